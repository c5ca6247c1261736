"""Thin Python binding of libpam (include/pam.h), argument marshalling only.

Every step of the fitting path runs in the CUDA library; this module turns
torch tensors into device pointers, fills the C structs and checks status
codes. PyTorch supplies the device memory (model arrays, workspace) and the
stream. If the library was not built, importing works but every call raises
``RuntimeError`` -- there is no other implementation to fall back to.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpam.so")

PAM_MAX_DIM = 3
PAM_INFO_N = 8
PAM_PREC_FP64 = 0
PAM_PREC_MIXED = 1

INFO_M, INFO_SUPPORT, INFO_LEVELS, INFO_ITERS, INFO_FLAGS, INFO_STOPPED, INFO_N_CELLS, INFO_MARKED = range(8)
FLAG_NOT_CERTIFIED, FLAG_CHOLESKY, FLAG_REFINE_DIVERGED = 1, 2, 4

STATUS = {0: "PAM_OK", 1: "PAM_ERR_INVALID_ARG", 2: "PAM_ERR_NONPOSITIVE_K", 3: "PAM_ERR_CUDA",
          4: "PAM_ERR_WORKSPACE", 5: "PAM_ERR_NOT_CONVERGED", 6: "PAM_ERR_UNSUPPORTED",
          7: "PAM_ERR_TIMEOUT"}
(PAM_OK, PAM_ERR_INVALID_ARG, PAM_ERR_NONPOSITIVE_K, PAM_ERR_CUDA, PAM_ERR_WORKSPACE, PAM_ERR_NOT_CONVERGED,
 PAM_ERR_UNSUPPORTED, PAM_ERR_TIMEOUT) = range(8)

EXPORTED = ["pam_version", "pam_status_string", "pam_plan_create", "pam_partition",
            "pam_fit_subdomains", "pam_refine", "pam_gram", "pam_eval_workspace_size", "pam_eval",
            "pam_errors", "pam_status_read", "pam_lambda_cv_workspace_size", "pam_lambda_cv",
            "pam_eval_glued_workspace_size", "pam_eval_glued", "pam_partition_cells", "pam_plan_create_cells",
            "pam_fit_cells", "pam_refine_cells", "pam_errors_cells", "pam_model_save", "pam_model_load",
            "pam_resume", "pam_resume_cells", "pam_tuning_set", "pam_tuning_get", "pam_autotune",
            "pam_autotune_cells", "pam_selftest_wait", "pam_error_sums", "pam_nn_inputs", "pam_group_layout",
            "pam_eval_bucket", "pam_eval_bucketed"]


class PamError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}")


class pam_problem(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_cells", C.c_int * 3), ("n_sub", C.c_int * 3),
                ("overlap", C.c_int), ("g_init", C.c_int * 3)]


class pam_params(C.Structure):
    _fields_ = [("lambda1_hat", C.c_double), ("lambda2_hat", C.c_double),
                ("eps_tol_rel", C.c_double), ("eta", C.c_double), ("k_top", C.c_int),
                ("m_max", C.c_int), ("levels", C.c_int), ("max_iters", C.c_int),
                ("precision", C.c_int), ("warm_start", C.c_int), ("quad", C.c_int),
                ("deferred_status", C.c_int), ("warm_start_event", C.c_void_p), ("sub_begin", C.c_int),
                ("sub_end", C.c_int)]


class pam_plan(C.Structure):
    _fields_ = [("n_subdomains", C.c_int), ("max_patch_cells", C.c_int), ("m0", C.c_int),
                ("m_cap", C.c_int), ("n_grid_cells", C.c_int64), ("workspace_bytes", C.c_size_t)]


class pam_cells(C.Structure):
    _fields_ = [("n_cells", C.c_int64), ("x", C.c_void_p), ("vol", C.c_void_p), ("patch_start", C.c_void_p),
                ("patch_cells", C.c_void_p)]


class pam_tuning(C.Structure):
    _fields_ = [("factor_kb", C.c_int), ("gram_stages", C.c_int), ("eval_block", C.c_int),
                ("solve_persistent", C.c_int), ("level_groups", C.c_int), ("reserved", C.c_int * 3)]


class pam_model(C.Structure):
    _fields_ = [("boxes", C.c_void_p), ("centres", C.c_void_p), ("beta", C.c_void_p),
                ("info", C.c_void_p)]


_lib = None


def lib():
    """The loaded libpam (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpam is not built ({LIB_PATH} missing): run "
                               "__graft_entry__.build() or python paper_2605_16564_gb300/build.py")
        L = C.CDLL(LIB_PATH)
        P = C.POINTER
        L.pam_version.restype = C.c_char_p
        L.pam_struct_sizes.argtypes = [P(C.c_size_t), C.c_int]
        L.pam_status_string.restype = C.c_char_p
        L.pam_status_string.argtypes = [C.c_int]
        L.pam_plan_create.argtypes = [P(pam_problem), P(pam_params), P(pam_plan)]
        L.pam_partition.argtypes = [P(pam_problem), C.c_void_p]
        L.pam_fit_subdomains.argtypes = [P(pam_problem), P(pam_params), P(pam_plan), C.c_void_p,
                                         P(pam_model), C.c_void_p, C.c_size_t, C.c_void_p]
        L.pam_refine.argtypes = [P(pam_problem), P(pam_params), P(pam_plan), C.c_void_p,
                                 P(pam_model), C.c_int, C.c_void_p, C.c_size_t, C.c_void_p]
        L.pam_status_read.argtypes = [P(pam_plan), C.c_void_p, C.c_size_t, C.c_void_p]
        L.pam_lambda_cv_workspace_size.argtypes = [P(pam_plan), P(C.c_size_t)]
        L.pam_lambda_cv.argtypes = [P(pam_problem), P(pam_params), P(pam_plan), C.c_void_p, P(pam_model),
                                    C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_size_t, C.c_void_p, C.c_size_t, C.c_void_p]
        L.pam_eval_workspace_size.argtypes = [P(pam_plan), C.c_int64, P(C.c_size_t)]
        L.pam_eval.argtypes = [P(pam_problem), P(pam_plan), P(pam_model), C.c_void_p, C.c_int64,
                               C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_size_t, C.c_void_p]
        L.pam_partition_cells.argtypes = [P(pam_problem), C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
        L.pam_plan_create_cells.argtypes = [P(pam_problem), P(pam_params), C.c_int64, C.c_void_p, P(pam_plan)]
        L.pam_fit_cells.argtypes = [P(pam_problem), P(pam_params), P(pam_plan), P(pam_cells), C.c_void_p,
                                    P(pam_model), C.c_void_p, C.c_size_t, C.c_void_p]
        L.pam_refine_cells.argtypes = [P(pam_problem), P(pam_params), P(pam_plan), P(pam_cells), C.c_void_p,
                                       P(pam_model), C.c_int, C.c_void_p, C.c_size_t, C.c_void_p]
        L.pam_errors_cells.argtypes = [P(pam_problem), P(pam_plan), P(pam_model), P(pam_cells), C.c_void_p,
                                       C.c_void_p, C.c_int, C.c_void_p, C.c_size_t, C.c_void_p]
        L.pam_model_save.argtypes = [P(pam_problem), P(pam_plan), P(pam_model), C.c_void_p, P(C.c_size_t),
                                     C.c_void_p]
        L.pam_model_load.argtypes = [P(pam_problem), P(pam_plan), C.c_void_p, C.c_size_t, P(pam_model), C.c_void_p]
        L.pam_resume.argtypes = [P(pam_problem), P(pam_params), P(pam_plan), C.c_void_p, P(pam_model), C.c_void_p,
                                 C.c_size_t, C.c_void_p]
        L.pam_resume_cells.argtypes = [P(pam_problem), P(pam_params), P(pam_plan), P(pam_cells), C.c_void_p,
                                       P(pam_model), C.c_void_p, C.c_size_t, C.c_void_p]
        L.pam_tuning_set.argtypes = [P(pam_tuning)]
        L.pam_tuning_get.argtypes = [P(pam_tuning)]
        L.pam_autotune.argtypes = [P(pam_problem), P(pam_params), P(pam_plan), C.c_void_p, P(pam_model), C.c_void_p,
                                   C.c_size_t, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p,
                                   P(pam_tuning), C.c_void_p]
        L.pam_autotune_cells.argtypes = [P(pam_problem), P(pam_params), P(pam_plan), P(pam_cells), C.c_void_p,
                                         P(pam_model), C.c_void_p, C.c_size_t, C.c_void_p, C.c_int64, C.c_void_p,
                                         C.c_void_p, C.c_size_t, C.c_void_p, P(pam_tuning), C.c_void_p]
        L.pam_selftest_wait.argtypes = [C.c_int, C.c_longlong, C.c_void_p, C.c_void_p]
        L.pam_selftest_wait.restype = C.c_int
        for name in ("pam_partition_cells", "pam_plan_create_cells", "pam_fit_cells", "pam_refine_cells",
                     "pam_errors_cells", "pam_model_save", "pam_model_load", "pam_resume", "pam_resume_cells",
                     "pam_tuning_set", "pam_tuning_get", "pam_autotune", "pam_autotune_cells"):
            getattr(L, name).restype = C.c_int
        L.pam_eval_glued_workspace_size.argtypes = [P(pam_problem), P(pam_plan), C.c_int64, P(C.c_size_t)]
        L.pam_eval_glued.argtypes = [P(pam_problem), P(pam_plan), P(pam_model), C.c_void_p, C.c_int64,
                                     C.c_double, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_size_t,
                                     C.c_void_p]
        L.pam_errors.argtypes = [P(pam_problem), P(pam_plan), P(pam_model), C.c_void_p, C.c_void_p,
                                 C.c_int, C.c_int, C.c_void_p, C.c_size_t, C.c_void_p]
        L.pam_error_sums.argtypes = [P(pam_problem), P(pam_plan), P(pam_model), C.c_void_p, C.c_void_p,
                                     C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_size_t, C.c_void_p]
        L.pam_error_sums.restype = C.c_int
        L.pam_gram.argtypes = [P(pam_problem), P(pam_params), P(pam_plan), C.c_void_p, P(pam_model),
                               C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
        L.pam_nn_sizes.argtypes = [C.c_int, C.c_int, P(C.c_int64), P(C.c_size_t)]
        L.pam_nn_geometry.argtypes = [C.c_int, C.c_void_p]
        L.pam_nn_layer_offsets.argtypes = [C.c_int, C.c_void_p]
        L.pam_nn_forward.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                     C.c_size_t, C.c_void_p]
        L.pam_nn_gradients.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
        L.pam_nn_adamw.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_float,
                                   C.c_float, C.c_float, C.c_float, C.c_float, C.c_int, C.c_void_p]
        L.pam_nn_layered_inputs.argtypes = [P(pam_problem), P(pam_plan), C.c_void_p, C.c_void_p, C.c_int,
                                            C.c_void_p]
        L.pam_nn_seed.argtypes = [P(pam_plan), C.c_int, C.c_void_p, C.c_float, P(pam_model), C.c_void_p]
        L.pam_nn_inputs.argtypes = [C.c_int, P(pam_problem), P(pam_plan), C.c_void_p, C.c_void_p, C.c_int,
                                    C.c_void_p]
        for name in ("pam_nn_sizes", "pam_nn_geometry", "pam_nn_layer_offsets", "pam_nn_forward",
                     "pam_nn_gradients", "pam_nn_adamw", "pam_nn_layered_inputs", "pam_nn_seed", "pam_nn_inputs"):
            getattr(L, name).restype = C.c_int
        L.pam_errors_noalloc.argtypes = [P(pam_problem), P(pam_plan), P(pam_model), C.c_void_p,
                                         C.c_void_p, C.c_void_p]
        for name in ("pam_plan_create", "pam_partition", "pam_fit_subdomains", "pam_refine",
                     "pam_eval", "pam_errors", "pam_errors_noalloc", "pam_gram",
                     "pam_eval_workspace_size", "pam_eval_glued", "pam_eval_glued_workspace_size"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(code, where):
    if code != 0:
        raise PamError(code, where)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _event_handle(event):
    """cudaEvent_t of a torch.cuda.Event (created by its first record), an
    integer handle as is, or None."""
    if event is None:
        return None
    h = int(getattr(event, "cuda_event", event))
    if h == 0:
        raise ValueError("the event has not been recorded")
    return h


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def make_problem(n_cells, n_sub, overlap, g_init):
    dim = len(n_cells)
    pad = lambda v, f: list(v) + [f] * (3 - len(v))
    pr = pam_problem()
    pr.dim = dim
    pr.n_cells[:] = pad(n_cells, 1)
    pr.n_sub[:] = pad(n_sub, 1)
    pr.overlap = overlap
    pr.g_init[:] = pad(g_init, 1)
    return pr


def make_params(lambda1_hat=4.59e-4, lambda2_hat=4.64e-6, eps_tol_rel=1e-3, eta=0.5, k_top=37,
                m_max=1 << 30, levels=3, max_iters=0, precision=PAM_PREC_FP64, warm_start=0, quad=0,
                deferred_status=0, sub_range=None):
    """quad: quadrature of the indicators R_T, 0 midpoint, 1 two-point Gauss-Legendre per axis.
    deferred_status: 1 = the fit calls never synchronise the host (read the
    status with pam_status_read), so they can be captured in a CUDA graph."""
    p = pam_params()
    p.warm_start = warm_start
    if sub_range is not None:  # fit only the subdomains [begin, end) (a shard of one field)
        p.sub_begin, p.sub_end = int(sub_range[0]), int(sub_range[1])
    p.quad = quad
    p.deferred_status = deferred_status
    p.lambda1_hat, p.lambda2_hat, p.eps_tol_rel, p.eta = lambda1_hat, lambda2_hat, eps_tol_rel, eta
    p.k_top, p.m_max, p.levels, p.max_iters, p.precision = k_top, min(m_max, (1 << 31) - 1), levels, \
        max_iters, precision
    return p


# ------------------------------------------------------------ entry points --

def pam_version():
    return lib().pam_version().decode()


def pam_plan_create(problem, params):
    plan = pam_plan()
    _check(lib().pam_plan_create(C.byref(problem), C.byref(params), C.byref(plan)), "pam_plan_create")
    return plan


def pam_partition(problem):
    S = int(np.prod(list(problem.n_sub)[:problem.dim]))
    boxes = np.zeros((S, 12), dtype=np.int32)
    _check(lib().pam_partition(C.byref(problem), boxes.ctypes.data), "pam_partition")
    return boxes


def pam_fit_subdomains(problem, params, plan, K, model, workspace, stream=None, check=True):
    code = lib().pam_fit_subdomains(C.byref(problem), C.byref(params), C.byref(plan), _ptr(K),
                                    C.byref(model.c_struct()), _ptr(workspace),
                                    workspace.numel() * workspace.element_size(), _stream(stream))
    if check:
        _check(code, "pam_fit_subdomains")
    return code


def pam_refine(problem, params, plan, K, model, n_levels, workspace, stream=None, check=True):
    code = lib().pam_refine(C.byref(problem), C.byref(params), C.byref(plan), _ptr(K),
                            C.byref(model.c_struct()), int(n_levels), _ptr(workspace),
                            workspace.numel() * workspace.element_size(), _stream(stream))
    if check:
        _check(code, "pam_refine")
    return code


def pam_status_read(plan, workspace, stream=None):
    """Status code (0 = ok) accumulated by deferred-status fit calls."""
    return lib().pam_status_read(C.byref(plan), _ptr(workspace), int(workspace.numel()), _stream(stream))


def pam_lambda_cv_workspace_size(plan):
    n = C.c_size_t(0)
    _check(lib().pam_lambda_cv_workspace_size(C.byref(plan), C.byref(n)), "pam_lambda_cv_workspace_size")
    return int(n.value)


def pam_lambda_cv(problem, params, plan, K, model, grid, n_folds, cv, choice, workspace, cv_workspace,
                  stream=None, check=True):
    """k-fold cross-validation of the grid of (lambda1_hat, lambda2_hat)
    pairs on every subdomain, then the refit with the chosen pair."""
    g = np.ascontiguousarray(np.asarray(grid, dtype=np.float64).reshape(-1, 2))
    code = lib().pam_lambda_cv(C.byref(problem), C.byref(params), C.byref(plan), _ptr(K),
                               C.byref(model.c_struct()), g.ctypes.data, int(g.shape[0]), int(n_folds),
                               _ptr(cv), _ptr(choice), _ptr(workspace), int(workspace.numel()),
                               _ptr(cv_workspace), int(cv_workspace.numel()), _stream(stream))
    if check and code not in (0, 5):
        _check(code, "pam_lambda_cv")
    return code


def pam_gram(problem, params, plan, K, model, G, b, workspace, stream=None):
    _check(lib().pam_gram(C.byref(problem), C.byref(params), C.byref(plan), _ptr(K),
                          C.byref(model.c_struct()), _ptr(G), _ptr(b), _ptr(workspace),
                          workspace.numel() * workspace.element_size(), _stream(stream)), "pam_gram")


def pam_eval_workspace_size(plan, n_pts):
    n = C.c_size_t(0)
    _check(lib().pam_eval_workspace_size(C.byref(plan), int(n_pts), C.byref(n)), "pam_eval_workspace_size")
    return n.value


def pam_eval(problem, plan, model, pts, out, log_space=False, precision=PAM_PREC_FP64, workspace=None,
             stream=None):
    n = pts.shape[0] if pts is not None else 0
    nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().pam_eval(C.byref(problem), C.byref(plan), C.byref(model.c_struct()), _ptr(pts),
                          int(n), _ptr(out), int(bool(log_space)), int(precision), _ptr(workspace),
                          nbytes, _stream(stream)), "pam_eval")


def pam_eval_bucket(problem, plan, pts, out, workspace=None, stream=None):
    n = pts.shape[0] if pts is not None else 0
    nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().pam_eval_bucket(C.byref(problem), C.byref(plan), _ptr(pts), int(n), _ptr(out), _ptr(workspace),
                                 nbytes, _stream(stream)), "pam_eval_bucket")


def pam_eval_bucketed(problem, plan, model, pts, out, log_space=False, precision=PAM_PREC_FP64, workspace=None,
                      stream=None):
    n = pts.shape[0] if pts is not None else 0
    nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().pam_eval_bucketed(C.byref(problem), C.byref(plan), C.byref(model.c_struct()), _ptr(pts),
                                   int(n), _ptr(out), int(bool(log_space)), int(precision), _ptr(workspace),
                                   nbytes, _stream(stream)), "pam_eval_bucketed")


def pam_eval_glued_workspace_size(problem, plan, n_pts):
    n = C.c_size_t(0)
    _check(lib().pam_eval_glued_workspace_size(C.byref(problem), C.byref(plan), int(n_pts), C.byref(n)),
           "pam_eval_glued_workspace_size")
    return n.value


def pam_eval_glued(problem, plan, model, pts, out, band, log_space=False, precision=PAM_PREC_FP64,
                   workspace=None, stream=None):
    """K*(x) blended across subdomain interfaces over a ramp of half-width
    band cells (0 < band <= half the narrowest core)."""
    n = pts.shape[0] if pts is not None else 0
    nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().pam_eval_glued(C.byref(problem), C.byref(plan), C.byref(model.c_struct()), _ptr(pts),
                                int(n), float(band), _ptr(out), int(bool(log_space)), int(precision),
                                _ptr(workspace), nbytes, _stream(stream)), "pam_eval_glued")


def pam_errors(problem, plan, model, K, err, workspace, precision=PAM_PREC_FP64, stream=None, quad=0):
    _check(lib().pam_errors(C.byref(problem), C.byref(plan), C.byref(model.c_struct()), _ptr(K),
                            _ptr(err), int(precision), int(quad), _ptr(workspace),
                            workspace.numel() * workspace.element_size(), _stream(stream)), "pam_errors")


def pam_error_sums(problem, plan, model, K, sums, sub_range, workspace, precision=PAM_PREC_FP64, stream=None,
                   quad=0):
    """The seven raw sums of the error measures over the cells owned by the
    subdomains [begin, end) into the device tensor sums [8] (a shard's share)."""
    _check(lib().pam_error_sums(C.byref(problem), C.byref(plan), C.byref(model.c_struct()), _ptr(K), _ptr(sums),
                                int(precision), int(quad), int(sub_range[0]), int(sub_range[1]), _ptr(workspace),
                                workspace.numel() * workspace.element_size(), _stream(stream)), "pam_error_sums")


def error_measures_from_sums(s):
    """pam_errors' four measures from the (summed) raw sums [8] (host array)."""
    import math
    return dict(l1=s[0] / s[1], l2=math.sqrt(s[2] / s[3]), l1_log=(s[4] / s[5]) if s[5] > 0 else s[4],
                max_log10=s[6] / math.log(10.0))


def pam_errors_noalloc(problem, plan, model, K, err, stream=None):
    """pam_errors for callers that cannot allocate device memory or provide
    a workspace (e.g. a host simulator that owns the whole GPU memory pool):
    its scratch is a fixed 256 KiB array inside the library."""
    _check(lib().pam_errors_noalloc(C.byref(problem), C.byref(plan), C.byref(model.c_struct()),
                                    _ptr(K), _ptr(err), _stream(stream)), "pam_errors_noalloc")


def pam_partition_cells(problem, x):
    """Patch lists of a mesh given as cells with sampling points x [n, dim]
    (host numpy): (patch_start int32 [S+1], patch_cells int32)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    n = x.shape[0]
    S = int(np.prod(list(problem.n_sub)[:problem.dim]))
    start = np.zeros(S + 1, dtype=np.int32)
    _check(lib().pam_partition_cells(C.byref(problem), x.ctypes.data, n, start.ctypes.data, None),
           "pam_partition_cells")
    cells = np.zeros(max(int(start[-1]), 1), dtype=np.int32)
    _check(lib().pam_partition_cells(C.byref(problem), x.ctypes.data, n, start.ctypes.data, cells.ctypes.data),
           "pam_partition_cells")
    return start, cells[:int(start[-1])]


def pam_plan_create_cells(problem, params, n_cells, patch_start):
    plan = pam_plan()
    ps = np.ascontiguousarray(np.asarray(patch_start, dtype=np.int32))
    _check(lib().pam_plan_create_cells(C.byref(problem), C.byref(params), int(n_cells), ps.ctypes.data,
                                       C.byref(plan)), "pam_plan_create_cells")
    return plan


def pam_fit_cells(problem, params, plan, cells, K, model, workspace, stream=None, check=True):
    code = lib().pam_fit_cells(C.byref(problem), C.byref(params), C.byref(plan), C.byref(cells), _ptr(K),
                               C.byref(model.c_struct()), _ptr(workspace),
                               workspace.numel() * workspace.element_size(), _stream(stream))
    if check:
        _check(code, "pam_fit_cells")
    return code


def pam_refine_cells(problem, params, plan, cells, K, model, n_levels, workspace, stream=None, check=True):
    code = lib().pam_refine_cells(C.byref(problem), C.byref(params), C.byref(plan), C.byref(cells), _ptr(K),
                                  C.byref(model.c_struct()), int(n_levels), _ptr(workspace),
                                  workspace.numel() * workspace.element_size(), _stream(stream))
    if check:
        _check(code, "pam_refine_cells")
    return code


def pam_errors_cells(problem, plan, model, cells, K, err, workspace, precision=PAM_PREC_FP64, stream=None):
    _check(lib().pam_errors_cells(C.byref(problem), C.byref(plan), C.byref(model.c_struct()), C.byref(cells),
                                  _ptr(K), _ptr(err), int(precision), _ptr(workspace),
                                  workspace.numel() * workspace.element_size(), _stream(stream)),
           "pam_errors_cells")


def pam_model_save(problem, plan, model, stream=None):
    """The model as a flat checkpoint blob (bytes)."""
    n = C.c_size_t(0)
    _check(lib().pam_model_save(C.byref(problem), C.byref(plan), C.byref(model.c_struct()), None, C.byref(n),
                                _stream(stream)), "pam_model_save")
    buf = np.zeros(int(n.value), dtype=np.uint8)
    _check(lib().pam_model_save(C.byref(problem), C.byref(plan), C.byref(model.c_struct()), buf.ctypes.data,
                                C.byref(n), _stream(stream)), "pam_model_save")
    return buf.tobytes()


def pam_model_load(problem, plan, blob, model, stream=None):
    """Copies a checkpoint blob (from pam_model_save) into a device model."""
    buf = np.frombuffer(blob, dtype=np.uint8)
    _check(lib().pam_model_load(C.byref(problem), C.byref(plan), buf.ctypes.data, buf.size,
                                C.byref(model.c_struct()), _stream(stream)), "pam_model_load")


def pam_resume(problem, params, plan, K, model, workspace, stream=None, check=True):
    code = lib().pam_resume(C.byref(problem), C.byref(params), C.byref(plan), _ptr(K), C.byref(model.c_struct()),
                            _ptr(workspace), workspace.numel() * workspace.element_size(), _stream(stream))
    if check:
        _check(code, "pam_resume")
    return code


def pam_resume_cells(problem, params, plan, cells, K, model, workspace, stream=None, check=True):
    code = lib().pam_resume_cells(C.byref(problem), C.byref(params), C.byref(plan), C.byref(cells), _ptr(K),
                                  C.byref(model.c_struct()), _ptr(workspace),
                                  workspace.numel() * workspace.element_size(), _stream(stream))
    if check:
        _check(code, "pam_resume_cells")
    return code


def pam_tuning_set(factor_kb=0, gram_stages=0, eval_block=0, solve_persistent=0, level_groups=0, reset=False):
    """Process-wide launch tuning (0 = built-in choice); reset=True restores all built-ins."""
    if reset:
        _check(lib().pam_tuning_set(None), "pam_tuning_set")
        return
    t = pam_tuning(int(factor_kb), int(gram_stages), int(eval_block), int(solve_persistent), int(level_groups))
    _check(lib().pam_tuning_set(C.byref(t)), "pam_tuning_set")


def pam_group_layout(n_subdomains):
    """The subdomain groups of the mixed form's levels for n_subdomains
    subdomains under the current tuning: a list of dicts, one per group."""
    out = np.zeros(14, dtype=np.int32)
    L = lib()
    L.pam_group_layout.restype = C.c_int
    n = L.pam_group_layout(int(n_subdomains), out.ctypes.data_as(C.c_void_p))
    if n < 1:
        raise PamError(PAM_ERR_INVALID_ARG, "pam_group_layout")
    keys = ("first", "stride", "count", "order_offset", "list_offset", "slots", "first_slot")
    return [dict(zip(keys, (int(v) for v in out[7 * q:7 * q + 7]))) for q in range(n)]


def pam_tuning_get():
    t = pam_tuning()
    _check(lib().pam_tuning_get(C.byref(t)), "pam_tuning_get")
    return dict(factor_kb=t.factor_kb, gram_stages=t.gram_stages, eval_block=t.eval_block,
                solve_persistent=t.solve_persistent, level_groups=t.level_groups)


def pam_autotune(problem, params, plan, K, model, workspace, pts=None, out=None, eval_workspace=None, stream=None,
                 cells=None):
    """Measures the tuning candidates on a fitted model (and pts, if given),
    keeps the fastest process-wide; returns (choice dict, medians in ms [14]).
    cells: the pam_cells of a mesh given as cells (pam_autotune_cells)."""
    t = pam_tuning()
    ms = np.zeros(14, dtype=np.float64)
    n = pts.shape[0] if pts is not None else 0
    ebytes = eval_workspace.numel() * eval_workspace.element_size() if eval_workspace is not None else 0
    wbytes = workspace.numel() * workspace.element_size()
    if cells is None:
        code = lib().pam_autotune(C.byref(problem), C.byref(params), C.byref(plan), _ptr(K), C.byref(model.c_struct()),
                                  _ptr(workspace), wbytes, _ptr(pts), int(n), _ptr(out), _ptr(eval_workspace), ebytes,
                                  _stream(stream), C.byref(t), ms.ctypes.data)
    else:
        code = lib().pam_autotune_cells(C.byref(problem), C.byref(params), C.byref(plan), C.byref(cells), _ptr(K),
                                        C.byref(model.c_struct()), _ptr(workspace), wbytes, _ptr(pts), int(n),
                                        _ptr(out), _ptr(eval_workspace), ebytes, _stream(stream), C.byref(t),
                                        ms.ctypes.data)
    _check(code, "pam_autotune")
    return dict(factor_kb=t.factor_kb, gram_stages=t.gram_stages, eval_block=t.eval_block,
                solve_persistent=t.solve_persistent, level_groups=t.level_groups), ms


def pam_selftest_wait(arrive, budget_cycles, flag, stream=None):
    """Bounded-wait self-test: returns the status code (PAM_ERR_TIMEOUT when
    nothing arrived and the wait gave up); flag: device int32 [1]."""
    return lib().pam_selftest_wait(int(arrive), int(budget_cycles), _ptr(flag), _stream(stream))


PAM_NN_PATCH2D, PAM_NN_LAYERED3D = 0, 1


def pam_nn_sizes(batch, arch=PAM_NN_PATCH2D):
    n, ws = C.c_int64(0), C.c_size_t(0)
    _check(lib().pam_nn_sizes(int(arch), int(batch), C.byref(n), C.byref(ws)), "pam_nn_sizes")
    return n.value, ws.value


def pam_nn_geometry(arch=PAM_NN_PATCH2D):
    """(input pixels per side, input channels, n_out)."""
    g = np.zeros(3, dtype=np.int32)
    _check(lib().pam_nn_geometry(int(arch), g.ctypes.data), "pam_nn_geometry")
    return int(g[0]), int(g[1]), int(g[2])


def pam_nn_layer_offsets(arch=PAM_NN_PATCH2D):
    off = np.zeros(24, dtype=np.int64)
    _check(lib().pam_nn_layer_offsets(int(arch), off.ctypes.data), "pam_nn_layer_offsets")
    return off.reshape(6, 4)


def pam_nn_forward(params, x, out, workspace, stream=None, arch=PAM_NN_PATCH2D):
    _check(lib().pam_nn_forward(int(arch), _ptr(params), _ptr(x), int(x.shape[0]), _ptr(out), _ptr(workspace),
                                workspace.numel(), _stream(stream)), "pam_nn_forward")


def pam_nn_gradients(params, x, support, beta, grads, loss, workspace, stream=None, arch=PAM_NN_PATCH2D):
    _check(lib().pam_nn_gradients(int(arch), _ptr(params), _ptr(x), _ptr(support), _ptr(beta),
                                  int(x.shape[0]), _ptr(grads), _ptr(loss), _ptr(workspace), workspace.numel(),
                                  _stream(stream)), "pam_nn_gradients")


def pam_nn_layered_inputs(problem, plan, K, x, stream=None):
    """x [n_rows][16][16][8] fp32 (n_rows >= S) from the patches of K."""
    _check(lib().pam_nn_layered_inputs(C.byref(problem), C.byref(plan), _ptr(K), _ptr(x), int(x.shape[0]),
                                       _stream(stream)), "pam_nn_layered_inputs")


def pam_nn_inputs(problem, plan, K, x, stream=None, arch=PAM_NN_PATCH2D):
    """The network inputs x [n_rows][h][h][c] fp32 of every subdomain's patch of K (on the device)."""
    _check(lib().pam_nn_inputs(int(arch), C.byref(problem), C.byref(plan), _ptr(K), _ptr(x), int(x.shape[0]),
                               _stream(stream)), "pam_nn_inputs")


def pam_nn_seed(plan, out, threshold, model, stream=None, arch=PAM_NN_LAYERED3D):
    """model.beta[s][j] = 4 out[s][n_out + j] where that exceeds threshold in magnitude, else 0."""
    _check(lib().pam_nn_seed(C.byref(plan), int(arch), _ptr(out), float(threshold), C.byref(model.c_struct()),
                             _stream(stream)), "pam_nn_seed")


def pam_nn_adamw(params, grads, m, v, lr, beta1, beta2, eps, weight_decay, step, stream=None):
    _check(lib().pam_nn_adamw(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), int(params.numel()),
                              float(lr), float(beta1), float(beta2), float(eps), float(weight_decay),
                              int(step), _stream(stream)), "pam_nn_adamw")


# ------------------------------------------------------------------ helpers --

@dataclass
class Model:
    """Device arrays of a fitted model (torch tensors, caller-owned)."""
    boxes: "object"
    centres: "object"
    beta: "object"
    info: "object"
    _c: pam_model = field(default=None, repr=False)

    def c_struct(self):
        self._c = pam_model(self.boxes.data_ptr(), self.centres.data_ptr(), self.beta.data_ptr(),
                            self.info.data_ptr())
        return self._c

    def to_host(self, n_cells, n_sub, m_cap):
        """The model as the numpy dict the oracle's evaluation takes."""
        info = self.info.cpu().numpy()
        return dict(boxes=self.boxes.cpu().numpy(), M=info[:, INFO_M].astype(np.int32),
                    c=self.centres.cpu().numpy(), beta=self.beta.cpu().numpy(), info=info,
                    m_cap=int(m_cap), n_cells=tuple(n_cells), n_sub=tuple(n_sub))


def alloc_model(plan, device="cuda"):
    import torch
    S, mc = plan.n_subdomains, plan.m_cap
    return Model(boxes=torch.zeros((S, 12), dtype=torch.int32, device=device),
                 centres=torch.zeros((S, mc, 4), dtype=torch.float64, device=device),
                 beta=torch.zeros((S, mc), dtype=torch.float64, device=device),
                 info=torch.zeros((S, PAM_INFO_N), dtype=torch.int32, device=device))


def alloc_workspace(plan, device="cuda"):
    import torch
    return torch.empty(int(plan.workspace_bytes), dtype=torch.uint8, device=device)


def error_dict(err):
    """Host dict of the error measures in a [4] tensor written by pam_errors."""
    e = err.cpu().numpy()
    return dict(l1=e[0], l2=e[1], l1_log=e[2], max_log10=e[3])


class Fitter:
    """A problem, its parameters and plan, with the device buffers they need."""

    def __init__(self, n_cells, n_sub, overlap, g_init, device="cuda", **params):
        self.n_cells, self.n_sub = tuple(n_cells), tuple(n_sub)
        self.problem = make_problem(n_cells, n_sub, overlap, g_init)
        self.params = make_params(**params)
        self.plan = pam_plan_create(self.problem, self.params)
        self.device = device
        self.model = alloc_model(self.plan, device)
        self.workspace = alloc_workspace(self.plan, device)

    def fit(self, K, levels=None, stream=None, check=True, warm_start=False, deferred=False,
            warm_start_event=None):
        """Step 2, then `levels` rounds of Step 3 (default: the planned levels).
        warm_start: the initial dictionary starts from the coefficients
        already in model.beta (e.g. seeded by pam_nn_seed).
        warm_start_event: a torch.cuda.Event recorded after the warm start
        was written on another stream; the level-0 solve waits for it.
        deferred: launch only, no host synchronisation (capturable in a CUDA
        graph); the status is read later with status()."""
        lv = self.params.levels if levels is None else levels
        self.params.warm_start = 1 if warm_start else 0
        self.params.deferred_status = 1 if deferred else 0
        self.params.warm_start_event = _event_handle(warm_start_event)
        try:
            c1 = pam_fit_subdomains(self.problem, self.params, self.plan, K, self.model, self.workspace,
                                    stream, check)
            c2 = pam_refine(self.problem, self.params, self.plan, K, self.model, lv, self.workspace,
                            stream, check) if lv > 0 else 0
        finally:
            self.params.warm_start = 0
            self.params.deferred_status = 0
            self.params.warm_start_event = None
        return c1 or c2

    def lambda_cv(self, K, grid, n_folds, stream=None, check=True):
        """Per-subdomain k-fold cross-validation of the grid pairs on the
        current dictionary and refit with the chosen pair (binary64 form).
        Returns (cv [S, n_grid] device, choice [S] device, status code)."""
        import torch
        S = self.plan.n_subdomains
        n_grid = int(np.asarray(grid).reshape(-1, 2).shape[0])
        cv = torch.empty((S, n_grid), dtype=torch.float64, device=self.device)
        choice = torch.empty(S, dtype=torch.int32, device=self.device)
        need = pam_lambda_cv_workspace_size(self.plan)
        ws = getattr(self, "_cv_ws", None)
        if ws is None or ws.numel() < need:
            ws = torch.empty(need, dtype=torch.uint8, device=self.device)
            self._cv_ws = ws
        code = pam_lambda_cv(self.problem, self.params, self.plan, K, self.model, grid, n_folds, cv, choice,
                             self.workspace, ws, stream, check)
        return cv, choice, code

    def status(self, stream=None):
        """Status of the deferred fit calls since the last fit (synchronises)."""
        return pam_status_read(self.plan, self.workspace, stream)

    def eval_workspace(self, n_pts):
        import torch
        need = pam_eval_workspace_size(self.plan, n_pts)
        ws = getattr(self, "_eval_ws", None)
        if ws is None or ws.numel() < need:
            ws = torch.empty(max(need, 256), dtype=torch.uint8, device=self.device)
            self._eval_ws = ws
        return ws

    def eval_bucket(self, pts, out, stream=None):
        """pam_eval_bucket: the points bucketed by owner in this fitter's
        evaluation workspace (no model read: it may run beside the fit on
        another stream). eval_bucketed with the same pts and out completes the
        evaluation; no other evaluation of more points may come in between
        (the workspace would be replaced)."""
        pam_eval_bucket(self.problem, self.plan, pts, out, self.eval_workspace(pts.shape[0]), stream)
        return out

    def eval_bucketed(self, pts, out, log_space=False, precision=None, stream=None):
        prec = self.params.precision if precision is None else precision
        pam_eval_bucketed(self.problem, self.plan, self.model, pts, out, log_space, prec,
                          self.eval_workspace(pts.shape[0]), stream)
        return out

    def eval(self, pts, out=None, log_space=False, precision=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(pts.shape[0], dtype=torch.float64, device=pts.device)
        prec = self.params.precision if precision is None else precision
        pam_eval(self.problem, self.plan, self.model, pts, out, log_space, prec,
                 self.eval_workspace(pts.shape[0]), stream)
        return out

    def _slice_bounds(self, n, chunks):
        k = max(1, min(int(chunks), n)) if n > 0 else 0
        return [(n * i // k, n * (i + 1) // k) for i in range(k)]

    def _slice_workspace(self, i, n_pts):
        import torch
        need = pam_eval_workspace_size(self.plan, n_pts)
        wss = getattr(self, "_slice_ws", None)
        if wss is None:
            wss = self._slice_ws = []
        while len(wss) <= i:
            wss.append(None)
        if wss[i] is None or wss[i].numel() < need:
            wss[i] = torch.empty(max(need, 256), dtype=torch.uint8, device=self.device)
        return wss[i]

    def bucket_slices(self, pts, out, chunks=4):
        """pam_eval_bucket of each slice eval_to_host(..., bucketed=True) will
        evaluate (the same pts, out and chunks), each slice in a workspace of
        its own, on the current stream: it reads no model, so it may run on
        another stream beside the fit."""
        for i, (a, b) in enumerate(self._slice_bounds(pts.shape[0], chunks)):
            pam_eval_bucket(self.problem, self.plan, pts[a:b], out[a:b], self._slice_workspace(i, b - a))
        return out

    def eval_to_host(self, pts, out, out_host, chunks=4, copy_stream=None, join=True, log_space=False,
                     precision=None, bucketed=False):
        """pam_eval of pts into the device buffer out in `chunks` contiguous
        slices, each slice's values copied to the pinned host buffer out_host
        on copy_stream as soon as they are ready, so that the copies overlap
        the evaluation of the later slices (the values are those of one
        pam_eval call: every point is evaluated on its own). Enqueued on the
        current stream; join: later work on it waits for the copies (else
        the caller joins copy_stream itself, and work enqueued meanwhile runs
        beside the copies). bucketed: the slices were bucketed already by
        bucket_slices (same pts, out and chunks; ordered before this call), and
        only pam_eval_bucketed runs here. Capturable in a CUDA graph."""
        import torch
        n = pts.shape[0]
        if out.shape[0] < n or out_host.shape[0] < n:
            raise ValueError(f"eval_to_host: {n} points, out holds {out.shape[0]}, out_host {out_host.shape[0]}")
        if not out.is_cuda or out.device != torch.device(self.device) or out.dtype != torch.float64:
            raise ValueError("eval_to_host: out must be a float64 tensor on the fitter's device (pam_eval writes "
                             "binary64 values there)")
        if out_host.device.type != "cpu" or out_host.dtype != out.dtype:
            raise ValueError("eval_to_host: out_host must be a host tensor of out's dtype (pinned for overlap)")
        cur = torch.cuda.current_stream()
        cs = copy_stream if copy_stream is not None else self._copy_stream()
        bounds = self._slice_bounds(n, chunks)
        k = len(bounds)
        evs = self._chunk_events(k)
        if not bucketed:
            self.eval_workspace(n)  # one workspace, sized for the whole set, serves every slice
        prec = self.params.precision if precision is None else precision
        for i, (a, b) in enumerate(bounds):
            if bucketed:
                pam_eval_bucketed(self.problem, self.plan, self.model, pts[a:b], out[a:b], log_space, prec,
                                  self._slice_workspace(i, b - a))
            else:
                self.eval(pts[a:b], out=out[a:b], log_space=log_space, precision=precision)
            evs[i].record(cur)
            cs.wait_event(evs[i])
            with torch.cuda.stream(cs):
                out_host[a:b].copy_(out[a:b], non_blocking=True)
        if join:
            cur.wait_stream(cs)
        else:
            out.record_stream(cs)  # out stays allocated until the copies on cs have run
        return out_host

    def _copy_stream(self):
        import torch
        if getattr(self, "_cs", None) is None:
            self._cs = torch.cuda.Stream(device=self.device)
        return self._cs

    def _chunk_events(self, k):
        import torch
        evs = getattr(self, "_chunk_evs", [])
        while len(evs) < k:
            evs.append(torch.cuda.Event())
        self._chunk_evs = evs
        return evs

    def eval_glued(self, pts, band, out=None, log_space=False, precision=None, stream=None):
        """K*(x) blended across the subdomain interfaces (pam_eval_glued)."""
        import torch
        if out is None:
            out = torch.empty(pts.shape[0], dtype=torch.float64, device=pts.device)
        prec = self.params.precision if precision is None else precision
        need = pam_eval_glued_workspace_size(self.problem, self.plan, pts.shape[0])
        ws = getattr(self, "_glue_ws", None)
        if ws is None or ws.numel() < need:
            ws = torch.empty(max(need, 256), dtype=torch.uint8, device=self.device)
            self._glue_ws = ws
        pam_eval_glued(self.problem, self.plan, self.model, pts, out, band, log_space, prec, ws, stream)
        return out

    def errors(self, K, precision=None, stream=None, quad=None):
        """quad: the errors' quadrature (default: the fit's indicator quadrature)."""
        import torch
        err = torch.zeros(4, dtype=torch.float64, device=K.device)
        self.errors_device(K, err, precision, stream, quad)
        return error_dict(err)

    def errors_device(self, K, err, precision=None, stream=None, quad=None):
        """The four error measures into the device tensor err [4] (no host
        synchronisation; read them with error_dict)."""
        prec = self.params.precision if precision is None else precision
        q = self.params.quad if quad is None else quad
        pam_errors(self.problem, self.plan, self.model, K, err, self.workspace, prec, stream, quad=q)
        return err

    def host_model(self):
        return self.model.to_host(self.n_cells, self.n_sub, self.plan.m_cap)

    def autotune(self, K, pts=None, stream=None):
        """pam_autotune on this fitter's fitted model (and evaluation points)."""
        import torch
        out = ws = None
        if pts is not None and pts.shape[0] > 0:
            out = torch.empty(pts.shape[0], dtype=torch.float64, device=pts.device)
            ws = self.eval_workspace(pts.shape[0])
        return pam_autotune(self.problem, self.params, self.plan, K, self.model, self.workspace, pts, out, ws, stream,
                            cells=getattr(self, "cells", None))

    def save(self, stream=None):
        """Checkpoint of the model (bytes, pam_model_save)."""
        return pam_model_save(self.problem, self.plan, self.model, stream)

    def load(self, blob, stream=None):
        """Loads a checkpoint into this fitter's model (pam_model_load)."""
        pam_model_load(self.problem, self.plan, blob, self.model, stream)

    def resume(self, K, levels=0, stream=None, check=True):
        """Readies the workspace for the loaded model and K (pam_resume), then
        runs `levels` more refinement rounds."""
        c1 = pam_resume(self.problem, self.params, self.plan, K, self.model, self.workspace, stream, check)
        c2 = pam_refine(self.problem, self.params, self.plan, K, self.model, levels, self.workspace, stream,
                        check) if levels > 0 else 0
        return c1 or c2


class CellFitter(Fitter):
    """A problem on a general mesh given as cells (sampling points x [n, dim]
    and measures vol [n], host arrays): the patch lists are built on the host
    (pam_partition_cells) and kept on the device with the points and
    measures; fit/errors take the element values K [n] on the device."""

    def __init__(self, n_cells, n_sub, overlap, g_init, x, vol, device="cuda", **params):
        import torch
        self.n_cells, self.n_sub = tuple(n_cells), tuple(n_sub)
        self.problem = make_problem(n_cells, n_sub, overlap, g_init)
        self.params = make_params(**params)
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, len(self.n_cells)))
        start, lists = pam_partition_cells(self.problem, x)
        self.plan = pam_plan_create_cells(self.problem, self.params, x.shape[0], start)
        self.device = device
        self.x = torch.from_numpy(x).to(device)
        self.vol = torch.from_numpy(np.ascontiguousarray(np.asarray(vol, dtype=np.float64))).to(device)
        self.patch_start = torch.from_numpy(start).to(device)
        self.patch_cells = torch.from_numpy(np.ascontiguousarray(lists) if lists.size else
                                            np.zeros(1, dtype=np.int32)).to(device)
        self.cells = pam_cells(x.shape[0], self.x.data_ptr(), self.vol.data_ptr(), self.patch_start.data_ptr(),
                               self.patch_cells.data_ptr())
        self.model = alloc_model(self.plan, device)
        self.workspace = alloc_workspace(self.plan, device)

    def fit(self, K, levels=None, stream=None, check=True, warm_start=False, deferred=False,
            warm_start_event=None):
        lv = self.params.levels if levels is None else levels
        self.params.warm_start = 1 if warm_start else 0
        self.params.deferred_status = 1 if deferred else 0
        self.params.warm_start_event = _event_handle(warm_start_event)
        try:
            c1 = pam_fit_cells(self.problem, self.params, self.plan, self.cells, K, self.model, self.workspace,
                               stream, check)
            c2 = pam_refine_cells(self.problem, self.params, self.plan, self.cells, K, self.model, lv,
                                  self.workspace, stream, check) if lv > 0 else 0
        finally:
            self.params.warm_start = 0
            self.params.deferred_status = 0
            self.params.warm_start_event = None
        return c1 or c2

    def errors_device(self, K, err, precision=None, stream=None, quad=None):
        prec = self.params.precision if precision is None else precision
        pam_errors_cells(self.problem, self.plan, self.model, self.cells, K, err, self.workspace, prec, stream)
        return err

    def resume(self, K, levels=0, stream=None, check=True):
        c1 = pam_resume_cells(self.problem, self.params, self.plan, self.cells, K, self.model, self.workspace,
                              stream, check)
        c2 = pam_refine_cells(self.problem, self.params, self.plan, self.cells, K, self.model, levels,
                              self.workspace, stream, check) if levels > 0 else 0
        return c1 or c2

    def lambda_cv(self, *a, **k):
        raise PamError(PAM_ERR_UNSUPPORTED, "lambda_cv on a mesh given as cells")
