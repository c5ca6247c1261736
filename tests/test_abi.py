"""The C ABI without a GPU: the library builds, loads, exports every entry
point include/pam.h declares, and its host-only calls (sizes, partition,
argument checks) behave as documented."""
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pam():
    from paper_2605_16564_gb300 import build
    build.build()
    from paper_2605_16564_gb300 import pam as p
    p.lib()
    return p


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(pam_\w+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_entry_point(pam):
    declared = _declared_functions()
    assert "pam_fit_subdomains" in declared and "pam_eval" in declared
    L = pam.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert set(pam.EXPORTED) <= set(declared)
    assert "sm_103a" in pam.pam_version()


@pytest.mark.parametrize("n_cells,n_sub,overlap", [
    ((256, 256), (8, 8), 2), ((60, 220, 85), (6, 22, 17), 1), ((37, 23), (4, 3), 3), ((50,), (7,), 2)])
def test_partition_matches_the_oracle(pam, n_cells, n_sub, overlap):
    pr = pam.make_problem(n_cells, n_sub, overlap, (2,) * len(n_cells))
    np.testing.assert_array_equal(pam.pam_partition(pr), oracle.partition(n_cells, n_sub, overlap))


def test_status_read_rejects_bad_arguments(pam):
    import ctypes as C
    pr = pam.make_problem((8, 8), (2, 2), 1, (2, 2))
    plan = pam.pam_plan_create(pr, pam.make_params())
    L = pam.lib()
    assert L.pam_status_read(None, None, 0, None) == 1
    assert L.pam_status_read(C.byref(plan), None, 1024, None) == 1
    buf = (C.c_int32 * 4)()
    assert L.pam_status_read(C.byref(plan), C.cast(buf, C.c_void_p), 16, None) == 1  # < 8 words


def test_lambda_cv_rejects_bad_arguments(pam):
    import ctypes as C
    pr = pam.make_problem((16, 16), (2, 2), 1, (2, 2))
    fake = C.c_void_p(256)  # never dereferenced: validation fails first
    for prec, grid, folds, want in [(pam.PAM_PREC_FP64, [(1e-4, 0.0)], 3, 1),    # lambda2_hat > 0
                                    (pam.PAM_PREC_MIXED, [(1e-4, 0.0)], 3, 1),
                                    (pam.PAM_PREC_FP64, [(-1e-4, 1e-6)], 3, 1),  # lambda1_hat >= 0
                                    (pam.PAM_PREC_FP64, [(1e-4, 1e-6)], 1, 1),   # at least two folds
                                    (pam.PAM_PREC_FP64, [(1e-4, 1e-6)] * 33, 3, 1)]:  # at most 32 pairs
        par = pam.make_params(precision=prec)
        plan = pam.pam_plan_create(pr, par)
        m = pam.pam_model(fake, fake, fake, fake)
        g = np.ascontiguousarray(np.asarray(grid, dtype=np.float64))
        code = pam.lib().pam_lambda_cv(C.byref(pr), C.byref(par), C.byref(plan), fake, C.byref(m),
                                       g.ctypes.data, len(grid), folds, fake, fake, fake, 1 << 40, fake,
                                       1 << 40, None)
        assert code == want, (prec, grid[:1], folds, code)
    n = C.c_size_t(0)
    assert pam.lib().pam_lambda_cv_workspace_size(C.byref(plan), C.byref(n)) == 0 and n.value > 0


def test_plan_sizes(pam):
    pr = pam.make_problem((60, 220, 85), (6, 22, 17), 1, (4, 4, 2))
    plan = pam.pam_plan_create(pr, pam.make_params(k_top=30, levels=3))
    assert plan.n_subdomains == 2244 and plan.m0 == 32
    assert plan.m_cap == 448 and plan.m_cap >= 32 + 3 * 4 * 30
    assert plan.max_patch_cells >= 12 * 12 * 7 and plan.max_patch_cells % 32 == 0
    assert plan.n_grid_cells == 60 * 220 * 85
    assert plan.workspace_bytes > 0
    # the m_max cap bounds the capacity
    plan2 = pam.pam_plan_create(pr, pam.make_params(k_top=30, levels=3, m_max=10))
    assert plan2.m_cap == 64


@pytest.mark.parametrize("bad", [
    dict(problem=dict(n_cells=(0, 8), n_sub=(1, 1))),
    dict(problem=dict(n_cells=(8, 8), n_sub=(9, 1))),
    dict(problem=dict(overlap=-1)),
    dict(problem=dict(g_init=(0, 2))),
    dict(params=dict(lambda2_hat=0.0)),
    dict(params=dict(lambda1_hat=-1.0)),
    dict(params=dict(eta=1.0)),
    dict(params=dict(k_top=-1)),
    dict(params=dict(precision=7)),
    dict(params=dict(quad=2)),
    dict(params=dict(warm_start=3)),
    dict(params=dict(deferred_status=2)),
])
def test_invalid_arguments_are_rejected(pam, bad):
    base = dict(n_cells=(8, 8), n_sub=(2, 2), overlap=1, g_init=(2, 2))
    base.update(bad.get("problem", {}))
    pr = pam.make_problem(base["n_cells"], base["n_sub"], base["overlap"], base["g_init"])
    par = pam.make_params(**bad.get("params", {}))
    with pytest.raises(pam.PamError) as e:
        pam.pam_plan_create(pr, par)
    assert e.value.code == 1


def test_oversized_dictionary_is_unsupported(pam):
    pr = pam.make_problem((64, 64), (1, 1), 0, (40, 40))
    with pytest.raises(pam.PamError) as e:
        pam.pam_plan_create(pr, pam.make_params())
    assert e.value.code == 6


def test_null_arguments_are_rejected(pam):
    import ctypes as C
    L = pam.lib()
    assert L.pam_plan_create(None, None, None) == 1
    assert L.pam_partition(None, None) == 1
    pr = pam.make_problem((8, 8), (2, 2), 1, (2, 2))
    par = pam.make_params()
    plan = pam.pam_plan_create(pr, par)
    assert L.pam_fit_subdomains(C.byref(pr), C.byref(par), C.byref(plan), None, None, None, 0, None) == 1
    assert L.pam_eval(C.byref(pr), C.byref(plan), None, None, 0, None, 0, 0, None, 0, None) == 1


def test_split_evaluation_checks_its_arguments(pam):
    # host-side checks of pam_eval_bucket / pam_eval_bucketed (no device work)
    import ctypes as C
    L = pam.lib()
    L.pam_eval_bucket.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                  C.c_size_t, C.c_void_p]
    L.pam_eval_bucketed.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                    C.c_int, C.c_int, C.c_void_p, C.c_size_t, C.c_void_p]
    pr = pam.make_problem((8, 8), (2, 2), 1, (2, 2))
    plan = pam.pam_plan_create(pr, pam.make_params())
    p, q = C.byref(pr), C.byref(plan)
    fake = C.c_void_p(256)  # never dereferenced: every call below fails its checks first
    need = pam.pam_eval_workspace_size(plan, 10)
    assert L.pam_eval_bucket(p, q, None, 0, None, None, 0, None) == 0  # no points: a no-op
    assert L.pam_eval_bucket(p, q, None, 10, fake, fake, need, None) == 1  # no points buffer
    assert L.pam_eval_bucket(p, q, fake, 10, fake, None, need, None) == 1  # no workspace
    assert L.pam_eval_bucket(p, q, fake, 10, fake, fake, need - 1, None) == 4  # workspace too small
    assert L.pam_eval_bucket(p, q, fake, -1, fake, fake, need, None) == 1
    assert L.pam_eval_bucketed(p, q, None, fake, 10, fake, 0, 1, fake, need, None) == 1  # no model
    assert L.pam_eval_bucket(None, q, fake, 10, fake, fake, need, None) == 1


def test_network_sizes_and_geometry(pam):
    # both architectures: parameter counts from the layer tables, geometry,
    # and rejection of unknown architectures and bad batches (host only)
    import oracle.nn as onn
    for arch in (0, 1):
        n, ws = pam.pam_nn_sizes(64, arch=arch)
        assert n == onn.layout(arch)[1] and ws > 0
        A = onn.ARCHS[arch]
        assert pam.pam_nn_geometry(arch) == (A["h0"], A["c0"], A["n_out"])
    L = pam.lib()
    import ctypes as C
    n, ws = C.c_int64(0), C.c_size_t(0)
    assert L.pam_nn_sizes(2, 64, C.byref(n), C.byref(ws)) == 1
    assert L.pam_nn_sizes(0, 33, C.byref(n), C.byref(ws)) == 1


def test_layered_inputs_reject_unsupported_problems(pam):
    import ctypes as C
    L = pam.lib()
    # a 2-D problem, and a 3-D one whose patches exceed 16 x 16 x 8 cells
    pr2 = pam.make_problem((8, 8), (2, 2), 1, (2, 2))
    plan2 = pam.pam_plan_create(pr2, pam.make_params())
    assert L.pam_nn_layered_inputs(C.byref(pr2), C.byref(plan2), C.c_void_p(8), C.c_void_p(8), 32, None) == 1
    pr3 = pam.make_problem((40, 20, 10), (1, 1, 1), 0, (4, 4, 2))
    plan3 = pam.pam_plan_create(pr3, pam.make_params())
    assert L.pam_nn_layered_inputs(C.byref(pr3), C.byref(plan3), C.c_void_p(8), C.c_void_p(8), 32, None) == 6


def test_network_inputs_check_the_arch_against_the_problem(pam):
    import ctypes as C
    L = pam.lib()
    fake = C.c_void_p(8)  # never dereferenced: validation fails first
    pr2 = pam.make_problem((64, 64), (2, 2), 0, (16, 16))
    plan2 = pam.pam_plan_create(pr2, pam.make_params())
    pr3 = pam.make_problem((30, 110, 85), (3, 11, 17), 1, (4, 4, 2))
    plan3 = pam.pam_plan_create(pr3, pam.make_params())
    wide = pam.make_problem((66, 64), (2, 2), 0, (16, 16))  # a 33-cell patch
    plan_w = pam.pam_plan_create(wide, pam.make_params())
    for arch, pr, plan, rows, want in [(0, pr3, plan3, 576, 1),   # a 3-D problem for the 2-D network
                                       (1, pr2, plan2, 32, 1),    # and the converse
                                       (2, pr2, plan2, 32, 1),    # no such network
                                       (0, pr2, plan2, 3, 1),     # fewer rows than subdomains
                                       (0, wide, plan_w, 32, 6)]:
        assert L.pam_nn_inputs(arch, C.byref(pr), C.byref(plan), fake, fake, rows, None) == want, (arch, rows)
    assert L.pam_nn_inputs(0, C.byref(pr2), C.byref(plan2), None, fake, 32, None) == 1


def test_eval_glued_checks_the_band_and_sizes(pam):
    import ctypes as C
    fake = C.c_void_p(256)  # never dereferenced: validation fails first
    for n_cells, n_sub, good, bad in [((64, 64), (4, 4), 8.0, 8.01),      # cores of 16
                                      ((37, 23), (4, 3), 3.5, 3.6),       # narrowest core 7
                                      ((24, 44, 17), (3, 4, 2), 4.0, 4.5),
                                      ((50,), (1,), 1e6, float("inf"))]:  # no interior face
        pr = pam.make_problem(n_cells, n_sub, 1, (2,) * len(n_cells))
        plan = pam.pam_plan_create(pr, pam.make_params())
        m = pam.pam_model(fake, fake, fake, fake)
        L = pam.lib()
        for band, want in [(bad, 1), (0.0, 1), (-1.0, 1), (float("nan"), 1)]:
            code = L.pam_eval_glued(C.byref(pr), C.byref(plan), C.byref(m), fake, 10, band, fake, 0, 0,
                                    fake, 1 << 40, None)
            assert code == want, (n_cells, band, code)
        # a valid band with no points enqueues nothing and succeeds
        assert L.pam_eval_glued(C.byref(pr), C.byref(plan), C.byref(m), None, 0, good, None, 0, 0,
                                None, 0, None) == 0
        # a valid band with a short workspace
        assert L.pam_eval_glued(C.byref(pr), C.byref(plan), C.byref(m), fake, 10, good, fake, 0, 0,
                                fake, 16, None) == 4
        assert L.pam_eval_glued(C.byref(pr), C.byref(plan), C.byref(m), fake, 10, good, fake, 0, 7,
                                fake, 1 << 40, None) == 1  # unknown precision
        n = pam.pam_eval_glued_workspace_size(pr, plan, 1000)
        assert n >= 1000 * (1 << len(n_cells)) * 16
        dim = len(n_cells)
        too_many = ((1 << 31) - 1) // (1 << dim) + 1
        assert L.pam_eval_glued_workspace_size(C.byref(pr), C.byref(plan), too_many,
                                               C.byref(C.c_size_t(0))) == 6


@pytest.mark.parametrize("mesh", ["triangles", "graded3d", "grid1d"])
def test_partition_cells_matches_the_oracle(pam, mesh):
    from paper_2605_16564_gb300 import fields
    if mesh == "triangles":
        shape, n_sub, ov = (40, 33), (3, 4), 2
        x, _ = fields.triangle_mesh(40, seed=5, ny=33)
    elif mesh == "graded3d":
        shape, n_sub, ov = (12, 14, 9), (2, 3, 2), 1
        x, _ = fields.graded_mesh(shape, seed=6)
    else:
        shape, n_sub, ov = (50,), (7,), 3
        x = fields.grid_as_cells(np.ones(50), shape)[0]
    pr = pam.make_problem(shape, n_sub, ov, (2,) * len(shape))
    start, cells = pam.pam_partition_cells(pr, x)
    _, ostart, ocells = oracle.partition_cells(shape, n_sub, ov, x)
    np.testing.assert_array_equal(start, ostart)
    np.testing.assert_array_equal(cells, ocells)


def test_cells_entry_points_check_their_arguments(pam):
    import ctypes as C
    from paper_2605_16564_gb300 import fields
    pr = pam.make_problem((16, 16), (2, 2), 1, (2, 2))
    x, vol = fields.triangle_mesh(16, seed=1)
    start, cells = pam.pam_partition_cells(pr, x)
    # a point outside the domain, or NaN
    for bad in ((1.5, 0.5), (np.nan, 0.2), (-0.01, 0.3)):
        xb = x.copy()
        xb[3] = bad
        with pytest.raises(pam.PamError):
            pam.pam_partition_cells(pr, xb)
    # the Gauss-Legendre rule needs element shapes
    with pytest.raises(pam.PamError) as e:
        pam.pam_plan_create_cells(pr, pam.make_params(quad=1), x.shape[0], start)
    assert e.value.code == pam.PAM_ERR_UNSUPPORTED
    plan = pam.pam_plan_create_cells(pr, pam.make_params(levels=1, k_top=3), x.shape[0], start)
    assert plan.max_patch_cells % 32 == 0 and plan.max_patch_cells >= int(np.diff(start).max())
    grid_plan = pam.pam_plan_create(pr, pam.make_params(levels=1, k_top=3))
    assert plan.workspace_bytes > grid_plan.workspace_bytes or plan.max_patch_cells != grid_plan.max_patch_cells
    fake = C.c_void_p(256)
    m = pam.pam_model(fake, fake, fake, fake)
    par = pam.make_params(levels=1, k_top=3)
    L = pam.lib()
    good = pam.pam_cells(x.shape[0], 256, 256, 256, 256)
    for cells_s in (pam.pam_cells(x.shape[0] + 1, 256, 256, 256, 256),   # count differs from the plan
                    pam.pam_cells(x.shape[0], 0, 256, 256, 256)):         # missing points
        assert L.pam_fit_cells(C.byref(pr), C.byref(par), C.byref(plan), C.byref(cells_s), fake, C.byref(m),
                               fake, 1 << 40, None) == 1
    assert L.pam_fit_cells(C.byref(pr), C.byref(par), C.byref(plan), C.byref(good), fake, C.byref(m),
                           fake, 16, None) == 4  # workspace too small
    assert L.pam_errors_cells(C.byref(pr), C.byref(plan), C.byref(m), C.byref(good), fake, fake, 5, fake,
                              1 << 40, None) == 1  # unknown precision


def test_model_blob_checks_without_a_gpu(pam):
    import ctypes as C
    pr = pam.make_problem((32, 32), (2, 2), 1, (3, 3))
    plan = pam.pam_plan_create(pr, pam.make_params(levels=1, k_top=4))
    fake = C.c_void_p(256)
    m = pam.pam_model(fake, fake, fake, fake)
    L = pam.lib()
    n = C.c_size_t(0)
    assert L.pam_model_save(C.byref(pr), C.byref(plan), C.byref(m), None, C.byref(n), None) == 0
    S, mc = plan.n_subdomains, plan.m_cap
    assert n.value == 80 + S * 12 * 4 + S * mc * 40 + S * 8 * 4
    small = C.c_size_t(16)
    buf = (C.c_uint8 * 16)()
    assert L.pam_model_save(C.byref(pr), C.byref(plan), C.byref(m), buf, C.byref(small), None) == 1
    assert small.value == n.value
    # a blob with the right header but boxes of another decomposition is rejected
    # before anything is copied
    blob = np.zeros(n.value, dtype=np.uint8)
    hdr = np.zeros(18, dtype=np.int32)
    hdr[0], hdr[1] = 1, 2                    # version, dim
    hdr[2:5] = (32, 32, 1); hdr[5:8] = (2, 2, 1); hdr[8] = 1; hdr[9:12] = (3, 3, 1)
    hdr[12], hdr[13] = S, mc
    blob[:8] = np.frombuffer(b"PAMMODEL", dtype=np.uint8)
    blob[8:80] = hdr.view(np.uint8)
    assert L.pam_model_load(C.byref(pr), C.byref(plan), blob.ctypes.data, blob.size, C.byref(m), None) == 1
    boxes = pam.pam_partition(pr)
    blob[80:80 + boxes.nbytes] = boxes.reshape(-1).view(np.uint8)
    # boxes right, but every M_i is 0
    assert L.pam_model_load(C.byref(pr), C.byref(plan), blob.ctypes.data, blob.size, C.byref(m), None) == 1
    blob2 = blob.copy()
    blob2[0] = ord("X")
    assert L.pam_model_load(C.byref(pr), C.byref(plan), blob2.ctypes.data, blob2.size, C.byref(m), None) == 1
    assert L.pam_model_load(C.byref(pr), C.byref(plan), blob.ctypes.data, blob.size - 1, C.byref(m), None) == 1


def test_tuning_set_get_and_checks(pam):
    pam.pam_tuning_set(reset=True)
    assert pam.pam_tuning_get() == dict(factor_kb=0, gram_stages=0, eval_block=0, solve_persistent=0,
                                        level_groups=0)
    pam.pam_tuning_set(factor_kb=48, gram_stages=2, eval_block=512, solve_persistent=1, level_groups=2)
    want = dict(factor_kb=48, gram_stages=2, eval_block=512, solve_persistent=1, level_groups=2)
    assert pam.pam_tuning_get() == want
    for bad in (dict(factor_kb=-1), dict(factor_kb=2), dict(gram_stages=4), dict(gram_stages=1), dict(eval_block=300),
                dict(solve_persistent=2), dict(solve_persistent=-1), dict(level_groups=3), dict(level_groups=-1)):
        with pytest.raises(pam.PamError):
            pam.pam_tuning_set(**bad)
    assert pam.pam_tuning_get() == want  # unchanged
    pam.pam_tuning_set(reset=True)
    assert pam.pam_tuning_get()["factor_kb"] == 0


def test_selftest_wait_checks_its_arguments(pam):
    import ctypes as C
    L = pam.lib()
    fake = C.c_void_p(256)
    assert L.pam_selftest_wait(2, 100000, fake, None) == 1
    assert L.pam_selftest_wait(0, 10, fake, None) == 1
    assert L.pam_selftest_wait(0, 100000, None, None) == 1


def test_partition_cells_on_faces_matches_the_oracle(pam):
    # sampling points exactly on cell faces, core faces, patch faces and the
    # outer faces of the domain (h = 1/16, so k h is exact): the half-open
    # rule, closed at the outer face
    shape, n_sub, ov = (16, 12), (4, 3), 2
    h = 1.0 / 16
    xs = np.arange(0, 17) * h
    ys = np.arange(0, 13) * h
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    x = np.stack([X.reshape(-1), Y.reshape(-1)], axis=1)
    pr = pam.make_problem(shape, n_sub, ov, (2, 2))
    start, cells = pam.pam_partition_cells(pr, x)
    _, ostart, ocells = oracle.partition_cells(shape, n_sub, ov, x)
    np.testing.assert_array_equal(start, ostart)
    np.testing.assert_array_equal(cells, ocells)
    # every point lies in some patch, and a point one ulp outside the outer
    # face is an input error (the library does not drop it silently)
    assert np.bincount(cells, minlength=x.shape[0]).min() >= 1
    with pytest.raises(pam.PamError):
        pam.pam_partition_cells(pr, np.array([[0.5, np.nextafter(0.75, 1.0)]]))


def test_binding_struct_layouts_match_the_library(pam):
    # the ctypes structs of the binding against sizeof in the compiled library
    import ctypes as C
    out = (C.c_size_t * 6)()
    assert pam.lib().pam_struct_sizes(out, 6) == 6
    mine = [C.sizeof(t) for t in (pam.pam_problem, pam.pam_params, pam.pam_plan, pam.pam_model,
                                  pam.pam_cells, pam.pam_tuning)]
    assert list(out) == mine
    # pam_params: 4 doubles, 8 ints, the warm-start event pointer
    assert C.sizeof(pam.pam_params) == 4 * 8 + 8 * 4 + 8 + 2 * 4  # ..., the event, the subdomain range
    assert pam.pam_params.warm_start_event.offset == 64


def test_event_handles(pam):
    class Ev:
        def __init__(self, h):
            self.cuda_event = h
    assert pam._event_handle(None) is None
    assert pam._event_handle(12345) == 12345
    assert pam._event_handle(Ev(777)) == 777
    with pytest.raises(ValueError):
        pam._event_handle(Ev(0))


def test_eval_to_host_checks_its_buffers_before_any_launch(pam):
    import torch
    pts = torch.zeros((10, 2), dtype=torch.float64)
    out = torch.zeros(10, dtype=torch.float64)
    with pytest.raises(ValueError):
        pam.Fitter.eval_to_host(None, pts, out[:9], torch.zeros(10, dtype=torch.float64))
    with pytest.raises(ValueError):
        pam.Fitter.eval_to_host(None, pts, out, torch.zeros(9, dtype=torch.float64))
    with pytest.raises(ValueError):
        pam.Fitter.eval_to_host(None, pts, out, torch.zeros(10, dtype=torch.float32))
    # pam_eval writes binary64 values on the fitter's device: a host or
    # float32 `out` is refused before anything is enqueued
    with pytest.raises(ValueError):
        pam.Fitter.eval_to_host(None, pts, out, torch.zeros(10, dtype=torch.float64))
    with pytest.raises(ValueError):
        pam.Fitter.eval_to_host(None, pts, out.float(), torch.zeros(10, dtype=torch.float32))


def test_subdomain_range_and_error_sums_are_checked(pam):
    prob = pam.make_problem((32, 32), (2, 2), 1, (3, 3))
    for bad in ((-1, 2), (3, 2), (0, 5)):
        with pytest.raises(pam.PamError):
            pam.pam_plan_create(prob, pam.make_params(k_top=2, levels=1, sub_range=bad))
    plan = pam.pam_plan_create(prob, pam.make_params(k_top=2, levels=1, sub_range=(1, 3)))
    assert plan.n_subdomains == 4
    import ctypes as C
    m = pam.pam_model()
    for bad in ((-1, 2), (3, 2), (0, 5)):
        code = pam.lib().pam_error_sums(C.byref(prob), C.byref(plan), C.byref(m), None, None, 0, 0, bad[0], bad[1],
                                        None, 0, None)
        assert code == pam.PAM_ERR_INVALID_ARG
    s = np.array([6.0, 12.0, 8.0, 32.0, 3.0, 6.0, np.log(10.0) * 0.5, 0.0])
    e = pam.error_measures_from_sums(s)
    assert e == dict(l1=0.5, l2=0.5, l1_log=0.5, max_log10=pytest.approx(0.5))


def _check_group_layout(groups, S):
    F = min(S, 32)
    subs, order, lists, slots = [], [], [], []
    for g in groups:
        subs += [g["first"] + i * g["stride"] for i in range(g["count"])]
        order += list(range(g["order_offset"], g["order_offset"] + g["count"]))
        lists += list(range(g["list_offset"], g["list_offset"] + 2 + g["slots"]))
        slots += list(range(g["first_slot"], g["first_slot"] + g["slots"]))
        assert g["slots"] >= 1
        if S <= 32:  # every subdomain of the group can take a slot, as in one list
            assert g["slots"] == g["count"]
    # the groups partition the subdomains, the order region, the slots; the
    # lists fit the 4 + F words carved for them, without overlap
    assert sorted(subs) == list(range(S))
    assert sorted(order) == list(range(S))
    assert sorted(slots) == list(range(F))
    assert len(set(lists)) == len(lists) and max(lists) < 4 + F


def test_subdomain_group_layout(pam):
    pam.pam_tuning_set(reset=True)
    try:
        for S in (1, 2, 3, 9, 25, 64, 1023):
            groups = pam.pam_group_layout(S)
            assert len(groups) == 1 and groups[0] == dict(first=0, stride=1, count=S, order_offset=0,
                                                          list_offset=0, slots=min(S, 32), first_slot=0)
        for S in (1024, 1025, 2244, 5001):
            groups = pam.pam_group_layout(S)
            assert len(groups) == 2 and [g["first"] for g in groups] == [0, 1]
            _check_group_layout(groups, S)
        pam.pam_tuning_set(level_groups=2)
        for S in (2, 3, 9, 25, 33, 64, 1023):
            groups = pam.pam_group_layout(S)
            assert len(groups) == 2
            _check_group_layout(groups, S)
        assert len(pam.pam_group_layout(1)) == 1  # one subdomain: one fallback slot, one group
        pam.pam_tuning_set(level_groups=1)
        assert len(pam.pam_group_layout(2244)) == 1
        with pytest.raises(pam.PamError):
            pam.pam_group_layout(0)
    finally:
        pam.pam_tuning_set(reset=True)
