"""Benchmark of the PAM fitting path on GB300.

One step = the whole path on one synthetic field: partition, Step 2 fit,
three refinement levels (Algorithm 1), evaluation of the surrogate on the
2x refined target mesh, and the error reduction. Workload (default): the
60 x 220 x 85 layered field (1,122,000 cells), 6 x 22 x 17 subdomains with a
1-cell overlap, 4 x 4 x 2 initial centres, 3 levels, evaluated on the
120 x 440 x 170 cell-centred mesh (8,976,000 points).

Prints ONE JSON line (rank 0). `value` = source cells fitted and evaluated
per second, whole job, inputs resident in HBM; `e2e` = the same through the
C ABI from pinned host buffers, copies included. Multi-GPU: every rank fits
its own field (weak scaling, no collective on the data path); the step time
is the maximum over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pam|reference]
                  [--precision auto|fp64|mixed] [--workload layered3d|voronoi2d|...]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2605_16564_gb300 import fields  # noqa: E402

METRIC = "cells fit/s & eval pts/s, chosen vs plain GPU form at equal L1 error"

WORKLOADS = {
    # name: (shape, n_sub, overlap, g_init, params, eval mesh counts, field maker)
    "layered3d": dict(shape=(60, 220, 85), n_sub=(6, 22, 17), overlap=1, g=(4, 4, 2),
                      params=dict(k_top=30, levels=3), eval_counts=(120, 440, 170),
                      field=lambda seed: fields.layered_field((60, 220, 85), seed=seed), seed=5),
    "layered3d_quarter": dict(shape=(30, 110, 85), n_sub=(3, 11, 17), overlap=1, g=(4, 4, 2),
                              params=dict(k_top=30, levels=3), eval_counts=(60, 220, 170),
                              field=lambda seed: fields.layered_field((30, 110, 85), seed=seed), seed=5),
    "channel2d": dict(shape=(1024, 1024), n_sub=(32, 32), overlap=2, g=(8, 8),
                      params=dict(k_top=37, levels=3), eval_counts=(1536, 1536),
                      field=lambda seed: fields.channel_field(1024, seed=seed), seed=3),
    "voronoi2d": dict(shape=(256, 256), n_sub=(8, 8), overlap=2, g=(8, 8),
                      params=dict(k_top=37, levels=3), eval_counts=(384, 384),
                      field=lambda seed: fields.voronoi_field(256, seed=seed), seed=2),
    # the channel workload on an unstructured mesh: every square of the
    # 1024 x 1024 grid cut along a seeded random diagonal into two triangles
    # (2,097,152 elements), each triangle carrying its square's value
    "triangles2d": dict(shape=(1024, 1024), n_sub=(32, 32), overlap=2, g=(8, 8),
                        params=dict(k_top=37, levels=3), eval_counts=(1536, 1536),
                        field=lambda seed: fields.channel_field(1024, seed=seed), seed=3,
                        mesh="triangles", mesh_seed=31, cpu_sample=32),
    "disc2d": dict(shape=(64, 64), n_sub=(1, 1), overlap=0, g=(16, 16),
                   params=dict(k_top=51, levels=2), eval_counts=(97, 97),
                   field=lambda seed: fields.disc_field(64), seed=0),
}

# slices of the end-to-end evaluation whose device-to-host copies overlap
# the evaluation of the next slices (--e2e-slices; each slice repeats the
# owner lookup and the per-owner staging of the dictionaries). Measured on
# the layered 3-D workload: 1 slice 16.15 ms, 2 slices 15.90, 4 slices 16.14
# per end-to-end step (the copies run at ~195-210 GB/s each way).
E2E_EVAL_CHUNKS = 2

# "eval_kernel" (the per-owner evaluation kernel alone) is timed inside "eval"
PHASES = ["prepare", "assemble", "gram", "solve", "residual", "mark", "eval", "errors", "stats",
          "gram_tc", "refine", "eval_kernel"]


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return rank, ws


def max_over_ranks(x: float, ws: int, device=None) -> float:
    """Maximum of a scalar over ranks (timing only; no data-path exchange)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def shard_ranges(costs, world: int):
    """Contiguous blocks of subdomains, one per rank, with about equal
    estimated cost (the prefix sums cut nearest to k/world of the total;
    section 2's subdomains are independent, so a rank fits its block alone):
    [(begin, end)] * world, covering every subdomain exactly once."""
    c = np.concatenate([[0.0], np.cumsum(np.asarray(costs, dtype=float))])
    S = len(c) - 1
    cuts = [0]
    for k in range(1, world):
        target = c[-1] * k / world
        i = int(np.searchsorted(c, target))
        i = min(max(i, 1), S)
        if abs(c[i - 1] - target) < abs(c[i] - target):
            i -= 1
        cuts.append(max(i, cuts[-1]))
    cuts.append(S)
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


def shard_costs(W):
    """Estimated cost of each subdomain: N_i M_cap^2, N_i its patch cells and
    M_cap the dictionary cap after the planned levels (the fit's Gram and
    solve scale with N M^2; the final M_i are not known before the fit)."""
    boxes = _patch_boxes(W)
    n = np.prod(boxes[:, 9:12] - boxes[:, 6:9], axis=1).astype(float)
    dim = len(W["shape"])
    m_cap = int(np.prod(W["g"])) + W["params"]["levels"] * (dim + 1) * W["params"]["k_top"]
    return n * float(m_cap) ** 2


def _patch_boxes(W):
    """Core and patch boxes [S, 12] of a workload (half-open cores, overlap clipped)."""
    shape, n_sub, ov = W["shape"], W["n_sub"], W["overlap"]
    dim = len(shape)
    S = int(np.prod(n_sub))
    boxes = np.zeros((S, 12), dtype=np.int64)
    for sidx in range(S):
        j, rem = [], sidx
        for a in range(dim):
            j.append(rem % n_sub[a])
            rem //= n_sub[a]
        for a in range(3):
            if a < dim:
                n, p = shape[a], n_sub[a]
                lo, hi = (j[a] * n) // p, ((j[a] + 1) * n) // p
                boxes[sidx, [a, 3 + a, 6 + a, 9 + a]] = [lo, hi, max(lo - ov, 0), min(hi + ov, n)]
            else:
                boxes[sidx, [a, 3 + a, 6 + a, 9 + a]] = [0, 1, 0, 1]
    return boxes


def shard_seed(base_seed: int, rank: int) -> int:
    """Each rank fits its own field: weak scaling over independent problems."""
    return base_seed + 1000 * rank


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# Nominal FP64 rate of GB300 (dense, per GPU), the peak of the binary64 path.
FP64_NOMINAL_TFLOPS = 1.25


def accounting(fit, Kd, levels, pam, seed=None):
    """Algorithmic work of one step, counted from the sizes each solve actually
    had (the fit is re-run level by level outside the timed region):
      gram_flops  sum N_i M_i (M_i + 1): the multiply-adds of the upper
                  triangle of the symmetric W^T W, two flops each;
      pairs       sum N_i M_i: Gaussians evaluated once per (cell, centre);
      chol_flops  sum iters * s^3 / 3 over the active-set steps (fp32 form);
      eval_pairs  filled in by the caller (points x their owner's M)."""
    out = dict(gram_flops=0.0, pairs=0.0, chol_flops=0.0, solve_bytes=0.0, m_final=None, solves=0,
               steps=0.0, passes=0.0, support_last=None, records=[])
    fit_levels = [0] + [1] * levels
    for r, _ in enumerate(fit_levels):
        if r == 0:
            if seed is not None:
                seed()
                fit.params.warm_start = 1
            if getattr(fit, "cells", None) is not None:
                pam.pam_fit_cells(fit.problem, fit.params, fit.plan, fit.cells, Kd, fit.model, fit.workspace)
            else:
                pam.pam_fit_subdomains(fit.problem, fit.params, fit.plan, Kd, fit.model, fit.workspace)
            fit.params.warm_start = 0
        elif getattr(fit, "cells", None) is not None:
            pam.pam_refine_cells(fit.problem, fit.params, fit.plan, fit.cells, Kd, fit.model, 1, fit.workspace)
        else:
            pam.pam_refine(fit.problem, fit.params, fit.plan, Kd, fit.model, 1, fit.workspace)
        info = fit.model.info.cpu().numpy()
        solved = info[:, pam.INFO_STOPPED] == 0 if r > 0 else np.ones(len(info), bool)
        n = info[solved, pam.INFO_N_CELLS].astype(float)
        m = info[solved, pam.INFO_M].astype(float)
        sup = info[solved, pam.INFO_SUPPORT].astype(float)
        iters = (info[solved, pam.INFO_ITERS] % 100).astype(float)
        passes = (info[solved, pam.INFO_ITERS] // 100).astype(float)
        out["gram_flops"] += float(np.sum(n * m * (m + 1.0)))
        out["pairs"] += float(np.sum(n * m))
        out["chol_flops"] += float(np.sum(iters * sup ** 3 / 3.0))
        # Gram streaming of the solve: every active-set step and refinement
        # pass reads the support block (s^2) and the support's rows (s M) of
        # the fp32 Gram (s = the final support, the step count of the solve)
        out["solve_bytes"] += float(np.sum((iters + passes) * (sup * sup + sup * m) * 4.0))
        out["solves"] += int(np.count_nonzero(solved))
        out["steps"] += float(np.sum(iters))
        out["passes"] += float(np.sum(passes))
        out["support_last"] = float(sup.mean()) if len(sup) else 0.0
        flags = info[solved, pam.INFO_FLAGS]
        for k, sd in enumerate(np.flatnonzero(solved)):
            out["records"].append({"level": r, "subdomain": int(sd), "cells": int(n[k]), "centres": int(m[k]),
                                   "support": int(sup[k]), "active_set_steps": int(iters[k]),
                                   "refinement_passes": int(passes[k]), "flags": int(flags[k])})
    out["m_final"] = fit.model.info.cpu().numpy()[:, pam.INFO_M].astype(float)
    return out


def solve_distribution(records):
    """Per level: how the solves' support sizes and active-set steps are
    spread (median, 90th percentile, maximum) and how many were flagged --
    where the solve's tail comes from."""
    out = {}
    for lv in sorted({r["level"] for r in records}):
        rs = [r for r in records if r["level"] == lv]
        d = {"solves": len(rs)}
        for key in ("centres", "support", "active_set_steps", "refinement_passes"):
            v = np.array([r[key] for r in rs], dtype=float)
            d[key] = {"p50": float(np.percentile(v, 50)), "p90": float(np.percentile(v, 90)), "max": float(v.max())}
        d["flagged"] = int(sum(1 for r in rs if r["flags"]))
        out[f"level{lv}"] = d
    return out


# Special-function-unit rate: 16 ex2 per SM per clock (4 per SM sub-partition)
# x 152 SMs x 2.07 GHz, the roof of the exp-bound kernels.
SFU_EX2_PER_S = 152 * 16 * 2.07e9
# fp32 FMA rate: 128 lanes per SM x 2 flops x 152 SMs x 2.07 GHz.
FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


# DRAM bytes (read + write) of one launch of each mixed-form kernel on the
# layered 3-D workload: ncu of the last level's launch on the quarter-size
# workload (561 of the 2,244 subdomains, same subdomain shape), scaled by 4
# (profiles/solve_layered3d_quarter_mixed.md for the solve,
# profiles/gram_tc_layered3d_quarter_mixed.md for the tensor-core Gram and the
# evaluation). Only valid for that workload and for the kernels as captured
# (the statistics changed after their last capture: none recorded).
TRAFFIC_LAYERED3D = {"k_solve_mixed": 1.378e9, "k_gram_tc": 1.224e9, "k_eval_bucket_f32": 2.94e8}
TRAFFIC_NOTE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the level-3 launch (eval: its one launch), "
                "captured on layered3d_quarter and scaled x4 by subdomains")


def roofline_entries(phase_ms, work, n_pts, mixed, peaks, peak_src):
    """Roofline objects per kernel family: achieved = algorithmic work per
    step / that family's CUDA-event time per step."""
    r = {}
    def t(k):
        return phase_ms[k][0] / 1e3 if k in phase_ms else None
    if t("gram_tc"):
        ach = work["gram_flops"] / t("gram_tc") / 1e12
        pk = peaks.get("bf16_tflops", 1900.0)
        r["gram_tc"] = {"kernel": "k_gram_tc", "bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                        "frac": ach / pk, "traffic": None,
                        "peak_source": f"bf16_tflops of {peak_src} (the kernel issues 3 bf16 products per flop pair)"}
    if t("gram"):
        ach = work["gram_flops"] / t("gram") / 1e12
        r["gram"] = {"kernel": "k_gram_f64", "bound": "alu", "achieved": ach, "peak": FP64_NOMINAL_TFLOPS,
                     "unit": "TFLOP/s", "frac": ach / FP64_NOMINAL_TFLOPS, "traffic": None,
                     "peak_source": "nominal GB300 fp64 dense rate"}
    if t("stats"):
        ach = work["pairs"] / t("stats")  # one pass of plain sums of 2^l
        r["stats"] = {"kernel": "k_stats_f32", "bound": "alu", "achieved": ach / 1e12,
                      "peak": SFU_EX2_PER_S / 1e12, "unit": "Texp/s", "frac": ach / SFU_EX2_PER_S,
                      "traffic": None, "peak_source": "SFU ex2 16/clk/SM x 152 SMs x 2.07 GHz"}
    if t("eval"):
        pairs = work.get("eval_pairs")
        if pairs:
            # the kernel's own time where it was recorded (the phase adds the
            # owner lookup, scan and scatter)
            te = t("eval_kernel") or t("eval")
            ach = pairs / te
            r["eval"] = {"kernel": "k_eval_bucket_f32" if mixed else "k_eval_bucket_f64", "bound": "alu",
                         "achieved": ach / 1e12, "peak": SFU_EX2_PER_S / 1e12, "unit": "Texp/s",
                         "frac": ach / SFU_EX2_PER_S, "traffic": None,
                         "peak_source": "SFU ex2 16/clk/SM x 152 SMs x 2.07 GHz",
                         "timed": "the kernel alone" if t("eval_kernel") else "the evaluation phase",
                         "phase_frac": pairs / t("eval") / SFU_EX2_PER_S}
    if t("solve") and mixed:
        ach = work["solve_bytes"] / t("solve") / 1e9
        pk = peaks.get("hbm_gbs", 6800.0)
        chol = work["chol_flops"] / t("solve") / 1e12
        r["solve"] = {"kernel": "k_solve_mixed", "bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s",
                      "frac": ach / pk, "traffic": None,
                      "peak_source": f"hbm_gbs of {peak_src}; work = Gram streaming, (steps + refinement passes) "
                                     "x (s^2 + s M) x 4 bytes per subdomain and level (latency-bound: one CTA "
                                     "per subdomain, see the clock-counter split)",
                      "cholesky_tflops": chol, "cholesky_frac_of_fp32": chol / FP32_TFLOPS}
        if work.get("solves"):
            # sweeps per subdomain: the solve's active-set steps (one support
            # factorisation each) and exact-gradient refinement passes, per
            # (subdomain, level) solve
            r["solve"]["solves_per_step"] = work["solves"]
            r["solve"]["active_set_steps_per_solve"] = work["steps"] / work["solves"]
            r["solve"]["refinement_passes_per_solve"] = work["passes"] / work["solves"]
            r["solve"]["mean_support_last_level"] = work["support_last"]
    return r


def attach_traffic(roofs, workload):
    """Fill `traffic` from the recorded ncu capture where it applies."""
    if workload != "layered3d":
        return roofs
    for v in roofs.values():
        t = TRAFFIC_LAYERED3D.get(v.get("kernel"))
        if t is not None:
            v["traffic"] = t
            v["traffic_note"] = TRAFFIC_NOTE
    return roofs


def workload_data(W, seed):
    """(K, x, vol): the cell values of the workload and, for a mesh given as
    cells, the element sampling points and measures (else None, None)."""
    K = W["field"](seed)
    if W.get("mesh") == "triangles":
        x, vol = fields.triangle_mesh(W["shape"][0], seed=W["mesh_seed"], ny=W["shape"][1])
        return np.repeat(np.ascontiguousarray(K).reshape(-1), 2), x, vol
    return K, None, None


def dictionary_agreement(pam, mixed, plain):
    """Where the mixed form's refinement took other decisions than the plain
    binary64 form's (which meets the oracle's to 1e-9): the fraction of
    subdomains whose final dictionary differs (fp32 rounding moved a marking
    decision), and how many of the mixed form's last solves fell back to
    binary64 or stayed uncertified."""
    S = len(plain["M"])
    differ = 0
    for s in range(S):
        m = int(plain["M"][s])
        if int(mixed["M"][s]) != m or not np.array_equal(mixed["c"][s, :m], plain["c"][s, :m]):
            differ += 1
    flags = mixed["info"][:, pam.INFO_FLAGS]
    return {"subdomains": S, "dictionaries_differing": differ, "fraction_differing": differ / max(S, 1),
            "mixed_solves_fallen_back_to_fp64": int(np.count_nonzero(flags & pam.FLAG_REFINE_DIVERGED)),
            "mixed_solves_uncertified": int(np.count_nonzero(flags & pam.FLAG_NOT_CERTIFIED))}


def combine_error_sums(sums, ws):
    """The shards' raw error sums (pam_error_sums, a tensor [8]) added over the
    ranks, the maximum taken for entry 6: the one collective of a sharded
    field (section 8(e)), a handful of scalars after the step."""
    if ws == 1:
        return sums
    import torch
    import torch.distributed as dist
    top = sums[6:7].clone()
    dist.all_reduce(sums, op=dist.ReduceOp.SUM)
    dist.all_reduce(top, op=dist.ReduceOp.MAX)
    sums[6] = top[0]
    return sums


def run_field_shard(args, rank, ws):
    """One field split over the ranks: rank r fits the contiguous block of
    subdomains shard_ranges gives it (pam_params.sub_begin/sub_end), evaluates
    the target points its block owns and reduces its error sums; the sums are
    added over the ranks after the timed steps. Strong scaling: the whole
    job's work is fixed."""
    import torch
    from paper_2605_16564_gb300 import build, pam
    build.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    W = WORKLOADS[args.workload]
    if W.get("mesh"):
        raise SystemExit("--shard field: grid workloads only")
    K, _, _ = workload_data(W, W["seed"])  # the same field on every rank
    b, e = shard_ranges(shard_costs(W), ws)[rank]
    h = fields.cell_size(W["shape"])
    pts = fields.cell_centred_points(W["eval_counts"], [n * h for n in W["shape"]])
    own = owner_index(W, pts)
    mine = np.ascontiguousarray(pts[(own >= b) & (own < e)])
    prec = pam.PAM_PREC_MIXED if (args.precision in ("auto", "mixed") and _mixed_available(pam)) \
        else pam.PAM_PREC_FP64
    fit = make_fitter(pam, W, None, None, dev, precision=prec, sub_range=(b, e), **W["params"])
    Kd = torch.from_numpy(np.ascontiguousarray(K)).to(dev)
    ptsd = torch.from_numpy(mine).to(dev)
    out = torch.empty(max(len(mine), 1), dtype=torch.float64, device=dev)
    sums = torch.zeros(8, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        fit.fit(Kd, deferred=True)
        if len(mine):
            fit.eval(ptsd, out=out[:len(mine)])
        pam.pam_error_sums(fit.problem, fit.plan, fit.model, Kd, sums, (b, e), fit.workspace, prec)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if fit.status() not in (0,):
        raise SystemExit(f"rank {rank}: fit status {fit.status()}")
    times = []
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(ws)
        torch.cuda.synchronize()
        e0.record()
        step()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = max_over_ranks(sum(times) / len(times), ws, dev)
    tot = combine_error_sums(sums, ws).cpu().numpy()
    if rank != 0:
        return
    err = pam.error_measures_from_sums(tot)
    n_cells = int(np.prod(W["shape"]))
    line = {"metric": METRIC, "value": n_cells / (ms / 1e3), "unit": "cells/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "bf16x3+f32+f64" if prec == pam.PAM_PREC_MIXED else "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "parallelism": f"one field, {ws} contiguous subdomain blocks",
                       "ranges_rank0": [b, e], "l2_flush": "256 MB buffer written between timed steps",
                       "launch": "eager"},
            "l1_rel": err["l1"], "l2_rel": err["l2"], "gpu_launches": None}
    print(json.dumps(line))


def make_fitter(pam, W, x, vol, dev, **params):
    if x is not None:
        return pam.CellFitter(W["shape"], W["n_sub"], W["overlap"], W["g"], x, vol, device=dev, **params)
    return pam.Fitter(W["shape"], W["n_sub"], W["overlap"], W["g"], device=dev, **params)


def run_pam(args, rank, ws):
    import torch
    from paper_2605_16564_gb300 import build, pam

    build.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    W = WORKLOADS[args.workload]
    K, x_el, vol_el = workload_data(W, shard_seed(W["seed"], rank))
    shape = W["shape"]
    h = fields.cell_size(shape)
    extent = [n * h for n in shape]
    pts = fields.cell_centred_points(W["eval_counts"], extent)
    n_cells = int(np.asarray(K).size)  # grid cells, or the elements of a mesh given as cells
    n_pts = pts.shape[0]

    prec_name = args.precision
    if prec_name == "auto":
        prec_name = "mixed" if _mixed_available(pam) else "fp64"
    prec = pam.PAM_PREC_MIXED if prec_name == "mixed" else pam.PAM_PREC_FP64

    fit = make_fitter(pam, W, x_el, vol_el, dev, precision=prec, quad=args.quad, **W["params"])
    Kd = torch.from_numpy(np.ascontiguousarray(K)).to(dev)
    ptsd = torch.from_numpy(pts).to(dev)
    out = torch.empty(n_pts, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    # learned warm start of the level-0 solves (3-D decompositions, mixed
    # form): trained once, outside the timed region, on other seeded fields
    # of the same workload; inference and seeding run inside every step
    lw, learned = None, None
    if prec == pam.PAM_PREC_MIXED and len(shape) == 3 and not args.no_learned:
        from paper_2605_16564_gb300 import warmstart
        t0 = time.perf_counter()
        lw = warmstart.LayeredWarmStart(dev, batch=256, seed=0)
        train = [torch.from_numpy(W["field"](shard_seed(W["seed"], rank) * 1000 + 100 + i)).to(dev)
                 for i in range(8)]
        lw.train(fit, train, epochs=8)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        del train
        it0 = lambda: (fit.model.info.cpu().numpy()[:, pam.INFO_ITERS] % 100).mean()
        fit.fit(Kd, levels=0)
        cold_it = float(it0())
        lw.seed(fit, Kd)
        fit.fit(Kd, levels=0, warm_start=True)
        warm_it = float(it0())
        learned = {"kind": "learned (PAM_NN_LAYERED3D network seeds the level-0 active set)",
                   "train_fields": 8, "train_samples": 8 * fit.plan.n_subdomains, "train_s": round(train_s, 2),
                   "seed_threshold": lw.threshold,
                   "inference_stream": "a high-priority side stream beside the level-0 partition, cell data "
                                       "and Gram products; the level-0 solve waits on its event",
                   "level0_active_set_steps_cold": round(cold_it, 3),
                   "level0_active_set_steps_learned": round(warm_it, 3)}

    # the inference runs on a side stream beside the level-0 partition, cell
    # data and Gram products; the level-0 solve waits for its event. The
    # stream has the high priority, so that the network's small kernels are
    # scheduled ahead of the set-up kernels they run beside
    seed_stream = torch.cuda.Stream(device=dev, priority=-1) if lw is not None else None
    seeded = torch.cuda.Event() if lw is not None else None

    def fit_step(deferred=False):
        if lw is not None:
            seed_stream.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(seed_stream):
                lw.seed(fit, Kd)
                seeded.record(seed_stream)
            fit.fit(Kd, warm_start=True, deferred=deferred, warm_start_event=seeded)
        else:
            fit.fit(Kd, deferred=deferred)

    errd = torch.zeros(4, dtype=torch.float64, device=dev)

    def step():
        fit_step()
        fit.eval(ptsd, out=out)
        return fit.errors(Kd)

    def step_body(seeded=True):
        # the same step without host synchronisation (deferred status), so
        # that it can be captured in a CUDA graph and replayed
        if seeded:
            fit_step(deferred=True)
        else:
            fit.fit(Kd, deferred=True)
        fit.eval(ptsd, out=out)
        fit.errors_device(Kd, errd)

    def check_status():
        code = fit.status()
        if code != 0:
            raise pam.PamError(code, "deferred fit")

    def capture(body, timed=False):
        cap = torch.cuda.Stream(device=dev)
        cap.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cap):
            body()  # one eager pass on a side stream before capture
        torch.cuda.current_stream().wait_stream(cap)
        torch.cuda.synchronize()
        check_status()
        g = torch.cuda.CUDAGraph()
        L.pam_timing_enable(1 if timed else 0)  # phase event pairs of the captured launches only
        try:
            with torch.cuda.graph(g):
                body()
        finally:
            L.pam_timing_enable(0)
        return g

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # launch tuning measured on this fitted problem (outside the timed region)
    tune = None
    if not args.no_autotune:
        choice, ms = fit.autotune(Kd, ptsd)
        names = ["gram_stages=3", "gram_stages=2", "factor_kb=builtin", "factor_kb=64", "factor_kb=48",
                 "factor_kb=32", "factor_kb=24", "factor_kb=16", "eval_block=128", "eval_block=256",
                 "eval_block=512", "eval_block=1024", "solve_persistent=0", "solve_persistent=1"]
        tune = {"chosen": choice, "median_ms": {n: round(float(v), 4) for n, v in zip(names, ms) if v >= 0}}
        for _ in range(2):
            step()
        torch.cuda.synchronize()

    L = pam.lib()
    import ctypes as C

    def read_phases():
        got = {}
        for i, name in enumerate(PHASES):
            tot, cnt = C.c_double(0), C.c_int(0)
            L.pam_timing_read(i, C.byref(tot), C.byref(cnt))
            if cnt.value:
                got[name] = (tot.value, cnt.value)
        return got

    # the timed step is a CUDA graph of the whole step (captured once), else
    # eager launches; the per-family phase times come from replays of a
    # second capture of the same step with the phase event pairs as graph
    # nodes, so that the timed replays carry no profiler nodes
    graph, graph_ph, mode = None, None, "eager"
    L.pam_timing_reset()
    if not args.no_graph:
        try:
            l0 = L.pam_kernel_launches()
            graph = capture(step_body, timed=False)
            launches_per_step = (L.pam_kernel_launches() - l0) // 2  # the eager pre-pass + the capture
            graph_ph = capture(step_body, timed=True)
            for _ in range(args.warmup):
                graph.replay()
            torch.cuda.synchronize()
            check_status()
            mode = "graph"
        except Exception as e:  # reported in the JSON line; the eager step is timed instead
            graph, graph_ph = None, None
            torch.cuda.synchronize()
            L.pam_timing_reset()
            mode = f"eager (graph capture failed: {type(e).__name__}: {str(e)[:160]})"
    if graph is None:
        L.pam_timing_enable(1)
        launches0 = L.pam_kernel_launches()
    times = []
    phase_tot = {}
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        for _ in range(args.steps):
            flush.fill_(1)  # L2 flush between timed steps (outside the events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            torch.cuda.nvtx.range_push("pam_step")  # lets a profiler select the timed steps
            if graph is not None:
                graph.replay()
            else:
                err = step()
            torch.cuda.nvtx.range_pop()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    if graph_ph is not None:
        # the phase times: as many replays of the profiled capture, each
        # after the same L2 flush, read one by one
        for _ in range(args.steps):
            flush.fill_(1)
            graph_ph.replay()
            torch.cuda.synchronize()
            for k, (t, c) in read_phases().items():
                a = phase_tot.setdefault(k, [0.0, c])
                a[0] += t
    barrier(ws)
    phase_ms = {}
    if graph is not None:
        check_status()
        err = pam.error_dict(errd)
        launches = launches_per_step * args.steps
        phase_ms = {k: (v[0] / args.steps, v[1]) for k, v in phase_tot.items()}
    else:
        launches = L.pam_kernel_launches() - launches0
        L.pam_timing_enable(0)
        for k, (t, c) in read_phases().items():
            phase_ms[k] = (t / args.steps, c // args.steps)
    del graph, graph_ph
    torch.cuda.synchronize()
    L.pam_timing_reset()

    step_ms = max_over_ranks(sum(times) / len(times), ws, dev)
    value = n_cells * ws / (step_ms / 1e3)
    info = fit.model.info.cpu().numpy()
    def time_variant(body):
        # mean step time of `body` in the same launch mode and with the same
        # L2 flush as the timed steps (a graph of its own, when graphs are used)
        g2 = capture(body) if mode == "graph" else None
        ts = []
        for i in range(args.warmup + args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if g2 is not None:
                g2.replay()
            else:
                body()
            e1.record(stream)
            torch.cuda.synchronize()
            if i >= args.warmup:
                ts.append(e0.elapsed_time(e1))
        check_status()
        del g2
        return sum(ts) / len(ts)

    groups = None
    if prec == pam.PAM_PREC_MIXED:
        # the levels as one pipeline of launches over every subdomain,
        # against the two subdomain groups on two streams
        tsave = pam.pam_tuning_get()
        n_groups = 2 if tsave["level_groups"] == 2 or (
            tsave["level_groups"] == 0 and fit.plan.n_subdomains >= 1024) else 1
        pam.pam_tuning_set(**dict(tsave, level_groups=1))
        try:
            one_ms = time_variant(step_body)
        finally:
            pam.pam_tuning_set(**tsave)
        groups = {"groups": n_groups, "step_ms": round(step_ms, 3), "step_ms_one_pipeline": round(one_ms, 3),
                  "note": "two groups (even and odd subdomains) run their levels (the initial lattices' "
                          "solve and the refinement levels) on two streams, so that one group's solve tail "
                          "overlaps the other's work; the phase times come from one pipeline"}
    if lw is not None:
        # the same step without the learned seed (level 0 from beta = 0), for
        # comparison, in the same launch mode
        plain_ms = time_variant(lambda: step_body(seeded=False))
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        lw.seed(fit, Kd)
        t1.record(stream)
        torch.cuda.synchronize()
        learned["step_ms_learned"] = round(step_ms, 3)
        learned["step_ms_without_learned"] = round(plain_ms, 3)
        learned["inference_ms"] = round(t0.elapsed_time(t1), 3)

    # --- end to end through the C ABI from pinned host buffers -------------
    Kh = torch.from_numpy(np.ascontiguousarray(K)).pin_memory()
    ptsh = torch.from_numpy(pts).pin_memory()
    outh = torch.empty(n_pts, dtype=torch.float64).pin_memory()
    errh = torch.empty(4, dtype=torch.float64).pin_memory()
    side = torch.cuda.Stream(device=dev)  # the evaluation points and the result travel beside the fit
    pts_ready = torch.cuda.Event()
    k_ready = torch.cuda.Event()

    def e2e_body():
        cur = torch.cuda.current_stream()
        # the field first: the fit waits for it, and a points copy enqueued
        # ahead of it on the same copy engine delayed it by the whole 215 MB
        # (measured: 15.50 ms per end-to-end step that way, 14.47 with the
        # field's copy alone on the path)
        Kd.copy_(Kh, non_blocking=True)
        k_ready.record(cur)
        side.wait_event(k_ready)
        with torch.cuda.stream(side):
            ptsd.copy_(ptsh, non_blocking=True)
            pts_ready.record(side)
        fit_step(deferred=True)
        cur.wait_event(pts_ready)
        # evaluated in slices, each copied back while the next evaluates
        fit.eval_to_host(ptsd, out, outh, chunks=args.e2e_slices, copy_stream=side, join=False)
        fit.errors_device(Kd, errd)
        errh.copy_(errd, non_blocking=True)
        cur.wait_stream(side)

    ge = None
    if mode == "graph":
        try:
            ge = capture(e2e_body)
        except Exception:
            ge = None
    e2e_times = []
    for it in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if ge is not None:
            ge.replay()
        else:
            e2e_body()
        torch.cuda.synchronize()
        if it >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
    check_status()
    e2e_mode = "graph" if ge is not None else "eager"
    del ge
    e2e_s = max_over_ranks(sum(e2e_times) / len(e2e_times), ws, dev)
    h2d = Kh.numel() * 8 + ptsh.numel() * 8
    d2h = outh.numel() * 8 + errh.numel() * 8

    # --- the plain binary64 form, for the chosen-vs-plain ratio -------------
    plain = None
    if prec == pam.PAM_PREC_MIXED and not args.skip_plain:
        pf = make_fitter(pam, W, x_el, vol_el, dev, precision=pam.PAM_PREC_FP64, quad=args.quad, **W["params"])
        pf.fit(Kd)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        flush.fill_(1)
        e0.record(stream)
        pf.fit(Kd)
        pf.eval(ptsd, out=out)
        perr = pf.errors(Kd)
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1)
        plain = {"ms_per_step": pms, "cells_per_s": n_cells / (pms / 1e3), "l1": perr["l1"],
                 "speedup_chosen_over_plain": pms / step_ms,
                 "l1_ratio_chosen_over_plain": err["l1"] / perr["l1"]}
        plain.update(dictionary_agreement(pam, fit.host_model(), pf.host_model()))
        del pf

    # --- per-subdomain lambda choice by k-fold cross-validation -------------
    lcv = None
    if args.lambda_cv:
        grid = [(W["params"].get("lambda1_hat", 4.59e-4) * f, W["params"].get("lambda2_hat", 4.64e-6) * f)
                for f in (0.25, 1.0, 4.0)]
        folds = 3
        lcv = {"grid": [list(map(float, g)) for g in grid], "folds": folds}
        forms = [("mixed", pam.PAM_PREC_MIXED)] if prec == pam.PAM_PREC_MIXED else []
        forms.append(("fp64", pam.PAM_PREC_FP64))
        first = None
        for name, pr in forms:
            cf = pam.Fitter(shape, W["n_sub"], W["overlap"], W["g"], device=dev, precision=pr, **W["params"])
            if first is None:
                cf.fit(Kd, check=False)
                first = [t.clone() for t in (cf.model.boxes, cf.model.centres, cf.model.beta, cf.model.info)]
            else:  # the same dictionary as the first form's fit
                for dst, src in zip((cf.model.boxes, cf.model.centres, cf.model.beta, cf.model.info), first):
                    dst.copy_(src)
            beta0 = cf.model.beta.clone()
            info0 = cf.model.info.clone()
            L.pam_timing_reset()
            cv_times = []
            for i in range(1 + args.steps):
                cf.model.beta.copy_(beta0)
                cf.model.info.copy_(info0)
                flush.fill_(1)
                if i == 1:
                    L.pam_timing_enable(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                cv, choice, code = cf.lambda_cv(Kd, grid, folds)
                e1.record(stream)
                torch.cuda.synchronize()
                if i >= 1:
                    cv_times.append(e0.elapsed_time(e1))
            L.pam_timing_enable(0)
            ph = {k: round(v[0] / args.steps, 3) for k, v in read_phases().items()}
            L.pam_timing_reset()
            ms = sum(cv_times) / len(cv_times)
            S = cf.plan.n_subdomains
            n_unc = int(((cf.model.info.cpu().numpy()[:, pam.INFO_FLAGS] & pam.FLAG_NOT_CERTIFIED) != 0).sum())
            lcv[name] = {"ms": round(ms, 3), "solves": S * (len(grid) * folds + 1),
                         "solves_per_s": S * (len(grid) * folds + 1) / (ms / 1e3),
                         "cells_per_s": n_cells / (ms / 1e3), "status": int(code),
                         "refit_not_certified": n_unc,
                         "choice_histogram": np.bincount(choice.cpu().numpy(), minlength=len(grid)).tolist(),
                         "phase_ms": ph}
            if name == "mixed":
                cv_m = cv.cpu().numpy()
            else:
                cv_d = cv.cpu().numpy()
                if "mixed" in lcv:
                    lcv["mixed_vs_fp64_cv_max_rel"] = float(np.max(np.abs(cv_m - cv_d) / cv_d))
            del cf, beta0, info0
        del first

    # --- glued evaluation across subdomain interfaces (optional) ------------
    glue = None
    if args.glue > 0:
        gout = torch.empty_like(out)
        fit.eval_glued(ptsd, args.glue, out=gout)
        gtimes = []
        for i in range(args.warmup + args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fit.eval_glued(ptsd, args.glue, out=gout)
            e1.record(stream)
            torch.cuda.synchronize()
            if i >= args.warmup:
                gtimes.append(e0.elapsed_time(e1))
        fit.eval(ptsd, out=out)
        pw = out.cpu().numpy()
        gl = gout.cpu().numpy()
        gms = sum(gtimes) / len(gtimes)
        pairs = glue_pairs_per_point(W, pts, args.glue)
        glue = {"band_cells": args.glue, "ms": round(gms, 3), "pts_per_s": n_pts / (gms / 1e3),
                "pairs_per_point": round(float(pairs.mean()), 4),
                "points_blended": int((pairs > 1).sum()),
                "max_abs_log_change": float(np.nanmax(np.abs(np.log(gl) - np.log(pw))))}

    # --- roofline of every kernel family, the dominant one first ------------
    peaks, peak_src = _peaks()
    work = accounting(fit, Kd, W["params"]["levels"], pam, seed=(lambda: lw.seed(fit, Kd)) if lw else None)
    if args.metrics_log and rank == 0:
        # one JSON object per subdomain and level of the step's fit
        with open(args.metrics_log, "w") as fh:
            for rec in work["records"]:
                fh.write(json.dumps(rec) + "\n")
    owners = owner_counts(W, pts)
    work["eval_pairs"] = float(np.sum(owners * work["m_final"]))
    roofs = attach_traffic(roofline_entries(phase_ms, work, n_pts, prec == pam.PAM_PREC_MIXED, peaks, peak_src),
                           args.workload)
    dom = max(phase_ms.items(), key=lambda kv: kv[1][0])[0] if phase_ms else None
    roof = roofs.get(dom) or {"kernel": dom, "bound": None, "achieved": None, "peak": None,
                              "unit": None, "frac": None, "traffic": None}

    return dict(value=value, step_ms=step_ms, times=times, err=err, phase_ms=phase_ms, launches=launches,
                clocks=clk.summary(), e2e_s=e2e_s, h2d=h2d, d2h=d2h, plain=plain, roof=roof, roofs=roofs,
                prec_name=prec_name, n_cells=n_cells, n_pts=n_pts, info=info, learned=learned, mode=mode,
                e2e_mode=e2e_mode, lambda_cv=lcv, glue=glue, tune=tune, groups=groups,
                solve_dist=solve_distribution(work["records"]))


def glue_pairs_per_point(W, pts, band):
    """(point, subdomain) pairs of the glued evaluation per point: along each
    axis two cores carry weight within band cells of an interior core face,
    one elsewhere (host geometry, for the report)."""
    shape, n_sub = W["shape"], W["n_sub"]
    nmax = max(shape)
    pairs = np.ones(pts.shape[0])
    for a, (n, p) in enumerate(zip(shape, n_sub)):
        faces = np.array([(j * n) // p for j in range(1, p)], dtype=np.float64)
        if faces.size == 0:
            continue
        u = pts[:, a] * nmax
        k = np.searchsorted(faces, u)
        d = np.minimum(np.abs(u - faces[np.clip(k - 1, 0, faces.size - 1)]),
                       np.abs(u - faces[np.clip(k, 0, faces.size - 1)]))
        pairs *= np.where(d < band, 2.0, 1.0)
    return pairs


def owner_counts(W, pts):
    """Target points per owner subdomain (half-open cores, outer face closed)."""
    return np.bincount(owner_index(W, pts), minlength=int(np.prod(W["n_sub"]))).astype(float)


def owner_index(W, pts):
    """Owner subdomain of each point (half-open cores, outer face closed)."""
    shape, n_sub = W["shape"], W["n_sub"]
    nmax = max(shape)
    idx = []
    for a, (n, p) in enumerate(zip(shape, n_sub)):
        i = np.minimum(np.floor(pts[:, a] * nmax).astype(np.int64), n - 1)
        j = (i * p) // n
        lo_next = ((j + 1) * n) // p
        j = np.where((j + 1 < p) & (lo_next <= i), j + 1, j)
        idx.append(j)
    s = idx[0]
    stride = n_sub[0]
    for a in range(1, len(shape)):
        s = s + stride * idx[a]
        stride *= n_sub[a]
    return s


def _mixed_available(pam):
    try:
        pr = pam.make_problem((8, 8), (1, 1), 0, (2, 2))
        pam.pam_plan_create(pr, pam.make_params(precision=pam.PAM_PREC_MIXED))
        return True
    except pam.PamError:
        return False


def oracle_sample(workload: str, n_sub_sample: int, seed_offset=0):
    """Time the FP64 oracle on a bounded, evenly spaced sample of subdomains of
    the workload (fit + evaluation of the target points inside their cores)."""
    import oracle
    W = WORKLOADS[workload]
    K, x_el, vol_el = workload_data(W, W["seed"] + seed_offset)
    shape = W["shape"]
    S = int(np.prod(W["n_sub"]))
    which = np.unique(np.linspace(0, S - 1, min(n_sub_sample, S)).astype(np.int32))
    boxes = oracle.partition(shape, W["n_sub"], W["overlap"])
    h = fields.cell_size(shape)
    ratio = [c / n for c, n in zip(W["eval_counts"], shape)]
    pts = []
    for s in which:
        lo, hi = boxes[s, :3], boxes[s, 3:6]
        axes = []
        for a in range(len(shape)):
            ia = np.arange(int(lo[a] * ratio[a]), int(hi[a] * ratio[a]))
            axes.append((ia + 0.5) * h / ratio[a])
        g = np.meshgrid(*reversed(axes), indexing="ij")
        pts.append(np.stack([x.reshape(-1) for x in reversed(g)], axis=1))
    pts = np.concatenate(pts)
    if x_el is not None:
        cells = int(np.isin(owner_index(W, x_el), which).sum())  # elements owned by the sample
        t0 = time.perf_counter()
        model = oracle.fit_cells(x_el, vol_el, K, shape, W["n_sub"], W["overlap"], W["g"],
                                 oracle.default_params(**W["params"]), which=which)
    else:
        cells = int(np.prod(boxes[which, 3:6] - boxes[which, 0:3], axis=1).sum())
        t0 = time.perf_counter()
        model = oracle.fit_all(K, shape, W["n_sub"], W["overlap"], W["g"],
                               oracle.default_params(**W["params"]), which=which)
    oracle.evaluate(model, pts)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return dict(cells=cells, seconds=dt, cores=cores, n_sub=len(which), n_pts=len(pts))


def oracle_patches(n_patches, seed=40):
    """Time the FP64 oracle's plain fit (16 x 16 dictionary, no refinement)
    of `n_patches` evenly spaced patches of a batch of 4,096 seeded 32 x 32
    patches tiled 64 x 64: the labelling fit of the learned warm start."""
    import oracle
    held = fields.patch_batch(4096, seed=seed)
    T, P = 64, 32
    grid = np.ascontiguousarray(held.reshape(T, T, P, P).transpose(0, 2, 1, 3).reshape(T * P, T * P))
    which = np.unique(np.linspace(0, 4095, n_patches).astype(np.int32))
    t0 = time.perf_counter()
    oracle.fit_all(grid, (T * P, T * P), (T, T), 0, (16, 16), oracle.default_params(k_top=1, levels=0),
                   which=which)
    return dict(cells=len(which) * P * P, seconds=time.perf_counter() - t0, n_sub=len(which))


def oracle_table():
    """The FP64 oracle on the host cores, per workload: the 64^2 disc, the
    256^2 Voronoi field and the 60 x 220 x 85 layered field in full, the
    1024^2 channel field and the 32 x 32 patches on evenly spaced samples
    (their full time extrapolated linearly by subdomains); each on all
    cores and on one thread (the layered field's one-thread figure on a
    sample). Every time is fit + evaluation of the target points in the
    timed subdomains' cores (the patches: the plain fit alone)."""
    import oracle
    n_all = oracle.threads()
    rows = []
    plan = [("disc2d", 1, 1), ("voronoi2d", 64, 64), ("channel2d", 64, 16), ("layered3d", 2244, 64),
            ("patches32", 64, 16)]
    for name, n_many, n_one in plan:
        for nt, n in ((n_all, n_many), (1, n_one)):
            oracle.threads(nt)
            if name == "patches32":
                r = oracle_patches(n)
                total = 50176 + 4096
            else:
                r = oracle_sample(name, n)
                total = int(np.prod(WORKLOADS[name]["n_sub"]))
            full = r["n_sub"] == total
            rows.append({"workload": name, "threads": nt, "subdomains": r["n_sub"], "of": total,
                         "cells": r["cells"], "seconds": round(r["seconds"], 3),
                         "cells_per_s": round(r["cells"] / r["seconds"], 1),
                         "full_seconds": round(r["seconds"] * total / r["n_sub"], 1),
                         "full_seconds_kind": "measured" if full else "extrapolated by subdomains"})
            print(json.dumps(rows[-1]), flush=True)
    oracle.threads(n_all)
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pam", choices=["pam", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp64", "mixed"])
    ap.add_argument("--workload", default="layered3d", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-sample", type=int, default=None,
                    help="subdomains in the oracle baseline sample (default: 192, 32 on the triangle mesh)")
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--e2e-slices", type=int, default=E2E_EVAL_CHUNKS,
                    help="evaluation slices of the end-to-end leg, each copied back while the next evaluates")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="3-D mixed form without the learned warm start")
    ap.add_argument("--lambda-cv", action="store_true",
                    help="also time the per-subdomain 3-fold cross-validation of 3 lambda pairs (binary64)")
    ap.add_argument("--no-graph", action="store_true", help="time eager launches instead of a CUDA graph replay")
    ap.add_argument("--no-autotune", action="store_true", help="keep the built-in launch tuning")
    ap.add_argument("--shard", choices=["replicas", "field"], default="replicas",
                    help="replicas: every rank fits its own field (weak scaling, the default); field: one "
                         "field's subdomains split into contiguous blocks over the ranks (strong scaling)")
    ap.add_argument("--metrics-log", default=None,
                    help="write one JSON line per subdomain and level (cells, centres, support, "
                         "active-set steps, refinement passes, flags) of the step's fit to this file")
    ap.add_argument("--glue", type=float, default=0.0,
                    help="also time the glued evaluation (pam_eval_glued) with this band in cells")
    ap.add_argument("--quad", type=int, default=0, choices=[0, 1],
                    help="indicator and error quadrature: 0 midpoint, 1 two-point Gauss-Legendre per axis")
    ap.add_argument("--oracle-table", action="store_true",
                    help="only time the FP64 oracle on every workload (all host cores and one thread)")
    args = ap.parse_args()
    if args.oracle_table:
        rows = oracle_table()
        print(json.dumps({"oracle_table": rows, "host_cores": os.cpu_count()}))
        return
    rank, ws = _dist()
    W = WORKLOADS[args.workload]
    if args.cpu_sample is None:
        args.cpu_sample = W.get("cpu_sample", 192)
    cfg = {"workload": f"{args.workload} {'x'.join(map(str, W['shape']))} cells, "
                       f"{'x'.join(map(str, W['n_sub']))} subdomains, overlap {W['overlap']}, "
                       f"{'x'.join(map(str, W['g']))} initial centres, {W['params']['levels']} levels, "
                       f"eval {'x'.join(map(str, W['eval_counts']))}"
                       + (", triangle mesh (each square cut in two, 2 elements per cell)"
                          if W.get("mesh") == "triangles" else ""),
           "cells_per_step": int(np.prod(W["shape"])) * (2 if W.get("mesh") == "triangles" else 1),
           "eval_pts_per_step": int(np.prod(W["eval_counts"])),
           "l2_flush": "256 MB buffer written between timed steps", "parallelism": f"replicas{ws}"}

    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "pam" else "gloo"
        dist.init_process_group(backend=backend)

    if args.impl == "reference":
        if rank != 0:
            return
        per_step = max(8, args.cpu_sample // 8)
        vals = []
        for i in range(args.warmup + args.steps):
            r = oracle_sample(args.workload, per_step)
            if i >= args.warmup:
                vals.append(r)
        secs = sum(v["seconds"] for v in vals) / len(vals)
        cells = vals[0]["cells"]
        value = cells / secs
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": cfg,
                "cpu_baseline": {"value": value, "unit": "cells/s", "cores": vals[0]["cores"], "kind": "oracle",
                                 "sample": f"{vals[0]['n_sub']} evenly spaced subdomains per step "
                                           f"({cells} core cells, {vals[0]['n_pts']} eval points)"},
                "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if args.shard == "field":
        run_field_shard(args, rank, ws)
        return
    r = run_pam(args, rank, ws)
    if rank != 0:
        return
    cpu = None
    if not args.skip_cpu:
        o = oracle_sample(args.workload, args.cpu_sample)
        cpu = {"value": o["cells"] / o["seconds"], "unit": "cells/s", "cores": o["cores"], "kind": "oracle",
               "sample": f"{o['n_sub']} evenly spaced subdomains of the workload: Algorithm 1 fit + "
                         f"evaluation of their {o['n_pts']} target points ({o['cells']} core cells, "
                         f"{o['seconds']:.1f} s)"}
    step_s = r["step_ms"] / 1e3
    eval_ms = r["phase_ms"].get("eval", (None,))[0]
    line = {
        "metric": METRIC, "value": r["value"], "unit": "cells/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["step_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if r["prec_name"] == "fp64" else "bf16x3+f32+f64",
        "data": "synthetic",
        "config": dict(cfg, precision=r["prec_name"],
                       quadrature="midpoint" if args.quad == 0 else "Gauss-Legendre 2^dim points",
                       warm_start=r["learned"]["kind"] if r["learned"] else "previous level (Algorithm 1)",
                       launch=r["mode"]),
        "eval_pts_per_s": r["n_pts"] * ws / (eval_ms / 1e3) if eval_ms else None,
        "fit_cells_per_s": None,
        "l1_rel": r["err"]["l1"], "l2_rel": r["err"]["l2"],
        "roofline": r["roof"],
        "cpu_baseline": cpu,
        "e2e": {"value": r["n_cells"] * ws / r["e2e_s"], "unit": "cells/s",
                "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"], "launch": r["e2e_mode"],
                "eval_slices": args.e2e_slices},
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
        "phase_ms_per_step": {k: round(v[0], 4) for k, v in r["phase_ms"].items()},
        "roofline_all": r["roofs"],
        "plain_fp64": r["plain"],
        "learned_warm_start": r["learned"],
        "level_groups": r["groups"],
    }
    if r["lambda_cv"] is not None:
        line["lambda_cv"] = r["lambda_cv"]
    if r["glue"] is not None:
        line["glued_eval"] = r["glue"]
    if r["tune"] is not None:
        line["tuning"] = r["tune"]
    line["solves_per_level"] = r["solve_dist"]
    fit_ms = sum(v[0] for k, v in r["phase_ms"].items() if k not in ("eval", "errors", "eval_kernel"))
    line["fit_cells_per_s"] = r["n_cells"] * ws / (fit_ms / 1e3) if fit_ms else None
    print(json.dumps(line))


if __name__ == "__main__":
    main()
