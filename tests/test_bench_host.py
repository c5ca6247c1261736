"""Host-side helpers of bench.py on CPU: the owner lookup and the glued
evaluation's pair count it reports, checked by brute force against the
partition, and the roofline objects' contract (every key, frac = achieved /
peak, recorded DRAM traffic only where it was captured)."""
import numpy as np
import pytest

import bench
import oracle


def _brute_owner(shape, n_sub, pts):
    boxes = oracle.partition(shape, n_sub, 0)
    nmax = max(shape)
    dim = len(shape)
    cell = np.stack([np.minimum(np.floor(pts[:, a] * nmax).astype(np.int64), shape[a] - 1) for a in range(dim)], 1)
    own = np.full(len(pts), -1)
    for s in range(boxes.shape[0]):
        inside = np.all((cell >= boxes[s, 0:dim]) & (cell < boxes[s, 3:3 + dim]), axis=1)
        assert np.all(own[inside] == -1)
        own[inside] = s
    return own


@pytest.mark.parametrize("name", ["layered3d", "voronoi2d", "triangles2d", "disc2d"])
def test_owner_index_is_the_core_box_containing_the_point(name):
    W = bench.WORKLOADS[name]
    shape = W["shape"]
    ext = np.asarray(shape, dtype=float) / max(shape)
    rng = np.random.default_rng(7)
    pts = rng.uniform(0, 1, size=(20000, len(shape))) * ext
    # points on core faces and on the outer faces
    faces = []
    for a, (n, p) in enumerate(zip(shape, W["n_sub"])):
        for j in range(p + 1):
            q = rng.uniform(0, 1, size=(20, len(shape))) * ext
            q[:, a] = ((j * n) // p) / max(shape)
            faces.append(q)
    pts = np.concatenate([pts] + faces)
    pts = np.minimum(pts, ext)
    np.testing.assert_array_equal(bench.owner_index(W, pts), _brute_owner(shape, W["n_sub"], pts))


def test_glue_pairs_per_point_counts_the_faces_within_the_band():
    W = bench.WORKLOADS["voronoi2d"]  # 256 x 256 cells, 8 x 8 cores of 32
    rng = np.random.default_rng(8)
    pts = rng.uniform(0, 1, size=(5000, 2))
    band = 2.5
    got = bench.glue_pairs_per_point(W, pts, band)
    u = pts * 256
    faces = np.arange(32, 256, 32, dtype=float)
    near = np.abs(u[:, :, None] - faces[None, None, :]).min(axis=2) < band
    np.testing.assert_array_equal(got, np.prod(np.where(near, 2.0, 1.0), axis=1))
    assert set(np.unique(got)) <= {1.0, 2.0, 4.0}


def test_roofline_objects_keep_their_contract():
    work = dict(gram_flops=2e12, pairs=3e11, chol_flops=1e9, solve_bytes=4e9, solves=8976, steps=4.7e4,
                passes=7.4e3, support_last=84.0, eval_pairs=3.5e12)
    phases = {"gram_tc": (4.4, 4), "stats": (0.62, 4), "eval": (1.53, 1), "solve": (9.6, 4)}
    peaks = {"hbm_gbs": 6783.5, "bf16_tflops": 1895.2}
    r = bench.roofline_entries(phases, work, 8_976_000, True, peaks, "measured")
    assert set(r) == {"gram_tc", "stats", "eval", "solve"}
    for v in r.values():
        for k in ("kernel", "bound", "achieved", "peak", "unit", "frac", "traffic", "peak_source"):
            assert k in v, k
        assert v["frac"] == pytest.approx(v["achieved"] / v["peak"])
        assert v["traffic"] is None
    assert r["solve"]["bound"] == "hbm" and r["solve"]["unit"] == "GB/s"
    assert r["solve"]["achieved"] == pytest.approx(4e9 / 9.6e-3 / 1e9)
    assert r["solve"]["active_set_steps_per_solve"] == pytest.approx(4.7e4 / 8976)
    assert r["gram_tc"]["bound"] == "tensor" and r["stats"]["bound"] == "alu"
    # recorded traffic: the layered 3-D workload only, and only for kernels captured as they are
    t = bench.attach_traffic({k: dict(v) for k, v in r.items()}, "layered3d")
    for name, v in t.items():
        assert v["traffic"] == bench.TRAFFIC_LAYERED3D.get(v["kernel"])
    assert t["stats"]["traffic"] is None
    assert all(v["traffic"] is None for v in bench.attach_traffic({k: dict(v) for k, v in r.items()},
                                                                   "channel2d").values())
    # with the evaluation kernel timed alone, its roofline uses that time
    # and keeps the whole phase's fraction beside it
    assert r["eval"]["timed"] == "the evaluation phase"
    phases["eval_kernel"] = (1.12, 1)
    r2 = bench.roofline_entries(phases, work, 8_976_000, True, peaks, "measured")
    assert r2["eval"]["timed"] == "the kernel alone"
    assert r2["eval"]["achieved"] == pytest.approx(3.5e12 / 1.12e-3 / 1e12)
    assert r2["eval"]["phase_frac"] == pytest.approx(3.5e12 / 1.53e-3 / bench.SFU_EX2_PER_S)
    assert "eval_kernel" not in r2


def test_dictionary_agreement_counts_differing_subdomains_and_flags():
    from paper_2605_16564_gb300 import pam
    S, mc = 4, 6
    c = np.random.default_rng(3).uniform(size=(S, mc, 4))
    plain = dict(M=np.array([4, 5, 6, 4]), c=c.copy(), info=np.zeros((S, 8), dtype=np.int32))
    mixed = dict(M=np.array([4, 5, 5, 4]), c=c.copy(), info=np.zeros((S, 8), dtype=np.int32))
    mixed["c"][3, 2, 0] += 1e-12          # one centre moved: differs
    mixed["c"][0, 5, 0] += 1.0            # past M: does not count
    mixed["info"][1, pam.INFO_FLAGS] = pam.FLAG_REFINE_DIVERGED
    mixed["info"][2, pam.INFO_FLAGS] = pam.FLAG_NOT_CERTIFIED
    a = bench.dictionary_agreement(pam, mixed, plain)
    assert a["dictionaries_differing"] == 2 and a["fraction_differing"] == 0.5
    assert a["mixed_solves_fallen_back_to_fp64"] == 1 and a["mixed_solves_uncertified"] == 1


def test_solve_distribution_summarises_each_level():
    recs = [{"level": lv, "subdomain": s, "cells": 100, "centres": 32 + lv, "support": s % 7,
             "active_set_steps": s % 5, "refinement_passes": s % 2, "flags": int(s == 3 and lv == 1)}
            for lv in (0, 1) for s in range(10)]
    d = bench.solve_distribution(recs)
    assert set(d) == {"level0", "level1"}
    assert d["level0"]["solves"] == 10 and d["level1"]["flagged"] == 1 and d["level0"]["flagged"] == 0
    assert d["level1"]["centres"] == {"p50": 33.0, "p90": 33.0, "max": 33.0}
    assert d["level0"]["support"]["max"] == 6.0 and d["level0"]["active_set_steps"]["p50"] == 2.0
