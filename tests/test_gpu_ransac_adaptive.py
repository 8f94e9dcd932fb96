"""RANSAC with the online adaptive stop (ransac_aca_adaptive; Sec. 6.2: the
loop count follows from the best inlier ratio so far at 99% confidence)
against the FP64 oracle's sequential loop.

Counts before the stop follow the count gate of the fixed-count tests (exact
except for points inside the oracle's ambiguity band).  Since the stop index
depends on the counts, it must lie between the oracle's stop index with every
count moved to the top of its band and to the bottom (the stop index never
increases with the counts); with no ambiguous point before the stop, it is
exact.  Every output is deterministic, whatever work the GPU skipped."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_2402_18008_gb300 import _lib, api
from paper_2402_18008_gb300._lib import AcaError
from tests.gpu_util import cuda
from tests.test_gpu_ransac import BAND_PX, _count_gate

pytestmark = pytest.mark.gpu
CONF = 0.99


def _run(corr, offsets, caps, thr, seed, **kw):
    caps = np.asarray(caps, np.int32)
    r = api.ransac(cuda(corr), cuda(np.asarray(offsets, np.int64)), cuda(caps), thr, seed,
                   total_hyps=int(caps.sum()), want_counts=True, want_mask=True, confidence=CONF, **kw)
    torch.cuda.synchronize()
    return {k: (None if v is None else v.cpu().numpy()) for k, v in r.__dict__.items()}


def _check_problem(g, o, hoff, k, N, p, label):
    ne = int(g["n_evaluated"][p])
    gc = g["hyp_counts"][hoff:hoff + k]
    oc = o["hyp_counts"][hoff:hoff + k]
    bi = o["band_in"][hoff:hoff + k]
    bo = o["band_out"][hoff:hoff + k]
    lo = oracle.adaptive_stop(np.where(oc < 0, oc, oc + bo), N, CONF)
    hi = oracle.adaptive_stop(np.where(oc < 0, oc, np.maximum(oc - bi, 0)), N, CONF)
    assert lo <= ne <= hi, (label, p, lo, ne, hi, int(o["n_eval"][p]))
    assert np.all(gc[ne:] == -2)
    m = min(ne, int(o["n_eval"][p]))
    _count_gate(gc[:m], oc[:m], bi[:m], bo[:m], f"{label} p={p}")
    if not (bi + bo)[:max(ne, int(o["n_eval"][p]))].any():
        assert ne == o["n_eval"][p] and g["best_hyp"][p] == o["best_hyp"][p]
    # the best is the argmax of the evaluated counts, ties to the lowest index
    ev = gc[:ne]
    if ev.max() >= 0:
        assert g["best_count"][p] == ev.max() and g["best_hyp"][p] == int(np.argmax(ev == ev.max()))
    else:
        assert g["best_hyp"][p] == -1 and g["best_count"][p] == 0
    return ne


def test_adaptive_one_pair_matches_the_sequential_loop():
    rp = workloads.ransac_problem(2000, 0.6, 1.0, seed=0)
    thr, seed, cap = 3.0, 2024, 4096
    g = _run(rp.corr, [0, 2000], [cap], thr, seed)
    o = oracle.ransac_adaptive(rp.corr, [0, 2000], [cap], thr, seed, CONF, band_px=BAND_PX)
    ne = _check_problem(g, o, 0, cap, 2000, 0, "one pair")
    print(f"one pair: stopped after {ne} of {cap} hypotheses (oracle {int(o['n_eval'][0])})")
    assert ne < cap


def test_adaptive_batched_uneven_matches_the_oracle():
    rb = workloads.ransac_batch(P=24, seed=6, n_max=3000)
    caps = np.full(24, 2048, np.int32)
    g = _run(rb.corr, rb.offsets, caps, 3.0, 99)
    o = oracle.ransac_adaptive(rb.corr, rb.offsets, caps, 3.0, 99, CONF, band_px=BAND_PX)
    nes = []
    for p in range(24):
        N = int(rb.offsets[p + 1] - rb.offsets[p])
        nes.append(_check_problem(g, o, 2048 * p, 2048, N, p, "batched 24"))
    print("batched 24: evaluated", nes)


def test_adaptive_equals_fixed_ransac_over_the_evaluated_prefix():
    rb = workloads.ransac_batch(P=16, seed=7, n_max=2000)
    caps = np.full(16, 1024, np.int32)
    g = _run(rb.corr, rb.offsets, caps, 3.0, 5)
    ne = g["n_evaluated"].astype(np.int32)
    f = api.ransac(cuda(rb.corr), cuda(rb.offsets), cuda(ne), 3.0, 5, total_hyps=int(ne.sum()),
                   want_counts=True, want_mask=True)
    torch.cuda.synchronize()
    assert np.array_equal(f.best_hyp.cpu().numpy(), g["best_hyp"])
    assert np.array_equal(f.best_count.cpu().numpy(), g["best_count"])
    assert np.array_equal(f.best_H.cpu().numpy(), g["best_H"])
    assert np.array_equal(f.inlier_mask.cpu().numpy(), g["inlier_mask"])
    fc = f.hyp_counts.cpu().numpy()
    off = np.concatenate([[0], np.cumsum(ne)])
    for p in range(16):
        assert np.array_equal(fc[off[p]:off[p + 1]], g["hyp_counts"][1024 * p:1024 * p + ne[p]])


@pytest.mark.parametrize("tuning", [dict(block_warps=4, hyps_per_thread=4, tile_points=2048),
                                    dict(block_warps=8, hyps_per_thread=1, tile_points=256),
                                    dict(block_warps=2, hyps_per_thread=2, tile_points=64, grid_blocks=7),
                                    # one block takes every item of both epochs (chunk 0 of all
                                    # problems, then the re-planned live chunks)
                                    dict(block_warps=4, hyps_per_thread=1, tile_points=512, grid_blocks=1)])
def test_adaptive_outputs_do_not_depend_on_tuning_or_skipped_work(tuning):
    rb = workloads.ransac_batch(P=40, seed=9, n_max=4000)
    caps = np.full(40, 4096, np.int32)
    ref = _run(rb.corr, rb.offsets, caps, 3.0, 11)
    for _ in range(2):
        g = _run(rb.corr, rb.offsets, caps, 3.0, 11, **tuning)
        for key in ("best_hyp", "best_count", "best_H", "hyp_counts", "inlier_mask", "n_evaluated"):
            assert np.array_equal(g[key], ref[key]), key


def test_adaptive_edge_cases_and_graph_replay():
    rp = workloads.ransac_problem(300, 0.0, 1.0, seed=42)       # pure outliers: the cap is reached
    rq = workloads.ransac_problem(500, 0.9, 0.5, seed=43)       # clean: stops after a few
    corr = np.concatenate([rq.corr[:3], rp.corr, rq.corr]).astype(np.float32)
    offsets = np.array([0, 3, 303, 303, 803], np.int64)         # N = 3, 300, 0, 500
    caps = np.array([64, 300, 10, 2000], np.int32)
    g = _run(corr, offsets, caps, 3.0, 3)
    o = oracle.ransac_adaptive(corr, offsets, caps, 3.0, 3, CONF, band_px=BAND_PX)
    assert list(g["n_evaluated"][:3]) == [0, 300, 0]
    assert g["best_hyp"][0] == -1 and g["best_hyp"][2] == -1
    assert np.all(g["hyp_counts"][:64] == -1) and np.all(g["hyp_counts"][364:374] == -1)
    assert 1 <= g["n_evaluated"][3] < 50
    assert g["n_evaluated"][1] == o["n_eval"][1]
    # graph capture and replay give the eager outputs
    plan = api.RansacPlan(cuda(corr), cuda(offsets), cuda(caps), 3.0, 3, int(caps.sum()), want_counts=True,
                          want_mask=True, confidence=CONF)
    e = plan.run()
    eager = {k: getattr(e, k).clone() for k in ("best_H", "best_hyp", "hyp_counts", "n_evaluated", "inlier_mask")}
    plan.capture()
    for _ in range(3):
        rep = plan.replay()
    torch.cuda.synchronize()
    for k, v in eager.items():
        assert torch.equal(v, getattr(rep, k)), k
    # arguments
    c, off, k = cuda(corr), cuda(offsets), cuda(caps)
    P = 4
    out = [torch.empty((P, 9), device="cuda"), torch.empty(P, dtype=torch.int32, device="cuda"),
           torch.empty(P, dtype=torch.int32, device="cuda")]
    ws = torch.empty(_lib.ransac_aca_adaptive_workspace_size(P, int(caps.sum())), dtype=torch.uint8, device="cuda")
    prm = _lib.RansacParams(threshold_px=3.0, seed=3)
    for conf in (0.0, 1.0, -0.5):
        with pytest.raises(AcaError):
            _lib.ransac_aca_adaptive(c, off, k, int(caps.sum()), prm, conf, *out, ws)
    with pytest.raises(AcaError):
        _lib.ransac_aca_adaptive(c, off, k, int(caps.sum()), prm, CONF, *out, ws[:1024])
    torch.cuda.synchronize()


def test_adaptive_full_size_512_pairs_sampled_against_the_oracle():
    # the batched workload at full size with the realistic cap (16384 for every
    # pair, no knowledge of the inlier ratio); 8 pairs checked one by one
    rb = workloads.ransac_batch(P=512, seed=0)
    caps = np.full(512, 16384, np.int32)
    g = _run(rb.corr, rb.offsets, caps, 3.0, 0, block_warps=4, hyps_per_thread=4, tile_points=2048)
    ne = g["n_evaluated"]
    print(f"512 pairs: evaluated {int(ne.sum())} of {int(caps.sum())} hypotheses, "
          f"median {int(np.median(ne))}, max {int(ne.max())}")
    assert np.all(ne >= 1) and ne.sum() < caps.sum()
    for p in np.random.default_rng(3).choice(512, 8, replace=False):
        a, b = int(rb.offsets[p]), int(rb.offsets[p + 1])
        o = oracle.ransac_adaptive(rb.corr[a:b], [0, b - a], [16384], 3.0, 0, CONF, problem_base=int(p),
                                   band_px=BAND_PX)
        gp = dict(g)
        gp["n_evaluated"] = g["n_evaluated"][p:p + 1]
        gp["best_hyp"] = g["best_hyp"][p:p + 1]
        gp["best_count"] = g["best_count"][p:p + 1]
        gp["hyp_counts"] = g["hyp_counts"][16384 * p:16384 * (p + 1)]
        _check_problem(gp, o, 0, 16384, b - a, 0, f"512 pairs, pair {p}")
