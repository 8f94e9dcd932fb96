"""Parity of the batched solvers (aca_solve, sks_solve, aca_rect_solve) with
the FP64 oracle, through the C ABI, on the seeded synthetic workloads."""
import os

import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_2402_18008_gb300 import _lib, api
from tests.gpu_util import H_TOL, bound_gate, cuda, planes_to_rows, unit_aligned_err

pytestmark = pytest.mark.gpu


def _solve(pts_np, n, ld, norm=0, solver="aca", flags=False, sentinel=12345.0):
    pts = torch.zeros((16, ld), dtype=torch.float32, device="cuda")
    pts[:, :n] = cuda(pts_np[:, :n])
    H = torch.full((9, ld), sentinel, dtype=torch.float32, device="cuda")
    fl = torch.full((ld,), 0xEE, dtype=torch.uint8, device="cuda") if flags else None
    (_lib.aca_solve if solver == "aca" else _lib.sks_solve)(pts, H, fl, n=n, norm=norm)
    torch.cuda.synchronize()
    return H, fl


def test_aca_config0_parity_within_1e4():
    ms = workloads.minimal_sets(4096, seed=0)
    H, _ = _solve(ms.pts, 4096, 4096)
    err = unit_aligned_err(planes_to_rows(H, 4096), oracle.aca(ms.pts))
    print(f"aca config0: max {err.max():.3e} median {np.median(err):.3e}")
    assert err.max() < H_TOL


@pytest.mark.parametrize("n,ld", [(1, 1), (1, 4), (3, 4), (3, 3), (4, 4), (5, 8), (5, 5), (31, 32), (1023, 1024),
                                  (1023, 1023), (4097, 4100), (4097, 4097)])
def test_aca_ragged_sizes_and_untouched_tail(n, ld):
    ms = workloads.minimal_sets(n, seed=5)
    H, _ = _solve(ms.pts, n, ld)
    err = unit_aligned_err(planes_to_rows(H, n), oracle.aca(ms.pts))
    bound_gate(err, oracle.aca_fp32_bound(ms.pts), f"ragged n={n} ld={ld}")
    if ld > n:
        assert torch.all(H[:, n:] == 12345.0)


def test_full_size_workload_sampled_against_oracle():
    """The 2^26-set workload of the benchmark, in the benchmark's launch
    configuration: 2^16 sampled sets against the oracle, flags of all sets
    against the generator's near-degenerate labels."""
    n = 1 << 26
    ms = workloads.minimal_sets(n, seed=0, degenerate_frac=0.01, keep_truth=False, workers=os.cpu_count() or 1)
    pts = cuda(ms.pts)
    H = torch.empty((9, n), dtype=torch.float32, device="cuda")
    fl = torch.empty(n, dtype=torch.uint8, device="cuda")
    _lib.aca_solve(pts, H, None, n=n)
    H2 = torch.empty_like(H)
    _lib.aca_solve(pts, H2, fl, n=n)
    torch.cuda.synchronize()
    assert torch.equal(H, H2)                        # flags do not change H
    labels = torch.from_numpy(ms.near_degenerate).cuda()
    assert torch.equal((fl & 1) > 0, labels)
    assert not torch.any(fl & 8)
    idx = np.sort(np.random.default_rng(0).choice(n, 1 << 16, replace=False))
    sub = ms.pts[:, idx]
    err = unit_aligned_err(H[:, idx].cpu().numpy().T, oracle.aca(sub))
    f = fl.cpu().numpy()[idx]
    ok = (f & 7) == 0
    beta = oracle.aca_fp32_bound(sub)
    bound_gate(err[ok], beta[ok], "full size 2^26 (sample 2^16)")
    print(f"flagged in sample: {int((~ok).sum())}, their max err {err[~ok].max():.3e}")
    # SKS on the same sets (sks_solve row of the benchmark)
    _lib.sks_solve(pts, H, None, n=n)
    torch.cuda.synchronize()
    err_s = unit_aligned_err(H[:, idx].cpu().numpy().T, oracle.sks(sub))
    bound_gate(err_s[ok], oracle.sks_fp32_bound(sub)[ok], "sks full size 2^26 (sample 2^16)")


@pytest.mark.parametrize("solver", ["aca", "sks"])
@pytest.mark.parametrize("n", [1 << 18, (1 << 18) + 5, (1 << 20) + 7])
def test_vector_and_scalar_paths_agree_bitwise(solver, n):
    # large batches (>= 2^18 sets) with ld % 4 == 0 take the float4 paths
    # (ACA without flags: the prefetching ring, several quads per thread at
    # 2^20 + 7 sets; with flags and SKS: direct loads), small batches, odd ld
    # and misaligned bases the one-set-per-thread path
    ms = workloads.minimal_sets(n, seed=6)
    ldv = (n + 4) & ~3                   # a multiple of 4 above n: float4 path with padding
    lds = n | 1                          # odd: the one-set-per-thread path
    for norm in (0, 1, 2):
        Hv, _ = _solve(ms.pts, n, ldv, norm=norm, solver=solver)
        Hs1, _ = _solve(ms.pts, n, lds, norm=norm, solver=solver)
        assert torch.equal(Hv[:, :n], Hs1[:, :n]), norm
        assert torch.all(Hv[:, n:] == 12345.0)
    H4, f4 = _solve(ms.pts, n, ldv, solver=solver, flags=True)        # float4 path, ragged tail
    H1, f1 = _solve(ms.pts, n, lds, solver=solver, flags=True)        # ld odd -> scalar path
    assert torch.equal(H4[:, :n], H1[:, :n])
    assert torch.equal(f4[:n], f1[:n])
    assert torch.all(H4[:, n:] == 12345.0) and torch.all(f4[n:] == 0xEE)
    pts = torch.zeros((16, n + 4), dtype=torch.float32, device="cuda")
    pts[:, 1:1 + n] = cuda(ms.pts)
    H = torch.empty((9, n + 4), dtype=torch.float32, device="cuda")
    (_lib.aca_solve if solver == "aca" else _lib.sks_solve)(pts[:, 1:], H[:, 1:], None, n=n)
    torch.cuda.synchronize()
    assert torch.equal(H[:, 1:1 + n], H4[:, :n])
    small = 1000                                                       # small batch: scalar path
    Hs, _ = _solve(ms.pts, small, 1000, solver=solver)
    assert torch.equal(Hs[:, :small], H4[:, :small])


def test_norm_modes():
    n = 4096
    ms = workloads.minimal_sets(n, seed=0)
    ref = oracle.aca(ms.pts)
    H33, _ = _solve(ms.pts, n, n, norm=_lib.ACA_NORM_H33)
    h = planes_to_rows(H33, n)
    assert np.all(h[:, 8] == 1.0)
    assert unit_aligned_err(h, ref).max() < H_TOL
    Hf, _ = _solve(ms.pts, n, n, norm=_lib.ACA_NORM_FROB)
    f = planes_to_rows(Hf, n)
    assert np.allclose(np.linalg.norm(f, axis=1), 1.0, atol=1e-6)
    rf = oracle.normalize_frob(ref)
    assert np.abs(f - rf).max() < H_TOL       # sign convention identical, no alignment


def test_flags_match_near_degenerate_labels_and_nonfinite():
    n = 1 << 16
    ms = workloads.minimal_sets(n, seed=7, degenerate_frac=0.01)
    _, fl = _solve(ms.pts, n, n, flags=True)
    f = fl.cpu().numpy()
    assert np.array_equal((f & 1) > 0, ms.near_degenerate)
    assert not np.any(f[~ms.near_degenerate] & 0x6)
    assert not np.any(f & 8)
    bad = ms.pts[:, :8].copy()
    bad[3, 2] = np.nan
    bad[12, 5] = np.inf
    _, fl2 = _solve(bad, 8, 8, flags=True)
    f2 = fl2.cpu().numpy()
    assert f2[2] & 8 and f2[5] & 8 and not f2[0] & 8
    # one non-finite coordinate in each of the 16 planes, as NaN, +inf and -inf
    m = 16 * 3
    bad = np.ascontiguousarray(np.repeat(ms.pts[:, :1], m + 4, axis=1))
    for j, v in enumerate((np.nan, np.inf, -np.inf)):
        for plane in range(16):
            bad[plane, 16 * j + plane] = v
    for n_, ld_ in ((m + 4, m + 4), (m + 3, m + 3)):          # vector and scalar kernels
        _, fl3 = _solve(bad, n_, ld_, flags=True)
        f3 = fl3.cpu().numpy()
        assert np.all(f3[:m] & 8) and not np.any(f3[m:n_] & 8)


def test_flag_tail_bytes_untouched():
    ms = workloads.minimal_sets(5, seed=8)
    _, fl = _solve(ms.pts, 5, 8, flags=True)
    assert torch.all(fl[5:] == 0xEE)


def test_sks_config0_parity():
    ms = workloads.minimal_sets(4096, seed=0)
    H, _ = _solve(ms.pts, 4096, 4096, solver="sks")
    err = unit_aligned_err(planes_to_rows(H, 4096), oracle.sks(ms.pts))
    print(f"sks config0: max {err.max():.3e} median {np.median(err):.3e} >1e-4: {(err > 1e-4).sum()}")
    assert np.median(err) < 1e-6
    assert err.max() < H_TOL
    bound_gate(err, oracle.sks_fp32_bound(ms.pts), "sks config0")


@pytest.mark.parametrize("n,ld", [(3, 3), (5, 8), (1023, 1024), (1023, 1023)])
def test_sks_ragged_sizes_and_untouched_tail(n, ld):
    ms = workloads.minimal_sets(n, seed=5)
    H, _ = _solve(ms.pts, n, ld, solver="sks")
    err = unit_aligned_err(planes_to_rows(H, n), oracle.sks(ms.pts))
    bound_gate(err, oracle.sks_fp32_bound(ms.pts), f"sks ragged n={n} ld={ld}")
    if ld > n:
        assert torch.all(H[:, n:] == 12345.0)


@pytest.mark.parametrize("B", [65536, (1 << 18) + 3])
def test_rect_solve_matches_eq42_and_general_aca(B):
    rb = workloads.rect_batch(B, seed=0)
    tgt = cuda(rb.tgt)
    H = torch.empty((9, B), dtype=torch.float32, device="cuda")
    _lib.aca_rect_solve(tgt, rb.rect, H)
    torch.cuda.synchronize()
    h = planes_to_rows(H, B)
    ref = oracle.aca_rect(rb.tgt, rb.rect)
    err = unit_aligned_err(h, ref)
    print(f"rect: max {err.max():.3e}")
    assert err.max() < H_TOL
    # unnormalised: same sign and scale as Eq. 42 (relative to |H|)
    rel = np.abs(h - ref).max(axis=1) / np.abs(ref).max(axis=1)
    assert rel.max() < 1e-3
    pts = np.concatenate([np.repeat(rb.src_corners.reshape(8, 1), 64, axis=1), rb.tgt[:, :64]], axis=0)
    assert unit_aligned_err(h[:64], oracle.aca(pts)).max() < H_TOL


def test_api_solve_and_layout_helpers():
    ms = workloads.minimal_sets(64, seed=9)
    s = oracle.sets_aos(ms.pts)
    src = torch.tensor(s[:, :8].reshape(64, 4, 2), dtype=torch.float32, device="cuda")
    tgt = torch.tensor(s[:, 8:].reshape(64, 4, 2), dtype=torch.float32, device="cuda")
    pts = api.to_planes(src, tgt, ld=64)
    H, fl = api.solve(pts, norm=_lib.ACA_NORM_FROB, with_flags=True)
    M = api.planes_to_mats(H, 64).cpu().numpy().reshape(64, 9)
    assert np.abs(M - oracle.normalize_frob(oracle.aca(ms.pts))).max() < H_TOL
    p12 = torch.from_numpy(np.ascontiguousarray(np.concatenate([ms.pts[0:6], ms.pts[8:14]], axis=0))).cuda()
    Ha = api.affine_solve(p12, norm=_lib.ACA_NORM_FROB)
    ref = oracle.normalize_frob(oracle.aca_affine(p12.cpu().numpy()))
    assert np.abs(planes_to_rows(Ha, 64) - ref).max() < H_TOL


def _affine_planes(ms):
    return np.ascontiguousarray(np.concatenate([ms.pts[0:6], ms.pts[8:14]], axis=0))


@pytest.mark.parametrize("n,ld", [(1, 1), (5, 8), (4096, 4096), (1023, 1023), ((1 << 18) + 3, (1 << 18) + 4)])
def test_affine_three_point_solver_parity(n, ld):
    ms = workloads.minimal_sets(n, seed=10)
    p12 = _affine_planes(ms)
    pts = torch.zeros((12, ld), dtype=torch.float32, device="cuda")
    pts[:, :n] = cuda(p12)
    H = torch.full((9, ld), 12345.0, dtype=torch.float32, device="cuda")
    _lib.aca_affine_solve(pts, H, n=n)
    torch.cuda.synchronize()
    h = planes_to_rows(H, n)
    err = unit_aligned_err(h, oracle.aca_affine(p12))
    print(f"affine n={n}: max {err.max():.3e}")
    assert err.max() < H_TOL
    assert np.all(h[:, 6] == 0) and np.all(h[:, 7] == 0)
    if ld > n:
        assert torch.all(H[:, n:] == 12345.0)
    H33 = torch.empty((9, ld), dtype=torch.float32, device="cuda")
    _lib.aca_affine_solve(pts, H33, n=n, norm=_lib.ACA_NORM_H33)
    torch.cuda.synchronize()
    a = planes_to_rows(H33, n)
    assert np.all(a[:, 8] == 1.0) and np.all(a[:, 6:8] == 0)
    # the affine map sends M1, N1, P1 to M2, N2, P2 (to FP32 accuracy)
    s = p12.astype(np.float64)
    for k in range(3):
        X = a[:, 0] * s[2 * k] + a[:, 1] * s[2 * k + 1] + a[:, 2]
        Y = a[:, 3] * s[2 * k] + a[:, 4] * s[2 * k + 1] + a[:, 5]
        assert np.max(np.hypot(X - s[6 + 2 * k], Y - s[7 + 2 * k])) < 1e-2


@pytest.mark.parametrize("n", [1 << 18, (1 << 20) + 7])
def test_affine_ring_and_scalar_paths_agree_bitwise(n):
    # the prefetching ring (ld % 4 == 0; at 2^20 + 7 several quads per thread
    # and a ragged last quad; 2^18 is the smallest batch it takes) against
    # the one-set-per-thread path (odd ld)
    p12 = _affine_planes(workloads.minimal_sets(n, seed=11))
    out = []
    for ld in ((n + 4) & ~3, n | 1):
        pts = torch.zeros((12, ld), dtype=torch.float32, device="cuda")
        pts[:, :n] = cuda(p12)
        for norm in (0, 1, 2):
            H = torch.full((9, ld), 12345.0, dtype=torch.float32, device="cuda")
            _lib.aca_affine_solve(pts, H, n=n, norm=norm)
            out.append(H)
    torch.cuda.synchronize()
    for k in range(3):
        assert torch.equal(out[k][:, :n], out[3 + k][:, :n]), k
        assert torch.all(out[k][:, n:] == 12345.0)


@pytest.mark.parametrize("n", [1000, (1 << 18) + 5])
def test_solve_on_pinned_host_buffers_matches_device_buffers(n):
    # zero-copy: the kernel reads the sets from and writes H and the flags to
    # page-locked host memory; results are bit-identical to HBM buffers
    ms = workloads.minimal_sets(n, seed=12)
    pts_d = cuda(ms.pts)
    H_d = torch.empty((9, n), device="cuda")
    f_d = torch.empty(n, dtype=torch.uint8, device="cuda")
    _lib.aca_solve(pts_d, H_d, f_d)
    pts_h = torch.from_numpy(ms.pts).pin_memory()
    H_h = torch.full((9, n), 7.0).pin_memory()
    f_h = torch.zeros(n, dtype=torch.uint8).pin_memory()
    _lib.aca_solve(pts_h, H_h, f_h)
    torch.cuda.synchronize()
    assert torch.equal(H_h, H_d.cpu()) and torch.equal(f_h, f_d.cpu())
    H_h2 = torch.full((9, n), 7.0).pin_memory()               # no flags: the prefetching ring at large n
    _lib.aca_solve(pts_h, H_h2)
    torch.cuda.synchronize()
    assert torch.equal(H_h2, H_d.cpu())
    with pytest.raises(ValueError):
        _lib.aca_solve(torch.from_numpy(ms.pts), H_h)        # pageable host memory is refused


@pytest.mark.parametrize("solver", ["aca", "sks"])
def test_all_24_correspondence_orders_of_a_rectangle_source(solver):
    # a rectangle source in every one of the 24 orders of its corners (the
    # orders for which a pivot-free elimination divides by zero included):
    # the same homography each time, within the FP32 bound gate
    import itertools
    rb = workloads.rect_batch(64, seed=21)
    x0, y0, w, r = rb.rect
    src = np.array([[x0, y0], [x0 + w, y0], [x0, y0 + w / r], [x0 + w, y0 + w / r]])   # M N P Q
    tgt = rb.tgt.T.reshape(64, 4, 2).astype(np.float64)
    sets = []
    for perm in itertools.permutations(range(4)):
        s = np.concatenate([src[list(perm)].reshape(1, 8).repeat(64, 0), tgt[:, list(perm)].reshape(64, 8)], axis=1)
        sets.append(s)
    S = np.concatenate(sets).astype(np.float32).T.copy()                # (16, 24 * 64)
    H = torch.empty((9, S.shape[1]), device="cuda")
    (_lib.aca_solve if solver == "aca" else _lib.sks_solve)(cuda(S), H)
    torch.cuda.synchronize()
    g = planes_to_rows(H, S.shape[1])
    ref = oracle.aca(S)
    beta = (oracle.aca_fp32_bound if solver == "aca" else oracle.sks_fp32_bound)(S)
    bound_gate(unit_aligned_err(g, ref), beta, f"{solver} 24 orders")
    # every order against the first order's H (the same map up to scale)
    per = unit_aligned_err(g.reshape(24, 64, 9).reshape(-1, 9), np.tile(ref[:64], (24, 1)))
    bound_gate(per, beta, f"{solver} 24 orders against order 0")


def test_solve_beyond_32_bit_offsets():
    # n = 2^30 + 3 sets, ld = 2^30 + 4: plane offsets reach 2^34 floats (64 GiB
    # in, 36 GiB out on the device).  The sets are 1024 copies of 2^20
    # generated ones plus 3 more: every copy must give bit-identical H, a
    # sample must pass the oracle gate, and the padding column stays untouched.
    m, reps = 1 << 20, 1 << 10
    n, ld = m * reps + 3, m * reps + 4
    ms = workloads.minimal_sets(m, seed=23)
    base = cuda(ms.pts)
    pts = torch.empty((16, ld), device="cuda")
    for r in range(reps):
        pts[:, r * m:(r + 1) * m].copy_(base)
    pts[:, m * reps:n].copy_(base[:, :3])
    H = torch.full((9, ld), 7.0, device="cuda")
    _lib.aca_solve(pts, H, n=n)
    torch.cuda.synchronize()
    first = H[:, :m]
    for r in (1, 511, reps - 1):
        assert torch.equal(H[:, r * m:(r + 1) * m], first), r
    assert torch.equal(H[:, m * reps:n], first[:, :3])
    assert torch.all(H[:, n:] == 7.0)
    idx = np.random.default_rng(4).choice(m, 4096, replace=False)
    g = first[:, torch.from_numpy(idx).cuda()].cpu().numpy().T.astype(np.float64)
    sub = ms.pts[:, idx]
    bound_gate(unit_aligned_err(g, oracle.aca(sub)), oracle.aca_fp32_bound(sub), "2^30 + 3 sets")
    del pts, H
    torch.cuda.empty_cache()


def test_prepared_calls_match_plain_calls():
    # one call bound to fixed buffers, checked once: the same bits as the
    # plain binding, on the current stream and on an explicit one
    ms = workloads.minimal_sets(5000, seed=31)
    pts = cuda(ms.pts)
    H1 = torch.empty((9, 5000), device="cuda")
    H2 = torch.full((9, 5000), 7.0, device="cuda")
    _lib.aca_solve(pts, H1)
    prep = _lib.prepare_aca_solve(pts, H2)
    prep()
    torch.cuda.synchronize()
    assert torch.equal(H1, H2)
    s = torch.cuda.Stream()
    H2.fill_(7.0)
    torch.cuda.synchronize()
    prep(stream=s)
    s.synchronize()
    assert torch.equal(H1, H2)
    rb = workloads.rect_batch(4096, seed=3)
    tgt = cuda(rb.tgt)
    gH = torch.randn((9, 4096), device="cuda")
    Ha, Hb = torch.empty((9, 4096), device="cuda"), torch.empty((9, 4096), device="cuda")
    ga, gb = torch.empty((8, 4096), device="cuda"), torch.empty((8, 4096), device="cuda")
    _lib.aca_rect_solve(tgt, rb.rect, Ha)
    _lib.aca_rect_backward(tgt, rb.rect, gH, ga)
    _lib.prepare_aca_rect_solve(tgt, rb.rect, Hb)()
    _lib.prepare_aca_rect_backward(tgt, rb.rect, gH, gb)()
    torch.cuda.synchronize()
    assert torch.equal(Ha, Hb) and torch.equal(ga, gb)
