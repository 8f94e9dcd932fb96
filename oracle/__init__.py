"""FP64 CPU oracle: TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` / ``--impl reference`` legs may import this package.  The
library (``paper_2402_18008_gb300``) never does, and this package never
imports the library: the two share no code.  Only ``workloads`` (seeded input
generators, none of the method's arithmetic) serves both.

``oracle.c`` holds the FP64 implementations (ACA Eq. 20-29, the independent
8x8 DLT of Eq. 2, SKS Eq. 4-14, the rectangle form Eq. 42 / Algorithm 1,
Philox sampling, brute-force RANSAC scoring, the online adaptive stop of
Sec. 6.2 and the analytic Jacobian);
``exact.py`` holds exact-rational versions used by the pins;
``inlier_refit.py`` the float64 refit on all inliers (normalised DLT, then
Levenberg-Marquardt: the global optimisation of Sec. 6.2, stage 5);
``fp32_bounds.c`` the tolerance model of the parity tests: first-order
rounding-error bounds of the library's stated FP32 evaluation orders (ACA,
SKS, the RANSAC inlier test), from which the solver gate and the per-point
ambiguity band of the RANSAC counts follow.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(exact agreement with an independent DLT, invariants, special cases, cuRAND's
Philox, brute-force enumeration; the bounds against exact rational arithmetic,
an FP32 host evaluation and their worst rounding corners).  None is "parity
unpinned", and tests/test_oracle_mutations.py checks that planted mistakes
fail the pins.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_SRC_BOUNDS = os.path.join(_HERE, "fp32_bounds.c")
_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_f = ctypes.POINTER(ctypes.c_float)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)
_u32 = ctypes.POINTER(ctypes.c_uint32)
_u8 = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (plain C, FP64, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_BOUNDS))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-fno-fast-math", _SRC, _SRC_BOUNDS, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.oracle_num_threads.restype = ctypes.c_int
            L.oracle_set_num_threads.argtypes = [ctypes.c_int]
            L.oracle_set_num_threads.restype = None
            for name in ("oracle_aca", "oracle_aca_divform", "oracle_sks", "oracle_aca_jacobian",
                         "oracle_aca_jacobian_src", "oracle_aca_condition"):
                getattr(L, name).argtypes = [_d, _d, ctypes.c_int64]
                getattr(L, name).restype = None
            L.oracle_aca_affine.argtypes = [_d, _d, ctypes.c_int64]
            L.oracle_aca_affine.restype = None
            L.oracle_dlt.argtypes = [_d, _d, ctypes.c_int64]
            L.oracle_dlt.restype = ctypes.c_int64
            for name in ("oracle_aca_rect", "oracle_aca_rect_alg1", "oracle_aca_rect_jacobian"):
                getattr(L, name).argtypes = [_d, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, _d, ctypes.c_int64]
                getattr(L, name).restype = None
            L.oracle_philox4x32_10.argtypes = [_u32, _u32, _u32]
            L.oracle_sample4.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64, _i64]
            L.oracle_sample_degenerate.argtypes = [_d]
            L.oracle_sample_degenerate.restype = ctypes.c_int
            L.oracle_normalize_frob.argtypes = [_d]
            L.oracle_score_problem.argtypes = [_f, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                               ctypes.c_uint64, ctypes.c_uint32, _i32, _i32, _i32, ctypes.c_double]
            L.oracle_ransac.argtypes = [_f, _i64, _i32, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64,
                                        ctypes.c_uint32, _d, _i32, _i32, _i32, _i32, _i32, ctypes.c_double, _u8]
            L.oracle_adaptive_k.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_double]
            L.oracle_adaptive_k.restype = ctypes.c_int32
            L.oracle_adaptive_stop.argtypes = [_i32, ctypes.c_int32, ctypes.c_int64, ctypes.c_double]
            L.oracle_adaptive_stop.restype = ctypes.c_int32
            L.oracle_ransac_adaptive.argtypes = [_f, _i64, _i32, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64,
                                                 ctypes.c_uint32, ctypes.c_double, _d, _i32, _i32, _i32, _i32,
                                                 _i32, _i32, ctypes.c_double, _u8]
            for name in ("oracle_aca_fp32_bound", "oracle_sks_fp32_bound"):
                getattr(L, name).argtypes = [_d, _d, _d, _d, ctypes.c_int64]
                getattr(L, name).restype = None
            L.oracle_score_band.argtypes = [_d, _f, ctypes.c_int64, ctypes.c_double, ctypes.c_double, _u8]
            L.oracle_score_band.restype = ctypes.c_int64
            L.oracle_score_band_px.argtypes = [_d, _f, ctypes.c_int64, ctypes.c_double, _d]
            L.oracle_score_band_px.restype = None
            L.oracle_fp32_rule_bound.argtypes = [ctypes.c_int, _d, _d]
            L.oracle_fp32_rule_bound.restype = ctypes.c_double
            L.oracle_score_bound_E.argtypes = [_d, _f, ctypes.c_int64, ctypes.c_double, _d, _d]
            L.oracle_score_bound_E.restype = None
            L.oracle_fp32_chain_corner.argtypes = [ctypes.c_int, _d, _d, _d, _d]
            L.oracle_fp32_chain_corner.restype = ctypes.c_double
            L.oracle_score_bound_E_fixed.argtypes = [_d, _f, ctypes.c_int64, ctypes.c_double, _d, _d]
            L.oracle_score_bound_E_fixed.restype = None
            L.oracle_score_corner.argtypes = [_d, _f, ctypes.c_double, _d, _d, _d]
            L.oracle_score_corner.restype = None
            _lib = L
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on."""
    lib().oracle_set_num_threads(int(n))


def sets_aos(pts16: np.ndarray, n: int | None = None) -> np.ndarray:
    """SoA (16, ld) float -> AoS (n, 16) float64 (values unchanged)."""
    n = pts16.shape[1] if n is None else n
    return np.ascontiguousarray(np.asarray(pts16[:, :n], dtype=np.float64).T)


def _solve(name: str, pts16: np.ndarray, n: int | None = None) -> np.ndarray:
    a = sets_aos(pts16, n)
    H = np.empty((a.shape[0], 9))
    getattr(lib(), name)(_ptr(a, _d), _ptr(H, _d), a.shape[0])
    return H


def aca(pts16, n=None):
    """ACA (Eq. 20-29), unnormalised, (n, 9) float64."""
    return _solve("oracle_aca", pts16, n)


def aca_divform(pts16, n=None):
    """ACA with the division-form core (Eq. 23, 26)."""
    return _solve("oracle_aca_divform", pts16, n)


def aca_affine(pts12, n=None):
    """Affine map from three correspondences, Eq. 38: H_A2^-1 H_A1, (n, 9),
    third row (0, 0, f_A1).  pts12: SoA (12, ld) = M1 N1 P1 M2 N2 P2."""
    n = pts12.shape[1] if n is None else n
    a = np.ascontiguousarray(np.asarray(pts12[:, :n], dtype=np.float64).T)
    H = np.empty((n, 9))
    lib().oracle_aca_affine(_ptr(a, _d), _ptr(H, _d), n)
    return H


def sks(pts16, n=None):
    """SKS (Eq. 4-14), (n, 9) float64."""
    return _solve("oracle_sks", pts16, n)


def dlt(pts16, n=None):
    """Independent 8x8 DLT with partial pivoting, h33 = 1, (n, 9)."""
    a = sets_aos(pts16, n)
    H = np.empty((a.shape[0], 9))
    lib().oracle_dlt(_ptr(a, _d), _ptr(H, _d), a.shape[0])
    return H


def aca_jacobian(pts16, n=None):
    """dH/d(target coordinates), (n, 9, 8)."""
    a = sets_aos(pts16, n)
    J = np.empty((a.shape[0], 9, 8))
    lib().oracle_aca_jacobian(_ptr(a, _d), _ptr(J, _d), a.shape[0])
    return J


def aca_jacobian_src(pts16, n=None):
    """dH/d(source coordinates), (n, 9, 8)."""
    a = sets_aos(pts16, n)
    J = np.empty((a.shape[0], 9, 8))
    lib().oracle_aca_jacobian_src(_ptr(a, _d), _ptr(J, _d), a.shape[0])
    return J


def aca_condition(pts16, n=None):
    """Componentwise condition number kappa of the unit-Frobenius ACA H
    w.r.t. relative perturbations of the 16 input coordinates, (n,)."""
    a = sets_aos(pts16, n)
    k = np.empty(a.shape[0])
    lib().oracle_aca_condition(_ptr(a, _d), _ptr(k, _d), a.shape[0])
    return k


def _rect(name, tgt8, rect, n=None, out_cols=9, per=1):
    n = tgt8.shape[1] if n is None else n
    t = np.ascontiguousarray(np.asarray(tgt8[:, :n], dtype=np.float64).T)
    x0, y0, w, r = (float(v) for v in rect)
    out = np.empty((n, out_cols * per))
    getattr(lib(), name)(_ptr(t, _d), x0, y0, w, r, _ptr(out, _d), n)
    return out


def aca_rect(tgt8, rect, n=None):
    """Rectangle source, Eq. 42, (n, 9)."""
    return _rect("oracle_aca_rect", tgt8, rect, n)


def aca_rect_alg1(tgt8, rect, n=None):
    """Rectangle source, Algorithm 1's operations, (n, 9)."""
    return _rect("oracle_aca_rect_alg1", tgt8, rect, n)


def aca_rect_jacobian(tgt8, rect, n=None):
    """dH/d(target corners) of Eq. 42, (n, 9, 8)."""
    return _rect("oracle_aca_rect_jacobian", tgt8, rect, n, per=8).reshape(-1, 9, 8)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.empty(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(c, _u32), _ptr(k, _u32), _ptr(out, _u32))
    return out


def sample4(seed: int, prob: int, hyp: int, N: int) -> np.ndarray:
    out = np.empty(4, dtype=np.int64)
    lib().oracle_sample4(seed, prob, hyp, N, _ptr(out, _i64))
    return out


def sample_degenerate(s16) -> bool:
    s = np.ascontiguousarray(np.asarray(s16, dtype=np.float64).reshape(16))
    return bool(lib().oracle_sample_degenerate(_ptr(s, _d)))


def normalize_frob(H) -> np.ndarray:
    """Unit Frobenius norm, sign fixed (h33 > 0, else largest entry > 0)."""
    H = np.array(H, dtype=np.float64).reshape(-1, 9)
    for row in H:
        r = np.ascontiguousarray(row)
        lib().oracle_normalize_frob(_ptr(r, _d))
        row[:] = r
    return H


def score_problem(corr, n_hyp: int, thr: float, seed: int, prob: int = 0, band_px: float = 1e-4):
    """Per-hypothesis counts (-1 = degenerate sample) and the ambiguous
    points of each hypothesis (oracle_score_problem): those within band_px
    of the threshold or within the first-order rounding bound of the FP32
    test (fp32_bounds.c), split by the exact decision.  Returns
    (counts, amb_in, amb_out); an FP32 count c is consistent when
    counts - amb_in <= c <= counts + amb_out."""
    c = np.ascontiguousarray(corr, dtype=np.float32)
    N = c.shape[0]
    cnt = np.empty(n_hyp, dtype=np.int32)
    ai = np.empty(n_hyp, dtype=np.int32)
    ao = np.empty(n_hyp, dtype=np.int32)
    lib().oracle_score_problem(_ptr(c, _f), N, n_hyp, thr, seed, prob, _ptr(cnt, _i32), _ptr(ai, _i32),
                               _ptr(ao, _i32), band_px)
    return cnt, ai, ao


def ransac(corr, offsets, n_hyp, thr: float, seed: int, problem_base: int = 0, band_px: float = 1e-4,
           want_counts: bool = True, want_mask: bool = False) -> dict:
    """Brute-force RANSAC over CSR problems; see oracle_ransac in oracle.c.
    band_in / band_out: ambiguous points per hypothesis (score_problem);
    band_counts = their sum."""
    c = np.ascontiguousarray(corr, dtype=np.float32)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    k = np.ascontiguousarray(n_hyp, dtype=np.int32)
    P = k.shape[0]
    tot = int(k.sum())
    best_H = np.empty((P, 9))
    best_count = np.empty(P, dtype=np.int32)
    best_hyp = np.empty(P, dtype=np.int32)
    counts = np.empty(tot, dtype=np.int32) if want_counts else None
    ai = np.empty(tot, dtype=np.int32) if want_counts else None
    ao = np.empty(tot, dtype=np.int32) if want_counts else None
    mask = np.empty(c.shape[0], dtype=np.uint8) if want_mask else None
    lib().oracle_ransac(_ptr(c, _f), _ptr(off, _i64), _ptr(k, _i32), P, thr, seed, problem_base,
                        _ptr(best_H, _d), _ptr(best_count, _i32), _ptr(best_hyp, _i32),
                        _ptr(counts, _i32), _ptr(ai, _i32), _ptr(ao, _i32), band_px, _ptr(mask, _u8))
    return dict(best_H=best_H, best_count=best_count, best_hyp=best_hyp, hyp_counts=counts, band_in=ai,
                band_out=ao, band_counts=None if ai is None else ai + ao, inlier_mask=mask)


def adaptive_k(c: int, N: int, cap: int, confidence: float = 0.99) -> int:
    """Hypotheses required by the online stop rule for a best count c of N
    (see oracle_adaptive_k)."""
    return int(lib().oracle_adaptive_k(int(c), int(N), int(cap), float(np.log(1.0 - confidence))))


def adaptive_stop(counts, N: int, confidence: float = 0.99) -> int:
    """Number of hypotheses the sequential loop evaluates over `counts`
    (cap = len(counts)); see oracle_adaptive_stop."""
    c = np.ascontiguousarray(counts, dtype=np.int32)
    return int(lib().oracle_adaptive_stop(_ptr(c, _i32), c.size, int(N), float(np.log(1.0 - confidence))))


def ransac_adaptive(corr, offsets, max_hyp, thr: float, seed: int, confidence: float = 0.99,
                    problem_base: int = 0, band_px: float = 1e-4, want_mask: bool = False,
                    want_band: bool = True) -> dict:
    """RANSAC with the online stop (oracle_ransac_adaptive): counts and
    ambiguous points (band_in / band_out, as in ransac; None without
    want_band) of all max_hyp hypotheses, n_eval, and the best over the
    evaluated ones."""
    c = np.ascontiguousarray(corr, dtype=np.float32)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    k = np.ascontiguousarray(max_hyp, dtype=np.int32)
    P = k.shape[0]
    tot = int(k.sum())
    best_H = np.empty((P, 9))
    best_count = np.empty(P, dtype=np.int32)
    best_hyp = np.empty(P, dtype=np.int32)
    n_eval = np.empty(P, dtype=np.int32)
    counts = np.empty(tot, dtype=np.int32)
    ai = np.empty(tot, dtype=np.int32) if want_band else None
    ao = np.empty(tot, dtype=np.int32) if want_band else None
    mask = np.empty(c.shape[0], dtype=np.uint8) if want_mask else None
    lib().oracle_ransac_adaptive(_ptr(c, _f), _ptr(off, _i64), _ptr(k, _i32), P, thr, seed, problem_base,
                                 confidence, _ptr(best_H, _d), _ptr(best_count, _i32), _ptr(best_hyp, _i32),
                                 _ptr(n_eval, _i32), _ptr(counts, _i32), _ptr(ai, _i32), _ptr(ao, _i32), band_px,
                                 _ptr(mask, _u8))
    return dict(best_H=best_H, best_count=best_count, best_hyp=best_hyp, n_eval=n_eval, hyp_counts=counts,
                band_in=ai, band_out=ao, band_counts=None if ai is None else ai + ao, inlier_mask=mask)


from .inlier_refit import hartley_normalization, refit, refit_dlt, refit_lm, refit_tolerance, reprojection_cost  # noqa: E402,F401


def _fp32_bound(name, pts16, n=None, per_entry=False):
    a = sets_aos(pts16, n)
    m = a.shape[0]
    beta = np.empty(m)
    Hv = np.empty((m, 9)) if per_entry else None
    He = np.empty((m, 9)) if per_entry else None
    getattr(lib(), name)(_ptr(a, _d), _ptr(beta, _d), _ptr(Hv, _d), _ptr(He, _d), m)
    return (beta, Hv, He) if per_entry else beta


def aca_fp32_bound(pts16, n=None, per_entry=False):
    """First-order bound on the error of the library's FP32 ACA evaluation
    order (running error analysis, fp32_bounds.c): beta per set, the bound on
    max |H^_fp32 - H^| at unit Frobenius norm; with per_entry, also the exact
    H of that order (n, 9) and per-entry absolute bounds (n, 9)."""
    return _fp32_bound("oracle_aca_fp32_bound", pts16, n, per_entry)


def sks_fp32_bound(pts16, n=None, per_entry=False):
    """As aca_fp32_bound, for the library's FP32 SKS evaluation order."""
    return _fp32_bound("oracle_sks_fp32_bound", pts16, n, per_entry)


def score_band(s16, corr, thr: float, band_px: float = 1e-4):
    """Per-point ambiguity of one hypothesis (minimal set s16, 16 coordinates)
    over corr (N, 4) float32: 1 where the FP32 inlier test may decide
    otherwise than the exact test, or where the exact residual is within
    band_px of the threshold.  Returns a (N,) uint8 array."""
    s = np.ascontiguousarray(np.asarray(s16, dtype=np.float64).ravel())
    c = np.ascontiguousarray(corr, dtype=np.float32)
    amb = np.empty(c.shape[0], np.uint8)
    lib().oracle_score_band(_ptr(s, _d), _ptr(c, _f), c.shape[0], float(thr), float(band_px), _ptr(amb, _u8))
    return amb


def score_band_px(s16, corr, thr: float):
    """The FP32 test's bound at each point in pixels of |r - thr| (N,)."""
    s = np.ascontiguousarray(np.asarray(s16, dtype=np.float64).ravel())
    c = np.ascontiguousarray(corr, dtype=np.float32)
    px = np.empty(c.shape[0])
    lib().oracle_score_band_px(_ptr(s, _d), _ptr(c, _f), c.shape[0], float(thr), _ptr(px, _d))
    return px


def fp32_rule_bound(op: int, args):
    """Bound of one rounding rule of fp32_bounds.c on FP32 operands (see
    oracle_fp32_rule_bound): returns (exact value, bound on |fl - exact|)."""
    a = np.zeros(8)
    a[:len(args)] = np.asarray(args, dtype=np.float32).astype(np.float64)
    v = np.zeros(1)
    b = lib().oracle_fp32_rule_bound(int(op), _ptr(a, _d), _ptr(v, _d))
    return float(v[0]), float(b)


def score_bound_E(s16, corr, thr: float):
    """Exact E = w^2 (r^2 - thr^2) of the inlier test at every point under the
    hypothesis of minimal set s16, and the first-order bound on the error of
    its FP32 evaluation (solve included).  Returns (E, B), each (N,)."""
    s = np.ascontiguousarray(np.asarray(s16, dtype=np.float64).ravel())
    c = np.ascontiguousarray(corr, dtype=np.float32)
    E = np.empty(c.shape[0])
    B = np.empty(c.shape[0])
    lib().oracle_score_bound_E(_ptr(s, _d), _ptr(c, _f), c.shape[0], float(thr), _ptr(E, _d), _ptr(B, _d))
    return E, B


def fp32_chain_corner(solver: str, s16, g9):
    """The worst corner of a solver's rounding events, re-evaluated (a pin of
    the bound's reverse sweep; fp32_bounds.c oracle_fp32_chain_corner).  For
    F = sum g_i H_i of the "aca" or "sks" chain at the set s16: returns
    (b1, dev, bound), the first-order bound on |fl(F) - F|, F re-run with every
    event at the sign of its weight times its bound, minus the exact F; and
    (third) the whole bound, with the allowance for products of events."""
    s = np.ascontiguousarray(np.asarray(s16, dtype=np.float64).ravel())
    g = np.ascontiguousarray(np.asarray(g9, dtype=np.float64).ravel())
    dev = np.zeros(1)
    b1 = np.zeros(1)
    b = lib().oracle_fp32_chain_corner({"aca": 0, "sks": 1}[solver], _ptr(s, _d), _ptr(g, _d), _ptr(dev, _d),
                                       _ptr(b1, _d))
    return float(b1[0]), float(dev[0]), float(b)


def score_bound_E_fixed(H9, corr, thr: float):
    """The inlier test at an exact H (nine values, no solve events): per
    point the exact E and the bound of the test's own rounding events.
    Returns (E, B), each (N,)."""
    h = np.ascontiguousarray(np.asarray(H9, dtype=np.float64).ravel())
    c = np.ascontiguousarray(corr, dtype=np.float32)
    E = np.empty(c.shape[0])
    B = np.empty(c.shape[0])
    lib().oracle_score_bound_E_fixed(_ptr(h, _d), _ptr(c, _f), c.shape[0], float(thr), _ptr(E, _d), _ptr(B, _d))
    return E, B


def score_corner(s16, c4, thr: float):
    """The inlier test at one point c4 under the hypothesis of the minimal set
    s16, with the solve's rounding events and then the test's placed at the
    signs of their first-order weights.  Returns (B1, dev, E): the
    first-order bound of e, the re-evaluated e minus E, and the exact E."""
    s = np.ascontiguousarray(np.asarray(s16, dtype=np.float64).ravel())
    c = np.ascontiguousarray(np.asarray(c4, dtype=np.float32).ravel())
    out = np.zeros(3)
    lib().oracle_score_corner(_ptr(s, _d), _ptr(c, _f), float(thr), _ptr(out[0:], _d), _ptr(out[1:], _d),
                              _ptr(out[2:], _d))
    return float(out[0]), float(out[1]), float(out[2])
