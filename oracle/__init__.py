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
Levenberg-Marquardt: the global optimisation of Sec. 6.2, stage 5).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(exact agreement with an independent DLT, invariants, special cases, cuRAND's
Philox, brute-force enumeration).  None is "parity unpinned".
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
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.oracle_num_threads.restype = ctypes.c_int
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
                                               ctypes.c_uint64, ctypes.c_uint32, _i32, _i32, ctypes.c_double,
                                               ctypes.c_double]
            L.oracle_ransac.argtypes = [_f, _i64, _i32, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64,
                                        ctypes.c_uint32, _d, _i32, _i32, _i32, _i32, ctypes.c_double,
                                        ctypes.c_double, _u8]
            L.oracle_adaptive_k.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_double]
            L.oracle_adaptive_k.restype = ctypes.c_int32
            L.oracle_adaptive_stop.argtypes = [_i32, ctypes.c_int32, ctypes.c_int64, ctypes.c_double]
            L.oracle_adaptive_stop.restype = ctypes.c_int32
            L.oracle_ransac_adaptive.argtypes = [_f, _i64, _i32, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64,
                                                 ctypes.c_uint32, ctypes.c_double, _d, _i32, _i32, _i32, _i32,
                                                 _i32, ctypes.c_double, ctypes.c_double, _u8]
            _lib = L
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def num_threads() -> int:
    return int(lib().oracle_num_threads())


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


def score_problem(corr, n_hyp: int, thr: float, seed: int, prob: int = 0, band_px: float = 1e-4,
                  herr: float = 0.0):
    """Per-hypothesis counts (-1 = degenerate sample) and band counts (see
    oracle_score_problem: band_px plus, when herr > 0, the first-order
    effect of an FP32-solver error of herr * kappa_h * 2^-24 + 2^-23 on H)."""
    c = np.ascontiguousarray(corr, dtype=np.float32)
    N = c.shape[0]
    cnt = np.empty(n_hyp, dtype=np.int32)
    band = np.empty(n_hyp, dtype=np.int32)
    lib().oracle_score_problem(_ptr(c, _f), N, n_hyp, thr, seed, prob, _ptr(cnt, _i32), _ptr(band, _i32), band_px,
                               herr)
    return cnt, band


def ransac(corr, offsets, n_hyp, thr: float, seed: int, problem_base: int = 0, band_px: float = 1e-4,
           want_counts: bool = True, want_mask: bool = False, herr: float = 0.0) -> dict:
    """Brute-force RANSAC over CSR problems; see oracle_ransac in oracle.c."""
    c = np.ascontiguousarray(corr, dtype=np.float32)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    k = np.ascontiguousarray(n_hyp, dtype=np.int32)
    P = k.shape[0]
    tot = int(k.sum())
    best_H = np.empty((P, 9))
    best_count = np.empty(P, dtype=np.int32)
    best_hyp = np.empty(P, dtype=np.int32)
    counts = np.empty(tot, dtype=np.int32) if want_counts else None
    band = np.empty(tot, dtype=np.int32) if want_counts else None
    mask = np.empty(c.shape[0], dtype=np.uint8) if want_mask else None
    lib().oracle_ransac(_ptr(c, _f), _ptr(off, _i64), _ptr(k, _i32), P, thr, seed, problem_base,
                        _ptr(best_H, _d), _ptr(best_count, _i32), _ptr(best_hyp, _i32),
                        _ptr(counts, _i32), _ptr(band, _i32), band_px, herr, _ptr(mask, _u8))
    return dict(best_H=best_H, best_count=best_count, best_hyp=best_hyp, hyp_counts=counts,
                band_counts=band, inlier_mask=mask)



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
                    herr: float = 0.0) -> dict:
    """RANSAC with the online stop (oracle_ransac_adaptive): counts and band
    counts of all max_hyp hypotheses, n_eval, and the best over the evaluated
    ones."""
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
    band = np.empty(tot, dtype=np.int32)
    mask = np.empty(c.shape[0], dtype=np.uint8) if want_mask else None
    lib().oracle_ransac_adaptive(_ptr(c, _f), _ptr(off, _i64), _ptr(k, _i32), P, thr, seed, problem_base,
                                 confidence, _ptr(best_H, _d), _ptr(best_count, _i32), _ptr(best_hyp, _i32),
                                 _ptr(n_eval, _i32), _ptr(counts, _i32), _ptr(band, _i32), band_px, herr,
                                 _ptr(mask, _u8))
    return dict(best_H=best_H, best_count=best_count, best_hyp=best_hyp, n_eval=n_eval, hyp_counts=counts,
                band_counts=band, inlier_mask=mask)


from .inlier_refit import hartley_normalization, refit, refit_dlt, refit_lm, refit_tolerance, reprojection_cost  # noqa: E402,F401
