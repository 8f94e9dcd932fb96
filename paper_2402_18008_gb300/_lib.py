"""ctypes binding of the C ABI in include/aca.h (argument marshalling only).

Every function here takes torch CUDA tensors, checks dtype / device / shape,
and passes raw device pointers plus the current CUDA stream to the library;
all computation happens in the CUDA kernels.  There is no CPU fallback: if
the shared library is missing or no CUDA device is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

_lock = threading.Lock()
_lib = None

ACA_NORM_NONE, ACA_NORM_H33, ACA_NORM_FROB = 0, 1, 2
ACA_FLAG_SRC_ANCHORS, ACA_FLAG_TGT_ANCHORS, ACA_FLAG_OTHER_TRIPLE, ACA_FLAG_NON_FINITE = 1, 2, 4, 8
_STATUS = {0: "ACA_OK", -1: "ACA_ERR_INVALID_ARG", -2: "ACA_ERR_CUDA", -3: "ACA_ERR_WORKSPACE", -4: "ACA_ERR_TIMEOUT"}

EXPORTED = ("aca_solve", "sks_solve", "aca_rect_solve", "aca_affine_solve", "aca_backward", "aca_rect_backward",
            "ransac_aca_workspace_size", "ransac_aca", "ransac_aca_noalloc", "ransac_aca_adaptive_workspace_size",
            "ransac_aca_adaptive", "aca_sample_indices", "aca_refit", "aca_fma_probe", "aca_fma_probe_flops",
            "aca_last_error", "aca_version")
ACA_NOALLOC_SCRATCH_BYTES = 8 * 1024 * 1024


class AcaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class RansacParams(ctypes.Structure):
    _fields_ = [("threshold_px", ctypes.c_float), ("problem_base", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("block_warps", ctypes.c_int32), ("hyps_per_thread", ctypes.c_int32),
                ("grid_blocks", ctypes.c_int32), ("tile_points", ctypes.c_int32)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load (building first if needed) the shared library."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise OSError(f"CUDA library not built: {path}")
            _build.build()
        L = ctypes.CDLL(path)
        vp, i64, i32, f32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float
        for name in ("aca_solve", "sks_solve"):
            getattr(L, name).argtypes = [vp, vp, vp, i64, i64, i32, vp]
        L.aca_rect_solve.argtypes = [vp, f32, f32, f32, f32, vp, i64, i64, vp]
        L.aca_affine_solve.argtypes = [vp, vp, i64, i64, i32, vp]
        L.aca_backward.argtypes = [vp, vp, vp, i64, i64, vp]
        L.aca_rect_backward.argtypes = [vp, f32, f32, f32, f32, vp, vp, i64, i64, vp]
        L.ransac_aca_workspace_size.argtypes = [i32, i64]
        L.ransac_aca_workspace_size.restype = ctypes.c_size_t
        L.ransac_aca.argtypes = [vp, vp, vp, i32, ctypes.POINTER(RansacParams), vp, vp, vp, vp, vp, vp,
                                 ctypes.c_size_t, vp]
        L.aca_sample_indices.argtypes = [i64, i32, ctypes.c_uint64, ctypes.c_uint32, vp, vp]
        L.ransac_aca_noalloc.argtypes = [vp, vp, vp, i32, i64, ctypes.POINTER(RansacParams), vp, vp, vp, vp, vp, vp]
        L.aca_refit.argtypes = [vp, vp, vp, i32, i32, vp, vp, vp, vp]
        L.ransac_aca_adaptive_workspace_size.argtypes = [i32, i64]
        L.ransac_aca_adaptive_workspace_size.restype = ctypes.c_size_t
        L.ransac_aca_adaptive.argtypes = [vp, vp, vp, i32, i64, ctypes.POINTER(RansacParams), ctypes.c_double, vp,
                                          vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
        L.aca_fma_probe.argtypes = [i32, i32, i32, i32, vp, vp]
        L.aca_fma_probe_flops.argtypes = [i32, i32, i32, i32]
        L.aca_fma_probe_flops.restype = ctypes.c_int64
        for name in EXPORTED:
            if name not in ("ransac_aca_workspace_size", "ransac_aca_adaptive_workspace_size", "aca_last_error",
                            "aca_version", "aca_fma_probe_flops"):
                getattr(L, name).restype = ctypes.c_int
        L.aca_last_error.restype = ctypes.c_char_p
        L.aca_version.restype = ctypes.c_char_p
        _lib = L
        return L


def _check(st: int):
    if st != 0:
        raise AcaError(st, load().aca_last_error().decode())


def _L():
    """The loaded library (no lock once it is loaded)."""
    return _lib if _lib is not None else load()


try:                                   # the current stream as a raw handle, without a Stream object
    _raw_stream = torch._C._cuda_getCurrentRawStream
except AttributeError:                 # pragma: no cover
    def _raw_stream(device: int) -> int:
        return int(torch.cuda.current_stream(device).cuda_stream)


def _stream(stream=None, like=None) -> int:
    """Raw handle of `stream`, else of the current stream of `like`'s device
    (of the current device for a host tensor or None)."""
    if stream is not None:
        return int(stream.cuda_stream)
    dev = like.get_device() if like is not None else -1
    return _raw_stream(dev if dev >= 0 else torch.cuda.current_device())


def _ptr(t):
    return None if t is None else t.data_ptr()


_F32, _U8 = torch.float32, torch.uint8


def _need(t, name, dtype, rows=None, host_ok=False):
    # host_ok: page-locked host tensors are accepted too (the kernel reads and
    # writes them over the host link itself; nothing runs on the CPU)
    if not isinstance(t, torch.Tensor) or not (t.is_cuda or (host_ok and t.is_pinned())):
        raise ValueError(f"{name} must be a CUDA tensor" + (" or a pinned host tensor" if host_ok else ""))
    if t.dtype is not dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if rows is not None:
        sh = t.shape
        if len(sh) != 2 or sh[0] != rows or t.stride(1) != 1:
            raise ValueError(f"{name} must be ({rows}, ld) with unit stride along ld")


def _planes(t, name, dtype, rows, host_ok=False):
    """_need for a (rows, ld) plane tensor, reading its shape and strides
    once: returns (row length, leading dimension)."""
    if not isinstance(t, torch.Tensor) or not (t.is_cuda or (host_ok and t.is_pinned())):
        raise ValueError(f"{name} must be a CUDA tensor" + (" or a pinned host tensor" if host_ok else ""))
    if t.dtype is not dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    sh, st = t.shape, t.stride()
    if len(sh) != 2 or sh[0] != rows or st[1] != 1:
        raise ValueError(f"{name} must be ({rows}, ld) with unit stride along ld")
    return sh[1], st[0]


def _shared_ld(*cols_lds):
    """The leading dimension that (row length, ld) pairs share."""
    ld = cols_lds[0][1]
    for cols, l in cols_lds:
        if l != ld:
            raise ValueError("all planes must share one leading dimension (row stride)")
        if cols > ld:
            raise ValueError("row length exceeds the leading dimension")
    return ld


def _ld(*ts):
    ld = None
    for t in ts:
        if t is None:
            continue
        s0 = t.stride(0)
        if ld is None:
            ld = s0
        elif s0 != ld:
            raise ValueError("all planes must share one leading dimension (row stride)")
        if t.shape[1] > ld:
            raise ValueError("row length exceeds the leading dimension")
    return ld


def aca_solve(pts, H, flags=None, n=None, norm=ACA_NORM_NONE, stream=None):
    """C ABI aca_solve on (16, ld) float32 planes -> (9, ld) float32.  Each
    tensor may be on the GPU or in pinned host memory (zero-copy)."""
    p = _planes(pts, "pts", _F32, 16, host_ok=True)
    ld = _shared_ld(p, _planes(H, "H", _F32, 9, host_ok=True))
    if flags is not None:
        _need(flags, "flags", torch.uint8, host_ok=True)
    r = _L().aca_solve(pts.data_ptr(), H.data_ptr(), _ptr(flags), p[0] if n is None else n, ld, norm,
                       _stream(stream, pts))
    if r:
        _check(r)


def sks_solve(pts, H, flags=None, n=None, norm=ACA_NORM_NONE, stream=None):
    """C ABI sks_solve on (16, ld) float32 planes -> (9, ld) float32."""
    p = _planes(pts, "pts", _F32, 16)
    ld = _shared_ld(p, _planes(H, "H", _F32, 9))
    if flags is not None:
        _need(flags, "flags", torch.uint8)
    r = _L().sks_solve(pts.data_ptr(), H.data_ptr(), _ptr(flags), p[0] if n is None else n, ld, norm,
                       _stream(stream, pts))
    if r:
        _check(r)


def aca_rect_solve(tgt, rect, H, n=None, stream=None):
    """C ABI aca_rect_solve: rect = (x0, y0, w, r)."""
    p = _planes(tgt, "tgt", _F32, 8)
    ld = _shared_ld(p, _planes(H, "H", _F32, 9))
    x0, y0, w, r = (float(v) for v in rect)
    st = _L().aca_rect_solve(tgt.data_ptr(), x0, y0, w, r, H.data_ptr(), p[0] if n is None else n, ld,
                             _stream(stream, tgt))
    if st:
        _check(st)


def aca_affine_solve(pts, H, n=None, norm=ACA_NORM_NONE, stream=None):
    """C ABI aca_affine_solve: (12, ld) planes M1 N1 P1 M2 N2 P2 -> (9, ld)."""
    _need(pts, "pts", torch.float32, 12)
    _need(H, "H", torch.float32, 9)
    ld = _ld(pts, H)
    n = pts.shape[1] if n is None else n
    _check(_L().aca_affine_solve(pts.data_ptr(), H.data_ptr(), n, ld, norm, _stream(stream, pts)))


def aca_backward(pts, grad_H, grad_tgt, n=None, stream=None):
    """C ABI aca_backward: (16, ld) sets, (9, ld) dL/dH -> (8, ld) dL/dtgt."""
    p = _planes(pts, "pts", _F32, 16)
    ld = _shared_ld(p, _planes(grad_H, "grad_H", _F32, 9), _planes(grad_tgt, "grad_tgt", _F32, 8))
    r = _L().aca_backward(pts.data_ptr(), grad_H.data_ptr(), grad_tgt.data_ptr(), p[0] if n is None else n, ld,
                          _stream(stream, pts))
    if r:
        _check(r)


def aca_rect_backward(tgt, rect, grad_H, grad_tgt, n=None, stream=None):
    """C ABI aca_rect_backward."""
    p = _planes(tgt, "tgt", _F32, 8)
    ld = _shared_ld(p, _planes(grad_H, "grad_H", _F32, 9), _planes(grad_tgt, "grad_tgt", _F32, 8))
    x0, y0, w, r = (float(v) for v in rect)
    st = _L().aca_rect_backward(tgt.data_ptr(), x0, y0, w, r, grad_H.data_ptr(), grad_tgt.data_ptr(),
                                p[0] if n is None else n, ld, _stream(stream, tgt))
    if st:
        _check(st)


class Prepared:
    """One C-ABI call bound to fixed tensors: the arguments are checked once,
    when it is made, and every call then passes the precomputed pointers and
    sizes and the current stream (for loops that call the same entry point
    on the same buffers, where per-call marshalling would exceed the kernel's
    own time).  It keeps references to its tensors."""

    __slots__ = ("_fn", "_args", "_dev", "_keep")

    def __init__(self, fn, args, like, keep):
        self._fn, self._args, self._keep = fn, tuple(args), keep
        dev = like.get_device()
        self._dev = dev if dev >= 0 else torch.cuda.current_device()

    def __call__(self, stream=None):
        st = int(stream.cuda_stream) if stream is not None else _raw_stream(self._dev)
        r = self._fn(*self._args, st)
        if r:
            _check(r)


def prepare_aca_solve(pts, H, flags=None, n=None, norm=ACA_NORM_NONE) -> Prepared:
    """aca_solve bound to pts, H (and flags): see aca_solve and Prepared."""
    _need(pts, "pts", torch.float32, 16, host_ok=True)
    _need(H, "H", torch.float32, 9, host_ok=True)
    if flags is not None:
        _need(flags, "flags", torch.uint8, host_ok=True)
    ld = _ld(pts, H)
    n = pts.shape[1] if n is None else int(n)
    return Prepared(_L().aca_solve, (pts.data_ptr(), H.data_ptr(), _ptr(flags), n, ld, int(norm)), pts,
                    (pts, H, flags))


def prepare_aca_rect_solve(tgt, rect, H, n=None) -> Prepared:
    """aca_rect_solve bound to tgt, rect and H: see Prepared."""
    _need(tgt, "tgt", torch.float32, 8)
    _need(H, "H", torch.float32, 9)
    ld = _ld(tgt, H)
    n = tgt.shape[1] if n is None else int(n)
    x0, y0, w, r = (float(v) for v in rect)
    return Prepared(_L().aca_rect_solve, (tgt.data_ptr(), x0, y0, w, r, H.data_ptr(), n, ld), tgt, (tgt, H))


def prepare_aca_rect_backward(tgt, rect, grad_H, grad_tgt, n=None) -> Prepared:
    """aca_rect_backward bound to its tensors: see Prepared."""
    _need(tgt, "tgt", torch.float32, 8)
    _need(grad_H, "grad_H", torch.float32, 9)
    _need(grad_tgt, "grad_tgt", torch.float32, 8)
    ld = _ld(tgt, grad_H, grad_tgt)
    n = tgt.shape[1] if n is None else int(n)
    x0, y0, w, r = (float(v) for v in rect)
    return Prepared(_L().aca_rect_backward,
                    (tgt.data_ptr(), x0, y0, w, r, grad_H.data_ptr(), grad_tgt.data_ptr(), n, ld), tgt,
                    (tgt, grad_H, grad_tgt))


def ransac_aca_workspace_size(P: int, total_hyps: int) -> int:
    return int(load().ransac_aca_workspace_size(P, total_hyps))


def ransac_aca(corr, offsets, n_hyp, params: RansacParams, best_H, best_count, best_hyp, workspace,
               hyp_counts=None, inlier_mask=None, stream=None):
    """C ABI ransac_aca.  corr (total, 4) float32; offsets (P+1,) int64;
    n_hyp (P,) int32; outputs best_H (P, 9) float32, best_count / best_hyp
    (P,) int32; workspace uint8 of ransac_aca_workspace_size bytes."""
    _need(corr, "corr", torch.float32)
    _need(offsets, "offsets", torch.int64)
    _need(n_hyp, "n_hyp", torch.int32)
    _need(best_H, "best_H", torch.float32)
    _need(best_count, "best_count", torch.int32)
    _need(best_hyp, "best_hyp", torch.int32)
    _need(workspace, "workspace", torch.uint8)
    if corr.dim() != 2 or corr.shape[1] != 4 or not corr.is_contiguous():
        raise ValueError("corr must be a contiguous (total, 4) tensor")
    P = n_hyp.numel()
    if offsets.numel() != P + 1:
        raise ValueError("offsets must have P+1 entries")
    for t, nm in ((offsets, "offsets"), (n_hyp, "n_hyp"), (best_H, "best_H"), (best_count, "best_count"),
                  (best_hyp, "best_hyp")):
        if not t.is_contiguous():
            raise ValueError(f"{nm} must be contiguous")
    if best_H.numel() < 9 * P or best_count.numel() < P or best_hyp.numel() < P:
        raise ValueError("output tensors too small")
    if hyp_counts is not None:
        _need(hyp_counts, "hyp_counts", torch.int32)
    if inlier_mask is not None:
        _need(inlier_mask, "inlier_mask", torch.uint8)
        if inlier_mask.numel() < corr.shape[0]:
            raise ValueError("inlier_mask too small")
    _check(load().ransac_aca(_ptr(corr), _ptr(offsets), _ptr(n_hyp), P, ctypes.byref(params), _ptr(best_H),
                             _ptr(best_count), _ptr(best_hyp), _ptr(hyp_counts), _ptr(inlier_mask),
                             _ptr(workspace), workspace.numel(), _stream(stream, corr)))


def aca_sample_indices(N: int, n_hyp: int, seed: int, problem: int, idx, stream=None):
    """C ABI aca_sample_indices into idx (n_hyp, 4) int32."""
    _need(idx, "idx", torch.int32)
    if not idx.is_contiguous() or idx.numel() < 4 * n_hyp:
        raise ValueError("idx must be a contiguous (n_hyp, 4) int32 tensor")
    _check(load().aca_sample_indices(int(N), int(n_hyp), int(seed), int(problem), _ptr(idx),
                                     _stream(stream, idx)))


def ransac_aca_noalloc(corr, offsets, n_hyp, total_hyps: int, params: RansacParams, best_H, best_count, best_hyp,
                       hyp_counts=None, inlier_mask=None, stream=None):
    """C ABI ransac_aca_noalloc: ransac_aca with the library's built-in scratch
    (no workspace argument, no device allocation); total_hyps = sum(n_hyp)."""
    _need(corr, "corr", torch.float32)
    _need(offsets, "offsets", torch.int64)
    _need(n_hyp, "n_hyp", torch.int32)
    _need(best_H, "best_H", torch.float32)
    _need(best_count, "best_count", torch.int32)
    _need(best_hyp, "best_hyp", torch.int32)
    if corr.dim() != 2 or corr.shape[1] != 4 or not corr.is_contiguous():
        raise ValueError("corr must be a contiguous (total, 4) tensor")
    P = n_hyp.numel()
    if offsets.numel() != P + 1:
        raise ValueError("offsets must have P+1 entries")
    for t, nm in ((offsets, "offsets"), (n_hyp, "n_hyp"), (best_H, "best_H"), (best_count, "best_count"),
                  (best_hyp, "best_hyp")):
        if not t.is_contiguous():
            raise ValueError(f"{nm} must be contiguous")
    if best_H.numel() < 9 * P or best_count.numel() < P or best_hyp.numel() < P:
        raise ValueError("output tensors too small")
    if hyp_counts is not None:
        _need(hyp_counts, "hyp_counts", torch.int32)
        if hyp_counts.numel() < total_hyps or not hyp_counts.is_contiguous():
            raise ValueError("hyp_counts must be a contiguous tensor of at least total_hyps entries")
    if inlier_mask is not None:
        _need(inlier_mask, "inlier_mask", torch.uint8)
        if inlier_mask.numel() < corr.shape[0]:
            raise ValueError("inlier_mask too small")
    _check(load().ransac_aca_noalloc(_ptr(corr), _ptr(offsets), _ptr(n_hyp), P, int(total_hyps), ctypes.byref(params),
                                     _ptr(best_H), _ptr(best_count), _ptr(best_hyp), _ptr(hyp_counts),
                                     _ptr(inlier_mask), _stream(stream, corr)))


def aca_refit(corr, offsets, H, mask=None, lm_iters=10, n_used=None, rms=None, stream=None):
    """C ABI aca_refit.  corr (total, 4) float32; offsets (P+1,) int64;
    mask (total,) uint8 or None (every point); outputs H (P, 9) float32,
    n_used (P,) int32 and rms (P,) float32, the last two optional."""
    _need(corr, "corr", torch.float32)
    _need(offsets, "offsets", torch.int64)
    _need(H, "H", torch.float32)
    if corr.dim() != 2 or corr.shape[1] != 4 or not corr.is_contiguous():
        raise ValueError("corr must be a contiguous (total, 4) tensor")
    P = offsets.numel() - 1
    if P < 0 or not offsets.is_contiguous() or not H.is_contiguous() or H.numel() < 9 * P:
        raise ValueError("offsets must be (P+1,) and H a contiguous (P, 9) tensor")
    if mask is not None:
        _need(mask, "mask", torch.uint8)
        if mask.numel() < corr.shape[0] or not mask.is_contiguous():
            raise ValueError("mask must be a contiguous (total,) tensor")
    for t, nm, dt in ((n_used, "n_used", torch.int32), (rms, "rms", torch.float32)):
        if t is not None:
            _need(t, nm, dt)
            if t.numel() < P or not t.is_contiguous():
                raise ValueError(f"{nm} must be a contiguous (P,) tensor")
    _check(load().aca_refit(_ptr(corr), _ptr(offsets), _ptr(mask), P, int(lm_iters), _ptr(H), _ptr(n_used),
                            _ptr(rms), _stream(stream, corr)))


def ransac_aca_adaptive_workspace_size(P: int, total_max_hyps: int) -> int:
    return int(load().ransac_aca_adaptive_workspace_size(int(P), int(total_max_hyps)))


def ransac_aca_adaptive(corr, offsets, max_hyp, total_max_hyps, params: RansacParams, confidence, best_H,
                        best_count, best_hyp, workspace, n_evaluated=None, hyp_counts=None, inlier_mask=None,
                        stream=None):
    """C ABI ransac_aca_adaptive: ransac_aca with the online stop at
    `confidence`; max_hyp (P,) int32 caps; n_evaluated (P,) int32."""
    _need(corr, "corr", torch.float32)
    _need(offsets, "offsets", torch.int64)
    _need(max_hyp, "max_hyp", torch.int32)
    _need(best_H, "best_H", torch.float32)
    _need(best_count, "best_count", torch.int32)
    _need(best_hyp, "best_hyp", torch.int32)
    _need(workspace, "workspace", torch.uint8)
    if corr.dim() != 2 or corr.shape[1] != 4 or not corr.is_contiguous():
        raise ValueError("corr must be a contiguous (total, 4) tensor")
    P = max_hyp.numel()
    if offsets.numel() != P + 1:
        raise ValueError("offsets must have P+1 entries")
    for t, nm in ((offsets, "offsets"), (max_hyp, "max_hyp"), (best_H, "best_H"), (best_count, "best_count"),
                  (best_hyp, "best_hyp")):
        if not t.is_contiguous():
            raise ValueError(f"{nm} must be contiguous")
    if best_H.numel() < 9 * P or best_count.numel() < P or best_hyp.numel() < P:
        raise ValueError("output tensors too small")
    if n_evaluated is not None:
        _need(n_evaluated, "n_evaluated", torch.int32)
        if n_evaluated.numel() < P:
            raise ValueError("n_evaluated too small")
    if hyp_counts is not None:
        _need(hyp_counts, "hyp_counts", torch.int32)
        if hyp_counts.numel() < total_max_hyps:
            raise ValueError("hyp_counts too small")
    if inlier_mask is not None:
        _need(inlier_mask, "inlier_mask", torch.uint8)
        if inlier_mask.numel() < corr.shape[0]:
            raise ValueError("inlier_mask too small")
    _check(load().ransac_aca_adaptive(_ptr(corr), _ptr(offsets), _ptr(max_hyp), P, int(total_max_hyps),
                                      ctypes.byref(params), float(confidence), _ptr(best_H), _ptr(best_count),
                                      _ptr(best_hyp), _ptr(n_evaluated), _ptr(hyp_counts), _ptr(inlier_mask),
                                      _ptr(workspace), workspace.numel(), _stream(stream, corr)))


def fma_probe(sink, packed: bool, blocks: int, threads: int, steps: int, stream=None) -> int:
    """One launch of the FP32 FMA throughput probe (aca_fma_probe); returns its
    FLOPs.  sink: float32 CUDA tensor of at least blocks * threads elements."""
    _need(sink, "sink", torch.float32)
    if sink.numel() < blocks * threads:
        raise ValueError("fma_probe: sink holds fewer than blocks * threads floats")
    L = _L()
    _check(L.aca_fma_probe(int(bool(packed)), blocks, threads, steps, sink.data_ptr(), _stream(stream, sink)))
    return int(L.aca_fma_probe_flops(int(bool(packed)), blocks, threads, steps))
