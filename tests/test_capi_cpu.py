"""The C-ABI library builds, loads and exports every entry point declared in
include/aca.h; argument validation happens on the host before any launch
(checked here without a GPU: only calls that are rejected up front)."""
import ctypes
import os
import re

import pytest

from paper_2402_18008_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "aca.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                                 src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("aca_solve", "sks_solve", "ransac_aca", "aca_backward", "ransac_aca_workspace_size",
                 "aca_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = _lib.load()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert set(declared_functions()) == set(_lib.EXPORTED)
    assert L.aca_version().startswith(b"aca-gb300")


def test_workspace_size_is_host_only_and_monotone():
    ws = _lib.ransac_aca_workspace_size
    assert ws(1, 4096) >= 4 * 4096
    assert ws(512, 700000) > ws(512, 1000) > ws(9, 1000)
    # at most 8 problems: four count slots per hypothesis (one per point
    # range of the one-launch path)
    assert ws(8, 1000) - ws(8, 0) >= 4 * 4 * 1000 > ws(9, 1000) - ws(9, 0)
    assert ws(-1, 10) == 0 and ws(4, -1) == 0
    assert ws(1, 0) % 256 == 0


def _call(name, *args):
    L = _lib.load()
    st = getattr(L, name)(*args)
    return st, L.aca_last_error().decode()


@pytest.mark.parametrize("name", ["aca_solve", "sks_solve"])
def test_solve_rejects_bad_sizes_before_launch(name):
    st, msg = _call(name, None, None, None, -1, 10, 0, None)
    assert st == -1 and "n <= ld" in msg
    st, msg = _call(name, None, None, None, 11, 10, 0, None)
    assert st == -1
    st, msg = _call(name, None, None, None, 4, 4, 7, None)
    assert st == -1 and "norm" in msg
    st, msg = _call(name, None, None, None, 4, 4, 0, None)
    assert st == -1 and "null" in msg
    st, _ = _call(name, None, None, None, 0, 0, 0, None)   # n = 0: nothing to do
    assert st == 0


def test_rect_and_backward_reject_bad_arguments():
    f = ctypes.c_float
    assert _call("aca_rect_solve", None, f(0), f(0), f(-1), f(1), None, 4, 4, None)[0] == -1
    assert _call("aca_rect_solve", None, f(0), f(0), f(1), f(1), None, 4, 4, None)[0] == -1
    assert _call("aca_backward", None, None, None, 5, 4, None)[0] == -1
    assert _call("aca_backward", None, None, None, 4, 4, None)[0] == -1
    assert _call("aca_rect_backward", None, f(0), f(0), f(1), f(0), None, None, 4, 4, None)[0] == -1
    assert _call("aca_sample_indices", 3, 10, 0, 0, None, None)[0] == -1
    assert _call("aca_sample_indices", 10, -1, 0, 0, None, None)[0] == -1


def test_ransac_rejects_bad_arguments():
    L = _lib.load()
    p = _lib.RansacParams(threshold_px=3.0, seed=1)
    buf = (ctypes.c_uint8 * 8192)()
    base = ctypes.addressof(buf)
    aligned = ctypes.c_void_p((base + 255) & ~255)
    misaligned = ctypes.c_void_p(((base + 255) & ~255) + 16)
    one = ctypes.c_void_p(((base + 255) & ~255) + 4096)

    def call(P, params, ws, nbytes, corr=one):
        return L.ransac_aca(corr, one, one, P, ctypes.byref(params) if params else None, one, one, one, None,
                            None, ws, nbytes, None)
    assert call(-1, p, aligned, 4096) == -1
    assert call(0, p, aligned, 4096) == 0                  # nothing to do
    assert call(1, None, aligned, 4096) == -1              # null params
    assert call(1, p, misaligned, 4096) == -1              # workspace alignment
    assert call(1, p, aligned, 16) == -3                   # workspace too small
    assert call(1, p, aligned, 4096, corr=ctypes.c_void_p(((base + 255) & ~255) + 4)) == -1
    for bad in (dict(threshold_px=0.0), dict(block_warps=17), dict(hyps_per_thread=3), dict(tile_points=48),
                dict(tile_points=16384), dict(block_warps=1, hyps_per_thread=2)):
        q = _lib.RansacParams(threshold_px=3.0, seed=1)
        for k, v in bad.items():
            setattr(q, k, v)
        assert call(1, q, aligned, 4096) == -1, bad


def test_adaptive_ransac_rejects_bad_arguments():
    L = _lib.load()
    p = _lib.RansacParams(threshold_px=3.0, seed=1)
    need = _lib.ransac_aca_adaptive_workspace_size(1, 64)
    assert need > _lib.ransac_aca_workspace_size(9, 64)
    assert _lib.ransac_aca_adaptive_workspace_size(512, 8388608) > _lib.ransac_aca_adaptive_workspace_size(512, 1000)
    assert _lib.ransac_aca_adaptive_workspace_size(-1, 5) == 0
    buf = (ctypes.c_uint8 * (need + 512))()
    base = (ctypes.addressof(buf) + 255) & ~255
    ws, one = ctypes.c_void_p(base), ctypes.c_void_p(base + 256)

    def call(P, conf, nbytes, params=p, total=64):
        return L.ransac_aca_adaptive(one, one, one, P, total, ctypes.byref(params), conf, one, one, one, None, None,
                                     None, ws, nbytes, None)
    assert call(-1, 0.99, need) == -1
    assert call(0, 0.99, need) == 0                        # nothing to do
    for conf in (0.0, 1.0, -0.1, float("nan")):
        assert call(1, conf, need) == -1, conf
    assert call(1, 0.99, need - 256) == -3                 # workspace smaller than the layout
    assert call(1, 0.99, need, total=-1) == -1
    q = _lib.RansacParams(threshold_px=3.0, seed=1, hyps_per_thread=3)
    assert call(1, 0.99, need, params=q) == -1


def test_refit_and_affine_reject_bad_arguments():
    buf = (ctypes.c_uint8 * 1024)()
    a = (ctypes.addressof(buf) + 255) & ~255
    good, odd = ctypes.c_void_p(a), ctypes.c_void_p(a + 4)
    assert _call("aca_refit", good, good, None, -1, 10, good, None, None, None)[0] == -1
    assert _call("aca_refit", good, good, None, 0, 10, good, None, None, None)[0] == 0      # P = 0
    assert _call("aca_refit", good, good, None, 1, -1, good, None, None, None)[0] == -1
    assert _call("aca_refit", good, good, None, 1, 10001, good, None, None, None)[0] == -1
    assert _call("aca_refit", None, good, None, 1, 10, good, None, None, None)[0] == -1
    st, msg = _call("aca_refit", odd, good, None, 1, 10, good, None, None, None)
    assert st == -1 and "aligned" in msg
    assert _call("aca_affine_solve", None, None, 5, 4, 0, None)[0] == -1
    assert _call("aca_affine_solve", None, None, 4, 4, 9, None)[0] == -1
    assert _call("aca_affine_solve", None, None, 0, 0, 0, None)[0] == 0


def test_fma_probe_rejects_bad_arguments_before_launch():
    L = _lib.load()
    assert L.aca_fma_probe(0, 0, 256, 4096, None, None) == -1
    assert L.aca_fma_probe(1, 4, 100, 4096, None, None) == -1
    assert L.aca_fma_probe(1, 4, 256, 4095, None, None) == -1
    assert b"steps" in L.aca_last_error()
    assert L.aca_fma_probe(1, 4, 256, 4096, None, None) == -1     # null sink
    assert L.aca_fma_probe_flops(1, 608, 256, 4096) == 608 * 256 * 4096 * 8 * 2 * 2


def test_binding_leading_dimension_rules():
    # the plane bindings' shared leading-dimension check (host logic only)
    assert _lib._shared_ld((5, 8), (8, 8), (0, 8)) == 8
    with pytest.raises(ValueError, match="one leading dimension"):
        _lib._shared_ld((5, 8), (5, 12))
    with pytest.raises(ValueError, match="exceeds the leading dimension"):
        _lib._shared_ld((9, 8), (5, 8))
