"""The FP32 FMA throughput probe (aca_fma_probe), the measured denominator
stated beside the derived FP32 peak of the RANSAC scoring rooflines: every
chain converges to the fixed point of x -> 0.5 x + 0.25, and the measured
rate lies within a plausible range of SMs x 128 lanes x 2 x clock."""
import pytest
import torch

from paper_2402_18008_gb300 import _lib

pytestmark = pytest.mark.gpu


def _rate(packed, blocks, threads, steps):
    sink = torch.full((blocks * threads,), float("nan"), device="cuda")
    flops = _lib.fma_probe(sink, packed, blocks, threads, steps)
    torch.cuda.synchronize()
    return sink, flops


@pytest.mark.parametrize("packed", [False, True])
def test_probe_values_and_flop_count(packed):
    sink, flops = _rate(packed, 3, 64, 256)
    # 256 steps of x -> 0.5 x + 0.25 from starts below 1.1: every chain is
    # 0.5 to FP32 precision; the thread sums 8 (scalar) or 16 (packed) of them
    want = 4.0 if not packed else 8.0
    assert torch.allclose(sink, torch.full_like(sink, want), rtol=0, atol=1e-5)
    assert flops == 3 * 64 * 256 * 8 * 2 * (2 if packed else 1)


def test_probe_rate_is_plausible():
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    blocks, threads, steps = 4 * sms, 256, 4096
    sink = torch.empty(blocks * threads, device="cuda")
    for packed in (False, True):
        for _ in range(2):
            _lib.fma_probe(sink, packed, blocks, threads, steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        flops = sum(_lib.fma_probe(sink, packed, blocks, threads, steps) for _ in range(5))
        e1.record()
        torch.cuda.synchronize()
        tflops = flops / (e0.elapsed_time(e1) * 1e-3) / 1e12
        derived = sms * 128 * 2 * 2.07e9 / 1e12       # at the part's 2070 MHz maximum
        print("packed" if packed else "scalar", f"{tflops:.1f} TFLOP/s, derived peak {derived:.1f}")
        assert 0.3 * derived < tflops < 1.5 * derived
