"""The FMA throughput microbenchmark behind the ALU rooflines (FP64 for the integrator, FP32 for the
mixed-precision form): its launches do the work they claim -- time grows in proportion to the FMA count --
and the measured rates stay below what the SM count and the observed clock allow."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def _time(ck, prec, dt, blocks, threads, iters):
    sink = torch.zeros(blocks * threads, dtype=dt, device="cuda")
    st = torch.cuda.current_stream()
    ck.cloak_fma_peak(prec, blocks, threads, 16, sink)  # warm-up
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    flops = ck.cloak_fma_peak(prec, blocks, threads, iters, sink)
    b.record(st)
    b.synchronize()
    assert not torch.any(sink != 0)  # the chains never satisfy the store condition
    return flops, a.elapsed_time(b) / 1e3


@pytest.mark.parametrize("fp64", [True, False])
def test_fma_peak_scales_and_stays_below_the_issue_limit(fp64):
    from paper_1209_6038_gb300 import cloak as ck
    ck.load()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    prec, dt = (ck.FP64, torch.float64) if fp64 else (ck.MIXED, torch.float32)
    iters = 2000 if fp64 else 40000
    f1, t1 = _time(ck, prec, dt, 8 * sms, 256, iters)
    f2, t2 = _time(ck, prec, dt, 8 * sms, 256, 2 * iters)
    assert f2 == pytest.approx(2 * f1)
    assert t2 / t1 == pytest.approx(2.0, rel=0.15)
    # an SM issues at most 128 FP32 lanes per clock (256 flop); FP64 runs far below that on this part;
    # 2.2 GHz is above the part's highest SM clock (2070 MHz)
    limit = sms * 256 * 2.2e9 / 1e12
    rate = f2 / t2 / 1e12
    assert 0 < rate < 1.05 * limit
