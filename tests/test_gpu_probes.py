"""The fp32 slab probes (apsp_probe_minplus variants 9-11): the tropical-GEMM engine's fp32 slab
arithmetic timed in isolation, by the SM clock, on every SM.  They separate what the engine's
fp32 instruction sequence costs from what feeding it costs: the same packed adds and 3-input
mins run on operands read from shared memory (9), on operands held in registers (10), and in
registers beside other work on the ALU pipe (11).  Prints the rates (pairs per SM clock) and
checks that each run completed and that the measured ordering holds."""
import json

import pytest
import torch

pytestmark = pytest.mark.gpu

PAIRS_PER_SLAB = 128 * 128 * 32
ISSUE_BOUND = 128.0  # pairs per SM clock: one issued instruction per pair, 128 lanes


@pytest.fixture(scope="module")
def apsp():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2310_03983_gb300 as m
    return m


def _slab_rate(apsp, variant, iters=2000):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    sink = torch.zeros(sms * 256, dtype=torch.int32, device="cuda")
    apsp.apsp_probe_minplus(variant, sms, 256, iters // 4, sink)  # warm-up
    apsp.apsp_probe_minplus(variant, sms, 256, iters, sink)
    torch.cuda.synchronize()
    clocks = sink.view(sms, 256)[:, 0].to(torch.int64) * 1024  # per block, thread 0's report
    assert int(clocks.min()) > 0
    return iters * PAIRS_PER_SLAB / float(clocks.max())


def test_fp32_slab_probes(apsp):
    rates = {v: _slab_rate(apsp, v) for v in (9, 10, 11)}
    print(json.dumps({"pairs_per_sm_clock": {
        "9 operands from shared memory (the engine's loop)": round(rates[9], 1),
        "10 operands in registers": round(rates[10], 1),
        "11 registers, one ALU-pipe XOR per 16 pairs": round(rates[11], 1)}}))
    for v, r in rates.items():
        assert 0.0 < r <= ISSUE_BOUND * 1.01, (v, r)
    # feeding the operands from shared memory costs throughput, and so does ALU-pipe work
    # beside the 3-input mins
    assert rates[9] < rates[10]
    assert rates[11] < rates[10]
    assert apsp.apsp_device_status() == 0
