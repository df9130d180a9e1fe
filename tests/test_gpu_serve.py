"""a9: the continuous-batching server on a short Poisson stream.

Every served result must equal the same request closed alone (int32 bit-exact; float32 within
1e-5 relative, in fact identical because the plan depends only on the request), a sample must
match the oracle, the arena must never exceed its budget, and both kinds of launch (batched and
solo) must occur."""
import pytest
import torch

import oracle
import workloads
from test_gpu_parity import assert_dist_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def apsp():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2310_03983_gb300 as m
    return m


def test_server_results_equal_alone_and_in_the_mix(apsp):
    from paper_2310_03983_gb300 import serve
    ns, ps, lib = workloads.request_library(24, n_lo=48, n_hi=1500, seed=3)
    t, _, _, _ = workloads.poisson_requests(rate=150.0, duration=0.8, seed=1)
    from paper_2310_03983_gb300 import planner
    model = planner.CostModel.load(planner.DEFAULT_MODEL)
    reqs = serve.make_requests(t, lib, density=list(ps))
    srv = serve.Server(arena_bytes=256 << 20, small_max=512, slots=4, keep_results=True, planner=model)
    st = srv.serve(reqs)
    assert st["requests"] == len(reqs) > 50
    assert st["launches"]["batch"] > 0 and st["launches"]["solo"] > 0
    assert st["arena_peak_bytes"] <= st["arena_bytes"]
    assert st["p50"] <= st["p99"]
    for r in reqs:
        alone = torch.from_numpy(lib[r.rid % len(lib)]).cuda()
        algo, param = r.plan
        if algo == "batched":
            apsp.apsp_close_cta(alone)
        else:  # the cost model's plan, run alone
            planner.run_config(alone, algo, param)
        assert_dist_equal(r.result.numpy(), alone.cpu().numpy(), f"request {r.rid} n={r.n}")
    for g in (0, 1, 5):  # and the oracle, on a few distinct graphs
        r = next(r for r in reqs if r.rid % len(lib) == g)
        assert_dist_equal(r.result.numpy(), oracle.fw(lib[g]), f"oracle graph {g}")
    base = serve.serve_one_at_a_time(serve.make_requests(t, lib))
    assert base["requests"] == len(reqs)
    print({"server": {k: st[k] for k in ("p50", "p99", "graphs_per_s")},
           "one_at_a_time": {k: base[k] for k in ("p50", "p99", "graphs_per_s")}})
