"""The overlapped split pass (cluster_options.overlap = 1; problems of at least
2^20 rows with the internal numbering): the update of each of 8 row chunks runs on a
second stream as soon as the gather has produced that chunk's rows, beside the
gather of the next chunks.  The update blocks, their row ranges and partial slots
are those of the plain schedule, so both schedules agree bit for bit, through the
captured graphs and the profiled launches alike; a batch holding such an instance
equals it solo."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2506_04045_b300")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.load()


def _solve(rp, c, v, U0, graph_iters, profiled_iters, **kw):
    s = pkg.Solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=graph_iters + profiled_iters, **kw)
    s.step(graph_iters)
    kt = s.enqueue_profiled(profiled_iters)
    rep = s.report()
    U = s.get_U()
    s.close()
    return U, rep, kt


# n just above 2^20 with a ragged last tile; the tcgen05 update (k = 32), the warp
# update (k = 64) and a small k
@pytest.mark.parametrize("k,precision", [(32, 0), (32, 1), (64, 0), (8, 1)])
def test_overlapped_pass_equals_plain_pass_bitwise(k, precision):
    spec = synth.GraphSpec("dcsbm", 1_100_011, k, 500 + k, mean_deg=16.0)
    rp, c, v = synth.make_graph(spec, device="cuda")
    U0 = synth.dirichlet_u0(spec.n, k, 500 + k, device="cuda")
    # the overlapped pass cuts the per-block update (engine 2) into chunks; the
    # plain pass of the same engine is its reference
    Uo, ro, kto = _solve(rp, c, v, U0, 10, 3, precision=precision, overlap=1, update_engine=2)
    Up, rp_, ktp = _solve(rp, c, v, U0, 10, 3, precision=precision, overlap=0, update_engine=2)
    assert ro["iters"] == rp_["iters"] == 13
    assert torch.equal(Uo, Up)
    assert ro["f"] == rp_["f"] and ro["pg_norm"] == rp_["pg_norm"] and ro["trace_SU"] == rp_["trace_SU"]
    # the overlapped schedule launches one gather and one update per chunk
    assert kto["kernels"] > ktp["kernels"]
    assert np.isfinite(ro["f"])


def test_batch_holding_an_overlapped_instance_equals_it_solo():
    specs = [synth.GraphSpec("dcsbm", 1_050_001, 32, 521, mean_deg=12.0),
             synth.GraphSpec("dcsbm", 3000, 16, 522, mean_deg=20.0)]
    inst = []
    for sp in specs:
        rp, c, v = synth.make_graph(sp)
        U0 = synth.dirichlet_u0(sp.n, sp.k, sp.seed)
        inst.append(tuple(t.cuda().contiguous() for t in (rp, c, v, U0)))
    b = pkg.Batch(inst, stop_rule=pkg.STOP_NONE, max_iter=12)
    b.step(12)
    for i, (rp, c, v, U0) in enumerate(inst):
        # a batch runs the per-block update (engine 2), also for instances of
        # at least 2^17 articles that stream when alone
        s = pkg.Solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=12, update_engine=2)
        s.step(12)
        assert torch.equal(b.get_U(i), s.get_U()), i
        s.close()
    b.close()
