"""cluster_objective_static: the objective for callers that may not allocate.

Some callers cannot call cudaMalloc when they need the objective (a service
whose pool allocator owns all free device memory, or a latency-critical loop
where cudaMalloc/cudaFree would synchronise the device).  The allocation-free
entry point keeps its scratch in a fixed array inside the library; here it is
checked against the allocating cluster_objective on two calls in a row with
different inputs (the shared scratch must not carry state from one call into
the next), and its size limits are checked to fail with EINVAL.  The file is
named so that pytest collects it last.
"""
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2506_04045_b300")

TOL_F = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.load()


@pytest.mark.parametrize("k", [32, 8])
def test_static_objective_matches_allocating_entry_point_twice(k):
    spec = synth.GraphSpec("dcsbm", 30001, k, 90 + k, mean_deg=25.0)
    rp, c, v = [t.cuda() for t in synth.make_graph(spec)]
    for call in range(2):
        U = synth.dirichlet_u0(spec.n, k, 1000 + 17 * call + k).cuda()
        f_ref = pkg.objective(rp, c, v, U)
        f = pkg.objective_static(rp, c, v, U)
        assert abs(f - f_ref) <= TOL_F * abs(f_ref), (call, f, f_ref)


def test_static_objective_rejects_what_it_cannot_do_without_memory():
    spec = synth.GraphSpec("dcsbm", 2000, 4, 7, mean_deg=10.0)
    rp, c, v = [t.cuda() for t in synth.make_graph(spec)]
    U3 = synth.dirichlet_u0(spec.n, 3, 7).cuda()
    with pytest.raises(pkg.ClusterError) as ei:
        pkg.objective_static(rp, c, v, U3)                   # k = 3 would need a padded copy
    assert ei.value.status == pkg.EINVAL and "k must be" in str(ei.value)
    U4 = synth.dirichlet_u0(spec.n, 4, 7).cuda()
    with pytest.raises(pkg.ClusterError) as ei:
        pkg.objective_static(rp.to(torch.int32), c, v, U4)   # int32 row pointers would need widening
    assert ei.value.status == pkg.EINVAL and "int64" in str(ei.value)
    f = pkg.objective_static(rp, c, v, U4)
    assert abs(f - pkg.objective(rp, c, v, U4)) <= TOL_F * abs(f)
