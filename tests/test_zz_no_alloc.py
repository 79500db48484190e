"""cluster_objective_static: the objective for callers that may not allocate.

Some callers cannot call cudaMalloc when they need the objective (a service
whose pool allocator owns all free device memory, or a latency-critical loop
where cudaMalloc/cudaFree would synchronise the device).  The allocation-free
entry point keeps its scratch in a fixed array inside the library; here it is
checked against the allocating cluster_objective on two calls in a row with
different inputs (the shared scratch must not carry state from one call into
the next) for every k it accepts, against the FP64 oracle on a graph with a
row adjacent to every article, and its size limits are checked to fail with
EINVAL.  The file is
named so that pytest collects it last.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2506_04045_b300")

TOL_F = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.load()


@pytest.mark.parametrize("k", [2, 4, 8, 16, 32])
def test_static_objective_matches_allocating_entry_point_twice(k):
    spec = synth.GraphSpec("dcsbm", 30001, k, 90 + k, mean_deg=25.0, blocks=max(k, 2))
    rp, c, v = [t.cuda() for t in synth.make_graph(spec)]
    for call in range(2):
        U = synth.dirichlet_u0(spec.n, k, 1000 + 17 * call + k).cuda()
        f_ref = pkg.objective(rp, c, v, U)
        f = pkg.objective_static(rp, c, v, U)
        assert abs(f - f_ref) <= TOL_F * abs(f_ref), (call, f, f_ref)


@pytest.mark.parametrize("k", [8, 32])
def test_static_objective_with_a_hub_row_matches_oracle(k):
    # the static path splits rows evenly (no chunking of high-degree rows): a
    # row adjacent to every article lands whole in one block
    n = 6000
    rng = np.random.default_rng(5 + k)
    src = np.concatenate([np.zeros(n - 1, np.int64), rng.integers(0, n, 40000)])
    dst = np.concatenate([np.arange(1, n, dtype=np.int64), rng.integers(0, n, 40000)])
    w = (1.0 - rng.random(src.size)).astype(np.float32)
    rp, c, v = oracle.csr_from_edges(n, src, dst, w)
    S = sp.csr_matrix((v.astype(np.float64), c, rp), shape=(n, n))
    g = [torch.from_numpy(x).cuda() for x in (rp, c, v)]
    for call in range(2):
        U = synth.dirichlet_u0(n, k, 300 + call)
        f_ref = oracle.objective_trace(S, U.numpy().astype(np.float64))
        f = pkg.objective_static(*g, U.cuda())
        assert abs(f - f_ref) <= TOL_F * f_ref, (call, f, f_ref)
        assert abs(f - pkg.objective(*g, U.cuda())) <= TOL_F * f_ref


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


def test_static_objective_refuses_a_capturing_stream():
    # it synchronises its stream and reads partials on the host: on a stream
    # under capture it returns EINVAL before enqueuing anything, and the
    # capture itself stays valid
    spec = synth.GraphSpec("dcsbm", 2000, 4, 8, mean_deg=10.0)
    rp, c, v = [t.cuda() for t in synth.make_graph(spec)]
    U4 = synth.dirichlet_u0(spec.n, 4, 8).cuda()
    f0 = pkg.objective_static(rp, c, v, U4)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        with pytest.raises(pkg.ClusterError) as ei:
            pkg.objective_static(rp, c, v, U4, stream=s)
        U4.add_(0.0)   # the capture still records work
    assert ei.value.status == pkg.EINVAL and "captured" in str(ei.value)
    g.replay()
    torch.cuda.synchronize()
    assert pkg.objective_static(rp, c, v, U4) == f0
