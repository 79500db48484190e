"""Second-order check (Sect. 4, Theorem 4.1) through cluster_hessian_apply:
H[W], the curvature <W, H[W]> and the slope <grad f(U), W> against the FP64
oracle on the same seeded inputs, and the paper's worked value -4."""
import numpy as np
import pytest
import torch

import oracle
import synth
from conftest import read_sections
from gpu_helpers import to_scipy

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2506_04045_b300")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.load()


def _scale(S, U, W):
    """Sum of the magnitudes of the terms of <W, H[W]> and <grad f, W>: the
    float32 path's rounding is relative to these, not to the (cancelled) result."""
    U = U.astype(np.float64)
    W = W.astype(np.float64)
    G, M, N = U.T @ U, U.T @ W, W.T @ W
    SW = S @ W
    curv = 4 * (abs(np.sum(W * SW)) + abs(np.sum(N * G)) + np.sum(M * M) + abs(np.sum(M * M.T)))
    slope = 4 * (abs(np.sum(U * SW)) + abs(np.sum(M * G)))
    return curv, slope


def _tangent(rng, n, k):
    W = rng.standard_normal((n, k))
    return (W - W.mean(axis=1, keepdims=True)).astype(np.float32)   # rows sum to zero


def test_toy_saddle_curvature_is_minus_four():
    g = read_sections("toy7.txt")
    e = np.array([[int(a) - 1, int(b) - 1] for a, b in g["edges"]])
    rp, c, v = oracle.csr_from_edges(7, e[:, 0], e[:, 1])
    X3 = np.array([[float(x) for x in r] for r in g["scenario3"][2:4]])
    U = torch.from_numpy(X3.T.astype(np.float32)).cuda().contiguous()
    Vbar = np.array([[float(x) for x in r] for r in g["hessian"][0:2]]).T
    W = torch.from_numpy(Vbar.astype(np.float32)).cuda().contiguous()
    dev = [torch.from_numpy(t).cuda() for t in (rp, c, v)]
    HW, curv, slope = pkg.hessian_apply(*dev, U, W)
    S = to_scipy(*dev, 7)
    assert abs(curv - float(g["hessian"][2][1])) <= 1e-5
    assert abs(slope - float(g["hessian"][3][1])) <= 1e-5
    ref = oracle.hessian_apply_sparse(S, X3.T, Vbar)
    assert np.max(np.abs(HW.cpu().numpy() - ref)) <= 1e-5


@pytest.mark.parametrize("k", [2, 3, 8, 20, 32, 64, 128])
def test_hessian_matches_oracle(k):
    spec = synth.GraphSpec("dcsbm", 4000, min(k, 32), 700 + k, mean_deg=25.0)
    rp, c, v = synth.make_graph(spec, device="cuda")
    n = spec.n
    rng = np.random.default_rng(k)
    U = synth.dirichlet_u0(n, k, 11, device="cuda")
    W = torch.from_numpy(_tangent(rng, n, k)).cuda()
    HW, curv, slope = pkg.hessian_apply(rp, c, v, U, W)
    S = to_scipy(rp, c, v, n)
    Uh, Wh = U.cpu().numpy().astype(np.float64), W.cpu().numpy().astype(np.float64)
    ref = oracle.hessian_apply_sparse(S, Uh, Wh)
    assert np.max(np.abs(HW.cpu().numpy() - ref)) <= 1e-5 * np.max(np.abs(ref))
    cs, ss = _scale(S, Uh, Wh)
    assert abs(curv - oracle.curvature(S, Uh, Wh)) <= 1e-5 * cs
    assert abs(slope - oracle.slope(S, Uh, Wh)) <= 1e-5 * ss


def test_hessian_with_chunked_rows_and_no_output_matrix():
    # rows above the chunk threshold go through the chunked product; HW may be omitted
    spec = synth.GraphSpec("dcsbm", 30000, 32, 5, mean_deg=60.0)
    rp, c, v = synth.make_graph(spec, device="cuda")
    n, k = spec.n, 32
    deg = (rp[1:] - rp[:-1]).max().item()
    assert deg > 16384 // 32
    U = synth.dirichlet_u0(n, k, 3, device="cuda")
    W = torch.from_numpy(_tangent(np.random.default_rng(1), n, k)).cuda()
    HW, curv, slope = pkg.hessian_apply(rp, c, v, U, W)
    none, curv2, slope2 = pkg.hessian_apply(rp, c, v, U, W, want_hw=False)
    assert none is None and curv2 == curv and slope2 == slope
    S = to_scipy(rp, c, v, n)
    Uh, Wh = U.cpu().numpy().astype(np.float64), W.cpu().numpy().astype(np.float64)
    ref = oracle.hessian_apply_sparse(S, Uh, Wh)
    assert np.max(np.abs(HW.cpu().numpy() - ref)) <= 1e-5 * np.max(np.abs(ref))
    cs, ss = _scale(S, Uh, Wh)
    assert abs(curv - oracle.curvature(S, Uh, Wh)) <= 1e-5 * cs
    assert abs(slope - oracle.slope(S, Uh, Wh)) <= 1e-5 * ss


def test_hessian_argument_errors():
    rp = torch.zeros(2, dtype=torch.int64, device="cuda")
    c = torch.zeros(0, dtype=torch.int32, device="cuda")
    v = torch.zeros(0, dtype=torch.float32, device="cuda")
    U = torch.ones(1, 129, device="cuda")
    with pytest.raises(pkg.ClusterError) as ei:
        pkg.hessian_apply(rp, c, v, U, U)
    assert ei.value.status == pkg.EINVAL
