"""Parity at the benchmark's own size: n = 70,000,000 articles, k = 32, about
2e9 nonzeros (the power-law citation-like graph and start point bench.py
times, in the same launch configuration).  The float64 state of the whole
problem does not fit a host, so the oracle is asked only what it can answer
from pieces: one Algorithm-4 step at about 2,000 sampled articles and the 50
highest-degree ones, from the GPU's own two previous iterates (their rows and
their neighbours' rows, with X^T X of the extrapolated point summed over row
blocks), and ||Xbar^T Xbar||_F^2 of the iterate whose loss the solver
reported, summed over row blocks in float64."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
import synth
from gpu_helpers import maxabs

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2506_04045_b300")

N, K, SEED, DEG = 70_000_000, 32, 2, 28.9
CHUNK = 1 << 21


@pytest.fixture(scope="module")
def graph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.load()
    spec = synth.GraphSpec("dcsbm", N, K, SEED, mean_deg=DEG)
    rp, c, v = synth.make_graph(spec, device="cuda")
    U0 = synth.dirichlet_u0(N, K, SEED, device="cuda")
    torch.cuda.synchronize()
    yield rp, c, v, U0
    del rp, c, v, U0
    torch.cuda.empty_cache()


def _blocks(X, Xp=None):
    """Consecutive row blocks of a device matrix on the host (pairs of blocks
    of X and Xp when Xp is given)."""
    for i in range(0, X.shape[0], CHUNK):
        if Xp is None:
            yield X[i:i + CHUNK].cpu().numpy()
        else:
            yield X[i:i + CHUNK].cpu().numpy(), Xp[i:i + CHUNK].cpu().numpy()


def _local_rows(rp, c, v, rows):
    """The rows of S at `rows`, with columns renumbered into `keep` (the rows
    and all their neighbours): a small host CSR for the oracle's step."""
    rpc = rp.cpu()
    r = torch.from_numpy(rows)
    lo, hi = rpc[r].numpy(), rpc[r + 1].numpy()
    idx = torch.from_numpy(np.concatenate([np.arange(a, b) for a, b in zip(lo, hi)])).cuda()
    cols = c[idx].cpu().numpy().astype(np.int64)
    vals = v[idx].cpu().numpy().astype(np.float64)
    keep = np.unique(np.concatenate([rows, cols]))
    pos = np.searchsorted(keep, rows)
    r_loc = np.repeat(pos, hi - lo)
    c_loc = np.searchsorted(keep, cols)
    S_loc = sp.csr_matrix((vals, (r_loc, c_loc)), shape=(keep.size, keep.size))
    return S_loc, keep, pos


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "mixed"])
def test_benchmark_scale_sampled_step_and_gram(graph, prec):
    rp, c, v, U0 = graph
    s = pkg.Solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=100, borrow=1, precision=prec)
    m = 8
    s.step(m - 2)
    X2 = s.get_U()
    s.step(1)
    X1 = s.get_U()
    rep = s.step(1)
    X0 = s.get_U()
    s.close()
    # step size: L = 4 ||S||_F + 12 n (Sect. 5), ||S||_F^2 summed over blocks
    S2 = sum(oracle.frob2(v[i:i + (1 << 26)].cpu().numpy()) for i in range(0, v.numel(), 1 << 26))
    tau = 1.0 / (4.0 * np.sqrt(S2) + 12.0 * N)
    assert abs(rep["tau"] - tau) <= 1e-12 * tau
    # ||Xbar^{m-1 T} Xbar^{m-1}||_F^2, the Gram term of the loss the last pass reported
    assert rep["f_iter"] == m - 1
    A = oracle.gram_blocks(_blocks(X1))
    gram2 = float((A * A).sum())
    err_g = abs(rep["gram_fro2"] - gram2) / gram2
    print(f"\nn=70M {'mixed' if prec else 'fp32'}: gram_fro2 rel err {err_g:.3e}")
    assert err_g <= 1e-6
    # one Algorithm-4 step at sampled articles from the GPU's Xbar^{m-1}, Xbar^{m-2}
    beta = oracle.momentum_factors(m)[m - 1]
    share = oracle.gram_blocks(_blocks(X1, X2), beta=beta)
    deg = rp[1:] - rp[:-1]
    hubs = torch.topk(deg, 50).indices.cpu().numpy()
    rng = np.random.default_rng(7)
    rows = np.unique(np.concatenate([rng.integers(0, N, 2000), hubs])).astype(np.int64)
    S_loc, keep, pos = _local_rows(rp, c, v, rows)
    kt = torch.from_numpy(keep).cuda()
    Xc = X1.index_select(0, kt).cpu().numpy()
    Xp = X2.index_select(0, kt).cpu().numpy()
    ref = oracle.fista_step_rows(S_loc, Xc, Xp, beta, tau, pos, share=share)
    got = X0.index_select(0, torch.from_numpy(rows).cuda()).cpu().numpy()
    err = maxabs(got, ref)
    print(f"n=70M {'mixed' if prec else 'fp32'}: sampled-step max-abs {err:.3e} over {rows.size} articles")
    assert err <= 1e-5
    del X0, X1, X2
    torch.cuda.empty_cache()
