"""The streaming row-local update (17 <= k <= 32: one CTA per SM over
128-row tiles loaded by TMA, y G(Y) as 3xTF32 and the Gram matrices as
scaled float16 splits on tcgen05) against the FP64 oracle: tiny and ragged
sizes (one partial tile, one row past a tile, one CTA with a single
warpgroup busy), k across the kernel's range, both precisions; reruns and
checkpoint resumes bit-identical; engine 0 chooses it from 2^17 articles; a
bounded wait that gives up ends the run with CLUSTER_ETIMEOUT and leaves the
context and the device usable."""
import time

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import maxabs, to_scipy

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2506_04045_b300")

STREAM = 3   # update_engine: the streaming update at any size


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.load()


def _run(rp, c, v, U0, iters, **kw):
    s = pkg.Solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=iters, **kw)
    rep = s.step(iters)
    U = s.get_U()
    s.close()
    return U, rep


def _oracle(rp, c, v, U0, iters):
    S = to_scipy(rp, c, v, U0.shape[0])
    o = oracle.fista(S, U0.cpu().numpy().astype(np.float64), 1.0 / oracle.lipschitz(S), max_iter=iters, stop="none")
    return S, o


# n = 5: one partial tile; 129: one row past a tile; 300: three tiles on three
# CTAs (the second warpgroup idle); 1000, 131149: many tiles, ragged last one
@pytest.mark.parametrize("n", [5, 129, 300, 1000, 131149])
def test_stream_update_matches_oracle(n):
    spec = synth.GraphSpec("dcsbm", n, 32, 500 + n, mean_deg=min(20.0, n / 2.0))
    rp, c, v = synth.make_graph(spec, device="cuda")
    U0 = synth.dirichlet_u0(n, 32, 500 + n, device="cuda")
    U, rep = _run(rp, c, v, U0, 30, update_engine=STREAM)
    assert rep["iters"] == 30 and rep["status"] == pkg.EMAXITER
    _, o = _oracle(rp, c, v, U0, 30)
    assert maxabs(U.cpu().numpy(), o.U) <= 1e-5
    # the loss terms are float32 sums of terms of size ||S||^2 (f can be far smaller)
    s2 = float((v.double() ** 2).sum())
    fo = o.losses[rep["f_iter"]]
    assert abs(rep["f"] - fo) <= 1e-6 * max(abs(fo), s2), (rep["f"], fo)
    assert abs(rep["pg_norm"] - o.pg_norms[-1]) <= 1e-4 * o.pg_norms[-1]


@pytest.mark.parametrize("k", [17, 24, 32])
@pytest.mark.parametrize("precision", [0, 1])
def test_stream_update_k_and_precision(k, precision):
    spec = synth.GraphSpec("dcsbm", 30011, k, 520 + k, mean_deg=25.0)
    rp, c, v = synth.make_graph(spec, device="cuda")
    U0 = synth.dirichlet_u0(spec.n, k, 520 + k, device="cuda")
    U, rep = _run(rp, c, v, U0, 50, update_engine=STREAM, precision=precision)
    _, o = _oracle(rp, c, v, U0, 50)
    assert maxabs(U.cpu().numpy(), o.U) <= (1e-5 if precision == 0 else 1e-4)
    f_ref = oracle.objective_trace(to_scipy(rp, c, v, spec.n), o.U)
    s = pkg.Solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=50, update_engine=STREAM, precision=precision)
    rep = s.solve()
    s.close()
    assert abs(rep["f"] - f_ref) <= (1e-6 if precision == 0 else 1e-5) * f_ref
    # the per-block tcgen05 form computes the same iteration (other Gram arithmetic)
    Ub, _ = _run(rp, c, v, U0, 50, update_engine=2, precision=precision)
    assert maxabs(U.cpu().numpy(), Ub.cpu().numpy()) <= 1e-5


# rows on faces of the simplex: most features of the start point are exactly
# zero, and after 20 steps more than half of the rows still have a zero
# feature, so the projection's active-set iteration runs for them (rows whose
# features all exceed the first threshold skip it); k = 32 takes the
# full-width kernel, k = 24 the padded one
@pytest.mark.parametrize("k", [24, 32])
def test_stream_update_projection_on_faces(k):
    n = 3000
    spec = synth.GraphSpec("dcsbm", n, k, 77 + k, mean_deg=20.0)
    rp, c, v = synth.make_graph(spec, device="cuda")
    U0 = synth.dirichlet_u0(n, k, 78 + k)
    keep = (torch.arange(n * k).view(n, k) * 2654435761 % 97) < 12   # about 1 feature in 8
    keep[:, 0] = True
    U0 = U0 * keep
    U0 = (U0 / U0.sum(dim=1, keepdim=True)).to(torch.float32).cuda()
    U, _ = _run(rp, c, v, U0, 20, update_engine=STREAM)
    _, o = _oracle(rp, c, v, U0, 20)
    assert (o.U == 0.0).mean() > 0.02                      # the faces are reached
    assert ((o.U > 0.0).sum(axis=1) < k).mean() > 0.4
    assert maxabs(U.cpu().numpy(), o.U) <= 1e-5


def test_stream_update_reruns_and_resume_are_bit_identical():
    spec = synth.GraphSpec("dcsbm", 40000, 32, 541, mean_deg=25.0)
    rp, c, v = synth.make_graph(spec, device="cuda")
    U0 = synth.dirichlet_u0(spec.n, 32, 541, device="cuda")
    a = pkg.Solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=40, update_engine=STREAM)
    a.step(13)
    state = a.get_state()
    ra = a.step(27)
    Ua = a.get_U()
    a.close()
    Ub, rb = _run(rp, c, v, U0, 40, update_engine=STREAM)
    assert torch.equal(Ua, Ub) and ra["f"] == rb["f"] and ra["pg_norm"] == rb["pg_norm"]
    b = pkg.Solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=40, update_engine=STREAM)
    b.set_state(state)
    rc = b.step(27)
    assert rc["iters"] == 40 and torch.equal(b.get_U(), Ua)
    b.close()


def test_engine_zero_streams_from_two_to_the_seventeen_articles():
    n = (1 << 17) + 5
    spec = synth.GraphSpec("dcsbm", n, 32, 551, mean_deg=20.0)
    rp, c, v = synth.make_graph(spec, device="cuda")
    U0 = synth.dirichlet_u0(n, 32, 551, device="cuda")
    U0_, r0 = _run(rp, c, v, U0, 12, update_engine=0)
    U3, r3 = _run(rp, c, v, U0, 12, update_engine=STREAM)
    assert torch.equal(U0_, U3) and r0["f"] == r3["f"]


def test_stream_wait_that_gives_up_is_a_status_and_the_context_survives():
    spec = synth.GraphSpec("dcsbm", 20000, 32, 561, mean_deg=20.0)
    rp, c, v = synth.make_graph(spec, device="cuda")
    U0 = synth.dirichlet_u0(spec.n, 32, 561, device="cuda")
    s = pkg.Solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=50, update_engine=STREAM)
    s.step(3)
    U3 = s.get_U().clone()
    s.test_hooks(1)
    t0 = time.time()
    rep = s.step(5)
    dt = time.time() - t0
    assert rep["status"] == pkg.ETIMEOUT and rep["done"] == 1 and rep["out_iter"] == 3
    assert dt < 60
    assert torch.equal(s.get_U(), U3)
    s.test_hooks(0)
    s.close()
    s2 = pkg.Solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=50, update_engine=STREAM)
    s2.step(3)
    assert torch.equal(s2.get_U(), U3)
    s2.close()
