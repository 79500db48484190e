"""The row-local update on the fifth-generation tensor cores (tcgen05.mma,
accumulators in tensor memory; k in 17..64) against the warp-level mma.sync
update: both compute the same 3xTF32 products in the same order, so every bit
of the iterates, losses and norms agrees.  Also the bounded-wait path: a wait
that gives up ends the run with CLUSTER_ETIMEOUT and leaves the context usable."""
import time

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import maxabs, to_scipy

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2506_04045_b300")


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


# n = 30011: 938 full tiles of 32 rows and a ragged one; k spans the kernel's range
@pytest.mark.parametrize("k", [17, 24, 32])
@pytest.mark.parametrize("precision", [0, 1])
def test_tcgen05_update_equals_warp_update_bitwise(k, precision):
    spec = synth.GraphSpec("dcsbm", 30011, k, 70 + k, mean_deg=25.0)
    rp, c, v = synth.make_graph(spec, device="cuda")
    U0 = synth.dirichlet_u0(spec.n, k, 70 + k, device="cuda")
    Ut, rt = _run(rp, c, v, U0, 25, precision=precision, update_engine=2)
    Uw, rw = _run(rp, c, v, U0, 25, precision=precision, update_engine=1)
    assert rt["iters"] == rw["iters"] == 25
    assert torch.equal(Ut, Uw)
    assert rt["f"] == rw["f"] and rt["pg_norm"] == rw["pg_norm"] and rt["trace_SU"] == rw["trace_SU"]
    if precision == 0 and k == 32:
        S = to_scipy(rp, c, v, spec.n)
        o = oracle.fista(S, U0.cpu().numpy().astype(np.float64), 1.0 / oracle.lipschitz(S), max_iter=25,
                         stop="none")
        assert maxabs(Ut.cpu().numpy(), o.U) <= 1e-5


def test_tcgen05_update_in_a_batch_equals_solo():
    specs = [synth.GraphSpec("dcsbm", 9001, 32, 81, mean_deg=20.0),
             synth.GraphSpec("dcsbm", 4000, 20, 82, mean_deg=30.0),
             synth.GraphSpec("dcsbm", 700, 8, 83, mean_deg=12.0),
             synth.GraphSpec("dcsbm", 3000, 50, 84, mean_deg=15.0)]
    inst = []
    for sp in specs:
        rp, c, v = synth.make_graph(sp)
        U0 = synth.dirichlet_u0(sp.n, sp.k, sp.seed)
        inst.append(tuple(t.cuda().contiguous() for t in (rp, c, v, U0)))
    # batch engine, solo engine: automatic (the warp form here) vs tcgen05,
    # warp vs tcgen05, tcgen05 for every k in 17..64 vs warp
    for eng_b, eng_s in ((0, 2), (1, 2), (2, 1)):
        b = pkg.Batch(inst, stop_rule=pkg.STOP_NONE, max_iter=20, update_engine=eng_b)
        b.step(20)
        for i, (rp, c, v, U0) in enumerate(inst):
            U, _ = _run(rp, c, v, U0, 20, update_engine=eng_s)
            assert torch.equal(b.get_U(i), U), (eng_b, i)
        b.close()


def test_wait_that_gives_up_is_a_status_and_the_context_survives():
    spec = synth.GraphSpec("dcsbm", 5000, 32, 91, mean_deg=20.0)
    rp, c, v = synth.make_graph(spec, device="cuda")
    U0 = synth.dirichlet_u0(spec.n, 32, 91, device="cuda")
    s = pkg.Solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=50, update_engine=2)
    s.step(3)
    U3 = s.get_U().clone()
    s.test_hooks(1)
    t0 = time.time()
    rep = s.step(5)
    dt = time.time() - t0
    assert rep["status"] == pkg.ETIMEOUT and rep["done"] == 1 and rep["out_iter"] == 3
    assert dt < 60
    assert torch.equal(s.get_U(), U3)          # the last complete iterate
    assert s.report()["status"] == pkg.ETIMEOUT
    assert s.state_size() > 0 and s.get_state().size > 0
    s.test_hooks(0)
    s.close()
    # the device is still fine for the next context: the same three iterations, the same bits
    s2 = pkg.Solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=50, update_engine=2)
    s2.step(3)
    assert torch.equal(s2.get_U(), U3)
    s2.close()


# a single partial tile (n = 5), one row past a tile (n = 33), fewer rows than
# update blocks, and a few full tiles with a ragged one
@pytest.mark.parametrize("n", [5, 33, 97, 1000])
def test_tcgen05_update_small_and_ragged_n(n):
    spec = synth.GraphSpec("dcsbm", n, 32, 300 + n, mean_deg=min(12.0, n / 2.0))
    rp, c, v = synth.make_graph(spec, device="cuda")
    U0 = synth.dirichlet_u0(n, 32, 300 + n, device="cuda")
    Ut, rt = _run(rp, c, v, U0, 30, update_engine=2)
    Uw, rw = _run(rp, c, v, U0, 30, update_engine=1)
    assert torch.equal(Ut, Uw)
    assert rt["f"] == rw["f"] and rt["pg_norm"] == rw["pg_norm"]
    S = to_scipy(rp, c, v, n)
    o = oracle.fista(S, U0.cpu().numpy().astype(np.float64), 1.0 / oracle.lipschitz(S), max_iter=30, stop="none")
    assert maxabs(Ut.cpu().numpy(), o.U) <= 1e-5
    # f = ||S||^2 - 2 sum_i p_i + ||A||^2: float32 sums of terms of size ||S||^2, so
    # the error bound scales with ||S||^2 (f itself can be far smaller)
    s2 = float((v.double() ** 2).sum())
    assert abs(rt["f"] - o.losses[rt["f_iter"]]) <= 1e-6 * max(abs(o.losses[rt["f_iter"]]), s2)


def test_tcgen05_update_with_a_stop_rule_inside_a_graph():
    # the relative PG rule fires inside a captured graph: the passes after it
    # return at once and both engines stop at the same iteration with the same bits
    spec = synth.GraphSpec("dcsbm", 6000, 20, 333, mean_deg=15.0)
    rp, c, v = synth.make_graph(spec, device="cuda")
    U0 = synth.dirichlet_u0(spec.n, 20, 333, device="cuda")
    outs = []
    for eng in (2, 1):
        s = pkg.Solver(rp, c, v, U0, stop_rule=pkg.STOP_PG_REL, tol=0.5, max_iter=400, update_engine=eng)
        rep = s.solve()
        outs.append((s.get_U(), rep))
        s.close()
    (Ut, rt), (Uw, rw) = outs
    assert rt["done"] == rw["done"] == 1 and rt["status"] == rw["status"] == pkg.OK
    assert rt["out_iter"] == rw["out_iter"] < 400
    assert torch.equal(Ut, Uw)


# ---- k in 33..64 (KP = 64): y G as M = 64, N = K = 64 with two swizzle atoms
# per row; the Gram as M = N = 128 over [Xbar | Y] ----
@pytest.mark.parametrize("k", [33, 48, 64])
@pytest.mark.parametrize("precision", [0, 1])
def test_tcgen05_k64_update_equals_warp_update_bitwise(k, precision):
    spec = synth.GraphSpec("dcsbm", 20011, k, 90 + k, mean_deg=25.0)
    rp, c, v = synth.make_graph(spec, device="cuda")
    U0 = synth.dirichlet_u0(spec.n, k, 90 + k, device="cuda")
    Ut, rt = _run(rp, c, v, U0, 25, precision=precision, update_engine=2)
    Uw, rw = _run(rp, c, v, U0, 25, precision=precision, update_engine=1)
    assert rt["iters"] == rw["iters"] == 25
    assert torch.equal(Ut, Uw)
    assert rt["f"] == rw["f"] and rt["pg_norm"] == rw["pg_norm"] and rt["trace_SU"] == rw["trace_SU"]
    if precision == 0:
        S = to_scipy(rp, c, v, spec.n)
        o = oracle.fista(S, U0.cpu().numpy().astype(np.float64), 1.0 / oracle.lipschitz(S), max_iter=25,
                         stop="none")
        assert maxabs(Ut.cpu().numpy(), o.U) <= 1e-5


# one partial tile of 16 rows (n = 5), one row past a tile (17), a few tiles
@pytest.mark.parametrize("n", [5, 17, 100, 1000])
def test_tcgen05_k64_update_small_and_ragged_n(n):
    spec = synth.GraphSpec("dcsbm", n, 64, 600 + n, mean_deg=min(12.0, n / 2.0))
    rp, c, v = synth.make_graph(spec, device="cuda")
    U0 = synth.dirichlet_u0(n, 64, 600 + n, device="cuda")
    Ut, rt = _run(rp, c, v, U0, 30, update_engine=2)
    S = to_scipy(rp, c, v, n)
    o = oracle.fista(S, U0.cpu().numpy().astype(np.float64), 1.0 / oracle.lipschitz(S), max_iter=30, stop="none")
    assert maxabs(Ut.cpu().numpy(), o.U) <= 1e-5
    s2 = float((v.double() ** 2).sum())
    assert abs(rt["f"] - o.losses[rt["f_iter"]]) <= 1e-6 * max(abs(o.losses[rt["f_iter"]]), s2)


def test_tcgen05_k64_wait_that_gives_up_is_a_status():
    spec = synth.GraphSpec("dcsbm", 3000, 64, 95, mean_deg=20.0)
    rp, c, v = synth.make_graph(spec, device="cuda")
    U0 = synth.dirichlet_u0(spec.n, 64, 95, device="cuda")
    s = pkg.Solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=50, update_engine=2)
    s.step(2)
    U2 = s.get_U().clone()
    s.test_hooks(1)
    rep = s.step(4)
    assert rep["status"] == pkg.ETIMEOUT and rep["done"] == 1 and rep["out_iter"] == 2
    assert torch.equal(s.get_U(), U2)
    s.test_hooks(0)
    s.close()
