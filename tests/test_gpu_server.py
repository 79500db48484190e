"""Serving with continuous batching: requests admitted by device-memory budget,
advanced together, finished and replaced while others keep running; each
result equals the same request solved alone."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2506_04045_b300")

SPECS = [
    synth.GraphSpec("dcsbm", 3000, 8, 401, mean_deg=20.0),
    synth.GraphSpec("dcsbm", 800, 4, 402, mean_deg=12.0),
    synth.GraphSpec("dcsbm", 12000, 32, 403, mean_deg=25.0),
    synth.GraphSpec("dcsbm", 5000, 20, 404, mean_deg=30.0),
    synth.GraphSpec("dcsbm", 2000, 64, 405, mean_deg=18.0),
    synth.GraphSpec("dcsbm", 7000, 16, 406, mean_deg=35.0),
    synth.GraphSpec("dcsbm", 1500, 2, 407, mean_deg=10.0, blocks=2),
    synth.GraphSpec("dcsbm", 9000, 128, 408, mean_deg=15.0),
]
OPTS = dict(stop_rule=1, tol=0.05, max_iter=150)   # PG_REL: instances stop at different iterations


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.load()


def _host(spec):
    rp, c, v = synth.make_graph(spec)
    U0 = synth.dirichlet_u0(spec.n, spec.k, spec.seed)
    return rp.numpy(), c.numpy(), v.numpy(), U0.numpy()


def _solo(rp, c, v, U0, **opts):
    s = pkg.Solver(*[torch.from_numpy(x).cuda() for x in (rp, c, v, U0)], **opts)
    rep = s.solve()
    U = s.get_U().cpu().numpy()
    s.close()
    return U, rep


def test_served_results_equal_solo_results():
    reqs = [_host(s) for s in SPECS]
    srv = pkg.Server(iters_per_tick=8, **OPTS)
    tickets = [srv.submit(*r) for r in reqs]
    outs = [srv.wait(t, timeout=300) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    iters = set()
    for r, (U, rep, times) in zip(reqs, outs):
        Us, reps = _solo(*r, **OPTS)
        assert np.array_equal(U, Us)
        assert rep["out_iter"] == reps["out_iter"] and rep["f"] == reps["f"]
        assert rep["done"] == 1
        assert 0 <= times["queue_s"] <= times["total_s"] and times["run_s"] > 0
        iters.add(rep["out_iter"])
    assert len(iters) > 1


def test_served_results_match_the_oracle():
    # a fixed iteration count (stop rule NONE) so that the oracle runs the same
    # 50 iterations; four requests share the GPU, two are checked in float64
    picks = [SPECS[2], SPECS[7], SPECS[0], SPECS[4]]      # k = 32 and k = 128 first
    reqs = [_host(s) for s in picks]
    srv = pkg.Server(iters_per_tick=8, stop_rule=3, max_iter=50)
    tickets = [srv.submit(*r) for r in reqs]
    outs = [srv.wait(t, timeout=300) for t in tickets]
    srv.close()
    for spec, (rp, c, v, U0), (U, rep, _) in list(zip(picks, reqs, outs))[:2]:
        S = sp.csr_matrix((v.astype(np.float64), c, rp), shape=(spec.n, spec.n))
        o = oracle.fista(S, U0.astype(np.float64), 1.0 / oracle.lipschitz(S), max_iter=50, stop="none")
        assert rep["iters"] == 50 and rep["out_iter"] == 50
        assert float(np.max(np.abs(U - o.U))) <= 1e-5, spec
        f_ref = oracle.objective_trace(S, o.U)
        assert abs(rep["f"] - f_ref) <= 1e-6 * f_ref, (spec, rep["f"], f_ref)


def test_budget_limits_residency_and_everything_completes():
    reqs = [_host(s) for s in SPECS[:5]]
    srv = pkg.Server(iters_per_tick=4, max_resident=2, **OPTS)
    tickets = [srv.submit(*r) for r in reqs]
    peak = 0
    done = {}
    while len(done) < len(tickets):
        peak = max(peak, srv.stats()["resident"])
        for t in tickets:
            if t not in done:
                out = srv.poll(t)
                if out is not None:
                    done[t] = out
    srv.close()
    assert peak <= 2
    for r, t in zip(reqs, tickets):
        Us, _ = _solo(*r, **OPTS)
        assert np.array_equal(done[t][0], Us)


def test_oversized_and_invalid_requests_fail_without_stopping_the_server():
    small = _host(SPECS[1])
    big = _host(SPECS[2])
    srv = pkg.Server(hbm_budget=8 << 20, iters_per_tick=8, **OPTS)    # 8 MB: the n = 12000, k = 32 request (~16 MB) cannot fit
    t_big = srv.submit(*big)
    bad = list(_host(SPECS[0]))
    bad[3] = bad[3].copy()
    bad[3][5, 0] += 0.5                                                 # U0 row off the simplex
    t_bad = srv.submit(*bad)
    t_ok = srv.submit(*small)
    with pytest.raises(pkg.ClusterError) as ei:
        srv.wait(t_big, timeout=120)
    assert ei.value.status == pkg.ENOMEM
    with pytest.raises(pkg.ClusterError) as ei:
        srv.wait(t_bad, timeout=120)
    assert ei.value.status == pkg.EINVAL and "U0-row-sum" in str(ei.value)
    U, rep, _ = srv.wait(t_ok, timeout=120)
    assert rep["done"] == 1
    st = srv.stats()
    srv.close()
    assert st["failed"] == 2 and st["completed"] == 1


def test_wait_times_out_then_succeeds():
    req = _host(SPECS[2])
    srv = pkg.Server(iters_per_tick=1, stop_rule=3, max_iter=400)
    t = srv.submit(*req)
    with pytest.raises(pkg.ClusterError) as ei:
        srv.wait(t, timeout=1e-4)
    assert ei.value.status == pkg.ETIMEOUT
    U, rep, _ = srv.wait(t, timeout=300)
    assert rep["iters"] == 400
    srv.close()


def test_queue_cap_refuses_and_borrowed_inputs_work():
    reqs = [_host(s) for s in SPECS[:3]]
    # copied requests: a queue cap below one request's host bytes refuses submissions beyond the first
    srv = pkg.Server(iters_per_tick=4, max_resident=1, queue_bytes_max=1, stop_rule=3, max_iter=200)
    accepted, refused = [], 0
    for r in [reqs[2], reqs[0], reqs[1]]:
        try:
            accepted.append(srv.submit(*r))
        except pkg.ClusterError as exc:
            assert exc.status == pkg.EAGAIN and "queue full" in str(exc)
            refused += 1
    for t in accepted:
        srv.wait(t, timeout=120)
    assert srv.stats()["rejected"] == refused >= 1
    srv.close()
    # borrowed host inputs give the same results as copied ones
    srv = pkg.Server(iters_per_tick=8, borrow_host=True, **OPTS)
    ts = [srv.submit(*r) for r in reqs]
    outs = [srv.wait(t, timeout=300) for t in ts]
    srv.close()
    for r, (U, rep, _) in zip(reqs, outs):
        Us, _ = _solo(*r, **OPTS)
        assert np.array_equal(U, Us)
