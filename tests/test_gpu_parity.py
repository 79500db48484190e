"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  Tolerances: iterates within 1e-5 max-abs after 50
iterations in FP32 and final objectives within 1e-6 relative; CSR and index
work bit-exact."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from conftest import read_sections
from gpu_helpers import maxabs, to_cuda, to_scipy

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2506_04045_b300")

TOL_U = 1e-5
TOL_F = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.load()


def _solver(rp, c, v, U0, **kw):
    rp, c, v, U0 = to_cuda(rp, c, v, U0)
    return pkg.Solver(rp, c, v, U0, **kw), (rp, c, v, U0)


def _toy():
    g = read_sections("toy7.txt")
    e = np.array([[int(a) - 1, int(b) - 1] for a, b in g["edges"]])
    rp, c, v = oracle.csr_from_edges(7, e[:, 0], e[:, 1])
    return g, torch.from_numpy(rp), torch.from_numpy(c), torch.from_numpy(v)


# ---------------------------------------------------------------------------
# worked example
# ---------------------------------------------------------------------------
def test_toy_scenarios_match_oracle_and_paper():
    g, rp, c, v = _toy()
    S = to_scipy(rp, c, v, 7)
    tau = float(g["step"][0][0])
    # scenario 3: the barycentre is a fixed point, loss 12.25, stop after one iteration
    U0 = torch.full((7, 2), 0.5)
    s, _ = _solver(rp, c, v, U0, step_rule=pkg.STEP_CONST, tau=tau, accel=0, tol=0.0, max_iter=100)
    rep = s.solve()
    assert rep["done"] == 1 and rep["out_iter"] == 1 and rep["f"] == 12.25
    assert torch.equal(s.get_U().cpu(), U0)
    # scenario 2 with plain GPA, stop when the loss stops decreasing
    U0 = torch.zeros((7, 2))
    U0[:, 0] = 1
    s, _ = _solver(rp, c, v, U0, step_rule=pkg.STEP_CONST, tau=tau, accel=0, tol=0.0, max_iter=1000)
    rep = s.solve()
    o = oracle.gpa(S, U0.numpy().astype(np.float64), tau, tol=0.0, max_iter=1000)
    assert round(rep["f"], 2) == float(g["scenario2"][1][1])
    assert abs(rep["f"] - o.losses[-1]) <= 1e-5 * o.losses[-1]
    assert maxabs(s.get_U().cpu().numpy(), o.U) < 1e-4


# ---------------------------------------------------------------------------
# fixed-iteration parity, several k (ragged padding) and both methods
# ---------------------------------------------------------------------------
CASES = [
    # (graph spec, k, accel)
    (synth.GraphSpec("sbm", 2000, 8, 0, p_in=0.02, p_out=0.001), 8, 1),     # config 1 workload
    (synth.GraphSpec("sbm", 2000, 8, 0, p_in=0.02, p_out=0.001), 8, 0),
    (synth.GraphSpec("dcsbm", 3001, 2, 11, mean_deg=20.0, blocks=2), 2, 1),
    (synth.GraphSpec("dcsbm", 4000, 3, 12, mean_deg=25.0, blocks=3), 3, 1),
    (synth.GraphSpec("dcsbm", 3333, 5, 13, mean_deg=18.0, blocks=5), 5, 1),
    (synth.GraphSpec("dcsbm", 5000, 16, 14, mean_deg=30.0), 16, 1),
    (synth.GraphSpec("dcsbm", 6007, 20, 15, mean_deg=30.0), 20, 1),
    (synth.GraphSpec("dcsbm", 8000, 32, 16, mean_deg=30.0), 32, 1),
    (synth.GraphSpec("dcsbm", 3000, 64, 17, mean_deg=24.0), 64, 1),
    (synth.GraphSpec("dcsbm", 2500, 100, 18, mean_deg=20.0), 100, 1),
    (synth.GraphSpec("dcsbm", 2000, 128, 19, mean_deg=16.0), 128, 1),
]


@pytest.mark.parametrize("spec,k,accel", CASES, ids=[f"{c[0].kind}-n{c[0].n}-k{c[1]}-a{c[2]}" for c in CASES])
def test_fifty_iterations_match_oracle(spec, k, accel):
    rp, c, v = synth.make_graph(spec)
    n = spec.n
    S = to_scipy(rp, c, v, n)
    U0 = synth.dirichlet_u0(n, k, spec.seed)
    s, _ = _solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=50, accel=accel)
    rep = s.solve()
    assert rep["iters"] == 50 and rep["out_iter"] == 50 and rep["status"] == pkg.EMAXITER
    tau = 1.0 / oracle.lipschitz(S)
    assert abs(rep["tau"] - tau) <= 1e-12 * tau
    o = oracle.fista(S, U0.numpy().astype(np.float64), tau, max_iter=50, stop="none", accel=bool(accel))
    U = s.get_U().cpu().numpy()
    assert maxabs(U, o.U) <= TOL_U
    f_ref = oracle.objective_trace(S, o.U)
    assert abs(rep["f"] - f_ref) <= TOL_F * f_ref
    assert np.all(U >= 0) and np.allclose(U.sum(1), 1.0, atol=1e-5)


@pytest.mark.parametrize("fused", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_split_and_fused_iterations_agree_with_oracle(fused, prec):
    spec = synth.GraphSpec("dcsbm", 12000, 32, 23, mean_deg=30.0)
    rp, c, v = synth.make_graph(spec)
    S = to_scipy(rp, c, v, spec.n)
    U0 = synth.dirichlet_u0(spec.n, 32, 23)
    s, _ = _solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=50, fused_pass=fused, precision=prec)
    rep = s.solve()
    o = oracle.fista(S, U0.numpy().astype(np.float64), 1.0 / oracle.lipschitz(S), max_iter=50, stop="none")
    tol = TOL_U if prec == 0 else 1e-4
    assert maxabs(s.get_U().cpu().numpy(), o.U) <= tol
    f_ref = oracle.objective_trace(S, o.U)
    assert abs(rep["f"] - f_ref) <= (TOL_F if prec == 0 else 1e-5) * f_ref


def test_heavy_rows_are_chunked_and_exact():
    # a hub row adjacent to everything exercises the chunked-row path
    n, k = 3000, 32
    rng = np.random.default_rng(3)
    src = np.concatenate([np.zeros(n - 1, np.int64), rng.integers(0, n, 20000)])
    dst = np.concatenate([np.arange(1, n, dtype=np.int64), rng.integers(0, n, 20000)])
    w = rng.random(src.size).astype(np.float32)
    rp, c, v = oracle.csr_from_edges(n, src, dst, w)
    assert rp[1] - rp[0] == n                                   # row 0 touches every column
    rp, c, v = torch.from_numpy(rp), torch.from_numpy(c), torch.from_numpy(v)
    S = to_scipy(rp, c, v, n)
    U0 = synth.dirichlet_u0(n, k, 3)
    s, _ = _solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=50)
    s.solve()
    o = oracle.fista(S, U0.numpy().astype(np.float64), 1.0 / oracle.lipschitz(S), max_iter=50, stop="none")
    assert maxabs(s.get_U().cpu().numpy(), o.U) <= TOL_U


def test_loss_stop_rule_matches_oracle():
    spec = synth.GraphSpec("dcsbm", 4000, 8, 21, mean_deg=20.0)
    rp, c, v = synth.make_graph(spec)
    S = to_scipy(rp, c, v, spec.n)
    U0 = synth.dirichlet_u0(spec.n, 8, 21)
    tau = 30.0 / oracle.lipschitz(S)          # large step: the loss test fires after a few dozen iterations
    # the tolerance sits midway between two consecutive decrements of the
    # oracle's loss (about 0.2 from each, 7e-7 of f), so that the decision is
    # far outside the float32 accuracy of the loss difference
    free = oracle.fista(S, U0.numpy().astype(np.float64), tau, max_iter=120, stop="none")
    dec = -np.diff(np.asarray(free.losses))
    m = int(np.nonzero(dec <= 5.0)[0][0])
    tol = 0.5 * (dec[m - 1] + dec[m])
    assert np.min(np.abs(dec[: m + 1] - tol)) > 0.15   # no decrement up to there is near tol
    o = oracle.fista(S, U0.numpy().astype(np.float64), tau, tol=tol, max_iter=400)
    assert o.stopped and o.iters == m + 1
    s, _ = _solver(rp, c, v, U0, step_rule=pkg.STEP_CONST, tau=tau, tol=tol, max_iter=400)
    rep = s.solve()
    assert rep["done"] == 1 and rep["status"] == pkg.OK
    assert rep["out_iter"] == o.iters
    assert maxabs(s.get_U().cpu().numpy(), o.U) <= TOL_U
    assert abs(rep["f"] - o.losses[-1]) <= TOL_F * o.losses[-1]


def test_pg_stop_rule():
    spec = synth.GraphSpec("dcsbm", 3000, 4, 22, mean_deg=20.0)
    rp, c, v = synth.make_graph(spec)
    S = to_scipy(rp, c, v, spec.n)
    U0 = synth.dirichlet_u0(spec.n, 4, 22)
    o = oracle.fista(S, U0.numpy().astype(np.float64), 1.0 / oracle.lipschitz(S), max_iter=500,
                     stop="pg_rel", pg_tol=0.3)
    s, _ = _solver(rp, c, v, U0, stop_rule=pkg.STOP_PG_REL, tol=0.3, max_iter=500)
    rep = s.solve()
    assert rep["done"] == 1 and rep["out_iter"] == o.iters
    assert abs(rep["pg_norm"] - o.pg_norms[-1]) <= 1e-4 * o.pg_norms[-1]
    assert maxabs(s.get_U().cpu().numpy(), o.U) <= TOL_U


def test_planted_factor_fixed_point_bit_exact():
    n, k = 4096, 16
    rng = np.random.default_rng(4)
    lab = rng.integers(0, k, n)
    # S* = U* U*^T: all-ones blocks, unit diagonal
    order = np.argsort(lab, kind="stable")
    src, dst = [], []
    for b in range(k):
        m = order[lab[order] == b]
        ii, jj = np.triu_indices(m.size, 1)
        src.append(m[ii]); dst.append(m[jj])
    rp, c, v = oracle.csr_from_edges(n, np.concatenate(src), np.concatenate(dst))
    Ustar = np.eye(k, dtype=np.float32)[lab]
    rp, c, v = torch.from_numpy(rp), torch.from_numpy(c), torch.from_numpy(v)
    s, _ = _solver(rp, c, v, torch.from_numpy(Ustar), stop_rule=pkg.STOP_NONE, max_iter=20)
    rep = s.solve()
    # exact in real arithmetic; the float32 threshold of the tie v_b = theta may leave a few ulps
    assert maxabs(s.get_U().cpu().numpy(), Ustar) <= 4e-7
    assert rep["f"] <= 1e-6 * n


# the start: after one pass the solver reports f(Xbar^0), whose Gram term comes
# from the start Gram (gram0_kernel: k <= 64, register blocks of 4 x 4 or 2 x 2,
# tiles of 64 to 256 rows, rows past a block's range zero-filled) and whose trace
# term from the first product with S; sizes below one tile, a ragged last tile,
# and many blocks
@pytest.mark.parametrize("k", [2, 3, 5, 8, 13, 16, 27, 32, 48, 64])
@pytest.mark.parametrize("n", [37, 1000, 20011])
def test_start_gram_and_loss_of_the_start_point(k, n):
    spec = synth.GraphSpec("dcsbm", n, k, 900 + k + n, mean_deg=min(20.0, n / 4.0))
    rp, c, v = synth.make_graph(spec)
    U0 = synth.dirichlet_u0(n, k, 901 + k)
    s, _ = _solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=1)
    rep = s.step(1)
    s.close()
    assert rep["f_iter"] == 0
    S = to_scipy(rp, c, v, n)
    terms = oracle.loss_terms(S, U0.numpy().astype(np.float64))
    assert abs(rep["gram_fro2"] - terms["gram_fro2"]) <= 1e-6 * terms["gram_fro2"]
    f0 = oracle.objective_trace(S, U0.numpy().astype(np.float64))
    assert abs(rep["f"] - f0) <= TOL_F * f0


def test_objective_entry_point():
    for spec, k in [(synth.GraphSpec("dcsbm", 5000, 32, 31, mean_deg=30.0), 32),
                    (synth.GraphSpec("sbm", 2000, 8, 0), 7)]:
        rp, c, v = synth.make_graph(spec)
        S = to_scipy(rp, c, v, spec.n)
        U = synth.dirichlet_u0(spec.n, k, 9)
        f_ref = oracle.objective_trace(S, U.numpy().astype(np.float64))
        g = to_cuda(rp, c, v, U)
        f = pkg.objective(*g)
        assert abs(f - f_ref) <= TOL_F * f_ref
        # int32 row pointers are accepted too
        f32 = pkg.objective(g[0].to(torch.int32), g[1], g[2], g[3])
        assert f32 == f


def test_reruns_are_bit_identical_and_resume_from_checkpoint():
    spec = synth.GraphSpec("dcsbm", 6000, 32, 41, mean_deg=30.0)
    rp, c, v = synth.make_graph(spec)
    U0 = synth.dirichlet_u0(spec.n, 32, 41)
    a, keep = _solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=40)
    a.step(17)
    state = a.get_state()
    a.step(23)
    Ua = a.get_U().cpu()
    b, _ = _solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=40)
    b.step(40)
    assert torch.equal(b.get_U().cpu(), Ua)
    c2, _ = _solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=40)
    c2.set_state(state)
    rep = c2.step(23)
    assert rep["iters"] == 40
    assert torch.equal(c2.get_U().cpu(), Ua)


def test_validation_rejects_bad_inputs():
    spec = synth.GraphSpec("dcsbm", 500, 4, 51, mean_deg=10.0)
    rp, c, v = synth.make_graph(spec)
    U0 = synth.dirichlet_u0(500, 4, 51)
    # U0 off the simplex
    bad = U0.clone()
    bad[3, 0] += 0.01
    with pytest.raises(pkg.ClusterError) as ei:
        _solver(rp, c, v, bad)
    assert ei.value.status == pkg.EINVAL and "U0-row-sum" in str(ei.value)
    # asymmetric values (validate=2 only)
    v2 = v.clone()
    j = int(rp[10]) if int(c[int(rp[10])]) != 10 else int(rp[10]) + 1   # an off-diagonal entry of row 10
    v2[j] = 0.123
    _solver(rp, c, v2, U0, validate=1)
    with pytest.raises(pkg.ClusterError) as ei:
        _solver(rp, c, v2, U0, validate=2)
    assert "asymmetric" in str(ei.value)
    # unsorted columns in a row
    c2 = c.clone()
    lo = int(rp[20])
    c2[lo], c2[lo + 1] = c[lo + 1], c[lo]
    with pytest.raises(pkg.ClusterError) as ei:
        _solver(rp, c2, v, U0)
    assert "col-order" in str(ei.value)
    # broken row pointer
    rp2 = rp.clone()
    rp2[5] = rp2[6] + 1
    with pytest.raises(pkg.ClusterError) as ei:
        _solver(rp2, c, v, U0)
    assert "row_ptr" in str(ei.value)


def test_nonfinite_weight_ends_the_run_with_enonfinite():
    # a NaN similarity (validate = 0 lets it through) poisons the first
    # product: the fold reports CLUSTER_ENONFINITE and keeps Xbar^0 as output
    spec = synth.GraphSpec("dcsbm", 3000, 8, 81, mean_deg=20.0)
    rp, c, v = synth.make_graph(spec)
    tau = 1.0 / oracle.lipschitz(to_scipy(rp, c, v, spec.n))
    v2 = v.clone()
    v2[int(rp[100]) + 1] = float("nan")
    U0 = synth.dirichlet_u0(spec.n, 8, 81)
    s, _ = _solver(rp, c, v2, U0, validate=0, step_rule=pkg.STEP_CONST, tau=tau, stop_rule=pkg.STOP_NONE,
                   max_iter=20)
    rep = s.step(20)
    assert rep["done"] == 1 and rep["status"] == pkg.ENONFINITE and rep["out_iter"] == 0
    assert rep["iters"] == 1
    assert torch.equal(s.get_U().cpu(), U0)
    s.close()


@pytest.mark.parametrize("k", [32, 8])
def test_nonfinite_iterate_mid_run_keeps_the_last_good_iterate(k):
    # a NaN planted from the host into the stored products S Xbar (checkpoint
    # buffers) at iteration 10 reaches the next update: the run ends with
    # CLUSTER_ENONFINITE, the output is the last complete iterate Xbar^10, and
    # restoring the clean checkpoint resumes bit for bit
    spec = synth.GraphSpec("dcsbm", 6000, k, 82, mean_deg=25.0)
    rp, c, v = synth.make_graph(spec)
    U0 = synth.dirichlet_u0(spec.n, k, 82)
    a, _ = _solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=40)
    a.step(10)
    U10 = a.get_U().cpu()
    clean = a.get_state()
    a.step(30)
    U40 = a.get_U().cpu()
    a.close()
    # state = header (32 B), FistaState, G(Y) (KP^2 float32), X0, X1, Z0, Z1 (n KP float32 each)
    KP = 1 << max(0, (k - 1).bit_length())
    nk, e2 = spec.n * KP * 4, KP * KP * 4
    fs = clean.size - 32 - e2 - 4 * nk
    assert 0 < fs < 4096
    bad = clean.copy()
    nan = np.frombuffer(np.float32(np.nan).tobytes(), np.uint8)
    for z in (32 + fs + e2 + 2 * nk, 32 + fs + e2 + 3 * nk):
        o = z + 5 * KP * 4
        bad[o:o + 4] = nan
    b, _ = _solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=40)
    b.set_state(bad)
    rep = b.step(30)
    assert rep["done"] == 1 and rep["status"] == pkg.ENONFINITE
    assert rep["out_iter"] == 10 and rep["iters"] == 11
    assert torch.equal(b.get_U().cpu(), U10)
    b.set_state(clean)
    rep = b.step(30)
    assert rep["status"] == pkg.EMAXITER and rep["out_iter"] == 40
    assert torch.equal(b.get_U().cpu(), U40)
    b.close()


def test_spectral_step_rule_matches_eigensolver():
    spec = synth.GraphSpec("dcsbm", 1500, 4, 61, mean_deg=12.0)
    rp, c, v = synth.make_graph(spec)
    S = to_scipy(rp, c, v, spec.n)
    U0 = synth.dirichlet_u0(spec.n, 4, 61)
    s, _ = _solver(rp, c, v, U0, step_rule=pkg.STEP_INV_L_SPEC)
    rep = s.step(0)
    L = oracle.lipschitz(S, "spectral")
    assert abs(rep["L"] - L) <= 1e-6 * L


@pytest.mark.parametrize("k", [8, 32])
def test_mixed_precision_error_against_oracle(k):
    spec = synth.GraphSpec("dcsbm", 20000, k, 71, mean_deg=30.0)
    rp, c, v = synth.make_graph(spec)
    S = to_scipy(rp, c, v, spec.n)
    U0 = synth.dirichlet_u0(spec.n, k, 71)
    s, _ = _solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=50, precision=pkg.MIXED_BF16)
    rep = s.solve()
    o = oracle.fista(S, U0.numpy().astype(np.float64), 1.0 / oracle.lipschitz(S), max_iter=50, stop="none")
    err = maxabs(s.get_U().cpu().numpy(), o.U)
    f_ref = oracle.objective_trace(S, o.U)
    # bfloat16 gathers perturb only the small data term of each step
    assert err <= 1e-4, err
    assert abs(rep["f"] - f_ref) <= 1e-5 * f_ref


def test_sampled_rows_at_one_million_articles():
    """Config-2 scale (n = 1e6, k = 32, power-law degrees): the GPU's Xbar^n at
    sampled articles against one oracle step from the GPU's own Xbar^{n-1},
    Xbar^{n-2} (the same launch configuration the benchmark times)."""
    spec = synth.GraphSpec("dcsbm", 1_000_000, 32, 1, mean_deg=30.0)
    rp, c, v = synth.make_graph(spec, device="cuda")
    n, k = spec.n, 32
    U0 = synth.dirichlet_u0(n, k, 1, device="cuda")
    s = pkg.Solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=100, borrow=1)
    m = 12
    s.step(m - 2)
    X2 = s.get_U().cpu().numpy()
    s.step(1)
    X1 = s.get_U().cpu().numpy()
    rep = s.step(1)
    X0 = s.get_U().cpu().numpy()
    S = to_scipy(rp, c, v, n)
    # loss terms in float64: each update block sums thousands of rows here, so
    # a drifting accumulation would show up above ordinary float32 rounding
    S2 = float((S.data.astype(np.float64) ** 2).sum())

    def loss_terms(X):
        Xd = X.astype(np.float64)
        Gm = Xd.T @ Xd
        gram2 = float((Gm * Gm).sum())
        tr = float((Xd * (S @ Xd)).sum())
        return gram2, tr, S2 - 2.0 * tr + gram2

    assert rep["f_iter"] == m - 1         # the pass that formed Xbar^m evaluated f(Xbar^{m-1})
    gram2, tr, f = loss_terms(X1)
    print(f"\nn=1M: rel err gram_fro2 {abs(rep['gram_fro2'] - gram2) / gram2:.3e} trace "
          f"{abs(rep['trace_SU'] - tr) / tr:.3e} f {abs(rep['f'] - f) / f:.3e}")
    # measured on a B300: 4.8e-7 (Gram and f), 6e-11 (trace)
    assert abs(rep["gram_fro2"] - gram2) <= TOL_F * gram2
    assert abs(rep["trace_SU"] - tr) <= TOL_F * tr
    assert abs(rep["f"] - f) <= TOL_F * f
    f0 = loss_terms(X0)[2]
    assert abs(pkg.objective(rp, c, v, s.get_U()) - f0) <= TOL_F * f0
    tau = 1.0 / oracle.lipschitz(S)
    beta = oracle.momentum_factors(m)[m - 1]
    deg = np.diff(S.indptr)
    rng = np.random.default_rng(0)
    rows = np.unique(np.concatenate([rng.integers(0, n, 3000), np.argsort(deg)[-50:]]))
    ref = oracle.fista_step_rows(S, X1, X2, beta, tau, rows)
    assert maxabs(X0[rows], ref) <= TOL_U


def test_internal_degree_numbering_is_invisible_to_the_caller():
    # relabel = 1 (default) numbers articles by degree inside the library; U0,
    # U and the losses stay in the caller's numbering and agree with relabel = 0
    spec = synth.GraphSpec("dcsbm", 20000, 16, 41, mean_deg=25.0)
    rp, c, v = synth.make_graph(spec, device="cuda")
    U0 = synth.dirichlet_u0(spec.n, 16, 41, device="cuda")
    runs = []
    for relabel in (1, 0):
        s = pkg.Solver(rp, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=30, relabel=relabel)
        rep = s.step(30)
        runs.append((s.get_U().cpu().numpy(), rep, s))
    (Ua, ra, sa), (Ub, rb, sb) = runs
    # the two numberings sum the Gram partials in different orders: float32 rounding only
    assert maxabs(Ua, Ub) <= TOL_U
    assert abs(ra["f"] - rb["f"]) <= TOL_F * abs(rb["f"])
    S = to_scipy(rp, c, v, spec.n)
    o = oracle.fista(S, U0.cpu().numpy().astype(np.float64), 1.0 / oracle.lipschitz(S), max_iter=30, stop="none")
    assert maxabs(Ua, o.U) <= TOL_U
    # a checkpoint records the numbering and is refused by a context with the other one
    buf = sa.get_state()
    with pytest.raises(pkg.ClusterError) as ei:
        sb.set_state(buf)
    assert ei.value.status == pkg.EINVAL
    sa.close()
    sb.close()
    # the L2 window is a cache hint and int32 row pointers are widened: neither changes a bit
    for kw, rpk in (({"l2_window": 0}, rp), ({}, rp.to(torch.int32))):
        s = pkg.Solver(rpk, c, v, U0, stop_rule=pkg.STOP_NONE, max_iter=30, **kw)
        s.step(30)
        assert torch.equal(s.get_U(), torch.from_numpy(Ua).cuda()), kw
        s.close()
