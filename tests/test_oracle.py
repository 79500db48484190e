"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: values the
paper prints for its 7-node example, brute force on tiny inputs, finite
differences, closed forms of the simplex projection, the invariants of
Theorem 2.1, and a planted exact factorisation.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth
from conftest import read_sections


def _toy():
    g = read_sections("toy7.txt")
    edges = np.array([[int(a) - 1, int(b) - 1] for a, b in g["edges"]])
    S_print = np.array([[float(v) for v in r] for r in g["S"]])
    return g, edges, S_print


def _toy_S():
    g, edges, S_print = _toy()
    rp, c, v = oracle.csr_from_edges(7, edges[:, 0], edges[:, 1])
    return sp.csr_matrix((v.astype(np.float64), c, rp), shape=(7, 7))


def _scenario(g, name):
    rows = g[name]
    loss = float(rows[1][1])
    X = np.array([[float(v) for v in r] for r in rows[2:4]])
    return rows[0][1], loss, X.T            # U = X^T


def _rand_simplex(rng, n, k):
    E = -np.log(rng.random((n, k)) + 1e-300)
    return E / E.sum(1, keepdims=True)


def _rand_sym_sparse(rng, n, density=0.2, weighted=True):
    A = sp.random(n, n, density=density, random_state=rng, format="csr")
    A.data[:] = rng.random(A.nnz) if weighted else 1.0
    A = A.maximum(A.T)
    A.setdiag(1.0)
    return sp.csr_matrix(A)


# ---------------------------------------------------------------------------
# similarity matrix
# ---------------------------------------------------------------------------
def test_csr_builder_reproduces_printed_toy_matrix():
    _, _, S_print = _toy()
    S = _toy_S()
    assert np.array_equal(S.toarray(), S_print)


def test_csr_builder_max_merge_and_diagonal():
    # duplicate (0,1) with weights 0.25 and 0.75, reversed duplicate (1,0) 0.5,
    # self-loop (2,2) weight 0.1 overridden by the unit diagonal
    rp, c, v = oracle.csr_from_edges(3, [0, 0, 1, 2], [1, 1, 0, 2], [0.25, 0.75, 0.5, 0.1])
    S = sp.csr_matrix((v, c, rp), shape=(3, 3)).toarray()
    assert np.array_equal(S, np.array([[1, .75, 0], [.75, 1, 0], [0, 0, 1]], dtype=np.float32))
    rp, c, v = oracle.csr_from_edges(3, [2], [2], [0.1], add_unit_diag=False)
    assert rp.tolist() == [0, 0, 0, 1] and c.tolist() == [2] and np.isclose(v[0], 0.1)
    with pytest.raises(ValueError):
        oracle.csr_from_edges(3, [0], [3])


# ---------------------------------------------------------------------------
# objective
# ---------------------------------------------------------------------------
def test_toy_printed_losses():
    g, _, _ = _toy()
    S = _toy_S()
    _, l1, U1 = _scenario(g, "scenario1")
    _, l2, U2 = _scenario(g, "scenario2")
    _, l3, U3 = _scenario(g, "scenario3")
    assert oracle.objective_trace(S, U3) == 12.25
    assert round(oracle.objective_trace(S, U1), 2) == l1
    assert round(oracle.objective_trace(S, U2), 2) == l2


@pytest.mark.parametrize("n,k,seed", [(5, 2, 0), (17, 3, 1), (40, 8, 2), (64, 5, 3)])
def test_trace_identity_matches_brute_force(n, k, seed):
    rng = np.random.default_rng(seed)
    S = _rand_sym_sparse(rng, n)
    U = _rand_simplex(rng, n, k)
    # brute force straight from the double sum, with Python loops
    Sd = S.toarray()
    bf = 0.0
    for i in range(n):
        for j in range(n):
            bf += (Sd[i, j] - float(np.dot(U[i], U[j]))) ** 2
    assert abs(oracle.objective_dense(S, U) - bf) <= 1e-12 * bf
    assert abs(oracle.objective_trace(S, U) - bf) <= 1e-12 * bf


# ---------------------------------------------------------------------------
# gradient and Hessian
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,k,seed", [(9, 2, 0), (30, 4, 1), (50, 7, 2)])
def test_gradient_finite_differences(n, k, seed):
    rng = np.random.default_rng(seed)
    S = _rand_sym_sparse(rng, n)
    U = rng.random((n, k))
    G = oracle.gradient_matrix(S, U)
    for _ in range(6):
        E = rng.standard_normal((n, k))
        h = 1e-6
        fd = (oracle.objective_dense(S, U + h * E) - oracle.objective_dense(S, U - h * E)) / (2 * h)
        an = float(np.sum(G * E))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
    # column form equals the matrix form
    Gc = oracle.gradient_columns(S, U)
    assert np.allclose(Gc, G, rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("n,k,seed", [(8, 2, 0), (25, 3, 4)])
def test_hessian_finite_differences(n, k, seed):
    rng = np.random.default_rng(seed)
    S = _rand_sym_sparse(rng, n)
    U = rng.random((n, k))
    V = rng.standard_normal((n, k))
    h = 1e-6
    fd = (oracle.gradient_matrix(S, U + h * V) - oracle.gradient_matrix(S, U - h * V)) / (2 * h)
    H = oracle.hessian_apply(S, U, V)
    assert np.allclose(H, fd, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("n,k,seed", [(8, 2, 0), (40, 5, 1), (120, 16, 2)])
def test_sparse_hessian_equals_dense_operator(n, k, seed):
    # the sparse grouping is the dense operator of Theorem 4.1 (itself pinned by
    # finite differences above); curvature and slope are its scalar forms
    rng = np.random.default_rng(seed)
    S = _rand_sym_sparse(rng, n)
    U = _rand_simplex(rng, n, k)
    W = rng.standard_normal((n, k))
    H = oracle.hessian_apply(S, U, W)
    assert np.allclose(oracle.hessian_apply_sparse(S, U, W), H, rtol=1e-12, atol=1e-10)
    assert abs(oracle.curvature(S, U, W) - float(np.sum(W * H))) <= 1e-10 * max(1.0, float(np.abs(W * H).sum()))
    G = oracle.gradient_matrix(S, U)
    assert abs(oracle.slope(S, U, W) - float(np.sum(W * G))) <= 1e-10 * max(1.0, float(np.abs(W * G).sum()))


def test_toy_curvature_and_slope_functions():
    # Sect. 4 after the table: curvature -4 and zero slope along the printed direction
    g, _, _ = _toy()
    S = _toy_S()
    _, _, U3 = _scenario(g, "scenario3")
    Vbar = np.array([[float(v) for v in r] for r in g["hessian"][0:2]]).T
    assert oracle.curvature(S, U3, Vbar) == float(g["hessian"][2][1])
    assert oracle.slope(S, U3, Vbar) == float(g["hessian"][3][1])


def test_toy_second_order_value():
    g, _, _ = _toy()
    S = _toy_S()
    _, _, U3 = _scenario(g, "scenario3")
    Vbar = np.array([[float(v) for v in r] for r in g["hessian"][0:2]]).T
    val = float(np.sum(oracle.hessian_apply(S, U3, Vbar) * Vbar))
    gin = float(np.sum(oracle.gradient_matrix(S, U3) * Vbar))
    assert val == float(g["hessian"][2][1])
    assert gin == float(g["hessian"][3][1])


def test_gradient_lipschitz_bound():
    # Theorem 2.1: ||grad f(X) - grad f(Y)||_F <= L ||X - Y||_F on Omega with
    # L = 4 ||S||_2 + 12 N (so also with the larger Frobenius variant)
    rng = np.random.default_rng(5)
    for n, k in [(20, 2), (60, 6)]:
        S = _rand_sym_sparse(rng, n)
        L2 = oracle.lipschitz(S, "spectral")
        LF = oracle.lipschitz(S, "frobenius")
        assert L2 <= LF
        assert abs(oracle.spectral_norm(S) - np.max(np.abs(np.linalg.eigvalsh(S.toarray())))) < 1e-9
        for _ in range(20):
            X = _rand_simplex(rng, n, k)
            Y = _rand_simplex(rng, n, k)
            lhs = np.linalg.norm(oracle.gradient_matrix(S, X) - oracle.gradient_matrix(S, Y))
            assert lhs <= L2 * np.linalg.norm(X - Y) * (1 + 1e-12)


def test_step_size_statements_consistent():
    from conftest import GOLDEN
    with open(GOLDEN + "/step_sizes.txt") as fh:
        rows = [l.split() for l in fh if l.strip() and not l.startswith("#")]
    for name, N, E, tau in rows:
        N, E, tau = int(N), int(E), float(tau)
        nnz = 2 * E + N                        # 0/1 adjacency plus unit diagonal
        tau_bar = 1.0 / (4.0 * math.sqrt(nnz) + 12.0 * N)
        assert tau <= tau_bar < 100 * tau, (name, tau_bar)


# ---------------------------------------------------------------------------
# simplex projection (Algorithm 1)
# ---------------------------------------------------------------------------
def _bisection_projection(v, iters=200):
    lo, hi = v.min() - 1.0, v.max()
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if np.maximum(v - mid, 0).sum() > 1.0:
            lo = mid
        else:
            hi = mid
    return np.maximum(v - 0.5 * (lo + hi), 0)


@pytest.mark.parametrize("k", [1, 2, 3, 8, 32, 128])
def test_duchi_kkt_and_bisection(k):
    rng = np.random.default_rng(k)
    for scale in (0.01, 1.0, 100.0):
        for _ in range(20):
            v = rng.standard_normal(k) * scale
            y = oracle.duchi(v)
            assert np.all(y >= 0)
            assert abs(y.sum() - 1.0) <= 1e-12 * max(1.0, np.abs(v).max())
            sup = y > 0
            thr = v[sup] - y[sup]
            assert np.ptp(thr) <= 1e-12 * max(1.0, np.abs(v).max())
            assert np.all(v[~sup] <= thr[0] + 1e-12 * max(1.0, np.abs(v).max()))
            assert np.allclose(y, _bisection_projection(v), atol=1e-9 * max(1.0, scale))


def test_duchi_closed_forms_and_invariances():
    rng = np.random.default_rng(7)
    # k = 2: projection onto the segment, y_1 = clip((a - b + 1) / 2, 0, 1)
    for _ in range(50):
        a, b = rng.standard_normal(2) * 3
        y = oracle.duchi(np.array([a, b]))
        y1 = min(1.0, max(0.0, (a - b + 1.0) / 2.0))
        assert np.allclose(y, [y1, 1.0 - y1], atol=1e-15)
    # points of the simplex are fixed; shifts by c*1 and permutations commute
    for k in (3, 7, 32):
        p = _rand_simplex(rng, 1, k)[0]
        assert np.allclose(oracle.duchi(p), p, atol=1e-15)
        v = rng.standard_normal(k)
        y = oracle.duchi(v)
        assert np.allclose(oracle.duchi(v + 3.7), y, atol=1e-12)
        perm = rng.permutation(k)
        assert np.allclose(oracle.duchi(v[perm]), y[perm], atol=1e-15)
    # ties: all-equal input projects to the barycentre
    assert np.allclose(oracle.duchi(np.full(5, 4.0)), np.full(5, 0.2))


def test_project_omega_rowwise_equals_duchi():
    rng = np.random.default_rng(8)
    V = rng.standard_normal((200, 13)) * rng.random((200, 1)) * 5
    P = oracle.project_omega(V)
    for i in range(V.shape[0]):
        assert np.allclose(P[i], oracle.duchi(V[i]), atol=1e-14)


# ---------------------------------------------------------------------------
# algorithms
# ---------------------------------------------------------------------------
def _config1():
    import torch  # noqa: F401
    import synth
    rp, c, v = synth.make_graph(synth.GraphSpec("sbm", 2000, 8, 0, p_in=0.02, p_out=0.001))
    S = sp.csr_matrix((v.numpy().astype(np.float64), c.numpy(), rp.numpy()), shape=(2000, 2000))
    U0 = synth.dirichlet_u0(2000, 8, 0).numpy().astype(np.float64)
    return S, U0


@pytest.mark.parametrize("frac", [1.0, 0.99])
def test_gpa_monotone_at_inverse_lipschitz(frac):
    # Theorem 2.1 (i): f(X^{n+1}) <= f(X^n) for tau < 1/L (and at 1/L here)
    S, U0 = _config1()
    tau = frac / oracle.lipschitz(S)
    r = oracle.gpa(S, U0, tau, max_iter=200, stop="none")
    l = np.array(r.losses)
    assert np.all(np.diff(l) <= 1e-9 * l[0])
    assert l[-1] < l[0]
    # (ii): step lengths shrink
    steps = np.array(r.pg_norms) * tau
    assert steps[-1] < steps[0]
    assert np.all(r.U >= 0) and np.allclose(r.U.sum(1), 1.0, atol=1e-12)


def test_fista_without_momentum_is_gpa():
    S, U0 = _config1()
    tau = 1.0 / oracle.lipschitz(S)
    g = oracle.gpa(S, U0, tau, max_iter=30, stop="none", keep_history=True)
    f = oracle.fista(S, U0, tau, max_iter=30, stop="none", accel=False, keep_history=True)
    for a, b in zip(g.history, f.history):
        assert np.array_equal(a, b)
    # with momentum, the first two steps still equal GPA (t_1 = 1 gives a zero factor twice)
    fa = oracle.fista(S, U0, tau, max_iter=3, stop="none", keep_history=True)
    assert np.array_equal(fa.history[0], g.history[0])
    assert np.array_equal(fa.history[1], g.history[1])
    assert not np.array_equal(fa.history[2], g.history[2])


def test_planted_factor_is_exact_fixed_point():
    rng = np.random.default_rng(11)
    n, k = 60, 4
    lab = rng.integers(0, k, n)
    Ustar = np.eye(k)[lab]
    S = sp.csr_matrix(Ustar @ Ustar.T)           # block-diagonal ones, unit diagonal
    assert oracle.objective_trace(S, Ustar) == 0.0
    assert np.all(oracle.gradient_matrix(S, Ustar) == 0.0)
    tau = 1.0 / oracle.lipschitz(S)
    r = oracle.fista(S, Ustar, tau, max_iter=5, stop="none")
    assert np.array_equal(r.U, Ustar)
    # from a perturbed start the loss falls towards 0
    U0 = oracle.project_omega(Ustar + 0.3 * rng.random((n, k)))
    r = oracle.fista(S, U0, tau, max_iter=200, stop="none")
    assert r.losses[-1] < 0.5 * r.losses[0]


def test_toy_scenario3_stops_after_first_iteration():
    g, _, _ = _toy()
    S = _toy_S()
    tau = float(g["step"][0][0])
    U0 = np.full((7, 2), 0.5)
    for r in (oracle.gpa(S, U0, tau, max_iter=100), oracle.fista(S, U0, tau, max_iter=100)):
        assert r.stopped and np.array_equal(r.U, U0)
        assert r.losses[-1] == 12.25
    assert oracle.fista(S, U0, tau, max_iter=100).iters == 1


def test_toy_scenario2_matches_printed_output():
    g, _, _ = _toy()
    S = _toy_S()
    tau = float(g["step"][0][0])
    _, loss, Xp = _scenario(g, "scenario2")
    U0 = np.zeros((7, 2))
    U0[:, 0] = 1.0
    r = oracle.gpa(S, U0, tau, tol=0.0, max_iter=1000)
    assert r.stopped
    assert round(r.losses[-1], 2) == loss
    # the printed matrix is an early-stopped iterate (4 decimals); agree to 1e-2
    assert np.max(np.abs(r.U - Xp)) < 1e-2
    # node 4 anchors cluster 1 exactly, the graph's mirror symmetry is kept
    assert r.U[3, 0] == 1.0
    assert np.allclose(r.U[[0, 1, 2]], r.U[[6, 5, 4]], atol=1e-12)


def test_toy_scenario1_random_starts():
    g, _, _ = _toy()
    S = _toy_S()
    tau = float(g["step"][0][0])
    _, loss, Xp = _scenario(g, "scenario1")
    rng = np.random.default_rng(3)
    for _ in range(5):
        U0 = _rand_simplex(rng, 7, 2)
        r = oracle.gpa(S, U0, tau, tol=0.0, max_iter=5000)
        assert round(r.losses[-1], 2) == loss
        c2, c6 = int(np.argmax(r.U[1])), int(np.argmax(r.U[5]))
        assert c2 != c6
        assert r.U[1, c2] > 0.99 and r.U[5, c6] > 0.99
        assert abs(r.U[3, 0] - 0.5) < 0.05


def test_step_rows_reproduces_fista_iterations():
    # the per-article step used for sampled checks equals Algorithm 4's own iterations
    S, U0 = _config1()
    tau = 1.0 / oracle.lipschitz(S)
    r = oracle.fista(S, U0, tau, max_iter=6, stop="none", keep_history=True)
    betas = oracle.momentum_factors(6)
    hist = [U0] + r.history                      # Xbar^0 .. Xbar^6
    rows = list(range(0, 2000, 37))
    for n in range(2, 7):                        # Xbar^n from Xbar^{n-1}, Xbar^{n-2}
        got = oracle.fista_step_rows(S, hist[n - 1], hist[n - 2], betas[n - 1], tau, rows)
        assert np.allclose(got, hist[n][rows], rtol=0, atol=1e-13)
    assert betas[:2] == [0.0, 0.0] and 0 < betas[2] < betas[3] < 1


def test_loss_terms_against_brute_force():
    # merge = sum_i sum_j s_ij <u_i, u_j> and ||U^T U||_F^2 = sum_ij <u_i, u_j>^2
    # as double loops over articles; f against the all-pairs definition
    rng = np.random.default_rng(12)
    n, k = 40, 3
    A = sp.random(n, n, density=0.15, random_state=3, data_rvs=lambda m: 1.0 - rng.random(m))
    S = ((A + A.T) / 2 + sp.eye(n)).tocsr()
    U = _rand_simplex(rng, n, k)
    Sd = S.toarray()
    merge = sum(Sd[i, j] * float(U[i] @ U[j]) for i in range(n) for j in range(n))
    g2 = sum(float(U[i] @ U[j]) ** 2 for i in range(n) for j in range(n))
    t = oracle.loss_terms(S, U)
    assert abs(t["trace"] - merge) <= 1e-12 * merge
    assert abs(t["gram_fro2"] - g2) <= 1e-12 * g2
    assert abs(t["f"] - oracle.objective_dense(S, U)) <= 1e-12 * t["f"]
    assert abs(t["frob2"] - float((Sd * Sd).sum())) <= 1e-12 * t["frob2"]


def test_blockwise_share_and_neighbour_only_step():
    # share = X^T X entry by entry (a double loop over articles) equals the
    # blockwise sum; one step evaluated from only the sampled articles and their
    # neighbours, with that share, equals the step from the whole arrays
    rng = np.random.default_rng(11)
    X = rng.random((37, 3))
    brute = np.array([[sum(X[i, a] * X[i, b] for i in range(37)) for b in range(3)] for a in range(3)])
    blocks = [X[0:5], X[5:6], X[6:30], X[30:37]]
    assert np.allclose(oracle.gram_blocks(blocks), brute, rtol=1e-14, atol=0)
    S, U0 = _config1()
    tau = 1.0 / oracle.lipschitz(S)
    r = oracle.fista(S, U0, tau, max_iter=4, stop="none", keep_history=True)
    Xc, Xp = r.history[-1], r.history[-2]
    beta = oracle.momentum_factors(5)[4]
    rows = np.array([3, 250, 1999])
    full = oracle.fista_step_rows(S, Xc, Xp, beta, tau, rows)
    keep = np.unique(np.concatenate([rows, S[rows].indices]))
    pos = -np.ones(S.shape[0], dtype=np.int64)
    pos[keep] = np.arange(keep.size)
    sub = S[rows].tocoo()
    local = sp.csr_matrix((sub.data, (pos[rows][sub.row], pos[sub.col])), shape=(keep.size, keep.size))
    share = oracle.gram_blocks(((Xc[i:i + 300], Xp[i:i + 300]) for i in range(0, S.shape[0], 300)), beta=beta)
    Y = Xc + beta * (Xc - Xp)
    assert np.allclose(share, Y.T @ Y, rtol=1e-13, atol=0)
    part = oracle.fista_step_rows(local, Xc[keep], Xp[keep], beta, tau, pos[rows], share=share)
    assert np.allclose(part, full, rtol=0, atol=1e-14)


def test_fista_momentum_sequence_is_fixed_by_mathematics():
    # Algorithm 4: t_1 = 1, t_{n+1} = (1 + sqrt(1 + 4 t_n^2)) / 2 and
    # X^{n+1} = Xbar^n + ((t_n - 1) / t_{n+1}) (Xbar^n - Xbar^{n-1}).  Values
    # that mathematics fixes independently of any implementation:
    #   t_2 = (1 + sqrt 5) / 2, the golden ratio (positive root of t^2 = t + 1);
    #   t_3 = (1 + sqrt(7 + 2 sqrt 5)) / 2, since 1 + 4 t_2^2 = 5 + 4 t_2;
    #   beta_3 = (t_2 - 1) / t_3 = 0.6180339887 / 2.1935270855 = 0.28175353;
    #   t_{n+1} is the positive root of t^2 - t = t_n^2, and t_n >= (n + 1) / 2
    #   (the standard FISTA bound, Beck and Teboulle 2009, by induction).
    S, U0 = _config1()
    tau = 1.0 / oracle.lipschitz(S)
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    t3 = (1.0 + math.sqrt(7.0 + 2.0 * math.sqrt(5.0))) / 2.0
    beta3 = (phi - 1.0) / t3
    assert abs(beta3 - 0.28175353) < 1e-8
    r = oracle.fista(S, U0, tau, max_iter=6, stop="none", keep_history=True)
    ts = r.t_values
    assert ts[0] == 1.0
    assert abs(ts[1] - phi) <= 1e-15 and abs(ts[2] - t3) <= 1e-15
    betas = oracle.momentum_factors(1001)
    assert betas[0] == 0.0 and betas[1] == 0.0 and abs(betas[2] - beta3) <= 1e-15
    # the momentum the oracle's iterates carry: Xbar^3 is one step from
    # X^3 = Xbar^2 + beta_3 (Xbar^2 - Xbar^1); the misreading (t_2 - 1) / t_2 is not
    hist = [U0] + r.history
    rows = list(range(0, 2000, 7))
    right = oracle.fista_step_rows(S, hist[2], hist[1], beta3, tau, rows)
    wrong = oracle.fista_step_rows(S, hist[2], hist[1], (phi - 1.0) / phi, tau, rows)
    assert np.max(np.abs(right - hist[3][rows])) <= 1e-13
    assert np.max(np.abs(wrong - hist[3][rows])) > 1e-9
    # 1000 iterations on the 7-node example: the quadratic identity and the bound
    g, _, _ = _toy()
    U7 = np.full((7, 2), 0.5)
    U7[0] = (0.9, 0.1)
    r = oracle.fista(_toy_S(), U7, float(g["step"][0][0]), max_iter=1000, stop="none")
    ts = np.array(r.t_values)
    assert ts.size == 1001
    n = np.arange(1, ts.size + 1)
    assert np.all(ts >= (n + 1) / 2.0)
    assert np.allclose(ts[1:] ** 2 - ts[1:], ts[:-1] ** 2, rtol=1e-13, atol=0)
    assert np.allclose(betas[2:], (ts[1:-1] - 1.0) / ts[2:], rtol=1e-14, atol=0)


def test_artificial_two_cluster_recovery():
    # Sect. 5, Experiment 2: from X^0 with ones in the second row, both GPA and
    # FISTA recover the two planted clusters in fewer than 10 iterations.  The
    # graph is the paper's construction at reduced size; the step keeps the
    # paper's 4 tau n = 1.5 (tau = 5e-7 at n = 750,000).
    rp, c, v, labels = synth.two_cluster_graph(8000, 4000, 480.0, 640.0, 20, seed=6)
    n = 12000
    S = sp.csr_matrix((v.numpy().astype(np.float64), c.numpy(), rp.numpy()), shape=(n, n))
    assert np.all(S.data == 1.0)
    U0 = synth.second_row_start(n).numpy().astype(np.float64)
    tau = 1.5 / (4 * n)
    truth = labels.numpy()
    for accel in (False, True):
        r = oracle.fista(S, U0, tau, max_iter=9, stop="none", accel=accel)
        lab = np.argmax(r.U, axis=1)
        agree = float((lab == truth).mean())
        assert max(agree, 1.0 - agree) == 1.0, (accel, agree)
        # first step in closed form: from rows e_2, U^T U = diag(0, n) and (S U)_i =
        # (0, d_i) with d_i the row sum of S, so grad_i = (0, 4 (n - d_i)) and the
        # projection of (0, 1 - 4 tau (n - d_i)) is (2 tau (n - d_i), 1 - 2 tau (n - d_i))
        r1 = oracle.fista(S, U0, tau, max_iter=1, stop="none", accel=accel)
        d = np.asarray(S.sum(axis=1)).ravel()
        x1 = 2.0 * tau * (n - d)
        assert np.allclose(r1.U, np.stack([x1, 1.0 - x1], axis=1), rtol=0, atol=1e-12)

