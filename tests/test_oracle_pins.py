"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test ties one part of the oracle to something other than itself:
brute-force enumeration, closed-form spectra, special cases with a textbook
answer, symmetry, and the descent guarantee of Sec. 3.2.  A dropped term, a
wrong sign or index, or a transposed mu in the oracle fails at least one.
"""
import math

import numpy as np
import pytest

from paper_1511_06103_gb300 import synth
from tests import helpers as H


def _f64(d, k):
    return np.asarray(d[k], np.float64)


def small_grid(oracle, Hh, Ww, L, conn, seed, symmetric=False, scale=1.0):
    d = synth.random_grid(Hh, Ww, L, conn, seed, symmetric=symmetric, coupling_scale=scale)
    return oracle.Model.grid(_f64(d, "U"), _f64(d, "mu"), _f64(d, "w"), Hh, Ww, conn), d


def random_q(n, L, seed):
    return np.exp(synth.random_logq(n, L, seed).astype(np.float64))


def renorm(q):
    return q / q.sum(axis=1, keepdims=True)


# ---------------------------------------------------------------- P1 ----

@pytest.mark.parametrize("conn,Hh,Ww,L", [(4, 3, 3, 3), (8, 3, 3, 3), (8, 2, 4, 3), (4, 4, 4, 2)])
def test_free_energy_equals_enumeration(oracle_mod, conn, Hh, Ww, L):
    """F(q) closed form == sum_x Q(x)[E(x) + log Q(x)] (Eq. related:mf-objective)."""
    m, _ = small_grid(oracle_mod, Hh, Ww, L, conn, seed=3, symmetric=False)
    for s in range(3):
        q = renorm(random_q(Hh * Ww, L, 100 + s))
        F = m.free_energy(q)
        Fb = m.brute_free_energy(q)
        assert abs(F - Fb) <= 1e-12 * max(1.0, abs(Fb))


def test_free_energy_dense_enumeration(oracle_mod):
    rng = np.random.default_rng(7)
    n, L = 6, 3
    U = rng.normal(size=(n, L))
    mu = rng.uniform(-1, 1, size=(L, L))          # asymmetric on purpose
    K = rng.uniform(0, 1, size=(n, n))
    K = (K + K.T) / 2
    m = oracle_mod.Model.dense(U, mu, K)
    q = renorm(random_q(n, L, 5))
    assert abs(m.free_energy(q) - m.brute_free_energy(q)) <= 1e-12 * abs(m.brute_free_energy(q))
    assert np.allclose(cond_from_grad(m, q), m.brute_cond_energy(q), rtol=0, atol=1e-12)


def cond_from_grad(m, q):
    """E_{Q(X\\X_i)}[E(x) | x_i = l] = g_il + E(q) - q_i . g_i: the terms of E(x)
    that involve x_i give g_il, the rest contribute their expectation, which
    is E(q) minus the expectation of the x_i terms."""
    g = m.grad(q)
    return g + (m.energy(q) - (q * g).sum(axis=1, keepdims=True))


@pytest.mark.parametrize("conn", [4, 8])
def test_gradient_is_conditional_expected_energy(oracle_mod, conn):
    """grad E(q) is the conditional expected energy E_{Q(X\\X_i)}[E(x) | x_i = l]
    of Eq. related:sweep-update (theta* of Eq. method:update_natural) up to the
    per-variable constant that the softmax removes, by enumeration."""
    m, _ = small_grid(oracle_mod, 3, 3, 3, conn, seed=11, symmetric=False)
    q = renorm(random_q(9, 3, 12))
    gb = m.brute_cond_energy(q)
    assert np.max(np.abs(cond_from_grad(m, q) - gb)) <= 1e-12 * max(1.0, np.max(np.abs(gb)))


def test_gibbs_inequality_and_equality(oracle_mod):
    """F(q) + log Z = KL(Q||P) >= 0 (Eq. related:kl), with equality for a
    decoupled model at its exact marginals."""
    m, d = small_grid(oracle_mod, 3, 3, 2, 8, seed=21)
    logZ, marg = m.brute_force()
    for s in range(5):
        q = renorm(random_q(9, 2, 200 + s))
        assert m.free_energy(q) + logZ >= -1e-12
    U = _f64(d, "U")
    m0 = oracle_mod.Model.grid(U, _f64(d, "mu"), np.zeros_like(_f64(d, "w")), 3, 3, 8)
    logZ0, marg0 = m0.brute_force()
    assert np.allclose(marg0, H.softmax_rows(-U), atol=1e-13)
    assert abs(m0.free_energy(marg0) + logZ0) <= 1e-12


def test_free_energy_finite_difference(oracle_mod):
    """dF/dq_il = grad E_il + log q_il + 1 on the open orthant."""
    m, _ = small_grid(oracle_mod, 3, 4, 3, 8, seed=31, symmetric=False)
    q = renorm(random_q(12, 3, 32)) + 0.05
    g = m.grad(q) + np.log(q) + 1.0
    h = 1e-6
    for (i, l) in [(0, 0), (5, 2), (11, 1), (7, 0)]:
        qp = q.copy(); qp[i, l] += h
        qm = q.copy(); qm[i, l] -= h
        fd = (m.free_energy(qp) - m.free_energy(qm)) / (2 * h)
        assert abs(fd - g[i, l]) <= 1e-6 * max(1.0, abs(g[i, l]))


def test_dense_and_edge_list_agree(oracle_mod):
    """The dense-matrix model and the same model as an i<j edge list agree."""
    rng = np.random.default_rng(41)
    n, L = 12, 4
    U = rng.normal(size=(n, L))
    mu = rng.uniform(-1, 1, size=(L, L))
    feats = np.concatenate([rng.uniform(0, 5, (n, 2)), rng.uniform(0, 255, (n, 3))], axis=1)
    K = oracle_mod.dense_gauss_kernel(feats, 3.0, 13.0)
    assert np.all(np.diag(K) == 0) and np.allclose(K, K.T)
    i0, j0 = 2, 7
    d = feats[i0] - feats[j0]
    assert math.isclose(K[i0, j0], math.exp(-(d[0] ** 2 + d[1] ** 2) / 18.0 - (d[2:] ** 2).sum() / 338.0),
                        rel_tol=1e-14)
    ei, ej = np.triu_indices(n, 1)
    md = oracle_mod.Model.dense(U, mu, K)
    ms = oracle_mod.Model.sparse(U, mu, ei, ej, K[ei, ej])
    q = renorm(random_q(n, L, 42))
    assert np.allclose(md.grad(q), ms.grad(q), atol=1e-13)
    assert abs(md.free_energy(q) - ms.free_energy(q)) <= 1e-12 * abs(ms.free_energy(q))
    s = np.log(q)
    assert np.allclose(md.prox_step(0.3, s), ms.prox_step(0.3, s), atol=1e-13)


def test_grid_edge_geometry(oracle_mod):
    Hh, Ww = 5, 7
    w = np.arange(4 * Hh * Ww, dtype=np.float64).reshape(4, Hh, Ww) + 1
    ei, ej, ew = oracle_mod.grid_edges(Hh, Ww, 8, w)
    assert ei.size == Hh * (Ww - 1) + (Hh - 1) * Ww + 2 * (Hh - 1) * (Ww - 1)
    ei4, _, _ = oracle_mod.grid_edges(Hh, Ww, 4, w[:2])
    assert ei4.size == Hh * (Ww - 1) + (Hh - 1) * Ww
    pairs = {(int(a), int(b)): float(c) for a, b, c in zip(ei, ej, ew)}
    y, x = 2, 3
    p = y * Ww + x
    assert pairs[(p, p + 1)] == w[0, y, x]
    assert pairs[(p, p + Ww)] == w[1, y, x]
    assert pairs[(p, p + Ww + 1)] == w[2, y, x]
    assert pairs[(p, p + Ww - 1)] == w[3, y, x]


# ---------------------------------------------------------------- P3 ----

def test_initial_state_is_the_unary_only_marginal(oracle_mod):
    """q^0 = softmax(-U) (reading of the unstated start): on a decoupled model
    (w = 0) this is the exact marginal, which enumeration fixes; the start
    does not depend on mu or w; and on one variable with costs (0, ln 2, ln 4)
    the probabilities are (4, 2, 1)/7 by hand (softmax(+U) would give
    (1, 2, 4)/7)."""
    d = synth.random_grid(3, 3, 3, 8, seed=41, symmetric=False)
    U = _f64(d, "U")
    m0 = oracle_mod.Model.grid(U, _f64(d, "mu"), np.zeros((4, 3, 3)), 3, 3, 8)
    _, marg = m0.brute_force()
    assert np.max(np.abs(np.exp(m0.init_logq()) - marg)) <= 1e-14
    m1 = oracle_mod.Model.grid(U, _f64(d, "mu"), _f64(d, "w"), 3, 3, 8)
    assert np.array_equal(m1.init_logq(), m0.init_logq())
    one = oracle_mod.Model.sparse(np.array([[0.0, math.log(2.0), math.log(4.0)]]), np.zeros((3, 3)),
                                  np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0))
    assert np.allclose(np.exp(one.init_logq()[0]), [4 / 7, 2 / 7, 1 / 7], rtol=0, atol=1e-15)


def test_decoupled_one_full_step_gives_exact_marginals(oracle_mod):
    """w = 0: one undamped step lands on softmax(-U), the exact marginals."""
    d = synth.random_grid(3, 3, 3, 4, seed=51)
    U = _f64(d, "U")
    m = oracle_mod.Model.grid(U, _f64(d, "mu"), np.zeros((2, 3, 3)), 3, 3, 4)
    s0 = np.log(renorm(random_q(9, 3, 52)))
    s1 = m.prox_step(1.0, s0)
    _, marg = m.brute_force()
    assert np.allclose(np.exp(s1), marg, atol=1e-14)


def test_decoupled_geometric_convergence(oracle_mod):
    """w = 0, eta < 1: the natural parameters contract geometrically,
    s^t = logsoftmax((1-eta)^t s^0 + (1 - (1-eta)^t) s*), s* = logsoftmax(-U)."""
    d = synth.random_grid(4, 4, 5, 8, seed=53)
    U = _f64(d, "U")
    m = oracle_mod.Model.grid(U, _f64(d, "mu"), np.zeros((4, 4, 4)), 4, 4, 8)
    eta = 0.3
    s0 = np.log(renorm(random_q(16, 5, 54)))
    z = -U - (-U).max(axis=1, keepdims=True)
    sstar = z - np.log(np.exp(z).sum(axis=1, keepdims=True))
    s = s0.copy()
    for t in range(1, 8):
        s = m.prox_step(eta, s)
        r = (1 - eta) ** t
        a = r * s0 + (1 - r) * sstar
        expect = a - a.max(axis=1, keepdims=True)
        expect = expect - np.log(np.exp(expect).sum(axis=1, keepdims=True))
        assert np.allclose(s, expect, atol=1e-13)


def test_gauge_invariance(oracle_mod):
    """Adding c_i to U_i, or a constant c to mu, leaves the q trajectory
    unchanged and shifts F by sum_i c_i, resp. c * sum of edge weights."""
    Hh, Ww, L, conn = 5, 4, 3, 8
    d = synth.random_grid(Hh, Ww, L, conn, seed=61, symmetric=False)
    U, mu, w = _f64(d, "U"), _f64(d, "mu"), _f64(d, "w")
    m = oracle_mod.Model.grid(U, mu, w, Hh, Ww, conn)
    ci = np.random.default_rng(62).normal(size=(Hh * Ww, 1))
    mU = oracle_mod.Model.grid(U + ci, mu, w, Hh, Ww, conn)
    mM = oracle_mod.Model.grid(U, mu + 0.7, w, Hh, Ww, conn)
    s0 = m.init_logq()
    sa, Fa = m.parallel_prox(0.2, 6, s0)
    sb, Fb = mU.parallel_prox(0.2, 6, s0)
    sc, Fc = mM.parallel_prox(0.2, 6, s0)
    assert np.allclose(sa, sb, atol=1e-12) and np.allclose(sa, sc, atol=1e-12)
    assert np.allclose(Fb - Fa, ci.sum(), atol=1e-10)
    assert np.allclose(Fc - Fa, 0.7 * w.sum(), atol=1e-10)


@pytest.mark.parametrize("conn", [4, 8])
def test_rotation_equivariance(oracle_mod, conn):
    """Rotating a grid instance by 90 degrees (symmetric mu) or 180 degrees
    (mu -> mu^T) rotates the whole trajectory: pins the grid geometry."""
    Hh, Ww, L = 5, 7, 3
    d = synth.random_grid(Hh, Ww, L, conn, seed=71, symmetric=True)
    U, mu, w = _f64(d, "U"), _f64(d, "mu"), _f64(d, "w")
    m = oracle_mod.Model.grid(U, mu, w, Hh, Ww, conn)
    s, F = m.parallel_prox(0.15, 5)
    Ur, wr, Hr, Wr = H.rot90_cw_grid(U, w, Hh, Ww, conn)
    mr = oracle_mod.Model.grid(Ur, mu, wr, Hr, Wr, conn)
    sr, Fr = mr.parallel_prox(0.15, 5)
    assert np.allclose(sr, H.rot90_cw_field(s, Hh, Ww), atol=1e-12)
    assert np.allclose(F, Fr, rtol=1e-12)
    da = synth.random_grid(Hh, Ww, L, conn, seed=72, symmetric=False)
    U, mu, w = _f64(da, "U"), _f64(da, "mu"), _f64(da, "w")
    m = oracle_mod.Model.grid(U, mu, w, Hh, Ww, conn)
    s, F = m.parallel_prox(0.15, 5)
    U2, w2 = H.rot180_grid(U, w, Hh, Ww, conn)
    m2 = oracle_mod.Model.grid(U2, mu.T.copy(), w2, Hh, Ww, conn)
    s2, F2 = m2.parallel_prox(0.15, 5)
    assert np.allclose(s2, s.reshape(Hh, Ww, L)[::-1, ::-1].reshape(-1, L), atol=1e-12)
    assert np.allclose(F, F2, rtol=1e-12)


# ---------------------------------------------------------------- P2 ----

@pytest.mark.parametrize("Hh,Ww,L,c", [(6, 5, 2, 0.8), (5, 4, 3, 0.7), (4, 6, 4, 1.3)])
def test_step_constant_closed_form_grid4(oracle_mod, Hh, Ww, L, c):
    """Potts on a uniform 4-connected grid: the tangent-space Hessian is
    A (x) (-c I), so Lambda = c * (2cos(pi/(H+1)) + 2cos(pi/(W+1))); without the
    projection the top eigenvalue is c (L-1) times the same grid value."""
    U = np.zeros((Hh * Ww, L))
    w = synth.constant_edge_weights(Hh, Ww, 4, 1.0)
    m = oracle_mod.Model.grid(U, synth.potts(L, c), w, Hh, Ww, 4)
    lam_grid = H.grid4_lambda_max(Hh, Ww)
    ev = m.hessian_eigenvalues(projected=True)
    assert math.isclose(ev[-1], c * lam_grid, rel_tol=1e-10)
    ev_full = m.hessian_eigenvalues(projected=False)
    assert math.isclose(ev_full[-1], c * (L - 1) * lam_grid, rel_tol=1e-10)


def test_step_constant_closed_form_grid8(oracle_mod):
    """8-connected (king's graph) Potts grid: Lambda = c |lambda_min(A_king)|."""
    Hh, Ww, L, c = 5, 6, 3, 0.6
    U = np.zeros((Hh * Ww, L))
    w = synth.constant_edge_weights(Hh, Ww, 8, 1.0)
    m = oracle_mod.Model.grid(U, synth.potts(L, c), w, Hh, Ww, 8)
    ev = m.hessian_eigenvalues(projected=True)
    assert math.isclose(ev[-1], -c * H.king_graph_lambda_min(Hh, Ww), rel_tol=1e-10)


def test_step_constant_binary_denoising_golden(oracle_mod):
    """The 64x64 binary denoising model: Lanczos on the tangent Hessian matches
    the closed form stored in tests/golden (Sec. 3.2, Sec. 4.3)."""
    g = H.read_golden("step_size_closed_form.txt")
    # the stored constant is the closed form (the file's generator is
    # tests/golden/make_step_size_closed_form.py): recompute it here
    c = float(np.float32(0.8))
    lam_cf = c * H.grid4_lambda_max(64, 64)
    assert g["coupling"] == float(f"{c:.15g}")
    assert math.isclose(g["Lambda"], lam_cf, rel_tol=1e-15)
    assert math.isclose(g["eta"], 1.0 / (1.0 + lam_cf), rel_tol=1e-15)
    d = synth.binary_denoising()
    m = oracle_mod.Model.grid(_f64(d, "U"), _f64(d, "mu"), _f64(d, "w"), 64, 64, 4)
    lo, hi, k = m.lanczos(260, synth.lanczos_start(64 * 64, 2))
    assert math.isclose(hi, g["Lambda"], rel_tol=1e-8), (hi, g["Lambda"], k)
    assert math.isclose(oracle_mod.step_size(hi), g["eta"], rel_tol=1e-8)
    assert math.isclose(-lo, g["Lambda"], rel_tol=1e-8)   # bipartite: symmetric spectrum


def test_lanczos_matches_dense_eigensolve(oracle_mod):
    m, _ = small_grid(oracle_mod, 6, 5, 4, 8, seed=81, symmetric=False)
    ev = m.hessian_eigenvalues(projected=True)
    lo, hi, _ = m.lanczos(120, synth.lanczos_start(30, 4, seed=3))
    # the tangent space has dimension n (L-1); the remaining n eigenvalues are 0
    assert math.isclose(hi, ev[-1], rel_tol=1e-9) and math.isclose(lo, ev[0], rel_tol=1e-9)


def test_step_size_rule(oracle_mod):
    assert oracle_mod.step_size(-2.0) == 1.0          # NSD potential matrix: full step
    assert oracle_mod.step_size(0.0) == 1.0
    assert math.isclose(oracle_mod.step_size(3.0), 0.25)


# ---------------------------------------------------------------- P4 ----

def test_parallel_fixed_point_is_sweep_stationary(oracle_mod):
    """A converged parallel-prox point satisfies q = softmax(-grad E(q)): one
    SWEEP pass leaves it unchanged."""
    d = synth.binary_denoising(H=20, W=20, coupling=0.8, seed=5)
    m = oracle_mod.Model.grid(_f64(d, "U"), _f64(d, "mu"), _f64(d, "w"), 20, 20, 4)
    lam = 0.8 * H.grid4_lambda_max(20, 20)
    s, F = m.parallel_prox(1 / (1 + lam), 1500)
    s2 = m.sweep(1, s)
    assert np.max(np.abs(np.exp(s2) - np.exp(s))) <= 1e-10


def test_weak_coupling_sweep_and_parallel_agree(oracle_mod):
    """Weak coupling (tangent Hessian norm < 1) makes F strictly convex on the
    simplex product: SWEEP and parallel prox reach the same unique minimiser."""
    Hh = Ww = 24
    d = synth.binary_denoising(H=Hh, W=Ww, coupling=0.2, seed=6)
    m = oracle_mod.Model.grid(_f64(d, "U"), _f64(d, "mu"), _f64(d, "w"), Hh, Ww, 4)
    lam = 0.2 * H.grid4_lambda_max(Hh, Ww)
    assert lam < 1
    sp, _ = m.parallel_prox(1 / (1 + lam), 400)
    ss = m.sweep(200)
    assert np.max(np.abs(np.exp(sp) - np.exp(ss))) <= 1e-10


# ---------------------------------------------------------------- P5 ----

def test_monotone_free_energy_binary_denoising(oracle_mod):
    """d >= Lambda: F never increases (Sec. 3.2).  The closed-form constant
    is the same for the attractive model and its repulsive mirror
    (mu -> -mu); undamped updates (eta = 1) on the repulsive one oscillate and
    F goes up, the failure of FULL-PARALLEL on repulsive grids (Sec. 4.3)."""
    g = H.read_golden("step_size_closed_form.txt")
    d = synth.binary_denoising()
    for sign in (1.0, -1.0):
        m = oracle_mod.Model.grid(_f64(d, "U"), sign * _f64(d, "mu"), _f64(d, "w"), 64, 64, 4)
        _, F = m.parallel_prox(g["eta"], 50)
        assert np.all(np.diff(F) <= 1e-12 * np.abs(F[1:]))
    _, F1 = m.parallel_prox(1.0, 50)
    assert np.any(np.diff(F1) > 1e-3 * np.abs(F1[1:]))


def test_monotone_free_energy_repulsive_grid(oracle_mod):
    m, d = small_grid(oracle_mod, 7, 6, 5, 8, seed=91, symmetric=False, scale=2.0)
    lam = m.hessian_eigenvalues(projected=True)[-1]
    _, F = m.parallel_prox(oracle_mod.step_size(lam), 60)
    assert np.all(np.diff(F) <= 1e-12 * np.abs(F[1:]))


def test_monotone_free_energy_dense(oracle_mod):
    d = synth.dense_gaussian(side=6, L=4, seed=92)
    K = oracle_mod.dense_gauss_kernel(_f64(d, "feats"), *d["theta"])
    m = oracle_mod.Model.dense(_f64(d, "U"), 3.0 * _f64(d, "mu"), K)
    lam = m.hessian_eigenvalues(projected=True)[-1]
    assert lam > 0
    _, F = m.parallel_prox(oracle_mod.step_size(lam), 60)
    assert np.all(np.diff(F) <= 1e-12 * np.abs(F[1:]))


# ---------------------------------------------------------------- P6 ----

def test_normalisation(oracle_mod):
    m, _ = small_grid(oracle_mod, 9, 8, 6, 8, seed=95, symmetric=False)
    s, _ = m.parallel_prox(0.1, 10)
    q = np.exp(s)
    assert np.all(q >= 0)
    assert np.max(np.abs(q.sum(axis=1) - 1)) <= 1e-12


def test_step_rows_matches_full_step(oracle_mod):
    """The row-subset step is the full step restricted to those rows."""
    d = synth.dense_gaussian(side=5, L=3, seed=97)
    K = oracle_mod.dense_gauss_kernel(_f64(d, "feats"), *d["theta"])
    m = oracle_mod.Model.dense(_f64(d, "U"), _f64(d, "mu"), K)
    s0 = np.log(renorm(random_q(25, 3, 98)))
    full = m.prox_step(0.4, s0)
    rows = np.array([0, 7, 24, 13])
    assert np.array_equal(m.prox_step_rows(0.4, s0, rows), full[rows])


# ---------------------------------------------------------------- P7 ----

@pytest.mark.parametrize("conn,sym", [(4, False), (8, True)])
def test_unrolled_gradient_matches_finite_differences(oracle_mod, conn, sym):
    """Reverse mode through K = 10 unrolled steps (fixed eta) against FP64
    central differences on an 8 x 8, L = 3 grid: unaries, mu and edge weights."""
    Hh = Ww = 8
    d = synth.random_grid(Hh, Ww, 3, conn, seed=123, symmetric=sym, coupling_scale=1.5)
    U, mu, w = _f64(d, "U"), _f64(d, "mu"), _f64(d, "w")
    y = np.random.default_rng(5).integers(0, 3, size=Hh * Ww)
    eta, K, h = 0.2, 10, 1e-6
    # central differences carry ~eps |loss| / h = 2e-10 of round-off: absolute floor 1e-9
    ei, ej, ew = oracle_mod.grid_edges(Hh, Ww, conn, w)
    m = oracle_mod.Model.sparse(U, mu, ei, ej, ew)
    loss, dU, dmu, dw = m.unrolled_grad(eta, K, y, ei.size)
    assert math.isclose(loss, m.unrolled_loss(eta, K, y), rel_tol=1e-14)

    def fd(make):
        return (make(h).unrolled_loss(eta, K, y) - make(-h).unrolled_loss(eta, K, y)) / (2 * h)

    for (i, l) in [(0, 0), (27, 2), (63, 1)]:
        def mk(dh, i=i, l=l):
            U2 = U.copy(); U2[i, l] += dh
            return oracle_mod.Model.sparse(U2, mu, ei, ej, ew)
        assert abs(fd(mk) - dU[i, l]) <= 1e-7 * abs(dU[i, l]) + 1e-9
    for (a, b) in [(0, 1), (2, 0), (1, 1)]:
        def mk(dh, a=a, b=b):
            mu2 = mu.copy(); mu2[a, b] += dh
            return oracle_mod.Model.sparse(U, mu2, ei, ej, ew)
        assert abs(fd(mk) - dmu[a, b]) <= 1e-7 * abs(dmu[a, b]) + 1e-9
    for e in [0, 17, ei.size - 1]:
        def mk(dh, e=e):
            ew2 = ew.copy(); ew2[e] += dh
            return oracle_mod.Model.sparse(U, mu, ei, ej, ew2)
        assert abs(fd(mk) - dw[e]) <= 1e-7 * abs(dw[e]) + 1e-9


# ---------------------------------------------------------------- P8 ----
# Adaptive binary step (Sec. 3.3, Eq. hessian): the proximal weights are
# d_i = d q_i0 q_i1, taken from q^t.

def _golden_min(f, lo, hi, tol=1e-14):
    """Minimiser of a strictly convex f on [lo, hi] by golden-section search."""
    r = (math.sqrt(5.0) - 1.0) / 2.0
    a, b = lo, hi
    c, e = b - r * (b - a), a + r * (b - a)
    fc, fe = f(c), f(e)
    while b - a > tol:
        if fc < fe:
            b, e, fe = e, c, fc
            c = b - r * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, e, fe
            e = a + r * (b - a)
            fe = f(e)
    return 0.5 * (a + b)


@pytest.mark.parametrize("conn", [4, 8])
def test_adaptive_step_is_the_proximal_argmin(oracle_mod, conn):
    """Each variable's adaptive update equals the minimiser over the simplex
    of <q_i, grad E(q^t)_i> - H(q_i) + d_i KL(q_i || q_i^t) (Eq.
    method:proxUpdateOurs with D^t of Eq. hessian), found by brute-force
    golden-section search on p = q_i0."""
    m, d = small_grid(oracle_mod, 5, 6, 2, conn, seed=41, symmetric=False, scale=1.5)
    n = 30
    s0 = synth.random_logq(n, 2, seed=42).astype(np.float64)
    q0 = np.exp(s0)
    dd = 3.7
    s1 = m.prox_step_adaptive(dd, s0)
    g = m.grad(q0)
    for i in range(n):
        di = dd * q0[i, 0] * q0[i, 1]

        def f(p):
            qa, qb = p, 1.0 - p
            return (qa * g[i, 0] + qb * g[i, 1] + qa * math.log(qa) + qb * math.log(qb)
                    + di * (qa * math.log(qa / q0[i, 0]) + qb * math.log(qb / q0[i, 1])))

        p = _golden_min(f, 1e-15, 1.0 - 1e-15)
        assert abs(math.exp(s1[i, 0]) - p) <= 1e-7


def test_adaptive_rejects_multilabel(oracle_mod):
    m, _ = small_grid(oracle_mod, 3, 3, 3, 4, seed=43)
    with pytest.raises(ValueError):
        m.prox_step_adaptive(2.0, m.init_logq())


def test_adaptive_fixed_point_is_sweep_stationary(oracle_mod):
    """Converged adaptive iterates are mean-field stationary points: one SWEEP
    pass leaves them unchanged."""
    d = synth.binary_denoising(H=20, W=20, coupling=0.8, seed=5)
    m = oracle_mod.Model.grid(_f64(d, "U"), _f64(d, "mu"), _f64(d, "w"), 20, 20, 4)
    lam = 0.8 * H.grid4_lambda_max(20, 20)
    s, F = m.parallel_prox_adaptive(lam, 1500)
    s2 = m.sweep(1, s)
    assert np.max(np.abs(np.exp(s2) - np.exp(s))) <= 1e-10
    assert np.all(np.isfinite(F))


# ---------------------------------------------------------------- P9 ----
# OURS-MOMENTUM and OURS-ADAM (Sec. 3.4-3.5).

def test_momentum_without_memory_is_the_fixed_step(oracle_mod):
    """gamma1 = 0 turns the average into the current gradient: the iterates
    are exactly those of the fixed step."""
    m, _ = small_grid(oracle_mod, 6, 5, 3, 8, seed=51, symmetric=False, scale=1.5)
    s1, F1 = m.parallel_prox_momentum(0.3, 0.0, 25)
    s2, F2 = m.parallel_prox(0.3, 25)
    assert np.array_equal(s1, s2) and np.array_equal(F1, F2)


def test_momentum_on_a_decoupled_model(oracle_mod):
    """Without edges the gradient is U at every step, so the average stays U
    and the trajectory is the fixed step's closed form."""
    d = synth.random_grid(4, 5, 3, 4, seed=52)
    m = oracle_mod.Model.grid(_f64(d, "U"), _f64(d, "mu"), 0.0 * _f64(d, "w"), 4, 5, 4)
    eta, T = 0.35, 12
    s, _ = m.parallel_prox_momentum(eta, 0.95, T)
    s0 = m.init_logq()
    a = (1 - eta) ** T * s0 + (1 - (1 - eta) ** T) * (-_f64(d, "U"))
    ref = a - np.log(np.exp(a).sum(axis=1, keepdims=True))
    assert np.max(np.abs(s - ref)) <= 1e-12


def test_adam_special_cases(oracle_mod):
    """d0 = 0 floors d at 0 (eta = 1, FULL-PARALLEL); gamma2 = 1 keeps v at
    its start 1, so d = d0 + eps - 1 and eta = 1/(d0 + eps): with gamma1 = 0
    both are fixed steps."""
    m, _ = small_grid(oracle_mod, 5, 6, 3, 4, seed=53, symmetric=True, scale=0.7)
    s1, _ = m.parallel_prox_adam(0.0, 0.0, 0.999, 1e-8, 15)
    s2, _ = m.parallel_prox(1.0, 15)
    assert np.max(np.abs(s1 - s2)) <= 1e-12
    d0 = 4.2
    s1, _ = m.parallel_prox_adam(d0, 0.0, 1.0, 1e-8, 15)
    s2, _ = m.parallel_prox(1.0 / (d0 + 1e-8), 15)
    assert np.max(np.abs(s1 - s2)) <= 1e-12


def _adam_binary_decoupled(U, s0, d0, gamma2, eps, T, centred=True, sign=1.0):
    """Per-label Adam on a decoupled binary model, written without the
    scalar reduction (used only to show what the pin below rejects)."""
    s = s0.copy()
    v = np.ones_like(s)
    for _ in range(T):
        t = U + sign * s
        r = t - t.mean(axis=1, keepdims=True) if centred else t
        v = gamma2 * v + (1 - gamma2) * r * r
        eta = 1.0 / (1.0 + np.maximum(np.sqrt(v) * d0 + eps - 1.0, 0.0))
        a = -eta * U + (1 - eta) * s
        s = a - a.max(axis=1, keepdims=True)
        s = s - np.log(np.exp(s).sum(axis=1, keepdims=True))
    return s


def test_adam_decoupled_binary_recursion(oracle_mod):
    """OURS-ADAM (Sec. 3.5, Eq. adamStepSize) on a binary model without edges.

    Derivation.  With w = 0 the gradient is U at every step, so the momentum
    average stays U (it starts at the first gradient).  Write
    delta = (U_0 + s_0) - (U_1 + s_1).  The centred natural gradient is
    r = (U + s) - mean_l(U + s) = (+delta/2, -delta/2): both labels see the
    same r^2 = delta^2/4, hence the same v and the same eta_t, with
        v_{t+1} = gamma2 v_t + (1 - gamma2) delta_t^2 / 4,   v_0 = 1,
        eta_t   = 1 / (1 + max(sqrt(v_{t+1}) d0 + eps - 1, 0)).
    The update a = -eta U + (1 - eta) s followed by a per-variable shift gives
    delta_{t+1} = (1 - eta_t) delta_t, and since s_0 - s_1 = delta - (U_0 - U_1)
    the state is s = log sigmoid(+-(s_0 - s_1)).  Dropping the centring gives
    each label its own r^2 = (U_l + s_l)^2 and thus its own eta; flipping the
    sign of log q in r changes delta; both are shown to leave this recursion."""
    rng = np.random.default_rng(71)
    n = 12
    U = rng.normal(scale=1.5, size=(n, 2))
    s0 = synth.random_logq(n, 2, seed=72).astype(np.float64)
    m = oracle_mod.Model.sparse(U, np.array([[0.0, 0.8], [0.8, 0.0]]),
                                np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0))
    d0, g1, g2, eps, T = 2.5, 0.9, 0.7, 1e-8, 9
    s, _ = m.parallel_prox_adam(d0, g1, g2, eps, T, s0)
    delta = (U[:, 0] + s0[:, 0]) - (U[:, 1] + s0[:, 1])
    v = np.ones(n)
    for _ in range(T):
        v = g2 * v + (1 - g2) * delta ** 2 / 4
        eta = 1.0 / (1.0 + np.maximum(np.sqrt(v) * d0 + eps - 1.0, 0.0))
        delta = (1 - eta) * delta
    x = delta - (U[:, 0] - U[:, 1])            # s_0 - s_1
    ref = np.stack([-np.logaddexp(0.0, -x), -np.logaddexp(0.0, x)], axis=1)
    assert np.max(np.abs(s - ref)) <= 1e-12
    # the pin is sensitive to the two readings it is meant to rule out
    for kw in ({"centred": False}, {"sign": -1.0}):
        alt = _adam_binary_decoupled(U, s0, d0, g2, eps, T, **kw)
        assert np.max(np.abs(alt - ref)) > 1e-4, kw
    assert np.max(np.abs(_adam_binary_decoupled(U, s0, d0, g2, eps, T) - ref)) <= 1e-12


@pytest.mark.parametrize("rule", ["momentum", "adam"])
def test_momentum_and_adam_fixed_points_are_sweep_stationary(oracle_mod, rule):
    d = synth.binary_denoising(H=16, W=16, coupling=0.4, seed=7)
    m = oracle_mod.Model.grid(_f64(d, "U"), _f64(d, "mu"), _f64(d, "w"), 16, 16, 4)
    lam = 0.4 * H.grid4_lambda_max(16, 16)
    if rule == "momentum":
        s, F = m.parallel_prox_momentum(1 / (1 + lam), 0.95, 3000)
    else:
        s, F = m.parallel_prox_adam(1 + lam, 0.99, 0.999, 1e-8, 6000)   # gamma1 = 0.99 settles slowly
    s2 = m.sweep(1, s)
    assert np.max(np.abs(np.exp(s2) - np.exp(s))) <= 1e-9


# ---------------------------------------------------------------- P10 ---
# ADHOC damping (Sec. 2.2.2, Eq. related:parallel-update).

def test_adhoc_undamped_is_full_parallel(oracle_mod):
    """eta = 1: both ADHOC and the natural-parameter step become
    q^{t+1} = softmax(-grad E(q^t))."""
    m, _ = small_grid(oracle_mod, 5, 6, 4, 8, seed=61, symmetric=False)
    s1, _ = m.parallel_adhoc(1.0, 10)
    s2, _ = m.parallel_prox(1.0, 10)
    assert np.max(np.abs(np.exp(s1) - np.exp(s2))) <= 1e-13


def test_adhoc_decoupled_closed_form(oracle_mod):
    """Without edges q* = softmax(-U) is fixed, so ADHOC mixes in mean
    parameters: q^t = (1-eta)^t q^0 + (1 - (1-eta)^t) q*, unlike the
    natural-parameter step (checked to differ)."""
    d = synth.random_grid(4, 5, 3, 4, seed=62)
    U = _f64(d, "U")
    m = oracle_mod.Model.grid(U, _f64(d, "mu"), 0.0 * _f64(d, "w"), 4, 5, 4)
    eta, T = 0.3, 7
    s0 = synth.random_logq(20, 3, seed=63).astype(np.float64)
    s, _ = m.parallel_adhoc(eta, T, s0)
    qs = np.exp(-U) / np.exp(-U).sum(axis=1, keepdims=True)
    q = (1 - eta) ** T * np.exp(s0) + (1 - (1 - eta) ** T) * qs
    assert np.max(np.abs(np.exp(s) - q)) <= 1e-12
    s_ours, _ = m.parallel_prox(eta, T, s0)
    assert np.max(np.abs(np.exp(s_ours) - q)) > 1e-3


def test_adhoc_fixed_point_is_sweep_stationary(oracle_mod):
    d = synth.binary_denoising(H=16, W=16, coupling=0.4, seed=7)
    m = oracle_mod.Model.grid(_f64(d, "U"), _f64(d, "mu"), _f64(d, "w"), 16, 16, 4)
    s, _ = m.parallel_adhoc(0.3, 1500)
    s2 = m.sweep(1, s)
    assert np.max(np.abs(np.exp(s2) - np.exp(s))) <= 1e-10
