"""GPU parity of general pairwise graphs (edge lists, CRF_SPARSE) against the
FP64 oracle's edge-list model, FP32 tolerances: single step |dq| <= 1e-6,
trajectories |dq| <= 1e-5 and |dF| <= 1e-6 |F| (tests.helpers.f_close)."""
import numpy as np
import pytest

from paper_1511_06103_gb300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    from paper_1511_06103_gb300 import binding, build
    build.build()
    import oracle
    oracle.build()
    return binding, oracle, torch


def f64(a):
    return np.asarray(a, np.float64)


def f_close(F, F_ref, n):
    F, F_ref = f64(F), f64(F_ref)
    return H.f_close(F, F_ref, n)


def model(oracle, d):
    return oracle.Model.sparse(f64(d["U"]), f64(d["mu"]), d["src"].astype(np.int64), d["dst"].astype(np.int64),
                               f64(d["w"]))


def crf_for(binding, d, batch=1):
    crf = binding.CRF(binding.CRF_SPARSE, d["L"], d["N"], 1, batch=batch)
    crf.set_unary(np.tile(d["U"], (batch, 1)) if batch > 1 else d["U"])
    crf.set_graph(d["mu"], d["src"], d["dst"], d["w"])
    return crf


@pytest.mark.parametrize("N,E,L,sym", [(500, 2000, 3, True), (500, 2000, 5, False), (333, 1500, 21, True),
                                       (257, 900, 32, False), (40, 0, 4, True), (1, 0, 2, True),
                                       # degrees above 32: several entries per lane in the
                                       # edge-parallel sums (L <= 8), and its largest L
                                       (300, 12000, 8, False), (200, 9000, 2, True), (150, 6000, 9, True)])
def test_sparse_single_step(env, N, E, L, sym):
    binding, oracle, torch = env
    d = synth.random_graph(N, E, L, seed=N + E + L, symmetric=sym)
    s0 = synth.random_logq(N, L, seed=L)
    s_ref = model(oracle, d).prox_step(0.35, f64(s0))
    with crf_for(binding, d) as crf:
        crf.set_state(s0)
        crf.iterate(1, eta=0.35)
        s = crf.log_marginals()[0].astype(np.float64)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= 1e-6


@pytest.mark.parametrize("maker", ["random", "dbn"])
def test_sparse_trajectory_auto_step(env, maker):
    """30 steps at the automatic step (the degree bound): parity with the
    oracle, and F never increases (the bound is >= Lambda)."""
    binding, oracle, torch = env
    d = synth.random_graph(600, 2400, 8, seed=3, symmetric=True) if maker == "random" else synth.dbn_layers()
    with crf_for(binding, d) as crf:
        lam, eta = crf.lipschitz()
        crf.iterate(30, eta=0.0, reset=True)
        s = crf.log_marginals()[0].astype(np.float64)
        trace = crf.free_energy_trace(30)[0]
    m = model(oracle, d)
    e = float(np.float32(eta[0]))
    s_ref, F_ref = m.parallel_prox(e, 30)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= 1e-5
    assert f_close(trace, F_ref[:-1], d["N"])
    assert np.all(np.diff(F_ref) <= 1e-12 * np.abs(F_ref[1:]))


def test_sparse_step_bound_is_above_lambda(env):
    binding, oracle, torch = env
    for sym in (True, False):
        d = synth.random_graph(30, 90, 3, seed=5, symmetric=sym)
        with crf_for(binding, d) as crf:
            lam, _ = crf.lipschitz()
        exact = model(oracle, d).hessian_eigenvalues(projected=True)[-1]
        assert lam[0] >= exact - 1e-5 * abs(exact)


def test_sparse_grid_edge_list_matches_grid_path(env):
    """A grid given as an edge list follows the grid path's trajectory."""
    binding, oracle, torch = env
    H, W, L = 21, 34, 6
    d = synth.random_grid(H, W, L, 8, seed=12, symmetric=False)
    ei, ej, ew = oracle.grid_edges(H, W, 8, f64(d["w"]))
    sp = dict(N=H * W, L=L, U=d["U"], mu=d["mu"], src=ei.astype(np.int32), dst=ej.astype(np.int32),
              w=ew.astype(np.float32))
    with crf_for(binding, sp) as crf:
        crf.iterate(20, eta=0.2, reset=True)
        s1 = crf.log_marginals()[0]
    with binding.CRF(binding.CRF_GRID8, L, H, W) as crf:
        crf.set_unary(d["U"])
        crf.set_pairwise(d["mu"], d["w"])
        crf.iterate(20, eta=0.2, reset=True)
        s2 = crf.log_marginals()[0]
    assert np.abs(np.exp(s1) - np.exp(s2)).max() <= 1e-5


def test_sparse_batch_and_errors(env):
    binding, oracle, torch = env
    d = synth.random_graph(200, 700, 4, seed=21)
    with crf_for(binding, d, batch=2) as crf:
        crf.iterate(10, eta=0.3, reset=True)
        s = crf.log_marginals()
    assert np.array_equal(s[0], s[1])
    with binding.CRF(binding.CRF_SPARSE, 4, 200, 1) as crf:
        with pytest.raises(binding.ProxMFError, match="INVALID"):
            crf.set_graph(d["mu"], d["src"], np.full_like(d["dst"], 200), d["w"])
        with pytest.raises(binding.ProxMFError, match="INVALID"):
            crf.set_pairwise(d["mu"], np.zeros((2, 10, 20), np.float32))


@pytest.mark.parametrize("N,E,L,sym,rows", [(9000, 36000, 5, False, None), (140000, 560000, 3, True, 3000)])
def test_sparse_step_several_variables_per_warp(env, N, E, L, sym, rows):
    """Graphs large enough that a warp takes 4 (N >= 8192) or 8 (N >= 131072)
    variables in turn: one step against the oracle (all rows, or a sample of
    rows at the larger size, which also exercises the last block's sum over
    fewer partials)."""
    binding, oracle, torch = env
    d = synth.random_graph(N, E, L, seed=N % 97 + L, symmetric=sym)
    s0 = synth.random_logq(N, L, seed=L + 1)
    m = model(oracle, d)
    with crf_for(binding, d) as crf:
        crf.set_state(s0)
        crf.iterate(1, eta=0.35)
        s = crf.log_marginals()[0].astype(np.float64)
        F_gpu = crf.free_energy_trace(1)[0][0]
    if rows is None:
        s_ref = m.prox_step(0.35, f64(s0))
        assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= 1e-6
    else:
        idx = np.random.default_rng(5).choice(N, size=rows, replace=False)
        s_ref = m.prox_step_rows(0.35, f64(s0), idx)
        assert np.abs(np.exp(s[idx]) - np.exp(s_ref)).max() <= 1e-6
    F_ref = m.free_energy(np.exp(f64(s0)))
    assert f_close(F_gpu, F_ref, N)
