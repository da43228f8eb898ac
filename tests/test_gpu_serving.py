"""Serving (continuous batching): requests of mixed size, label count and
connectivity join and leave between steps while one launch per iteration
advances all of them.  Each result is the same alone and in the mix
(bitwise), matches a solve through the handle API and the oracle within the
FP32 tolerances, and stops after the same number of steps."""
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


def requests(n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        side = int(round(np.exp(rng.uniform(np.log(24), np.log(80)))))
        L = int(rng.choice([2, 8, 21]))
        if L == 2:
            d = synth.binary_denoising(H=side, W=side + 3, seed=100 + i)
            eta = 0.24
        else:
            d = synth.segmentation_grid(H=side, W=side + 5, L=L, conn=8, seed=200 + i)
            eta = 0.05
        d["eta"] = eta
        out.append(d)
    return out


def solve_alone(binding, d, rel_tol, max_iters):
    topo = binding.CRF_GRID8 if d["conn"] == 8 else binding.CRF_GRID4
    with binding.CRF(topo, d["L"], d["H"], d["W"]) as crf:
        crf.use_resident(False)   # the serving loop shares the step-by-step kernel's arithmetic
        crf.set_unary(d["U"])
        crf.set_pairwise(d["mu"], d["w"])
        it = crf.iterate(max_iters, eta=d["eta"], rel_tol=rel_tol, want_iters=True)[0]
        q = crf.marginals()[0]
        tr = crf.free_energy_trace(int(it))[0]
    return q, tr[-1], int(it)


def run_server(binding, reqs, budget, rel_tol, max_iters, stagger=0, slots=64):
    with binding.Server(budget, max_slots=slots) as srv:
        tickets = []
        pending = list(reqs)
        steps = 0
        while pending or any(srv.poll(t)[0] != 2 for t in tickets):
            # continuous batching: one new arrival every `stagger` steps
            if pending and (stagger == 0 or steps % stagger == 0):
                batch = pending if stagger == 0 else pending[:1]
                for d in batch:
                    tickets.append(srv.submit(d["U"], d["mu"], d["w"], d["H"], d["W"], d["conn"], eta=d["eta"],
                                              max_iters=max_iters, rel_tol=rel_tol))
                pending = pending[len(batch):]
            srv.step(1)
            steps += 1
            assert steps < 100000
        srv.sync()
        return [srv.poll(t) for t in tickets]


def test_server_matches_single_solves(env):
    """The serving tile and the handle API's step group their FP32 arithmetic
    differently, so results agree within the trajectory bounds (the stopping
    step may differ by one where |dF|/|F| sits at the tolerance)."""
    binding, oracle, torch = env
    reqs = requests(6, seed=1)
    res = run_server(binding, reqs, 1 << 30, rel_tol=1e-6, max_iters=400)
    for d, (st, F, it, q) in zip(reqs, res):
        q1, F1, it1 = solve_alone(binding, d, 1e-6, 400)
        assert st == 2 and abs(it - it1) <= 1
        assert np.abs(q - q1).max() <= 1e-5
        assert H.f_close(F, F1, d["H"] * d["W"])


def test_alone_and_in_the_mix_are_identical(env):
    binding, oracle, torch = env
    reqs = requests(7, seed=2)
    alone = run_server(binding, reqs[:1], 1 << 30, rel_tol=1e-6, max_iters=300)[0]
    mixed = run_server(binding, reqs[1:4] + reqs[:1] + reqs[4:], 1 << 30, rel_tol=1e-6, max_iters=300, stagger=3)
    st, F, it, q = mixed[3]
    assert st == 2 and it == alone[2] and F == alone[1]
    assert np.array_equal(q, alone[3])


def test_small_budget_queues_and_completes(env):
    binding, oracle, torch = env
    reqs = requests(5, seed=3)
    big = run_server(binding, reqs, 1 << 30, rel_tol=0.0, max_iters=25)
    # room for about one request at a time: the rest wait in the queue
    small = run_server(binding, reqs, 12 << 20, rel_tol=0.0, max_iters=25, slots=2)
    for a, b in zip(big, small):
        assert a[0] == b[0] == 2 and a[2] == b[2] == 25
        assert np.array_equal(a[3], b[3]) and a[1] == b[1]


def test_server_against_oracle(env):
    binding, oracle, torch = env
    d = synth.segmentation_grid(H=20, W=27, L=8, conn=8, seed=9)
    d["eta"] = 0.1
    st, F, it, q = run_server(binding, [d], 1 << 28, rel_tol=0.0, max_iters=40)[0]
    m = oracle.Model.grid(np.asarray(d["U"], np.float64), np.asarray(d["mu"], np.float64),
                          np.asarray(d["w"], np.float64), 20, 27, 8)
    s_ref, F_ref = m.parallel_prox(0.1, 40)
    assert np.abs(q - np.exp(s_ref)).max() <= 1e-5
    assert H.f_close(F, F_ref[-2], 540)


def test_step_bound_is_an_upper_bound(env):
    """eta <= 0: eta = 1/(1 + D max|nu|) >= the exact 1/(1+Lambda) bound's
    damping, i.e. the bound is at least the device Lanczos constant."""
    binding, oracle, torch = env
    d = synth.segmentation_grid(H=30, W=33, L=8, conn=8, seed=4)
    with binding.CRF(binding.CRF_GRID8, 8, 30, 33) as crf:
        crf.set_unary(d["U"])
        crf.set_pairwise(d["mu"], d["w"])
        lam, eta_exact = crf.lipschitz()
    d["eta"] = 0.0
    st, F, it, q = run_server(binding, [d], 1 << 28, rel_tol=0.0, max_iters=30)[0]
    # the same request solved with the explicit bound
    w = np.asarray(d["w"], np.float64)
    deg = w.sum(axis=0)
    deg[:, 1:] += w[0][:, :-1]
    deg[1:, :] += w[1][:-1, :]
    deg[1:, 1:] += w[2][:-1, :-1]
    deg[1:, :-1] += w[3][:-1, 1:]
    C = np.eye(8) - 1.0 / 8
    nu = np.linalg.eigvalsh(C @ np.asarray(d["mu"], np.float64) @ C)
    bound = deg.max() * np.abs(nu).max()
    assert bound >= lam[0] * (1 - 1e-6)
    d["eta"] = float(np.float32(1.0 / (1.0 + bound)))
    q2, F2, it2 = solve_alone(binding, d, 0.0, 30)
    assert np.abs(q - q2).max() <= 1e-5


def test_mixed_classes_in_one_launch_against_oracle(env):
    """Label counts 3, 5, 13, 21 and 32, 4- and 8-connected, symmetric and
    asymmetric mu, all in flight together (one launch per iteration walks
    them all); each against the oracle's trajectory."""
    binding, oracle, torch = env
    specs = [(3, 4, False), (5, 8, True), (13, 8, False), (21, 4, True), (32, 8, False)]
    reqs = []
    for i, (L, conn, sym) in enumerate(specs):
        d = synth.random_grid(19 + 3 * i, 41 - 2 * i, L, conn, seed=700 + i, symmetric=sym)
        d["eta"] = 0.2
        reqs.append(d)
    res = run_server(binding, reqs, 1 << 28, rel_tol=0.0, max_iters=25)
    for d, (st, F, it, q) in zip(reqs, res):
        assert st == 2 and it == 25
        m = oracle.Model.grid(np.asarray(d["U"], np.float64), np.asarray(d["mu"], np.float64),
                              np.asarray(d["w"], np.float64), d["H"], d["W"], d["conn"])
        s_ref, F_ref = m.parallel_prox(float(np.float32(0.2)), 25)
        assert np.abs(q - np.exp(s_ref)).max() <= 1e-5, (d["L"], d["conn"])
        assert H.f_close(F, F_ref[-2], d["H"] * d["W"])
