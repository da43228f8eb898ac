"""GPU parity of the grid path against the FP64 oracle, through the C ABI.

Tolerances (FP32 form): single step |dq|max <= 1e-6; trajectories
|dq|max <= 1e-5 and |dF|/|F| <= 1e-6.
"""
import math

import numpy as np
import pytest

from paper_1511_06103_gb300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

TOL_Q_STEP = 1e-6
TOL_Q = 1e-5
TOL_F = 1e-6


def f_close(F, F_ref, n_vars):
    """|dF| <= 1e-6 |F| (see tests.helpers.f_close for cancelling instances)."""
    return H.f_close(F, F_ref, n_vars, TOL_F)


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


def topo(binding, conn):
    return binding.CRF_GRID8 if conn == 8 else binding.CRF_GRID4


def make(binding, torch, d, batch=1):
    crf = binding.CRF(topo(binding, d["conn"]), d["L"], d["H"], d["W"], batch=batch)
    return crf


def oracle_model(oracle, d):
    return oracle.Model.grid(f64(d["U"]), f64(d["mu"]), f64(d["w"]), d["H"], d["W"], d["conn"])


def gpu_run(binding, torch, d, eta, iters, s0=None):
    dev = torch.device("cuda:0")
    with make(binding, torch, d) as crf:
        crf.set_unary(torch.from_numpy(d["U"]).to(dev))
        crf.set_pairwise(torch.from_numpy(d["mu"]).to(dev), torch.from_numpy(d["w"]).to(dev))
        if s0 is not None:
            crf.set_state(torch.from_numpy(np.ascontiguousarray(s0, np.float32)).to(dev))
        crf.iterate(iters, eta=eta)
        s = torch.empty((1, d["H"] * d["W"], d["L"]), device=dev)
        crf.log_marginals(s)
        F = crf.free_energy()[0]
        trace = crf.free_energy_trace(iters)[0] if iters > 0 else np.zeros(0)
        torch.cuda.synchronize()
        return s[0].cpu().numpy().astype(np.float64), F, trace


CASES = [
    # (H, W, L, conn, symmetric)   -- several tiles and ragged tails
    (37, 45, 2, 4, True), (37, 45, 3, 8, False), (21, 70, 5, 4, False), (33, 33, 8, 8, True),
    (19, 40, 13, 8, False), (40, 33, 21, 8, True), (17, 35, 21, 4, False), (9, 65, 24, 8, True),
    (12, 34, 32, 8, False), (1, 1, 3, 8, False), (1, 50, 4, 4, True), (50, 1, 4, 8, False),
    (5, 7, 1, 8, True),
]


@pytest.mark.parametrize("Hh,Ww,L,conn,sym", CASES)
def test_single_step_parity(env, Hh, Ww, L, conn, sym):
    binding, oracle, torch = env
    d = synth.random_grid(Hh, Ww, L, conn, seed=Hh * 131 + Ww * 7 + L, symmetric=sym)
    s0 = synth.random_logq(Hh * Ww, L, seed=5 + L)
    m = oracle_model(oracle, d)
    s_ref = m.prox_step(0.37, f64(s0))
    F_ref = m.free_energy(np.exp(f64(s0)))
    s, _, trace = gpu_run(binding, torch, d, 0.37, 1, s0=s0)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= TOL_Q_STEP
    assert f_close(trace[0], F_ref, Hh * Ww)


@pytest.mark.parametrize("Hh,Ww,L,conn,sym,eta,iters", [
    (40, 52, 3, 8, False, 0.15, 60), (33, 70, 21, 8, True, 0.05, 100), (30, 41, 8, 4, False, 0.3, 50),
])
def test_trajectory_parity(env, Hh, Ww, L, conn, sym, eta, iters):
    binding, oracle, torch = env
    d = synth.random_grid(Hh, Ww, L, conn, seed=1000 + L, symmetric=sym)
    m = oracle_model(oracle, d)
    s_ref, F_ref = m.parallel_prox(eta, iters)
    s, F, trace = gpu_run(binding, torch, d, eta, iters)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= TOL_Q
    assert f_close(trace, F_ref[:-1], Hh * Ww)
    assert f_close(F, F_ref[-1], Hh * Ww)


def test_binary_denoising_trajectory(env):
    """The 64x64 binary denoising workload: 50 steps at the closed-form step."""
    binding, oracle, torch = env
    g = H.read_golden("step_size_closed_form.txt")
    d = synth.binary_denoising()
    m = oracle_model(oracle, d)
    s_ref, F_ref = m.parallel_prox(g["eta"], 50)
    s, F, trace = gpu_run(binding, torch, d, g["eta"], 50)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= TOL_Q
    assert f_close(F, F_ref[-1], 64 * 64)
    assert f_close(trace, F_ref[:-1], 64 * 64)


def test_segmentation_grid_full_size_first_steps(env):
    """512x512, L=21, 8-connected (the segmentation-shaped workload) in the
    launch configuration of the benchmark: 8 steps against the oracle."""
    binding, oracle, torch = env
    d = synth.segmentation_grid()
    m = oracle_model(oracle, d)
    eta = 0.04
    s_ref, F_ref = m.parallel_prox(eta, 8)
    s, F, trace = gpu_run(binding, torch, d, eta, 8)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= TOL_Q
    assert f_close(F, F_ref[-1], 512 * 512)
    assert f_close(trace, F_ref[:-1], 512 * 512)


def test_step_constant_binary_denoising(env):
    binding, oracle, torch = env
    g = H.read_golden("step_size_closed_form.txt")
    d = synth.binary_denoising()
    with make(binding, torch, d) as crf:
        crf.set_unary(d["U"])
        crf.set_pairwise(d["mu"], d["w"])
        lam, eta = crf.lipschitz()
    assert math.isclose(lam[0], g["Lambda"], rel_tol=1e-8)
    assert math.isclose(eta[0], g["eta"], rel_tol=1e-6)   # eta is held in FP32


@pytest.mark.parametrize("sym,conn", [(True, 8), (False, 8), (False, 4)])
def test_step_constant_vs_dense_eigensolve(env, sym, conn):
    binding, oracle, torch = env
    d = synth.random_grid(6, 7, 4, conn, seed=77, symmetric=sym, coupling_scale=1.5)
    lam_ref = oracle_model(oracle, d).hessian_eigenvalues(projected=True)[-1]
    with make(binding, torch, d) as crf:
        crf.set_unary(d["U"])
        crf.set_pairwise(d["mu"], d["w"])
        lam, _ = crf.lipschitz()
    assert math.isclose(lam[0], lam_ref, rel_tol=1e-8, abs_tol=1e-12)


def test_auto_step_is_monotone(env):
    """eta = 1/(1+Lambda) from the device estimate: F does not increase."""
    binding, oracle, torch = env
    d = synth.random_grid(48, 64, 6, 8, seed=91, symmetric=False, coupling_scale=2.0)
    dev = torch.device("cuda:0")
    with make(binding, torch, d) as crf:
        crf.set_unary(d["U"])
        crf.set_pairwise(d["mu"], d["w"])
        crf.iterate(40, eta=0.0)
        trace = crf.free_energy_trace(40)[0]
    assert np.all(np.diff(trace) <= 2e-7 * np.abs(trace[1:]))


def test_batch_instances_are_independent(env):
    """A batch gives, per instance, exactly the result of solving it alone."""
    binding, oracle, torch = env
    ds = [synth.random_grid(23, 41, 5, 8, seed=300 + i, symmetric=(i % 2 == 0)) for i in range(3)]
    # one shared mu for the batch
    for d in ds:
        d["mu"] = ds[0]["mu"]
    U = np.stack([d["U"] for d in ds])
    w = np.stack([d["w"] for d in ds])
    dev = torch.device("cuda:0")
    with binding.CRF(binding.CRF_GRID8, 5, 23, 41, batch=3) as crf:
        crf.set_unary(torch.from_numpy(U).to(dev))
        crf.set_pairwise(torch.from_numpy(ds[0]["mu"]).to(dev), torch.from_numpy(w).to(dev))
        crf.iterate(20, eta=0.25)
        sb = crf.log_marginals()
        Fb = crf.free_energy()
    for i, d in enumerate(ds):
        s, F, _ = gpu_run(binding, torch, d, 0.25, 20)
        assert np.array_equal(sb[i].astype(np.float64), s)
        assert Fb[i] == F


def test_stopping_rule(env):
    binding, oracle, torch = env
    d = synth.binary_denoising(H=48, W=40, seed=3)
    tol = 1e-6
    m = oracle_model(oracle, d)
    g = 1.0 / (1.0 + 0.8 * H.grid4_lambda_max(48, 40))
    _, F_ref = m.parallel_prox(g, 300)
    stop_ref = next(t + 1 for t in range(1, 300) if abs(F_ref[t] - F_ref[t - 1]) <= tol * abs(F_ref[t]))
    with make(binding, torch, d) as crf:
        crf.set_unary(d["U"])
        crf.set_pairwise(d["mu"], d["w"])
        it = crf.iterate(300, eta=g, rel_tol=tol, want_iters=True)[0]
        tr = crf.free_energy_trace(int(it))[0]
    t = it - 1
    assert abs(tr[t] - tr[t - 1]) <= tol * abs(tr[t])
    assert all(abs(tr[k] - tr[k - 1]) > tol * abs(tr[k]) for k in range(1, t))
    assert abs(int(it) - stop_ref) <= 1


def test_zero_iterations_and_reset(env):
    binding, oracle, torch = env
    d = synth.random_grid(10, 12, 4, 4, seed=5)
    m = oracle_model(oracle, d)
    with make(binding, torch, d) as crf:
        crf.set_unary(d["U"])
        crf.set_pairwise(d["mu"], d["w"])
        crf.iterate(0, eta=0.5)
        s0 = crf.log_marginals()[0].astype(np.float64)
        assert np.abs(np.exp(s0) - np.exp(m.init_logq())).max() <= TOL_Q_STEP
        crf.iterate(5, eta=0.5)
        crf.iterate(0, eta=0.5, reset=True)
        s1 = crf.log_marginals()[0].astype(np.float64)
        assert np.array_equal(s0, s1)


def test_full_parallel_step(env):
    binding, oracle, torch = env
    d = synth.random_grid(20, 30, 3, 8, seed=8, symmetric=False)
    m = oracle_model(oracle, d)
    s_ref, F_ref = m.parallel_prox(1.0, 6)
    s, F, _ = gpu_run(binding, torch, d, 1.0, 6)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= TOL_Q


def test_non_finite_unaries_are_reported(env):
    binding, oracle, torch = env
    d = synth.random_grid(8, 8, 3, 4, seed=9)
    U = d["U"].copy()
    U[5, 1] = np.nan
    with make(binding, torch, d) as crf:
        crf.set_unary(U)
        crf.set_pairwise(d["mu"], d["w"])
        crf.iterate(2, eta=0.5)
        with pytest.raises(binding.ProxMFError) as e:
            crf.free_energy()
        assert e.value.status == -6


def test_rotation_equivariance_gpu(env):
    """The device stencil honours the grid geometry: rotating the instance
    rotates the result (symmetric mu, 90 degrees)."""
    binding, oracle, torch = env
    d = synth.random_grid(14, 37, 5, 8, seed=12, symmetric=True)
    s, F, _ = gpu_run(binding, torch, d, 0.3, 7)
    Ur, wr, Hr, Wr = H.rot90_cw_grid(d["U"], d["w"], d["H"], d["W"], 8)
    dr = dict(d, U=np.ascontiguousarray(Ur), w=np.ascontiguousarray(wr), H=Hr, W=Wr)
    sr, Fr, _ = gpu_run(binding, torch, dr, 0.3, 7)
    assert np.abs(np.exp(sr) - np.exp(H.rot90_cw_field(s, d["H"], d["W"]))).max() <= 1e-6
    assert abs(F - Fr) <= 1e-6 * abs(F)


@pytest.mark.parametrize("rel_tol", [0.0, 1e-6])
def test_graph_replay_matches_eager(env, rel_tol):
    """mf_use_graphs: captured and replayed step loops give bit-identical
    states, traces and iteration counts (first replay and cached replays)."""
    binding, oracle, torch = env
    d = synth.binary_denoising()
    res = []
    for graphs in (False, True):
        with make(binding, torch, d) as crf:
            crf.use_graphs(graphs)
            crf.use_resident(False)   # the step-by-step loop (eager or replayed)
            crf.set_unary(d["U"])
            crf.set_pairwise(d["mu"], d["w"])
            out = []
            for _ in range(3):
                its = crf.iterate(50, eta=0.0, reset=True, rel_tol=rel_tol, want_iters=True)
                out.append((crf.log_marginals().copy(), crf.free_energy_trace(50).copy(), its.copy()))
            # an odd count flips the buffer parity; the next call needs another graph
            crf.iterate(7, eta=0.3)
            out.append((crf.log_marginals().copy(), crf.free_energy_trace(7).copy(), None))
            crf.iterate(7, eta=0.3)
            out.append((crf.log_marginals().copy(), crf.free_energy_trace(7).copy(), None))
            res.append(out)
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a[0], b[0])
        assert np.array_equal(a[1], b[1])
        if a[2] is not None:
            assert np.array_equal(a[2], b[2])


def test_device_allocation_failure_is_reported(env):
    """A handle whose arrays exceed device memory fails with CRF_E_OOM (a
    failed cudaMalloc, nothing launched) and leaves the context usable: a
    handle created afterwards still matches the oracle.  The request is
    64 x 8192 x 8192 pixels x 24 stored labels x 4 bytes = 412 GB per array,
    within the size limits of the ABI but above the 288 GB of the device."""
    binding, oracle, torch = env
    with pytest.raises(binding.ProxMFError) as e:
        binding.CRF(binding.CRF_GRID8, 21, 8192, 8192, batch=64)
    assert e.value.status == -2
    with pytest.raises(binding.ProxMFError) as e:
        binding.Server(1 << 42)
    assert e.value.status == -2
    d = synth.random_grid(9, 14, 3, 8, seed=31, symmetric=True)
    s_ref = oracle_model(oracle, d).prox_step(0.5, oracle_model(oracle, d).init_logq())
    s, _, _ = gpu_run(binding, torch, d, 0.5, 1)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= TOL_Q


@pytest.mark.parametrize("B,Hh,Ww,L,conn", [(5, 9, 11, 3, 8), (2, 1, 13, 4, 4), (3, 16, 5, 5, 8)])
def test_step_constant_batch_vs_dense_eigensolve(env, B, Hh, Ww, L, conn):
    """Every instance of a batch gets its own constant (symmetric mu: the
    scalar Lanczos form, one cooperative launch per chunk of steps), equal to
    the top eigenvalue of its tangent-projected Hessian."""
    binding, oracle, torch = env
    ds = [synth.random_grid(Hh, Ww, L, conn, seed=900 + 7 * i, symmetric=True, coupling_scale=1.3)
          for i in range(B)]
    for d in ds:
        d["mu"] = ds[0]["mu"]
    topo_ = binding.CRF_GRID8 if conn == 8 else binding.CRF_GRID4
    with binding.CRF(topo_, L, Hh, Ww, batch=B) as crf:
        crf.set_unary(np.stack([d["U"] for d in ds]))
        crf.set_pairwise(ds[0]["mu"], np.stack([d["w"] for d in ds]))
        lam, eta = crf.lipschitz()
    for i, d in enumerate(ds):
        ref = oracle_model(oracle, d).hessian_eigenvalues(projected=True)[-1]
        assert math.isclose(lam[i], ref, rel_tol=1e-8, abs_tol=1e-12)
        assert math.isclose(eta[i], 1.0 / (1.0 + max(ref, 0.0)), rel_tol=1e-6)


def _lipschitz(binding, d, B=1, w_scale=1.0, ds=None):
    ds = ds or [d]
    topo_ = binding.CRF_GRID8 if d["conn"] == 8 else binding.CRF_GRID4
    with binding.CRF(topo_, d["L"], d["H"], d["W"], batch=B) as crf:
        crf.set_unary(np.stack([x["U"] for x in ds]) if B > 1 else d["U"])
        w = np.stack([x["w"] for x in ds]) if B > 1 else d["w"]
        crf.set_pairwise(d["mu"], (w * w_scale).astype(np.float32))
        lam, _ = crf.lipschitz()
    return lam


def test_step_constant_large_batch_strided_form(env):
    """40 instances of 128 x 128: too many pixels per block for the shared-
    memory form, so the cooperative launch takes the strided form; every
    instance's constant equals the one its single-instance handle (staged
    form) computes."""
    binding, oracle, torch = env
    ds = [synth.random_grid(128, 128, 5, 8, seed=1200 + i, symmetric=True) for i in range(40)]
    for d in ds:
        d["mu"] = ds[0]["mu"]
    lam_b = _lipschitz(binding, ds[0], B=40, ds=ds)
    for i in (0, 17, 39):
        lam_1 = _lipschitz(binding, ds[i])
        assert math.isclose(lam_b[i], lam_1[0], rel_tol=1e-8)


def test_step_constant_fp64_form_for_extreme_weights(env):
    """Weights scaled by 2^-45 fall outside the double-float range test and
    take the FP64 two-kernel form; Lambda scales exactly with the weights."""
    binding, oracle, torch = env
    d = synth.random_grid(61, 47, 6, 8, seed=1300, symmetric=True)
    lam = _lipschitz(binding, d)[0]
    lam_s = _lipschitz(binding, d, w_scale=2.0 ** -45)[0]
    assert math.isclose(lam_s * 2.0 ** 45, lam, rel_tol=1e-8)


def test_step_constant_fp64_form_for_many_instances(env):
    """More instances than SMs: the FP64 two-kernel form runs (no
    cooperative launch); each constant equals the dense eigen-solve."""
    binding, oracle, torch = env
    ds = [synth.random_grid(5, 6, 3, 8, seed=1400 + i, symmetric=True) for i in range(160)]
    for d in ds:
        d["mu"] = ds[0]["mu"]
    lam = _lipschitz(binding, ds[0], B=160, ds=ds)
    for i in (0, 81, 159):
        ref = oracle_model(oracle, ds[i]).hessian_eigenvalues(projected=True)[-1]
        assert math.isclose(lam[i], ref, rel_tol=1e-8, abs_tol=1e-12)


@pytest.mark.parametrize("Hh,Ww,L,conn,sym,B", [(64, 64, 2, 4, True, 1), (37, 45, 3, 8, False, 2),
                                              (21, 30, 8, 8, True, 1), (19, 23, 13, 4, False, 3),
                                              (1, 1, 2, 8, True, 1), (7, 1, 5, 8, False, 1)])
def test_resident_loop_matches_step_loop(env, Hh, Ww, L, conn, sym, B):
    """The one-launch loop of small grids against the launch-per-step loop:
    states, free-energy traces, stop counts and the final F agree to FP32
    rounding, and the trajectory against the oracle's."""
    binding, oracle, torch = env
    ds = [synth.random_grid(Hh, Ww, L, conn, seed=1500 + 11 * i + L, symmetric=sym) for i in range(B)]
    for d in ds:
        d["mu"] = ds[0]["mu"]
    topo_ = binding.CRF_GRID8 if conn == 8 else binding.CRF_GRID4
    out = []
    for resident in (True, False):
        with binding.CRF(topo_, L, Hh, Ww, batch=B) as crf:
            crf.use_resident(resident)
            crf.set_unary(np.stack([d["U"] for d in ds]) if B > 1 else ds[0]["U"])
            crf.set_pairwise(ds[0]["mu"], np.stack([d["w"] for d in ds]) if B > 1 else ds[0]["w"])
            crf.iterate(40, eta=0.35, final_free_energy=True)
            out.append((crf.log_marginals().astype(np.float64), crf.free_energy_trace(40),
                        crf.free_energy()))
            crf.iterate(9, eta=0.3, reset=True)   # odd count: the final buffer flips
            out.append((crf.log_marginals().astype(np.float64), crf.free_energy_trace(9), None))
            its = crf.iterate(400, eta=0.35, reset=True, rel_tol=1e-6, want_iters=True)
            out.append((None, None, its.copy()))
    (s_r, tr_r, F_r), (s9_r, tr9_r, _), (_, _, it_r), (s_s, tr_s, F_s), (s9_s, tr9_s, _), (_, _, it_s) = out
    # the stopping rule fires at the same step, up to a tie decided by rounding
    assert np.abs(it_r.astype(int) - it_s.astype(int)).max() <= 1
    assert np.abs(np.exp(s_r) - np.exp(s_s)).max() <= 2e-5
    assert np.abs(np.exp(s9_r) - np.exp(s9_s)).max() <= 2e-5
    for b in range(B):
        scale = max(1.0, float(np.abs(tr_s[b]).max()))
        assert np.abs(tr_r[b] - tr_s[b]).max() <= 1e-5 * scale
        assert abs(F_r[b] - F_s[b]) <= 1e-5 * max(1.0, abs(F_s[b]))
        assert np.abs(tr9_r[b] - tr9_s[b]).max() <= 1e-5 * max(1.0, float(np.abs(tr9_s[b]).max()))
    # against the oracle, 9 steps from q^0
    d = ds[0]
    s_ref, F_ref = oracle_model(oracle, d).parallel_prox(0.3, 9)
    assert np.abs(np.exp(s9_r[0]) - np.exp(s_ref)).max() <= TOL_Q
    assert np.abs(tr9_r[0] - F_ref[:9]).max() <= 1e-5 * max(1.0, float(np.abs(F_ref).max()))


def test_pinned_host_buffers_match_pageable(env):
    """Host buffers in page-locked memory are read and written in place by the
    layout kernels (no staging copy); results are bit-identical to pageable
    buffers, also for a view at an odd float offset inside a larger pinned
    allocation."""
    binding, oracle, torch = env
    d = synth.random_grid(37, 45, 5, 8, seed=77, symmetric=False)
    n = 37 * 45
    out = []
    for mode in ("pageable", "pinned", "pinned_view"):
        U = torch.from_numpy(d["U"]).clone()
        q = torch.empty((1, n, 5))
        s = torch.empty((1, n, 5))
        if mode == "pinned":
            U, q, s = U.pin_memory(), q.pin_memory(), s.pin_memory()
        elif mode == "pinned_view":
            big = torch.empty(3 * n * 5 + 7).pin_memory()
            Uv = big[3:3 + n * 5].view(n, 5)
            Uv.copy_(U)
            U = Uv
            q = big[3 + n * 5:3 + 2 * n * 5].view(1, n, 5)
            s = big[3 + 2 * n * 5:3 + 3 * n * 5].view(1, n, 5)
        with make(binding, torch, d) as crf:
            crf.use_resident(False)
            crf.set_unary(U)
            crf.set_pairwise(d["mu"], d["w"])
            crf.iterate(6, eta=0.3)
            crf.marginals(q)
            crf.log_marginals(s)
            out.append((q.clone().numpy(), s.clone().numpy(), crf.free_energy()[0]))
    for q_, s_, F_ in out[1:]:
        assert np.array_equal(q_, out[0][0]) and np.array_equal(s_, out[0][1]) and F_ == out[0][2]
