"""GPU parity of the fully connected (dense Gaussian kernel) path against the
FP64 oracle, through the C ABI."""
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


def oracle_model(oracle, d):
    K = oracle.dense_gauss_kernel(f64(d["feats"]), *d["theta"])
    return oracle.Model.dense(f64(d["U"]), f64(d["mu"]), K)


def make(binding, d, batch=1):
    side = int(round(math.sqrt(d["N"])))
    return binding.CRF(binding.CRF_DENSE_GAUSS, d["L"], side, d["N"] // side, batch=batch)


def gpu_run(binding, torch, d, eta, iters, s0=None):
    dev = torch.device("cuda:0")
    with make(binding, d) as crf:
        crf.set_unary(torch.from_numpy(d["U"]).to(dev))
        crf.set_pairwise(torch.from_numpy(d["mu"]).to(dev), torch.from_numpy(d["feats"]).to(dev),
                         theta=np.array(d["theta"], np.float32))
        if s0 is not None:
            crf.set_state(torch.from_numpy(np.ascontiguousarray(s0, np.float32)).to(dev))
        crf.iterate(iters, eta=eta)
        s = crf.log_marginals()[0].astype(np.float64)
        F = crf.free_energy()[0]
        trace = crf.free_energy_trace(iters)[0] if iters > 0 else np.zeros(0)
        torch.cuda.synchronize()
        return s, F, trace


@pytest.mark.parametrize("side,L", [(10, 2), (10, 3), (9, 5), (12, 8), (10, 21), (11, 24), (7, 1)])
def test_dense_single_step_parity(env, side, L):
    binding, oracle, torch = env
    d = synth.dense_gaussian(side=side, L=L, seed=side * 31 + L)
    s0 = synth.random_logq(d["N"], L, seed=3 + L)
    m = oracle_model(oracle, d)
    s_ref = m.prox_step(0.3, f64(s0))
    F_ref = m.free_energy(np.exp(f64(s0)))
    s, _, trace = gpu_run(binding, torch, d, 0.3, 1, s0=s0)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= TOL_Q_STEP
    assert f_close(trace[0], F_ref, d["N"])


def test_dense_trajectory_parity(env):
    binding, oracle, torch = env
    d = synth.dense_gaussian(side=16, L=21, seed=5)
    m = oracle_model(oracle, d)
    lam = m.hessian_eigenvalues(projected=True)[-1] if d["N"] * d["L"] <= 2048 else None
    eta = 0.2 if lam is None else oracle.step_size(lam)
    s_ref, F_ref = m.parallel_prox(eta, 30)
    s, F, trace = gpu_run(binding, torch, d, eta, 30)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= TOL_Q
    assert f_close(trace, F_ref[:-1], d["N"])
    assert f_close(F, F_ref[-1], d["N"])


def test_dense_full_size_first_step_sampled(env):
    """N = 96 x 96 = 9216, L = 21 (the fully connected workload): one step from
    q^0 = softmax(-U), compared on sampled variables, and F(q^0)."""
    binding, oracle, torch = env
    d = synth.dense_gaussian()
    m = oracle_model(oracle, d)
    s0 = m.init_logq()
    rows = np.random.default_rng(0).choice(d["N"], size=64, replace=False)
    eta = 0.05
    s_ref = m.prox_step_rows(eta, s0, rows)
    s, F, trace = gpu_run(binding, torch, d, eta, 1)
    assert np.abs(np.exp(s[rows]) - np.exp(s_ref)).max() <= TOL_Q_STEP
    F0 = m.free_energy(np.exp(s0))
    assert f_close(trace[0], F0, d["N"])


def test_dense_step_constant(env):
    binding, oracle, torch = env
    d = synth.dense_gaussian(side=6, L=4, seed=92)
    d["mu"] = (3.0 * d["mu"]).astype(np.float32)
    lam_ref = oracle_model(oracle, d).hessian_eigenvalues(projected=True)[-1]
    with make(binding, d) as crf:
        crf.set_unary(d["U"])
        crf.set_pairwise(d["mu"], d["feats"], theta=np.array(d["theta"], np.float32))
        lam, _ = crf.lipschitz()
    # the device builds K in FP32: agreement to FP32 rounding of the weights
    assert math.isclose(lam[0], lam_ref, rel_tol=2e-6)


@pytest.mark.parametrize("side,L,B", [(8, 5, 2), (9, 2, 3)])
def test_dense_batch_independent(env, side, L, B):
    """Instances of a batch solve as they do alone (9 x 9, L = 2: odd N with
    two stored labels, so later instances start off a 16-byte boundary)."""
    binding, oracle, torch = env
    ds = [synth.dense_gaussian(side=side, L=L, seed=40 + i) for i in range(B)]
    for d in ds:
        d["mu"] = ds[0]["mu"]
    with binding.CRF(binding.CRF_DENSE_GAUSS, L, side, side, batch=B) as crf:
        crf.set_unary(np.stack([d["U"] for d in ds]))
        crf.set_pairwise(ds[0]["mu"], np.stack([d["feats"] for d in ds]), theta=np.array(ds[0]["theta"], np.float32))
        crf.iterate(10, eta=0.3)
        sb = crf.log_marginals()
    for i, d in enumerate(ds):
        s, _, _ = gpu_run(binding, torch, d, 0.3, 10)
        assert np.array_equal(sb[i].astype(np.float64), s)


def test_dense_rejects_asymmetric_mu(env):
    binding, oracle, torch = env
    d = synth.dense_gaussian(side=4, L=3, seed=1)
    mu = d["mu"].copy()
    mu[0, 1] += 0.5
    with make(binding, d) as crf:
        crf.set_unary(d["U"])
        with pytest.raises(binding.ProxMFError) as e:
            crf.set_pairwise(mu, d["feats"], theta=np.array(d["theta"], np.float32))
        assert e.value.status == -1


# ---------------------------------------------------------------- BF16 form
# BF16 tensor-core messages, FP32 state; tolerances after FP32 refinement:
# |dq|max <= 1e-2 and |dF|/|F| <= 1e-3.

TOL_Q_BF16 = 1e-2
TOL_F_BF16 = 1e-3


def gpu_run_bf16(binding, torch, d, eta, iters, refine=0, s0=None, fly=False):
    dev = torch.device("cuda:0")
    side = int(round(math.sqrt(d["N"])))
    with binding.CRF(binding.CRF_DENSE_GAUSS, d["L"], side, d["N"] // side, precision=binding.CRF_BF16) as crf:
        crf.dense_on_the_fly(fly)
        crf.set_unary(torch.from_numpy(d["U"]).to(dev))
        crf.set_pairwise(torch.from_numpy(d["mu"]).to(dev), torch.from_numpy(d["feats"]).to(dev),
                         theta=np.array(d["theta"], np.float32))
        if s0 is not None:
            crf.set_state(torch.from_numpy(np.ascontiguousarray(s0, np.float32)).to(dev))
        crf.iterate(iters, eta=eta, refine_fp32=refine)
        s = crf.log_marginals()[0].astype(np.float64)
        F = crf.free_energy()[0]
        trace = crf.free_energy_trace(iters + refine)[0]
        torch.cuda.synchronize()
        return s, F, trace


@pytest.mark.parametrize("side,L", [(10, 21), (12, 5), (9, 2)])
def test_dense_bf16_single_step(env, side, L):
    binding, oracle, torch = env
    d = synth.dense_gaussian(side=side, L=L, seed=side * 7 + L)
    s0 = synth.random_logq(d["N"], L, seed=11 + L)
    m = oracle_model(oracle, d)
    s_ref = m.prox_step(0.3, f64(s0))
    s, _, _ = gpu_run_bf16(binding, torch, d, 0.3, 1, s0=s0)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= TOL_Q_BF16
    assert np.all(np.isfinite(s))


def test_dense_bf16_trajectory_refined(env):
    binding, oracle, torch = env
    d = synth.dense_gaussian(side=16, L=21, seed=5)
    m = oracle_model(oracle, d)
    s_ref, F_ref = m.parallel_prox(0.2, 35)
    s, F, trace = gpu_run_bf16(binding, torch, d, 0.2, 30, refine=5)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= TOL_Q_BF16
    assert H.f_close(F, F_ref[-1], d["N"], TOL_F_BF16)


def test_dense_bf16_full_size_sampled(env):
    """N = 9216, L = 21: one BF16 step from q^0 on sampled rows, and the
    tensor-core run is deterministic."""
    binding, oracle, torch = env
    d = synth.dense_gaussian()
    m = oracle_model(oracle, d)
    s0 = m.init_logq()
    rows = np.random.default_rng(1).choice(d["N"], size=64, replace=False)
    s_ref = m.prox_step_rows(0.05, s0, rows)
    s, _, _ = gpu_run_bf16(binding, torch, d, 0.05, 1)
    assert np.abs(np.exp(s[rows]) - np.exp(s_ref)).max() <= TOL_Q_BF16
    s1, F1, _ = gpu_run_bf16(binding, torch, d, 0.05, 6, refine=1)
    s2, F2, _ = gpu_run_bf16(binding, torch, d, 0.05, 6, refine=1)
    assert np.array_equal(s1, s2) and F1 == F2


def test_dense_mid_size_trajectories(env):
    """N = 40 x 40 = 1600, L = 21, 30 steps at the step-size constant: the FP32
    form within the FP32 tolerances, the BF16 form (28 tensor-core + 2 FP32
    steps) within the BF16 ones."""
    binding, oracle, torch = env
    d = synth.dense_gaussian(side=40, L=21, seed=8)
    with make(binding, d) as crf:
        crf.set_unary(d["U"])
        crf.set_pairwise(d["mu"], d["feats"], theta=np.array(d["theta"], np.float32))
        _, eta = crf.lipschitz()
    eta = float(np.float32(eta[0]))
    m = oracle_model(oracle, d)
    s_ref, F_ref = m.parallel_prox(eta, 30)
    s, F, _ = gpu_run(binding, torch, d, eta, 30)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= TOL_Q
    assert f_close(F, F_ref[-1], d["N"])
    s, F, _ = gpu_run_bf16(binding, torch, d, eta, 28, refine=2)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= TOL_Q_BF16
    assert H.f_close(F, F_ref[-1], d["N"], TOL_F_BF16)


# ------------------------------------------------ BF16 form, K computed in the kernel
# The on-the-fly form builds each 128 x 64 block of K from the features in
# the kernel (K_ij = 2^(-|s (f_i - f_j)|^2), zero diagonal) instead of reading
# the BF16 copy: the same rounding to BF16 and the same tolerances.


@pytest.mark.parametrize("side,L", [(10, 21), (12, 5), (9, 2), (13, 17)])
def test_dense_on_the_fly_single_step(env, side, L):
    binding, oracle, torch = env
    d = synth.dense_gaussian(side=side, L=L, seed=side * 7 + L)
    s0 = synth.random_logq(d["N"], L, seed=11 + L)
    m = oracle_model(oracle, d)
    s_ref = m.prox_step(0.3, f64(s0))
    s, _, _ = gpu_run_bf16(binding, torch, d, 0.3, 1, s0=s0, fly=True)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= TOL_Q_BF16
    assert np.all(np.isfinite(s))


def test_dense_on_the_fly_trajectory_refined(env):
    binding, oracle, torch = env
    d = synth.dense_gaussian(side=16, L=21, seed=5)
    m = oracle_model(oracle, d)
    s_ref, F_ref = m.parallel_prox(0.2, 35)
    s, F, trace = gpu_run_bf16(binding, torch, d, 0.2, 30, refine=5, fly=True)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= TOL_Q_BF16
    assert H.f_close(F, F_ref[-1], d["N"], TOL_F_BF16)
    for t in range(35):
        assert H.f_close(trace[t], F_ref[t], d["N"], 2e-2)


def test_dense_on_the_fly_agrees_with_the_stored_copy(env):
    """Both forms round K to BF16; the weights differ only where the two
    exponentials round to neighbouring BF16 values, so one step from the same
    state agrees far inside the BF16 tolerance, and repeated runs are
    bit-identical."""
    binding, oracle, torch = env
    d = synth.dense_gaussian(side=20, L=21, seed=3)
    s0 = synth.random_logq(d["N"], 21, seed=4)
    s_a, F_a, _ = gpu_run_bf16(binding, torch, d, 0.3, 1, s0=s0, fly=False)
    s_b, F_b, _ = gpu_run_bf16(binding, torch, d, 0.3, 1, s0=s0, fly=True)
    s_c, F_c, _ = gpu_run_bf16(binding, torch, d, 0.3, 1, s0=s0, fly=True)
    assert np.abs(np.exp(s_a) - np.exp(s_b)).max() <= 2e-3
    assert np.array_equal(s_b, s_c) and F_b == F_c


def test_dense_on_the_fly_rejected_on_fp32_handles(env):
    binding, _, _ = env
    d = synth.dense_gaussian(side=8, L=3, seed=1)
    with make(binding, d) as crf:
        with pytest.raises(binding.ProxMFError):
            crf.dense_on_the_fly(True)
