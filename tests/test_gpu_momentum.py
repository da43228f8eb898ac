"""GPU parity of OURS-MOMENTUM and OURS-ADAM (Sec. 3.4-3.5) against the FP64
oracle, with the FP32 tolerances of the fixed step: |dq|max <= 1e-5 and
|dF| <= 1e-6 |F| (tests.helpers.f_close) along the trajectory."""
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
    return oracle.Model.grid(f64(d["U"]), f64(d["mu"]), f64(d["w"]), d["H"], d["W"], d["conn"])


def run(binding, inst, iters, resident=True, **kw):
    topo = binding.CRF_GRID8 if inst["conn"] == 8 else binding.CRF_GRID4
    with binding.CRF(topo, inst["L"], inst["H"], inst["W"]) as crf:
        crf.use_resident(resident)
        crf.set_unary(inst["U"])
        crf.set_pairwise(inst["mu"], inst["w"])
        crf.iterate(iters, reset=True, **kw)
        s = crf.log_marginals()[0].astype(np.float64)
        trace = crf.free_energy_trace(iters)[0]
        F = crf.free_energy()[0]
        return s, trace, F


@pytest.mark.parametrize("Hh,Ww,L,conn,sym", [(40, 37, 5, 8, False), (33, 70, 21, 8, True), (21, 30, 2, 4, True)])
def test_momentum_trajectory(env, Hh, Ww, L, conn, sym):
    binding, oracle, torch = env
    d = synth.random_grid(Hh, Ww, L, conn, seed=600 + L, symmetric=sym)
    eta, g1, T = 0.12, 0.95, 40
    s, trace, F = run(binding, d, T, eta=eta, rule=binding.MF_RULE_MOMENTUM, gamma1=g1)
    s_ref, F_ref = model(oracle, d).parallel_prox_momentum(eta, g1, T)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= 1e-5
    assert f_close(trace, F_ref[:-1], Hh * Ww)
    assert f_close(F, F_ref[-1], Hh * Ww)


@pytest.mark.parametrize("Hh,Ww,L,conn,sym", [(40, 37, 5, 8, False), (33, 70, 21, 8, True), (21, 30, 2, 4, True)])
def test_adam_trajectory(env, Hh, Ww, L, conn, sym):
    binding, oracle, torch = env
    d = synth.random_grid(Hh, Ww, L, conn, seed=700 + L, symmetric=sym)
    d0, g1, g2, eps, T = 6.0, 0.99, 0.999, 1e-8, 40
    s, trace, F = run(binding, d, T, rule=binding.MF_RULE_ADAM, d=d0, gamma1=g1, gamma2=g2, epsilon=eps)
    s_ref, F_ref = model(oracle, d).parallel_prox_adam(d0, g1, g2, eps, T)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= 1e-5
    assert f_close(trace, F_ref[:-1], Hh * Ww)
    assert f_close(F, F_ref[-1], Hh * Ww)


def test_adam_with_lambda_damping_on_denoising(env):
    """d <= 0 takes the step-size constant as the damping d0."""
    binding, oracle, torch = env
    d = synth.binary_denoising()
    topo = binding.CRF_GRID4
    with binding.CRF(topo, 2, 64, 64) as crf:
        crf.set_pairwise(d["mu"], d["w"])
        lam, _ = crf.lipschitz()
    s, trace, F = run(binding, d, 50, rule=binding.MF_RULE_ADAM, d=0.0, gamma1=0.99, gamma2=0.999, epsilon=1e-8)
    s_ref, F_ref = model(oracle, d).parallel_prox_adam(float(np.float32(lam[0])), 0.99, 0.999, 1e-8, 50)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= 1e-5
    assert f_close(F, F_ref[-1], 64 * 64)


def test_momentum_without_memory_is_the_fixed_step(env):
    """gamma1 = 0: the momentum rule takes the fixed step.  The fixed rule's
    kernel groups its FP32 arithmetic differently (a = -eta m + c with
    c = -eta U + (1 - eta) log q), so the two agree to FP32 rounding, within
    the trajectory bounds."""
    binding, oracle, torch = env
    d = synth.random_grid(19, 45, 8, 8, seed=9, symmetric=False)
    a = run(binding, d, 20, eta=0.3, rule=binding.MF_RULE_MOMENTUM, gamma1=0.0)
    b = run(binding, d, 20, resident=False, eta=0.3)
    assert np.abs(np.exp(a[0]) - np.exp(b[0])).max() <= 1e-5
    assert f_close(a[1], b[1], 19 * 45)


def test_momentum_rejected_on_dense_and_bf16(env):
    binding, oracle, torch = env
    dd = synth.dense_gaussian(side=8, L=3, seed=1)
    with binding.CRF(binding.CRF_DENSE_GAUSS, 3, 8, 8) as crf:
        crf.set_unary(dd["U"])
        crf.set_pairwise(dd["mu"], dd["feats"], theta=np.array(dd["theta"], np.float32))
        with pytest.raises(binding.ProxMFError, match="UNSUPPORTED"):
            crf.iterate(2, eta=0.3, rule=binding.MF_RULE_MOMENTUM)
    d = synth.random_grid(8, 8, 3, 4, seed=2)
    with binding.CRF(binding.CRF_GRID4, 3, 8, 8, precision=binding.CRF_BF16) as crf:
        crf.set_unary(d["U"])
        crf.set_pairwise(d["mu"], d["w"])
        with pytest.raises(binding.ProxMFError, match="UNSUPPORTED"):
            crf.iterate(2, rule=binding.MF_RULE_ADAM, d=2.0)
