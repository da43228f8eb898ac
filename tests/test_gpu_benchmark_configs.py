"""GPU parity against the FP64 oracle at the full sizes the benchmark times,
in the launch configuration it times (mf_iterate from q^0 with the automatic
step eta = 1/(1 + max(Lambda, 0)) computed on the device, whole trajectories).

  - segmentation-shaped grid, 512 x 512, L = 21, 8-connected, 100 steps:
    FP32 form |dq|max <= 1e-5 on every variable and label, and the whole F
    trace within |dF| <= 1e-6 |F|; BF16 tensor-core form (98 steps + 2 FP32
    refinement steps) |dq|max <= 1e-2 and |dF| <= 1e-3 |F|;
  - fully connected Gaussian CRF, N = 96 x 96 = 9216, L = 21, 30 steps: the
    same bounds, the BF16 form with 28 + 2 steps.
The free-energy bound is the plain relative one, with no floor.  For the
BF16 form it applies after refinement (the final F and the F read by the two
FP32 steps); the F of a tensor-core grid step uses its BF16 messages (mu and
the neighbour sums rounded to BF16) and is held to a sanity bound of 2e-2.

The oracle runs at the device's step size rounded to FP32 (the device holds
eta in FP32), so both sides take the same step.
"""
import math

import numpy as np
import pytest

from paper_1511_06103_gb300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

TOL_Q, TOL_F = 1e-5, 1e-6
TOL_Q_BF16, TOL_F_BF16 = 1e-2, 1e-3


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


# ------------------------------------------------------------ 512 x 512 grid

SEG_ITERS = 100


@pytest.fixture(scope="module")
def seg(env):
    """The benchmark instance, its device step size and the oracle's 100-step
    trajectory at that step (about 10 s of CPU)."""
    binding, oracle, torch = env
    d = synth.segmentation_grid()
    with binding.CRF(binding.CRF_GRID8, 21, 512, 512) as crf:
        crf.set_unary(d["U"])
        crf.set_pairwise(d["mu"], d["w"])
        lam, eta = crf.lipschitz()
    eta32 = float(np.float32(eta[0]))
    m = oracle.Model.grid(f64(d["U"]), f64(d["mu"]), f64(d["w"]), 512, 512, 8)
    s_ref, F_ref = m.parallel_prox(eta32, SEG_ITERS)
    return d, float(lam[0]), eta32, s_ref, F_ref


def run_seg(binding, torch, d, iters, precision, refine=0):
    dev = torch.device("cuda:0")
    with binding.CRF(binding.CRF_GRID8, 21, 512, 512, precision=precision) as crf:
        crf.set_unary(torch.from_numpy(d["U"]).to(dev))
        crf.set_pairwise(torch.from_numpy(d["mu"]).to(dev), torch.from_numpy(d["w"]).to(dev))
        crf.iterate(iters, eta=0.0, reset=True, final_free_energy=True, refine_fp32=refine)
        s = crf.log_marginals()[0].astype(np.float64)
        F = crf.free_energy()[0]
        trace = crf.free_energy_trace(iters + refine)[0]
        _, eta = crf.lipschitz()
        torch.cuda.synchronize()
    return s, F, trace, float(np.float32(eta[0]))


def test_segmentation_grid_full_solve(env, seg):
    binding, oracle, torch = env
    d, lam, eta, s_ref, F_ref = seg
    s, F, trace, eta_dev = run_seg(binding, torch, d, SEG_ITERS, binding.CRF_FP32)
    assert eta_dev == eta
    dq = np.abs(np.exp(s) - np.exp(s_ref)).max()
    assert dq <= TOL_Q, dq
    assert H.f_rel_close(trace, F_ref[:-1], TOL_F), H.f_rel_err(trace, F_ref[:-1])
    assert H.f_rel_close(F, F_ref[-1], TOL_F), H.f_rel_err(F, F_ref[-1])


def test_segmentation_grid_full_solve_bf16(env, seg):
    binding, oracle, torch = env
    d, lam, eta, s_ref, F_ref = seg
    s, F, trace, eta_dev = run_seg(binding, torch, d, SEG_ITERS - 2, binding.CRF_BF16, refine=2)
    assert eta_dev == eta
    dq = np.abs(np.exp(s) - np.exp(s_ref)).max()
    assert dq <= TOL_Q_BF16, dq
    # after refinement: the final F and the F of the two FP32 steps
    assert H.f_rel_close(F, F_ref[-1], TOL_F_BF16), H.f_rel_err(F, F_ref[-1])
    assert H.f_rel_close(trace[-2:], F_ref[-3:-1], TOL_F_BF16), H.f_rel_err(trace[-2:], F_ref[-3:-1])
    # the F of a tensor-core step is taken with its BF16 messages, i.e. with
    # mu and the neighbour sums rounded to BF16: a sanity bound only
    assert H.f_rel_close(trace[:-2], F_ref[:-3], 2e-2), H.f_rel_err(trace[:-2], F_ref[:-3])


# ------------------------------------------------------- dense N = 9216

DENSE_ITERS = 30


@pytest.fixture(scope="module")
def dense(env):
    binding, oracle, torch = env
    d = synth.dense_gaussian()
    side = int(round(math.sqrt(d["N"])))
    with binding.CRF(binding.CRF_DENSE_GAUSS, d["L"], side, side) as crf:
        crf.set_unary(d["U"])
        crf.set_pairwise(d["mu"], d["feats"], theta=np.array(d["theta"], np.float32))
        _, eta = crf.lipschitz()
    eta32 = float(np.float32(eta[0]))
    K = oracle.dense_gauss_kernel(f64(d["feats"]), *d["theta"])
    m = oracle.Model.dense(f64(d["U"]), f64(d["mu"]), K)
    s_ref, F_ref = m.parallel_prox(eta32, DENSE_ITERS)
    return d, side, eta32, s_ref, F_ref


def run_dense(binding, torch, d, side, iters, precision, refine=0, fly=False):
    dev = torch.device("cuda:0")
    with binding.CRF(binding.CRF_DENSE_GAUSS, d["L"], side, side, precision=precision) as crf:
        if fly:
            crf.dense_on_the_fly(True)
        crf.set_unary(torch.from_numpy(d["U"]).to(dev))
        crf.set_pairwise(torch.from_numpy(d["mu"]).to(dev), torch.from_numpy(d["feats"]).to(dev),
                         theta=np.array(d["theta"], np.float32))
        crf.iterate(iters, eta=0.0, reset=True, final_free_energy=True, refine_fp32=refine)
        s = crf.log_marginals()[0].astype(np.float64)
        F = crf.free_energy()[0]
        trace = crf.free_energy_trace(iters + refine)[0]
        torch.cuda.synchronize()
    return s, F, trace


def test_dense_full_solve(env, dense):
    binding, oracle, torch = env
    d, side, eta, s_ref, F_ref = dense
    s, F, trace = run_dense(binding, torch, d, side, DENSE_ITERS, binding.CRF_FP32)
    dq = np.abs(np.exp(s) - np.exp(s_ref)).max()
    assert dq <= TOL_Q, dq
    assert H.f_rel_close(trace, F_ref[:-1], TOL_F), H.f_rel_err(trace, F_ref[:-1])
    assert H.f_rel_close(F, F_ref[-1], TOL_F), H.f_rel_err(F, F_ref[-1])


@pytest.mark.parametrize("fly", [False, True], ids=["stored_K", "K_in_kernel"])
def test_dense_full_solve_bf16(env, dense, fly):
    binding, oracle, torch = env
    d, side, eta, s_ref, F_ref = dense
    s, F, trace = run_dense(binding, torch, d, side, DENSE_ITERS - 2, binding.CRF_BF16, refine=2, fly=fly)
    dq = np.abs(np.exp(s) - np.exp(s_ref)).max()
    assert dq <= TOL_Q_BF16, dq
    assert H.f_rel_close(F, F_ref[-1], TOL_F_BF16), H.f_rel_err(F, F_ref[-1])
    # the dense form keeps mu in FP32 (only K and q are BF16): its whole trace
    # is within the bound
    assert H.f_rel_close(trace, F_ref[:-1], TOL_F_BF16), H.f_rel_err(trace, F_ref[:-1])
