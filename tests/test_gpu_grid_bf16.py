"""GPU parity of the BF16 tensor-core form of the grid step.

The L x L product m = mu S runs on the tensor cores with BF16 operands and
FP32 accumulation; everything else stays FP32.  Three kinds of checks:
  - exact: one-hot states, weights that are multiples of 1/8 and mu entries
    that are multiples of 1/16 make every operand exactly representable in
    BF16, so one tensor-core step must match the oracle to FP32 rounding
    (catches any layout, transposition or padding error of the operands);
  - rounding: a general single step within |dq|max <= 1e-2;
  - trajectories after FP32 refinement: |dq|max <= 1e-2, |dF| <= 1e-3 |F|
    (tests.helpers.f_close).
"""
import numpy as np
import pytest

from paper_1511_06103_gb300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

TOL_Q_BF16 = 1e-2
TOL_F_BF16 = 1e-3


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
    return oracle.Model.grid(f64(d["U"]), f64(d["mu"]), f64(d["w"]), d["H"], d["W"], d["conn"])


def run(binding, torch, d, eta, iters, precision, refine=0, s0=None):
    dev = torch.device("cuda:0")
    topo = binding.CRF_GRID8 if d["conn"] == 8 else binding.CRF_GRID4
    with binding.CRF(topo, d["L"], d["H"], d["W"], precision=precision) as crf:
        crf.set_unary(torch.from_numpy(d["U"]).to(dev))
        crf.set_pairwise(torch.from_numpy(d["mu"]).to(dev), torch.from_numpy(d["w"]).to(dev))
        if s0 is not None:
            crf.set_state(torch.from_numpy(np.ascontiguousarray(s0, np.float32)).to(dev))
        crf.iterate(iters, eta=eta, refine_fp32=refine)
        s = crf.log_marginals()[0].astype(np.float64)
        F = crf.free_energy()[0]
        torch.cuda.synchronize()
        return s, F


def exact_instance(H, W, L, conn, sym, seed):
    rng = np.random.default_rng(seed)
    d = synth.random_grid(H, W, L, conn, seed=seed, symmetric=sym)
    mu = rng.integers(-16, 17, size=(L, L)) / 16.0
    if sym:
        mu = np.triu(mu) + np.triu(mu, 1).T
    d["mu"] = mu.astype(np.float32)
    mask = d["w"] != 0
    d["w"] = (rng.integers(1, 17, size=d["w"].shape) / 8.0 * mask).astype(np.float32)
    lab = rng.integers(0, L, H * W)
    s0 = np.full((H * W, L), -1e30, np.float32)
    s0[np.arange(H * W), lab] = 0.0
    return d, s0


@pytest.mark.parametrize("Hh,Ww,L,conn,sym", [
    (19, 45, 21, 8, True), (19, 45, 21, 8, False), (13, 70, 21, 4, False), (9, 33, 32, 8, False),
    (11, 40, 17, 4, True), (10, 35, 16, 8, False), (12, 34, 8, 4, True), (8, 40, 3, 8, False),
    (7, 9, 2, 4, True), (1, 1, 5, 8, False),
])
def test_bf16_step_exact_operands(env, Hh, Ww, L, conn, sym):
    binding, oracle, torch = env
    d, s0 = exact_instance(Hh, Ww, L, conn, sym, seed=Hh * 17 + L * 3 + conn + int(sym))
    s_ref = oracle_model(oracle, d).prox_step(0.45, f64(s0))
    s, _ = run(binding, torch, d, 0.45, 1, binding.CRF_BF16, s0=s0)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= 1e-5


@pytest.mark.parametrize("L,conn,sym", [(21, 8, True), (21, 4, False), (32, 8, False), (12, 8, True), (5, 4, True)])
def test_bf16_single_step_rounding(env, L, conn, sym):
    binding, oracle, torch = env
    d = synth.random_grid(21, 50, L, conn, seed=300 + L, symmetric=sym)
    s0 = synth.random_logq(21 * 50, L, seed=7 + L)
    s_ref = oracle_model(oracle, d).prox_step(0.4, f64(s0))
    s, _ = run(binding, torch, d, 0.4, 1, binding.CRF_BF16, s0=s0)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= TOL_Q_BF16
    assert np.all(np.isfinite(s))


@pytest.mark.parametrize("conn,sym", [(8, True), (4, False)])
def test_bf16_trajectory_refined(env, conn, sym):
    """40 x 37, L = 21, 100 steps at the step-size constant: 98 tensor-core
    steps and 2 FP32 refinement steps against 100 oracle steps."""
    binding, oracle, torch = env
    d = synth.random_grid(40, 37, 21, conn, seed=500 + conn, symmetric=sym)
    topo = binding.CRF_GRID8 if conn == 8 else binding.CRF_GRID4
    with binding.CRF(topo, 21, 40, 37) as crf:
        crf.set_pairwise(d["mu"], d["w"])
        _, eta = crf.lipschitz()
    eta = float(np.float32(eta[0]))
    s_ref, F_ref = oracle_model(oracle, d).parallel_prox(eta, 100)
    s, F = run(binding, torch, d, eta, 98, binding.CRF_BF16, refine=2)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= TOL_Q_BF16
    assert H.f_close(F, F_ref[-1], 40 * 37, TOL_F_BF16)


def test_bf16_segmentation_full_size(env):
    """512 x 512, L = 21, 8-connected: 98 + 2 refined steps against the FP32
    form at equal iterations, and the tensor-core run repeats bit for bit."""
    binding, oracle, torch = env
    d = synth.segmentation_grid()
    with binding.CRF(binding.CRF_GRID8, 21, 512, 512) as crf:
        crf.set_pairwise(d["mu"], d["w"])
        _, eta = crf.lipschitz()
    eta = float(eta[0])
    s32, F32 = run(binding, torch, d, eta, 100, binding.CRF_FP32)
    s16, F16 = run(binding, torch, d, eta, 98, binding.CRF_BF16, refine=2)
    s16b, F16b = run(binding, torch, d, eta, 98, binding.CRF_BF16, refine=2)
    assert np.array_equal(s16, s16b) and F16 == F16b
    assert np.abs(np.exp(s16) - np.exp(s32)).max() <= TOL_Q_BF16
    assert H.f_close(F16, F32, 512 * 512, TOL_F_BF16)
    # sampled pixels of the first step against the oracle
    m = oracle_model(oracle, d)
    s0 = m.init_logq()
    s1_ref = m.prox_step(eta, s0)
    s1, _ = run(binding, torch, d, eta, 1, binding.CRF_BF16)
    rows = np.random.default_rng(3).choice(512 * 512, size=4096, replace=False)
    assert np.abs(np.exp(s1[rows]) - np.exp(s1_ref[rows])).max() <= TOL_Q_BF16
