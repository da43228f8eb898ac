"""GPU parity of the adaptive binary step (Sec. 3.3, Eq. hessian):
eta_i = 1/(1 + d q_i0 q_i1) per variable, taken from q^t.  FP32 tolerances
as for the fixed step: single step |dq|max <= 1e-6, trajectories 1e-5 and
|dF| <= 1e-6 |F| (tests.helpers.f_close)."""
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


def crf_for(binding, d, **kw):
    topo = binding.CRF_GRID8 if d["conn"] == 8 else binding.CRF_GRID4
    crf = binding.CRF(topo, d["L"], d["H"], d["W"], **kw)
    crf.set_unary(d["U"])
    crf.set_pairwise(d["mu"], d["w"])
    return crf


@pytest.mark.parametrize("Hh,Ww,conn,sym,dd", [(37, 45, 4, True, 3.0), (21, 70, 8, False, 5.5), (1, 1, 4, True, 2.0)])
def test_adaptive_single_step(env, Hh, Ww, conn, sym, dd):
    binding, oracle, torch = env
    d = synth.random_grid(Hh, Ww, 2, conn, seed=Hh + Ww + conn, symmetric=sym)
    s0 = synth.random_logq(Hh * Ww, 2, seed=8)
    s_ref = model(oracle, d).prox_step_adaptive(dd, f64(s0))
    with crf_for(binding, d) as crf:
        crf.set_state(s0)
        crf.iterate(1, rule=binding.MF_RULE_ADAPTIVE, d=dd)
        s = crf.log_marginals()[0].astype(np.float64)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= 1e-6


def test_adaptive_binary_denoising_trajectory(env):
    """64 x 64 binary denoising, 50 adaptive steps with d = Lambda (the
    step-size constant computed on the device)."""
    binding, oracle, torch = env
    d = synth.binary_denoising()
    with crf_for(binding, d) as crf:
        lam, _ = crf.lipschitz()
        crf.iterate(50, rule=binding.MF_RULE_ADAPTIVE, d=0.0, reset=True)
        s = crf.log_marginals()[0].astype(np.float64)
        trace = crf.free_energy_trace(50)[0]
        F = crf.free_energy()[0]
    dd = float(np.float32(max(lam[0], 0.0)))
    s_ref, F_ref = model(oracle, d).parallel_prox_adaptive(dd, 50)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= 1e-5
    assert f_close(trace, F_ref[:-1], 64 * 64)
    assert f_close(F, F_ref[-1], 64 * 64)


def test_adaptive_graph_replay_and_batch(env):
    """A batch of two instances with their own d (from Lambda), eager and
    replayed as a graph, bit for bit."""
    binding, oracle, torch = env
    ds = [synth.binary_denoising(seed=s) for s in (1, 2)]
    out = []
    for graphs in (False, True):
        with binding.CRF(binding.CRF_GRID4, 2, 64, 64, batch=2) as crf:
            crf.use_graphs(graphs)
            crf.set_unary(np.stack([x["U"] for x in ds]))
            crf.set_pairwise(ds[0]["mu"], np.stack([x["w"] for x in ds]))
            for _ in range(2):
                crf.iterate(30, rule=binding.MF_RULE_ADAPTIVE, reset=True)
            out.append(crf.log_marginals().copy())
    assert np.array_equal(out[0], out[1])


def test_adaptive_rejected_off_binary_grids(env):
    binding, oracle, torch = env
    d = synth.random_grid(8, 8, 3, 4, seed=1)
    with crf_for(binding, d) as crf:
        with pytest.raises(binding.ProxMFError, match="UNSUPPORTED"):
            crf.iterate(1, rule=binding.MF_RULE_ADAPTIVE, d=1.0)
