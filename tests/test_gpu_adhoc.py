"""GPU parity of the ADHOC baseline (mean-parameter damping, Sec. 2.2.2,
Eq. related:parallel-update) against the FP64 oracle, FP32 tolerances."""
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


@pytest.mark.parametrize("Hh,Ww,L,conn,sym,eta", [(40, 37, 5, 8, False, 0.3), (33, 70, 21, 8, True, 0.1),
                                                  (64, 64, 2, 4, True, 0.5), (1, 1, 3, 8, False, 0.7)])
def test_adhoc_trajectory(env, Hh, Ww, L, conn, sym, eta):
    binding, oracle, torch = env
    d = synth.random_grid(Hh, Ww, L, conn, seed=800 + L, symmetric=sym)
    T = 30
    topo = binding.CRF_GRID8 if conn == 8 else binding.CRF_GRID4
    with binding.CRF(topo, L, Hh, Ww) as crf:
        crf.set_unary(d["U"])
        crf.set_pairwise(d["mu"], d["w"])
        crf.iterate(T, eta=eta, reset=True, rule=binding.MF_RULE_ADHOC)
        s = crf.log_marginals()[0].astype(np.float64)
        trace = crf.free_energy_trace(T)[0]
    m = oracle.Model.grid(f64(d["U"]), f64(d["mu"]), f64(d["w"]), Hh, Ww, conn)
    s_ref, F_ref = m.parallel_adhoc(eta, T)
    assert np.abs(np.exp(s) - np.exp(s_ref)).max() <= 1e-5
    assert H.f_close(trace, F_ref[:-1], Hh * Ww)
