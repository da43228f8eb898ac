"""The allocation-free step entry point (for callers that cannot call
cudaMalloc: code under an allocator or memory pool that owns the device, or
in a region where allocation is forbidden) gives, on two calls in a row, the
same result as the handle API and as the FP64 oracle.

Collected last on purpose: it calls the library through raw ctypes with its
own device buffers, and must pass both alone in a fresh process and after the
other GPU tests (its scratch array is shared by every call)."""
import ctypes as C

import numpy as np
import pytest

from paper_1511_06103_gb300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu


def storage_labels(L):
    return 2 if L <= 2 else (L + 3) // 4 * 4


def padded(a, pad):
    """[N][L] rows -> [N][Lp] with the padding labels set to pad."""
    N, L = a.shape
    out = np.full((N, storage_labels(L)), pad, np.float32)
    out[:, :L] = a
    return out


def pixel_major_weights(w):
    """[n_dirs][H][W] -> [H*W][n_dirs] (entries off the image are already 0)."""
    nd = w.shape[0]
    return np.ascontiguousarray(w.reshape(nd, -1).T)


@pytest.mark.parametrize("Hh,Ww,L,conn,sym", [(37, 45, 21, 8, True), (20, 70, 5, 4, False)])
def test_noalloc_step_matches_handle_api(Hh, Ww, L, conn, sym):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    from paper_1511_06103_gb300 import binding, build
    build.build()
    lib = binding.lib()
    fn = lib.mf_grid_step_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_int32, C.c_int32, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                   C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]
    dev = torch.device("cuda:0")
    d = synth.random_grid(Hh, Ww, L, conn, seed=4242 + L, symmetric=sym)
    s0 = synth.random_logq(Hh * Ww, L, seed=17)
    eta = 0.31
    topo = binding.CRF_GRID8 if conn == 8 else binding.CRF_GRID4

    # the FP64 oracle: two steps from the same state
    import oracle
    oracle.build()
    m = oracle.Model.grid(np.asarray(d["U"], np.float64), np.asarray(d["mu"], np.float64),
                          np.asarray(d["w"], np.float64), Hh, Ww, conn)
    orc_s, orc_F = [], []
    s_cur = np.asarray(s0, np.float64)
    for _ in range(2):
        orc_F.append(m.free_energy(np.exp(s_cur)))
        s_cur = m.prox_step(float(np.float32(eta)), s_cur)
        orc_s.append(s_cur)

    # reference: two steps through the handle API
    ref_s, ref_F = [], []
    with binding.CRF(topo, L, Hh, Ww) as crf:
        crf.set_unary(d["U"])
        crf.set_pairwise(d["mu"], d["w"])
        crf.set_state(s0)
        for _ in range(2):
            crf.iterate(1, eta=eta)
            ref_F.append(crf.free_energy_trace(1)[0, 0])
            ref_s.append(crf.log_marginals()[0])

    # the same two steps through the allocation-free entry point
    U = torch.from_numpy(padded(d["U"], 0.0)).to(dev)
    w = torch.from_numpy(pixel_major_weights(d["w"])).to(dev)
    mu = np.ascontiguousarray(d["mu"], np.float32)
    bufs = [torch.from_numpy(padded(s0, -1e30)).to(dev),
            torch.empty((Hh * Ww, storage_labels(L)), device=dev)]
    F = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for k in range(2):
        rc = fn(topo, L, Hh, Ww, U.data_ptr(), w.data_ptr(), mu.ctypes.data, bufs[k % 2].data_ptr(),
                bufs[(k + 1) % 2].data_ptr(), eta, F.data_ptr(), stream)
        assert rc == 0
        torch.cuda.synchronize()
        out = bufs[(k + 1) % 2].cpu().numpy()[:, :L]
        q = np.exp(out.astype(np.float64))
        assert np.abs(q - np.exp(ref_s[k].astype(np.float64))).max() <= 1e-6
        assert H.f_close(F.item(), ref_F[k], Hh * Ww)
        assert np.abs(q - np.exp(orc_s[k])).max() <= 1e-6
        assert H.f_close(F.item(), orc_F[k], Hh * Ww)

    # a state holding NaN gives a non-finite F, reported as NaN in F_out;
    # the next call with a clean state starts from a cleared status word
    bad = padded(s0, -1e30)
    bad[3, 0] = np.nan
    bufs[0].copy_(torch.from_numpy(bad).to(dev))
    assert fn(topo, L, Hh, Ww, U.data_ptr(), w.data_ptr(), mu.ctypes.data, bufs[0].data_ptr(),
              bufs[1].data_ptr(), eta, F.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    assert np.isnan(F.item())
    bufs[0].copy_(torch.from_numpy(padded(s0, -1e30)).to(dev))
    assert fn(topo, L, Hh, Ww, U.data_ptr(), w.data_ptr(), mu.ctypes.data, bufs[0].data_ptr(),
              bufs[1].data_ptr(), eta, F.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    assert H.f_close(F.item(), orc_F[0], Hh * Ww)


def test_noalloc_rejects_oversize_and_bad_arguments():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_06103_gb300 import binding, build
    build.build()
    fn = binding.lib().mf_grid_step_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_int32, C.c_int32, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                   C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]
    mu = np.zeros((3, 3), np.float32)
    fake = 256  # never dereferenced: every case below is rejected before any launch
    # 4096 x 4096 needs 65536 tiles > 64480
    assert fn(1, 3, 4096, 4096, fake, fake, mu.ctypes.data, fake, fake * 2, 0.5, fake, None) == -1
    assert fn(1, 0, 8, 8, fake, fake, mu.ctypes.data, fake, fake * 2, 0.5, fake, None) == -1
    assert fn(1, 3, 8, 8, fake, fake, mu.ctypes.data, fake, fake, 0.5, fake, None) == -1
    assert fn(1, 3, 8, 8, fake, fake, mu.ctypes.data, fake, fake * 2, 0.0, fake, None) == -1
