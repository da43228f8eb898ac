"""Thin ctypes binding of the C ABI in include/proxmf.h.

Argument marshalling only: every step of the method runs in the CUDA
library.  If the compiled library is missing, loading fails loudly -- there
is no CPU fallback.

Two levels:
  - module functions with the C names (crf_create, crf_set_unary, ...),
    taking raw pointers / ctypes objects and raising ProxMFError on a
    non-zero status;
  - ``CRF``, a small convenience wrapper taking torch tensors (device or
    host) or numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# PROXMF_LIB selects another build of the same library (e.g. an experimental
# variant); the default is the in-tree build.
LIB_PATH = os.environ.get("PROXMF_LIB") or os.path.join(HERE, "_build", "libproxmf.so")

CRF_GRID4, CRF_GRID8, CRF_DENSE_GAUSS, CRF_SPARSE = 0, 1, 2, 3
CRF_FP32, CRF_BF16 = 0, 1

STATUS = {
    0: "CRF_OK", -1: "CRF_E_INVALID", -2: "CRF_E_OOM", -3: "CRF_E_CUDA", -4: "CRF_E_STATE",
    -5: "CRF_E_TIMEOUT", -6: "CRF_E_NUMERIC", -7: "CRF_E_UNSUPPORTED",
}


class ProxMFError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({error_string(status)})")


class crf_desc(C.Structure):
    _fields_ = [("topology", C.c_int32), ("n_labels", C.c_int32), ("batch", C.c_int32),
                ("precision", C.c_int32), ("height", C.c_int64), ("width", C.c_int64),
                ("stream", C.c_void_p)]


MF_RULE_FIXED, MF_RULE_ADAPTIVE, MF_RULE_MOMENTUM, MF_RULE_ADAM, MF_RULE_ADHOC = 0, 1, 2, 3, 4


class mf_params(C.Structure):
    _fields_ = [("eta", C.c_double), ("max_iters", C.c_int32), ("reset", C.c_int32),
                ("rel_tol", C.c_double), ("refine_fp32", C.c_int32),
                ("final_free_energy", C.c_int32), ("rule", C.c_int32), ("d", C.c_double),
                ("gamma1", C.c_double), ("gamma2", C.c_double), ("epsilon", C.c_double)]


_lock = threading.Lock()
_lib = None

_vp = C.c_void_p
_i = C.c_int
_SIGS = {
    "crf_create": [C.POINTER(crf_desc), C.POINTER(_vp)],
    "crf_destroy": [_vp],
    "crf_set_unary": [_vp, _vp, _i],
    "crf_set_pairwise": [_vp, _vp, _vp, _vp, _i],
    "crf_set_state": [_vp, _vp, _i],
    "crf_set_graph": [_vp, _vp, C.c_int64, _vp, _vp, _vp, C.c_int32],
    "mf_iterate": [_vp, C.POINTER(mf_params), _vp],
    "mf_free_energy": [_vp, _vp],
    "mf_free_energy_trace": [_vp, _vp, C.c_int32],
    "mf_marginals": [_vp, _vp, _i],
    "mf_log_marginals": [_vp, _vp, _i],
    "mf_lipschitz": [_vp, _vp, _vp],
    "mf_server_create": [C.c_int64, C.c_int32, _vp, C.POINTER(_vp)],
    "mf_server_destroy": [_vp],
    "mf_server_submit": [_vp, C.POINTER(crf_desc), _vp, _vp, _vp, C.POINTER(mf_params), _vp,
                         C.POINTER(C.c_uint64)],
    "mf_server_step": [_vp, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
    "mf_server_poll": [_vp, C.c_uint64, C.POINTER(C.c_int32), C.POINTER(C.c_double), C.POINTER(C.c_int32)],
    "mf_server_sync": [_vp],
    "mf_profile": [_vp, C.c_int32],
    "mf_profile_read": [_vp, _vp, _vp],
    "crf_launch_count": [_vp, _vp],
    "mf_use_graphs": [_vp, C.c_int32],
    "mf_use_resident": [_vp, C.c_int32],
    "mf_dense_on_the_fly": [_vp, C.c_int32],
    "mf_unrolled_checkpoint_floats": [_vp, C.c_int32, _vp],
    "mf_unrolled_forward": [_vp, C.c_int32, C.c_double, _vp],
    "mf_unrolled_backward": [_vp, C.c_int32, C.c_double, _vp, _vp, _vp, _vp, _vp, C.c_int32],
}


def lib():
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run paper_1511_06103_gb300.build.build())")
        h = C.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(h, name)
            f.argtypes = args
            f.restype = C.c_int
        h.crf_error_string.argtypes = [C.c_int]
        h.crf_error_string.restype = C.c_char_p
        h.crf_version.argtypes = []
        h.crf_version.restype = C.c_char_p
        _lib = h
        return h


def error_string(status: int) -> str:
    try:
        return lib().crf_error_string(int(status)).decode()
    except Exception:  # noqa: BLE001 - message only
        return "?"


def _call(name: str, *args) -> None:
    rc = getattr(lib(), name)(*args)
    if rc != 0:
        raise ProxMFError(rc, name)


# -- C-named entry points ------------------------------------------------------

def crf_create(desc: crf_desc) -> int:
    h = _vp()
    _call("crf_create", C.byref(desc), C.byref(h))
    return h.value


def crf_destroy(h: int) -> None:
    _call("crf_destroy", h)


def crf_set_unary(h, U_ptr, is_device: int) -> None:
    _call("crf_set_unary", h, U_ptr, is_device)


def crf_set_pairwise(h, mu_ptr, w_ptr, theta_ptr, is_device: int) -> None:
    _call("crf_set_pairwise", h, mu_ptr, w_ptr, theta_ptr, is_device)


def crf_set_state(h, logq_ptr, is_device: int) -> None:
    _call("crf_set_state", h, logq_ptr, is_device)


def mf_iterate(h, params: mf_params, iters_done_ptr=None) -> None:
    _call("mf_iterate", h, C.byref(params), iters_done_ptr)


def mf_free_energy(h, F_ptr) -> None:
    _call("mf_free_energy", h, F_ptr)


def mf_free_energy_trace(h, F_ptr, n: int) -> None:
    _call("mf_free_energy_trace", h, F_ptr, n)


def mf_marginals(h, q_ptr, is_device: int) -> None:
    _call("mf_marginals", h, q_ptr, is_device)


def mf_log_marginals(h, logq_ptr, is_device: int) -> None:
    _call("mf_log_marginals", h, logq_ptr, is_device)


def mf_lipschitz(h, Lambda_ptr, eta_ptr) -> None:
    _call("mf_lipschitz", h, Lambda_ptr, eta_ptr)


def mf_profile(h, enable: int) -> None:
    _call("mf_profile", h, int(enable))


def mf_profile_read(h) -> tuple[float, int]:
    ms = C.c_double(0.0)
    n = C.c_int32(0)
    _call("mf_profile_read", h, C.byref(ms), C.byref(n))
    return ms.value, n.value


def crf_launch_count(h) -> int:
    n = C.c_int64(0)
    _call("crf_launch_count", h, C.byref(n))
    return n.value


def mf_unrolled_checkpoint_floats(h, K: int) -> int:
    n = C.c_int64(0)
    _call("mf_unrolled_checkpoint_floats", h, int(K), C.byref(n))
    return n.value


def mf_unrolled_forward(h, K: int, eta: float, ckpt_ptr) -> None:
    _call("mf_unrolled_forward", h, int(K), float(eta), ckpt_ptr)


def mf_unrolled_backward(h, K: int, eta: float, ckpt_ptr, dlogq_ptr, dU_ptr, dmu_ptr, dw_ptr,
                         is_device: int) -> None:
    _call("mf_unrolled_backward", h, int(K), float(eta), ckpt_ptr, dlogq_ptr, dU_ptr, dmu_ptr, dw_ptr,
          int(is_device))


def crf_version() -> str:
    return lib().crf_version().decode()


# -- convenience wrapper -------------------------------------------------------

def _as_buffer(a):
    """(pointer, is_device, keepalive) for a float32 torch tensor or numpy array."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float32 or not a.is_contiguous():
                raise ValueError("expected a contiguous float32 tensor")
            return a.data_ptr(), int(a.is_cuda), a
    except ImportError:  # pragma: no cover
        pass
    arr = np.ascontiguousarray(a, dtype=np.float32)
    return arr.ctypes.data, 0, arr


def current_stream_handle() -> int | None:
    import torch
    if torch.cuda.is_available() and torch.cuda.is_initialized():
        return torch.cuda.current_stream().cuda_stream
    return None


class CRF:
    """One handle of the library: a batch of same-shaped grid CRFs."""

    def __init__(self, topology: int, n_labels: int, height: int, width: int, batch: int = 1,
                 precision: int = CRF_FP32, stream: int | None = None):
        if stream is None:
            stream = current_stream_handle()
        self.desc = crf_desc(topology, n_labels, batch, precision, height, width, stream)
        self.L, self.H, self.W, self.B = n_labels, height, width, batch
        self.N = height * width
        self.h = crf_create(self.desc)

    def close(self) -> None:
        if getattr(self, "h", None):
            crf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_unary(self, U) -> None:
        p, dev, keep = _as_buffer(U)
        crf_set_unary(self.h, p, dev)

    def set_pairwise(self, mu, w, theta=None) -> None:
        pm, dm, km = _as_buffer(mu)
        pw, dw, kw = _as_buffer(w)
        if dm != dw:
            # mu and w travel with one is_device flag; bring mu to w's side
            import torch
            km = torch.as_tensor(np.asarray(km.cpu() if hasattr(km, "cpu") else km, np.float32))
            if dw:
                km = km.cuda()
            pm, dm, km = _as_buffer(km)
        pt = None
        if theta is not None:
            th = np.ascontiguousarray(theta, np.float32)
            pt = th.ctypes.data
        crf_set_pairwise(self.h, pm, pw, pt, dw)

    def set_graph(self, mu, src, dst, w) -> None:
        """Pairwise term of a CRF_SPARSE handle: oriented edges src[e] -> dst[e]
        with weights w[e] (host arrays), mu [L][L]."""
        src = np.ascontiguousarray(src, np.int32)
        dst = np.ascontiguousarray(dst, np.int32)
        w = np.ascontiguousarray(w, np.float32)
        mu = np.ascontiguousarray(mu, np.float32)
        if not (src.shape == dst.shape == w.shape):
            raise ValueError("src, dst and w must have the same length")
        _call("crf_set_graph", self.h, mu.ctypes.data, int(src.size), src.ctypes.data, dst.ctypes.data,
              w.ctypes.data, 0)

    def set_state(self, logq) -> None:
        p, dev, keep = _as_buffer(logq)
        crf_set_state(self.h, p, dev)

    def iterate(self, max_iters: int, eta: float = 0.0, reset: bool = False, rel_tol: float = 0.0,
                refine_fp32: int = 0, want_iters: bool = False, final_free_energy: bool = False,
                rule: int = MF_RULE_FIXED, d: float = 0.0, gamma1: float = 0.95, gamma2: float = 0.999,
                epsilon: float = 1e-8):
        prm = mf_params(float(eta), int(max_iters), int(bool(reset)), float(rel_tol), int(refine_fp32),
                        int(bool(final_free_energy)), int(rule), float(d), float(gamma1), float(gamma2),
                        float(epsilon))
        if want_iters:
            out = np.zeros(self.B, np.int32)
            mf_iterate(self.h, prm, out.ctypes.data)
            return out
        mf_iterate(self.h, prm, None)
        return None

    def free_energy(self) -> np.ndarray:
        F = np.zeros(self.B, np.float64)
        mf_free_energy(self.h, F.ctypes.data)
        return F

    def free_energy_trace(self, n: int) -> np.ndarray:
        F = np.zeros((self.B, n), np.float64)
        mf_free_energy_trace(self.h, F.ctypes.data, n)
        return F

    def _export(self, fn, out):
        if out is None:
            out = np.zeros((self.B, self.N, self.L), np.float32)
        p, dev, keep = _as_buffer(out)
        fn(self.h, p, dev)
        return out

    def marginals(self, out=None):
        return self._export(mf_marginals, out)

    def log_marginals(self, out=None):
        return self._export(mf_log_marginals, out)

    def profile(self, enable: bool = True) -> None:
        mf_profile(self.h, int(enable))

    def profile_read(self) -> tuple[float, int]:
        return mf_profile_read(self.h)

    def launch_count(self) -> int:
        return crf_launch_count(self.h)

    def use_graphs(self, enable: bool = True) -> None:
        _call("mf_use_graphs", self.h, int(bool(enable)))

    def dense_on_the_fly(self, enable: bool = True) -> None:
        """BF16 dense handles: the tensor-core steps compute K in the kernel (mf_dense_on_the_fly)."""
        _call("mf_dense_on_the_fly", self.h, int(bool(enable)))

    def use_resident(self, enable: bool = True) -> None:
        """Small grids: the whole iteration loop in one launch (the default)."""
        _call("mf_use_resident", self.h, int(bool(enable)))

    def checkpoint_floats(self, K: int) -> int:
        return mf_unrolled_checkpoint_floats(self.h, K)

    def unrolled_forward(self, K: int, eta: float, ckpt) -> None:
        """K steps from softmax(-U), states s^0..s^K into ``ckpt`` (a device
        float32 tensor of checkpoint_floats(K) elements)."""
        p, dev, keep = _as_buffer(ckpt)
        if not dev:
            raise ValueError("checkpoints live on the device")
        mf_unrolled_forward(self.h, K, eta, p)

    def unrolled_backward(self, K: int, eta: float, ckpt, dlogq, dU=None, dmu=None, dw=None):
        """(dU, dmu, dw) from d loss / d log q^K.  Outputs are allocated like
        ``dlogq`` (device tensor or host array) when not given."""
        pc, dc, kc = _as_buffer(ckpt)
        pg, dg, kg = _as_buffer(dlogq)
        nd = 4 if self.desc.topology == CRF_GRID8 else 2
        if dg:
            import torch
            dev = kg.device
            dU = torch.empty((self.B, self.N, self.L), dtype=torch.float32, device=dev) if dU is None else dU
            dmu = torch.empty((self.L, self.L), dtype=torch.float32, device=dev) if dmu is None else dmu
            dw = torch.empty((self.B, nd, self.H, self.W), dtype=torch.float32, device=dev) if dw is None else dw
        else:
            dU = np.zeros((self.B, self.N, self.L), np.float32) if dU is None else dU
            dmu = np.zeros((self.L, self.L), np.float32) if dmu is None else dmu
            dw = np.zeros((self.B, nd, self.H, self.W), np.float32) if dw is None else dw
        bufs = [_as_buffer(a) for a in (dU, dmu, dw)]
        if any(b[1] != dg for b in bufs):
            raise ValueError("gradient outputs must be on the same side as dlogq")
        mf_unrolled_backward(self.h, K, eta, pc, pg, bufs[0][0], bufs[1][0], bufs[2][0], dg)
        return dU, dmu, dw

    def lipschitz(self):
        lam = np.zeros(self.B, np.float64)
        eta = np.zeros(self.B, np.float64)
        mf_lipschitz(self.h, lam.ctypes.data, eta.ctypes.data)
        return lam, eta


# -- serving -------------------------------------------------------------------

class Server:
    """Continuous-batching server over the mf_server_* calls."""

    def __init__(self, budget_bytes: int, max_slots: int = 64, stream: int | None = None):
        if stream is None:
            stream = current_stream_handle()
        h = _vp()
        _call("mf_server_create", int(budget_bytes), int(max_slots), stream, C.byref(h))
        self.h = h.value
        self._keep = {}

    def close(self) -> None:
        if getattr(self, "h", None):
            _call("mf_server_destroy", self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, U, mu, w, H: int, W: int, conn: int, eta: float = 0.0, max_iters: int = 1000,
               rel_tol: float = 0.0) -> int:
        L = mu.shape[0]
        topo = CRF_GRID8 if conn == 8 else CRF_GRID4
        d = crf_desc(topo, L, 1, CRF_FP32, H, W, None)
        prm = mf_params(float(eta), int(max_iters), 1, float(rel_tol), 0, 0, MF_RULE_FIXED, 0.0, 0.0, 0.0, 0.0)
        U = np.ascontiguousarray(U, np.float32)
        mu = np.ascontiguousarray(mu, np.float32)
        w = np.ascontiguousarray(w, np.float32)
        q = np.zeros((H * W, L), np.float32)
        t = C.c_uint64(0)
        _call("mf_server_submit", self.h, C.byref(d), U.ctypes.data, mu.ctypes.data, w.ctypes.data,
              C.byref(prm), q.ctypes.data, C.byref(t))
        self._keep[t.value] = q
        return t.value

    def step(self, iters: int = 1) -> tuple[int, int]:
        a = C.c_int32(0)
        b = C.c_int32(0)
        _call("mf_server_step", self.h, int(iters), C.byref(a), C.byref(b))
        return a.value, b.value

    def poll(self, ticket: int):
        """(state, F, iters, q or None): state 0 queued, 1 running, 2 done."""
        st = C.c_int32(0)
        F = C.c_double(0.0)
        it = C.c_int32(0)
        _call("mf_server_poll", self.h, C.c_uint64(ticket), C.byref(st), C.byref(F), C.byref(it))
        q = self._keep.get(ticket) if st.value == 2 else None
        return st.value, F.value, it.value, q

    def sync(self) -> None:
        _call("mf_server_sync", self.h)
