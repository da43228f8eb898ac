"""FP64 CPU oracle for parallel proximal mean-field inference.

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the CPU
baseline leg of ``bench.py`` use this module; the product path never does.
It shares no code with the CUDA library.

The arithmetic lives in ``mf_oracle.c`` (plain C, FP64, libm); this file
compiles it with gcc on first use and wraps it with ctypes and numpy.
Conventions: ``U[i, l]`` unary costs, ``mu[l, m]`` the cost of
``(x_i=l, x_j=m)`` on an edge oriented ``i -> j``, state ``s = log q``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mf_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = C.c_double
_i32 = C.c_int32
_i64 = C.c_int64
_vp = C.c_void_p


def build(force: bool = False) -> str:
    """Compile ``mf_oracle.c`` into ``oracle/_build/liboracle.so``."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        sig = {
            "orc_num_threads": (_i32, []),
            "orc_model_sparse": (_vp, [_i64, _i32, _vp, _vp, _i64, _vp, _vp, _vp]),
            "orc_model_dense": (_vp, [_i64, _i32, _vp, _vp, _vp]),
            "orc_model_free": (None, [_vp]),
            "orc_grid_edge_count": (_i64, [_i64, _i64, _i32]),
            "orc_grid_edges": (None, [_i64, _i64, _i32, _vp, _vp, _vp, _vp]),
            "orc_dense_gauss_kernel": (None, [_i64, _vp, _d, _d, _vp]),
            "orc_hess_vec": (None, [_vp, _vp, _vp]),
            "orc_grad": (None, [_vp, _vp, _vp]),
            "orc_energy": (_d, [_vp, _vp]),
            "orc_neg_entropy": (_d, [_vp, _vp]),
            "orc_free_energy": (_d, [_vp, _vp]),
            "orc_init_logq": (None, [_vp, _vp]),
            "orc_prox_step": (None, [_vp, _d, _vp, _vp]),
            "orc_parallel_prox": (None, [_vp, _d, _i32, _vp, _vp]),
            "orc_prox_step_adaptive": (_i32, [_vp, _d, _vp, _vp]),
            "orc_parallel_prox_momentum": (None, [_vp, _d, _d, _i32, _vp, _vp]),
            "orc_parallel_adhoc": (None, [_vp, _d, _i32, _vp, _vp]),
            "orc_parallel_prox_adam": (None, [_vp, _d, _d, _d, _d, _i32, _vp, _vp]),
            "orc_parallel_prox_adaptive": (_i32, [_vp, _d, _i32, _vp, _vp]),
            "orc_prox_step_rows": (None, [_vp, _d, _vp, _vp, _i64, _vp]),
            "orc_sweep": (None, [_vp, _i32, _vp]),
            "orc_state_energy": (_d, [_vp, _vp]),
            "orc_brute_force": (C.c_int, [_vp, _vp, _vp]),
            "orc_brute_free_energy": (_d, [_vp, _vp]),
            "orc_brute_cond_energy": (C.c_int, [_vp, _vp, _vp]),
            "orc_jacobi_eigenvalues": (None, [_i64, _vp, _vp]),
            "orc_hessian_eigenvalues": (C.c_int, [_vp, C.c_int, _vp]),
            "orc_lanczos_tangent": (_i32, [_vp, _i32, _vp, _vp, _vp]),
            "orc_step_size": (_d, [_d]),
            "orc_unrolled_loss_grad": (_d, [_vp, _d, _i32, _vp, _vp, _vp, _vp]),
            "orc_unrolled_loss": (_d, [_vp, _d, _i32, _vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_vp)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def grid_edges(H: int, W: int, conn: int, w: np.ndarray):
    """Oriented edge list of a 4- or 8-connected H x W grid.

    ``w`` is ``[n_dirs][H][W]``: direction 0 right, 1 down, 2 down-right,
    3 down-left; the entry at (y, x) weights the edge leaving (y, x)."""
    lib = _load()
    nd = 4 if conn == 8 else 2
    w = _f64(w)
    assert w.shape == (nd, H, W)
    ne = int(lib.orc_grid_edge_count(H, W, conn))
    ei = np.zeros(ne, np.int64)
    ej = np.zeros(ne, np.int64)
    ew = np.zeros(ne, np.float64)
    lib.orc_grid_edges(H, W, conn, _ptr(w), _ptr(ei), _ptr(ej), _ptr(ew))
    return ei, ej, ew


def dense_gauss_kernel(feats: np.ndarray, theta_pos: float, theta_rgb: float) -> np.ndarray:
    """N x N Gaussian kernel over (x, y, r, g, b) features, zero diagonal."""
    lib = _load()
    f = _f64(feats)
    n = f.shape[0]
    assert f.shape == (n, 5)
    K = np.zeros((n, n), np.float64)
    lib.orc_dense_gauss_kernel(n, _ptr(f), float(theta_pos), float(theta_rgb), _ptr(K))
    return K


def jacobi_eigenvalues(A: np.ndarray) -> np.ndarray:
    lib = _load()
    A = _f64(A).copy()
    n = A.shape[0]
    ev = np.zeros(n, np.float64)
    lib.orc_jacobi_eigenvalues(n, _ptr(A), _ptr(ev))
    return ev


def step_size(Lambda: float) -> float:
    """eta = 1 / (1 + max(Lambda, 0))."""
    return float(_load().orc_step_size(float(Lambda)))


class Model:
    """A pairwise CRF held by the oracle (sparse edge list or dense matrix)."""

    def __init__(self, handle, n: int, L: int, U: np.ndarray, mu: np.ndarray):
        self._h = handle
        self.n = n
        self.L = L
        self.U = U
        self.mu = mu

    @classmethod
    def sparse(cls, U, mu, ei, ej, ew) -> "Model":
        lib = _load()
        U = _f64(U)
        mu = _f64(mu)
        n, L = U.shape
        assert mu.shape == (L, L)
        ei = np.ascontiguousarray(ei, np.int64)
        ej = np.ascontiguousarray(ej, np.int64)
        ew = _f64(ew)
        assert ei.shape == ej.shape == ew.shape
        if ei.size:
            assert ei.min() >= 0 and ej.min() >= 0 and ei.max() < n and ej.max() < n
        h = lib.orc_model_sparse(n, L, _ptr(U), _ptr(mu), ei.size, _ptr(ei), _ptr(ej), _ptr(ew))
        if not h:
            raise MemoryError("oracle model allocation failed")
        return cls(h, n, L, U, mu)

    @classmethod
    def grid(cls, U, mu, w, H: int, W: int, conn: int) -> "Model":
        """U is [H*W][L] (pixel p = y*W + x), w is [n_dirs][H][W]."""
        ei, ej, ew = grid_edges(H, W, conn, w)
        return cls.sparse(U, mu, ei, ej, ew)

    @classmethod
    def dense(cls, U, mu, K) -> "Model":
        lib = _load()
        U = _f64(U)
        mu = _f64(mu)
        K = _f64(K)
        n, L = U.shape
        assert K.shape == (n, n)
        h = lib.orc_model_dense(n, L, _ptr(U), _ptr(mu), _ptr(K))
        if not h:
            raise MemoryError("oracle model allocation failed")
        return cls(h, n, L, U, mu)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_model_free(h)
            self._h = None

    # -- quantities ------------------------------------------------------
    def _nl(self, a) -> np.ndarray:
        a = _f64(a)
        assert a.shape == (self.n, self.L), a.shape
        return a

    def init_logq(self) -> np.ndarray:
        s = np.zeros((self.n, self.L))
        _load().orc_init_logq(self._h, _ptr(s))
        return s

    def grad(self, q) -> np.ndarray:
        q = self._nl(q)
        g = np.zeros_like(q)
        _load().orc_grad(self._h, _ptr(q), _ptr(g))
        return g

    def hess_vec(self, v) -> np.ndarray:
        v = self._nl(v)
        out = np.zeros_like(v)
        _load().orc_hess_vec(self._h, _ptr(v), _ptr(out))
        return out

    def energy(self, q) -> float:
        return float(_load().orc_energy(self._h, _ptr(self._nl(q))))

    def neg_entropy(self, q) -> float:
        return float(_load().orc_neg_entropy(self._h, _ptr(self._nl(q))))

    def free_energy(self, q) -> float:
        return float(_load().orc_free_energy(self._h, _ptr(self._nl(q))))

    def prox_step(self, eta: float, s) -> np.ndarray:
        s = self._nl(s)
        out = np.zeros_like(s)
        _load().orc_prox_step(self._h, float(eta), _ptr(s), _ptr(out))
        return out

    def prox_step_rows(self, eta: float, s, rows) -> np.ndarray:
        """One proximal step evaluated for the listed variables only."""
        s = self._nl(s)
        rows = np.ascontiguousarray(rows, np.int64)
        out = np.zeros((rows.size, self.L))
        _load().orc_prox_step_rows(self._h, float(eta), _ptr(s), _ptr(rows), rows.size, _ptr(out))
        return out

    def parallel_prox(self, eta: float, iters: int, s=None, trace: bool = True):
        """Returns (s after iters steps, F(q^t) for t = 0..iters)."""
        s = self.init_logq() if s is None else self._nl(s).copy()
        F = np.zeros(iters + 1) if trace else None
        _load().orc_parallel_prox(self._h, float(eta), int(iters), _ptr(s),
                                  _ptr(F) if trace else None)
        return s, F

    def prox_step_adaptive(self, d: float, s) -> np.ndarray:
        """One adaptive step of a binary model (Sec. 3.3): eta_i = 1/(1 + d q_i0 q_i1)."""
        s = self._nl(s)
        out = np.zeros_like(s)
        if _load().orc_prox_step_adaptive(self._h, float(d), _ptr(s), _ptr(out)) != 0:
            raise ValueError("the adaptive step is defined for binary models only")
        return out

    def parallel_prox_adaptive(self, d: float, iters: int, s=None, trace: bool = True):
        """(s after iters adaptive steps, F(q^t) for t = 0..iters)."""
        s = self.init_logq() if s is None else self._nl(s).copy()
        F = np.zeros(iters + 1) if trace else None
        if _load().orc_parallel_prox_adaptive(self._h, float(d), int(iters), _ptr(s),
                                              _ptr(F) if trace else None) != 0:
            raise ValueError("the adaptive step is defined for binary models only")
        return s, F

    def parallel_adhoc(self, eta: float, iters: int, s=None):
        """(s, F(q^t) for t = 0..iters) of ADHOC damping (Eq. related:parallel-update)."""
        s = self.init_logq() if s is None else self._nl(s).copy()
        F = np.zeros(iters + 1)
        _load().orc_parallel_adhoc(self._h, float(eta), int(iters), _ptr(s), _ptr(F))
        return s, F

    def parallel_prox_momentum(self, eta: float, gamma1: float, iters: int, s=None):
        """(s, F(q^t) for t = 0..iters) of OURS-MOMENTUM (Sec. 3.4)."""
        s = self.init_logq() if s is None else self._nl(s).copy()
        F = np.zeros(iters + 1)
        _load().orc_parallel_prox_momentum(self._h, float(eta), float(gamma1), int(iters), _ptr(s), _ptr(F))
        return s, F

    def parallel_prox_adam(self, d0: float, gamma1: float, gamma2: float, eps: float, iters: int, s=None):
        """(s, F(q^t) for t = 0..iters) of OURS-ADAM (Sec. 3.5)."""
        s = self.init_logq() if s is None else self._nl(s).copy()
        F = np.zeros(iters + 1)
        _load().orc_parallel_prox_adam(self._h, float(d0), float(gamma1), float(gamma2), float(eps), int(iters),
                                       _ptr(s), _ptr(F))
        return s, F

    def sweep(self, sweeps: int, s=None) -> np.ndarray:
        s = self.init_logq() if s is None else self._nl(s).copy()
        _load().orc_sweep(self._h, int(sweeps), _ptr(s))
        return s

    def state_energy(self, x) -> float:
        x = np.ascontiguousarray(x, np.int32)
        return float(_load().orc_state_energy(self._h, _ptr(x)))

    def brute_force(self):
        """(log Z, exact marginals) by enumeration."""
        logZ = C.c_double(0.0)
        marg = np.zeros((self.n, self.L))
        rc = _load().orc_brute_force(self._h, C.byref(logZ), _ptr(marg))
        if rc != 0:
            raise ValueError("model too large to enumerate")
        return logZ.value, marg

    def brute_free_energy(self, q) -> float:
        return float(_load().orc_brute_free_energy(self._h, _ptr(self._nl(q))))

    def brute_cond_energy(self, q) -> np.ndarray:
        q = self._nl(q)
        out = np.zeros_like(q)
        if _load().orc_brute_cond_energy(self._h, _ptr(q), _ptr(out)) != 0:
            raise ValueError("model too large to enumerate")
        return out

    def unrolled_loss(self, eta: float, K: int, y) -> float:
        """-(1/n) sum_i log q^K_{i,y_i} after K steps from softmax(-U)."""
        y = np.ascontiguousarray(y, np.int32)
        return float(_load().orc_unrolled_loss(self._h, float(eta), int(K), _ptr(y)))

    def unrolled_grad(self, eta: float, K: int, y, n_edges: int):
        """(loss, dU [n][L], dmu [L][L], dw [n_edges]) by reverse mode."""
        y = np.ascontiguousarray(y, np.int32)
        dU = np.zeros((self.n, self.L))
        dmu = np.zeros((self.L, self.L))
        dw = np.zeros(max(1, n_edges))
        loss = _load().orc_unrolled_loss_grad(self._h, float(eta), int(K), _ptr(y), _ptr(dU), _ptr(dmu), _ptr(dw))
        return float(loss), dU, dmu, dw[:n_edges]

    def hessian_eigenvalues(self, projected: bool = True) -> np.ndarray:
        ev = np.zeros(self.n * self.L)
        if _load().orc_hessian_eigenvalues(self._h, int(projected), _ptr(ev)) != 0:
            raise ValueError("model too large for a dense eigen-solve")
        return ev

    def lanczos(self, iters: int, v0) -> tuple[float, float, int]:
        """(lambda_min, lambda_max, steps) of the tangent-space Hessian."""
        v0 = self._nl(v0)
        lo = C.c_double(0.0)
        hi = C.c_double(0.0)
        k = _load().orc_lanczos_tangent(self._h, int(iters), _ptr(v0), C.byref(lo), C.byref(hi))
        if k < 0:
            raise MemoryError("lanczos allocation failed")
        return lo.value, hi.value, int(k)
