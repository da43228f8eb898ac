"""Seeded synthetic CRF instances shaped like the paper's workloads.

This module only *draws inputs*: it holds none of the mean-field arithmetic,
so both the CUDA path and the FP64 oracle consume its output.  Every array is
returned as float32 (what the device library takes); the oracle promotes the
same values to float64, so both sides solve exactly the same model.

Layouts (shared by the C-ABI and the oracle):
  U   [N][L]         unary costs, pixel p = y*W + x
  mu  [L][L]         mu[l, m] = cost of (x_i=l, x_j=m) on an edge i -> j
  w   [n_dirs][H][W] grid edge weights; direction 0 right, 1 down,
                     2 down-right, 3 down-left; the entry at (y, x) weights
                     the edge leaving (y, x); entries whose edge would leave
                     the image are 0
  feats [N][5]       (x, y, r, g, b) for fully connected models

Recipes (the workloads of the paper's Sec. 4.2, with the readings listed in
the design notes):
  binary_denoising   64x64 4-connected, L=2, 6 random rectangles, 20% flips,
                     U = -log likelihood of the flip noise, Potts 0.8
  segmentation_grid  8-connected, L labels, U = -log softmax(N(0, 2^2)
                     logits), symmetric mu ~ U(-1,1) with zero diagonal,
                     w = exp(-|dc|^2 / (2 * 0.1^2)) over a smooth RGB field
  dense_gaussian     96x96 positions, RGB in [0,255] smooth field,
                     mu = (1 - I) + 0.5 S, S symmetric U(-1,1) zero diagonal
"""
from __future__ import annotations

import math

import numpy as np

DIRS_DY = (0, 1, 1, 1)
DIRS_DX = (1, 0, 1, -1)


def n_dirs(conn: int) -> int:
    if conn not in (4, 8):
        raise ValueError("conn must be 4 or 8")
    return 2 if conn == 4 else 4


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def _blur_axis(a: np.ndarray, sigma: float, axis: int) -> np.ndarray:
    r = int(math.ceil(3 * sigma))
    x = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-x * x / (2 * sigma * sigma))
    k /= k.sum()
    pad = [(0, 0)] * a.ndim
    pad[axis] = (r, r)
    p = np.pad(a, pad, mode="reflect")
    out = np.zeros_like(a, dtype=np.float64)
    n = a.shape[axis]
    for t in range(2 * r + 1):
        sl = [slice(None)] * a.ndim
        sl[axis] = slice(t, t + n)
        out += k[t] * p[tuple(sl)]
    return out


def smooth_field(H: int, W: int, channels: int, rng: np.random.Generator,
                 sigma_blur: float = 8.0) -> np.ndarray:
    """[channels][H][W] uniform noise blurred by a Gaussian, rescaled to [0,1]."""
    out = np.empty((channels, H, W), np.float64)
    sb = min(sigma_blur, max(1.0, (min(H, W) - 1) / 3.0))
    for c in range(channels):
        a = rng.random((H, W))
        a = _blur_axis(_blur_axis(a, sb, 0), sb, 1)
        lo, hi = a.min(), a.max()
        out[c] = (a - lo) / (hi - lo) if hi > lo else 0.5
    return out


def edge_weights_from_colour(rgb: np.ndarray, conn: int, sigma: float) -> np.ndarray:
    """w[k][y][x] = exp(-|c(y,x) - c(neighbour_k)|^2 / (2 sigma^2)); 0 off-image."""
    _, H, W = rgb.shape
    nd = n_dirs(conn)
    w = np.zeros((nd, H, W), np.float64)
    for k in range(nd):
        dy, dx = DIRS_DY[k], DIRS_DX[k]
        y0, y1 = 0, H - dy
        x0, x1 = max(0, -dx), W - max(0, dx)
        a = rgb[:, y0:y1, x0:x1]
        b = rgb[:, y0 + dy:y1 + dy, x0 + dx:x1 + dx]
        d2 = ((a - b) ** 2).sum(axis=0)
        w[k, y0:y1, x0:x1] = np.exp(-d2 / (2 * sigma * sigma))
    return w


def constant_edge_weights(H: int, W: int, conn: int, value: float) -> np.ndarray:
    nd = n_dirs(conn)
    w = np.zeros((nd, H, W), np.float64)
    for k in range(nd):
        dy, dx = DIRS_DY[k], DIRS_DX[k]
        w[k, 0:H - dy, max(0, -dx):W - max(0, dx)] = value
    return w


def random_edge_weights(H: int, W: int, conn: int, rng: np.random.Generator,
                        lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    w = constant_edge_weights(H, W, conn, 1.0)
    return w * rng.uniform(lo, hi, size=w.shape)


def unary_from_logits(logits: np.ndarray) -> np.ndarray:
    """U = -log softmax(logits) along the last axis (costs of a classifier)."""
    z = logits - logits.max(axis=-1, keepdims=True)
    return -(z - np.log(np.exp(z).sum(axis=-1, keepdims=True)))


def symmetric_uniform(L: int, rng: np.random.Generator, zero_diag: bool = True) -> np.ndarray:
    A = rng.uniform(-1.0, 1.0, size=(L, L))
    A = np.triu(A, 1)
    A = A + A.T
    if not zero_diag:
        A += np.diag(rng.uniform(-1.0, 1.0, size=L))
    return A


def potts(L: int, c: float) -> np.ndarray:
    return c * (1.0 - np.eye(L))


def binary_denoising(H: int = 64, W: int = 64, n_rects: int = 6, flip: float = 0.2,
                     coupling: float = 0.8, seed: int = 0) -> dict:
    rng = np.random.default_rng(seed)
    clean = np.zeros((H, W), np.int32)
    for _ in range(n_rects):
        ya, yb = np.sort(rng.integers(0, H, size=2))
        xa, xb = np.sort(rng.integers(0, W, size=2))
        clean[ya:yb + 1, xa:xb + 1] = 1
    flips = rng.random((H, W)) < flip
    noisy = np.where(flips, 1 - clean, clean)
    y = noisy.reshape(-1)
    U = np.empty((H * W, 2), np.float64)
    U[np.arange(H * W), y] = -math.log(1.0 - flip)
    U[np.arange(H * W), 1 - y] = -math.log(flip)
    return dict(kind="grid", H=H, W=W, L=2, conn=4, U=_f32(U), mu=_f32(potts(2, coupling)),
                w=_f32(constant_edge_weights(H, W, 4, 1.0)), clean=clean, noisy=noisy,
                seed=seed)


def segmentation_grid(H: int = 512, W: int = 512, L: int = 21, conn: int = 8,
                      logit_std: float = 2.0, sigma_rgb: float = 0.1, seed: int = 1,
                      mu: np.ndarray | None = None) -> dict:
    rng = np.random.default_rng(seed)
    U = unary_from_logits(rng.normal(0.0, logit_std, size=(H * W, L)))
    m = symmetric_uniform(L, rng) if mu is None else np.asarray(mu, np.float64)
    rgb = smooth_field(H, W, 3, rng)
    w = edge_weights_from_colour(rgb, conn, sigma_rgb)
    return dict(kind="grid", H=H, W=W, L=L, conn=conn, U=_f32(U), mu=_f32(m), w=_f32(w),
                seed=seed)


def unrolled_batch(B: int = 16, H: int = 256, W: int = 256, L: int = 21, conn: int = 4,
                   logit_std: float = 2.0, sigma_rgb: float = 0.1, seed: int = 4) -> dict:
    """A batch for training through unrolled inference: per-instance unaries
    and colour-derived edge weights (as segmentation_grid), one mu shared by
    the batch, and a seeded label map y per instance (argmax of a smooth
    random field, so labels come in regions like a segmentation)."""
    rng = np.random.default_rng(seed)
    m = symmetric_uniform(L, rng)
    U = np.empty((B, H * W, L))
    w = np.empty((B, n_dirs(conn), H, W))
    y = np.empty((B, H * W), np.int32)
    for b in range(B):
        U[b] = unary_from_logits(rng.normal(0.0, logit_std, size=(H * W, L)))
        w[b] = edge_weights_from_colour(smooth_field(H, W, 3, rng), conn, sigma_rgb)
        y[b] = np.argmax(smooth_field(H, W, L, rng), axis=0).reshape(-1)
    return dict(kind="grid", B=B, H=H, W=W, L=L, conn=conn, U=_f32(U), mu=_f32(m), w=_f32(w), y=y,
                seed=seed)


def random_graph(N: int, n_edges: int, L: int, seed: int, symmetric: bool = True,
                 coupling_scale: float = 1.0) -> dict:
    """General pairwise graph: n_edges oriented edges between distinct random
    variables, weights U(0.2, 1), random (a)symmetric mu, random unaries."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, N, n_edges)
    dst = (src + rng.integers(1, N, n_edges)) % N
    w = rng.uniform(0.2, 1.0, n_edges)
    m = symmetric_uniform(L, rng) if symmetric else rng.uniform(-1.0, 1.0, size=(L, L))
    U = unary_from_logits(rng.normal(0.0, 2.0, size=(N, L)))
    return dict(kind="sparse", N=N, L=L, U=_f32(U), mu=_f32(coupling_scale * m),
                src=src.astype(np.int32), dst=dst.astype(np.int32), w=_f32(w), seed=seed)


def dbn_layers(n_top: int = 256, n_bottom: int = 512, fan: int = 32, L: int = 2, seed: int = 11) -> dict:
    """Bipartite graph shaped like the layers of a deep belief network: each
    top variable connects to `fan` random bottom variables (weights U(0.2,1)),
    Potts-like symmetric coupling, random unaries."""
    rng = np.random.default_rng(seed)
    src = np.repeat(np.arange(n_top), fan)
    dst = np.concatenate([n_top + rng.choice(n_bottom, fan, replace=False) for _ in range(n_top)])
    w = rng.uniform(0.2, 1.0, src.size)
    N = n_top + n_bottom
    U = unary_from_logits(rng.normal(0.0, 1.0, size=(N, L)))
    m = 0.3 * symmetric_uniform(L, rng)
    return dict(kind="sparse", N=N, L=L, U=_f32(U), mu=_f32(m), src=src.astype(np.int32),
                dst=dst.astype(np.int32), w=_f32(w), seed=seed)


def random_grid(H: int, W: int, L: int, conn: int, seed: int, symmetric: bool = True,
                coupling_scale: float = 1.0, unary_scale: float = 2.0) -> dict:
    """Generic test instance: random unaries, random (a)symmetric mu, random w."""
    rng = np.random.default_rng(seed)
    U = unary_from_logits(rng.normal(0.0, unary_scale, size=(H * W, L)))
    if symmetric:
        m = symmetric_uniform(L, rng)
    else:
        m = rng.uniform(-1.0, 1.0, size=(L, L))
    w = random_edge_weights(H, W, conn, rng)
    return dict(kind="grid", H=H, W=W, L=L, conn=conn, U=_f32(U),
                mu=_f32(coupling_scale * m), w=_f32(w), seed=seed)


def dense_gaussian(side: int = 96, L: int = 21, theta_pos: float = 3.0,
                   theta_rgb: float = 13.0, logit_std: float = 2.0, seed: int = 2) -> dict:
    rng = np.random.default_rng(seed)
    N = side * side
    U = unary_from_logits(rng.normal(0.0, logit_std, size=(N, L)))
    mu = (1.0 - np.eye(L)) + 0.5 * symmetric_uniform(L, rng)
    rgb = smooth_field(side, side, 3, rng) * 255.0
    yy, xx = np.meshgrid(np.arange(side, dtype=np.float64), np.arange(side, dtype=np.float64),
                         indexing="ij")
    feats = np.stack([xx.reshape(-1), yy.reshape(-1), rgb[0].reshape(-1), rgb[1].reshape(-1),
                      rgb[2].reshape(-1)], axis=1)
    return dict(kind="dense", N=N, L=L, U=_f32(U), mu=_f32(mu), feats=_f32(feats),
                theta=(float(theta_pos), float(theta_rgb)), seed=seed)


def random_logq(N: int, L: int, seed: int, concentration: float = 0.5) -> np.ndarray:
    """log of a random point of the simplex product (Dirichlet draw per
    variable), as float32; zeros are avoided by flooring at 1e-30."""
    rng = np.random.default_rng(seed)
    q = rng.dirichlet(np.full(L, concentration), size=N)
    return _f32(np.log(np.maximum(q, 1e-30)))


def lanczos_start(N: int, L: int, seed: int = 12345) -> np.ndarray:
    """Start vector for Krylov eigenvalue estimates (the random draw of the
    power / Lanczos method)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((N, L))
