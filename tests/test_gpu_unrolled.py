"""GPU reverse mode through K unrolled proximal steps against the FP64 oracle.

The loss is the cross-entropy of q^K against a label map,
    loss = -(1/(B n)) sum_b sum_i log q^K_{b,i,y_bi},
so d loss / d log q^K is -1/(B n) at the labelled entries.  The oracle's
reverse mode is itself pinned by central differences (CPU suite); here the
GPU gradients (FP32 arithmetic) must agree with it to
    |g - g_ref|max <= TOL_G * max|g_ref| + 1e-7,
TOL_G = 1e-4: FP32 messages carry about 1e-6 relative error per step, and the
backward pass of K = 10 steps goes through 2K products with the same
operators.  A few coordinates are also checked directly against FP64
central differences of the oracle's loss.
"""
import numpy as np
import pytest

from paper_1511_06103_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_G = 1e-4


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


def edge_mask(H, W, conn):
    """[n_dirs][H][W] True where direction k leaves (y, x) inside the grid
    (direction 0 right, 1 down, 2 down-right, 3 down-left)."""
    dy, dx = [0, 1, 1, 1], [1, 0, 1, -1]
    nd = 4 if conn == 8 else 2
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    return np.stack([(yy + dy[k] < H) & (xx + dx[k] >= 0) & (xx + dx[k] < W) for k in range(nd)])


def oracle_grads(oracle, U, mu, w, H, W, conn, eta, K, y):
    """(loss, dU [n][L], dmu [L][L], dw [n_dirs][H][W]) of one instance."""
    m = oracle.Model.grid(f64(U), f64(mu), f64(w), H, W, conn)
    mask = edge_mask(H, W, conn)
    loss, dU, dmu, dw_e = m.unrolled_grad(eta, K, y, int(mask.sum()))
    dw = np.zeros(mask.shape)
    dw[mask] = dw_e      # the oracle lists edges direction-major, then row, then column
    return loss, dU, dmu, dw


def gpu_grads(binding, torch, d, eta, K, on_device=True, precision=0):
    B = d["U"].shape[0] if d["U"].ndim == 3 else 1
    U = d["U"].reshape(B, d["H"] * d["W"], d["L"])
    w = d["w"].reshape(B, -1, d["H"], d["W"])
    y = np.asarray(d["y"]).reshape(B, -1)
    topo = binding.CRF_GRID8 if d["conn"] == 8 else binding.CRF_GRID4
    crf = binding.CRF(topo, d["L"], d["H"], d["W"], batch=B, precision=precision)
    crf.set_unary(torch.from_numpy(U).cuda())
    crf.set_pairwise(torch.from_numpy(d["mu"]).cuda(), torch.from_numpy(np.ascontiguousarray(w)).cuda())
    ckpt = torch.empty(crf.checkpoint_floats(K), dtype=torch.float32, device="cuda")
    crf.unrolled_forward(K, eta, ckpt)
    logq = crf.log_marginals(torch.empty((B, crf.N, d["L"]), dtype=torch.float32, device="cuda"))
    n = crf.N
    g = np.zeros((B, n, d["L"]), np.float32)
    g[np.arange(B)[:, None], np.arange(n)[None, :], y] = -1.0 / (B * n)
    if on_device:
        dU, dmu, dw = crf.unrolled_backward(K, eta, ckpt, torch.from_numpy(g).cuda())
        dU, dmu, dw = dU.cpu().numpy(), dmu.cpu().numpy(), dw.cpu().numpy()
    else:
        dU, dmu, dw = crf.unrolled_backward(K, eta, ckpt, g)
    lq = logq.cpu().numpy()
    loss = -lq[np.arange(B)[:, None], np.arange(n)[None, :], y].mean()
    crf.close()
    return float(loss), dU, dmu, dw


def close(g, ref):
    g, ref = f64(g), f64(ref)
    return np.abs(g - ref).max() <= TOL_G * np.abs(ref).max() + 1e-7


@pytest.mark.parametrize("conn,sym,eta", [(4, True, 0.3), (4, False, 0.5), (8, True, 0.25), (8, False, 1.0)])
def test_adjoint_matches_oracle_8x8_L3(env, conn, sym, eta):
    binding, oracle, torch = env
    d = synth.random_grid(8, 8, 3, conn, seed=70 + conn + int(sym), symmetric=sym)
    d["y"] = np.random.default_rng(5).integers(0, 3, 64).astype(np.int32)
    K = 10
    loss, dU, dmu, dw = gpu_grads(binding, torch, d, eta, K)
    lref, dUr, dmur, dwr = oracle_grads(oracle, d["U"], d["mu"], d["w"], 8, 8, conn, eta, K, d["y"])
    assert abs(loss - lref) <= 1e-5 * abs(lref)
    assert close(dU[0], dUr)
    assert close(dmu, dmur)
    assert close(dw[0], dwr)


@pytest.mark.parametrize("L,conn,sym", [(2, 4, True), (2, 8, False), (12, 8, True), (16, 4, False),
                                         (20, 8, True), (24, 4, True), (24, 8, False)])
def test_adjoint_label_counts(env, L, conn, sym):
    """Every label-count instantiation; 13 x 70 grids span three 32-wide
    and four 4-high tiles with ragged tails."""
    binding, oracle, torch = env
    H, W, K, eta = 13, 70, 4, 0.3
    d = synth.random_grid(H, W, L, conn, seed=200 + L + conn, symmetric=sym)
    d["y"] = np.random.default_rng(L).integers(0, L, H * W).astype(np.int32)
    loss, dU, dmu, dw = gpu_grads(binding, torch, d, eta, K)
    lref, dUr, dmur, dwr = oracle_grads(oracle, d["U"], d["mu"], d["w"], H, W, conn, eta, K, d["y"])
    assert abs(loss - lref) <= 1e-5 * abs(lref)
    assert close(dU[0], dUr)
    assert close(dmu, dmur)
    assert close(dw[0], dwr)


def test_adjoint_matches_finite_differences(env):
    """Direct FP64 central differences of the oracle's loss at a few
    coordinates of U, mu and w (h = 1e-6)."""
    binding, oracle, torch = env
    H = W = 8
    L, conn, K, eta = 3, 4, 10, 0.4
    d = synth.random_grid(H, W, L, conn, seed=91, symmetric=False)
    d["y"] = np.random.default_rng(6).integers(0, L, H * W).astype(np.int32)
    _, dU, dmu, dw = gpu_grads(binding, torch, d, eta, K)
    U, mu, w = f64(d["U"]), f64(d["mu"]), f64(d["w"])
    h = 1e-6

    def loss(U_, mu_, w_):
        return oracle.Model.grid(U_, mu_, w_, H, W, conn).unrolled_loss(eta, K, d["y"])

    checks = []
    for (i, l) in [(0, 0), (27, 2), (63, 1)]:
        Up, Um = U.copy(), U.copy()
        Up[i, l] += h
        Um[i, l] -= h
        checks.append((dU[0, i, l], (loss(Up, mu, w) - loss(Um, mu, w)) / (2 * h)))
    for (a, c) in [(0, 1), (2, 0), (1, 1)]:
        mp, mm = mu.copy(), mu.copy()
        mp[a, c] += h
        mm[a, c] -= h
        checks.append((dmu[a, c], (loss(U, mp, w) - loss(U, mm, w)) / (2 * h)))
    for (k, y, x) in [(0, 3, 4), (1, 0, 7), (1, 6, 2)]:
        wp, wm = w.copy(), w.copy()
        wp[k, y, x] += h
        wm[k, y, x] -= h
        checks.append((dw[0, k, y, x], (loss(U, mu, wp) - loss(U, mu, wm)) / (2 * h)))
    scale = max(abs(f) for _, f in checks)
    for g, fd in checks:
        assert abs(g - fd) <= TOL_G * scale + 1e-7, (g, fd)


@pytest.mark.parametrize("conn", [4, 8])
def test_adjoint_matches_oracle_L21_batch(env, conn):
    """Batch of 2 ragged grids (40 x 37: tail tiles), L = 21, Lambda-based eta."""
    binding, oracle, torch = env
    d = synth.unrolled_batch(B=2, H=40, W=37, L=21, conn=conn, seed=8)
    K = 10
    crf = binding.CRF(binding.CRF_GRID8 if conn == 8 else binding.CRF_GRID4, 21, 40, 37, batch=2)
    crf.set_pairwise(d["mu"], d["w"])
    _, eta_b = crf.lipschitz()
    crf.close()
    loss, dU, dmu, dw = gpu_grads(binding, torch, d, 0.0, K)
    dmu_ref = np.zeros((21, 21))
    lref = 0.0
    for b in range(2):
        # eta in FP32 as the device applies it
        e = float(np.float32(eta_b[b]))
        lb, dUr, dmur, dwr = oracle_grads(oracle, d["U"][b], d["mu"], d["w"][b], 40, 37, conn, e, K, d["y"][b])
        assert close(dU[b], dUr / 2)
        assert close(dw[b], dwr / 2)
        dmu_ref += dmur / 2
        lref += lb / 2
    assert close(dmu, dmu_ref)
    assert abs(loss - lref) <= 1e-5 * abs(lref)


def test_adjoint_host_and_device_outputs_agree_bitwise(env):
    binding, oracle, torch = env
    d = synth.random_grid(19, 23, 5, 8, seed=12, symmetric=False)
    d["y"] = np.random.default_rng(7).integers(0, 5, 19 * 23).astype(np.int32)
    a = gpu_grads(binding, torch, d, 0.35, 6, on_device=True)
    b = gpu_grads(binding, torch, d, 0.35, 6, on_device=False)
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_autograd_function(env):
    binding, oracle, torch = env
    from paper_1511_06103_gb300.unrolled import unrolled_log_marginals
    d = synth.random_grid(8, 8, 3, 4, seed=33, symmetric=True)
    y = np.random.default_rng(8).integers(0, 3, 64)
    U = torch.from_numpy(d["U"]).cuda()[None].requires_grad_(True)
    mu = torch.from_numpy(d["mu"]).cuda().requires_grad_(True)
    w = torch.from_numpy(d["w"]).cuda()[None].requires_grad_(True)
    logq = unrolled_log_marginals(U, mu, w, 8, 8, 4, 10, 0.3)
    yt = torch.from_numpy(y).cuda()
    loss = -logq[0, torch.arange(64, device="cuda"), yt].mean()
    loss.backward()
    lref, dUr, dmur, dwr = oracle_grads(oracle, d["U"], d["mu"], d["w"], 8, 8, 4, 0.3, 10, y.astype(np.int32))
    assert abs(loss.item() - lref) <= 1e-5 * abs(lref)
    assert close(U.grad[0].cpu().numpy(), dUr)
    assert close(mu.grad.cpu().numpy(), dmur)
    assert close(w.grad[0].cpu().numpy(), dwr)


def test_adjoint_full_size_sampled(env):
    """16 x 256 x 256, L = 21, 4-connected, K = 10 (the training workload):
    instances 0 and 15 against the oracle, and a repeat run bit for bit."""
    binding, oracle, torch = env
    d = synth.unrolled_batch()
    B, H, W, L, K, eta = 16, 256, 256, 21, 10, 0.25
    r1 = gpu_grads(binding, torch, d, eta, K)
    r2 = gpu_grads(binding, torch, d, eta, K)
    for x, y in zip(r1[1:], r2[1:]):
        assert np.array_equal(x, y)
    _, dU, dmu, dw = r1
    assert np.all(np.isfinite(dmu))
    for b in (0, 15):
        _, dUr, _, dwr = oracle_grads(oracle, d["U"][b], d["mu"], d["w"][b], H, W, 4, eta, K, d["y"][b])
        assert close(dU[b], dUr / B)
        assert close(dw[b], dwr / B)


def test_adjoint_bf16_forward(env):
    """BF16 tensor-core messages in the forward steps (16 x 64 x 64, L = 21,
    4-connected, K = 10): the loss and the gradients stay within 2% of the
    FP64 reference (the trajectory itself carries the BF16 message error)."""
    binding, oracle, torch = env
    d = synth.unrolled_batch(B=2, H=64, W=64, L=21, conn=4, seed=9)
    K, eta = 10, 0.25
    loss, dU, dmu, dw = gpu_grads(binding, torch, d, eta, K, precision=binding.CRF_BF16)
    dmu_ref = np.zeros((21, 21))
    lref = 0.0
    for b in range(2):
        lb, dUr, dmur, dwr = oracle_grads(oracle, d["U"][b], d["mu"], d["w"][b], 64, 64, 4, eta, K, d["y"][b])
        assert np.abs(dU[b] - dUr / 2).max() <= 2e-2 * np.abs(dUr / 2).max()
        assert np.abs(dw[b] - dwr / 2).max() <= 2e-2 * np.abs(dwr / 2).max()
        dmu_ref += dmur / 2
        lref += lb / 2
    assert np.abs(dmu - dmu_ref).max() <= 2e-2 * np.abs(dmu_ref).max()
    assert abs(loss - lref) <= 1e-3 * abs(lref)


def test_adjoint_rejects_unsupported(env):
    binding, oracle, torch = env
    crf = binding.CRF(binding.CRF_GRID4, 28, 8, 8)
    with pytest.raises(binding.ProxMFError, match="UNSUPPORTED"):
        crf.checkpoint_floats(3)
    crf.close()
    crf = binding.CRF(binding.CRF_GRID4, 3, 8, 8)
    with pytest.raises(binding.ProxMFError, match="INVALID"):
        crf.checkpoint_floats(0)
    crf.close()
