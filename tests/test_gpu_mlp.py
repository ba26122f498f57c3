"""Tensor-core (tcgen05) GEMM and the surrogate MLP vs the FP64 oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ms():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2207_09334_gb300 as ms
    ms.load()
    return ms


def bf16_round(a):
    import torch
    return torch.tensor(np.asarray(a, np.float32)).bfloat16().float().numpy().astype(np.float64)


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 384, 320), (1024, 512, 2048), (512, 2048, 1024)])
def test_gemm_matches_fp64(ms, M, N, K):
    import torch
    g = torch.Generator().manual_seed(M + N + K)
    A = torch.randn(M, K, generator=g).bfloat16()
    B = torch.randn(N, K, generator=g).bfloat16()
    ref = A.double() @ B.double().T
    out = ms.gemm_bf16(A.cuda(), B.cuda()).double().cpu()
    err = (out - ref).abs().max().item()
    bound = 1e-5 * (A.double().abs() @ B.double().abs().T).max().item()
    assert err <= bound, (err, bound)


@pytest.mark.parametrize("M,N,K", [(19456, 256, 192), (18944, 512, 1024)])
def test_gemm_wide_tiles_match_fp64(ms, M, N, K):
    """Problems with at least 148 tiles of 128 x 256 take the 256-wide tile
    (two B boxes per stage, 256 TMEM columns); K = 192 is shorter than the
    stage ring.  Checked on every 37th row against FP64."""
    import torch
    g = torch.Generator().manual_seed(M + N + K)
    A = torch.randn(M, K, generator=g).bfloat16()
    B = torch.randn(N, K, generator=g).bfloat16()
    out = ms.gemm_bf16(A.cuda(), B.cuda()).double().cpu()
    rows = torch.arange(0, M, 37)
    ref = A[rows].double() @ B.double().T
    err = (out[rows] - ref).abs().max().item()
    bound = 1e-5 * (A[rows].double().abs() @ B.double().abs().T).max().item()
    assert err <= bound, (err, bound)


@pytest.mark.parametrize("B", [1024, 16384])
def test_onehot_tiles_equal_the_materialised_input(ms, B):
    """Inference on a batch of materials builds the one-hot A tiles in shared
    memory (128-byte swizzled) instead of reading X: the predictions equal,
    bit for bit, those from the same one-hot matrix given as bf16 input, and
    those of the entry point that reads the caller's materials in place.
    B = 16384 takes the 128 x 256 tiles, B = 1024 the 128 x 128 ones."""
    import torch
    rng = np.random.default_rng(B)
    mats = torch.tensor(rng.integers(0, 4, size=(B, 512)).astype(np.uint8), device="cuda")
    x = torch.nn.functional.one_hot(mats.long(), 4).reshape(B, 2048).to(torch.bfloat16).contiguous()
    net = ms.Surrogate(2048, 512, max_batch=16384, seed=3)
    y1 = torch.empty(B, device="cuda"); y2 = torch.empty(B, device="cuda")
    net.load_materials(mats)
    net.forward(B, y1)
    net.load_input(x)
    net.forward(B, y2)
    y3 = net.forward_materials(mats)
    net.sync()
    assert torch.equal(y1, y2) and torch.equal(y1, y3)
    net.close()


def _mlp_case(ms, B=256, n_in=2048, h=512, seed=1):
    import torch
    rng = np.random.default_rng(seed)
    mats = rng.integers(0, 4, size=(B, n_in // 4)).astype(np.uint8)
    t = rng.normal(0, 1, B).astype(np.float32)
    net = ms.Surrogate(n_in, h, max_batch=max(B, 128), seed=seed)
    p = net.params().astype(np.float64)
    # the kernels multiply with bf16 copies of W1 and W2: give the oracle the same weights
    from oracle import mlp
    W1, b1, W2, b2, w3, b3 = mlp.unpack(p, n_in, h)
    pq = np.concatenate([bf16_round(W1).ravel(), b1, bf16_round(W2).ravel(), b2, w3, [b3]])
    X = mlp.one_hot(mats)
    dmats = torch.tensor(mats, device="cuda")
    dt = torch.tensor(t, device="cuda")
    return net, mlp, pq, X, t, dmats, dt


def close_elementwise(name, got, want, rel=1e-2, floor=1e-2):
    """Every element within rel of its reference value plus an absolute floor
    of `floor` times the block's largest reference magnitude (entries near
    zero have no meaningful relative error).  The BF16 storage of the
    activations (H1, H2), of the kept pre-activations (Z1, Z2) and of the
    back-propagated dZ1, dZ2 puts the kernel 2e-3 to 4e-3 of each block's
    largest entry away from the FP64 definition (an FP64 emulation of those
    rounding points, batch 256); a zeroed column of dW1 or a wrong bias entry
    is far outside this gate."""
    got = np.asarray(got, np.float64); want = np.asarray(want, np.float64)
    bound = rel * np.abs(want) + floor * np.abs(want).max()
    bad = np.abs(got - want) > bound
    assert not bad.any(), (name, int(bad.sum()), float(np.abs(got - want).max()), float(np.abs(want).max()))


def test_forward_and_gradients_match_oracle(ms):
    """Predictions, loss and every gradient block against the FP64 oracle
    (given the kernel's BF16 weights), element by element."""
    net, mlp, pq, X, t, dmats, dt = _mlp_case(ms)
    with net:
        B = X.shape[0]
        net.load_materials(dmats)
        y = net.forward(B).cpu().numpy()
        loss = float(net.backward(dt, B).item())
        g = net.grads().astype(np.float64)
    y_o, _ = mlp.forward(pq, X, 2048, 512)
    loss_o, g_o = mlp.loss_and_grad(pq, X, t, 2048, 512)
    close_elementwise("y", y, y_o)
    assert abs(loss - loss_o) <= 1e-2 * loss_o
    got = mlp.unpack(g, 2048, 512)
    want = mlp.unpack(g_o, 2048, 512)
    for name, a, b in zip(("W1", "b1", "W2", "b2", "w3"), got[:5], want[:5]):
        close_elementwise("d" + name, a, b)
    assert abs(got[5] - want[5]) <= 1e-2 * abs(want[5]) + 1e-7


def test_screening_pass_matches_oracle_on_sampled_rows(ms):
    """The screening configuration itself: 65 536 designs per forward pass,
    so both GEMMs take 128 x 256 tiles in the persistent grid (layer 1 with
    the one-hot tiles built on chip, layer 2 with the head folded into its
    epilogue).  512 sampled predictions against the FP64 oracle given the
    kernel's BF16 weights, element by element as in the forward test."""
    import torch
    from oracle import mlp
    B, n_in, h = 65536, 2048, 512
    rng = np.random.default_rng(17)
    mats = rng.integers(0, 4, size=(B, n_in // 4)).astype(np.uint8)
    with ms.Surrogate(n_in, h, max_batch=B, seed=5) as net:
        p = net.params().astype(np.float64)
        y = net.predict(torch.tensor(mats, device="cuda"), chunk=B).cpu().numpy()
        net.sync()
    W1, b1, W2, b2, w3, b3 = mlp.unpack(p, n_in, h)
    pq = np.concatenate([bf16_round(W1).ravel(), b1, bf16_round(W2).ravel(), b2, w3, [b3]])
    rows = rng.choice(B, size=512, replace=False)
    y_o, _ = mlp.forward(pq, mlp.one_hot(mats[rows]), n_in, h)
    close_elementwise("y", y[rows], y_o)


def test_fp32_accumulators_on_the_mlp_layers(ms):
    """Given bit-identical BF16 operands, the tensor-core accumulators are
    FP32 sums: the layer-1 pre-activation X W1^T (one-hot X, the model's own
    BF16 W1) and the layer-2 product H1 W2^T (H1 = the oracle's activations
    rounded to BF16, the model's BF16 W2) agree with FP64 products of the same
    operands to 1e-5 of each element's sum of |a||b|."""
    import torch
    net, mlp, pq, X, t, dmats, dt = _mlp_case(ms)
    with net:
        W1, b1, W2, b2, w3, b3 = mlp.unpack(pq, 2048, 512)     # already BF16-valued
        Xb = torch.tensor(X, dtype=torch.bfloat16)
        W1b = torch.tensor(W1, dtype=torch.bfloat16); W2b = torch.tensor(W2, dtype=torch.bfloat16)
        assert np.array_equal(W1b.double().numpy(), W1) and np.array_equal(W2b.double().numpy(), W2)
        H1b = torch.tensor(mlp.gelu(X @ W1.T + b1), dtype=torch.float32).bfloat16()
        for A, Bm in ((Xb, W1b), (H1b, W2b)):
            out = ms.gemm_bf16(A.cuda(), Bm.cuda()).double().cpu().numpy()
            Ad, Bd = A.double().numpy(), Bm.double().numpy()
            ref = Ad @ Bd.T
            scale = np.abs(Ad) @ np.abs(Bd).T
            err = np.abs(out - ref)
            assert (err <= 1e-5 * scale).all(), (err.max(), float((err / np.maximum(scale, 1e-30)).max()))


def test_adam_step_matches_oracle(ms):
    net, mlp, pq, X, t, dmats, dt = _mlp_case(ms, B=128)
    with net:
        p0 = net.params().astype(np.float64)
        net.load_materials(dmats)
        net.backward(dt, 128)
        g = net.grads().astype(np.float64)
        net.adam(1e-3)
        p1 = net.params().astype(np.float64)
    ref, _, _ = mlp.adam(p0, g, np.zeros_like(p0), np.zeros_like(p0), 1, lr=1e-3)
    np.testing.assert_allclose(p1, ref, rtol=0, atol=1e-6)


def test_training_fits_a_learnable_target(ms):
    """A target that is a fixed function of the one-hot design: Adam on the
    tensor-core kernels cuts the loss by 10x."""
    import torch
    rng = np.random.default_rng(5)
    N, B = 4096, 512
    mats = rng.integers(0, 4, size=(N, 512)).astype(np.uint8)
    from oracle import mlp
    wt = rng.normal(0, 1, 2048)
    tt = mlp.one_hot(mats) @ wt
    tt = ((tt - tt.mean()) / tt.std()).astype(np.float32)
    dm = torch.tensor(mats, device="cuda"); dtt = torch.tensor(tt, device="cuda")
    with ms.Surrogate(2048, 512, max_batch=B, seed=2) as net:
        first = None
        for it in range(400):
            s = (it * B) % N
            loss = float(net.train_step(dm[s:s + B], dtt[s:s + B], lr=1e-3).item())
            first = first if first is not None else loss
        net.sync()
    assert loss < 0.1 * first, (first, loss)


def _bf16_nearest(x):
    """bf16 nearest to each FP64 value (ties to even), computed exactly."""
    x = np.asarray(x, np.float64)
    m, e = np.frexp(np.abs(x))
    r = np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)       # np.rint: ties to even
    return np.where(x < 0, -r, r)


def test_gelu_of_every_input_range_matches_the_definition(ms):
    """The forward epilogues apply GELU(z) = z Phi(z) to bf16 pre-activations.
    A model whose unit k reads only voxel k (Z1_k = W1[k][4k + m], exact), with
    W2 = I (Z2 = H1, exact) and w3 = e_j, predicts y = GELU(GELU(z)) rounded to
    bf16 after each GELU.  512 values of z over +-[2^-12, 128] (both signs,
    zero, and the powers of two where the bf16 step changes) are checked
    against the FP64 definition: within one bf16 step of the value, plus the
    FP32 cancellation of 1 + erf(z / sqrt 2) in the negative tail (1e-7 |z|),
    and bit-equal for at least 98 % of the values with z >= -2."""
    import torch
    from oracle import mlp
    n_in, h, B = 512, 128, 128
    rng = np.random.default_rng(11)
    edges = [2.0 ** -7, 2.0 ** -7 * (1 - 2 ** -8), 7.96875, 8.0, 8.0625, 0.0, 2.0 ** -12, 100.0, 1.0, 0.5]
    z = np.concatenate([edges, [-e for e in edges]])
    mag = 2.0 ** rng.uniform(-12, 7, 4 * h - z.size)
    z = _bf16_nearest(np.concatenate([z, mag * rng.choice([-1.0, 1.0], mag.size)]))
    W1 = np.zeros((h, n_in)); W2 = np.eye(h)
    for k in range(h):
        W1[k, 4 * k:4 * k + 4] = z[4 * k:4 * k + 4]
    mats = torch.tensor(np.tile((np.arange(B) % 4)[:, None], (1, n_in // 4)).astype(np.uint8), device="cuda")
    got = np.empty(4 * h)
    with ms.Surrogate(n_in, h, max_batch=B, seed=0) as net:
        for j in range(h):
            w3 = np.zeros(h); w3[j] = 1.0
            net.set_params(np.concatenate([W1.ravel(), np.zeros(h), W2.ravel(), np.zeros(h), w3, [0.0]]))
            net.load_materials(mats)
            y = net.forward(B).cpu().numpy().astype(np.float64)
            got[4 * j:4 * j + 4] = y[:4]
        net.sync()
    e1 = _bf16_nearest(mlp.gelu(z))
    want = _bf16_nearest(mlp.gelu(e1))
    err = np.abs(got - want)
    assert (err <= 2.0 ** -7 * np.abs(want) + 1e-7 * np.abs(z) + 1e-30).all(), err.max()
    mild = z >= -2.0
    assert np.mean(got[mild] == want[mild]) >= 0.98, np.mean(got[mild] == want[mild])
