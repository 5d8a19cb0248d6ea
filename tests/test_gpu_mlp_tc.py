"""The surrogate MLP's tensor-core GEMM (tcgen05.mma fed by TMA, FP32
accumulators in tensor memory) against a float64 product of the same BF16
operands, element by element, and against the mma.sync path.

Bound for an FP32 accumulation of K = 256 products of BF16 values (exact in
FP32) in any order: |Z - Z_exact| <= K u_32 sum_k |a_k w_k| + |b| u_32, with
u_32 = 2^-24; BF16(SiLU(Z)) may then differ by one BF16 unit where Z sits at
a rounding boundary.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2312_07440_gb300 import rwgt  # noqa: E402

DEV = torch.device("cuda", 0)
HIDDEN = 256


def model(seed=5, n_layers=4, max_batch=8192):
    return rwgt.Mlp(0, torch.cuda.current_stream(DEV).cuda_stream, n_in=40, hidden=HIDDEN, n_layers=n_layers,
                    max_batch=max_batch, seed=seed)


def layer_weights(m, layer):
    """(W [K][N] rounded to BF16 as float64, b [N] float64) of a hidden layer."""
    p = m.get_state()["params"]
    off, K, N = 0, 40, HIDDEN
    for l in range(layer):
        off += K * N + N
        K = HIDDEN
    W = torch.from_numpy(p[off:off + K * N].reshape(K, N)).to(torch.bfloat16).to(torch.float64).numpy()
    b = p[off + K * N:off + K * N + N].astype(np.float64)
    return W, b


def random_bf16(n, seed):
    g = torch.Generator().manual_seed(seed)
    return (torch.randn(n, HIDDEN, generator=g) * 1.5).to(torch.bfloat16)


@pytest.mark.parametrize("n", [1, 127, 128, 1000, 128 * 300 + 17])
@pytest.mark.parametrize("layer", [1, 3])
def test_tensor_core_layer_matches_float64_product(n, layer):
    m = model()
    W, b = layer_weights(m, layer)
    a = random_bf16(n, seed=n + layer)
    z = torch.empty(n, HIDDEN, dtype=torch.float32, device=DEV)
    h = torch.empty(n, HIDDEN, dtype=torch.bfloat16, device=DEV)
    m.set_gemm("tcgen05")
    m.hidden_layer(layer, a.to(DEV), z, h)
    m.status()
    A = a.to(torch.float64).numpy()
    exact = A @ W + b
    bound = HIDDEN * 2.0 ** -24 * (np.abs(A) @ np.abs(W) + np.abs(b)) + 1e-30
    zg = z.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(zg - exact) <= bound), f"max excess {np.max(np.abs(zg - exact) / bound):.3g}"
    # the activation: BF16 of SiLU of the GPU's own Z (SiLU in FP32 with the fast exponential)
    hz = torch.from_numpy(zg).float()
    h_ref = (hz * torch.sigmoid(hz)).to(torch.bfloat16).to(torch.float32)
    hg = h.float().cpu()
    ulp = torch.abs(h_ref) * 2.0 ** -7 + 1e-30
    assert torch.all(torch.abs(hg - h_ref) <= ulp)
    m.close()


def test_tensor_core_and_mma_sync_agree():
    m = model()
    n = 5000
    a = random_bf16(n, seed=3).to(DEV)
    out = {}
    for kind in ("tcgen05", "mma_sync"):
        z = torch.empty(n, HIDDEN, dtype=torch.float32, device=DEV)
        h = torch.empty(n, HIDDEN, dtype=torch.bfloat16, device=DEV)
        m.set_gemm(kind)
        m.hidden_layer(2, a, z, h)
        m.status()
        out[kind] = z.cpu().numpy().astype(np.float64)
    W, b = layer_weights(m, 2)
    scale = np.abs(a.to(torch.float64).cpu().numpy()) @ np.abs(W) + np.abs(b)
    assert np.all(np.abs(out["tcgen05"] - out["mma_sync"]) <= 2 * HIDDEN * 2.0 ** -24 * scale)
    m.close()


def test_inference_with_the_fused_output_layer():
    """rw_mlp_forward layer by layer: the last hidden layer's epilogue
    computes the output layer itself on the tensor-core path; it agrees with
    the unfused path to FP32 accumulation error (the chunks of max_batch rows
    included)."""
    m = model(max_batch=4096)
    g = torch.Generator().manual_seed(11)
    x = torch.randn(10007, 40, generator=g).to(DEV)
    outs = {}
    for kind in ("tcgen05_layers", "mma_sync"):
        o = torch.empty(10007, 2, dtype=torch.float32, device=DEV)
        m.set_gemm(kind)
        m.forward(x, o)
        m.status()
        outs[kind] = o.cpu().numpy()
    d = np.abs(outs["tcgen05_layers"] - outs["mma_sync"])
    assert np.max(d / (np.abs(outs["mma_sync"]) + 1e-2)) < 2e-2  # BF16 activations may round differently
    assert np.median(d / (np.abs(outs["mma_sync"]) + 1e-2)) < 1e-3
    m.close()


# --------------------------------------------------------------------------
# The whole network in one kernel (rw_mlp_forward on the tensor-core path)
# --------------------------------------------------------------------------
U32 = 2.0 ** -24
N_IN = 40
# rows: several 128-row tile pairs per CTA on a 152-SM GPU, an odd tile count
# (the last pair has one tile) and a ragged last tile
ROWS = [1, 127, 129, 128 * 152 * 4 + 77]


def _bf16(a32):
    return torch.from_numpy(np.ascontiguousarray(a32, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _f32_down(a):
    f = a.astype(np.float32)
    return np.where(f.astype(np.float64) > a, np.nextafter(f, np.float32(-np.inf)), f)


def _f32_up(a):
    f = a.astype(np.float32)
    return np.where(f.astype(np.float64) < a, np.nextafter(f, np.float32(np.inf)), f)


def _silu(z):
    return z / (1.0 + np.exp(-z))


def random_model(n_layers, seed):
    """A model with random weights and biases (every parameter nonzero)."""
    m = rwgt.Mlp(0, torch.cuda.current_stream(DEV).cuda_stream, n_in=N_IN, hidden=HIDDEN, n_layers=n_layers,
                 max_batch=4096, seed=seed)
    rng = np.random.default_rng(seed)
    p = np.empty(m.n_params, np.float32)
    off, K = 0, N_IN
    for l in range(n_layers + 1):
        N = 2 if l == n_layers else HIDDEN
        p[off:off + K * N] = rng.normal(0, 1.3 / np.sqrt(K), K * N)
        p[off + K * N:off + K * N + N] = rng.normal(0, 0.4, N)
        off += K * N + N
        K = HIDDEN
    m.set_state(p)
    return m, p


def interval_forward(p, x32, n_layers):
    """The kernel's arithmetic in float64 with every rounding bounded:
    (mid, rad) of the output such that the GPU's value lies in mid +- rad.
    Input layer: [x_h | x_l | x_h] . [W_h ; W_h ; W_l] (parts rounded to BF16)
    with FP32 accumulation over K = 128; hidden layers: BF16 activations
    (the interval keeps both BF16 neighbours where the rounding could go
    either way) times BF16 weights, FP32 accumulation over K = 256; SiLU in
    FP32 with the fast exponential and division (relative error <= 2^-20);
    output layer in FP32 from the unrounded last activation."""
    off, K = 0, N_IN
    Ws, bs = [], []
    for l in range(n_layers + 1):
        N = 2 if l == n_layers else HIDDEN
        Ws.append(p[off:off + K * N].reshape(K, N))
        bs.append(p[off + K * N:off + K * N + N].astype(np.float64))
        off += K * N + N
        K = HIDDEN
    xh = _bf16(x32)
    xl = _bf16((x32.astype(np.float32) - xh.astype(np.float32)))
    Wh = _bf16(Ws[0])
    Wl = _bf16(Ws[0].astype(np.float32) - Wh.astype(np.float32))
    z = xh @ Wh + xl @ Wh + xh @ Wl + bs[0]
    zr = 128 * U32 * (np.abs(xh) @ np.abs(Wh) + np.abs(xl) @ np.abs(Wh) + np.abs(xh) @ np.abs(Wl) + np.abs(bs[0]))
    for l in range(1, n_layers):
        s = _silu(z)
        sr = 1.1 * zr + 2.0 ** -20 * np.abs(s) + 1e-30
        h_lo, h_hi = _bf16(_f32_down(s - sr)), _bf16(_f32_up(s + sr))
        hm, hr = (h_lo + h_hi) / 2, (h_hi - h_lo) / 2
        Wb = _bf16(Ws[l])
        z = hm @ Wb + bs[l]
        zr = hr @ np.abs(Wb) + 256 * U32 * ((np.abs(hm) + hr) @ np.abs(Wb) + np.abs(bs[l]))
    s = _silu(z)
    sr = 1.1 * zr + 2.0 ** -20 * np.abs(s) + 1e-30
    Wo = Ws[n_layers].astype(np.float64)
    out = s @ Wo + bs[n_layers]
    out_r = sr @ np.abs(Wo) + 261 * U32 * ((np.abs(s) + sr) @ np.abs(Wo) + np.abs(bs[n_layers]))
    return out, out_r


@pytest.mark.parametrize("n_layers", [1, 2])
@pytest.mark.parametrize("n", ROWS)
def test_whole_network_kernel_matches_interval_reference(n_layers, n):
    """Element by element against the interval reference.  One layer: no
    BF16 activation in between, so the bound is tight (~1e-3 of the output's
    size; dropping one of the split input layer's three products exceeds it
    ninefold).  Two layers: one hidden layer's BF16 A operand written by the
    epilogue, the interval ~2 % of the output (a wrong bias, weight block or
    swizzle is far outside it).  Deeper networks: the interval grows with
    every BF16 rounding that could go either way, so they are compared with
    the layer-by-layer path below."""
    m, p = random_model(n_layers, seed=17 + n_layers)
    g = torch.Generator().manual_seed(n)
    x = (torch.randn(n, N_IN, generator=g) * 1.5).float()
    out = torch.full((n, 2), float("nan"), dtype=torch.float32, device=DEV)
    m.set_gemm("tcgen05")
    m.forward(x.to(DEV), out)
    m.status()
    mid, rad = interval_forward(p, x.numpy(), n_layers)
    og = out.cpu().numpy().astype(np.float64)
    excess = np.abs(og - mid) / rad
    assert np.all(excess <= 1.0), f"max excess {excess.max():.3g} at {np.unravel_index(excess.argmax(), excess.shape)}"
    if n_layers == 1:
        # no BF16 activation in between: the split input layer is FP32 up to
        # the dropped x_l W_l, so the output is within ~2^-15 of the FP32 network
        off = N_IN * HIDDEN
        W0, b0 = p[:off].reshape(N_IN, HIDDEN).astype(np.float64), p[off:off + HIDDEN].astype(np.float64)
        Wo = p[off + HIDDEN:off + HIDDEN + 2 * HIDDEN].reshape(HIDDEN, 2).astype(np.float64)
        bo = p[off + HIDDEN + 2 * HIDDEN:].astype(np.float64)
        s = _silu(x.numpy().astype(np.float64) @ W0 + b0)
        exact = s @ Wo + bo
        scale = (np.abs(x.numpy()) @ np.abs(W0) + np.abs(b0)) @ np.abs(Wo) * 1.1 + np.abs(s) @ np.abs(Wo)
        assert np.all(np.abs(og - exact) <= 2.0 ** -15 * scale)
    m.close()


def test_whole_network_kernel_and_layer_by_layer_agree():
    """The one-kernel inference and the layer-by-layer tensor-core path (FP32
    input layer, the output layer fused into the last hidden layer) compute
    the same network; they differ only where a BF16 rounding of an activation
    goes the other way."""
    m, _ = random_model(4, seed=3)
    g = torch.Generator().manual_seed(4)
    x = (torch.randn(20011, N_IN, generator=g) * 1.5).to(DEV)
    outs = {}
    for kind in ("tcgen05", "tcgen05_layers"):
        o = torch.empty(20011, 2, dtype=torch.float32, device=DEV)
        m.set_gemm(kind)
        m.forward(x, o)
        m.status()
        outs[kind] = o.cpu().numpy().astype(np.float64)
    # the hidden layers and the output layer are the same instructions on the
    # same operands: rows where no activation rounds the other way agree to
    # the bit; elsewhere a few BF16 units of activations move the output by
    # a small fraction of its spread
    a, b = outs["tcgen05"], outs["tcgen05_layers"]
    same = np.mean(a == b)
    d = np.abs(a - b) / np.std(b, axis=0)
    assert same > 0.5 and np.max(d) < 2e-2, (same, np.median(d), np.max(d))
    # deterministic: a second run gives the same bits
    o = torch.empty(20011, 2, dtype=torch.float32, device=DEV)
    m.set_gemm("tcgen05")
    m.forward(x, o)
    m.status()
    assert np.array_equal(o.cpu().numpy().astype(np.float64), outs["tcgen05"])
    m.close()
