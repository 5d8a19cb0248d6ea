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
    """rw_mlp_forward: the last hidden layer's epilogue computes the output
    layer itself on the tensor-core path; it agrees with the unfused path
    to FP32 accumulation error (the chunks of max_batch rows included)."""
    m = model(max_batch=4096)
    g = torch.Generator().manual_seed(11)
    x = torch.randn(10007, 40, generator=g).to(DEV)
    outs = {}
    for kind in ("tcgen05", "mma_sync"):
        o = torch.empty(10007, 2, dtype=torch.float32, device=DEV)
        m.set_gemm(kind)
        m.forward(x, o)
        m.status()
        outs[kind] = o.cpu().numpy()
    d = np.abs(outs["tcgen05"] - outs["mma_sync"])
    assert np.max(d / (np.abs(outs["mma_sync"]) + 1e-2)) < 2e-2  # BF16 activations may round differently
    assert np.median(d / (np.abs(outs["mma_sync"]) + 1e-2)) < 1e-3
    m.close()
