"""Tensor-core kernels of the initial-guess network against the numpy layers of
oracle/warmstart_oracle.py, evaluated on the same BF16-rounded operands.  Needs a GB300 (sm_103a).

Tolerances: a product of two BF16 numbers is exact in FP32, so the tensor-core results differ from
the FP64 reference only by the FP32 summation of at most 432 products per output (convolutions) or
27 x 16 x n^3 / 27 products per weight (weight gradient): ~1e-6 and ~1e-5 relative to the largest
entry.  Convolution outputs are stored as BF16 (8 significant bits), so they are compared with the
reference rounded to BF16, within one BF16 step.
"""
import numpy as np
import pytest
import torch

from oracle import warmstart_oracle as wo

pytestmark = pytest.mark.gpu

smg = pytest.importorskip("paper_2312_10615_gb300")
DEV = torch.device("cuda:0")


def _bf(a):
    """BF16-rounded copy as float64 (numpy) and the BF16 device tensor."""
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.to(torch.float64).numpy(), t.to(DEV)


def _within_bf16_step(y, ref):
    scale = np.max(np.abs(ref))
    return np.all(np.abs(y - ref) <= 2.0 ** -7 * np.abs(ref) + 1e-5 * scale)


def test_tcgen05_mma_operand_layout():
    """one 128 x 16 x 16 MMA on small integers (exact in BF16 and FP32): D = A B^T exactly"""
    rng = np.random.default_rng(0)
    A = rng.integers(-8, 9, (128, 16)).astype(np.float32)
    B = rng.integers(-8, 9, (16, 16)).astype(np.float32)
    a = torch.from_numpy(A).to(torch.bfloat16).to(DEV)
    b = torch.from_numpy(B).to(torch.bfloat16).to(DEV)
    d = torch.zeros(128, 16, dtype=torch.float32, device=DEV)
    assert smg.warmstart_mma_check(a, b, d) == smg.OK
    assert np.array_equal(d.cpu().numpy(), A @ B.T)


@pytest.mark.parametrize("n,ci", [(16, 16), (24, 16), (32, 4), (64, 16), (128, 16), (128, 4)])
def test_tensor_core_convolution(n, ci):
    rng = np.random.default_rng(n + ci)
    x64, x = _bf(rng.standard_normal((n, n, n, ci)))
    w = (rng.standard_normal((27, ci, 16)) / np.sqrt(27 * ci)).astype(np.float32)
    w64, _ = _bf(w)
    y = torch.zeros(n, n, n, 16, dtype=torch.bfloat16, device=DEV)
    assert smg.warmstart_conv_check(n, ci, 0, 1, x, torch.from_numpy(w).to(DEV), y) == smg.OK
    ref = torch.from_numpy(wo.act(wo.conv(x64, w64))).to(torch.bfloat16).to(torch.float64).numpy()
    assert _within_bf16_step(y.to(torch.float64).cpu().numpy(), ref)
    # the CUDA-core kernel (FP32 weights) agrees to the weights' BF16 rounding
    y0 = torch.zeros_like(y)
    assert smg.warmstart_conv_check(n, ci, 0, 0, x, torch.from_numpy(w).to(DEV), y0) == smg.OK
    d = (y0.to(torch.float64) - y.to(torch.float64)).abs().max().item()
    assert d <= 2e-2 * np.max(np.abs(ref))


@pytest.mark.parametrize("n", [16, 40, 128])
def test_tensor_core_data_gradient(n):
    rng = np.random.default_rng(n)
    g = rng.standard_normal((n, n, n, 16)).astype(np.float32)
    g64, _ = _bf(g)
    w = (rng.standard_normal((27, 16, 16)) / np.sqrt(432)).astype(np.float32)
    w64, _ = _bf(w)
    out = torch.zeros(n, n, n, 16, dtype=torch.float32, device=DEV)
    assert smg.warmstart_conv_check(n, 16, 1, 1, torch.from_numpy(g).to(DEV), torch.from_numpy(w).to(DEV), out) == smg.OK
    ref = wo.conv_bwd_data(g64, w64)
    err = np.max(np.abs(out.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err < 1e-5, err


@pytest.mark.parametrize("n,ci", [(16, 16), (24, 4), (64, 16)])
def test_tensor_core_weight_gradient(n, ci):
    rng = np.random.default_rng(7 * n + ci)
    x64, x = _bf(rng.standard_normal((n, n, n, ci)))
    g = rng.standard_normal((n, n, n, 16)).astype(np.float32)
    g64, _ = _bf(g)
    out = torch.zeros(27, ci, 16, dtype=torch.float32, device=DEV)
    w_unused = torch.zeros(27 * ci * 16, dtype=torch.float32, device=DEV)
    assert smg.warmstart_conv_check(n, ci, 2, 1, x, w_unused, out, g=torch.from_numpy(g).to(DEV)) == smg.OK
    ref = wo.conv_bwd_weight(x64, g64)
    err = np.max(np.abs(out.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err < 1e-4, err


def test_bf16_network_on_tensor_cores_matches_cuda_cores():
    """the whole network (forward and gradient) with BF16 activations: tensor cores vs CUDA cores"""
    import synthetic
    n = 32
    w = (synthetic.net_weights(2) * 0.5).astype(np.float32)
    m = (n + 1) * n * n * 3 + n ** 3
    b = torch.from_numpy(np.random.default_rng(1).standard_normal(m)).to(DEV)
    xs = torch.from_numpy(np.random.default_rng(2).standard_normal(m)).to(DEV)
    outs, grads = [], []
    for engine in (1, 0):
        ws = smg.WarmStart(n, smg.STORE_BF16, scale=0.7)
        ws.set_engine(engine)
        ws.set_weights(w)
        outs.append(ws.predict(b).cpu().numpy())
        grads.append(ws.loss_grad(b, xs, want_grad=True)[1].astype(np.float64))
        ws.close()
    assert np.max(np.abs(outs[0] - outs[1])) / np.max(np.abs(outs[1])) < 5e-2
    cos = float(grads[0] @ grads[1] / (np.linalg.norm(grads[0]) * np.linalg.norm(grads[1])))
    assert cos > 0.99, cos
