"""tcgen05 BF16 GEMMs of the MLP surrogate against plain PyTorch FP32
references of the same ops (on the same BF16-rounded operands)."""
import numpy as np
import pytest

from paper_1802_05839_gb300 import wx

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def rnd(*shape, scale=1.0, seed=0):
    g = torch.Generator(device="cpu").manual_seed(seed)
    return (torch.randn(*shape, generator=g) * scale).to(torch.bfloat16).cuda()


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 512, 256), (384, 128, 512), (4096, 512, 512),
                                   (128, 256, 4096)])
def test_gemm_f32_epilogue(M, N, K):
    A, B = rnd(M, K, seed=1), rnd(N, K, seed=2)
    bias = torch.randn(N, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    C = wx.wx_gemm_bf16(A, B, 0, bias=bias, status=st)
    torch.cuda.synchronize()
    ref = A.float() @ B.float().T + bias
    err = (C - ref).abs().max().item() / ref.abs().max().item()
    assert int(st.item()) == 0
    assert err < 1e-5, err


def gelu(z):
    return 0.5 * z * (1 + torch.erf(z / np.sqrt(2)))


def test_gemm_gelu_and_dgelu_epilogues():
    M, N, K = 256, 512, 256
    A, B = rnd(M, K, scale=0.1, seed=3), rnd(N, K, scale=0.1, seed=4)
    bias = torch.randn(N, device="cuda") * 0.1
    H = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    Z = torch.empty_like(H)
    wx.wx_gemm_bf16(A, B, 1, bias=bias, out=H, out2=Z)
    z = A.float() @ B.float().T + bias
    assert (Z.float() - z).abs().max().item() <= 1e-2 * z.abs().max().item()
    assert (H.float() - gelu(z)).abs().max().item() <= 1e-2 * gelu(z).abs().max().item()
    # backward epilogue: (dY . W) * GELU'(Z)
    dY, W = rnd(M, K, scale=0.1, seed=5), rnd(N, K, scale=0.1, seed=6)
    D = wx.wx_gemm_bf16(dY, W, 2, aux=Z, out=torch.empty(M, N, dtype=torch.bfloat16, device="cuda"))
    zz = Z.float().requires_grad_(True)
    gelu(zz).backward(torch.ones_like(zz))
    ref = (dY.float() @ W.float().T) * zz.grad
    torch.cuda.synchronize()
    assert (D.float() - ref).abs().max().item() <= 2e-2 * ref.abs().max().item()


def test_gemm_rejects_bad_shapes():
    A, B = rnd(100, 64), rnd(128, 64)
    with pytest.raises(wx.WxError):
        wx.wx_gemm_bf16(A, B, 0)
