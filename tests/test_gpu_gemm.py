"""The network's BF16 tensor-core GEMMs through the C ABI (rt_gemm_bf16):
the TMA-fed warp-specialised kernel and the register-staged one against an
FP64 product of the same BF16 values, on ragged and full-size shapes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mlp as OM  # noqa: E402
from paper_1811_05784_gb300 import rt  # noqa: E402


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (300, 200, 96), (1000, 1568, 512), (65, 33, 8), (4096, 512, 960),
                                   (512, 960, 4096), (1000, 1002, 1000), (130, 2000, 72)])
@pytest.mark.parametrize("kernel,split", [(rt.RT_GEMM_TMA, False), (rt.RT_GEMM_TMA, True), (rt.RT_GEMM_STAGED, False)])
def test_gemm_matches_fp64(M, N, K, kernel, split):
    """Ragged M, N and K (zero-filled tile edges), tile widths that do not
    divide 32, N not a multiple of 4 (scalar stores), several K steps and
    tiles, with and without the cut along K: |C - A B^T| <= max(K, 16) 2^-24
    sum |a b| per element, the bound of an FP32 sum of K exact BF16
    products."""
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    ws = torch.empty(16 * M * N, dtype=torch.float32, device="cuda") if split else None
    C = rt.rt_gemm_bf16(A.cuda(), B.cuda(), kernel=kernel, workspace=ws).cpu().numpy().astype(np.float64)
    a, b = A.float().numpy().astype(np.float64), B.float().numpy().astype(np.float64)
    ref = a @ b.T
    scale = np.abs(a) @ np.abs(b).T
    tol = max(K, 16) * 2.0 ** -24
    assert np.all(np.abs(C - ref) <= tol * scale + 1e-30), np.max(np.abs(C - ref) / (scale + 1e-30))


def test_both_kernels_agree_on_the_network_shapes():
    """The surrogate network's forward products at batch 1024 (960 -> 512 ->
    512 -> 1568): the two kernels give the same FP32 sums within rounding."""
    g = torch.Generator(device="cpu").manual_seed(5)
    for K, N in ((960, 512), (512, 512), (512, 1568)):
        A = torch.randn(1024, K, generator=g).to(torch.bfloat16).cuda()
        B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
        c1 = rt.rt_gemm_bf16(A, B, kernel=rt.RT_GEMM_TMA)
        c2 = rt.rt_gemm_bf16(A, B, kernel=rt.RT_GEMM_STAGED)
        scale = (A.float().abs() @ B.float().abs().T)
        assert torch.all((c1 - c2).abs() <= 2 * K * 2.0 ** -24 * scale)
    assert OM.to_bf16(np.array([1.0]))[0] == 1.0


def test_split_products_are_deterministic_and_timed():
    """A weight-gradient shape (M = 512, N = 960, K = 65,536: 16 tiles, cut
    into K ranges): two calls give the same bits, the uncut product agrees
    within the FP32 summation bound, and the reported kernel time is
    positive."""
    g = torch.Generator(device="cuda").manual_seed(11)
    A = torch.randn(512, 65536, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(960, 65536, device="cuda", generator=g).to(torch.bfloat16)
    ws = torch.empty(16 * 512 * 960, dtype=torch.float32, device="cuda")
    c1, ms1 = rt.rt_gemm_bf16(A, B, workspace=ws, timed=True)
    c2, ms2 = rt.rt_gemm_bf16(A, B, workspace=ws, timed=True)
    c3 = rt.rt_gemm_bf16(A, B)
    assert torch.equal(c1, c2) and ms1 > 0 and ms2 > 0
    scale = A.float().abs() @ B.float().abs().T
    assert torch.all((c1 - c3).abs() <= 2 * 65536 * 2.0 ** -24 * scale)


def test_gemm_arguments_are_checked():
    A = torch.zeros((4, 8), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(rt.RtError):
        rt.rt_gemm_bf16(A, A, kernel=5)
    with pytest.raises(rt.RtError):
        rt.rt_gemm_bf16(A[:, :6].contiguous(), A[:, :6].contiguous())
