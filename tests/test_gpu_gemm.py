"""The tcgen05 BF16 GEMM against a float64 product of the same BF16 operands:
ragged M, small and large N (every tile width), long K, split-K, bias, ReLU
and the BF16 copy of the result."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_02779_b300.rimg as R
    return R


def _ref(A, B):
    return A.float().cpu().numpy().astype(np.float64) @ B.float().cpu().numpy().astype(np.float64).T


@pytest.mark.parametrize("M,N,K", [(128, 32, 64), (300, 6, 128), (1000, 64, 576), (257, 128, 1152),
                                   (64, 256, 64), (5, 200, 192), (4096, 48, 64)])
def test_gemm_matches_float64(R, M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    C = torch.full((M, N), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    R.rimg_gemm_bf16(A, B, C, err=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    ref = _ref(A, B)
    # FP32 accumulation of K products of BF16 values: |error| <= K u sum|a b|
    bound = K * 2.0 ** -23 * (np.abs(A.float().cpu().numpy()) @ np.abs(B.float().cpu().numpy()).T) + 1e-6
    assert np.all(np.abs(C.cpu().numpy() - ref) <= bound)


def test_gemm_bias_relu_bf16_copy(R):
    M, N, K = 333, 96, 256
    A = torch.randn(M, K, device="cuda").to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda").to(torch.bfloat16)
    bias = torch.randn(N, device="cuda")
    C = torch.zeros(M, N, device="cuda")
    Cb = torch.zeros(M, N, device="cuda", dtype=torch.bfloat16)
    R.rimg_gemm_bf16(A, B, C, C_bf16=Cb, bias=bias, relu=True)
    torch.cuda.synchronize()
    ref = np.maximum(_ref(A, B) + bias.cpu().numpy()[None, :], 0.0)
    np.testing.assert_allclose(C.cpu().numpy(), ref, rtol=1e-4, atol=1e-3)
    assert torch.equal(Cb, C.to(torch.bfloat16))


def test_gemm_split_k(R):
    M, N, K, S = 200, 64, 1024, 4
    A = torch.randn(M, K, device="cuda").to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda").to(torch.bfloat16)
    C = torch.zeros(S, M, N, device="cuda")
    R.rimg_gemm_bf16(A, B, C, splits=S)
    torch.cuda.synchronize()
    np.testing.assert_allclose(C.sum(0).cpu().numpy(), _ref(A, B), rtol=1e-4, atol=1e-3)
    # each split is the product over its own quarter of K
    q = K // S
    np.testing.assert_allclose(C[1].cpu().numpy(), _ref(A[:, q:2 * q], B[:, q:2 * q]), rtol=1e-4, atol=1e-3)
