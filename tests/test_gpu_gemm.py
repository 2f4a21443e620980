"""The tcgen05 BF16 GEMM (the learned depth prior's contraction) against an
FP64 product of the same BF16 values.  FP32 accumulation over K terms is held to
|C - ref| <= 2e-6 * sum_k |a_k b_k| (K * 2^-24 with margin); BF16 outputs to one
BF16 rounding (2^-8 relative) on top."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2409_09295_gb300 import _abi, raster  # noqa: E402


def bf16_round(x):
    """Round float32 values to bfloat16 (nearest even); returns (values, bits)."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32)
    b = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    return (b.astype(np.uint32) << 16).view(np.float32), b


def to_dev_bf16(bits):
    return torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (1000, 48, 200), (300, 256, 1728),
                                   (77, 300, 96), (4096, 128, 576), (130, 32, 8)])
def test_gemm_bf16_fp32_out(M, N, K):
    rs = np.random.default_rng(M + N + K)
    a, abits = bf16_round(rs.normal(size=(M, K)).astype(np.float32))
    b, bbits = bf16_round(rs.normal(size=(N, K)).astype(np.float32))
    bias = rs.normal(size=N).astype(np.float32)
    ws = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    C = torch.zeros(M, N, dtype=torch.float32, device="cuda")
    tb = torch.from_numpy(bias).cuda()
    _abi.gevo_gemm_bf16(M, N, K, to_dev_bf16(abits), K, to_dev_bf16(bbits), K, C, N, False, tb,
                        False, 0.0, ws)
    torch.cuda.synchronize()
    assert _abi.gevo_last_error(ws) == 0
    ref = a.astype(np.float64) @ b.astype(np.float64).T + bias
    scale = np.abs(a).astype(np.float64) @ np.abs(b).astype(np.float64).T + np.abs(bias)
    err = np.abs(C.cpu().numpy() - ref)
    assert (err <= 2e-6 * scale + 1e-30).all(), (err / scale).max()


def test_gemm_bf16_relu_bf16_out_and_accumulate():
    M, N, K = 513, 64, 144
    rs = np.random.default_rng(7)
    a, abits = bf16_round(rs.normal(size=(M, K)).astype(np.float32))
    b, bbits = bf16_round(rs.normal(size=(N, K)).astype(np.float32))
    ws = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    C = torch.zeros(M, N, dtype=torch.bfloat16, device="cuda")
    _abi.gevo_gemm_bf16(M, N, K, to_dev_bf16(abits), K, to_dev_bf16(bbits), K, C, N, True, None,
                        True, 0.0, ws)
    ref = np.maximum(a.astype(np.float64) @ b.astype(np.float64).T, 0)
    got = C.float().cpu().numpy()
    scale = np.abs(a).astype(np.float64) @ np.abs(b).astype(np.float64).T
    assert (np.abs(got - ref) <= 2 ** -8 * np.abs(ref) + 2e-6 * scale + 1e-30).all()
    # accumulate: C = A B^T + 1.0 * C (FP32 output)
    C2 = torch.full((M, N), 0.5, dtype=torch.float32, device="cuda")
    _abi.gevo_gemm_bf16(M, N, K, to_dev_bf16(abits), K, to_dev_bf16(bbits), K, C2, N, False,
                        None, False, 1.0, ws)
    ref2 = a.astype(np.float64) @ b.astype(np.float64).T + 0.5
    assert (np.abs(C2.cpu().numpy() - ref2) <= 2e-6 * scale + 1e-6).all()
    assert _abi.gevo_last_error(ws) == 0
