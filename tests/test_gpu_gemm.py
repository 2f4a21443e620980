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


@pytest.mark.parametrize("nb,H,W,Cin,Cout", [(2, 6, 10, 24, 8), (1, 12, 20, 8, 40), (3, 5, 8, 16, 16)])
def test_conv_and_weight_gradient_ragged_sizes(nb, H, W, Cin, Cout):
    """The implicit-GEMM convolution and weight gradient (gathered A operands) on
    sizes that leave partial row tiles, partial column tiles and a partial last
    K slice (P = nb H W not a multiple of 64, 9 Cin not of 128), against the
    FP64 oracle convolution on the same BF16 values."""
    from oracle import unet as ounet
    rs = np.random.default_rng(nb * 1000 + H * 10 + Cin)
    P = nb * H * W
    x, xb = bf16_round(rs.normal(size=(nb, H, W, Cin)).astype(np.float32))
    w, wb = bf16_round(rs.normal(size=(Cout, 9, Cin)).astype(np.float32) * 0.2)
    dz, dzb = bf16_round(rs.normal(size=(nb, H, W, Cout)).astype(np.float32))
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    X = to_dev_bf16(xb.reshape(-1))
    Wt = to_dev_bf16(wb.reshape(-1))
    Y = torch.zeros(P * Cout, dtype=torch.float32, device="cuda")
    _abi.prior_call("gevo_conv3x3", nb, H, W, Cin, X, Cout, Wt, None, Y, Cout, 0, 0, 0.0, ws)
    dZt = to_dev_bf16(np.ascontiguousarray(dzb.reshape(P, Cout).T).reshape(-1))
    dW = torch.zeros(Cout * 9 * Cin, dtype=torch.float32, device="cuda")
    _abi.prior_call("gevo_conv3x3_wgrad", nb, H, W, Cin, X, Cout, dZt, dW, ws)
    torch.cuda.synchronize()
    assert _abi.gevo_last_error(ws) == 0
    x64, w64, dz64 = (a.astype(np.float64) for a in (x, w, dz))
    ref = ounet.conv3x3(x64, w64, np.zeros(Cout))
    mag = ounet.conv3x3(np.abs(x64), np.abs(w64), np.zeros(Cout))
    got = Y.cpu().numpy().reshape(nb, H, W, Cout)
    assert (np.abs(got - ref) <= 2e-6 * mag + 1e-30).all()
    _, dw_ref, _ = ounet.conv3x3_bwd(x64, w64, dz64)
    _, dw_mag, _ = ounet.conv3x3_bwd(np.abs(x64), w64, np.abs(dz64))
    got_dw = dW.cpu().numpy().reshape(Cout, 9, Cin)
    assert (np.abs(got_dw - dw_ref) <= 2e-6 * np.abs(dw_mag) + 1e-30).all()
