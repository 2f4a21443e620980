"""The BF16 tensor-core U-Net (learned depth prior) against the FP64 oracle on
the same BF16 weights and inputs, the oracle storing activations and masked
gradients in BF16 at the same points (each layer computed in double).  What
remains is binary32 accumulation (K * 2^-24) and the rare BF16 rounding that
binary32 and double decide differently (one BF16 ulp, 2^-8), which then
propagates down the backward chain (up to 14 layers to the first one).
A rounding decides differently where the binary32 accumulation error, about
K 2^-24 ~ 7e-5 relative at K = 1152, straddles a BF16 rounding boundary: for
a fraction of about 7e-5 / 2^-8 ~ 2% of a layer's activations, each then off
by one BF16 ulp; over 14 layers that is a relative L2 error of about
2^-8 sqrt(14 x 0.02) ~ 2e-3 to be expected.  Bound: forward within twice that, 4e-3.
Gradients: how much BF16 storage moves a weight gradient depends on how much
its sum cancels (the first layer's, over centred inputs of both signs, moves
by about 17% between storing and not storing activations in BF16, the last
layers' by under 1%).  The two sides store at the same points and differ only
in the ~2% of roundings decided differently, so each gradient tensor must lie
within half of the oracle's own storage effect on it (the relative L2 error
and 1 - cosine between the oracle storing and not storing in BF16), plus 5e-3
relative L2 and 5e-4 in cosine."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import unet as ounet  # noqa: E402
from paper_2409_09295_gb300 import _abi  # noqa: E402
from paper_2409_09295_gb300.prior import DepthUNet  # noqa: E402


def _bf(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).bfloat16().float().numpy().astype(np.float64)


def _case(nb, H, W, chans, seed):
    net = DepthUNet(nb, H, W, chans, seed=seed)
    rs = np.random.default_rng(seed + 1)
    rgb = rs.uniform(size=(nb, 3, H, W)).astype(np.float32)
    target = rs.normal(1.0, 0.3, size=nb * H * W).astype(np.float32)
    weight = (rs.uniform(size=nb * H * W) > 0.1).astype(np.float32)
    # oracle parameters: the GPU's BF16 weights, FP32 biases / head
    params = {}
    for name, lay in net.layers.items():
        w = lay["W16"].float().cpu().numpy().astype(np.float64).reshape(lay["cout"], 9, lay["cin"])
        params[name] = (w, lay["b32"].cpu().numpy().astype(np.float64))
    params["head"] = (net.head_w.cpu().numpy().astype(np.float64), net.head_b.cpu().numpy().astype(np.float64))
    x = np.zeros((nb, H, W, 8))
    x[..., :3] = _bf(rgb.transpose(0, 2, 3, 1) - 0.5)   # the network input: centred RGB
    return net, rgb, target, weight, params, x


@pytest.mark.parametrize("nb,H,W,chans", [(2, 16, 16, (8, 16)), (2, 48, 64, (16, 32, 64, 128))])
def test_prior_forward_and_gradients_match_oracle(nb, H, W, chans):
    net, rgb, target, weight, params, x = _case(nb, H, W, chans, seed=11)
    t_rgb = torch.from_numpy(rgb).cuda()
    pred = net.forward(t_rgb).cpu().numpy().astype(np.float64)
    ref, cache = ounet.forward(params, x, chans, store_bf16=True)
    rel = np.linalg.norm(pred - ref) / np.linalg.norm(ref)
    assert rel <= 4e-3, rel
    # pixels whose prediction lies within 0.05 of the target could take the L1
    # sign either way on the two sides: weight 0 there on both sides (decided
    # from the oracle's prediction), then each side uses its own loss gradient
    weight = (weight * (np.abs(ref.reshape(-1) - target) > 0.05)).astype(np.float32)
    assert weight.mean() > 0.8
    net.depth_loss(torch.from_numpy(target).cuda(), torch.from_numpy(weight).cuda())
    net.backward()
    torch.cuda.synchronize()
    _, dpred = ounet.loss_l1(ref.reshape(-1), target.astype(np.float64), weight.astype(np.float64))
    np.testing.assert_array_equal(np.sign(net.dpred.cpu().numpy()), np.sign(dpred))
    g = ounet.backward(params, cache, dpred.reshape(ref.shape), chans, store_bf16=True)
    # the oracle's own storage effect: the same pass without BF16 storage
    _, cache_d = ounet.forward(params, x, chans, store_bf16=False)
    g_d = ounet.backward(params, cache_d, dpred.reshape(ref.shape), chans, store_bf16=False)

    def rel_cos(a, b):
        return (np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-300),
                a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300))
    for name, lay in net.layers.items():
        for i, (got, what) in enumerate(((lay["dW"].cpu().numpy(), "W"), (lay["db"].cpu().numpy(), "b"))):
            got = got.astype(np.float64).reshape(-1)
            want = g[name][i].reshape(-1)
            rel, cos = rel_cos(got, want)
            rel_s, cos_s = rel_cos(want, g_d[name][i].reshape(-1))
            assert rel <= 0.5 * rel_s + 5e-3, (name, what, rel, rel_s)
            assert 1 - cos <= 0.5 * (1 - cos_s) + 5e-4, (name, what, cos, cos_s)
    gw = net.head_state[0].cpu().numpy()
    assert np.dot(gw, g["head"][0]) / (np.linalg.norm(gw) * np.linalg.norm(g["head"][0])) >= 0.9995
    assert _abi.gevo_last_error(net.ws) == 0


def test_prior_training_reduces_loss():
    nb, H, W = 4, 32, 32
    net = DepthUNet(nb, H, W, (16, 32, 64), seed=3)
    rs = np.random.default_rng(5)
    # a learnable synthetic mapping: log-depth = 1 + brightness of the image
    rgb = rs.uniform(size=(nb, 3, H, W)).astype(np.float32)
    target = (1.0 + rgb.mean(axis=1)).reshape(-1).astype(np.float32)
    t_rgb = torch.from_numpy(rgb).cuda()
    t_tar = torch.from_numpy(target).cuda()
    t_w = torch.ones_like(t_tar)
    losses = [float(net.train_step(t_rgb, t_tar, t_w, lr=3e-3).item()) for _ in range(60)]
    assert losses[-1] < 0.5 * losses[0], losses[::10]
