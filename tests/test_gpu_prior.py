"""The BF16 tensor-core U-Net (learned depth prior) against the FP64 oracle on
the same BF16 weights and inputs, the oracle storing activations and masked
gradients in BF16 at the same points (each layer computed in double).  What
remains is binary32 accumulation (K * 2^-24) and the rare BF16 rounding that
binary32 and double decide differently (one BF16 ulp, 2^-8), which then
propagates down the backward chain (up to 14 layers to the first one):
forward within a relative L2 error of 2e-3, each gradient tensor within a
relative L2 error of 3e-2 and a cosine similarity of 0.9995."""
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
    x[..., :3] = _bf(rgb.transpose(0, 2, 3, 1))
    return net, rgb, target, weight, params, x


@pytest.mark.parametrize("nb,H,W,chans", [(2, 16, 16, (8, 16)), (2, 48, 64, (16, 32, 64, 128))])
def test_prior_forward_and_gradients_match_oracle(nb, H, W, chans):
    net, rgb, target, weight, params, x = _case(nb, H, W, chans, seed=11)
    t_rgb = torch.from_numpy(rgb).cuda()
    pred = net.forward(t_rgb).cpu().numpy().astype(np.float64)
    ref, cache = ounet.forward(params, x, chans, store_bf16=True)
    rel = np.linalg.norm(pred - ref) / np.linalg.norm(ref)
    assert rel <= 2e-3, rel
    net.depth_loss(torch.from_numpy(target).cuda(), torch.from_numpy(weight).cuda())
    net.backward()
    torch.cuda.synchronize()
    # the oracle's gradient through the GPU's own loss gradient (same sign pattern)
    dpred = net.dpred.cpu().numpy().astype(np.float64)
    g = ounet.backward(params, cache, dpred, chans, store_bf16=True)
    for name, lay in net.layers.items():
        for got, want, what in ((lay["dW"].cpu().numpy(), g[name][0], "W"),
                                (lay["db"].cpu().numpy(), g[name][1], "b")):
            got = got.astype(np.float64).reshape(-1)
            want = want.reshape(-1)
            cos = got @ want / (np.linalg.norm(got) * np.linalg.norm(want) + 1e-300)
            rel = np.linalg.norm(got - want) / (np.linalg.norm(want) + 1e-300)
            assert cos >= 0.9995 and rel <= 3e-2, (name, what, cos, rel)
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
