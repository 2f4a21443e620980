"""Learned depth prior: a small U-Net trained on (RGB, depth) pairs rendered
from the map, proposing depths for the Gaussians of newly observed regions.

GEVO initialises those Gaussians from a photometric cost volume (Eq. 1) with
belief propagation and SPGF* (Section III-A); the prior replaces the depth
proposal with one network evaluation and is judged against that plain
initialisation after the same optimisation.

Architecture (levels l = 0..L-1, channels c_l, default 16/32/64/128): per level
two 3x3 conv + ReLU; 2x2 max pool between encoder levels; x2 nearest upsample,
concatenation with the encoder's skip, two 3x3 conv + ReLU per decoder level;
1x1 head to log-depth.  BF16 weights and activations, FP32 accumulation (in
tensor memory), FP32 master weights with Adam.  Every step runs in libgevo's
kernels (include/gevo_prior.h); torch only holds the buffers.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi

BF16 = torch.bfloat16


def _ptr(t: torch.Tensor, offset_elems: int = 0):
    return ctypes.c_void_p(t.data_ptr() + offset_elems * t.element_size())


class DepthUNet:
    def __init__(self, nb: int, H: int, W: int, chans=(16, 32, 64, 128), device="cuda",
                 seed: int = 0):
        L = len(chans)
        assert H % (1 << (L - 1)) == 0 and W % (1 << (L - 1)) == 0
        assert all(c % 8 == 0 for c in chans) and chans[0] <= 16
        self.nb, self.H, self.W, self.L, self.chans = nb, H, W, L, tuple(chans)
        self.dev = torch.device(device)
        self.hw = [(H >> i, W >> i) for i in range(L)]
        self.P = [nb * h * w for h, w in self.hw]
        self.ccat = [chans[i + 1] + chans[i] for i in range(L - 1)]
        rs = np.random.default_rng(seed)
        self.layers = {}
        for i in range(L):
            self._layer(f"enc{i}a", 8 if i == 0 else chans[i - 1], chans[i], rs, 3 if i == 0 else None)
            self._layer(f"enc{i}b", chans[i], chans[i], rs)
        for i in range(L - 2, -1, -1):
            self._layer(f"dec{i}a", self.ccat[i], chans[i], rs)
            self._layer(f"dec{i}b", chans[i], chans[i], rs)
        f32 = torch.float32
        d = self.dev
        self.head_w = torch.from_numpy((rs.normal(size=chans[0]) * np.sqrt(1.0 / chans[0]))
                                       .astype(np.float32)).to(d)
        self.head_b = torch.full((1,), 1.0, dtype=f32, device=d)   # log(2.7 m): room-scale start
        self.head_state = [torch.zeros_like(self.head_w) for _ in range(3)] + \
            [torch.zeros_like(self.head_b) for _ in range(3)]       # dw, m, v, db, m, v
        # activations
        z16 = lambda p, c: torch.zeros(p, c, dtype=BF16, device=d)
        z32 = lambda p, c: torch.zeros(p, c, dtype=f32, device=d)
        self.X0 = z16(self.P[0], 8)
        self.A = [z16(self.P[i], chans[i]) for i in range(L)]
        self.CAT = [z16(self.P[i], self.ccat[i]) for i in range(L - 1)]
        self.BOT = z16(self.P[L - 1], chans[L - 1])
        self.POOL = [None] + [z16(self.P[i], chans[i - 1]) for i in range(1, L)]
        self.DA = [z16(self.P[i], chans[i]) for i in range(L - 1)]
        self.DB = [z16(self.P[i], chans[i]) for i in range(L - 1)]
        self.pred = torch.zeros(self.P[0], dtype=f32, device=d)
        self.dpred = torch.zeros_like(self.pred)
        self.loss = torch.zeros(1, dtype=f32, device=d)
        # gradients of activations (FP32)
        self.dDB = [z32(self.P[i], chans[i]) for i in range(L - 1)]
        self.dDA = [z32(self.P[i], chans[i]) for i in range(L - 1)]
        self.dCAT = [z32(self.P[i], self.ccat[i]) for i in range(L - 1)]
        self.dBOT = z32(self.P[L - 1], chans[L - 1])
        self.dA = [z32(self.P[i], chans[i]) for i in range(L)]
        self.dPOOL = [None] + [z32(self.P[i], chans[i - 1]) for i in range(1, L)]
        zmax = max(self.P[i] * chans[i] for i in range(L))
        self.dZ = torch.zeros(zmax, dtype=BF16, device=d)
        self.dZt = torch.zeros(zmax, dtype=BF16, device=d)
        self.ws = torch.zeros(256, dtype=torch.uint8, device=d)
        self.step_count = 0

    # ---- parameters ----------------------------------------------------------------
    def _layer(self, name, cin, cout, rs, cin_real=None):
        fan_in = 9 * (cin_real if cin_real is not None else cin)
        w = (rs.normal(size=(cout, 9, cin)) * np.sqrt(2.0 / fan_in)).astype(np.float32)
        if cin_real is not None:
            w[:, :, cin_real:] = 0.0
        d = self.dev
        W32 = torch.from_numpy(w.reshape(cout, 9 * cin)).to(d)
        lay = dict(cin=cin, cout=cout, W32=W32, b32=torch.zeros(cout, device=d),
                   W16=torch.zeros(cout, 9 * cin, dtype=BF16, device=d),
                   Wf16=torch.zeros(cin, 9 * cout, dtype=BF16, device=d),
                   dW=torch.zeros_like(W32), db=torch.zeros(cout, device=d),
                   mW=torch.zeros_like(W32), vW=torch.zeros_like(W32),
                   mb=torch.zeros(cout, device=d), vb=torch.zeros(cout, device=d))
        self.layers[name] = lay
        _abi.prior_call("gevo_to_bf16", W32.numel(), W32, lay["W16"])
        _abi.prior_call("gevo_flip3x3", cout, cin, lay["W16"], lay["Wf16"])

    def parameters_numpy(self):
        """FP32 masters (for the oracle comparison)."""
        out = {k: (v["W32"].cpu().numpy().reshape(v["cout"], 9, v["cin"]), v["b32"].cpu().numpy())
               for k, v in self.layers.items()}
        out["head"] = (self.head_w.cpu().numpy(), self.head_b.cpu().numpy())
        return out

    # ---- forward -------------------------------------------------------------------
    def _conv(self, name, nb, h, w, X, Y, ldy, y_off=0, relu=True):
        lay = self.layers[name]
        _abi.prior_call("gevo_conv3x3", nb, h, w, lay["cin"], X, lay["cout"], lay["W16"],
                        lay["b32"], _ptr(Y, y_off), ldy, 1, int(relu), 0.0, self.ws)

    def forward(self, rgb_planar: torch.Tensor):
        """rgb_planar: FP32 [nb, 3, H, W] (contiguous).  Returns pred (log-depth, [nb*H*W])."""
        nb, L, c = self.nb, self.L, self.chans
        _abi.prior_call("gevo_rgb_pack", nb, self.H, self.W, rgb_planar, self.X0)
        for i in range(L):
            h, w = self.hw[i]
            Xin = self.X0 if i == 0 else self.POOL[i]
            self._conv(f"enc{i}a", nb, h, w, Xin, self.A[i], c[i])
            if i < L - 1:
                self._conv(f"enc{i}b", nb, h, w, self.A[i], self.CAT[i], self.ccat[i], c[i + 1])
                _abi.prior_call("gevo_maxpool2", nb, h, w, c[i], _ptr(self.CAT[i], c[i + 1]),
                                self.ccat[i], self.POOL[i + 1])
            else:
                self._conv(f"enc{i}b", nb, h, w, self.A[i], self.BOT, c[i])
        up = self.BOT
        for i in range(L - 2, -1, -1):
            h, w = self.hw[i]
            _abi.prior_call("gevo_upsample2", nb, h // 2, w // 2, c[i + 1], up, self.CAT[i],
                            self.ccat[i])
            self._conv(f"dec{i}a", nb, h, w, self.CAT[i], self.DA[i], c[i])
            self._conv(f"dec{i}b", nb, h, w, self.DA[i], self.DB[i], c[i])
            up = self.DB[i]
        last = self.DB[0] if L > 1 else self.BOT
        _abi.prior_call("gevo_head_fwd", self.P[0], c[0], last, self.head_w, self.head_b, self.pred)
        return self.pred

    # ---- backward ------------------------------------------------------------------
    def _layer_bwd(self, name, nb, h, w, Xin, dY, lddy, Y, ldy, dX, lddx, y_off=0, dy_off=0,
                   need_dx=True):
        lay = self.layers[name]
        P = nb * h * w
        cin, cout = lay["cin"], lay["cout"]
        _abi.prior_call("gevo_relu_bwd", P, cout, _ptr(dY, dy_off), lddy, _ptr(Y, y_off), ldy,
                        self.dZ, self.dZt, lay["db"])
        _abi.prior_call("gevo_conv3x3_wgrad", nb, h, w, cin, Xin, cout, self.dZt, lay["dW"],
                        self.ws)
        if need_dx:
            _abi.prior_call("gevo_conv3x3", nb, h, w, cout, self.dZ, cin, lay["Wf16"], None,
                            dX, lddx, 0, 0, 0.0, self.ws)

    def backward(self):
        """Gradients of self.loss (after depth_loss) w.r.t. every parameter."""
        nb, L, c = self.nb, self.L, self.chans
        for lay in self.layers.values():
            lay["db"].zero_()
        last = self.DB[0] if L > 1 else self.BOT
        dlast = self.dDB[0] if L > 1 else self.dBOT
        dw, _, _, db, _, _ = self.head_state
        _abi.prior_call("gevo_head_bwd", self.P[0], c[0], last, self.head_w, self.dpred, dlast,
                        dw, db)
        for i in range(L - 1):
            h, w = self.hw[i]
            self._layer_bwd(f"dec{i}b", nb, h, w, self.DA[i], self.dDB[i], c[i], self.DB[i], c[i],
                            self.dDA[i], c[i])
            self._layer_bwd(f"dec{i}a", nb, h, w, self.CAT[i], self.dDA[i], c[i], self.DA[i], c[i],
                            self.dCAT[i], self.ccat[i])
            dst = self.dBOT if i + 1 == L - 1 else self.dDB[i + 1]
            _abi.prior_call("gevo_upsample2_bwd", nb, h // 2, w // 2, c[i + 1], self.dCAT[i],
                            self.ccat[i], dst)
        i = L - 1
        h, w = self.hw[i]
        self._layer_bwd(f"enc{i}b", nb, h, w, self.A[i], self.dBOT, c[i], self.BOT, c[i],
                        self.dA[i], c[i])
        Xin = self.X0 if i == 0 else self.POOL[i]
        self._layer_bwd(f"enc{i}a", nb, h, w, Xin, self.dA[i], c[i], self.A[i], c[i],
                        self.dPOOL[i] if i > 0 else None, c[i - 1] if i > 0 else 8, need_dx=i > 0)
        for i in range(L - 2, -1, -1):
            h, w = self.hw[i]
            off = c[i + 1]
            _abi.prior_call("gevo_maxpool2_bwd", nb, h, w, c[i], _ptr(self.CAT[i], off),
                            self.ccat[i], self.dPOOL[i + 1], _ptr(self.dCAT[i], off),
                            self.ccat[i], 1.0)
            self._layer_bwd(f"enc{i}b", nb, h, w, self.A[i], self.dCAT[i], self.ccat[i], self.CAT[i],
                            self.ccat[i], self.dA[i], c[i], y_off=off, dy_off=off)
            Xin = self.X0 if i == 0 else self.POOL[i]
            self._layer_bwd(f"enc{i}a", nb, h, w, Xin, self.dA[i], c[i], self.A[i], c[i],
                            self.dPOOL[i] if i > 0 else None, c[i - 1] if i > 0 else 8,
                            need_dx=i > 0)

    def depth_loss(self, target: torch.Tensor, weight: torch.Tensor):
        _abi.prior_call("gevo_depth_l1", self.P[0], self.pred, target, weight, self.loss, self.dpred)
        return self.loss

    def adam_step(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step_count += 1
        t = self.step_count
        for lay in self.layers.values():
            _abi.prior_call("gevo_adam", lay["W32"].numel(), lay["W32"], lay["dW"], lay["mW"],
                            lay["vW"], lay["W16"], lr, b1, b2, eps, t)
            _abi.prior_call("gevo_adam", lay["b32"].numel(), lay["b32"], lay["db"], lay["mb"],
                            lay["vb"], None, lr, b1, b2, eps, t)
            _abi.prior_call("gevo_flip3x3", lay["cout"], lay["cin"], lay["W16"], lay["Wf16"])
        dw, mw, vw, db, mb, vb = self.head_state
        _abi.prior_call("gevo_adam", self.head_w.numel(), self.head_w, dw, mw, vw, None, lr, b1, b2,
                        eps, t)
        _abi.prior_call("gevo_adam", 1, self.head_b, db, mb, vb, None, lr, b1, b2, eps, t)

    def train_step(self, rgb_planar, target, weight, lr=1e-3):
        self.forward(rgb_planar)
        self.depth_loss(target, weight)
        self.backward()
        self.adam_step(lr)
        return self.loss
