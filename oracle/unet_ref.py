"""Reference forward pass of the U-Net with temporal conditioning (FP64, CPU, PyTorch ops).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only tests, the smoke
check and the benchmark's CPU baseline may import it.

What it computes ("U-Net with temporal conditioning", Methods; readings where
the paper is silent are marked READING):

  f(dt)      = w2 sin(w1 sin(w0 dt + b0) + b1) + b2          (MLP, 2 hidden layers of 128, sin activation)
  conv(u)    = cross-correlation with a 3x3 kernel, zero 'same' padding, no bias
               (READING: kernel size 3x3 and zero padding; GroupNorm follows, so a bias would cancel)
  GN(u)      = per-sample group normalisation with affine gamma/beta, eps 1e-5 (READING: 8 groups)
  GELU(u)    = 0.5 u (1 + tanh(sqrt(2/pi)(u + 0.044715 u^3)))  (the paper's tanh form)
  block(u)   = GELU(GN(conv(u)))
  down       = 2x2 max pooling, stride 2
  up         = transposed convolution, 2x2 kernel, stride 2, channel-mixing, no bias
               (READING: the printed up-sampling formula omits the channel sums)

  encoder    z1 = block(x), zp = block(down(z_{p-1})), p = 2, 3, 4       (unconditioned chain)
  condition  zc_p = z_p * (W_p f(dt))  (per-channel product, p = 1..4)
  decoder    d3 = up(block(zc4)); d2 = up(block(zc3 ++ d3)); d1 = up(block(zc2 ++ d2))
  output     y  = x_fields + gamma * conv(block(zc1 ++ d1)) + beta
             (READING: the paper writes GN(conv(...)) for its single normalised composition field; here
             the network predicts two fields whose per-sample mean and spread vary with the film's
             thickness and the incident composition, which a final normalisation would pin, so the
             last convolution instead gives a per-channel affine increment added to the input fields)

Channels 32-64-128-256.  Input x = lb = 3 look-back frames of the state (phi, c, rho),
oldest first, then a plane holding the jump length dt / dt_ref; output y = the newest
frame plus the predicted increments of (phi, c, rho).  The paper's operator reads lb
consecutive frames [c(t - lb + 1), ..., c(t)] of its single field and its look-back
study finds lb = 1 markedly worse (the process is non-Markovian in that field).
READING: here the state is the three coupled fields, so every frame carries all three
(9 planes), and the vapor density is predicted too (resetting it instead costs 12.6 %
relative L2 in phi after 25 exact jumps).  The frames are 1000 steps apart and the
jump is 2000 steps: the two older frames are the start and the middle of the DNS
stretch that precedes a jump.

Weights come from ``paper_2312_05410_gb300.inputs.unet_weights`` (seeded numbers,
no arithmetic of the method).

Precision model of the GPU path that this mirrors: the first convolution reads the
FP32 fields and frames with FP32 weights (the composition fluctuations that seed the
spinodal pattern are about 0.01 on c ~ 0.5, a few BF16 units, so BF16 inputs would
quantize them away); every other weight and every stored activation is BF16 (round to
nearest even); products are exact and sums are kept in high precision (FP64 here, FP32
on the GPU); group statistics are taken from the unrounded convolution outputs; GN +
GELU are evaluated in high precision on the rounded stored values.  ``bf16`` below is
written from the format definition (1 sign, 8 exponent, 7 fraction bits), not taken
from a library.
"""
from __future__ import annotations

import math

import numpy as np
import torch
import torch.nn.functional as F

DT = torch.float64
CH = (32, 64, 128, 256)
GROUPS = 8
EPS = 1e-5
FDIM = 128       # width of the MLP's hidden layers and of the basis f(dt)
LB = 3                   # look-back frames
IN_CH, OUT_CH = 3 * LB + 1, 3


def bf16(a) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64.

    The FP32 value's 16 low bits are dropped after adding 0x7FFF plus the
    lowest kept bit (round half to even on the discarded half-word)."""
    x = np.array(a, dtype=np.float32, copy=True)
    shape = x.shape
    x = x.reshape(-1)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[np.isnan(x)] = np.nan
    return out.reshape(shape)


def _t(a) -> torch.Tensor:
    return torch.as_tensor(np.asarray(a, dtype=np.float64), dtype=DT)


def _rb(t: torch.Tensor) -> torch.Tensor:
    return _t(bf16(t.numpy()))


def basis(W: dict, tau: float) -> np.ndarray:
    """f(dt) of the MLP with sin activations, in FP64 (tau = dt / dt_ref)."""
    h = np.sin(W["mlp_w0"].astype(np.float64)[:, 0] * tau + W["mlp_b0"])
    h = np.sin(W["mlp_w1"].astype(np.float64) @ h + W["mlp_b1"])
    return W["mlp_w2"].astype(np.float64) @ h + W["mlp_b2"]


def scales(W: dict, tau: float) -> list[np.ndarray]:
    """Per-channel conditioning factors W_p f(dt) of the four levels, in FP64."""
    f = basis(W, tau)
    return [W[f"proj{p}"].astype(np.float64) @ f for p in range(1, 5)]


def conv3x3(x: torch.Tensor, w, weights_bf16: bool = True) -> torch.Tensor:
    """Zero-padded 'same' 3x3 cross-correlation of NCHW x with w [Cout, Cin, 3, 3] (BF16 weights, or the
    FP32 weights as given)."""
    wt = bf16(w) if weights_bf16 else np.asarray(w, dtype=np.float32).astype(np.float64)
    return F.conv2d(x, _t(wt), padding=1)


def group_stats(y: torch.Tensor, groups: int):
    n, c, h, w = y.shape
    v = y.reshape(n, groups, (c // groups) * h * w)
    mean = v.mean(dim=2)
    var = ((v - mean[:, :, None]) ** 2).mean(dim=2)
    return mean, var


def group_norm(y_store: torch.Tensor, mean, var, gamma, beta, groups: int) -> torch.Tensor:
    n, c, h, w = y_store.shape
    cg = c // groups
    m = mean.repeat_interleave(cg, dim=1)[:, :, None, None]
    r = (1.0 / torch.sqrt(var + EPS)).repeat_interleave(cg, dim=1)[:, :, None, None]
    return (y_store - m) * r * _t(gamma)[None, :, None, None] + _t(beta)[None, :, None, None]


def gelu(u: torch.Tensor) -> torch.Tensor:
    return 0.5 * u * (1.0 + torch.tanh(math.sqrt(2.0 / math.pi) * (u + 0.044715 * u ** 3)))


def block(x: torch.Tensor, W: dict, name: str, groups: int = GROUPS, act: bool = True,
          weights_bf16: bool = True) -> torch.Tensor:
    """conv -> (stats of the unrounded output) -> BF16 store -> GN -> GELU -> BF16 store."""
    y = conv3x3(x, W[name], weights_bf16)
    mean, var = group_stats(y, groups)
    y = group_norm(_rb(y), mean, var, W[name + "_gamma"], W[name + "_beta"], groups)
    return _rb(gelu(y)) if act else y


def down(x: torch.Tensor) -> torch.Tensor:
    return F.max_pool2d(x, 2, 2)


def up(x: torch.Tensor, w) -> torch.Tensor:
    return _rb(F.conv_transpose2d(x, _t(bf16(w)), stride=2))


def forward(W: dict, x, tau: float, taps: dict | None = None) -> np.ndarray:
    """Network output for x [N, 10, H, W] (3 frames of phi, c, rho, oldest first, then the dt plane;
    rounded to FP32 here); returns [N, 3, H, W] FP64: the newest frame plus the increments.
    If `taps` is a dict it receives the intermediate tensors by name."""
    newest = 3 * (LB - 1)
    x_fields = _t(np.asarray(x, dtype=np.float32)[:, newest:newest + OUT_CH])  # the residual adds the newest frame
    x = _t(np.asarray(x, dtype=np.float32))        # the first convolution reads the FP32 fields
    s = [_t(bf16(v)) for v in scales(W, tau)]     # conditioning factors are stored as BF16
    z1 = block(x, W, "enc1", weights_bf16=False)
    z2 = block(down(z1), W, "enc2")
    z3 = block(down(z2), W, "enc3")
    z4 = block(down(z3), W, "enc4")
    zc = [_rb(z * sp[None, :, None, None]) for z, sp in zip((z1, z2, z3, z4), s)]
    d3 = up(block(zc[3], W, "dec4"), W["up4"])
    d2 = up(block(torch.cat([zc[2], d3], 1), W, "dec3"), W["up3"])
    d1 = up(block(torch.cat([zc[1], d2], 1), W, "dec2"), W["up2"])
    h1 = block(torch.cat([zc[0], d1], 1), W, "dec1")
    inc = conv3x3(h1, W["out"])
    y = x_fields + inc * _t(W["out_gamma"])[None, :, None, None] + _t(W["out_beta"])[None, :, None, None]
    if taps is not None:
        taps.update(z1=z1, z2=z2, z3=z3, z4=z4, zc1=zc[0], zc2=zc[1], zc3=zc[2], zc4=zc[3], d3=d3, d2=d2,
                    d1=d1, h1=h1, inc=inc, y=y)
    return y.numpy()


def flops_per_sample(h: int, w: int) -> float:
    """Multiply-add FLOPs (2 per MAC) of one forward pass on an h x w input."""
    tot = 0.0
    cin = IN_CH
    for p, c in enumerate(CH):
        tot += 2 * 9 * cin * c * (h >> p) * (w >> p)
        cin = c
    for cin, cout, p in ((256, 256, 3), (256, 128, 2), (128, 64, 1), (64, 32, 0)):
        tot += 2 * 9 * cin * cout * (h >> p) * (w >> p)
    for cin, cout, p in ((256, 128, 3), (128, 64, 2), (64, 32, 1)):
        tot += 2 * cin * cout * 4 * (h >> p) * (w >> p)
    tot += 2 * 9 * 32 * OUT_CH * h * w
    return tot
