"""Multiply-add work of one U-Net forward pass (2 FLOPs per multiply-add), by layer."""
from __future__ import annotations

from .inputs import UNET_IN


def layer_flops(h: int, w: int) -> list[tuple[str, float]]:
    """(layer, FLOPs) of one sample on an h x w input: 3x3 convolutions of the encoder and decoder
    blocks, the stride-2 transposed convolutions, and the output convolution."""
    out = []
    enc = [(UNET_IN, 32), (32, 64), (64, 128), (128, 256)]
    for lvl, (ci, co) in enumerate(enc):
        out.append((f"enc{lvl + 1}", 2.0 * 9 * ci * co * (h >> lvl) * (w >> lvl)))
    dec = [("dec4", 256, 256, 3), ("dec3", 256, 128, 2), ("dec2", 128, 64, 1), ("dec1", 64, 32, 0)]
    for name, ci, co, lvl in dec:
        out.append((name, 2.0 * 9 * ci * co * (h >> lvl) * (w >> lvl)))
    ups = [("up4", 256, 128, 3), ("up3", 128, 64, 2), ("up2", 64, 32, 1)]
    for name, ci, co, lvl in ups:
        out.append((name, 2.0 * ci * co * 4 * (h >> lvl) * (w >> lvl)))
    out.append(("out", 2.0 * 9 * 32 * 3 * h * w))
    return out


def flops_per_sample(h: int, w: int) -> float:
    return sum(f for _, f in layer_flops(h, w))


def tensor_core_flops_per_sample(h: int, w: int) -> float:
    """The part that runs on the tensor cores (all but the first and the output convolutions)."""
    return sum(f for n, f in layer_flops(h, w) if n not in ("enc1", "out"))
