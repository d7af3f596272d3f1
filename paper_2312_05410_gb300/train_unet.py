"""Train the time-conditioned U-Net on trajectories that the GPU DNS generates.

    python -m paper_2312_05410_gb300.train_unet --out weights.npz [--runs 200] [--budget 1800]

This is offline tooling, not the solver's path.
- **Data.** The batched ensemble kernel advances `runs` seeded films of 256 x 256 cells
  (another seed than the hybrid benchmark's runs).  A snapshot of (phi, c, rho) is kept
  every 1000 steps, 100 snapshots per run.
- **Samples.** The network's input is three look-back frames 1000 steps apart, oldest
  first (the paper's operator reads lb = 3 consecutive frames), and the jump length
  tau = 1 (2000 steps); the target is the state 2000 steps after the newest frame.  This
  is what the hybrid solver feeds it: the two older frames are the start and the middle
  of the DNS stretch before the jump.  Samples are shifted and mirrored in x at random:
  the domain is periodic in x and, at normal incidence, mirror-symmetric.
- **Training.** The network is the one the inference kernels compute (pf_unet_jump),
  written a second time with PyTorch operations so that autograd can differentiate it.
  Adam on the summed relative squared error of the three fields ("Training of the
  network", "Error metrics"), cosine learning-rate decay over the time budget, BF16 autocast.
- **Output.** The weights are written under the names pf.UNet expects.  Prediction
  with them runs only in the hand-written BF16 tensor-core kernels.
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np

from . import inputs as I

CH = I.UNET_CHANNELS
FDIM = I.UNET_FDIM


def generate(pf, runs: int, side: int = 256, seed: int = 11, every: int = 1000, snapshots: int = 100):
    """(phi, c, rho) snapshots [snapshots + 1, runs, 3, side, side] (FP32, on the GPU) of seeded films,
    one every `every` steps."""
    import torch

    ms = []
    for m in I.hybrid_members(runs, side, seed=seed):
        p = I.default_params(v_mag=m["v_mag"])
        p["dt"] = 0.5 * pf.pf_dt_limit(p)[0]
        ms.append((p, *I.film_state(m["spec"], p)))
    probe = pf.Ensemble(ms)  # the autotuner's tile shape, timed on a throwaway copy of the batch
    tile, _ = probe.autotune(20)
    probe.close()
    ens = pf.Ensemble(ms)
    ens.set_tile(tile)
    out = torch.empty((snapshots + 1, runs, 3, side, side), dtype=torch.float32, device="cuda")

    def grab(k):
        for r, run in enumerate(ens.fields):
            for q in range(3):
                out[k, r, q].copy_(run[q][:, :side])

    grab(0)
    for k in range(1, snapshots + 1):
        ens.step(every)
        grab(k)
    torch.cuda.synchronize()
    ens.close()
    return out


def make_model(seed: int = 0):
    import torch
    import torch.nn.functional as F

    class Net(torch.nn.Module):
        def __init__(self):
            super().__init__()
            W = I.unet_weights(seed)
            W["out_gamma"] = np.full(I.UNET_OUT, 0.1, np.float32)  # start close to the identity jump
            W["out_beta"] = np.zeros(I.UNET_OUT, np.float32)
            self.p = torch.nn.ParameterDict({k: torch.nn.Parameter(torch.from_numpy(v.copy())) for k, v in W.items()})

        def block(self, x, name, fp32=False):
            if fp32:  # the first convolution reads the FP32 fields with FP32 weights, as the kernel does
                with torch.autocast("cuda", enabled=False):
                    y = F.conv2d(x.float(), self.p[name].float(), padding=1)
            else:
                y = F.conv2d(x, self.p[name], padding=1)
            y = F.group_norm(y, 8, self.p[name + "_gamma"], self.p[name + "_beta"], eps=1e-5)
            return F.gelu(y, approximate="tanh")

        def forward(self, x, tau):
            p = self.p
            t = torch.full((1, 1), float(tau), device=x.device)
            h = torch.sin(t @ p["mlp_w0"].t() + p["mlp_b0"])
            h = torch.sin(h @ p["mlp_w1"].t() + p["mlp_b1"])
            f = (h @ p["mlp_w2"].t() + p["mlp_b2"])[0]
            s = [p[f"proj{k}"] @ f for k in range(1, 5)]
            z1 = self.block(x, "enc1", fp32=True)
            z2 = self.block(F.max_pool2d(z1, 2), "enc2")
            z3 = self.block(F.max_pool2d(z2, 2), "enc3")
            z4 = self.block(F.max_pool2d(z3, 2), "enc4")
            zc = [z * sp[None, :, None, None] for z, sp in zip((z1, z2, z3, z4), s)]
            d3 = F.conv_transpose2d(self.block(zc[3], "dec4"), p["up4"], stride=2)
            d2 = F.conv_transpose2d(self.block(torch.cat([zc[2], d3], 1), "dec3"), p["up3"], stride=2)
            d1 = F.conv_transpose2d(self.block(torch.cat([zc[1], d2], 1), "dec2"), p["up2"], stride=2)
            h1 = self.block(torch.cat([zc[0], d1], 1), "dec1")
            inc = F.conv2d(h1, p["out"], padding=1)
            k = 3 * (I.UNET_LB - 1)  # the newest frame
            return x[:, k:k + 3] + inc * p["out_gamma"][None, :, None, None] + p["out_beta"][None, :, None, None]

    return Net()


def train(pf, runs: int = 200, budget_s: float = 1800.0, batch: int = 8, lr: float = 1e-3, seed: int = 0,
          held_out: int = 4, field_weights=(1.0, 1.0, 1.0), log=print) -> dict:
    import torch

    torch.manual_seed(seed)
    lb, gap, ahead = I.UNET_LB, 1, 2  # frames 1 snapshot apart, target 2 snapshots after the newest frame
    data = generate(pf, runs)          # [101, runs, 3, H, W]
    S, R = data.shape[0], data.shape[1]
    first = (lb - 1) * gap
    idx = [(k, r) for k in range(first, S - ahead) for r in range(R)]
    val = [(k, r) for (k, r) in idx if r >= R - held_out]  # the last runs are held out
    trn = [(k, r) for (k, r) in idx if r < R - held_out]
    net = make_model(seed).cuda()
    opt = torch.optim.Adam(net.parameters(), lr=lr)
    g = np.random.default_rng(seed)

    def sample(ids, augment=False):
        x = torch.stack([torch.cat([data[k - (lb - 1 - f) * gap, r] for f in range(lb)]
                                   + [torch.ones_like(data[k, r, :1])]) for k, r in ids])
        y = torch.stack([data[k + ahead, r] for k, r in ids])
        if augment:  # x is periodic and, at normal incidence, mirror-symmetric: random shifts and flips
            shift = int(g.integers(0, x.shape[-1]))
            x, y = torch.roll(x, shift, dims=-1), torch.roll(y, shift, dims=-1)
            if g.integers(0, 2):
                x, y = torch.flip(x, dims=(-1,)), torch.flip(y, dims=(-1,))
        return x, y

    def loss_fn(pred, y):  # relative squared error of each field, weighted
        return sum(field_weights[q] * ((pred[:, q] - y[:, q]) ** 2).sum() / (y[:, q] ** 2).sum() for q in range(3))

    def validate():
        """Held-out relative squared error per field (phi, c, rho), one jump from DNS frames."""
        num, den = torch.zeros(3), torch.zeros(3)
        with torch.no_grad(), torch.autocast("cuda", dtype=torch.bfloat16):
            for i in range(0, len(val), 16):
                x, y = sample(val[i:i + 16])
                pred = net(x, 1.0).float()
                for q in range(3):
                    num[q] += float(((pred[:, q] - y[:, q]) ** 2).sum())
                    den[q] += float((y[:, q] ** 2).sum())
        return (num / den).tolist()

    t0 = time.time()
    step = epoch = 0
    loss = torch.zeros(())
    while time.time() - t0 < budget_s:
        order = g.permutation(len(trn))
        for i in range(0, len(order) - batch + 1, batch):
            frac = min(1.0, (time.time() - t0) / budget_s)
            for gr in opt.param_groups:
                gr["lr"] = lr * 0.5 * (1 + math.cos(math.pi * frac))  # cosine decay over the budget
            x, y = sample([trn[j] for j in order[i:i + batch]], augment=True)
            with torch.autocast("cuda", dtype=torch.bfloat16):
                pred = net(x, 1.0)
            loss = loss_fn(pred.float(), y)
            opt.zero_grad(set_to_none=True)
            loss.backward()
            opt.step()
            step += 1
            if time.time() - t0 > budget_s:
                break
        epoch += 1
        v = validate()
        log(f"epoch {epoch} step {step} t {time.time() - t0:.0f}s train {float(loss.detach()) / sum(field_weights):.3e} "
            f"val rel L2 phi {math.sqrt(v[0]):.3e} c {math.sqrt(v[1]):.3e} rho {math.sqrt(v[2]):.3e}")
    return {k: v.detach().float().cpu().numpy() for k, v in net.p.items()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--runs", type=int, default=200)
    ap.add_argument("--budget", type=float, default=1800.0)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--field-weights", type=float, nargs=3, default=(1.0, 1.0, 1.0),
                    help="loss weights of the relative squared errors of phi, c, rho")
    args = ap.parse_args()
    from . import build as B
    B.build()
    from . import pf
    W = train(pf, args.runs, args.budget, args.batch, args.lr, field_weights=tuple(args.field_weights))
    np.savez(args.out, **W)
    print(f"wrote {args.out}")


if __name__ == "__main__":
    main()
