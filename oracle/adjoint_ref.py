"""Reference gradients of the explicit phase-field PVD step (FP64, CPU, PyTorch autograd).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.  This is a plain
PyTorch restatement of the same discrete scheme as ``pf_oracle.c``
(Materials and Methods: [CH-c], [Mc], [MBulk], [MSurf], [CH-phi], [S], [rho];
"Dataset": central differences and the explicit midpoint method; boundary
and closure readings as in the C oracle).  Autograd through it gives the
exact discrete gradient of a loss of the final state with respect to the
initial fields and to three scalar parameters:

  v_mag    the incident vapor speed V (deposition rate),
  m_scale  a factor on the composition mobility, M_c -> m_scale * M_c (at 1),
  kappa_c  the composition gradient-energy coefficient.

The time step dt is held fixed.  Its forward is checked against the C oracle
and its gradients against central finite differences of the C oracle.
"""
from __future__ import annotations

import math

import numpy as np
import torch

DT = torch.float64


def _pad(u, top=None):
    """One ghost ring: periodic in x, mirror at the bottom, mirror or a constant at the top."""
    u = torch.cat([u[:, -1:], u, u[:, :1]], dim=1)
    bottom = u[:1]
    above = u[-1:] if top is None else torch.full_like(u[-1:], top)
    return torch.cat([bottom, u, above], dim=0)


def _lap(up, dx2):
    return (up[1:-1, 2:] + up[1:-1, :-2] + up[2:, 1:-1] + up[:-2, 1:-1] - 4.0 * up[1:-1, 1:-1]) / dx2


def rhs(p: dict, phi, c, rho, v_mag, m_scale, kappa_c):
    dx = p["dx"]
    dx2 = dx * dx
    pp, cp = _pad(phi), _pad(c)
    P = 0.25 * (2.0 - phi) * (1.0 + phi) ** 2
    dP = 0.75 * (1.0 - phi ** 2)
    g = c ** 2 * (1.0 - c) ** 2
    dg = 2.0 * c * (1.0 - c) * (1.0 - 2.0 * c)
    mu_c = P * p["W_c"] * dg - kappa_c * _lap(cp, dx2)
    mu_f = -p["W_phi"] * phi * (1.0 - phi ** 2) + dP * p["W_c"] * g - p["kappa_phi"] * _lap(pp, dx2)
    h = c ** 2 * (3.0 - 2.0 * c)
    M = P * (h * p["MA_bulk"] + (1.0 - h) * p["MB_bulk"])
    M = M + torch.exp(-(phi / p["sigma_surf"]) ** 2) * (h * p["MA_surf"] + (1.0 - h) * p["MB_surf"])
    M = m_scale * M
    Mp, mp = _pad(M), _pad(mu_c)
    Rc = torch.zeros_like(c)
    for sl in ((slice(1, -1), slice(2, None)), (slice(1, -1), slice(None, -2)),
               (slice(2, None), slice(1, -1)), (slice(None, -2), slice(1, -1))):
        Rc = Rc + 0.5 * (M + Mp[sl]) * (mp[sl] - mu_c)
    Rc = Rc / dx2
    if p["deposition"]:
        th = math.radians(p["v_angle_deg"])
        vx, vy = v_mag * math.cos(th), -v_mag * math.sin(th)
    else:
        vx = vy = 0.0 * v_mag
    S = rho * (vx * (pp[1:-1, 2:] - pp[1:-1, :-2]) + vy * (pp[2:, 1:-1] - pp[:-2, 1:-1])) / (2.0 * dx)
    if p["phi_mode"] == 0:
        Rf = p["M_phi"] * _lap(_pad(mu_f), dx2) + S
    else:
        Rf = -p["L_phi"] * mu_f + S
    rp = _pad(rho, top=p["rho_top"])
    adv = (vx * (rp[1:-1, 2:] - rp[1:-1, :-2]) + vy * (rp[2:, 1:-1] - rp[:-2, 1:-1])) / (2.0 * dx)
    Rr = p["D_rho"] * _lap(rp, dx2) - adv - S
    return Rf, Rc, Rr


def run(p: dict, phi, c, rho, nsteps: int, v_mag=None, m_scale=None, kappa_c=None):
    """nsteps explicit midpoint steps; returns the final (phi, c, rho)."""
    v_mag = torch.tensor(p["v_mag"], dtype=DT) if v_mag is None else v_mag
    m_scale = torch.tensor(1.0, dtype=DT) if m_scale is None else m_scale
    kappa_c = torch.tensor(p["kappa_c"], dtype=DT) if kappa_c is None else kappa_c
    dt = p["dt"]
    for _ in range(nsteps):
        Rf, Rc, Rr = rhs(p, phi, c, rho, v_mag, m_scale, kappa_c)
        fs, cs, rs = phi + 0.5 * dt * Rf, c + 0.5 * dt * Rc, rho + 0.5 * dt * Rr
        Rf, Rc, Rr = rhs(p, fs, cs, rs, v_mag, m_scale, kappa_c)
        phi, c, rho = phi + dt * Rf, c + dt * Rc, rho + dt * Rr
    return phi, c, rho


def gradients(p: dict, phi0, c0, rho0, nsteps: int, w_phi, w_c, w_rho=None):
    """Gradient of L = sum(w_phi * phi_N + w_c * c_N [+ w_rho * rho_N]) (a linear functional of the
    final state, i.e. the vector-Jacobian product with cotangent w) with respect to the initial fields
    and (v_mag, m_scale, kappa_c).  Returns a dict of numpy arrays / floats."""
    t = lambda a: torch.tensor(np.asarray(a, dtype=np.float64), dtype=DT, requires_grad=True)
    phi, c, rho = t(phi0), t(c0), t(rho0)
    v = torch.tensor(float(p["v_mag"]), dtype=DT, requires_grad=True)
    ms = torch.tensor(1.0, dtype=DT, requires_grad=True)
    kc = torch.tensor(float(p["kappa_c"]), dtype=DT, requires_grad=True)
    f, cc, r = run(p, phi, c, rho, nsteps, v, ms, kc)
    L = (torch.as_tensor(np.asarray(w_phi, dtype=np.float64)) * f).sum() + \
        (torch.as_tensor(np.asarray(w_c, dtype=np.float64)) * cc).sum()
    if w_rho is not None:
        L = L + (torch.as_tensor(np.asarray(w_rho, dtype=np.float64)) * r).sum()
    L.backward()
    return {"phi0": phi.grad.numpy(), "c0": c.grad.numpy(), "rho0": rho.grad.numpy(),
            "v_mag": float(v.grad), "m_scale": float(ms.grad), "kappa_c": float(kc.grad)}
