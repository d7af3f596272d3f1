"""Pins of the FP64 reference adjoint (oracle/adjoint_ref.py).

Its forward must reproduce the C oracle, and its gradients must match central
finite differences of the C oracle (an independent implementation of the
forward) for every parameter and for sampled entries of every initial field.
"""
import numpy as np
import pytest

import oracle as O
from paper_2312_05410_gb300 import inputs as I

torch = pytest.importorskip("torch")
from oracle import adjoint_ref as A  # noqa: E402


def setup_case(phi_mode=0, surf=True, nx=24, ny=20, seed=4):
    over = dict(v_angle_deg=70.0, v_mag=0.6, phi_mode=phi_mode, MA_bulk=1.6, MB_bulk=0.7)
    if surf:
        over.update(MA_surf=2.0, MB_surf=1.0, sigma_surf=0.6)
    p = O.with_dt(I.default_params(**over))
    st = [a.astype(np.float64) for a in I.film_state(I.FilmSpec(nx, ny, ny / 3.0, seed=seed), p)]
    rng = np.random.default_rng(seed)
    w = [rng.standard_normal((ny, nx)) for _ in range(3)]
    return p, st, w


def linear_loss(p, st, w, n):
    f, c, r = O.step(p, *st, n)
    return float((w[0] * f).sum() + (w[1] * c).sum() + (w[2] * r).sum())


def test_reference_forward_matches_the_c_oracle():
    p, st, _ = setup_case()
    ref = O.step(p, *st, 25)
    got = A.run(p, *(torch.tensor(a) for a in st), 25)
    for a, b in zip(got, ref):
        np.testing.assert_allclose(a.numpy(), b, rtol=0, atol=1e-12)


@pytest.mark.parametrize("phi_mode", [0, 1])
def test_reference_gradients_match_finite_differences(phi_mode):
    p, st, w = setup_case(phi_mode=phi_mode)
    n = 30
    g = A.gradients(p, *st, n, *w)
    # parameters (central differences, FP64)
    for name, perturb in (
        ("v_mag", lambda q, e: dict(q, v_mag=q["v_mag"] + e)),
        ("kappa_c", lambda q, e: dict(q, kappa_c=q["kappa_c"] + e)),
        ("m_scale", lambda q, e: dict(q, **{k: q[k] * (1.0 + e) for k in ("MA_bulk", "MB_bulk", "MA_surf", "MB_surf")})),
    ):
        e = 1e-5
        fd = (linear_loss(perturb(p, e), st, w, n) - linear_loss(perturb(p, -e), st, w, n)) / (2 * e)
        assert g[name] == pytest.approx(fd, rel=2e-6, abs=1e-8), name
    # sampled entries of the initial fields, including boundary rows and the wrap column
    for fi, key in enumerate(("phi0", "c0", "rho0")):
        for (j, i) in ((0, 0), (1, 5), (9, 11), (19, 23), (18, 0)):
            e = 1e-6
            up = [a.copy() for a in st]
            dn = [a.copy() for a in st]
            up[fi][j, i] += e
            dn[fi][j, i] -= e
            fd = (linear_loss(p, up, w, n) - linear_loss(p, dn, w, n)) / (2 * e)
            assert g[key][j, i] == pytest.approx(fd, rel=1e-5, abs=1e-7), (key, j, i)
