"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
the variational structure of the (read) free energy, continuum derivatives of
analytic fields, conservation laws, energy dissipation, the equilibrium tanh
interface, the discrete and continuum dispersion relations, the midpoint
method's time order, symmetries and the explicit stability limit.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2312_05410_gb300 import inputs as I


# ------------------------------------------------------------------ closed forms
def test_switching_and_indicator_closed_forms():
    # p(phi) = 1/4 (2-phi)(1+phi)^2: 0 in vapor (phi=-1), 1 in solid (phi=+1), flat at both.
    assert O.p_fn(-1.0) == 0.0 and O.p_fn(1.0) == 1.0
    assert O.dp_fn(-1.0) == 0.0 and O.dp_fn(1.0) == 0.0
    # h(c): 0, 1/2, 1 at c = 0, 1/2, 1; the reading makes p(phi) = h((1+phi)/2) exactly.
    assert O.h_fn(0.0) == 0.0 and O.h_fn(1.0) == 1.0 and O.h_fn(0.5) == 0.5
    for x in np.linspace(-1.3, 1.3, 27):
        assert O.p_fn(x) == pytest.approx(O.h_fn(0.5 * (1.0 + x)), abs=1e-15)
    # g(c) = c^2 (1-c)^2: zeros at 0 and 1, maximum 1/16 at 1/2.
    assert O.g_fn(0.0) == 0.0 and O.g_fn(1.0) == 0.0 and O.g_fn(0.5) == 0.0625
    # derivatives by central differences
    e = 1e-6
    for x in np.linspace(-1.2, 1.2, 13):
        assert O.dp_fn(x) == pytest.approx((O.p_fn(x + e) - O.p_fn(x - e)) / (2 * e), abs=1e-8)
        assert O.dg_fn(x) == pytest.approx((O.g_fn(x + e) - O.g_fn(x - e)) / (2 * e), abs=1e-8)


def test_mobility_limits():
    # Bulk term vanishes in vapor and equals the interpolated bulk mobility in the solid.
    pd = I.default_params(MA_bulk=3.0, MB_bulk=1.0, MA_surf=0.0, MB_surf=0.0)
    assert O.mobility(pd, -1.0, 0.3) == 0.0
    assert O.mobility(pd, 1.0, 1.0) == pytest.approx(3.0)
    assert O.mobility(pd, 1.0, 0.0) == pytest.approx(1.0)
    assert O.mobility(pd, 1.0, 0.5) == pytest.approx(2.0)
    # Surface term: exp(-(phi/sigma)^2) weight, full at phi = 0 where p(0) = 1/2.
    pd = I.default_params(MA_bulk=0.0, MB_bulk=0.0, MA_surf=10.0, MB_surf=4.0, sigma_surf=0.5)
    assert O.mobility(pd, 0.0, 1.0) == pytest.approx(10.0)
    assert O.mobility(pd, 0.5, 0.0) == pytest.approx(4.0 * math.exp(-1.0))
    assert O.mobility(pd, 1.0, 0.5) == pytest.approx(7.0 * math.exp(-4.0))


def test_dt_limit_closed_form_small_config():
    # dx = 1, M = 1, kappa = 2, W = 1: dt_phi = 2 / (kappa 64 + (2 + 3/32) 8) = 2 / 144.75,
    # dt_c = 2 / (2 * 64 + 2 * 8) = 2/144; vapor limited by diffusion, dx^2 / (4 D) = 1/4.
    d = O.dt_limit(I.default_params())
    assert d["dt_phi"] == pytest.approx(2.0 / 144.75, rel=1e-15)
    assert d["dt_c"] == pytest.approx(2.0 / 144.0, rel=1e-15)
    assert d["dt_rho"] == pytest.approx(0.25, rel=1e-12)
    assert d["dt_lim"] == d["dt_phi"]
    # Allen-Cahn phi: dt = 2 / (L (kappa 8 + 2 W + 3/32 W_c))
    d = O.dt_limit(I.default_params(phi_mode=1))
    assert d["dt_phi"] == pytest.approx(2.0 / (16.0 + 2.09375), rel=1e-15)
    # Pure advection of vapor is unstable for the midpoint method at any dt; the
    # limit collapses to the scan's round-off tolerance (|gain| <= 1 + 1e-13).
    assert O.dt_limit(I.default_params(D_rho=0.0))["dt_rho"] < 0.01


# --------------------------------------------------------- variational structure
def test_chemical_potentials_are_energy_gradients():
    """mu_u,i = dx^-2 dF_h/du_i: pins signs, kappa, p', g', the Laplacian and its mirror BCs."""
    pd = I.default_params(dx=0.7, W_c=1.3, W_phi=0.8, kappa_c=1.7, kappa_phi=2.3)
    rng = np.random.default_rng(5)
    ny, nx = 6, 7
    phi = rng.uniform(-1.1, 1.1, (ny, nx))
    c = rng.uniform(-0.1, 1.1, (ny, nx))
    mu_c, mu_f = O.chem_pot(pd, phi, c)
    e = 1e-6
    for j in range(ny):
        for i in range(nx):
            for arr, mu, which in ((c, mu_c, "c"), (phi, mu_f, "phi")):
                a = arr.copy(); a[j, i] += e
                b = arr.copy(); b[j, i] -= e
                if which == "c":
                    Fp, Fm = O.free_energy(pd, phi, a), O.free_energy(pd, phi, b)
                else:
                    Fp, Fm = O.free_energy(pd, a, c), O.free_energy(pd, b, c)
                fd = (Fp - Fm) / (2 * e) / pd["dx"] ** 2
                assert mu[j, i] == pytest.approx(fd, rel=1e-6, abs=1e-7), (which, j, i)


def test_free_energy_uniform_state():
    pd = I.default_params(dx=0.5)
    phi = np.full((5, 6), 0.3)
    c = np.full((5, 6), 0.2)
    f = 0.25 * (1 - 0.09) ** 2 + O.p_fn(0.3) * (0.2 * 0.8) ** 2
    assert O.free_energy(pd, phi, c) == pytest.approx(30 * 0.25 * f, rel=1e-14)
    out = O.diag(pd, phi, c, np.full((5, 6), 0.7))
    assert out[0] == pytest.approx(30 * 0.25 * 0.2)
    assert out[1] == pytest.approx(30 * 0.25 * 0.3)
    assert out[2] == pytest.approx(30 * 0.25 * 0.7)


# ----------------------------------------------------- continuum right-hand side
def _continuum_rhs(pd, L):
    sympy = pytest.importorskip("sympy")
    x, y = sympy.symbols("x y", real=True)
    k = 2 * sympy.pi / L
    q = sympy.pi / L
    phi = sympy.Rational(1, 5) + sympy.Rational(3, 5) * sympy.cos(k * x) * sympy.cos(q * y)
    c = sympy.Rational(1, 2) + sympy.Rational(1, 5) * sympy.sin(k * x) * sympy.cos(2 * q * y)
    rho = sympy.Rational(1, 2) + sympy.Rational(3, 10) * sympy.cos(k * x + 1) * sympy.cos(q * y)
    W_c, W_f, kc, kf = (sympy.Float(pd[n]) for n in ("W_c", "W_phi", "kappa_c", "kappa_phi"))
    p = sympy.Rational(1, 4) * (2 - phi) * (1 + phi) ** 2
    dp = sympy.Rational(3, 4) * (1 - phi ** 2)
    g = c ** 2 * (1 - c) ** 2
    dg = 2 * c * (1 - c) * (1 - 2 * c)
    h = c ** 2 * (3 - 2 * c)
    lap = lambda u: sympy.diff(u, x, 2) + sympy.diff(u, y, 2)
    mu_c = p * W_c * dg - kc * lap(c)
    mu_f = -W_f * phi * (1 - phi ** 2) + dp * W_c * g - kf * lap(phi)
    M = p * (h * pd["MA_bulk"] + (1 - h) * pd["MB_bulk"]) + sympy.exp(-(phi / pd["sigma_surf"]) ** 2) * (
        h * pd["MA_surf"] + (1 - h) * pd["MB_surf"])
    th = math.radians(pd["v_angle_deg"])
    vx, vy = pd["v_mag"] * math.cos(th), -pd["v_mag"] * math.sin(th)
    S = rho * (vx * sympy.diff(phi, x) + vy * sympy.diff(phi, y))
    Rc = sympy.diff(M * sympy.diff(mu_c, x), x) + sympy.diff(M * sympy.diff(mu_c, y), y)
    if pd["phi_mode"] == 0:
        Rf = pd["M_phi"] * lap(mu_f) + S
    else:
        Rf = -pd["L_phi"] * mu_f + S
    Rr = pd["D_rho"] * lap(rho) - (sympy.diff(rho * vx, x) + sympy.diff(rho * vy, y)) - S
    f = lambda e: sympy.lambdify((x, y), e, "numpy")
    return [f(e) for e in (phi, c, rho, Rf, Rc, Rr)]


@pytest.mark.parametrize("phi_mode", [0, 1])
def test_rhs_matches_continuum_to_second_order(phi_mode):
    """Discrete R against the continuum PDE right-hand sides on smooth analytic fields.

    Fields are even about y = 0 and y = L (so the mirror BCs are exact) and periodic in x.
    The top row of rho is excluded: its ghost holds rho_top, a first-order Dirichlet closure.
    """
    L = 32.0
    pd = I.default_params(MA_bulk=2.0, MB_bulk=0.5, MA_surf=3.0, MB_surf=1.0, sigma_surf=0.6,
                          v_angle_deg=60.0, v_mag=0.7, D_rho=0.8, M_phi=1.3, L_phi=0.9,
                          phi_mode=phi_mode, kappa_c=2.0, kappa_phi=3.0, rho_top=0.5)
    fphi, fc, frho, gRf, gRc, gRr = _continuum_rhs(pd, L)
    errs = []
    for N in (32, 64, 128):
        dx = L / N
        q = dict(pd, dx=dx)
        xc = (np.arange(N) + 0.5) * dx
        X, Y = np.meshgrid(xc, xc)
        Rf, Rc, Rr = O.rhs(q, fphi(X, Y), fc(X, Y), frho(X, Y))
        e = (np.abs(Rf - gRf(X, Y)).max(), np.abs(Rc - gRc(X, Y)).max(),
             np.abs(Rr - gRr(X, Y))[:-1].max())
        errs.append(np.array(e))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert np.all((r1 > 3.5) & (r1 < 4.6)), (errs, r1)
    assert np.all((r2 > 3.7) & (r2 < 4.3)), (errs, r2)


# ----------------------------------------------------------- conservation, energy
def _small_state(deposition, phi_mode=0, steps_params=None):
    pd = I.default_params(deposition=deposition, phi_mode=phi_mode, **(steps_params or {}))
    pd = O.with_dt(pd)
    spec = I.FilmSpec(32, 32, 8.0, seed=4)
    return pd, I.film_state(spec, pd)


@pytest.mark.parametrize("deposition", [0, 1])
def test_composition_is_conserved(deposition):
    # No c-flux through any boundary and no c-source: sum(c) is constant in both modes.
    pd, (phi, c, rho) = _small_state(deposition)
    d0 = O.diag(pd, phi, c, rho)
    f, cc, r = O.step(pd, phi, c, rho, 2000)
    d1 = O.diag(pd, f, cc, r)
    assert abs(d1[0] - d0[0]) <= 1e-12 * abs(d0[0])
    if deposition == 0:
        # Cahn-Hilliard phi without source conserves sum(phi) as well
        assert abs(d1[1] - d0[1]) <= 1e-11 * abs(d0[1]) + 1e-11
    else:
        # the source deposits solid: sum(phi) grows
        assert d1[1] > d0[1] + 1.0


@pytest.mark.parametrize("phi_mode", [0, 1])
def test_free_energy_decreases_without_deposition(phi_mode):
    pd, (phi, c, rho) = _small_state(0, phi_mode)
    F = [O.free_energy(pd, phi, c)]
    f, cc, r = phi, c, rho
    for _ in range(100):
        f, cc, r = O.step(pd, f, cc, r, 10)
        F.append(O.free_energy(pd, f, cc))
    F = np.array(F)
    assert np.all(np.diff(F) <= 1e-12 * abs(F[0])), np.diff(F).max()
    assert F[-1] < F[0]


# ------------------------------------------------------------ flat interface
def _tanh_profile_error(kappa):
    ny, nx, H = 64, 4, 32.0
    pd = I.default_params(phi_mode=1, deposition=0, kappa_phi=kappa, kappa_c=kappa)
    pd = O.with_dt(pd)
    xi = math.sqrt(kappa / pd["W_phi"])
    y = np.arange(ny) + 0.5
    exact = -np.tanh((y - H) / (math.sqrt(2.0) * xi))
    phi = np.repeat(exact[:, None], nx, axis=1)
    c = np.ones_like(phi)
    rho = np.zeros_like(phi)
    steps = int(round(60.0 / pd["dt"]))
    f, cc, _ = O.step(pd, phi, c, rho, steps)
    assert np.all(cc == 1.0)  # g = g' = 0 at c = 1 decouples phi
    return np.abs(f[:, 0] - exact).max(), f


def test_flat_interface_matches_tanh_profile():
    """Relaxed discrete interface vs the closed-form -tanh((y-H)/(sqrt(2) xi)); error O((dx/xi)^2)."""
    e1, f1 = _tanh_profile_error(8.0)
    e2, _ = _tanh_profile_error(32.0)
    assert e1 < 0.2 * (1.0 / 8.0)  # (dx/xi)^2 = 1/8
    assert 3.0 < e1 / e2 < 5.0, (e1, e2)
    # the profile is antisymmetric about H (equal wells at c = 1)
    assert np.allclose(f1[:32, 0], -f1[::-1, 0][:32], atol=1e-10)


# ---------------------------------------------------------- linear stability
def _mode(nx, ny, mx, my):
    i = np.arange(nx)
    j = np.arange(ny)
    return np.outer(np.cos(math.pi * my * (j + 0.5) / ny), np.cos(2 * math.pi * mx * i / nx))


def _lam_hat(nx, ny, mx, my, dx):
    return 4.0 / dx ** 2 * (math.sin(math.pi * mx / nx) ** 2 + math.sin(math.pi * my / (2 * ny)) ** 2)


@pytest.mark.parametrize("mx,my", [(3, 2), (1, 1), (10, 9)])
def test_composition_dispersion_relation(mx, my):
    """Small c-mode about c = 1/2 in the solid: per-step gain 1 + z + z^2/2 with
    z = dt M lam (W - kappa lam), lam the 5-point eigenvalue (exact discrete form)."""
    nx, ny = 32, 16
    pd = O.with_dt(I.default_params(deposition=0))
    mode = _mode(nx, ny, mx, my)
    amp = 1e-6
    phi = np.ones((ny, nx))
    c = 0.5 + amp * mode
    n = 300
    f, cc, _ = O.step(pd, phi, c, np.zeros_like(phi), n)
    assert np.all(f == 1.0)
    a = ((cc - 0.5) * mode).sum() / (mode * mode).sum()
    lam = _lam_hat(nx, ny, mx, my, pd["dx"])
    z = pd["dt"] * 1.0 * lam * (pd["W_c"] - pd["kappa_c"] * lam)
    expect = amp * (1 + z + 0.5 * z * z) ** n
    assert a == pytest.approx(expect, rel=1e-8)


@pytest.mark.parametrize("phi_mode", [0, 1])
def test_order_parameter_dispersion_relation(phi_mode):
    """Small phi-mode about phi = +1 at c = 1: CH z = -dt M lam (2W + kappa lam),
    AC z = -dt L (2W + kappa lam)."""
    nx, ny, mx, my = 16, 16, 2, 3
    pd = O.with_dt(I.default_params(deposition=0, phi_mode=phi_mode, M_phi=1.4, L_phi=0.7))
    mode = _mode(nx, ny, mx, my)
    amp = 1e-7
    phi = 1.0 + amp * mode
    n = 200
    f, _, _ = O.step(pd, phi, np.ones_like(phi), np.zeros_like(phi), n)
    a = ((f - 1.0) * mode).sum() / (mode * mode).sum()
    lam = _lam_hat(nx, ny, mx, my, pd["dx"])
    rate = pd["M_phi"] * lam if phi_mode == 0 else pd["L_phi"]
    z = -pd["dt"] * rate * (2 * pd["W_phi"] + pd["kappa_phi"] * lam)
    assert a == pytest.approx(amp * (1 + z + 0.5 * z * z) ** n, rel=1e-6)


def test_continuum_growth_rate_long_wave():
    """Long-wave c-mode grows at the continuum rate M k^2 (W - kappa k^2) up to O((k dx)^2)."""
    nx, ny, mx = 128, 4, 3
    pd = O.with_dt(I.default_params(deposition=0, kappa_c=20.0))
    mode = _mode(nx, ny, mx, 0)
    amp = 1e-6
    n = 2000
    _, cc, _ = O.step(pd, np.ones((ny, nx)), 0.5 + amp * mode, np.zeros((ny, nx)), n)
    a = ((cc - 0.5) * mode).sum() / (mode * mode).sum()
    omega_meas = math.log(a / amp) / (n * pd["dt"])
    k = 2 * math.pi * mx / (nx * pd["dx"])
    omega = k * k * (pd["W_c"] - pd["kappa_c"] * k * k)
    assert omega > 0
    assert abs(omega_meas / omega - 1) < 2 * (k * pd["dx"]) ** 2


# ---------------------------------------------------------- time order
def test_midpoint_method_is_second_order_in_time():
    pd0 = I.default_params(deposition=1, v_angle_deg=70.0)
    base = O.dt_limit(pd0)["dt_lim"] * 0.4
    spec = I.FilmSpec(16, 16, 6.0, seed=9)
    phi, c, rho = I.film_state(spec, pd0)
    T = 200 * base
    sols = []
    for m in (1, 2, 4, 8):
        q = dict(pd0, dt=base / m)
        sols.append(O.step(q, phi, c, rho, 200 * m))
    err = [max(np.abs(a - b).max() for a, b in zip(sols[i], sols[i + 1])) for i in range(3)]
    assert 3.6 < err[0] / err[1] < 4.4, err
    assert 3.8 < err[1] / err[2] < 4.2, err
    assert T > 0


# ---------------------------------------------------------- symmetries
def test_x_shift_equivariance_is_exact():
    pd = O.with_dt(I.default_params(v_angle_deg=60.0))
    phi, c, rho = I.random_state(12, 10, seed=2)
    a = O.step(pd, phi, c, rho, 20)
    b = O.step(pd, np.roll(phi, 5, 1), np.roll(c, 5, 1), np.roll(rho, 5, 1), 20)
    for u, v in zip(a, b):
        assert np.array_equal(np.roll(u, 5, 1), v)


def test_x_mirror_symmetry_at_normal_incidence():
    pd = O.with_dt(I.default_params(v_angle_deg=90.0))
    phi, c, rho = I.random_state(12, 10, seed=3)
    a = O.step(pd, phi, c, rho, 20)
    b = O.step(pd, phi[:, ::-1], c[:, ::-1], rho[:, ::-1], 20)
    for u, v in zip(a, b):
        assert np.allclose(u[:, ::-1], v, atol=1e-12, rtol=0)


# ---------------------------------------------------------- stability limit
def _max_mode(nx, ny):
    i = np.arange(nx)
    j = np.arange(ny)
    return np.outer(np.cos(math.pi * (ny - 1) * (j + 0.5) / ny), (-1.0) ** i)


@pytest.mark.parametrize("frac,grows", [(1.05, True), (0.95, False)])
def test_stability_limit_order_parameter(frac, grows):
    # phi = -1, c = 1/2 is where f_phiphi reaches 2 W_phi + 3/32 W_c, the bound used for dt_phi
    nx, ny = 16, 16
    pd = I.default_params(deposition=0)
    q = dict(pd, dt=frac * O.dt_limit(pd)["dt_phi"])
    eps = 1e-9
    phi = -1.0 + eps * _max_mode(nx, ny)
    f, _, _ = O.step(q, phi, np.full((ny, nx), 0.5), np.zeros((ny, nx)), 400)
    amp = np.nan_to_num(np.abs(f + 1.0).max(), nan=np.inf)
    assert (amp > 100 * eps) == grows, amp


@pytest.mark.parametrize("frac,grows", [(1.05, True), (0.95, False)])
def test_stability_limit_composition(frac, grows):
    # c = 0 in the solid: f_cc = 2 W_c and M = 1, the bound used for dt_c
    nx, ny = 16, 16
    pd = I.default_params(deposition=0)
    q = dict(pd, dt=frac * O.dt_limit(pd)["dt_c"])
    eps = 1e-9
    c = eps * _max_mode(nx, ny)
    _, cc, _ = O.step(q, np.ones((ny, nx)), c, np.zeros((ny, nx)), 400)
    amp = np.nan_to_num(np.abs(cc).max(), nan=np.inf)
    assert (amp > 100 * eps) == grows, amp


@pytest.mark.parametrize("frac,grows", [(1.05, True), (0.95, False)])
def test_stability_limit_vapor(frac, grows):
    # pure vapor (phi = -1): phi and c are frozen, only rho evolves
    nx, ny = 16, 16
    pd = I.default_params(deposition=1, v_mag=0.5, v_angle_deg=70.0)
    q = dict(pd, dt=frac * O.dt_limit(pd)["dt_rho"])
    eps = 1e-9
    rho = 1.0 + eps * _max_mode(nx, ny)
    f, cc, r = O.step(q, -np.ones((ny, nx)), np.full((ny, nx), 0.5), rho, 400)
    assert np.all(f == -1.0) and np.all(cc == 0.5)
    amp = np.nan_to_num(np.abs(r - 1.0).max(), nan=np.inf)
    assert (amp > 100 * eps) == grows, amp


# ---------------------------------------------------------- deposition direction
def test_film_grows_at_the_incident_rate():
    """Source only (AC mode with L_phi = 0): phi is advected up at speed rho V sin(theta).

    With rho held near 1 by a wide vapor reservoir, the interface (phi = 0 crossing)
    rises by about V t over a short time.
    """
    ny, nx = 128, 4
    pd = I.default_params(phi_mode=1, L_phi=0.0, v_mag=0.5, v_angle_deg=90.0, D_rho=1.0)
    pd = O.with_dt(pd)
    y = np.arange(ny) + 0.5
    phi = np.repeat((-np.tanh((y - 40.0) / 8.0))[:, None], nx, 1)
    rho = np.ones_like(phi)
    c = np.ones_like(phi)
    steps = int(round(4.0 / pd["dt"]))
    f, _, r = O.step(pd, phi, c, rho, steps)
    col = f[:, 0]
    k = np.where((col[:-1] > 0) & (col[1:] <= 0))[0][0]
    y0 = y[k] + col[k] / (col[k] - col[k + 1])
    t = steps * pd["dt"]
    # rho is depleted at the interface, so the rise is at most V t and clearly positive
    assert 0.5 * 0.5 * t < y0 - 40.0 <= 0.5 * t * 1.02


# ---------------------------------------------------------- vapor boundary fluxes
def test_vapor_mass_balance_through_reservoir_and_substrate():
    """Pure vapor (phi = -1, S = 0): one midpoint step changes dx^2 sum(rho) by exactly
    dt dx sum_x (F_bottom - F_top) at the midpoint state, with the face fluxes
    F = -D drho/dy + v_y rho of the two ghost rules: reservoir value rho_top above the
    top row, mirror below the bottom row (so F_bottom = v_y rho_0)."""
    nx, ny = 9, 7
    pd = O.with_dt(I.default_params(v_mag=0.6, v_angle_deg=65.0, D_rho=0.7, rho_top=0.8, dx=0.9))
    rng = np.random.default_rng(8)
    phi = -np.ones((ny, nx))
    c = np.full((ny, nx), 0.4)
    rho = rng.uniform(0.0, 1.0, (ny, nx))
    _, _, Rr = O.rhs(pd, phi, c, rho)
    mid = rho + 0.5 * pd["dt"] * Rr
    _, _, r1 = O.step(pd, phi, c, rho, 1)
    dx, D, rt = pd["dx"], pd["D_rho"], pd["rho_top"]
    vy = -pd["v_mag"] * math.sin(math.radians(pd["v_angle_deg"]))
    F_top = -D * (rt - mid[-1]) / dx + vy * 0.5 * (rt + mid[-1])
    F_bot = vy * mid[0]
    expect = pd["dt"] * dx * (F_bot - F_top).sum()
    assert (r1.sum() - rho.sum()) * dx * dx == pytest.approx(expect, rel=1e-11, abs=1e-13)


def test_vapor_relaxes_to_reservoir_value():
    # deposition off, no film: diffusion from the reservoir fills the box to rho_top
    nx, ny = 4, 16
    pd = I.default_params(deposition=0, rho_top=0.75)
    pd["dt"] = 0.5 * O.dt_limit(pd)["dt_rho"]  # phi = -1 and c are frozen in pure vapor
    _, _, r = O.step(pd, -np.ones((ny, nx)), np.full((ny, nx), 0.5), np.zeros((ny, nx)), 30000)
    assert np.allclose(r, 0.75, atol=1e-6)


def test_all_cores_build_gives_the_checker_results_bit_for_bit():
    """The CPU baseline's OpenMP build of the same source splits rows over threads; every cell is
    computed by the same expressions, so its states equal the single-thread checker's exactly."""
    p = O.with_dt(I.default_params(v_angle_deg=70.0, MA_bulk=2.0, MB_bulk=0.5, MA_surf=3.0, MB_surf=1.0,
                                   sigma_surf=0.5))
    st = I.film_state(I.FilmSpec(70, 45, 12.0, seed=8), p)
    a = O.step(p, *st, 30)
    b = O.step_all_cores(p, *st, 30)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
