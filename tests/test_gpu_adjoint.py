"""Hand-written adjoint of the fused step (pf_adjoint) against the FP64 reference
adjoint (PyTorch autograd on CPU, itself pinned to finite differences of the C
oracle) and against FP64 central finite differences of the C oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2312_05410_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pf(cuda_ok):
    from paper_2312_05410_gb300 import build as B
    B.build()
    from paper_2312_05410_gb300 import pf as mod
    return mod


def case(phi_mode=0, nx=37, ny=29, seed=5, surf=True):
    over = dict(v_angle_deg=70.0, v_mag=0.6, phi_mode=phi_mode, MA_bulk=1.6, MB_bulk=0.7)
    if surf:
        over.update(MA_surf=2.0, MB_surf=1.0, sigma_surf=0.6)
    p = O.with_dt(I.default_params(**over))
    st = I.film_state(I.FilmSpec(nx, ny, ny / 3.0, seed=seed), p)
    rng = np.random.default_rng(seed)
    w = [rng.standard_normal((ny, nx)).astype(np.float32) for _ in range(3)]
    return p, st, w


def rel_err(a, b):
    return float(np.abs(np.asarray(a, dtype=np.float64) - b).max() / max(np.abs(b).max(), 1e-30))


@pytest.mark.parametrize("phi_mode,K", [(0, 7), (1, 40)])
def test_adjoint_matches_the_reference_adjoint(pf, phi_mode, K):
    from oracle import adjoint_ref as A

    p, st, w = case(phi_mode)
    n = 40
    ny, nx = st[0].shape
    res = pf.adjoint(p, pf.device_fields(st), nx, n, K, *pf.device_fields(w))
    ref = A.gradients(p, *(a.astype(np.float64) for a in st), n, *(x.astype(np.float64) for x in w))
    for key in ("phi0", "c0", "rho0"):
        got = res[key][:, :nx].cpu().numpy()
        assert rel_err(got, ref[key]) <= 1e-3, (key, rel_err(got, ref[key]))
    for key in ("v_mag", "m_scale", "kappa_c"):
        assert res[key] == pytest.approx(ref[key], rel=1e-3), key
    # the forward inside the adjoint is the plain step
    sim = pf.Sim(p, *st)
    sim.step(n)
    for a, b in zip(sim.numpy(), res["final"]):
        assert np.array_equal(a, b[:, :nx].cpu().numpy())
    sim.close()


def test_checkpoint_interval_does_not_change_the_gradient(pf):
    p, st, w = case(nx=48, ny=32)
    ny, nx = st[0].shape
    outs = [pf.adjoint(p, pf.device_fields(st), nx, 30, K, *pf.device_fields(w)) for K in (1, 13, 30)]
    for o in outs[1:]:
        for key in ("phi0", "c0", "rho0"):
            assert torch.equal(o[key], outs[0][key])
        for key in ("v_mag", "m_scale", "kappa_c"):
            assert o[key] == outs[0][key]


def test_adjoint_of_a_target_loss_matches_oracle_finite_differences(pf):
    """64 x 64, loss = sum (phi_N - phi_T)^2 + (c_N - c_T)^2 against a target run of the same
    film deposited faster and with a different kappa_c (an inverse-design setting); gradients in
    V, mobility scale, kappa_c and sampled c0 entries vs FP64 central differences."""
    p = O.with_dt(I.default_params(v_mag=0.5, v_angle_deg=80.0))
    nx = ny = 64
    n, K = 150, 50
    st = I.film_state(I.FilmSpec(nx, ny, 8.0, seed=0), p)
    tgt = O.step(dict(p, v_mag=0.65, kappa_c=2.2), *st, n)

    def loss(q, s):
        f, c, _ = O.step(q, *s, n)
        return float(((f - tgt[0]) ** 2).sum() + ((c - tgt[1]) ** 2).sum())

    sim = pf.Sim(p, *st)
    sim.step(n)
    f, c, _ = sim.numpy()
    sim.close()
    wf = (2.0 * (f.astype(np.float64) - tgt[0])).astype(np.float32)
    wc = (2.0 * (c.astype(np.float64) - tgt[1])).astype(np.float32)
    res = pf.adjoint(p, pf.device_fields(st), nx, n, K, *pf.device_fields([wf, wc]))
    st64 = [a.astype(np.float64) for a in st]
    for key, pert in (("v_mag", lambda q, e: dict(q, v_mag=q["v_mag"] + e)),
                      ("kappa_c", lambda q, e: dict(q, kappa_c=q["kappa_c"] + e)),
                      ("m_scale", lambda q, e: dict(q, MA_bulk=q["MA_bulk"] * (1 + e), MB_bulk=q["MB_bulk"] * (1 + e)))):
        e = 1e-5
        fd = (loss(pert(p, e), st64) - loss(pert(p, -e), st64)) / (2 * e)
        assert res[key] == pytest.approx(fd, rel=1e-3), (key, res[key], fd)
    g = res["c0"][:, :nx].cpu().numpy()
    for (j, i) in ((9, 10), (6, 33), (0, 5)):
        e = 1e-6
        up = [a.copy() for a in st64]
        dn = [a.copy() for a in st64]
        up[1][j, i] += e
        dn[1][j, i] -= e
        fd = (loss(p, up) - loss(p, dn)) / (2 * e)
        assert g[j, i] == pytest.approx(fd, rel=1e-3, abs=1e-3 * np.abs(g).max()), (j, i, g[j, i], fd)


def test_autograd_function_gives_the_adjoint_gradients(pf):
    p, st, w = case(nx=40, ny=24)
    ny, nx = st[0].shape
    PFRun = pf.make_run_function()
    v = torch.tensor(p["v_mag"], dtype=torch.float64, requires_grad=True)
    m = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    kc = torch.tensor(p["kappa_c"], dtype=torch.float64, requires_grad=True)
    init = [t.requires_grad_(True) for t in pf.device_fields(st)]
    out = PFRun.apply(v, m, kc, *init, p, nx, 25, 10)
    wt = pf.device_fields(w)
    L = sum((o * x).sum() for o, x in zip(out, wt))
    L.backward()
    res = pf.adjoint(p, pf.device_fields(st), nx, 25, 10, *wt)
    assert float(v.grad) == pytest.approx(res["v_mag"], rel=1e-12)
    assert float(m.grad) == pytest.approx(res["m_scale"], rel=1e-12)
    assert float(kc.grad) == pytest.approx(res["kappa_c"], rel=1e-12)
    assert torch.equal(init[1].grad, res["c0"])


def test_autograd_forward_binds_the_device_tensors(pf, monkeypatch):
    """The forward copies the given CUDA tensors device to device: with host copies of tensors made
    impossible it still runs, and its final state equals a run started from host arrays bit for bit."""
    p, st, _ = case(nx=40, ny=24)
    ny, nx = st[0].shape
    PFRun = pf.make_run_function()
    init = pf.device_fields(st)

    def no_host_copy(*a, **k):
        raise AssertionError("device-to-host copy in the forward")

    monkeypatch.setattr(torch.Tensor, "cpu", no_host_copy)
    monkeypatch.setattr(torch.Tensor, "numpy", no_host_copy)
    v = torch.tensor(p["v_mag"], dtype=torch.float64)
    out = PFRun.apply(v, torch.tensor(1.0, dtype=torch.float64), torch.tensor(p["kappa_c"], dtype=torch.float64),
                      *init, p, nx, 25, 10)
    monkeypatch.undo()
    sim = pf.Sim(p, *st, history_rows=1)
    sim.step(25)
    for a, b in zip(out, sim.fields):
        assert torch.equal(a[:, :nx], b[:, :nx])
    sim.close()
