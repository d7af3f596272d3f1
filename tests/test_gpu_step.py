"""GPU parity of the fused step against the FP64 oracle, through the C ABI.

Tolerances are the project's targets: max-abs 1e-5 after 100 steps and 1e-4
after 2000 steps on every field (FP32 state against FP64; the spinodal growth
of the composition amplifies round-off by about e^{t/8}).
"""
import numpy as np
import pytest

import oracle as O
from paper_2312_05410_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf(cuda_ok):
    from paper_2312_05410_gb300 import build as B
    B.build()
    from paper_2312_05410_gb300 import pf as mod
    return mod


def run_gpu(pf, params, state, steps, history_rows=64):
    sim = pf.Sim(params, *state, history_rows=history_rows)
    sim.step(steps)
    out = sim.numpy()
    hist = sim.history()
    sim.close()
    return out, hist


def max_err(a, b):
    return max(float(np.abs(x.astype(np.float64) - y).max()) for x, y in zip(a, b))


def test_small_film_100_and_2000_steps(pf):
    cfg = I.SMALL_64
    p = O.with_dt(I.default_params(**cfg["params"]))
    state = I.film_state(cfg["spec"], p)
    ref100 = O.step(p, *state, 100)
    ref2000 = O.step(p, *ref100, 1900)
    g100, _ = run_gpu(pf, p, state, 100)
    g2000, _ = run_gpu(pf, p, state, 2000)
    e100, e2000 = max_err(g100, ref100), max_err(g2000, ref2000)
    assert e100 <= 1e-5, e100
    assert e2000 <= 1e-4, e2000
    # the run did something: the film grew and the composition coarsened
    assert ref2000[0].sum() > state[0].astype(np.float64).sum() + 10


@pytest.mark.parametrize("nx,ny", [(37, 23), (65, 64), (130, 70), (64, 33), (1, 5), (3, 2), (200, 9), (511, 513)])
def test_odd_and_ragged_sizes(pf, nx, ny):
    p = O.with_dt(I.default_params(v_angle_deg=65.0))
    state = I.film_state(I.FilmSpec(nx, ny, ny / 3.0, seed=nx * 1000 + ny), p)
    ref = O.step(p, *state, 100)
    got, _ = run_gpu(pf, p, state, 100)
    assert max_err(got, ref) <= 1e-5


@pytest.mark.parametrize("over", [
    dict(phi_mode=1),
    dict(MA_bulk=2.0, MB_bulk=0.5),
    dict(MA_bulk=2.0, MB_bulk=0.5, MA_surf=10.0, MB_surf=4.0, sigma_surf=0.5),
    dict(v_angle_deg=50.0, v_mag=1.0),
    dict(deposition=0),
    dict(dx=0.7, kappa_c=1.5, W_c=1.2, rho_top=0.8),
])
def test_model_variants(pf, over):
    p = O.with_dt(I.default_params(**over))
    state = I.film_state(I.FilmSpec(96, 80, 20.0, seed=7), p)
    ref = O.step(p, *state, 100)
    got, _ = run_gpu(pf, p, state, 100)
    assert max_err(got, ref) <= 1e-5


def test_rough_random_fields(pf):
    p = O.with_dt(I.default_params(v_angle_deg=70.0))
    state = I.random_state(72, 40, seed=21)
    ref = O.step(p, *state, 20)
    got, _ = run_gpu(pf, p, state, 20)
    assert max_err(got, ref) <= 1e-5


def test_tma_staged_small_tiles_match_oracle(pf):
    """Grids up to 2^20 cells use the 56 x 8 tile; interior tiles are TMA-staged once the grid has one
    (nx >= 116, ny >= 20).  Ragged sizes mix both staging paths."""
    p = O.with_dt(I.default_params(v_angle_deg=70.0))
    for nx, ny in ((116, 20), (130, 70), (200, 64)):
        state = I.film_state(I.FilmSpec(nx, ny, ny / 3.0, seed=nx + ny), p)
        got, _ = run_gpu(pf, p, state, 100)
        assert max_err(got, O.step(p, *state, 100)) <= 1e-5, (nx, ny)


def test_tma_staged_large_grid_matches_oracle(pf):
    """A grid above 2^20 cells (56 x 24 tiles, interior tiles staged by TMA, boundary tiles by
    per-thread copies with ghost rows) against the oracle."""
    p = O.with_dt(I.default_params(v_angle_deg=75.0))
    state = I.film_state(I.FilmSpec(1100, 1000, 40.0, seed=12), p)
    ref = O.step(p, *state, 12)
    got, _ = run_gpu(pf, p, state, 12)
    assert max_err(got, ref) <= 1e-5


def test_paper_scale_grid_graph_path(pf):
    """512 x 512, the benchmark's kernel and graph replay (diagnostics every 100 steps)."""
    cfg = I.PAPER_512
    p = O.with_dt(I.default_params(**dict(cfg["params"], diag_every=100)))
    state = I.film_state(cfg["spec"], p)
    ref = O.step(p, *state, 200)
    got, hist = run_gpu(pf, p, state, 200)
    assert max_err(got, ref) <= 1e-5
    # history: records of the states at steps 0 and 100
    assert hist.shape == (2, 5)
    assert list(hist[:, 0]) == [0.0, 100.0]
    d0 = O.diag(p, *state)
    d100 = O.diag(p, *O.step(p, *state, 100))
    np.testing.assert_allclose(hist[0, 1:], d0, rtol=2e-6)
    np.testing.assert_allclose(hist[1, 1:], d100, rtol=2e-6)


def test_diag_matches_oracle(pf):
    p = O.with_dt(I.default_params(kappa_c=1.7, W_phi=0.8, dx=0.9))
    state = I.film_state(I.FilmSpec(100, 60, 15.0, seed=3), p)
    sim = pf.Sim(p, *state)
    got = sim.diag()
    sim.close()
    np.testing.assert_allclose(got, O.diag(p, *state), rtol=1e-6)


def test_composition_conserved_long_run(pf):
    """sum(c) has no source and no boundary flux: FP32 drift stays tiny over 20000 steps."""
    cfg = I.PAPER_512
    p = O.with_dt(I.default_params(**dict(cfg["params"], diag_every=1000)))
    state = I.film_state(cfg["spec"], p)
    sim = pf.Sim(p, *state)
    d0 = sim.diag()
    sim.step(20000)
    d1 = sim.diag()
    hist = sim.history()
    sim.close()
    assert abs(d1[0] - d0[0]) <= 2e-5 * abs(d0[0]), (d0, d1)
    assert d1[1] > d0[1]  # film grew
    assert np.all(np.isfinite(hist))
    assert hist.shape[0] == 20


def test_tma_staging_is_used_where_tiles_fit(pf):
    p = O.with_dt(I.default_params())
    for (nx, ny), mode in (((2048, 1024), 1), ((1120, 960), 1), ((512, 512), 1), ((116, 20), 1), ((115, 40), 0),
                           ((200, 19), 0), ((64, 64), 0), ((37, 23), 0)):
        sim = pf.Sim(p, *I.film_state(I.FilmSpec(nx, ny, ny / 3.0, seed=1), p))
        assert pf.pf_staging_mode(sim.h) == mode, (nx, ny)
        sim.close()


def test_runs_are_bitwise_deterministic(pf):
    p = O.with_dt(I.default_params())
    state = I.film_state(I.FilmSpec(128, 96, 12.0, seed=5), p)
    a, _ = run_gpu(pf, p, state, 300)
    b, _ = run_gpu(pf, p, state, 300)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_resume_from_checkpoint_is_bitwise(pf):
    p = O.with_dt(I.default_params(diag_every=100))
    state = I.film_state(I.FilmSpec(96, 96, 12.0, seed=6), p)
    full, hfull = run_gpu(pf, p, state, 1000)
    sim = pf.Sim(p, *state)
    sim.step(500)
    ckpt = sim.numpy()
    sim.close()
    sim = pf.Sim(p, *ckpt)
    sim.set_step(500)
    sim.step(500)
    resumed = sim.numpy()
    hres = sim.history()
    sim.close()
    for x, y in zip(full, resumed):
        assert np.array_equal(x, y)
    np.testing.assert_array_equal(hres, hfull[5:])


def test_step_counts_odd_and_zero(pf):
    p = O.with_dt(I.default_params())
    state = I.film_state(I.FilmSpec(64, 64, 8.0, seed=0), p)
    sim = pf.Sim(p, *state)
    sim.step(0)
    assert all(np.array_equal(a, b) for a, b in zip(sim.numpy(), state))
    sim.step(7)
    sim.step(6)
    got = sim.numpy()
    assert sim.step_index == 13
    sim.close()
    assert max_err(got, O.step(p, *state, 13)) <= 1e-5


def test_nonfinite_is_reported(pf):
    p = O.with_dt(I.default_params())
    phi, c, rho = I.film_state(I.FilmSpec(64, 64, 8.0, seed=0), p)
    c = c.copy()
    c[10, 10] = np.nan
    sim = pf.Sim(p, phi, c, rho)
    sim.step(3)
    rc, _ = pf.pf_diag(sim.h)
    assert rc == pf.PF_ERR_NONFINITE
    assert pf.pf_clear_error(sim.h) == 0
    sim.close()


@pytest.mark.parametrize("loop", [1, 0])
def test_staging_wait_timeout_is_reported_and_recoverable(pf, loop):
    """A bounded TMA wait that runs out (limit of zero polls) sets the error word; pf_diag reports
    PF_ERR_TIMEOUT, the context stays usable, and with the default limit the run is correct again.
    Both the persistent tile loop (loop = 1) and one CTA per tile (loop = 0)."""
    p = O.with_dt(I.default_params())
    state = I.film_state(I.FilmSpec(1120, 960, 16.0, seed=4), p)  # above 2^20 cells: TMA-staged tiles
    sim = pf.Sim(p, *state)
    assert pf.pf_staging_mode(sim.h) == 1
    assert pf.pf_set_tile_loop(sim.h, loop) == 0
    assert pf.pf_set_wait_limit(sim.h, 0) == 0
    sim.step(1)
    rc, _ = pf.pf_diag(sim.h)
    assert rc == pf.PF_ERR_TIMEOUT
    sim.close()
    sim = pf.Sim(p, *state)
    assert pf.pf_set_wait_limit(sim.h, 1 << 22) == 0
    assert pf.pf_clear_error(sim.h) == 0
    sim.step(10)
    rc, _ = pf.pf_diag(sim.h)
    assert rc == 0
    got = sim.numpy()
    sim.close()
    assert max_err(got, O.step(p, *state, 10)) <= 1e-5


@pytest.mark.parametrize("nx,ny", [(1100, 1000), (1101, 960), (1456, 744)])
def test_tile_loop_equals_one_cta_per_tile_bitwise(pf, nx, ny):
    """The persistent tile loop (next tile staged while one computes; TMA for interior tiles, cp.async or,
    for nx % 4 != 0, plain loads for the rest) runs the same per-tile arithmetic as one CTA per tile:
    identical fields after 603 steps, through single launches and graph replays alike."""
    p = O.with_dt(I.default_params(v_angle_deg=80.0))
    state = I.film_state(I.FilmSpec(nx, ny, 30.0, seed=nx + ny), p)
    out = []
    for loop in (1, 0):
        sim = pf.Sim(p, *state, history_rows=1)
        assert pf.pf_set_tile_loop(sim.h, loop) == 0
        sim.step(3)
        sim.step(600)
        out.append(sim.numpy())
        sim.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("nx,ny,diag_every,steps", [(64, 64, 0, 1001), (37, 23, 0, 37), (512, 512, 1000, 2000),
                                                     (130, 70, 10, 251), (1, 5, 0, 7), (200, 9, 7, 60),
                                                     (116, 40, 4, 130), (1000, 1000, 0, 515)])
def test_two_steps_per_launch_equal_one_bitwise(pf, nx, ny, diag_every, steps):
    """Two explicit midpoint steps per launch (u^{n+1} kept in shared memory) against one step per launch:
    identical fields and diagnostic history, for ragged sizes, graph replays, odd step counts and even and
    odd diagnostic periods (where a record would fall between two steps, single steps are taken)."""
    p = O.with_dt(I.default_params(v_angle_deg=70.0, diag_every=diag_every))
    state = I.film_state(I.FilmSpec(nx, ny, max(2.0, ny / 3.0), seed=nx * 7 + ny), p)
    out = []
    for spl in (2, 1):
        sim = pf.Sim(p, *state, history_rows=8)
        assert pf.pf_set_steps_per_launch(sim.h, spl) == 1
        sim.step(3)
        sim.step(steps - 3)
        out.append((sim.numpy(), sim.history()))
        sim.close()
    (a, ha), (b, hb) = out
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    np.testing.assert_array_equal(ha, hb)


def test_two_step_wait_timeout_is_reported(pf):
    """The two-step kernel's bounded TMA wait (512^2: interior tiles are TMA-staged) run out: PF_ERR_TIMEOUT."""
    p = O.with_dt(I.default_params())
    state = I.film_state(I.FilmSpec(512, 512, 16.0, seed=1), p)
    sim = pf.Sim(p, *state, history_rows=1)
    assert pf.pf_set_steps_per_launch(sim.h, 2) == 1
    assert pf.pf_set_wait_limit(sim.h, 0) == 0
    sim.step(2)
    rc, _ = pf.pf_diag(sim.h)
    assert rc == pf.PF_ERR_TIMEOUT
    sim.close()
    assert pf.pf_set_steps_per_launch(None, 2) == pf.PF_ERR_ARG


def test_tile_loop_is_refused_on_small_grids(pf):
    p = O.with_dt(I.default_params())
    sim = pf.Sim(p, *I.film_state(I.FilmSpec(512, 512, 16.0, seed=1), p), history_rows=1)
    assert pf.pf_set_tile_loop(sim.h, 1) == pf.PF_ERR_ARG
    sim.close()


def test_host_buffer_load_step_store(pf):
    """pf_load_host / pf_step / pf_store_host with pinned host arrays: the same state as the device path,
    bit for bit, and nothing outside the nx model columns of the host rows is touched."""
    import torch

    p = O.with_dt(I.default_params(v_angle_deg=60.0))
    st = I.film_state(I.FilmSpec(150, 70, 20.0, seed=31), p)
    other = I.film_state(I.FilmSpec(150, 70, 10.0, seed=32), p)
    sim = pf.Sim(p, *other, history_rows=1)        # a different state, overwritten by the load
    host_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in st]
    host_out = [torch.full((70, 152), 7.0).pin_memory() for _ in range(3)]
    sim.load_host(*host_in)
    sim.step(40)
    ptrs = [int(t.data_ptr()) for t in host_out]
    assert pf.lib.pf_store_host(sim.h, *ptrs, 152) == 0
    sim.stream.synchronize()
    sim.close()
    ref = pf.Sim(p, *st, history_rows=1)
    ref.step(40)
    want = ref.numpy()
    ref.close()
    for h, w in zip(host_out, want):
        a = h.numpy()
        assert np.array_equal(a[:, :150], w)
        assert np.all(a[:, 150:] == 7.0)
    assert pf.lib.pf_load_host(None, None, None, None, 150) == pf.PF_ERR_ARG


@pytest.mark.parametrize("nx,ny,spl,loop", [(37, 23, 1, 0), (511, 513, 1, 0), (511, 513, 2, 0), (130, 70, 2, 0),
                                            (1100, 1000, 1, 0), (1100, 1000, 1, 1), (1101, 960, 1, 1),
                                            (1101, 960, 1, 0)])
def test_guard_bands_stay_untouched(pf, nx, ny, spl, loop):
    """Out-of-bounds writes would land in canaries: the caller's fields sit inside buffers with 8 canary rows
    above and below and canary columns from nx to the padded pitch (and the workspace has a canary tail).
    After steps through the chosen kernel path, every canary still holds its value and the state equals
    the one of plain fields."""
    import torch

    G, CAN = 8, -12345.5
    p = O.with_dt(I.default_params(v_angle_deg=70.0, diag_every=10))
    st = I.film_state(I.FilmSpec(nx, ny, max(2.0, ny / 3.0), seed=nx + 3 * ny), p)
    pitch = pf.padded_pitch(nx)
    bufs = []
    for a in st:
        t = torch.full((ny + 2 * G, pitch), CAN, dtype=torch.float32, device="cuda")
        t[G:G + ny, :nx] = torch.from_numpy(a).cuda()
        bufs.append(t)
    need = pf.pf_workspace_size(nx, ny, pitch, 8)
    work = torch.full((need + 256 + 4096,), 0x5A, dtype=torch.uint8, device="cuda")
    wp = (work.data_ptr() + 255) // 256 * 256
    tail = work[wp - work.data_ptr() + need:].clone()
    stream = torch.cuda.current_stream().cuda_stream
    rc, h = pf.pf_init(p, nx, ny, pitch, *(t[G:].data_ptr() for t in bufs), wp, need, 8, stream)
    assert rc == 0, pf.last_error()
    if spl == 2:
        assert pf.pf_set_steps_per_launch(h, 2) == 1
    if loop:
        assert pf.pf_set_tile_loop(h, 1) == 0
    assert pf.pf_step(h, 3) == 0 and pf.pf_step(h, 40) == 0
    torch.cuda.synchronize()
    assert pf.pf_destroy(h) == 0
    for t in bufs:
        assert torch.all(t[:G] == CAN) and torch.all(t[G + ny:] == CAN)
        assert torch.all(t[G:G + ny, nx:] == CAN)
    assert torch.equal(work[wp - work.data_ptr() + need:], tail)
    ref = pf.Sim(p, *st, history_rows=8)
    ref.step(43)
    for t, w in zip(bufs, ref.numpy()):
        assert np.array_equal(t[G:G + ny, :nx].cpu().numpy(), w)
    ref.close()


def test_standalone_diagnostics_entry_point(pf):
    import torch

    p = O.with_dt(I.default_params())
    state = I.film_state(I.FilmSpec(80, 50, 10.0, seed=2), p)
    sim = pf.Sim(p, *state)
    ws = torch.zeros(pf.pf_diag_workspace_size(80, 50) + 256, dtype=torch.uint8, device="cuda")
    wp = (ws.data_ptr() + 255) // 256 * 256
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = pf.pf_diagnostics(p, 80, 50, sim.pitch, sim.phi.data_ptr(), sim.c.data_ptr(), sim.rho.data_ptr(), wp,
                           pf.pf_diag_workspace_size(80, 50), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), sim.diag(), rtol=1e-12)
    sim.close()
