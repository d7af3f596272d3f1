"""Batched ensemble of uneven runs (one launch per step for all runs) through the C ABI.

The per-cell arithmetic of the fused step does not depend on which tile or
which launch computes a cell, so every run of an ensemble must match the
single-run path bit for bit, for every tile shape; small runs are also
checked against the FP64 oracle.
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


SHAPES = [(128, 128), (192, 128), (64, 96), (37, 23), (256, 64), (112, 56)]


def members(shapes=SHAPES, seed=11):
    out = []
    u = I.uniform01(seed, 5, 2 * len(shapes)).reshape(len(shapes), 2)
    for k, (nx, ny) in enumerate(shapes):
        v = 0.1 + 0.8 * u[k, 0]
        ci = 0.3 + 0.4 * u[k, 1]
        p = O.with_dt(I.default_params(v_mag=float(v), v_angle_deg=60.0 + 5 * k))
        st = I.film_state(I.FilmSpec(nx, ny, max(2.0, ny / 5.0), seed=seed * 100 + k, c_inc=float(ci)), p)
        out.append((p, *st))
    return out


def single(pf, m, steps):
    sim = pf.Sim(m[0], *m[1:])
    sim.step(steps)
    out = sim.numpy()
    sim.close()
    return out


@pytest.mark.parametrize("steps", [37, 250])
def test_every_run_matches_the_single_run_path_bitwise(pf, steps):
    ms = members()
    ens = pf.Ensemble(ms)
    ens.step(steps)
    assert ens.step_index == steps
    for r, m in enumerate(ms):
        got = ens.numpy(r)
        ref = single(pf, m, steps)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), r
    ens.close()


TMA_SHAPES = [(128, 128), (192, 128), (64, 96), (37, 23), (256, 64), (112, 56), (300, 40), (150, 70), (132, 200)]


@pytest.mark.parametrize("tile", [0, 1])
def test_tma_staging_equals_per_thread_staging_bitwise(pf, tile):
    """Tile kinds 0 and 1 stage every tile that lies inside its run's grid in x by TMA (every run's maps
    travel with the launch), the bottom and top tiles included: their rows outside the domain arrive as
    zeros and get the ghost values in shared memory.  Per-thread staging of every tile must give the same
    states bit for bit.  The runs include widths that are not multiples of 56 or of 4, grids narrower
    than a window (per-thread only) and grids shorter than the large tile's window."""
    ms = members(TMA_SHAPES, seed=16)
    out = []
    for tma in (True, False):
        ens = pf.Ensemble(ms)
        ens.set_tile(tile)
        ens.set_tma(tma)
        assert ens.staging_mode == (1 if tma else 0)
        ens.step(37)
        out.append([ens.numpy(r) for r in range(len(ms))])
        ens.close()
    for r, (ra, rb) in enumerate(zip(*out)):
        for a, b in zip(ra, rb):
            assert np.array_equal(a, b), r


def test_single_runs_with_tma_edges_equal_per_thread_staging(pf):
    """A single run TMA-stages its bottom and top tiles too; against the ensemble with per-thread staging
    of every tile (the same per-cell arithmetic), bit for bit after 250 steps."""
    ms = members([(128, 128), (256, 64), (300, 40), (132, 200)], seed=18)
    ens = pf.Ensemble(ms)
    ens.set_tma(False)
    ens.step(250)
    for r, m in enumerate(ms):
        sim = pf.Sim(m[0], *m[1:])
        assert pf.pf_staging_mode(sim.h) == 1
        sim.step(250)
        ref = sim.numpy()
        sim.close()
        for a, b in zip(ens.numpy(r), ref):
            assert np.array_equal(a, b), r
    ens.close()


def test_tma_staging_timeout_is_reported(pf):
    """A TMA staging wait limited to zero polls runs out; the CTA lets its copies land and leaves,
    pf_ens_diag reports PF_ERR_TIMEOUT, and the context stays usable."""
    ms = members([(256, 256), (192, 128)], seed=17)
    ens = pf.Ensemble(ms)
    ens.set_tile(1)
    assert ens.staging_mode == 1
    ens.set_wait_limit(0)
    ens.step(3)
    with pytest.raises(pf.PFError) as e:
        ens.diag(0)
    assert e.value.code == pf.PF_ERR_TIMEOUT
    ens.close()
    ok = pf.Ensemble(ms)
    ok.set_tile(1)
    ok.step(3)
    ok.diag(0)
    ok.close()


def test_tile_shapes_give_identical_results(pf):
    ms = members(SHAPES[:4])
    results = []
    for tile in (0, 1, 2, 3):
        ens = pf.Ensemble(ms)
        ens.set_tile(tile)
        ens.step(24)
        results.append([ens.numpy(r) for r in range(len(ms))])
        ens.close()
    for other in results[1:]:
        for ra, rb in zip(results[0], other):
            for a, b in zip(ra, rb):
                assert np.array_equal(a, b)


@pytest.mark.parametrize("steps", [1, 37, 250])
def test_persistent_launch_equals_one_launch_per_step_bitwise(pf, steps):
    """Tile kind 4: every run advanced by one cooperative launch per chunk of up to 100 steps (graph
    replays of such launches for the full chunks), with a bounded grid barrier between steps, against one
    launch per step (kind 0), bit for bit."""
    ms = members([(128, 128), (192, 128), (64, 96), (256, 64), (112, 56)], seed=13)
    out = []
    for tile in (4, 0):
        ens = pf.Ensemble(ms)
        ens.set_tile(tile)
        ens.step(steps)
        out.append([ens.numpy(r) for r in range(len(ms))])
        assert ens.step_index == steps
        ens.close()
    for ra, rb in zip(*out):
        for a, b in zip(ra, rb):
            assert np.array_equal(a, b)


def test_persistent_launch_needs_widths_in_multiples_of_four(pf):
    ens = pf.Ensemble(members([(128, 128), (37, 23)], seed=14))
    with pytest.raises(pf.PFError) as e:
        ens.set_tile(4)
    assert e.value.code == pf.PF_ERR_ARG
    chosen, secs = ens.autotune(2)
    assert chosen != 4 and secs[4] == 0.0
    ens.close()


def test_persistent_barrier_timeout_is_reported(pf):
    """A grid-barrier wait limited to zero polls runs out on the CTAs that arrive early; pf_ens_diag reports
    PF_ERR_TIMEOUT and the context stays usable."""
    ms = members([(256, 256), (192, 128)], seed=15)
    ens = pf.Ensemble(ms)
    ens.set_tile(4)
    ens.set_wait_limit(0)
    ens.step(3)
    with pytest.raises(pf.PFError) as e:
        ens.diag(0)
    assert e.value.code == pf.PF_ERR_TIMEOUT
    ens.close()
    ok = pf.Ensemble(ms)
    ok.set_tile(4)
    ok.step(3)
    ok.diag(0)
    ok.close()


def test_small_runs_match_the_oracle(pf):
    ms = members([(48, 40), (37, 23), (96, 32)], seed=3)
    ens = pf.Ensemble(ms)
    ens.step(100)
    for r, m in enumerate(ms):
        ref = O.step(m[0], *m[1:], 100)
        got = ens.numpy(r)
        err = max(float(np.abs(a.astype(np.float64) - b).max()) for a, b in zip(got, ref))
        assert err <= 1e-5, (r, err)
        np.testing.assert_allclose(ens.diag(r), O.diag(m[0], *ref), rtol=1e-5)
    ens.close()


def test_autotune_picks_a_tile_and_keeps_stepping_the_runs(pf):
    ms = members(SHAPES[:3])
    ens = pf.Ensemble(ms)
    chosen, secs = ens.autotune(4)
    assert chosen in (0, 1, 2, 3, 4) and ens.tile == chosen
    assert len(secs) == 5 and all(s > 0 for s in secs)
    assert ens.step_index == 5 * (4 + 2)
    ens.step(2)
    for r, m in enumerate(ms):
        for a, b in zip(ens.numpy(r), single(pf, m, 5 * 6 + 2)):
            assert np.array_equal(a, b)
    ens.close()


def test_mixed_mobility_forms_are_rejected(pf):
    ms = members(SHAPES[:2])
    p2 = dict(ms[1][0], MA_bulk=2.0)
    with pytest.raises(pf.PFError) as e:
        pf.Ensemble([ms[0], (p2, *ms[1][1:])])
    assert e.value.code == pf.PF_ERR_ARG
