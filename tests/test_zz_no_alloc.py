"""pf_diagnostics_static: the diagnostics entry point for callers that cannot
allocate device memory themselves (a plug-in whose host application owns all
device memory through its own pool, or a latency-critical loop where
cudaMalloc/cudaFree would synchronise the device).  It keeps its reduction
scratch in a static device array instead of a caller workspace.

Checked here through the C ABI: two calls in a row give the same sums as
pf_diagnostics (the workspace-taking entry point), and its NaN flag is cleared
between calls.  This file is collected last on purpose.
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


def _fields(pf, nx, ny, seed, nan=False):
    import torch

    p = O.with_dt(I.default_params())
    phi, c, rho = I.film_state(I.FilmSpec(nx, ny, ny / 4.0, seed=seed), p)
    if nan:
        c = c.copy()
        c[ny // 2, nx // 3] = np.nan
    pitch = pf.padded_pitch(nx)
    ts = []
    for a in (phi, c, rho):
        t = torch.zeros((ny, pitch), dtype=torch.float32, device="cuda")
        t[:, :nx] = torch.from_numpy(a).cuda()
        ts.append(t)
    return p, pitch, ts


def _with_workspace(pf, p, nx, ny, pitch, ts, stream):
    import torch

    need = pf.pf_diag_workspace_size(nx, ny)
    ws = torch.zeros(need + 256, dtype=torch.uint8, device="cuda")
    wp = (ws.data_ptr() + 255) // 256 * 256
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = pf.pf_diagnostics(p, nx, ny, pitch, *(t.data_ptr() for t in ts), wp, need, out.data_ptr(), stream)
    assert rc == 0
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _static(pf, p, nx, ny, pitch, ts, stream):
    import torch

    out = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    err = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    rc = pf.pf_diagnostics_static(p, nx, ny, pitch, *(t.data_ptr() for t in ts), out.data_ptr(), err.data_ptr(),
                                  stream)
    assert rc == 0, pf.strerror(rc)
    torch.cuda.synchronize()
    return out.cpu().numpy(), int(err.item())


@pytest.mark.parametrize("nx,ny", [(512, 512), (37, 23), (2048, 1024)])
def test_static_scratch_matches_workspace_entry_point(pf, nx, ny):
    import torch

    stream = torch.cuda.current_stream().cuda_stream
    p, pitch, ts = _fields(pf, nx, ny, seed=nx + ny)
    ref = _with_workspace(pf, p, nx, ny, pitch, ts, stream)
    for _ in range(2):  # two calls in a row share the static scratch
        got, err = _static(pf, p, nx, ny, pitch, ts, stream)
        np.testing.assert_allclose(got, ref, rtol=1e-12)
        assert err == 0


def test_static_scratch_capacity_is_the_reduction_block_cap(pf):
    """The static array holds the partials of the most reduction blocks any accepted grid uses
    (1216, documented in pf.h): the workspace entry point's size stops growing there, and
    2048 x 1024 (run above) already reaches it."""
    cap = 1216
    full = (4 * 8 * cap + 255) // 256 * 256 + 256
    assert pf.pf_diag_workspace_size(2048, 1024) == full
    assert pf.pf_diag_workspace_size(1 << 20, 1 << 20) == full
    assert pf.pf_diag_workspace_size(1024, 1024) < full


def test_static_scratch_error_word_is_cleared_between_calls(pf):
    import torch

    stream = torch.cuda.current_stream().cuda_stream
    p, pitch, bad = _fields(pf, 64, 48, seed=1, nan=True)
    _, err = _static(pf, p, 64, 48, pitch, bad, stream)
    assert err == 1
    p, pitch, good = _fields(pf, 64, 48, seed=1)
    got, err = _static(pf, p, 64, 48, pitch, good, stream)
    assert err == 0
    np.testing.assert_allclose(got, _with_workspace(pf, p, 64, 48, pitch, good, stream), rtol=1e-12)


def test_static_entry_point_rejects_bad_sizes(pf):
    p = I.default_params()
    fake = 1 << 20
    assert pf.pf_diagnostics_static(p, 0, 8, 32, fake, fake, fake, fake, None, 0) == pf.PF_ERR_ARG
    assert pf.pf_diagnostics_static(p, (1 << 20) + 4, 8, (1 << 20) + 4, fake, fake, fake, fake, None, 0) \
        == pf.PF_ERR_ARG
    assert pf.pf_diagnostics_static(p, 40, 8, 42, fake, fake, fake, fake, None, 0) == pf.PF_ERR_LAYOUT
    assert pf.pf_diagnostics_static(p, 40, 8, 40, fake, fake, fake, fake + 4, None, 0) == pf.PF_ERR_LAYOUT
    assert "8-byte aligned" in pf.last_error()
    assert pf.pf_diagnostics_static(p, 40, 8, 42, fake, fake, fake, fake, None, 0) == pf.PF_ERR_LAYOUT
    assert "pitch" in pf.last_error()
