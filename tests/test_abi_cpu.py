"""C-ABI checks that need no GPU: exported symbols, the host-side stability
limit against the oracle's, and every argument/layout/stability error path of
pf_init and pf_diagnostics (they return before any CUDA call)."""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2312_05410_gb300 import build as B
from paper_2312_05410_gb300 import inputs as I


@pytest.fixture(scope="module")
def pf():
    B.build()
    from paper_2312_05410_gb300 import pf as mod
    return mod


def declared_symbols():
    text = open(os.path.join(B.INCLUDE, "pf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pf_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(pf):
    names = declared_symbols()
    assert len(names) >= 15, names
    for n in names:
        assert hasattr(pf.lib, n), n


def test_binding_declares_the_argument_types_of_every_entry_point(pf):
    """ctypes passes undeclared arguments as C ints: a pointer, size_t, long or double argument would be
    truncated or mis-passed.  Every entry point the header declares has its argument types set."""
    import ctypes as C

    missing = [s for s in declared_symbols() if getattr(pf.lib, s).argtypes is None]
    assert not missing, missing
    # entry points that return something other than an int declare it (return types read from the header)
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(B.INCLUDE, "pf.h")).read(), flags=re.S)
    kinds = {"size_t": C.c_size_t, "long": C.c_long, "const char*": C.c_char_p}
    wide = {}
    for ret, name in re.findall(r"^(size_t|long|const char\*)\s+(pf_[a-z_0-9]+)\s*\(", text, flags=re.M):
        wide[name] = kinds[ret]
    assert len(wide) >= 10, wide
    for name, rt in wide.items():
        assert getattr(pf.lib, name).restype is rt, name


def test_ctypes_struct_mirrors_match_the_c_layout(pf, tmp_path):
    """The binding's mirrors of pf_params, pf_hybrid_params and pf_hybrid_stats have the C structs' size and
    field offsets: a small C program compiled against include/pf.h prints them."""
    import ctypes as C
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"pf_params": pf.Params, "pf_hybrid_params": pf.HybridParams, "pf_hybrid_stats": pf.HybridStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pf.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'    printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c11", "-I", B.INCLUDE, "-o", str(exe), str(src)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        cname, key, val = line.split()
        got[(cname, key)] = int(val)
    assert len(got) == sum(1 + len(py._fields_) for py in mirrors.values())
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)


def test_strerror(pf):
    assert pf.strerror(0) == "ok"
    assert "stability" in pf.strerror(pf.PF_ERR_UNSTABLE)
    assert pf.strerror(-99) == "unknown error"


@pytest.mark.parametrize("over", [
    {}, dict(phi_mode=1), dict(v_angle_deg=55.0, v_mag=0.9, D_rho=0.3), dict(MA_surf=10.0, MB_surf=3.0, MA_bulk=2.0),
    dict(deposition=0, dx=0.5), dict(D_rho=0.05, v_mag=1.0, v_angle_deg=50.0), dict(kappa_c=8.0, W_c=3.0),
])
def test_dt_limit_matches_oracle(pf, over):
    p = I.default_params(**over)
    got = pf.pf_dt_limit(p)
    ref = O.dt_limit(p)
    np.testing.assert_allclose(got, [ref["dt_lim"], ref["dt_c"], ref["dt_phi"], ref["dt_rho"]], rtol=1e-12)


FAKE = 1 << 20  # aligned non-null address; never dereferenced on these paths


def _init(pf, p, nx=64, ny=64, pitch=64, ptrs=(FAKE, FAKE, FAKE), work=FAKE, work_bytes=None, hist=4):
    if work_bytes is None:
        work_bytes = pf.pf_workspace_size(nx, ny, max(pitch, 1), hist) or 1 << 30
    rc, h = pf.pf_init(p, nx, ny, pitch, *ptrs, work, work_bytes, hist, 0)
    return rc


def test_init_error_paths(pf):
    good = O.with_dt(I.default_params())
    assert _init(pf, good, nx=0) == pf.PF_ERR_ARG
    assert _init(pf, good, ny=0) == pf.PF_ERR_ARG
    assert _init(pf, good, pitch=66) == pf.PF_ERR_LAYOUT
    assert _init(pf, good, pitch=60) == pf.PF_ERR_LAYOUT
    assert _init(pf, good, ptrs=(FAKE + 4, FAKE, FAKE)) == pf.PF_ERR_LAYOUT
    assert _init(pf, good, ptrs=(0, FAKE, FAKE)) == pf.PF_ERR_ARG
    assert _init(pf, good, work=FAKE + 64) == pf.PF_ERR_LAYOUT
    assert _init(pf, good, work_bytes=1024) == pf.PF_ERR_LAYOUT
    assert _init(pf, dict(good, phi_mode=2)) == pf.PF_ERR_ARG
    assert _init(pf, dict(good, dt=0.0)) == pf.PF_ERR_ARG
    assert _init(pf, dict(good, W_c=float("nan"))) == pf.PF_ERR_ARG
    assert _init(pf, dict(good, MA_surf=1.0, sigma_surf=0.0)) == pf.PF_ERR_ARG
    assert _init(pf, good, hist=-1) == pf.PF_ERR_ARG
    lim = pf.pf_dt_limit(good)[0]
    rc = _init(pf, dict(good, dt=1.01 * lim))
    assert rc == pf.PF_ERR_UNSTABLE
    assert "stability limit" in pf.last_error()


def test_workspace_size(pf):
    assert pf.pf_workspace_size(0, 4, 32, 1) == 0
    assert pf.pf_workspace_size(40, 4, 32, 1) == 0  # pitch < nx
    s1 = pf.pf_workspace_size(512, 512, 512, 64)
    assert s1 >= 3 * 512 * 512 * 4
    assert pf.pf_workspace_size(512, 512, 512, 128) > s1
    assert s1 % 256 == 0


def test_diagnostics_error_paths(pf):
    p = I.default_params()
    need = pf.pf_diag_workspace_size(64, 64)
    assert need > 0 and pf.pf_diag_error_offset(64, 64) < need
    assert pf.pf_diagnostics(p, 64, 64, 64, FAKE, FAKE, FAKE, FAKE, need - 1, FAKE, 0) == pf.PF_ERR_LAYOUT
    assert pf.pf_diagnostics(p, 64, 64, 64, FAKE, FAKE, 0, FAKE, need, FAKE, 0) == pf.PF_ERR_ARG
    assert pf.pf_diagnostics(p, 0, 64, 64, FAKE, FAKE, FAKE, FAKE, need, FAKE, 0) == pf.PF_ERR_ARG
    assert pf.pf_diagnostics(p, 64, 64, 64, FAKE, FAKE, FAKE, FAKE + 8, need, FAKE, 0) == pf.PF_ERR_LAYOUT


def test_static_diagnostics_error_paths_report_their_reason(pf):
    """The allocation-free diagnostics reject bad arguments before any CUDA call, through the same
    checks and error text as the workspace entry point."""
    p = I.default_params()
    cases = [
        ((p, 64, 64, 64, FAKE, FAKE, 0, FAKE, None, 0), pf.PF_ERR_ARG, "null pointer"),
        ((p, 0, 64, 64, FAKE, FAKE, FAKE, FAKE, None, 0), pf.PF_ERR_ARG, "empty grid"),
        ((p, (1 << 20) + 4, 8, (1 << 20) + 4, FAKE, FAKE, FAKE, FAKE, None, 0), pf.PF_ERR_ARG, "grid side above"),
        ((p, 40, 8, 42, FAKE, FAKE, FAKE, FAKE, None, 0), pf.PF_ERR_LAYOUT, "pitch"),
        ((p, 40, 8, 40, FAKE, FAKE, FAKE, FAKE + 4, None, 0), pf.PF_ERR_LAYOUT, "8-byte aligned"),
        ((dict(p, dx=0.0), 40, 8, 40, FAKE, FAKE, FAKE, FAKE, None, 0), pf.PF_ERR_ARG, "dx"),
    ]
    for args, code, text in cases:
        assert pf.pf_diagnostics_static(*args) == code, text
        assert text in pf.last_error(), (text, pf.last_error())


def test_new_entry_points_reject_null_handles_before_any_cuda_call(pf):
    import ctypes as C
    lib = pf.lib
    assert lib.pf_hybrid_workspace_size(None) == 0
    hp = pf.HybridParams(2000, 2000, 1000, 2000.0, -1.5, 1.5, -0.5, 1.5, -0.5, 1.5)
    st = pf.HybridStats()
    assert lib.pf_hybrid_run(None, None, C.byref(hp), 100, None, 0, C.byref(st)) == pf.PF_ERR_ARG
    assert "null" in lib.pf_hybrid_last_error().decode()
    assert lib.pf_unet_reset_frames(None) == pf.PF_ERR_ARG
    assert lib.pf_unet_frame(None, 1, None, None, None, 256) == pf.PF_ERR_ARG
    assert pf.pf_set_tile_loop(None, True) == pf.PF_ERR_ARG
    assert lib.pf_ens_set_tma(None, 1) == pf.PF_ERR_ARG
    assert lib.pf_ens_staging_mode(None) == -1


def _ens_init(pf, plist, shapes, work_bytes=None, ptr=FAKE):
    import ctypes as C

    n = len(plist)
    I_ = C.c_int * n
    nx = I_(*[s[0] for s in shapes])
    ny = I_(*[s[1] for s in shapes])
    pitch = I_(*[((s[0] + 31) // 32) * 32 for s in shapes])
    params = (pf.Params * n)(*[pf.Params.from_dict(p) for p in plist])
    V = C.c_void_p * n
    f = V(*([ptr] * n))
    if work_bytes is None:
        work_bytes = pf.lib.pf_ens_workspace_size(n, nx, ny, pitch)
    h = C.c_void_p()
    return pf.lib.pf_ens_init(n, params, nx, ny, pitch, f, f, f, FAKE, work_bytes, None, C.byref(h))


def test_ensemble_init_error_paths(pf):
    good = O.with_dt(I.default_params())
    shapes = [(64, 64), (37, 23)]
    assert pf.lib.pf_ens_workspace_size(0, None, None, None) == 0
    assert _ens_init(pf, [good, dict(good, phi_mode=1)], shapes) == pf.PF_ERR_ARG
    assert _ens_init(pf, [good, dict(good, MA_bulk=2.0)], shapes) == pf.PF_ERR_ARG
    lim = pf.pf_dt_limit(good)[0]
    assert _ens_init(pf, [good, dict(good, dt=1.1 * lim)], shapes) == pf.PF_ERR_UNSTABLE
    assert _ens_init(pf, [good, good], shapes, work_bytes=4096) == pf.PF_ERR_LAYOUT
    assert _ens_init(pf, [good, good], [(64, 64), (0, 5)]) == pf.PF_ERR_ARG
    assert _ens_init(pf, [good, good], shapes, ptr=FAKE + 4) == pf.PF_ERR_LAYOUT


def test_unet_workspace_shape_rules(pf):
    """Host-side shape rules of the U-Net surrogate: sides >= 128 and multiples of 8, the quarter-resolution
    width dividing or a multiple of the 128-pixel tile, and fewer than 2^27 pixels in the batch (the range
    of the convolutions' tile indices)."""
    ws = pf.lib.pf_unet_workspace_size
    s16 = ws(16, 256, 256)
    assert s16 > 0 and s16 % 256 == 0
    # at least the full-resolution activations: pre1, cat1 (64 channels), h1, in BF16
    assert s16 >= 2 * 16 * 256 * 256 * (32 + 64 + 32)
    assert ws(32, 256, 256) > s16 > ws(8, 256, 256) > 0
    assert ws(1, 128, 128) > 0 and ws(1, 512, 512) > 0 and ws(2, 1024, 128) > 0
    for n, nx, ny in ((0, 256, 256), (1, 120, 256), (1, 256, 120), (1, 260, 256), (1, 384, 256),
                      (4097, 128, 128)):
        assert ws(n, nx, ny) == 0, (n, nx, ny)
    # 2^27 pixels: 2047 runs of 256^2 fit, 2048 do not
    assert ws(2047, 256, 256) > 0
    assert ws(2048, 256, 256) == 0
