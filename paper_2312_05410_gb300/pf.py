"""Python binding of libpf.so (include/pf.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; PyTorch provides device
memory and the CUDA stream.  Importing this module loads the in-tree
``_build/libpf.so`` and raises if it is missing (build it with
``python -m paper_2312_05410_gb300.build``); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB as _LIB_PATH

PF_OK = 0
PF_ERR_ARG = -1
PF_ERR_LAYOUT = -2
PF_ERR_UNSTABLE = -3
PF_ERR_NONFINITE = -4
PF_ERR_TIMEOUT = -5
PF_ERR_CUDA = -6


class PFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class Params(C.Structure):
    """Mirror of struct pf_params."""
    _fields_ = [(n, C.c_double) for n in (
        "dx", "dt", "W_c", "W_phi", "kappa_c", "kappa_phi",
        "MA_bulk", "MB_bulk", "MA_surf", "MB_surf", "sigma_surf",
        "M_phi", "L_phi", "D_rho", "v_mag", "v_angle_deg", "rho_top")] + [
        ("phi_mode", C.c_int), ("deposition", C.c_int), ("diag_every", C.c_int)]

    @classmethod
    def from_dict(cls, d: dict) -> "Params":
        p = cls()
        for name, _ in cls._fields_:
            setattr(p, name, d[name])
        return p


# Ensemble tile kinds (pf_ens_set_tile), by index.
TILE_KINDS = ("56x8", "56x24", "56x16", "56x24, persistent tile walk", "56x24, cooperative launch of up to 100 steps")
ENS_STEPS_PER_PERSISTENT_LAUNCH = 100


class HybridParams(C.Structure):
    """Mirror of struct pf_hybrid_params."""
    _fields_ = [("dns_stretch", C.c_long), ("jump_steps", C.c_long), ("frame_every", C.c_long),
                ("dt_ref_steps", C.c_double)] + [(n, C.c_double) for n in (
                    "phi_lo", "phi_hi", "c_lo", "c_hi", "rho_lo", "rho_hi")] + [("dns_lead", C.c_long)]


class HybridStats(C.Structure):
    """Mirror of struct pf_hybrid_stats."""
    _fields_ = [("jumps", C.c_long), ("fallbacks", C.c_long), ("dns_steps", C.c_long)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libpf.so not built ({_LIB_PATH}); run python -m paper_2312_05410_gb300.build")
    L = C.CDLL(_LIB_PATH)
    P = C.POINTER(Params)
    vp, sz = C.c_void_p, C.c_size_t
    L.pf_dt_limit.argtypes, L.pf_dt_limit.restype = [P, C.POINTER(C.c_double)], C.c_int
    L.pf_workspace_size.argtypes, L.pf_workspace_size.restype = [C.c_int, C.c_int, C.c_int, C.c_int], sz
    L.pf_init.argtypes = [P, C.c_int, C.c_int, C.c_int, vp, vp, vp, vp, sz, C.c_int, vp, C.POINTER(vp)]
    L.pf_init.restype = C.c_int
    L.pf_step.argtypes, L.pf_step.restype = [vp, C.c_long], C.c_int
    L.pf_diag.argtypes, L.pf_diag.restype = [vp, C.POINTER(C.c_double)], C.c_int
    L.pf_diag_history.argtypes = [vp, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int)]
    L.pf_diag_history.restype = C.c_int
    L.pf_get_step.argtypes, L.pf_get_step.restype = [vp], C.c_long
    L.pf_set_step.argtypes, L.pf_set_step.restype = [vp, C.c_long], C.c_int
    L.pf_clear_error.argtypes, L.pf_clear_error.restype = [vp], C.c_int
    L.pf_set_wait_limit.argtypes, L.pf_set_wait_limit.restype = [vp, C.c_int], C.c_int
    L.pf_staging_mode.argtypes, L.pf_staging_mode.restype = [vp], C.c_int
    L.pf_set_tile_loop.argtypes, L.pf_set_tile_loop.restype = [vp, C.c_int], C.c_int
    L.pf_set_steps_per_launch.argtypes, L.pf_set_steps_per_launch.restype = [vp, C.c_int], C.c_int
    L.pf_load_host.argtypes, L.pf_load_host.restype = [vp, vp, vp, vp, C.c_int], C.c_int
    L.pf_store_host.argtypes, L.pf_store_host.restype = [vp, vp, vp, vp, C.c_int], C.c_int
    L.pf_destroy.argtypes, L.pf_destroy.restype = [vp], C.c_int
    L.pf_diag_workspace_size.argtypes, L.pf_diag_workspace_size.restype = [C.c_int, C.c_int], sz
    L.pf_diag_error_offset.argtypes, L.pf_diag_error_offset.restype = [C.c_int, C.c_int], sz
    L.pf_diagnostics.argtypes = [P, C.c_int, C.c_int, C.c_int, vp, vp, vp, vp, sz, vp, vp]
    L.pf_diagnostics.restype = C.c_int
    L.pf_diagnostics_static.argtypes = [P, C.c_int, C.c_int, C.c_int, vp, vp, vp, vp, vp, vp]
    L.pf_diagnostics_static.restype = C.c_int
    ip, pp = C.POINTER(C.c_int), C.POINTER(C.c_void_p)
    L.pf_ens_workspace_size.argtypes, L.pf_ens_workspace_size.restype = [C.c_int, ip, ip, ip], sz
    L.pf_ens_init.argtypes = [C.c_int, P, ip, ip, ip, pp, pp, pp, vp, sz, vp, C.POINTER(vp)]
    L.pf_ens_init.restype = C.c_int
    L.pf_ens_step.argtypes, L.pf_ens_step.restype = [vp, C.c_long], C.c_int
    L.pf_ens_autotune.argtypes = [vp, C.c_int, ip, C.POINTER(C.c_double)]
    L.pf_ens_autotune.restype = C.c_int
    L.pf_ens_set_tile.argtypes, L.pf_ens_set_tile.restype = [vp, C.c_int], C.c_int
    L.pf_ens_set_wait_limit.argtypes, L.pf_ens_set_wait_limit.restype = [vp, C.c_int], C.c_int
    L.pf_ens_set_tma.argtypes, L.pf_ens_set_tma.restype = [vp, C.c_int], C.c_int
    L.pf_ens_staging_mode.argtypes, L.pf_ens_staging_mode.restype = [vp], C.c_int
    L.pf_ens_get_tile.argtypes, L.pf_ens_get_tile.restype = [vp], C.c_int
    L.pf_ens_get_step.argtypes, L.pf_ens_get_step.restype = [vp], C.c_long
    L.pf_ens_diag.argtypes, L.pf_ens_diag.restype = [vp, C.c_int, C.POINTER(C.c_double)], C.c_int
    L.pf_ens_destroy.argtypes, L.pf_ens_destroy.restype = [vp], C.c_int
    L.pf_ens_last_error.argtypes, L.pf_ens_last_error.restype = [], C.c_char_p
    L.pf_adjoint_workspace_size.argtypes = [C.c_int, C.c_int, C.c_int, C.c_long, C.c_int]
    L.pf_adjoint_workspace_size.restype = sz
    L.pf_adjoint.argtypes = [P, C.c_int, C.c_int, C.c_int, vp, vp, vp, C.c_long, C.c_int, vp, vp, vp, vp, vp, vp,
                             C.POINTER(C.c_double), vp, vp, vp, vp, sz, vp]
    L.pf_adjoint.restype = C.c_int
    L.pf_adjoint_last_error.argtypes, L.pf_adjoint_last_error.restype = [], C.c_char_p
    L.pf_conv3x3_bf16.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, C.c_int, vp, C.c_int, C.c_int,
                                  C.c_int, vp, vp, vp]
    L.pf_conv3x3_bf16.restype = C.c_int
    L.pf_tconv2x2_bf16.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, C.c_int, vp, C.c_int, C.c_int,
                                   vp, vp]
    L.pf_tconv2x2_bf16.restype = C.c_int
    L.pf_conv_halo.argtypes, L.pf_conv_halo.restype = [C.c_int], C.c_int
    L.pf_unet_last_error.argtypes, L.pf_unet_last_error.restype = [], C.c_char_p
    L.pf_unet_workspace_size.argtypes, L.pf_unet_workspace_size.restype = [C.c_int, C.c_int, C.c_int], sz
    L.pf_unet_init.argtypes = [C.POINTER(C.POINTER(C.c_float)), C.c_int, C.c_int, C.c_int, C.c_int, vp, sz, vp,
                               C.POINTER(vp)]
    L.pf_unet_init.restype = C.c_int
    L.pf_unet_frame.argtypes = [vp, C.c_int, pp, pp, pp, C.c_int]
    L.pf_unet_frame.restype = C.c_int
    L.pf_unet_reset_frames.argtypes, L.pf_unet_reset_frames.restype = [vp], C.c_int
    L.pf_unet_jump.argtypes = [vp, C.c_int, pp, pp, pp, C.c_int, C.c_double]
    L.pf_unet_jump.restype = C.c_int
    L.pf_unet_sync.argtypes, L.pf_unet_sync.restype = [vp], C.c_int
    L.pf_unet_check.argtypes = [vp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, ip]
    L.pf_unet_check.restype = C.c_int
    L.pf_unet_buffer.argtypes = [vp, C.c_int, C.POINTER(vp), C.POINTER(C.c_int)]
    L.pf_unet_buffer.restype = C.c_int
    L.pf_unet_destroy.argtypes, L.pf_unet_destroy.restype = [vp], C.c_int
    L.pf_hybrid_workspace_size.argtypes, L.pf_hybrid_workspace_size.restype = [vp], sz
    L.pf_hybrid_run.argtypes = [vp, vp, C.POINTER(HybridParams), C.c_long, vp, sz, C.POINTER(HybridStats)]
    L.pf_hybrid_run.restype = C.c_int
    L.pf_hybrid_last_error.argtypes, L.pf_hybrid_last_error.restype = [], C.c_char_p
    L.pf_s2_counts.argtypes = [vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp]
    L.pf_s2_counts.restype = C.c_int
    L.pf_strerror.argtypes, L.pf_strerror.restype = [C.c_int], C.c_char_p
    L.pf_last_error.argtypes, L.pf_last_error.restype = [], C.c_char_p
    return L


lib = _load()


def _check(rc: int) -> int:
    if rc != PF_OK:
        raise PFError(rc, f"{lib.pf_strerror(rc).decode()}: {lib.pf_last_error().decode()}")
    return rc


def strerror(code: int) -> str:
    return lib.pf_strerror(code).decode()


def last_error() -> str:
    return lib.pf_last_error().decode()


# ---------------------------------------------------------------- thin wrappers
def pf_dt_limit(params: dict) -> np.ndarray:
    out = (C.c_double * 4)()
    _check(lib.pf_dt_limit(C.byref(Params.from_dict(params)), out))
    return np.array(out[:])


def pf_workspace_size(nx: int, ny: int, pitch: int, history_rows: int) -> int:
    return int(lib.pf_workspace_size(nx, ny, pitch, history_rows))


def pf_init(params: dict, nx: int, ny: int, pitch: int, phi_ptr: int, c_ptr: int, rho_ptr: int,
            work_ptr: int, work_bytes: int, history_rows: int, stream: int) -> int:
    """Returns the raw return code and handle (no exception), for error-path tests."""
    h = C.c_void_p()
    rc = lib.pf_init(C.byref(Params.from_dict(params)), nx, ny, pitch, phi_ptr, c_ptr, rho_ptr, work_ptr,
                     work_bytes, history_rows, stream, C.byref(h))
    return rc, h


def pf_step(h, n: int) -> int:
    return lib.pf_step(h, n)


def pf_diag(h):
    out = (C.c_double * 4)()
    rc = lib.pf_diag(h, out)
    return rc, np.array(out[:])


def pf_diag_history(h, max_rows: int = 4096):
    buf = (C.c_double * (5 * max(1, max_rows)))()
    rows = C.c_int(0)
    _check(lib.pf_diag_history(h, buf, max_rows, C.byref(rows)))
    return np.array(buf[: 5 * rows.value]).reshape(rows.value, 5)


def pf_get_step(h) -> int:
    return int(lib.pf_get_step(h))


def pf_set_step(h, step: int) -> int:
    return lib.pf_set_step(h, step)


def pf_clear_error(h) -> int:
    return lib.pf_clear_error(h)


def pf_set_wait_limit(h, polls: int) -> int:
    return lib.pf_set_wait_limit(h, int(polls))


def pf_staging_mode(h) -> int:
    return int(lib.pf_staging_mode(h))


def pf_set_steps_per_launch(h, steps: int) -> int:
    return int(lib.pf_set_steps_per_launch(h, int(steps)))


def pf_set_tile_loop(h, on: bool) -> int:
    return int(lib.pf_set_tile_loop(h, 1 if on else 0))


def pf_destroy(h) -> int:
    return lib.pf_destroy(h)


def pf_diag_workspace_size(nx: int, ny: int) -> int:
    return int(lib.pf_diag_workspace_size(nx, ny))


def pf_diag_error_offset(nx: int, ny: int) -> int:
    return int(lib.pf_diag_error_offset(nx, ny))


def pf_diagnostics(params: dict, nx: int, ny: int, pitch: int, phi_ptr: int, c_ptr: int, rho_ptr: int,
                   work_ptr: int, work_bytes: int, out_dev_ptr: int, stream: int) -> int:
    return lib.pf_diagnostics(C.byref(Params.from_dict(params)), nx, ny, pitch, phi_ptr, c_ptr, rho_ptr,
                              work_ptr, work_bytes, out_dev_ptr, stream)


def pf_diagnostics_static(params: dict, nx: int, ny: int, pitch: int, phi_ptr: int, c_ptr: int, rho_ptr: int,
                          out_dev_ptr: int, err_dev_ptr, stream: int) -> int:
    """Diagnostics with no caller workspace (for callers that cannot allocate device memory)."""
    return lib.pf_diagnostics_static(C.byref(Params.from_dict(params)), nx, ny, pitch, phi_ptr, c_ptr, rho_ptr,
                                     out_dev_ptr, err_dev_ptr, stream)


# ---------------------------------------------------------------- torch-backed simulation
def padded_pitch(nx: int) -> int:
    """Row pitch in floats: nx rounded up to 32 (128-byte rows)."""
    return (nx + 31) // 32 * 32


class Sim:
    """One simulation bound to torch-owned device fields and workspace.

    ``phi``, ``c``, ``rho`` are (ny, pitch) float32 CUDA tensors; the model
    state is their first nx columns.  All launches go to ``stream`` (default:
    torch's current stream).
    """

    def __init__(self, params: dict, phi, c, rho, history_rows: int = 256, stream=None, device="cuda", nx=None):
        """phi, c, rho: (ny, nx) arrays, or CUDA tensors (ny, >= nx) whose first nx columns (default: all)
        are the state; tensors are copied device to device on the launch stream."""
        import torch

        self.stream = stream if stream is not None else torch.cuda.current_stream()
        on_device = all(isinstance(a, torch.Tensor) and a.is_cuda for a in (phi, c, rho))
        if not on_device:
            phi, c, rho = (np.asarray(a, dtype=np.float32) for a in (phi, c, rho))
        ny = phi.shape[0]
        nx = int(nx) if nx is not None else phi.shape[1]
        self.nx, self.ny, self.pitch = nx, ny, padded_pitch(nx)
        self.params = dict(params)
        self.fields = []
        # the fields are filled on the launch stream, after whatever the caller's stream has queued
        self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            for a in (phi, c, rho):
                t = torch.zeros((ny, self.pitch), dtype=torch.float32, device=device)
                if on_device:
                    t[:, :nx].copy_(a[:, :nx])
                else:
                    t[:, :nx] = torch.from_numpy(a).to(device)
                self.fields.append(t)
        self.phi, self.c, self.rho = self.fields
        nbytes = pf_workspace_size(nx, ny, self.pitch, history_rows)
        if nbytes == 0:
            raise PFError(PF_ERR_ARG, "bad grid size")
        self.work = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = self.work.data_ptr()
        self._work_ptr = (base + 255) // 256 * 256
        self._work_bytes = nbytes
        rc, h = pf_init(self.params, nx, ny, self.pitch, self.phi.data_ptr(), self.c.data_ptr(),
                        self.rho.data_ptr(), self._work_ptr, nbytes, history_rows, self.stream.cuda_stream)
        _check(rc)
        self.h = h

    def step(self, n: int):
        _check(pf_step(self.h, int(n)))

    def diag(self) -> np.ndarray:
        rc, out = pf_diag(self.h)
        _check(rc)
        return out

    def history(self) -> np.ndarray:
        return pf_diag_history(self.h)

    @property
    def step_index(self) -> int:
        return pf_get_step(self.h)

    def set_step(self, step: int):
        _check(pf_set_step(self.h, step))

    def load_host(self, phi, c, rho):
        """pf_load_host: (ny, nx) float32 host arrays or CPU tensors (pinned for an overlapping copy)."""
        ptr = [int(a.data_ptr()) if hasattr(a, "data_ptr") else a.ctypes.data for a in (phi, c, rho)]
        _check(lib.pf_load_host(self.h, *ptr, int(phi.shape[1])))

    def store_host(self, phi, c, rho):
        """pf_store_host into (ny, nx) float32 host arrays or CPU tensors."""
        ptr = [int(a.data_ptr()) if hasattr(a, "data_ptr") else a.ctypes.data for a in (phi, c, rho)]
        _check(lib.pf_store_host(self.h, *ptr, int(phi.shape[1])))

    def numpy(self):
        """(phi, c, rho) of the current state as float32 numpy arrays (synchronises)."""
        self.stream.synchronize()
        return tuple(t[:, : self.nx].cpu().numpy() for t in self.fields)

    def close(self):
        if getattr(self, "h", None) is not None:
            _check(pf_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ensemble:
    """Independent runs of uneven sizes stepped together by one launch per step.

    members: list of (params, phi, c, rho) with numpy (ny, nx) arrays; every
    run gets torch-owned (ny, pitch) float32 device fields.
    """

    def __init__(self, members, stream=None, device="cuda"):
        import torch

        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.n = len(members)
        self.fields, self.shapes, self.params = [], [], []
        nxs, nys, pitches = [], [], []
        for params, phi, c, rho in members:
            ny, nx = np.asarray(phi).shape
            pitch = padded_pitch(nx)
            ts = []
            for a in (phi, c, rho):
                t = torch.zeros((ny, pitch), dtype=torch.float32, device=device)
                t[:, :nx] = torch.from_numpy(np.asarray(a, dtype=np.float32)).to(device)
                ts.append(t)
            self.fields.append(ts)
            self.shapes.append((ny, nx))
            self.params.append(dict(params))
            nxs.append(nx), nys.append(ny), pitches.append(pitch)
        I = C.c_int * self.n
        self._nx, self._ny, self._pitch = I(*nxs), I(*nys), I(*pitches)
        nbytes = int(lib.pf_ens_workspace_size(self.n, self._nx, self._ny, self._pitch))
        if nbytes == 0:
            raise PFError(PF_ERR_ARG, "bad ensemble sizes")
        self.work = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        wp = (self.work.data_ptr() + 255) // 256 * 256
        self._params = (Params * self.n)(*[Params.from_dict(p) for p in self.params])
        V = C.c_void_p * self.n
        ptr = [V(*[self.fields[r][q].data_ptr() for r in range(self.n)]) for q in range(3)]
        torch.cuda.synchronize()
        h = C.c_void_p()
        rc = lib.pf_ens_init(self.n, self._params, self._nx, self._ny, self._pitch, ptr[0], ptr[1], ptr[2], wp,
                             nbytes, self.stream.cuda_stream, C.byref(h))
        if rc != PF_OK:
            raise PFError(rc, f"{strerror(rc)}: {lib.pf_ens_last_error().decode()}")
        self.h = h

    def _check(self, rc):
        if rc != PF_OK:
            raise PFError(rc, f"{strerror(rc)}: {lib.pf_ens_last_error().decode()}")

    def step(self, n: int):
        self._check(lib.pf_ens_step(self.h, int(n)))

    def autotune(self, trial_steps: int = 20):
        chosen = C.c_int(-1)
        secs = (C.c_double * 5)()
        self._check(lib.pf_ens_autotune(self.h, int(trial_steps), C.byref(chosen), secs))
        return chosen.value, list(secs)

    def set_tile(self, tile: int):
        self._check(lib.pf_ens_set_tile(self.h, int(tile)))

    def set_wait_limit(self, polls: int):
        self._check(lib.pf_ens_set_wait_limit(self.h, int(polls)))

    def set_tma(self, on: bool):
        """TMA staging of the short and large tiles inside each run's grid in x (default on)."""
        self._check(lib.pf_ens_set_tma(self.h, int(bool(on))))

    @property
    def staging_mode(self) -> int:
        """1 if the current tile kind stages by TMA, else 0."""
        return int(lib.pf_ens_staging_mode(self.h))

    @property
    def tile(self) -> int:
        return int(lib.pf_ens_get_tile(self.h))

    @property
    def step_index(self) -> int:
        return int(lib.pf_ens_get_step(self.h))

    def diag(self, run: int) -> np.ndarray:
        out = (C.c_double * 4)()
        self._check(lib.pf_ens_diag(self.h, int(run), out))
        return np.array(out[:])

    def numpy(self, run: int):
        self.stream.synchronize()
        ny, nx = self.shapes[run]
        return tuple(t[:, :nx].cpu().numpy() for t in self.fields[run])

    def close(self):
        if getattr(self, "h", None) is not None:
            self._check(lib.pf_ens_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- adjoint
def device_fields(arrays, device="cuda"):
    """(ny, pitch) float32 CUDA tensors holding the given (ny, nx) arrays."""
    import torch

    out = []
    for a in arrays:
        a = np.asarray(a, dtype=np.float32)
        ny, nx = a.shape
        t = torch.zeros((ny, padded_pitch(nx)), dtype=torch.float32, device=device)
        t[:, :nx] = torch.from_numpy(a).to(device)
        out.append(t)
    return out


def adjoint(params: dict, init, nx: int, nsteps: int, K: int, w_phi, w_c, w_rho=None, stream=None):
    """Gradient of sum(w . u_N) through nsteps steps (pf_adjoint).

    init, w_*: (ny, pitch) float32 CUDA tensors (as made by device_fields), model
    width nx; returns {"phi0", "c0", "rho0": tensors, "v_mag", "m_scale", "kappa_c":
    floats, "final": (phi, c, rho)}.
    """
    import torch

    phi0, c0, rho0 = init
    ny, pitch = phi0.shape
    stream = stream if stream is not None else torch.cuda.current_stream()
    nbytes = int(lib.pf_adjoint_workspace_size(nx, ny, pitch, int(nsteps), int(K)))
    if nbytes == 0:
        raise PFError(PF_ERR_ARG, "bad adjoint sizes")
    work = torch.empty(nbytes + 256, dtype=torch.uint8, device=phi0.device)
    wp = (work.data_ptr() + 255) // 256 * 256
    g = [torch.zeros_like(phi0) for _ in range(3)]
    fin = [torch.zeros_like(phi0) for _ in range(3)]
    gp = (C.c_double * 3)()
    # the inputs and the zeroed outputs were written on the caller's stream: order the call after them
    stream.wait_stream(torch.cuda.current_stream())
    rc = lib.pf_adjoint(C.byref(Params.from_dict(params)), nx, ny, pitch, phi0.data_ptr(), c0.data_ptr(),
                        rho0.data_ptr(), int(nsteps), int(K), w_phi.data_ptr(), w_c.data_ptr(),
                        None if w_rho is None else w_rho.data_ptr(), g[0].data_ptr(), g[1].data_ptr(),
                        g[2].data_ptr(), gp, fin[0].data_ptr(), fin[1].data_ptr(), fin[2].data_ptr(), wp, nbytes,
                        stream.cuda_stream)
    if rc != PF_OK:
        raise PFError(rc, f"{strerror(rc)}: {lib.pf_adjoint_last_error().decode()}")
    return {"phi0": g[0], "c0": g[1], "rho0": g[2], "v_mag": gp[0], "m_scale": gp[1], "kappa_c": gp[2],
            "final": tuple(fin)}


def _scaled(params: dict, v_mag: float, m_scale: float, kappa_c: float) -> dict:
    q = dict(params, v_mag=v_mag, kappa_c=kappa_c)
    for k in ("MA_bulk", "MB_bulk", "MA_surf", "MB_surf"):
        q[k] = params[k] * m_scale
    return q


def make_run_function():
    """torch.autograd.Function: (v_mag, m_scale, kappa_c, phi0, c0, rho0) -> final (phi, c, rho).

    m_scale multiplies the four composition-mobility coefficients.  Forward runs the
    fused step kernels; backward runs the hand-written adjoint (checkpoints every K).
    Fields are (ny, pitch) float32 CUDA tensors of model width nx.
    """
    import torch

    class PFRun(torch.autograd.Function):
        @staticmethod
        def forward(ctx, v_mag, m_scale, kappa_c, phi0, c0, rho0, params, nx, nsteps, K):
            q = _scaled(params, float(v_mag), float(m_scale), float(kappa_c))
            # the given device tensors are bound by a device-to-device copy (no host round trip)
            sim = Sim(q, phi0.detach(), c0.detach(), rho0.detach(), history_rows=1, nx=nx)
            sim.step(int(nsteps))
            torch.cuda.current_stream().wait_stream(sim.stream)
            out = tuple(t.clone() for t in sim.fields)
            sim.close()
            ctx.save_for_backward(v_mag, m_scale, kappa_c, phi0, c0, rho0)
            ctx.q, ctx.nx, ctx.nsteps, ctx.K = q, int(nx), int(nsteps), int(K)
            return out

        @staticmethod
        def backward(ctx, gf, gc, gr):
            v_mag, m_scale, kappa_c, phi0, c0, rho0 = ctx.saved_tensors
            z = torch.zeros_like(phi0)
            gf = z if gf is None else gf.contiguous()
            gc = z if gc is None else gc.contiguous()
            gr = z if gr is None else gr.contiguous()
            res = adjoint(ctx.q, (phi0.contiguous(), c0.contiguous(), rho0.contiguous()), ctx.nx, ctx.nsteps,
                          ctx.K, gf, gc, gr)
            dv = torch.tensor(res["v_mag"], dtype=v_mag.dtype, device=v_mag.device)
            dm = torch.tensor(res["m_scale"] / float(m_scale), dtype=m_scale.dtype, device=m_scale.device)
            dk = torch.tensor(res["kappa_c"], dtype=kappa_c.dtype, device=kappa_c.device)
            return dv, dm, dk, res["phi0"], res["c0"], res["rho0"], None, None, None, None

    return PFRun


# ---------------------------------------------------------------------------------------------
# U-Net surrogate: tensor-core convolution primitives (BF16 NHWC tensors on the device)

def _ucheck(rc: int) -> int:
    if rc != PF_OK:
        raise PFError(rc, f"{strerror(rc)}: {lib.pf_unet_last_error().decode()}")
    return rc


def conv_weight_layout(w):
    """[Cout, Cin, 3, 3] (PyTorch convention) -> BF16 [9][Cout][Cin] on the device (tap = 3 ky + kx)."""
    import torch
    t = torch.as_tensor(np.asarray(w, dtype=np.float32))
    return t.permute(2, 3, 0, 1).reshape(9, t.shape[0], t.shape[1]).contiguous().to("cuda", torch.bfloat16)


def tconv_weight_layout(w):
    """[Cin, Cout, 2, 2] (PyTorch convention) -> BF16 [4 Cout][Cin] on the device (row (2 dy + dx) Cout + co)."""
    import torch
    t = torch.as_tensor(np.asarray(w, dtype=np.float32))
    return t.permute(2, 3, 1, 0).reshape(4 * t.shape[1], t.shape[0]).contiguous().to("cuda", torch.bfloat16)


def conv3x3_bf16(x, w_dev, groups: int, out=None, out_coff: int = 0, partials=None, err=None, stream=None):
    """x: BF16 NHWC [n, h, w, cin] on the device; w_dev from conv_weight_layout.  Returns (out, partials)."""
    import torch
    n, h, wd, cin = x.shape
    cout = w_dev.shape[1]
    if out is None:
        out = torch.empty((n, h, wd, cout), dtype=torch.bfloat16, device=x.device)
    if partials is None:
        partials = torch.zeros((n, groups, h * wd // 128, 4, 2), dtype=torch.float32, device=x.device)
    if err is None:
        err = torch.zeros(1, dtype=torch.int32, device=x.device)
    s = (stream or torch.cuda.current_stream()).cuda_stream
    _ucheck(lib.pf_conv3x3_bf16(x.data_ptr(), n, h, wd, cin, w_dev.data_ptr(), cout, out.data_ptr(), out.shape[3],
                                out_coff, groups, partials.data_ptr(), err.data_ptr(), s))
    return out, partials


def conv_halo(on: bool) -> bool:
    """Select the halo staging of 64-channel 3x3 convolutions (default on); returns the previous setting."""
    return bool(lib.pf_conv_halo(1 if on else 0))


def tconv2x2_bf16(x, w_dev, out=None, out_coff: int = 0, err=None, stream=None):
    """x: BF16 NHWC [n, h, w, cin]; w_dev from tconv_weight_layout.  Returns out [n, 2h, 2w, cout]."""
    import torch
    n, h, wd, cin = x.shape
    cout = w_dev.shape[0] // 4
    if out is None:
        out = torch.empty((n, 2 * h, 2 * wd, cout), dtype=torch.bfloat16, device=x.device)
    if err is None:
        err = torch.zeros(1, dtype=torch.int32, device=x.device)
    s = (stream or torch.cuda.current_stream()).cuda_stream
    _ucheck(lib.pf_tconv2x2_bf16(x.data_ptr(), n, h, wd, cin, w_dev.data_ptr(), cout, out.data_ptr(), out.shape[3],
                                 out_coff, err.data_ptr(), s))
    return out


UNET_WEIGHT_NAMES = (["mlp_w0", "mlp_b0", "mlp_w1", "mlp_b1", "mlp_w2", "mlp_b2", "proj1", "proj2", "proj3", "proj4",
                      "enc1", "enc2", "enc3", "enc4", "dec4", "dec3", "dec2", "dec1", "up4", "up3", "up2", "out"]
                     + [f"{n}_{g}" for n in ("enc1", "enc2", "enc3", "enc4", "dec4", "dec3", "dec2", "dec1", "out")
                        for g in ("gamma", "beta")])
UNET_BUFFERS = ("pre1", "cat1", "p1", "pre2", "cat2", "p2", "pre3", "cat3", "p3", "pre4", "zc4", "h4", "h3", "h2",
                "h1")
_UNET_LEVEL = (0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3, 3, 2, 1, 0)


class UNet:
    """The time-conditioned U-Net surrogate (pf_unet_*): weights in PyTorch layouts by name (see
    UNET_WEIGHT_NAMES), a batch of `batch` runs of ny x nx cells."""

    def __init__(self, weights: dict, batch: int, nx: int, ny: int, stream=None):
        import torch
        self.batch, self.nx, self.ny = batch, nx, ny
        self.stream = stream or torch.cuda.current_stream()
        size = lib.pf_unet_workspace_size(batch, nx, ny)
        if size == 0:
            raise PFError(PF_ERR_ARG, f"U-Net shape {batch} x {ny} x {nx} unsupported")
        self._arrays = [np.ascontiguousarray(np.asarray(weights[k], dtype=np.float32)) for k in UNET_WEIGHT_NAMES]
        ptrs = (C.POINTER(C.c_float) * len(self._arrays))(
            *[a.ctypes.data_as(C.POINTER(C.c_float)) for a in self._arrays])
        self.work = torch.empty(size + 256, dtype=torch.uint8, device="cuda")
        self._base = (self.work.data_ptr() + 255) // 256 * 256
        h = C.c_void_p()
        _ucheck(lib.pf_unet_init(ptrs, len(self._arrays), batch, nx, ny, self._base, size, self.stream.cuda_stream,
                                 C.byref(h)))
        self.h = h

    @staticmethod
    def _tables(fields):
        n = len(fields)
        return n, [(C.c_void_p * n)(*[int(f[q].data_ptr()) for f in fields]) for q in range(3)], fields[0][0].shape[1]

    def frame(self, fields):
        """Push `batch` tuples (phi, c, rho) of (ny, pitch) float32 CUDA tensors as the newest look-back frame."""
        n, arr, pitch = self._tables(fields)
        _ucheck(lib.pf_unet_frame(self.h, n, arr[0], arr[1], arr[2], pitch))

    def reset_frames(self):
        _ucheck(lib.pf_unet_reset_frames(self.h))

    def jump(self, fields, tau: float):
        """fields: `batch` tuples (phi, c, rho) of (ny, pitch) float32 CUDA tensors, updated in place; the
        frames pushed with frame() are the look-back."""
        n, arr, pitch = self._tables(fields)
        _ucheck(lib.pf_unet_jump(self.h, n, arr[0], arr[1], arr[2], pitch, float(tau)))

    def sync(self):
        _ucheck(lib.pf_unet_sync(self.h))

    def check(self, phi_range=(-1.5, 1.5), c_range=(-0.5, 1.5), rho_range=(-0.5, 1.5)) -> list[bool]:
        """Per run: is the last jump's prediction finite and inside the given ranges?  (Synchronises.)"""
        ok = (C.c_int * self.batch)()
        _ucheck(lib.pf_unet_check(self.h, phi_range[0], phi_range[1], c_range[0], c_range[1], rho_range[0],
                                  rho_range[1], ok))
        return [bool(v) for v in ok]

    def buffer(self, name: str):
        """Activation buffer `name` (see UNET_BUFFERS) as a BF16 NHWC tensor view of the workspace."""
        import torch
        k = UNET_BUFFERS.index(name)
        ptr, ch = C.c_void_p(), C.c_int()
        _ucheck(lib.pf_unet_buffer(self.h, k, C.byref(ptr), C.byref(ch)))
        lev = _UNET_LEVEL[k]
        hh, ww = self.ny >> lev, self.nx >> lev
        off = ptr.value - self.work.data_ptr()
        nel = self.batch * hh * ww * ch.value
        return self.work[off:off + 2 * nel].view(torch.bfloat16).view(self.batch, hh, ww, ch.value)

    def close(self):
        if getattr(self, "h", None) is not None:
            _ucheck(lib.pf_unet_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hybrid:
    """The hybrid DNS / U-Net solver (pf_hybrid_run): an Ensemble of equal grids and a UNet of the same
    batch and grid, sharing one stream.  The first `dns_lead` steps are DNS alone; then each cycle
    runs `dns_stretch` DNS steps (pushing look-back
    frames `2 frame_every` and `frame_every` steps before its end), backs the state up, jumps
    `jump_steps` steps with the U-Net and falls back to DNS for the jumped steps when a prediction
    fails the plausibility ranges."""

    def __init__(self, ens: "Ensemble", net: "UNet", dns_stretch: int = 2000, jump_steps: int = 2000,
                 frame_every: int = 1000, dt_ref_steps: float = 2000.0, phi_range=(-1.5, 1.5),
                 c_range=(-0.5, 1.5), rho_range=(-0.5, 1.5), dns_lead: int = 0):
        import torch
        self.ens, self.net = ens, net
        self.params = HybridParams(int(dns_stretch), int(jump_steps), int(frame_every), float(dt_ref_steps),
                                   *phi_range, *c_range, *rho_range, int(dns_lead))
        size = int(lib.pf_hybrid_workspace_size(ens.h))
        self.work = torch.empty(size + 256, dtype=torch.uint8, device="cuda")
        self._wp = (self.work.data_ptr() + 255) // 256 * 256
        self._size = size

    def run(self, total_steps: int) -> dict:
        st = HybridStats()
        rc = lib.pf_hybrid_run(self.ens.h, self.net.h, C.byref(self.params), int(total_steps), self._wp,
                               self._size, C.byref(st))
        if rc != PF_OK:
            raise PFError(rc, f"{strerror(rc)}: {lib.pf_hybrid_last_error().decode()}")
        return {"jumps": st.jumps, "fallbacks": st.fallbacks, "dns_steps": st.dns_steps}


def s2_counts(phi, c, nx: int, ny: int, R: int, stream=None):
    """S2 pair counts [2R+1, 2R+1] of the solid A phase of (phi, c) ((ny, pitch) FP32 CUDA tensors)."""
    import torch
    scratch = torch.empty(nx * ny, dtype=torch.uint8, device=phi.device)
    counts = torch.empty((2 * R + 1, 2 * R + 1), dtype=torch.int64, device=phi.device)
    s = (stream or torch.cuda.current_stream()).cuda_stream
    _check(lib.pf_s2_counts(phi.data_ptr(), c.data_ptr(), nx, ny, phi.shape[1], R, scratch.data_ptr(),
                            counts.data_ptr(), s))
    return counts


def s2_rel_l2(counts_true, counts_pred) -> float:
    """Relative L2 distance of two S2 maps (the normalisation by the cell count cancels)."""
    a = counts_true.double()
    return float((a - counts_pred.double()).norm() / a.norm())
