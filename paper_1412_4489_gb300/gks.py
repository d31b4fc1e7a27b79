"""ctypes binding of ``libgks.so`` (the C ABI declared in ``include/gks.h``).

Argument marshalling only: every step of the scheme runs in the CUDA kernels of the
library.  Functions keep the C names (``gks_create``, ``gks_set_state``, ``gks_step``,
``gks_advance``, ``gks_get_state``, ``gks_destroy`` ...); ``Solver`` wraps one handle.
Host arrays are float64 numpy arrays in the layouts of ``gks.h``; device arrays are
float64 torch CUDA tensors.  Loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

GKS_OK, GKS_EINVAL, GKS_ENOMEM, GKS_ECUDA, GKS_ENONPHYSICAL, GKS_ETIMEOUT, GKS_EUNSUPPORTED = range(7)
GKS_BC_PERIODIC, GKS_BC_OUTFLOW, GKS_BC_SLIPWALL, GKS_BC_NOSLIP_ISOTHERMAL, GKS_BC_NOSLIP_ADIABATIC = range(5)
GKS_BC_EXCHANGE = 5
GKS_PART_STATE, GKS_PART_RECORDS = 0, 1
GKS_FP64, GKS_FP32_BULK = 0, 1
STATUS_NAMES = ["GKS_OK", "GKS_EINVAL", "GKS_ENOMEM", "GKS_ECUDA", "GKS_ENONPHYSICAL", "GKS_ETIMEOUT",
                "GKS_EUNSUPPORTED"]


class gks_bc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("u_wall", ctypes.c_double), ("v_wall", ctypes.c_double),
                ("T_wall", ctypes.c_double)]


class gks_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("weno_eps", ctypes.c_double), ("weno_C", ctypes.c_double),
                ("tau_eps", ctypes.c_double), ("tau_C", ctypes.c_double), ("viscous_dt", ctypes.c_int),
                ("characteristic", ctypes.c_int)]


class gks_grid_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("Lx", ctypes.c_double), ("Ly", ctypes.c_double),
                ("gamma", ctypes.c_double), ("Pr", ctypes.c_double), ("mu", ctypes.c_double), ("bc", gks_bc * 4)]


class GKSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


def load(path: str | None = None):
    """Loads (building first if needed) the CUDA library; raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        _build.build()
    L = ctypes.CDLL(path)
    H = ctypes.c_void_p
    D = ctypes.c_double
    L.gks_default_options.argtypes = [ctypes.POINTER(gks_options)]
    L.gks_default_options.restype = None
    L.gks_create.argtypes = [ctypes.c_int, ctypes.c_int, D, D, D, D, D, ctypes.POINTER(gks_bc),
                             ctypes.POINTER(gks_options), ctypes.c_void_p, ctypes.POINTER(H)]
    L.gks_set_state.argtypes = [H, _dp, _dp, _dp, D]
    L.gks_set_state_device.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, D]
    L.gks_step.argtypes = [H, D, D, _dp]
    L.gks_advance.argtypes = [H, ctypes.c_int, D, D]
    L.gks_sync.argtypes = [H, _dp, ctypes.POINTER(ctypes.c_longlong)]
    L.gks_get_state.argtypes = [H, _dp, _dp, _dp, _dp]
    L.gks_get_state_device.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, _dp]
    L.gks_destroy.argtypes = [H]
    L.gks_destroy.restype = None
    L.gks_last_error.argtypes = [H]
    L.gks_last_error.restype = ctypes.c_char_p
    L.gks_launches_per_step.argtypes = [H]
    L.gks_profile_step.argtypes = [H, D, ctypes.POINTER(ctypes.c_float)]
    L.gks_face_op_count.argtypes = [_dp, _dp, _dp, D, D, D, D, D, D, D, D, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_longlong)]
    L.gks_measure_alu_peak.argtypes = [ctypes.c_int, _dp]
    L.gks_part_halo_bytes.argtypes = [H, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
    L.gks_part_bound.argtypes = [H, _dp]
    L.gks_part_recon.argtypes = [H, D]
    L.gks_part_finish.argtypes = [H]
    L.gks_part_get_edge.argtypes = [H, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    L.gks_part_set_halo.argtypes = [H, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    for name in ("gks_part_halo_bytes", "gks_part_bound", "gks_part_recon", "gks_part_finish", "gks_part_get_edge",
                 "gks_part_set_halo"):
        getattr(L, name).restype = ctypes.c_int
    L.gks_step_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, D, D, D, D, D, ctypes.POINTER(gks_bc),
                                   ctypes.POINTER(gks_options), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, D, D,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, _dp, ctypes.c_void_p]
    B = ctypes.c_void_p
    LL = ctypes.POINTER(ctypes.c_longlong)
    L.gks_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(gks_grid_desc), ctypes.POINTER(gks_options),
                                   ctypes.c_void_p, ctypes.POINTER(B)]
    L.gks_batch_set_state.argtypes = [B, ctypes.c_int, _dp, _dp, _dp, D]
    L.gks_batch_get_state.argtypes = [B, ctypes.c_int, _dp, _dp, _dp, _dp, LL]
    L.gks_batch_step.argtypes = [B, ctypes.c_int, D]
    L.gks_batch_sync.argtypes = [B, LL, LL]
    L.gks_batch_grid_info.argtypes = [B, ctypes.c_int, _dp, LL, ctypes.POINTER(ctypes.c_int)]
    L.gks_batch_configure.argtypes = [B, ctypes.c_int, ctypes.c_int]
    L.gks_batch_profile.argtypes = [B, ctypes.c_int, D, _dp]
    L.gks_batch_profile.restype = ctypes.c_int
    L.gks_batch_autotune.argtypes = [B, D, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]
    L.gks_batch_configure_tiles.argtypes = [B, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.gks_batch_configure_tiles.restype = ctypes.c_int
    L.gks_batch_set_wait_limit.argtypes = [B, D, ctypes.c_int]
    L.gks_batch_cells.argtypes = [B]
    L.gks_batch_cells.restype = ctypes.c_longlong
    L.gks_batch_launches_per_call.argtypes = [B]
    L.gks_batch_destroy.argtypes = [B]
    L.gks_batch_destroy.restype = None
    L.gks_batch_last_error.argtypes = [B]
    L.gks_batch_last_error.restype = ctypes.c_char_p
    for name in ("gks_batch_create", "gks_batch_set_state", "gks_batch_get_state", "gks_batch_step", "gks_batch_sync",
                 "gks_batch_grid_info", "gks_batch_configure", "gks_batch_autotune", "gks_batch_set_wait_limit",
                 "gks_batch_launches_per_call"):
        getattr(L, name).restype = ctypes.c_int
    L.gks_debug_recon.argtypes = [H, _dp]
    L.gks_debug_flux.argtypes = [H, D, _dp, _dp, _dp, _dp]
    for name in ("gks_create", "gks_set_state", "gks_set_state_device", "gks_step", "gks_advance", "gks_sync",
                 "gks_get_state", "gks_get_state_device", "gks_debug_recon", "gks_debug_flux", "gks_profile_step", "gks_step_noalloc", "gks_face_op_count", "gks_measure_alu_peak",
                 "gks_launches_per_step"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _ptr(a):
    if a is None:
        return None
    assert isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _dev(t):
    if t is None:
        return None
    assert t.is_cuda and str(t.dtype) == "torch.float64" and t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr())


def _check(h, st):
    if st != GKS_OK:
        raise GKSError(st, load().gks_last_error(h).decode())


def _buf(b):
    """Address of a contiguous byte buffer: a numpy array (host) or a torch tensor (host or CUDA)."""
    if isinstance(b, np.ndarray):
        assert b.flags["C_CONTIGUOUS"]
        return ctypes.c_void_p(b.ctypes.data)
    assert b.is_contiguous()
    return ctypes.c_void_p(b.data_ptr())


# ---- partitioned step (row slabs of one grid; see gks.h) ----
def gks_part_halo_bytes(h, what):
    n = ctypes.c_size_t(0)
    _check(h, load().gks_part_halo_bytes(h, int(what), ctypes.byref(n)))
    return n.value


def gks_part_bound(h):
    b = ctypes.c_double(0.0)
    _check(h, load().gks_part_bound(h, ctypes.byref(b)))
    return b.value


def gks_part_recon(h, dt):
    _check(h, load().gks_part_recon(h, float(dt)))


def gks_part_finish(h):
    _check(h, load().gks_part_finish(h))


def gks_part_get_edge(h, side, what, dst):
    _check(h, load().gks_part_get_edge(h, int(side), int(what), _buf(dst)))


def gks_part_set_halo(h, side, what, src):
    _check(h, load().gks_part_set_halo(h, int(side), int(what), _buf(src)))


def gks_default_options(precision=GKS_FP64, **kw) -> gks_options:
    o = gks_options()
    load().gks_default_options(ctypes.byref(o))
    o.precision = precision
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def make_bcs(spec):
    """spec: 4 entries (kind, u_wall, v_wall, T_wall) or kinds; order x-low, x-high, y-low, y-high."""
    arr = (gks_bc * 4)()
    for k in range(4):
        s = spec[k] if isinstance(spec[k], (tuple, list)) else (spec[k], 0.0, 0.0, 1.0)
        arr[k] = gks_bc(int(s[0]), float(s[1]), float(s[2]), float(s[3]))
    return arr


def gks_create(nx, ny, Lx, Ly, gamma, Pr, mu, bc=None, options=None, stream=None):
    h = ctypes.c_void_p()
    bcs = make_bcs(bc) if bc is not None else None
    st = load().gks_create(int(nx), int(ny), float(Lx), float(Ly), float(gamma), float(Pr), float(mu), bcs,
                           ctypes.byref(options) if options is not None else None,
                           ctypes.c_void_p(stream) if stream else None, ctypes.byref(h))
    _check(None, st)
    return h


def gks_set_state(h, U, Wx=None, Wy=None, t=0.0):
    _check(h, load().gks_set_state(h, _ptr(U), _ptr(Wx), _ptr(Wy), float(t)))


def gks_set_state_device(h, U, Wx=None, Wy=None, t=0.0):
    _check(h, load().gks_set_state_device(h, _dev(U), _dev(Wx), _dev(Wy), float(t)))


def gks_step(h, CFL, dt_max=float("inf")):
    dt = ctypes.c_double(0.0)
    _check(h, load().gks_step(h, float(CFL), float(dt_max), ctypes.byref(dt)))
    return dt.value


def gks_advance(h, nsteps, CFL, t_end=float("inf")):
    _check(h, load().gks_advance(h, int(nsteps), float(CFL), float(t_end)))


def gks_sync(h):
    t = ctypes.c_double(0.0)
    n = ctypes.c_longlong(0)
    _check(h, load().gks_sync(h, ctypes.byref(t), ctypes.byref(n)))
    return t.value, n.value


def gks_get_state(h, U=None, Wx=None, Wy=None):
    t = ctypes.c_double(0.0)
    _check(h, load().gks_get_state(h, _ptr(U), _ptr(Wx), _ptr(Wy), ctypes.byref(t)))
    return t.value


def gks_get_state_device(h, U=None, Wx=None, Wy=None):
    t = ctypes.c_double(0.0)
    _check(h, load().gks_get_state_device(h, _dev(U), _dev(Wx), _dev(Wy), ctypes.byref(t)))
    return t.value


def gks_step_noalloc(nx, ny, Lx, Ly, gamma, Pr, mu, bc, options, U, Wx, Wy, U_out, Wx_out, Wy_out, CFL,
                     dt_max=float("inf"), stream=None):
    """One FP64 step between caller-owned torch CUDA tensors, using the library's static
    scratch instead of any device allocation (see gks.h).  Returns dt."""
    dt = ctypes.c_double(0.0)
    st = load().gks_step_noalloc(int(nx), int(ny), float(Lx), float(Ly), float(gamma), float(Pr), float(mu),
                                 make_bcs(bc) if bc is not None else None,
                                 ctypes.byref(options) if options is not None else None,
                                 _dev(U), _dev(Wx), _dev(Wy), float(CFL), float(dt_max), _dev(U_out), _dev(Wx_out),
                                 _dev(Wy_out), ctypes.byref(dt), ctypes.c_void_p(stream) if stream else None)
    _check(None, st)
    return dt.value


def gks_destroy(h):
    if h:
        load().gks_destroy(h)


def gks_last_error(h=None) -> str:
    return load().gks_last_error(h).decode()


def gks_launches_per_step(h) -> int:
    return load().gks_launches_per_step(h)


KERNEL_NAMES = ["recon", "flux_x", "flux_y", "update", "update2", "update3", "end"]


def gks_profile_step(h, CFL):
    """One step with per-kernel CUDA-event timing; returns {kernel name: ms}."""
    ms = (ctypes.c_float * len(KERNEL_NAMES))()
    _check(h, load().gks_profile_step(h, float(CFL), ms))
    return dict(zip(KERNEL_NAMES, list(ms)))


OP_NAMES = ["add", "mul", "div", "cmp", "sqrt", "rsqrt", "exp", "expm1", "erfc"]


def gks_face_op_count(L, R, avg, dn, dtan, dt, gamma, mu, Pr, tau_eps=0.05, tau_C=1.0, precision=GKS_FP64):
    """Arithmetic of one face evaluation, counted on the host: {op: count}."""
    L = np.ascontiguousarray(L, dtype=np.float64).reshape(6, 4)
    R = np.ascontiguousarray(R, dtype=np.float64).reshape(6, 4)
    avg = np.ascontiguousarray(avg, dtype=np.float64).reshape(2, 3, 4)
    c = (ctypes.c_longlong * 9)()
    _check(None, load().gks_face_op_count(_ptr(L), _ptr(R), _ptr(avg), dn, dtan, dt, gamma, mu, Pr, tau_eps, tau_C,
                                          int(precision), c))
    return dict(zip(OP_NAMES, list(c)))


def gks_measure_alu_peak(precision):
    t = ctypes.c_double(0.0)
    _check(None, load().gks_measure_alu_peak(int(precision), ctypes.byref(t)))
    return t.value


def gks_debug_recon(h, nx, ny):
    coef = np.zeros((4, 6, ny, nx))
    _check(h, load().gks_debug_recon(h, _ptr(coef)))
    return coef


def gks_debug_flux(h, nx, ny, dt):
    Fx, Fy = np.zeros((4, ny, nx + 1)), np.zeros((4, ny + 1, nx))
    Wx, Wy = np.zeros((4, 2, ny, nx + 1)), np.zeros((4, 2, ny + 1, nx))
    _check(h, load().gks_debug_flux(h, float(dt), _ptr(Fx), _ptr(Fy), _ptr(Wx), _ptr(Wy)))
    return Fx, Fy, Wx, Wy


class Solver:
    """One grid on the GPU.  ``problem`` is a workloads.Problem (or any object with the same
    attributes); the state is loaded at construction."""

    def __init__(self, problem, precision=GKS_FP64, stream=None, **opts):
        self.p = problem
        self.nx, self.ny = problem.nx, problem.ny
        o = gks_default_options(precision, **opts)
        self.h = gks_create(problem.nx, problem.ny, problem.Lx, problem.Ly, problem.gamma, problem.Pr, problem.mu,
                            problem.bc, o, stream)
        gks_set_state(self.h, np.ascontiguousarray(problem.U), np.ascontiguousarray(problem.Wx),
                      np.ascontiguousarray(problem.Wy), 0.0)

    def step(self, CFL, dt_max=float("inf")):
        return gks_step(self.h, CFL, dt_max)

    def advance(self, nsteps, CFL, t_end=float("inf")):
        gks_advance(self.h, nsteps, CFL, t_end)

    def sync(self):
        return gks_sync(self.h)

    def state(self):
        U = np.zeros((4, self.ny, self.nx))
        Wx = np.zeros((4, 2, self.ny, self.nx + 1))
        Wy = np.zeros((4, 2, self.ny + 1, self.nx))
        t = gks_get_state(self.h, U, Wx, Wy)
        return U, Wx, Wy, t

    def close(self):
        if self.h:
            gks_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- batched form ----

def _bcheck(b, st):
    if st != GKS_OK:
        raise GKSError(st, load().gks_batch_last_error(b).decode() if b else "")


def grid_desc(p) -> gks_grid_desc:
    d = gks_grid_desc()
    d.nx, d.ny, d.Lx, d.Ly, d.gamma, d.Pr, d.mu = p.nx, p.ny, p.Lx, p.Ly, p.gamma, p.Pr, p.mu
    bcs = make_bcs(p.bc)
    for k in range(4):
        d.bc[k] = bcs[k]
    return d


def gks_batch_create(problems, options=None, stream=None):
    arr = (gks_grid_desc * len(problems))(*[grid_desc(p) for p in problems])
    b = ctypes.c_void_p()
    st = load().gks_batch_create(len(problems), arr, ctypes.byref(options) if options is not None else None,
                                 ctypes.c_void_p(stream) if stream else None, ctypes.byref(b))
    _bcheck(None, st)
    return b


def gks_batch_set_state(b, g, U, Wx, Wy, t=0.0):
    _bcheck(b, load().gks_batch_set_state(b, int(g), _ptr(U), _ptr(Wx), _ptr(Wy), float(t)))


def gks_batch_get_state(b, g, U=None, Wx=None, Wy=None):
    t = ctypes.c_double(0.0)
    n = ctypes.c_longlong(0)
    _bcheck(b, load().gks_batch_get_state(b, int(g), _ptr(U), _ptr(Wx), _ptr(Wy), ctypes.byref(t), ctypes.byref(n)))
    return t.value, n.value


def gks_batch_step(b, nsteps, CFL):
    _bcheck(b, load().gks_batch_step(b, int(nsteps), float(CFL)))


def gks_batch_sync(b):
    lo, hi = ctypes.c_longlong(0), ctypes.c_longlong(0)
    _bcheck(b, load().gks_batch_sync(b, ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


def gks_batch_grid_info(b, g):
    t, n, s = ctypes.c_double(0.0), ctypes.c_longlong(0), ctypes.c_int(0)
    _bcheck(b, load().gks_batch_grid_info(b, int(g), ctypes.byref(t), ctypes.byref(n), ctypes.byref(s)))
    return t.value, n.value, s.value


def gks_batch_configure(b, face_tile_width, blocks_per_sm):
    _bcheck(b, load().gks_batch_configure(b, int(face_tile_width), int(blocks_per_sm)))


def gks_batch_configure_tiles(b, width_x, width_y, blocks_per_sm):
    _bcheck(b, load().gks_batch_configure_tiles(b, int(width_x), int(width_y), int(blocks_per_sm)))


def gks_batch_autotune(b, CFL, trial_steps=2):
    """Returns ((x-face tile width, y-face tile width), blocks per SM, ms per step)."""
    wx, wy, k, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_float(0.0)
    _bcheck(b, load().gks_batch_autotune(b, float(CFL), int(trial_steps), ctypes.byref(wx), ctypes.byref(wy),
                                         ctypes.byref(k), ctypes.byref(ms)))
    return (wx.value, wy.value), k.value, ms.value


BATCH_PHASES = ["open", "recon", "faces", "update", "update2", "update3"]


def gks_batch_profile(b, nsteps, CFL):
    """Mean ms per step of each phase of the persistent batch kernel over nsteps steps."""
    ms = (ctypes.c_double * len(BATCH_PHASES))()
    _bcheck(b, load().gks_batch_profile(b, int(nsteps), float(CFL), ms))
    return dict(zip(BATCH_PHASES, list(ms)))


def gks_batch_set_wait_limit(b, seconds, test_skip_block=-1):
    _bcheck(b, load().gks_batch_set_wait_limit(b, float(seconds), int(test_skip_block)))


def gks_batch_cells(b) -> int:
    return load().gks_batch_cells(b)


def gks_batch_destroy(b):
    if b:
        load().gks_batch_destroy(b)


class Batch:
    """Independent grids (workloads.Problem list) advanced together in one persistent launch."""

    def __init__(self, problems, precision=GKS_FP64, stream=None, **opts):
        self.problems = list(problems)
        self.b = gks_batch_create(self.problems, gks_default_options(precision, **opts), stream)
        for g, p in enumerate(self.problems):
            gks_batch_set_state(self.b, g, np.ascontiguousarray(p.U), np.ascontiguousarray(p.Wx),
                                np.ascontiguousarray(p.Wy), 0.0)

    def step(self, nsteps, CFL):
        gks_batch_step(self.b, nsteps, CFL)

    def sync(self):
        return gks_batch_sync(self.b)

    def state(self, g):
        p = self.problems[g]
        U = np.zeros((4, p.ny, p.nx))
        Wx = np.zeros((4, 2, p.ny, p.nx + 1))
        Wy = np.zeros((4, 2, p.ny + 1, p.nx))
        t, n = gks_batch_get_state(self.b, g, U, Wx, Wy)
        return U, Wx, Wy, t, n

    def close(self):
        if self.b:
            gks_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
