"""Oracle of the compact third-order gas-kinetic scheme (Pan & Xu, arXiv:1412.4489).

TEST INFRASTRUCTURE ONLY.  A plain FP64 C restatement of the paper (``gks_oracle2d.c``,
``gks_oracle1d.c``) and this ctypes binding.  Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import it; the CUDA library never does.

``build()`` compiles ``liboracle.so`` next to the sources with gcc -O2 (no fast-math),
with OpenMP over grid rows (used only to time the oracle on all host cores).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")
SOURCES = ["gks_oracle2d.c", "gks_oracle1d.c"]

BC_PERIODIC, BC_OUTFLOW, BC_SLIPWALL, BC_NOSLIP_ISOTHERMAL, BC_NOSLIP_ADIABATIC = 0, 1, 2, 3, 4


class Params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("mu", ctypes.c_double), ("Pr", ctypes.c_double),
                ("weno_eps", ctypes.c_double), ("weno_C", ctypes.c_double),
                ("tau_eps", ctypes.c_double), ("tau_C", ctypes.c_double), ("characteristic", ctypes.c_int)]


class BC(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("u_wall", ctypes.c_double),
                ("v_wall", ctypes.c_double), ("T_wall", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle library if it is missing or older than its sources."""
    srcs = [os.path.join(HERE, s) for s in SOURCES] + [os.path.join(HERE, "gks_oracle.h")]
    if not force and os.path.exists(LIB_PATH):
        if os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(s) for s in srcs):
            return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp", "-o", tmp]
    cmd += [os.path.join(HERE, s) for s in SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB_PATH)
        D = ctypes.c_double
        P = ctypes.POINTER
        dp = P(D)
        L.orc_moments.argtypes = [D, D, D, D, ctypes.c_int, dp, dp, dp]
        L.orc_solve_coef.argtypes = [D, D, D, D, D, dp, dp]
        L.orc_time_coefs.argtypes = [D, D, dp]
        L.orc_time_integrals.argtypes = [D, D, dp]
        L.orc_face.argtypes = [P(Params), dp, dp, dp, D, D, D, dp, dp, dp]
        L.orc_bc_image.argtypes = [P(Params), ctypes.c_int, D, D, dp, dp]
        L.orc_face_first_order.argtypes = [P(Params), dp, dp, D, D, D, dp, dp, dp]
        L.orc_recon_cell.argtypes = [P(Params), dp, dp, dp, D, D, dp]
        L.orc_char_basis.argtypes = [dp, D, dp, dp]
        L.orc_dt2d.argtypes = [P(Params), ctypes.c_int, ctypes.c_int, D, D, dp, D, D, ctypes.c_int]
        L.orc_dt2d.restype = D
        L.orc_recon2d.argtypes = [P(Params), ctypes.c_int, ctypes.c_int, D, D, P(BC), dp, dp, dp, dp]
        L.orc_flux2d.argtypes = [P(Params), ctypes.c_int, ctypes.c_int, D, D, P(BC), dp, dp, dp, D,
                                 dp, dp, dp, dp]
        L.orc_flux2d_faces.argtypes = [P(Params), ctypes.c_int, ctypes.c_int, D, D, P(BC), dp, dp, dp, D,
                                       ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp, dp]
        L.orc_step2d.argtypes = [P(Params), ctypes.c_int, ctypes.c_int, D, D, P(BC), D, D,
                                 ctypes.c_int, dp, dp, dp, dp]
        L.orc_step2d.restype = ctypes.c_int
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        L.orc1d_face.argtypes = [P(Params), dp, dp, dp, D, D, dp, dp, dp]
        L.orc1d_recon_cell.argtypes = [P(Params), dp, dp, D, dp]
        L.orc1d_dt.argtypes = [P(Params), ctypes.c_int, D, dp, D, D]
        L.orc1d_dt.restype = D
        L.orc1d_step.argtypes = [P(Params), ctypes.c_int, D, ctypes.c_int, D, D, dp, dp, dp]
        L.orc1d_step.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def params(gamma=1.4, mu=0.0, Pr=1.0, weno_eps=1e-6, weno_C=10.0, tau_eps=0.05, tau_C=1.0,
           characteristic=0) -> Params:
    return Params(gamma, mu, Pr, weno_eps, weno_C, tau_eps, tau_C, int(characteristic))


def bcs(kinds, walls=None):
    """kinds: 4 BC kinds (x-low, x-high, y-low, y-high); walls: optional 4 (u, v, T)."""
    arr = (BC * 4)()
    for k in range(4):
        u, v, T = (walls[k] if walls is not None else (0.0, 0.0, 1.0))
        arr[k] = BC(int(kinds[k]), u, v, T)
    return arr


def moments(U, V, lam, K, half):
    mu, mv, mx = np.zeros(10), np.zeros(10), np.zeros(3)
    lib().orc_moments(U, V, lam, K, half, _p(mu), _p(mv), _p(mx))
    return mu, mv, mx


def solve_coef(rho, U, V, lam, K, rhs):
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    out = np.zeros(4)
    lib().orc_solve_coef(rho, U, V, lam, K, _p(rhs), _p(out))
    return out


def time_coefs(t, tau):
    out = np.zeros(11)
    lib().orc_time_coefs(t, tau, _p(out))
    return out


def time_integrals(T, tau):
    out = np.zeros(11)
    lib().orc_time_integrals(T, tau, _p(out))
    return out


def face(P, L, R, avg, dn, dtan, dt):
    """One interface in the face frame; returns (Fhat[4], Wg[2,4], dbg[64])."""
    L = np.ascontiguousarray(L, dtype=np.float64).reshape(6, 4)
    R = np.ascontiguousarray(R, dtype=np.float64).reshape(6, 4)
    avg = np.ascontiguousarray(avg, dtype=np.float64).reshape(2, 3, 4)
    F, W, dbg = np.zeros(4), np.zeros((2, 4)), np.zeros(64)
    lib().orc_face(ctypes.byref(P), _p(L), _p(R), _p(avg), dn, dtan, dt, _p(F), _p(W), _p(dbg))
    return F, W, dbg


def face_first_order(P, L, R, dn, dtan, dt):
    """First-order evolution of the positivity fallback: L, R used as constant states."""
    L = np.ascontiguousarray(L, dtype=np.float64).reshape(6, 4)
    R = np.ascontiguousarray(R, dtype=np.float64).reshape(6, 4)
    F, W, dbg = np.zeros(4), np.zeros((2, 4)), np.zeros(64)
    lib().orc_face_first_order(ctypes.byref(P), _p(L), _p(R), dn, dtan, dt, _p(F), _p(W), _p(dbg))
    return F, W, dbg


def char_basis(w, gamma=1.4):
    """(L, R): left (rows) and right (columns) eigenvectors of the x-flux Jacobian at w."""
    L = np.zeros((4, 4))
    R = np.zeros((4, 4))
    lib().orc_char_basis(_p(np.ascontiguousarray(w, dtype=np.float64)), ctypes.c_double(gamma), _p(L), _p(R))
    return L, R


def bc_image(P, kind, u_wall_t, T_wall, inside):
    inside = np.ascontiguousarray(inside, dtype=np.float64).reshape(6, 4)
    out = np.zeros((6, 4))
    lib().orc_bc_image(ctypes.byref(P), int(kind), u_wall_t, T_wall, _p(inside), _p(out))
    return out


def recon_cell(P, nb, fx, fy, dx, dy):
    nb = np.ascontiguousarray(nb, dtype=np.float64).reshape(5, 4)
    fx = np.ascontiguousarray(fx, dtype=np.float64).reshape(4, 4)
    fy = np.ascontiguousarray(fy, dtype=np.float64).reshape(4, 4)
    out = np.zeros((4, 6))
    lib().orc_recon_cell(ctypes.byref(P), _p(nb), _p(fx), _p(fy), dx, dy, _p(out))
    return out


class State2D:
    """Host copy of a 2D state in the library's SoA layout."""

    def __init__(self, nx, ny, Lx, Ly, U, Wx, Wy):
        self.nx, self.ny, self.Lx, self.Ly = nx, ny, Lx, Ly
        self.U = np.ascontiguousarray(U, dtype=np.float64).reshape(4, ny, nx).copy()
        self.Wx = np.ascontiguousarray(Wx, dtype=np.float64).reshape(4, 2, ny, nx + 1).copy()
        self.Wy = np.ascontiguousarray(Wy, dtype=np.float64).reshape(4, 2, ny + 1, nx).copy()
        self.t = 0.0

    def copy(self):
        s = State2D(self.nx, self.ny, self.Lx, self.Ly, self.U, self.Wx, self.Wy)
        s.t = self.t
        return s


def dt2d(P, st: State2D, CFL, dt_max=np.inf, viscous_dt=0):
    return lib().orc_dt2d(ctypes.byref(P), st.nx, st.ny, st.Lx, st.Ly, _p(st.U), CFL, dt_max,
                          int(viscous_dt))


def recon2d(P, st: State2D, bc):
    coef = np.zeros((4, 6, st.ny, st.nx))
    lib().orc_recon2d(ctypes.byref(P), st.nx, st.ny, st.Lx, st.Ly, bc, _p(st.U), _p(st.Wx),
                      _p(st.Wy), _p(coef))
    return coef


def flux2d(P, st: State2D, bc, dt):
    nx, ny = st.nx, st.ny
    Fx, Fy = np.zeros((4, ny, nx + 1)), np.zeros((4, ny + 1, nx))
    Wxn, Wyn = np.zeros_like(st.Wx), np.zeros_like(st.Wy)
    lib().orc_flux2d(ctypes.byref(P), nx, ny, st.Lx, st.Ly, bc, _p(st.U), _p(st.Wx), _p(st.Wy), dt,
                     _p(Fx), _p(Fy), _p(Wxn), _p(Wyn))
    return Fx, Fy, Wxn, Wyn


def flux2d_faces(P, st: State2D, bc, dt, faces):
    """Flux and point values at listed faces [(axis, i, j), ...] of a (large) grid."""
    fl = np.ascontiguousarray(np.asarray(faces, dtype=np.int32).reshape(-1, 3))
    n = fl.shape[0]
    F, W = np.zeros((n, 4)), np.zeros((n, 2, 4))
    lib().orc_flux2d_faces(ctypes.byref(P), st.nx, st.ny, st.Lx, st.Ly, bc, _p(st.U), _p(st.Wx), _p(st.Wy), dt, n,
                           fl.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(F), _p(W))
    return F, W


def step2d(P, st: State2D, bc, CFL, dt_max=np.inf, viscous_dt=0):
    """One step in place; returns (status, dt)."""
    dt = ctypes.c_double(0.0)
    rc = lib().orc_step2d(ctypes.byref(P), st.nx, st.ny, st.Lx, st.Ly, bc, CFL, dt_max,
                          int(viscous_dt), _p(st.U), _p(st.Wx), _p(st.Wy), ctypes.byref(dt))
    if rc == 0:
        st.t += dt.value
    return rc, dt.value


def run2d(P, st: State2D, bc, CFL, t_end=None, nsteps=None, viscous_dt=0):
    """Advance by nsteps steps, or until t_end (last step clipped)."""
    k = 0
    while True:
        if nsteps is not None and k >= nsteps:
            break
        if t_end is not None and st.t >= t_end * (1 - 1e-14):
            break
        dt_max = (t_end - st.t) if t_end is not None else np.inf
        rc, _ = step2d(P, st, bc, CFL, dt_max, viscous_dt)
        if rc != 0:
            raise RuntimeError(f"oracle step {k}: non-physical state")
        k += 1
    return k


def set_threads(n: int):
    lib().orc_set_num_threads(int(n))


def num_threads() -> int:
    return lib().orc_num_threads()


# ---- 1D ----

def face1d(P, L, R, avg, dx, dt):
    L = np.ascontiguousarray(L, dtype=np.float64).reshape(3, 3)
    R = np.ascontiguousarray(R, dtype=np.float64).reshape(3, 3)
    avg = np.ascontiguousarray(avg, dtype=np.float64).reshape(2, 3)
    F, W, dbg = np.zeros(3), np.zeros(3), np.zeros(8)
    lib().orc1d_face(ctypes.byref(P), _p(L), _p(R), _p(avg), dx, dt, _p(F), _p(W), _p(dbg))
    return F, W, dbg


def step1d(P, nx, Lx, U, W, CFL, dt_max=np.inf, periodic=True):
    dt = ctypes.c_double(0.0)
    rc = lib().orc1d_step(ctypes.byref(P), nx, Lx, int(periodic), CFL, dt_max, _p(U), _p(W),
                          ctypes.byref(dt))
    return rc, dt.value


def run1d(P, nx, Lx, U, W, CFL, t_end, periodic=True):
    t = 0.0
    n = 0
    while t < t_end * (1 - 1e-14):
        rc, dt = step1d(P, nx, Lx, U, W, CFL, t_end - t, periodic)
        if rc != 0:
            raise RuntimeError("oracle 1D: non-physical state")
        t += dt
        n += 1
    return n
