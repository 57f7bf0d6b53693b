"""Plain FP64 CPU oracle for the zero-centered MRT lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
product path (``paper_2211_02435_b300``) never imports it and shares no code
with it.

The arithmetic lives in ``lbm_oracle.c`` (plain C, double precision, explicit
moment matrices); this module only compiles it with gcc and marshals numpy
arrays through ctypes.  Function-by-function citations of the paper are in the
C header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblbm_oracle.so")

D2Q9, D3Q19, D3Q27 = 0, 1, 2
SPACE_POPULATIONS, SPACE_RAW, SPACE_CENTRAL, SPACE_CUMULANT, SPACE_TRT = 0, 1, 2, 3, 4
SPACE_RAW_WEIGHTED, SPACE_NONE = 5, 6
EQ_DELTA, EQ_ABSOLUTE, EQ_DISCRETE2 = 0, 1, 2
GROUP_CONSERVED, GROUP_SHEAR, GROUP_BULK = -1, 0, 1
Q_OF = {D2Q9: 9, D3Q19: 19, D3Q27: 27}


class OracleError(RuntimeError):
    pass


class Method(ctypes.Structure):
    _fields_ = [
        ("stencil", ctypes.c_int),
        ("space", ctypes.c_int),
        ("equilibrium", ctypes.c_int),
        ("rates", ctypes.c_double * 6),
    ]


def method(stencil, space, equilibrium, rates):
    r = list(rates) + [1.0] * (6 - len(rates))
    return Method(stencil, space, equilibrium, (ctypes.c_double * 6)(*r))


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) into ``liblbm_oracle.so``."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC[:-1] + "h")):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-Wall", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER
        d, i32, i64 = P(ctypes.c_double), P(ctypes.c_int), P(ctypes.c_int64)
        m = P(Method)
        L.lbm_oracle_lattice.argtypes = [ctypes.c_int, i32, i32, i32, d, i32]
        L.lbm_oracle_matrices.argtypes = [ctypes.c_int, d, d, d, d, i32]
        L.lbm_oracle_central_matrix.argtypes = [ctypes.c_int, d, d]
        L.lbm_oracle_weighted_basis.argtypes = [ctypes.c_int, d]
        L.lbm_oracle_cumulants.argtypes = [ctypes.c_int, d, d]
        L.lbm_oracle_moments_from_cumulants.argtypes = [ctypes.c_int, d, d]
        L.lbm_oracle_cumulant_of.argtypes = [d, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.lbm_oracle_cumulant_of.restype = ctypes.c_double
        L.lbm_oracle_collide.argtypes = [m, ctypes.c_int64, d, d]
        L.lbm_oracle_equilibrium.argtypes = [m, ctypes.c_int64, d, d, d]
        L.lbm_oracle_init.argtypes = [m, i64, d, d, d]
        L.lbm_oracle_step.argtypes = [m, i64, d, ctypes.c_int64, ctypes.c_int]
        L.lbm_oracle_macroscopic.argtypes = [m, i64, d, d, d]
        L.lbm_oracle_collide_forced.argtypes = [m, ctypes.c_int64, d, d, ctypes.c_int, d]
        L.lbm_oracle_step_forced.argtypes = [m, i64, d, d, ctypes.c_int, ctypes.c_int64,
                                             ctypes.c_int]
        L.lbm_oracle_macroscopic_forced.argtypes = [m, i64, d, d, d, d]
        L.lbm_oracle_swe_equilibrium.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                 d, d]
        L.lbm_oracle_swe_collide.argtypes = [m, ctypes.c_double, ctypes.c_int64, d, d]
        L.lbm_oracle_swe_init.argtypes = [m, ctypes.c_double, i64, d, d, d]
        L.lbm_oracle_swe_step.argtypes = [m, ctypes.c_double, i64, d, ctypes.c_int64,
                                          ctypes.c_int]
        L.lbm_oracle_closure_features.argtypes = [ctypes.c_int, d, ctypes.c_double, d]
        L.lbm_oracle_closure_mlp.argtypes = [d, d, d, d, d]
        L.lbm_oracle_closure_step.argtypes = [m, i64, d, d, d, d, ctypes.c_int]
        L.lbm_oracle_closure_loss.argtypes = [m, i64, d, d, d, d, d, ctypes.c_int]
        L.lbm_oracle_closure_loss.restype = ctypes.c_double
        L.lbm_oracle_closure_rollout_loss.argtypes = [m, i64, d, ctypes.c_int, d, d, d,
                                                      ctypes.c_int]
        L.lbm_oracle_closure_rollout_loss.restype = ctypes.c_double
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _check(rc):
    if rc != 0:
        raise OracleError(f"oracle call failed with code {rc}")


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def lattice(stencil):
    """(xi[q,3] int, w[q], expo[q,3]) in the documented velocity order."""
    q = Q_OF[stencil]
    xi = np.zeros((q, 3), np.int32)
    ex = np.zeros((q, 3), np.int32)
    w = np.zeros(q)
    _check(lib().lbm_oracle_lattice(stencil, None, None, _ip(xi), _dp(w), _ip(ex)))
    return xi.astype(np.int64), w, ex.astype(np.int64)


def weighted_basis(stencil):
    """Weighted orthogonal raw basis Pw (q x q) of WO-MRT."""
    q = Q_OF[stencil]
    out = np.zeros((q, q))
    _check(lib().lbm_oracle_weighted_basis(stencil, _dp(out)))
    return out


def matrices(stencil):
    """dict with M, Minv, Praw, Pcm (q x q) and group (q,)."""
    q = Q_OF[stencil]
    out = {k: np.zeros((q, q)) for k in ("M", "Minv", "Praw", "Pcm")}
    g = np.zeros(q, np.int32)
    _check(lib().lbm_oracle_matrices(stencil, _dp(out["M"]), _dp(out["Minv"]),
                                     _dp(out["Praw"]), _dp(out["Pcm"]), _ip(g)))
    out["group"] = g.astype(np.int64)
    return out


def central_matrix(stencil, u):
    q = Q_OF[stencil]
    K = np.zeros((q, q))
    _check(lib().lbm_oracle_central_matrix(stencil, _dp(_f64(u)), _dp(K)))
    return K


def cumulants(stencil, f):
    q = Q_OF[stencil]
    out = np.zeros(q)
    _check(lib().lbm_oracle_cumulants(stencil, _dp(_f64(f)), _dp(out)))
    return out


def moments_from_cumulants(stencil, c):
    q = Q_OF[stencil]
    out = np.zeros(q)
    _check(lib().lbm_oracle_moments_from_cumulants(stencil, _dp(_f64(c)), _dp(out)))
    return out


def cumulant_of(mu, a, b, c):
    """Joint cumulant for exponents (a,b,c) from normalized raw moments mu[3,3,3]."""
    return lib().lbm_oracle_cumulant_of(_dp(_f64(mu).reshape(27)), a, b, c)


def collide(m, df):
    """Collide cells; df is [ncells, q] (or [q]) of zero-centered deviations."""
    df = _f64(df)
    flat = df.reshape(-1, Q_OF[m.stencil])
    out = np.empty_like(flat)
    _check(lib().lbm_oracle_collide(ctypes.byref(m), flat.shape[0], _dp(flat), _dp(out)))
    return out.reshape(df.shape)


FORCE_GUO, FORCE_HE = 0, 1


def collide_forced(m, df, force, model=FORCE_GUO):
    """Collide cells under a body force (Guo or He; see lbm_oracle.h):
    df [ncells, q], force [ncells, 3] (or [3] for one cell)."""
    df = _f64(df)
    flat = df.reshape(-1, Q_OF[m.stencil])
    F = _f64(np.broadcast_to(np.asarray(force, dtype=np.float64).reshape(-1, 3),
                             (flat.shape[0], 3))).copy()
    out = np.empty_like(flat)
    _check(lib().lbm_oracle_collide_forced(ctypes.byref(m), flat.shape[0], _dp(flat), _dp(F),
                                           int(model), _dp(out)))
    return out.reshape(df.shape)


def equilibrium(m, rho, u):
    """Method equilibrium deviations for rho[n], u[n,3] -> [n, q]."""
    rho = _f64(np.atleast_1d(rho))
    u = _f64(np.atleast_2d(u))
    out = np.empty((rho.size, Q_OF[m.stencil]))
    _check(lib().lbm_oracle_equilibrium(ctypes.byref(m), rho.size, _dp(rho), _dp(u), _dp(out)))
    return out


def _dims(dims):
    d = list(dims) + [1] * (3 - len(dims))
    return np.asarray(d, dtype=np.int64)


def init(m, dims, rho, u):
    """SoA pre-collision state df[q, Nz, Ny, Nx] at equilibrium with rho, u.

    rho is [Nz, Ny, Nx]; u is [3 (or 2), Nz, Ny, Nx].
    """
    dm = _dims(dims)
    N = int(np.prod(dm))
    df = np.empty((Q_OF[m.stencil], N))
    u = _f64(u).reshape(-1, N)
    _check(lib().lbm_oracle_init(ctypes.byref(m), dm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 _dp(_f64(rho).reshape(N)), _dp(u), _dp(df)))
    return df.reshape(Q_OF[m.stencil], dm[2], dm[1], dm[0])


def step(m, dims, df, nsteps, nthreads=0):
    """Advance the SoA pre-collision state df[q, ...] by nsteps (returns a copy)."""
    dm = _dims(dims)
    out = _f64(df).copy()
    _check(lib().lbm_oracle_step(ctypes.byref(m), dm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 _dp(out), int(nsteps), int(nthreads)))
    return out


def _force_field(m, dims, force):
    """Force as SoA [D, N] (D = 2 for D2Q9); force may be a constant vector."""
    dm = _dims(dims)
    N = int(np.prod(dm))
    d = 2 if m.stencil == D2Q9 else 3
    F = np.asarray(force, dtype=np.float64)
    if F.size == 3 or F.size == d:
        F = np.repeat(F.reshape(-1)[:d, None], N, axis=1)
    return np.ascontiguousarray(F.reshape(d, N))


def step_forced(m, dims, df, force, nsteps, nthreads=0, model=FORCE_GUO):
    """step() under a time-constant body force (a vector or a [D, ...] field)."""
    dm = _dims(dims)
    out = _f64(df).copy()
    F = _force_field(m, dims, force)
    _check(lib().lbm_oracle_step_forced(ctypes.byref(m),
                                        dm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                        _dp(out), _dp(F), int(model), int(nsteps),
                                        int(nthreads)))
    return out


def macroscopic_forced(m, dims, df, force):
    """(rho, u) with the fluid velocity u = (j + F/2) / rho of a forced state."""
    dm = _dims(dims)
    N = int(np.prod(dm))
    d = 2 if m.stencil == D2Q9 else 3
    rho = np.empty(N)
    u = np.zeros((d, N))
    F = _force_field(m, dims, force)
    _check(lib().lbm_oracle_macroscopic_forced(
        ctypes.byref(m), dm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(_f64(df)),
        _dp(F), _dp(rho), _dp(u)))
    shp = (dm[2], dm[1], dm[0])
    return rho.reshape(shp), u.reshape((d,) + shp)


def macroscopic(m, dims, df):
    """(rho[Nz,Ny,Nx], u[3,Nz,Ny,Nx]) of the SoA state (u has 2 rows in 2-D)."""
    dm = _dims(dims)
    N = int(np.prod(dm))
    d = 2 if m.stencil == D2Q9 else 3
    rho = np.empty(N)
    u = np.zeros((d, N))
    _check(lib().lbm_oracle_macroscopic(ctypes.byref(m), dm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                        _dp(_f64(df)), _dp(rho), _dp(u)))
    shp = (dm[2], dm[1], dm[0])
    return rho.reshape(shp), u.reshape((d,) + shp)


# ------------------------------------------------------------ shallow water
def swe_equilibrium(space, g, h, u):
    """Absolute D2Q9 equilibrium populations [9] of the shallow-water method
    (SPACE_CENTRAL: Zhou's discrete f_eq; SPACE_CUMULANT: Maxwellian with
    c_s^2 = g h / 2) at depth h and velocity u[2]."""
    out = np.zeros(9)
    _check(lib().lbm_oracle_swe_equilibrium(int(space), float(g), float(h),
                                            _dp(_f64(np.asarray(u, dtype=np.float64)[:2])), _dp(out)))
    return out


def swe_collide(m, g, df):
    df = _f64(df)
    flat = df.reshape(-1, 9)
    out = np.empty_like(flat)
    _check(lib().lbm_oracle_swe_collide(ctypes.byref(m), float(g), flat.shape[0], _dp(flat),
                                        _dp(out)))
    return out.reshape(df.shape)


def swe_init(m, g, dims, h, u):
    dm = _dims(dims)
    N = int(np.prod(dm))
    df = np.empty((9, N))
    _check(lib().lbm_oracle_swe_init(ctypes.byref(m), float(g),
                                     dm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                     _dp(_f64(h).reshape(N)), _dp(_f64(u).reshape(-1, N)),
                                     _dp(df)))
    return df.reshape(9, dm[2], dm[1], dm[0])


def swe_step(m, g, dims, df, nsteps, nthreads=0):
    dm = _dims(dims)
    out = _f64(df).copy()
    _check(lib().lbm_oracle_swe_step(ctypes.byref(m), float(g),
                                     dm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                     _dp(out), int(nsteps), int(nthreads)))
    return out


# ------------------------------------------------------------ learned closure
CLOSURE_NPARAM = 1444


def closure_features(stencil, df, omega_shear):
    """Raw features [7] of one cell's zero-centered populations."""
    out = np.zeros(7)
    _check(lib().lbm_oracle_closure_features(stencil, _dp(_f64(df)), float(omega_shear), _dp(out)))
    return out


def closure_mlp(params, shift, scale, raw):
    """Per-cell rates of orders 3..6 from raw features."""
    om = np.zeros(4)
    _check(lib().lbm_oracle_closure_mlp(_dp(_f64(params)), _dp(_f64(shift)), _dp(_f64(scale)),
                                        _dp(_f64(raw)), _dp(om)))
    return om


def closure_step(m, dims, df, params, shift, scale, nthreads=0):
    dm = _dims(dims)
    out = _f64(df).copy()
    _check(lib().lbm_oracle_closure_step(ctypes.byref(m), dm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                         _dp(out), _dp(_f64(params)), _dp(_f64(shift)),
                                         _dp(_f64(scale)), int(nthreads)))
    return out


def closure_loss(m, dims, df_s, df_t, params, shift, scale, nthreads=0):
    dm = _dims(dims)
    return lib().lbm_oracle_closure_loss(ctypes.byref(m), dm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                         _dp(_f64(df_s)), _dp(_f64(df_t)), _dp(_f64(params)),
                                         _dp(_f64(shift)), _dp(_f64(scale)), int(nthreads))


def closure_rollout_loss(m, dims, states, params, shift, scale, nthreads=0):
    """K-step rollout loss from states[0] against targets states[1..K]
    (states: K + 1 SoA populations, stacked along the first axis)."""
    dm = _dims(dims)
    st = np.ascontiguousarray(np.asarray(states, dtype=np.float64))
    K = st.shape[0] - 1
    return lib().lbm_oracle_closure_rollout_loss(
        ctypes.byref(m), dm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(st), int(K),
        _dp(_f64(params)), _dp(_f64(shift)), _dp(_f64(scale)), int(nthreads))
