"""GPU parity of the body-force collision (source term of Eq. 2.1a, q^F of
Eq. 2.4, Guo's model; include/lbm.h) against the FP64 oracle: every stencil
and collision space, uniform force and per-cell force field, pull and AA,
FP64 (1e-12) and FP32 (1e-5) storage; the fluid velocity (j + F/2) / rho of
lbm_macroscopic; the Kolmogorov steady state; and the combinations the
library refuses."""
import functools

import numpy as np
import pytest

import oracle as O
from paper_2211_02435_b300 import build as B
from paper_2211_02435_b300 import inputs as I
from paper_2211_02435_b300 import lbm as L

pytestmark = pytest.mark.gpu

TOL = {L.STORE_F64: 1e-12, L.STORE_F32: 1e-5}
DIMS = {0: (133, 37, 1), 1: (133, 6, 5), 2: (133, 6, 5)}
RATES_GEN = [1.7, 1.2, 1.3, 1.4, 1.5, 1.6]
RATES_UNIT = [1.9, 1.0, 1.0, 1.0, 1.0, 1.0]
METHODS = [  # (space, equilibrium, rates)
    (L.SPACE_POPULATIONS, L.EQ_DELTA, "srt"),
    (L.SPACE_RAW, L.EQ_DELTA, "gen"), (L.SPACE_RAW, L.EQ_ABSOLUTE, "unit"),
    (L.SPACE_CENTRAL, L.EQ_DELTA, "gen"), (L.SPACE_CENTRAL, L.EQ_ABSOLUTE, "unit"),
    (L.SPACE_CUMULANT, L.EQ_ABSOLUTE, "gen"), (L.SPACE_CUMULANT, L.EQ_ABSOLUTE, "unit"),
    (L.SPACE_TRT, L.EQ_DELTA, "trt"), (L.SPACE_RAW_WEIGHTED, L.EQ_DELTA, "gen"),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    O.build()


def rates_of(kind):
    return {"srt": [1.6] * 6, "gen": RATES_GEN, "unit": RATES_UNIT,
            "trt": [1.3, 1.0, 1.75, 1.0, 1.0, 1.0]}[kind]


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def force_of(st, kind):
    dims = DIMS[st]
    d = 2 if st == 0 else 3
    if kind == "uniform":
        return np.array([2e-5, -1e-5, 3e-5][:d])
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    F = np.zeros((d, nz, ny, nx))
    F[0] = 3e-5 * np.sin(2 * np.pi * y / ny) + 1e-5 * np.cos(2 * np.pi * x / nx)
    F[1] = -2e-5 * np.cos(2 * np.pi * x / nx)
    if d == 3:
        F[2] = 1e-5 * np.sin(2 * np.pi * (x / nx + z / nz))
    return F


@functools.lru_cache(maxsize=None)
def case(st, mi, fkind, model=0):
    space, eq, rk = METHODS[mi]
    dims = DIMS[st]
    d = 2 if st == 0 else 3
    rho, u = I.taylor_green(dims, 0.05, d=d)
    u = I.add_uniform_noise(u, 1e-3, seed=31)
    m = O.method(st, space, eq, rates_of(rk))
    df = O.init(m, dims, rho, u)
    _, w, _ = O.lattice(st)
    pert = I.random_deviations(len(w), int(np.prod(dims)), 2e-3, seed=32)
    df0 = df + (w[:, None] * pert).reshape(df.shape)
    F = force_of(st, fkind)
    ref = {n: O.step_forced(m, dims, df0, F, n, model=model) for n in (3, 4)}
    return m, dims, df0, F, ref


@pytest.mark.parametrize("fkind", ["uniform", "field"])
@pytest.mark.parametrize("streaming", L.STREAMING_PATTERNS)
@pytest.mark.parametrize("storage", [L.STORE_F64, L.STORE_F32])
@pytest.mark.parametrize("mi", range(len(METHODS)),
                         ids=[f"sp{m[0]}eq{m[1]}{m[2]}" for m in METHODS])
@pytest.mark.parametrize("st", [0, 1, 2], ids=["D2Q9", "D3Q19", "D3Q27"])
def test_forced_step_parity(st, mi, storage, streaming, fkind):
    m, dims, df0, F, ref = case(st, mi, fkind)
    space, eq, rk = METHODS[mi]
    with L.Lattice(st, space, eq, storage, streaming, rates_of(rk), dims) as lat:
        if fkind == "uniform":
            lat.set_force(F)
        else:
            lat.set_force_field(F)
        lat.set_populations(df0)
        done = 0
        for n in (3, 4):
            lat.step(n - done)
            done = n
            assert rel_linf(lat.get_populations(), ref[n]) < TOL[storage], n
            rho_r, u_r = O.macroscopic_forced(m, dims, ref[n], F)
            rho_g, u_g = lat.macroscopic()
            assert rel_linf(u_g, u_r) < TOL[storage]


HE_METHODS = [i for i, m in enumerate(METHODS) if m[0] != L.SPACE_CUMULANT]


@pytest.mark.parametrize("fkind", ["uniform", "field"])
@pytest.mark.parametrize("streaming", [L.PULL, L.ESOTERIC_TWIST, L.ESOTERIC_PULL, L.ESOTERIC_PUSH])
@pytest.mark.parametrize("storage", [L.STORE_F64, L.STORE_F32])
@pytest.mark.parametrize("mi", HE_METHODS, ids=[f"sp{METHODS[i][0]}eq{METHODS[i][1]}{METHODS[i][2]}"
                                                for i in HE_METHODS])
@pytest.mark.parametrize("st", [0, 1, 2], ids=["D2Q9", "D3Q19", "D3Q27"])
def test_he_forced_step_parity(st, mi, storage, streaming, fkind):
    m, dims, df0, F, ref = case(st, mi, fkind, O.FORCE_HE)
    space, eq, rk = METHODS[mi]
    with L.Lattice(st, space, eq, storage, streaming, rates_of(rk), dims) as lat:
        lat.set_force_model(L.FORCE_HE)
        if fkind == "uniform":
            lat.set_force(F)
        else:
            lat.set_force_field(F)
        lat.set_populations(df0)
        lat.step(3)
        assert rel_linf(lat.get_populations(), ref[3]) < TOL[storage]


def test_he_model_refused_for_cumulants():
    with L.Lattice(2, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, L.STORE_F32, L.PULL, RATES_UNIT,
                   (8, 8, 8)) as lat:
        with pytest.raises(L.LBMError) as e:
            lat.set_force_model(L.FORCE_HE)
        assert e.value.code == -2
        with pytest.raises(L.LBMError) as e:
            lat.set_force_model(7)
        assert e.value.code == -1


def test_removing_the_force_restores_the_plain_step():
    st, dims = 2, DIMS[2]
    rho, u = I.taylor_green(dims, 0.05)
    out = []
    for forced in (False, True):
        with L.Lattice(st, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, L.STORE_F32, L.PULL, RATES_UNIT,
                       dims) as lat:
            if forced:
                lat.set_force([1e-5, 0, 0])
                lat.set_force_field(force_of(st, "field"))
                lat.set_force(None)
                lat.set_force_field(None)
            lat.init_velocity(rho.reshape(-1), u.reshape(-1))
            lat.step(3)
            out.append(lat.get_populations())
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("space", [L.SPACE_POPULATIONS, L.SPACE_RAW, L.SPACE_CENTRAL,
                                   L.SPACE_CUMULANT])
def test_kolmogorov_flow_steady_state(space):
    """F_x = F0 sin(k y) on a 4 x 64 x 2 D3Q27 lattice, FP64: the steady
    u_x = F0 / (nu k^2) sin(k y) within the lattice's O(k^2) error."""
    nx, ny, nz = 4, 64, 2
    k = 2 * np.pi / ny
    omega = 1.6
    nu = (1.0 / omega - 0.5) / 3.0
    F0 = 1e-6
    F = np.zeros((3, nz, ny, nx))
    F[0] = F0 * np.sin(k * np.arange(ny))[None, :, None]
    with L.Lattice(2, space, L.EQ_ABSOLUTE, L.STORE_F64, L.PULL, [omega] + [1.0] * 5,
                   (nx, ny, nz)) as lat:
        lat.set_force_field(F)
        lat.init_velocity(np.ones(nx * ny * nz), np.zeros(3 * nx * ny * nz))
        lat.step(int(14 / (nu * k * k)))
        _, u = lat.macroscopic()
    u = u.reshape(3, nz, ny, nx)
    amp = F0 / (nu * k * k)
    err = np.abs(u[0] - amp * np.sin(k * np.arange(ny))[None, :, None]).max() / amp
    assert err < 3e-3, err  # O(k^2): ~0.1 % at L = 64
    assert np.abs(u[1:]).max() < 1e-6 * amp


def test_force_refusals():
    dims = (16, 8, 4)
    for storage, arith in ((L.STORE_F16_DELTA, 0), (L.STORE_BF16_DELTA, 0),
                           (L.STORE_F64_ABSOLUTE, 0), (L.STORE_F64, L.ARITH_AS_WRITTEN)):
        with L.Lattice(2, L.SPACE_CENTRAL, L.EQ_ABSOLUTE, storage, L.PULL, RATES_UNIT, dims,
                       arithmetic=arith) as lat:
            with pytest.raises(L.LBMError) as e:
                lat.set_force([1e-5, 0, 0])
            assert e.value.code == -2
    with L.Lattice(2, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, L.STORE_F32, L.PULL, RATES_UNIT,
                   dims) as lat:
        with pytest.raises(L.LBMError) as e:
            lat.set_force([np.nan, 0, 0])
        assert e.value.code == -1
        lat.set_force([1e-5, 0, 0])
        with pytest.raises(L.LBMError) as e:  # the staged kernel has no force
            lat.set_step_kernel(L.STEP_STAGED)
        assert e.value.code == -2
        w = L.ClosureWeights()
        w.scale[:] = [1.0] * 7
        with pytest.raises(L.LBMError) as e:  # nor the learned closure
            lat.set_closure(w)
        assert e.value.code == -2
