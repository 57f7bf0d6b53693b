"""GPU parity: the CUDA stream-collide path (through the C ABI) against the
FP64 CPU oracle, element by element, on seeded inputs.

Tolerances (relative L-infinity over the zero-centered populations, and over
the velocity): 1e-12 for FP64 storage, 1e-5 for FP32 storage.  FP16/BF16
delta storage is measured against the oracle and held to a bound derived
from its rounding unit (see test_half_storage_error_bound).

Lattices are non-cubic, span two x-blocks with a ragged tail (Nx = 133 with
128-thread blocks) and are run for an odd and an even number of steps, so
both AA parities are read out.
"""
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
RATES_REG = [1.9, 1.0, 1.0, 1.0, 1.0, 1.0]
METHODS = [  # (space, equilibrium, regularised)
    (L.SPACE_POPULATIONS, L.EQ_DELTA, False),
    (L.SPACE_RAW, L.EQ_DELTA, False), (L.SPACE_RAW, L.EQ_DELTA, True),
    (L.SPACE_RAW, L.EQ_ABSOLUTE, False),
    (L.SPACE_CENTRAL, L.EQ_DELTA, False), (L.SPACE_CENTRAL, L.EQ_ABSOLUTE, True),
    (L.SPACE_CENTRAL, L.EQ_ABSOLUTE, False),
    (L.SPACE_CUMULANT, L.EQ_ABSOLUTE, False), (L.SPACE_CUMULANT, L.EQ_ABSOLUTE, True),
    (L.SPACE_TRT, L.EQ_DELTA, False), (L.SPACE_TRT, L.EQ_ABSOLUTE, False),
    (L.SPACE_RAW_WEIGHTED, L.EQ_DELTA, False), (L.SPACE_RAW_WEIGHTED, L.EQ_ABSOLUTE, True),
]
RATES_TRT = [1.3, 1.0, 1.75, 1.0, 1.0, 1.0]  # w+ (even part), w- (odd part) in slot 2


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    O.build()


def rates_of(space, reg):
    if space == L.SPACE_POPULATIONS:
        return [1.6] * 6
    if space == L.SPACE_TRT:
        return RATES_TRT
    return RATES_REG if reg else RATES_GEN


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@functools.lru_cache(maxsize=None)
def initial_state(st, space, eq, reg):
    """Seeded non-equilibrium start: the method's equilibrium of a noisy
    Taylor-Green field plus a random deviation on every population."""
    dims = DIMS[st]
    d = 2 if st == 0 else 3
    rho, u = I.taylor_green(dims, 0.05, d=d)
    u = I.add_uniform_noise(u, 1e-3, seed=11)
    m = O.method(st, space, eq, rates_of(space, reg))
    df = O.init(m, dims, rho, u)
    _, w, _ = O.lattice(st)
    pert = I.random_deviations(len(w), int(np.prod(dims)), 2e-3, seed=12)
    return m, dims, df + (w[:, None] * pert).reshape(df.shape)


@functools.lru_cache(maxsize=None)
def oracle_run(st, space, eq, reg, nsteps):
    m, dims, df0 = initial_state(st, space, eq, reg)
    return O.step(m, dims, df0, nsteps)


def gpu_lattice(st, space, eq, reg, storage, streaming):
    return L.Lattice(st, space, eq, storage, streaming, rates_of(space, reg), DIMS[st])


@pytest.mark.parametrize("streaming", L.STREAMING_PATTERNS)
@pytest.mark.parametrize("storage", [L.STORE_F64, L.STORE_F32])
@pytest.mark.parametrize("method", METHODS, ids=lambda m: f"sp{m[0]}eq{m[1]}reg{int(m[2])}")
@pytest.mark.parametrize("st", [0, 1, 2], ids=["D2Q9", "D3Q19", "D3Q27"])
def test_step_parity(st, method, storage, streaming):
    space, eq, reg = method
    _, dims, df0 = initial_state(st, space, eq, reg)
    m, _, _ = initial_state(st, space, eq, reg)
    with gpu_lattice(st, space, eq, reg, storage, streaming) as lat:
        lat.set_populations(df0)
        got0 = lat.get_populations()
        tol0 = 0.0 if storage == L.STORE_F64 else 1e-7
        assert rel_linf(got0, df0) <= tol0
        done = 0
        for n in (3, 4):
            lat.step(n - done)
            done = n
            ref = oracle_run(st, space, eq, reg, n)
            got = lat.get_populations()
            assert rel_linf(got, ref) < TOL[storage], n
            rho_r, u_r = O.macroscopic(m, dims, ref)
            rho_g, u_g = lat.macroscopic()
            assert rel_linf(u_g, u_r) < TOL[storage]
            assert rel_linf(rho_g - 1, rho_r - 1) < TOL[storage]
            assert lat.time() == (n, (n % 2) if streaming != L.PULL else 0)


@pytest.mark.parametrize("space", [L.SPACE_RAW, L.SPACE_CENTRAL, L.SPACE_CUMULANT])
@pytest.mark.parametrize("st", [0, 1, 2])
@pytest.mark.parametrize("streaming", L.STREAMING_PATTERNS)
def test_init_velocity_is_the_method_equilibrium(st, space, streaming):
    eq = L.EQ_DELTA if space == L.SPACE_RAW else L.EQ_ABSOLUTE
    dims = DIMS[st]
    d = 2 if st == 0 else 3
    rho, u = I.taylor_green(dims, 0.08, d=d)
    u = I.add_uniform_noise(u, 1e-2, seed=3)
    m = O.method(st, space, eq, RATES_GEN)
    ref = O.init(m, dims, rho, u)
    with L.Lattice(st, space, eq, L.STORE_F64, streaming, RATES_GEN, dims) as lat:
        lat.init_velocity(rho.reshape(-1), u.reshape(-1))
        assert rel_linf(lat.get_populations(), ref) < 1e-13
        r, uu = lat.macroscopic()
        assert np.abs(uu - u).max() < 1e-15
        assert np.abs(r - rho).max() < 1e-15
        # equilibrium is a fixed point of the collision: one step = streaming
        lat.step(1)
        shifted = O.step(O.method(st, O.SPACE_NONE, 0, [1.0] * 6), dims, ref, 1)
        assert rel_linf(lat.get_populations(), shifted) < 1e-12


@pytest.mark.parametrize("storage", [L.STORE_F32, L.STORE_F64])
def test_pull_and_aa_are_bitwise_identical(storage):
    """Pull, AA and the three esoteric patterns run the same per-cell
    arithmetic; odd and even step counts end on both in-place parities."""
    st, space, eq, reg = 2, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, False
    _, dims, df0 = initial_state(st, space, eq, reg)
    for n in (4, 5):
        out = []
        for streaming in L.STREAMING_PATTERNS:
            with gpu_lattice(st, space, eq, reg, storage, streaming) as lat:
                lat.set_populations(df0)
                lat.step(n)
                out.append(lat.get_populations())
        for k in range(1, len(out)):
            assert np.array_equal(out[0], out[k]), (n, k)


@pytest.mark.parametrize("streaming", L.STREAMING_PATTERNS)
def test_checkpoint_resume_is_bitwise(streaming):
    st, space, eq, reg = 1, L.SPACE_RAW, L.EQ_DELTA, False
    _, dims, df0 = initial_state(st, space, eq, reg)
    with gpu_lattice(st, space, eq, reg, L.STORE_F32, streaming) as a:
        a.set_populations(df0)
        a.step(3)
        state = a.get_state()
        a.step(4)
        straight = a.get_populations()
    with gpu_lattice(st, space, eq, reg, L.STORE_F32, streaming) as b:
        b.set_state(state)
        assert b.time() == (3, 1 if streaming != L.PULL else 0)
        b.step(4)
        assert np.array_equal(b.get_populations(), straight)
    # a state of another configuration is refused
    with L.Lattice(st, space, eq, L.STORE_F64, streaming, RATES_GEN, dims) as c:
        with pytest.raises(L.LBMError) as e:
            c.set_state(state)
        assert e.value.code == -7


def test_invariants_match_oracle_and_conserve():
    st, space, eq, reg = 2, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, False
    m, dims, df0 = initial_state(st, space, eq, reg)
    with gpu_lattice(st, space, eq, reg, L.STORE_F64, L.PULL) as lat:
        lat.set_populations(df0)
        inv0 = lat.invariants()
        lat.step(4)
        inv = lat.invariants()
    ref = oracle_run(st, space, eq, reg, 4)
    rho, u = O.macroscopic(m, dims, ref)
    assert inv["cells"] == np.prod(dims) and inv["nonfinite"] == 0
    assert abs(inv["mass_dev"] - (rho - 1).sum()) < 1e-12
    for k, d in (("jx", 0), ("jy", 1), ("jz", 2)):
        assert abs(inv[k] - (rho * u[d]).sum()) < 1e-12
        assert abs(inv[k] - inv0[k]) < 1e-12  # momentum conservation
    assert abs(inv["mass_dev"] - inv0["mass_dev"]) < 1e-12
    e_ref = 0.5 * (rho * (u ** 2).sum(0)).sum()
    assert abs(inv["energy"] - e_ref) < 1e-12 * e_ref
    assert abs(inv["max_u"] - np.sqrt((u ** 2).sum(0)).max()) < 1e-14


def test_nonfinite_population_is_reported():
    st = 1
    dims = DIMS[st]
    with L.Lattice(st, L.SPACE_RAW, L.EQ_DELTA, L.STORE_F32, L.AA, RATES_GEN, dims) as lat:
        df = np.zeros((19, int(np.prod(dims))))
        df[4, 17] = np.nan  # host-made failure: a poisoned population
        lat.set_populations(df)
        with pytest.raises(L.LBMError) as e:
            lat.invariants()
        assert e.value.code == -6
        inv = lat.invariants(check=False)
        assert inv["nonfinite"] == 1


@pytest.mark.parametrize("streaming", [L.PULL, L.AA])
def test_divergence_watch_stops_the_step(streaming):
    """A poisoned population (host-made) spreads through the collision; the
    step call with the watch on returns DIVERGED at the first watched step,
    and without the watch it runs on."""
    st = 1
    dims = DIMS[st]
    df = np.zeros((19, int(np.prod(dims))))
    df[4, 17] = np.nan
    with L.Lattice(st, L.SPACE_RAW, L.EQ_DELTA, L.STORE_F32, streaming, RATES_GEN, dims) as lat:
        lat.set_populations(df)
        lat.step(3)  # watch off
        assert lat.time()[0] == 3
        lat.set_divergence_check(2)
        with pytest.raises(L.LBMError) as e:
            lat.step(5)
        assert e.value.code == -6
        assert lat.time()[0] == 4  # stopped at the first watched step
        lat.set_divergence_check(0)
        lat.step(2)
        assert lat.time()[0] == 6
    with L.Lattice(st, L.SPACE_RAW, L.EQ_DELTA, L.STORE_F32, streaming, RATES_GEN, dims) as lat:
        lat.set_populations(np.zeros_like(df))
        lat.set_divergence_check(1)
        lat.step(4)  # finite: no error
        assert lat.time()[0] == 4


def test_device_pointer_path_matches_host_path():
    torch = pytest.importorskip("torch")
    st, space, eq, reg = 2, L.SPACE_CENTRAL, L.EQ_ABSOLUTE, True
    _, dims, df0 = initial_state(st, space, eq, reg)
    N = int(np.prod(dims))
    with gpu_lattice(st, space, eq, reg, L.STORE_F32, L.AA) as lat:
        lat.set_stream(torch.cuda.current_stream())
        lat.set_populations(torch.from_numpy(df0.reshape(-1).copy()).cuda())
        lat.step(3)
        dev = torch.empty(27 * N, dtype=torch.float64, device="cuda")
        lat.get_populations(dev)
        r = torch.empty(N, dtype=torch.float64, device="cuda")
        uu = torch.empty(3 * N, dtype=torch.float64, device="cuda")
        lat.macroscopic(r, uu)
        torch.cuda.synchronize()
        host = lat.get_populations()
        rh, uh = lat.macroscopic()
    assert np.array_equal(dev.cpu().numpy().reshape(host.shape), host)
    assert np.array_equal(uu.cpu().numpy().reshape(uh.shape), uh)
    assert np.array_equal(r.cpu().numpy().reshape(rh.shape), rh)


@pytest.mark.parametrize("storage,p", [(L.STORE_F16_DELTA, 10), (L.STORE_BF16_DELTA, 7)])
@pytest.mark.parametrize("space", [L.SPACE_CENTRAL, L.SPACE_CUMULANT])
@pytest.mark.parametrize("streaming", L.STREAMING_PATTERNS)
def test_half_storage_error_bound(storage, p, space, streaming):
    """FP16 / BF16 delta storage: every store rounds each scaled deviation
    to p explicit mantissa bits, an error of at most 2^-(p+1) of |df_i|;
    with the collision a contraction on non-conserved parts, n steps stay
    within (n + 1) * 2^-(p+1) * max|df| (the +1 for the initial encode)."""
    st, eq, reg = 2, L.EQ_ABSOLUTE, True
    m, dims, df0 = initial_state(st, space, eq, reg)
    n = 4
    with gpu_lattice(st, space, eq, reg, storage, streaming) as lat:
        lat.set_populations(df0)
        lat.step(n)
        got = lat.get_populations()
        rho_g, u_g = lat.macroscopic()
    ref = oracle_run(st, space, eq, reg, n)
    bound = (n + 1) * 2.0 ** -(p + 1)
    err = rel_linf(got, ref)
    assert err < bound, (err, bound)
    _, u_r = O.macroscopic(m, dims, ref)
    assert rel_linf(u_g, u_r) < 4 * bound


def test_taylor_green_config_d3q19_omrt_fp64():
    """32^3 D3Q19 O-MRT (R-) Taylor-Green vortex, u0 = 0.05, nu = 0.01,
    FP64, 100 steps: GPU equals the oracle to 1e-12, pull and AA."""
    L_, u0, nu, steps = 32, 0.05, 0.01, 100
    rates = [I.shear_viscosity_rate(nu)] + [1.0] * 5
    dims = (L_, L_, L_)
    rho, u = I.taylor_green(dims, u0)
    m = O.method(1, O.SPACE_RAW, O.EQ_DELTA, rates)
    ref = O.step(m, dims, O.init(m, dims, rho, u), steps)
    rho_r, u_r = O.macroscopic(m, dims, ref)
    for streaming in (L.PULL, L.AA):
        with L.Lattice(1, L.SPACE_RAW, L.EQ_DELTA, L.STORE_F64, streaming, rates, dims) as lat:
            lat.init_velocity(rho.reshape(-1), u.reshape(-1))
            lat.step(steps)
            assert rel_linf(lat.get_populations(), ref) < 1e-12
            _, u_g = lat.macroscopic()
            assert rel_linf(u_g, u_r) < 1e-12


# Nx = 134 (2 mod 4): two cells per thread; Nx = 532 (0 mod 4): four cells
# per thread, 133 threads per row, so two blocks of 128 with a ragged tail
EVEN_DIMS = {0: (134, 37, 1), 1: (134, 6, 5), 2: (134, 6, 5)}
QUAD_DIMS = {0: (532, 9, 1), 1: (532, 6, 5), 2: (532, 6, 5)}


@pytest.mark.parametrize("streaming", L.STREAMING_PATTERNS)
@pytest.mark.parametrize("storage,p", [(L.STORE_F16_DELTA, 10), (L.STORE_BF16_DELTA, 7)])
@pytest.mark.parametrize("method", METHODS, ids=lambda m: f"sp{m[0]}eq{m[1]}reg{int(m[2])}")
@pytest.mark.parametrize("st", [0, 1, 2], ids=["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("cells", [2, 4], ids=["pairs", "quads"])
def test_packed_half_kernel_error_bound(cells, st, method, storage, p, streaming):
    """Even Nx routes FP16 / BF16 steps, pull and in place, to the
    two- (Nx % 4 == 2) or four-cells-per-thread (Nx % 4 == 0) kernels with
    packed FP32 arithmetic; same rounding bound as the scalar kernel (see
    test_half_storage_error_bound)."""
    space, eq, reg = method
    dims = (EVEN_DIMS if cells == 2 else QUAD_DIMS)[st]
    d = 2 if st == 0 else 3
    rho, u = I.taylor_green(dims, 0.05, d=d)
    u = I.add_uniform_noise(u, 1e-3, seed=11)
    m = O.method(st, space, eq, rates_of(space, reg))
    df0 = O.init(m, dims, rho, u)
    _, w, _ = O.lattice(st)
    pert = I.random_deviations(len(w), int(np.prod(dims)), 2e-3, seed=12)
    df0 = df0 + (w[:, None] * pert).reshape(df0.shape)
    n = 4
    with L.Lattice(st, space, eq, storage, streaming, rates_of(space, reg), dims) as lat:
        lat.set_populations(df0)
        lat.step(n)
        got = lat.get_populations()
    ref = O.step(m, dims, df0, n)
    assert rel_linf(got, ref) < (n + 1) * 2.0 ** -(p + 1)


@pytest.mark.parametrize("storage", [L.STORE_F16_DELTA, L.STORE_BF16_DELTA], ids=["f16", "bf16"])
@pytest.mark.parametrize("st", [0, 1, 2], ids=["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("cells", [2, 4], ids=["pairs", "quads"])
def test_packed_half_pull_and_in_place_are_bitwise_identical(cells, st, storage):
    """The packed in-place kernels run the packed pull kernels' arithmetic:
    identical FP16 / BF16 states after odd and even step counts."""
    space, eq, reg = L.SPACE_CUMULANT, L.EQ_ABSOLUTE, True
    dims = (EVEN_DIMS if cells == 2 else QUAD_DIMS)[st]
    rho, u = I.taylor_green(dims, 0.05, d=2 if st == 0 else 3)
    u = I.add_uniform_noise(u, 1e-3, seed=11)
    for n in (4, 5):
        out = []
        for streaming in L.STREAMING_PATTERNS:
            with L.Lattice(st, space, eq, storage, streaming, rates_of(space, reg), dims) as lat:
                lat.init_velocity(rho.reshape(-1), u.reshape(-1))
                lat.step(n)
                out.append(lat.get_populations())
        for k in range(1, len(out)):
            assert np.array_equal(out[0], out[k]), (n, k)


@pytest.mark.parametrize("streaming", L.STREAMING_PATTERNS)
@pytest.mark.parametrize("storage", [L.STORE_F16_DELTA, L.STORE_BF16_DELTA], ids=["f16", "bf16"])
@pytest.mark.parametrize("method", [(L.SPACE_CUMULANT, L.EQ_ABSOLUTE, True),
                                    (L.SPACE_RAW, L.EQ_DELTA, False),
                                    (L.SPACE_TRT, L.EQ_ABSOLUTE, False)],
                         ids=lambda m: f"sp{m[0]}eq{m[1]}reg{int(m[2])}")
@pytest.mark.parametrize("st", [0, 1, 2], ids=["D2Q9", "D3Q19", "D3Q27"])
def test_four_cell_kernels_equal_two_cell_kernels_on_a_periodic_replica(st, method, storage,
                                                                        streaming):
    """Two copies along x of an Nx = 266 state (2 mod 4: two cells per
    thread) form an Nx = 532 state (0 mod 4: four cells per thread) whose
    periodic neighbours are the same values: after odd and even step counts
    the large lattice holds exactly two copies of the small one."""
    space, eq, reg = method
    ny, nz = (9, 1) if st == 0 else (6, 5)
    small, big = (266, ny, nz), (532, ny, nz)
    rho, u = I.taylor_green(small, 0.05, d=2 if st == 0 else 3)
    u = I.add_uniform_noise(u, 1e-3, seed=13)
    m = O.method(st, space, eq, rates_of(space, reg))
    df0 = O.init(m, small, rho, u)
    _, w, _ = O.lattice(st)
    pert = I.random_deviations(len(w), int(np.prod(small)), 2e-3, seed=14)
    df0 = df0 + (w[:, None] * pert).reshape(df0.shape)
    q = len(w)

    def tile(df):
        a = np.asarray(df).reshape(q, nz, ny, 266)
        return np.concatenate([a, a], axis=3).reshape(q, -1)

    for n in (4, 5):
        got = []
        for dims, d in ((small, df0), (big, tile(df0))):
            with L.Lattice(st, space, eq, storage, streaming, rates_of(space, reg), dims) as lat:
                lat.set_populations(d)
                lat.step(n)
                got.append(lat.get_populations())
        assert np.array_equal(tile(got[0]).reshape(got[1].shape), got[1]), n
