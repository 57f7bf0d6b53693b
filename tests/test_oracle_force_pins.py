"""Pins of the oracle's body-force collision (source term of Eq. 2.1a, q^F of
Eq. 2.4; Guo's model, see oracle/lbm_oracle.h) against what the physics
fixes independently of the formulas typed in the oracle:

* a body force changes the momentum of every cell by exactly F per step and
  leaves its mass unchanged (any force model);
* with F = 0 the forced collision is the plain one;
* for cumulants with every rate 1 the collision lands on the method's own
  equilibrium at the advanced velocity (j + F) / rho;
* Kolmogorov flow: the steady state of a periodic shear force
  F_x = F0 sin(k y) is u_x = F0 / (rho nu k^2) sin(k y) for the
  incompressible Navier-Stokes equations, nu = (1/omega - 1/2) / 3; every
  collision space reaches it within the lattice's O(k^2) error;
* total momentum of a periodic lattice grows by N F per step.
"""
import numpy as np
import pytest

import oracle as O

SPACES = [O.SPACE_POPULATIONS, O.SPACE_RAW, O.SPACE_CENTRAL, O.SPACE_CUMULANT]


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


def random_cells(st, n, seed):
    rng = np.random.default_rng(seed)
    _, w, _ = O.lattice(st)
    m = O.method(st, O.SPACE_RAW, O.EQ_DELTA, [1.0] * 6)
    rho = 1.0 + 0.02 * rng.standard_normal(n)
    u = 0.05 * rng.standard_normal((n, 3))
    if st == O.D2Q9:
        u[:, 2] = 0
    df = O.equilibrium(m, rho, u)
    return df + w[None, :] * 3e-3 * rng.standard_normal(df.shape)


def moments(st, df):
    xi = O.lattice(st)[0]
    return df.sum(1), df @ xi


@pytest.mark.parametrize("eq", [O.EQ_DELTA, O.EQ_ABSOLUTE])
@pytest.mark.parametrize("space", SPACES)
@pytest.mark.parametrize("st", [O.D2Q9, O.D3Q19, O.D3Q27])
def test_force_adds_exactly_F_to_the_momentum(st, space, eq):
    if space == O.SPACE_CUMULANT and eq == O.EQ_DELTA:
        pytest.skip("inadmissible")
    df = random_cells(st, 16, seed=st * 10 + space)
    rng = np.random.default_rng(7)
    F = 1e-3 * rng.standard_normal((16, 3))
    if st == O.D2Q9:
        F[:, 2] = 0
    m = O.method(st, space, eq, [1.3, 1.1, 1.2, 1.4, 1.5, 1.6])
    out = O.collide_forced(m, df, F)
    rho0, j0 = moments(st, df)
    rho1, j1 = moments(st, out)
    assert np.abs(rho1 - rho0).max() < 1e-15
    assert np.abs(j1 - (j0 + F)).max() < 1e-15
    # no force: the plain collision
    assert np.abs(O.collide_forced(m, df, np.zeros((16, 3))) - O.collide(m, df)).max() < 1e-16


@pytest.mark.parametrize("st", [O.D3Q19, O.D3Q27])
def test_cumulant_with_unit_rates_lands_on_the_shifted_equilibrium(st):
    df = random_cells(st, 12, seed=3)
    F = np.tile([2e-3, -1e-3, 5e-4], (12, 1))
    m = O.method(st, O.SPACE_CUMULANT, O.EQ_ABSOLUTE, [1.0] * 6)
    out = O.collide_forced(m, df, F)
    rho, j = moments(st, df)
    rho = 1.0 + rho
    ref = O.equilibrium(m, rho, (j + F) / rho[:, None])
    assert np.abs(out - ref).max() < 1e-15


@pytest.mark.parametrize("space", SPACES)
@pytest.mark.parametrize("st", [O.D2Q9, O.D3Q19, O.D3Q27])
def test_kolmogorov_flow_steady_state(st, space):
    ny = 32
    dims = (1, ny, 1)
    k = 2 * np.pi / ny
    omega = 1.6
    nu = (1.0 / omega - 0.5) / 3.0
    F0 = 1e-6
    y = np.arange(ny)
    d = 2 if st == O.D2Q9 else 3
    force = np.zeros((d, 1, ny, 1))
    force[0, 0, :, 0] = F0 * np.sin(k * y)
    eq = O.EQ_ABSOLUTE
    m = O.method(st, space, eq, [omega] + [1.0] * 5)
    rho0 = np.ones((1, ny, 1))
    u0 = np.zeros((d, 1, ny, 1))
    df = O.init(m, dims, rho0, u0)
    steps = int(12 / (nu * k * k))  # e^-12 of the start-up transient left
    df = O.step_forced(m, dims, df, force, steps)
    _, u = O.macroscopic_forced(m, dims, df, force)
    amp = F0 / (nu * k * k)
    want = amp * np.sin(k * y)
    err = np.abs(u[0, 0, :, 0] - want).max() / amp
    assert err < 0.01, err  # O(k^2) lattice error: 0.4 - 0.6 % at L = 32
    assert np.abs(u[1]).max() < 1e-6 * amp


def test_total_momentum_grows_by_N_F_per_step():
    st, dims = O.D3Q27, (6, 5, 4)
    N = 6 * 5 * 4
    F = np.array([1e-4, -2e-4, 3e-4])
    for space in SPACES:
        m = O.method(st, space, O.EQ_ABSOLUTE, [1.7, 1.0, 1.2, 1.1, 1.0, 1.3])
        rng = np.random.default_rng(1)
        u = 0.02 * rng.standard_normal((3, 4, 5, 6))
        df = O.init(m, dims, np.ones((4, 5, 6)), u)
        j0 = np.einsum("iz,id->d", df.reshape(27, -1), O.lattice(st)[0].astype(float))
        out = O.step_forced(m, dims, df, F, 5)
        j5 = np.einsum("iz,id->d", out.reshape(27, -1), O.lattice(st)[0].astype(float))
        assert np.abs(j5 - (j0 + 5 * N * F)).max() < 1e-13, space


@pytest.mark.parametrize("forced", [False, True])
@pytest.mark.parametrize("eq", [O.EQ_DELTA, O.EQ_ABSOLUTE])
@pytest.mark.parametrize("st", [O.D2Q9, O.D3Q19, O.D3Q27])
def test_trt_is_raw_mrt_with_rates_by_parity(st, eq, forced):
    """The population-space TRT (even part w+, odd part w-) equals raw-moment
    MRT with every even-order group at w+ and every odd-order group at w-:
    even-order monomial moments see only f+, odd-order ones only f- (the
    orthogonal basis keeps each polynomial's parity); the Guo source splits
    the same way, and the momentum row is exact in both."""
    wp, wm = 1.3, 1.75
    df = random_cells(st, 20, seed=5)
    trt = O.method(st, O.SPACE_TRT, eq, [wp, 0.5, wm, 0.5, 0.5, 0.5])
    mrt = O.method(st, O.SPACE_RAW, eq, [wp, wp, wm, wp, wm, wp])
    if forced:
        F = 1e-3 * np.random.default_rng(2).standard_normal((20, 3))
        if st == O.D2Q9:
            F[:, 2] = 0
        a, b = O.collide_forced(trt, df, F), O.collide_forced(mrt, df, F)
    else:
        a, b = O.collide(trt, df), O.collide(mrt, df)
    assert np.abs(a - b).max() < 1e-15


# --------------------------------------------------------------- He's model
HE_SPACES = [O.SPACE_POPULATIONS, O.SPACE_RAW, O.SPACE_CENTRAL, O.SPACE_TRT,
             O.SPACE_RAW_WEIGHTED]


@pytest.mark.parametrize("space", HE_SPACES)
@pytest.mark.parametrize("st", [O.D2Q9, O.D3Q19, O.D3Q27])
def test_he_force_adds_exactly_F_and_keeps_mass(st, space):
    df = random_cells(st, 16, seed=40 + space)
    F = 1e-3 * np.random.default_rng(9).standard_normal((16, 3))
    if st == O.D2Q9:
        F[:, 2] = 0
    m = O.method(st, space, O.EQ_ABSOLUTE, [1.3, 1.1, 1.2, 1.4, 1.5, 1.6])
    out = O.collide_forced(m, df, F, model=O.FORCE_HE)
    rho0, j0 = moments(st, df)
    rho1, j1 = moments(st, out)
    assert np.abs(rho1 - rho0).max() < 1e-15
    assert np.abs(j1 - (j0 + F)).max() < 1e-15


@pytest.mark.parametrize("st", [O.D2Q9, O.D3Q19, O.D3Q27])
def test_he_and_guo_agree_to_second_order_for_central_moments(st):
    """He's source has Guo's moments up to order 2 except for terms of order
    u^3 F (the lattice aliases the equilibrium's odd central moments), so
    the two collisions' second-order raw moments differ by O(u^3 F): halving
    the velocity divides the difference by 8."""
    _, w, ex = O.lattice(st)
    M = O.matrices(st)["M"]
    low = ex.sum(1) <= 2
    rng = np.random.default_rng(10)
    F = 1e-3 * rng.standard_normal((16, 3))
    u0 = 0.08 * rng.standard_normal((16, 3))
    if st == O.D2Q9:
        F[:, 2] = 0
        u0[:, 2] = 0
    rho = 1 + 0.02 * rng.standard_normal(16)
    m = O.method(st, O.SPACE_CENTRAL, O.EQ_ABSOLUTE, [1.3, 1.1, 1.2, 1.4, 1.5, 1.6])
    diff = []
    for sc in (1.0, 0.5):
        df = O.equilibrium(m, rho, sc * u0)
        a = O.collide_forced(m, df, F, model=O.FORCE_HE)
        b = O.collide_forced(m, df, F, model=O.FORCE_GUO)
        diff.append(np.abs((a - b) @ M.T[:, low]).max())
        assert np.abs((a - b) @ M.T[:, ~low]).max() > 1e-9  # different models
    assert diff[0] < 10 * np.abs(u0).max() ** 3 * np.abs(F).max()
    assert 6.5 < diff[0] / diff[1] < 9.5, diff


@pytest.mark.parametrize("space", [O.SPACE_POPULATIONS, O.SPACE_RAW, O.SPACE_CENTRAL])
def test_he_kolmogorov_flow_steady_state(space):
    ny, st = 32, O.D3Q27
    dims = (1, ny, 1)
    k = 2 * np.pi / ny
    omega = 1.6
    nu = (1.0 / omega - 0.5) / 3.0
    F0 = 1e-6
    force = np.zeros((3, 1, ny, 1))
    force[0, 0, :, 0] = F0 * np.sin(k * np.arange(ny))
    m = O.method(st, space, O.EQ_ABSOLUTE, [omega] + [1.0] * 5)
    df = O.init(m, dims, np.ones((1, ny, 1)), np.zeros((3, 1, ny, 1)))
    df = O.step_forced(m, dims, df, force, int(12 / (nu * k * k)), model=O.FORCE_HE)
    _, u = O.macroscopic_forced(m, dims, df, force)
    amp = F0 / (nu * k * k)
    err = np.abs(u[0, 0, :, 0] - amp * np.sin(k * np.arange(ny))).max() / amp
    assert err < 0.01, err


def test_he_is_undefined_for_cumulants():
    m = O.method(O.D3Q27, O.SPACE_CUMULANT, O.EQ_ABSOLUTE, [1.3] + [1.0] * 5)
    with pytest.raises(RuntimeError):
        O.collide_forced(m, random_cells(O.D3Q27, 2, seed=1), [1e-3, 0, 0], model=O.FORCE_HE)
