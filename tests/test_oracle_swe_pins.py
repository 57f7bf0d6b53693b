"""Pins of the oracle's shallow-water methods (Sec. 5.2: Zhou's discrete
equilibrium with the central-moment collision of de Rosis, and the cumulant
collision with c_s^2 = g h / 2 of Venturi) against what the shallow-water
equations fix:

* both equilibria carry depth h, discharge h u and the shallow-water
  momentum flux h u u + g h^2 / 2 I;
* the lake at rest is a fixed point, and every collision keeps h and h u;
* with every rate 1 the cumulant collision lands on its own equilibrium;
* a small surface wave h0 + eps cos(k x) oscillates at the gravity-wave
  frequency sqrt(g h0) k.
"""
import numpy as np
import pytest

import oracle as O

G = 0.0613  # 9.81 m/s^2 with dx = 0.4 m, dt = 0.05 s (the dam-break lattice)
SPACES = [O.SPACE_CENTRAL, O.SPACE_CUMULANT]


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


def method(space, omega=0.696):
    return O.method(O.D2Q9, space, O.EQ_ABSOLUTE, [omega, 1.0, 1.0, 1.0, 1.0, 1.0])


def xi2():
    return O.lattice(O.D2Q9)[0][:, :2].astype(float)


@pytest.mark.parametrize("space", SPACES)
def test_equilibrium_moments_are_the_shallow_water_fluxes(space):
    rng = np.random.default_rng(1)
    xi = xi2()
    for _ in range(20):
        h = rng.uniform(0.5, 6.0)
        u = rng.uniform(-0.1, 0.1, 2)
        f = O.swe_equilibrium(space, G, h, u)
        assert abs(f.sum() - h) < 1e-14 * h
        assert np.abs(xi.T @ f - h * u).max() < 1e-14 * h
        flux = np.einsum("ia,ib,i->ab", xi, xi, f)
        want = h * np.outer(u, u) + 0.5 * G * h * h * np.eye(2)
        assert np.abs(flux - want).max() < 1e-14 * h


@pytest.mark.parametrize("space", SPACES)
def test_lake_at_rest_and_conservation(space):
    m = method(space)
    _, w, _ = O.lattice(O.D2Q9)
    for h in (0.8, 2.5, 6.25):
        feq = O.swe_equilibrium(space, G, h, [0.0, 0.0])
        out = O.swe_collide(m, G, (feq - w)[None, :])[0] + w
        assert np.abs(out - feq).max() < 1e-14 * h
    rng = np.random.default_rng(2)
    xi = xi2()
    for _ in range(10):
        h = rng.uniform(0.8, 5.0)
        u = rng.uniform(-0.05, 0.05, 2)
        f = O.swe_equilibrium(space, G, h, u) * (1 + 0.01 * rng.standard_normal(9))
        out = O.swe_collide(m, G, (f - w)[None, :])[0] + w
        assert abs(out.sum() - f.sum()) < 1e-14 * h
        assert np.abs(xi.T @ out - xi.T @ f).max() < 1e-14 * h


def test_cumulant_with_unit_rates_lands_on_its_equilibrium():
    m = O.method(O.D2Q9, O.SPACE_CUMULANT, O.EQ_ABSOLUTE, [1.0] * 6)
    _, w, _ = O.lattice(O.D2Q9)
    xi = xi2()
    rng = np.random.default_rng(3)
    for _ in range(10):
        h = rng.uniform(0.8, 5.0)
        u = rng.uniform(-0.05, 0.05, 2)
        f = O.swe_equilibrium(O.SPACE_CUMULANT, G, h, u) * (1 + 0.02 * rng.standard_normal(9))
        out = O.swe_collide(m, G, (f - w)[None, :])[0] + w
        hh = f.sum()
        ref = O.swe_equilibrium(O.SPACE_CUMULANT, G, hh, xi.T @ f / hh)
        assert np.abs(out - ref).max() < 1e-14 * h


@pytest.mark.parametrize("space", SPACES)
def test_gravity_wave_frequency(space):
    nx, h0, eps = 64, 2.0, 1e-4
    k = 2 * np.pi / nx
    dims = (nx, 1, 1)
    x = np.arange(nx)
    h = (h0 + eps * np.cos(k * x)).reshape(1, 1, nx)
    u = np.zeros((2, 1, 1, nx))
    m = method(space, omega=1.8)  # low viscosity: weak damping
    df = O.swe_init(m, G, dims, h, u)
    amp = []
    for _ in range(400):
        df = O.swe_step(m, G, dims, df, 1)
        hh, _ = O.macroscopic(m, dims, df)
        amp.append(float(((hh.reshape(-1) - h0) * np.cos(k * x)).sum()) * 2 / nx)
    amp = np.array(amp)
    t = np.arange(1, 401)
    # frequency of the damped cosine from its zero crossings
    zc = np.where(np.sign(amp[:-1]) != np.sign(amp[1:]))[0]
    tz = t[zc] + amp[zc] / (amp[zc] - amp[zc + 1])  # linear interpolation
    period = 2 * np.mean(np.diff(tz))
    want = 2 * np.pi / (np.sqrt(G * h0) * k)
    assert len(tz) >= 3
    assert abs(period / want - 1) < 5e-3, (period, want)  # measured 0.05 %
