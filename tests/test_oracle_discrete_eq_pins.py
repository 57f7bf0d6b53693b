"""Pins of the oracle's discrete second-order equilibrium (EQ_DISCRETE2: the
equilibrium prescribed as a population vector, q_eq = T(f_eq), Sec. 2.4):

* f_eq reproduces the hydrodynamic moments exactly: sum f = rho,
  sum xi f = rho u, sum xi xi f = rho (u u + I / 3), on every stencil;
* on D2Q9 / D3Q27 its raw moments equal the truncated Maxwellian ones
  (product weights), so raw-space collisions equal EQ_ABSOLUTE ones; on
  D3Q19 the x^2 y^2-type moments differ by exactly -rho u_z^2 / 6 (and
  cyclically), every other moment agrees;
* raw-moment MRT with every rate equal to w is the textbook BGK step
  f* = f - w (f - f_eq) (brute force); SRT and TRT with w+ = w- likewise;
* with every rate 1 every space (raw, central, cumulant) collides to f_eq;
* f_eq is a fixed point of every space at any rates; mass and momentum are
  conserved;
* central moments of f_eq are not the Maxwellian's (third order is
  -rho u_x^2 u_y-like), so the central method with this equilibrium is a
  different method from the default one.
"""
import numpy as np
import pytest

import oracle as O

STENCILS = [O.D2Q9, O.D3Q19, O.D3Q27]
RATES = [1.3, 1.1, 1.6, 0.9, 1.2, 1.4]


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


def cells(st, n=12, seed=3):
    rng = np.random.default_rng(seed + st)
    rho = 1.0 + 0.03 * rng.standard_normal(n)
    u = 0.06 * rng.standard_normal((n, 3))
    if st == O.D2Q9:
        u[:, 2] = 0.0
    return rho, u


def feq_populations(st, rho, u):
    m = O.method(st, O.SPACE_RAW, O.EQ_DISCRETE2, [1.0] * 6)
    _, w, _ = O.lattice(st)
    return O.equilibrium(m, rho, u) + w[None, :]


@pytest.mark.parametrize("st", STENCILS)
def test_hydrodynamic_moments_exact(st):
    xi, _, _ = O.lattice(st)
    rho, u = cells(st)
    f = feq_populations(st, rho, u)
    assert np.abs(f.sum(1) - rho).max() < 1e-15
    np.testing.assert_allclose(f @ xi, rho[:, None] * u, rtol=0, atol=1e-15)
    d = 2 if st == O.D2Q9 else 3
    for a in range(d):
        for b in range(d):
            pi = f @ (xi[:, a] * xi[:, b])
            want = rho * (u[:, a] * u[:, b] + (1.0 / 3.0 if a == b else 0.0))
            assert np.abs(pi - want).max() < 1e-15


@pytest.mark.parametrize("st", STENCILS)
def test_raw_moments_against_truncated_maxwellian(st):
    _, _, ex = O.lattice(st)
    M = O.matrices(st)["M"]
    rho, u = cells(st)
    disc = feq_populations(st, rho, u) @ M.T
    _, w, _ = O.lattice(st)
    cont = (O.equilibrium(O.method(st, O.SPACE_RAW, O.EQ_ABSOLUTE, [1.0] * 6), rho, u)
            + w[None, :]) @ M.T
    diff = disc - cont
    for k, e in enumerate(ex):
        if st == O.D3Q19 and sorted(e) == [0, 2, 2]:
            other = int(np.argmin(e))  # the axis with exponent 0
            np.testing.assert_allclose(diff[:, k], -rho * u[:, other] ** 2 / 6.0,
                                       rtol=0, atol=1e-15)
        else:
            assert np.abs(diff[:, k]).max() < 1e-15, e


@pytest.mark.parametrize("st", [O.D2Q9, O.D3Q27])
def test_product_lattices_raw_collision_equals_absolute(st):
    rho, u = cells(st)
    _, w, _ = O.lattice(st)
    rng = np.random.default_rng(9)
    df = feq_populations(st, rho, u) - w + w * 4e-3 * rng.standard_normal((len(rho), len(w)))
    for space in (O.SPACE_RAW, O.SPACE_RAW_WEIGHTED, O.SPACE_POPULATIONS, O.SPACE_TRT):
        a = O.collide(O.method(st, space, O.EQ_DISCRETE2, RATES), df)
        b = O.collide(O.method(st, space, O.EQ_ABSOLUTE, RATES), df)
        assert np.abs(a - b).max() < 1e-15, space


@pytest.mark.parametrize("st", STENCILS)
def test_equal_rates_raw_mrt_is_textbook_bgk(st):
    xi, w, _ = O.lattice(st)
    rng = np.random.default_rng(11)
    n = 10
    f = w[None, :] * (1.0 + 0.05 * rng.standard_normal((n, len(w))))
    rho = f.sum(1)
    u = (f @ xi) / rho[:, None]
    # brute-force BGK with the polynomial equilibrium, written out per population
    om = 1.37
    feq = np.empty_like(f)
    for c in range(n):
        uu = u[c] @ u[c]
        for i in range(len(w)):
            xu = xi[i] @ u[c]
            feq[c, i] = w[i] * rho[c] * (1 + 3 * xu + 4.5 * xu * xu - 1.5 * uu)
    bgk = f - om * (f - feq)
    df = f - w
    for space, rates in ((O.SPACE_RAW, [om] * 6), (O.SPACE_RAW_WEIGHTED, [om] * 6),
                         (O.SPACE_POPULATIONS, [om] * 6), (O.SPACE_TRT, [om] * 6)):
        got = O.collide(O.method(st, space, O.EQ_DISCRETE2, rates), df) + w
        assert np.abs(got - bgk).max() < 2e-15, space


@pytest.mark.parametrize("st", STENCILS)
def test_unit_rates_collide_to_feq_in_every_space(st):
    rho0, u0 = cells(st)
    _, w, _ = O.lattice(st)
    rng = np.random.default_rng(5)
    df = feq_populations(st, rho0, u0) - w + w * 5e-3 * rng.standard_normal((len(rho0), len(w)))
    xi, _, _ = O.lattice(st)
    f = df + w
    rho = f.sum(1)
    u = (f @ xi) / rho[:, None]
    want = feq_populations(st, rho, u) - w
    for space in (O.SPACE_RAW, O.SPACE_CENTRAL, O.SPACE_CUMULANT, O.SPACE_POPULATIONS):
        got = O.collide(O.method(st, space, O.EQ_DISCRETE2, [1.0] * 6), df)
        assert np.abs(got - want).max() < 5e-15, space


@pytest.mark.parametrize("st", STENCILS)
def test_feq_is_fixed_point_and_conservation(st):
    rho, u = cells(st)
    xi, w, _ = O.lattice(st)
    df_eq = feq_populations(st, rho, u) - w
    rng = np.random.default_rng(6)
    df = df_eq + w * 5e-3 * rng.standard_normal(df_eq.shape)
    for space in (O.SPACE_RAW, O.SPACE_RAW_WEIGHTED, O.SPACE_CENTRAL, O.SPACE_CUMULANT,
                  O.SPACE_POPULATIONS, O.SPACE_TRT):
        m = O.method(st, space, O.EQ_DISCRETE2, RATES)
        assert np.abs(O.collide(m, df_eq) - df_eq).max() < 5e-15, space
        out = O.collide(m, df)
        assert np.abs(out.sum(1) - df.sum(1)).max() < 1e-15
        assert np.abs(out @ xi - df @ xi).max() < 1e-15


def test_central_equilibrium_differs_from_maxwellian():
    st = O.D3Q27
    rho, u = cells(st)
    f = feq_populations(st, rho[:1], u[:1])[0]
    xi, _, _ = O.lattice(st)
    c = xi - u[0][None, :]
    k_xxy = f @ (c[:, 0] ** 2 * c[:, 1])
    # third-order central moment of the polynomial f_eq: -rho u_x^2 u_y
    # (the Maxwellian's is 0)
    assert abs(k_xxy - (-rho[0] * u[0, 0] ** 2 * u[0, 1])) < 1e-15
    rng = np.random.default_rng(7)
    _, w, _ = O.lattice(st)
    df = f - w + w * 3e-3 * rng.standard_normal(27)
    a = O.collide(O.method(st, O.SPACE_CENTRAL, O.EQ_DISCRETE2, [1.0] * 6), df)
    b = O.collide(O.method(st, O.SPACE_CENTRAL, O.EQ_ABSOLUTE, [1.0] * 6), df)
    assert np.abs(a - b).max() > 1e-7
