"""Pins of the oracle's weighted orthogonal raw-moment basis (WO-MRT, Sec. 4.2
and Table 3) against closed forms:

* the rows are orthogonal under <p,q> = sum_i w_i p(xi_i) q(xi_i) and keep
  the degree filtration (each row is its leading monomial plus lower-degree
  terms);
* on the tensor-product lattices D2Q9 / D3Q27 the rows of order >= 3 are the
  products of the 1-D weighted orthogonal polynomials 1, x, x^2 - 1/3;
* WO-MRT with every rate equal is BGK, and with every rate 1 it is O-MRT
  with every rate 1 (both set every non-conserved moment to equilibrium);
* with shear and bulk rates other than 1 the two bases are different methods.
"""
import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


@pytest.mark.parametrize("st", [O.D2Q9, O.D3Q19, O.D3Q27])
def test_rows_are_weight_orthogonal_with_degree_filtration(st):
    _, w, ex = O.lattice(st)
    M = O.matrices(st)["M"]
    Pw = O.weighted_basis(st)
    V = Pw @ M  # V[r, i] = p_r(xi_i)
    G = V @ np.diag(w) @ V.T
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() < 1e-14
    deg = ex.sum(1)
    for r in range(len(w)):
        lead = int(np.argmax(deg * (np.abs(Pw[r]) > 1e-14)))
        assert all(deg[k] < deg[lead] or k == lead or abs(Pw[r, k]) < 1e-14 or deg[k] == deg[lead]
                   for k in range(len(w)))


@pytest.mark.parametrize("st", [O.D2Q9, O.D3Q27])
def test_tensor_product_rows(st):
    xi, w, ex = O.lattice(st)
    M = O.matrices(st)["M"]
    Pw = O.weighted_basis(st)
    V = Pw @ M
    p1 = {0: lambda t: np.ones_like(t, dtype=float), 1: lambda t: t.astype(float),
          2: lambda t: t.astype(float) ** 2 - 1.0 / 3.0}
    deg = ex.sum(1)
    checked = 0
    for r in range(len(w)):
        # rows of order >= 3 are monomial rows: leading monomial of max degree
        k = int(np.argmax(np.where(np.abs(Pw[r]) > 1e-14, deg, -1)))
        if deg[k] < 3:
            continue
        want = p1[ex[k, 0]](xi[:, 0]) * p1[ex[k, 1]](xi[:, 1]) * p1[ex[k, 2]](xi[:, 2])
        assert np.abs(V[r] - want).max() < 1e-14, (r, ex[k])
        checked += 1
    assert checked == (3 if st == O.D2Q9 else 17)


@pytest.mark.parametrize("st", [O.D2Q9, O.D3Q19, O.D3Q27])
def test_equal_rates_is_bgk_and_unit_rates_match_o_mrt(st):
    rng = np.random.default_rng(4)
    _, w, _ = O.lattice(st)
    m0 = O.method(st, O.SPACE_RAW, O.EQ_DELTA, [1.0] * 6)
    rho = 1 + 0.02 * rng.standard_normal(10)
    u = 0.05 * rng.standard_normal((10, 3))
    if st == O.D2Q9:
        u[:, 2] = 0
    df = O.equilibrium(m0, rho, u) + w[None, :] * 3e-3 * rng.standard_normal((10, len(w)))
    for eq in (O.EQ_DELTA, O.EQ_ABSOLUTE):
        wo = O.collide(O.method(st, O.SPACE_RAW_WEIGHTED, eq, [1.4] * 6), df)
        bgk = O.collide(O.method(st, O.SPACE_POPULATIONS, eq, [1.4] * 6), df)
        assert np.abs(wo - bgk).max() < 1e-15
        wo1 = O.collide(O.method(st, O.SPACE_RAW_WEIGHTED, eq, [1.0] * 6), df)
        o1 = O.collide(O.method(st, O.SPACE_RAW, eq, [1.0] * 6), df)
        assert np.abs(wo1 - o1).max() < 1e-15
    # with shear and bulk rates other than 1 the bases give different methods
    # (on D2Q9 a unit bulk rate alone hides the difference: x^2 y^2 sees the
    # trace of the second-order non-equilibrium only)
    r = [1.8, 1.4] + [1.0] * 4
    a = O.collide(O.method(st, O.SPACE_RAW_WEIGHTED, O.EQ_DELTA, r), df)
    b = O.collide(O.method(st, O.SPACE_RAW, O.EQ_DELTA, r), df)
    assert np.abs(a - b).max() > 1e-8
