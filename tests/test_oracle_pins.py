"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

None of these tests re-types the oracle's own formula: each one checks the
oracle against an independent route (a textbook value, a generating-function
expansion, a brute-force step, an invariant or a closed-form flow solution).
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2211_02435_b300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
STENCILS = [0, 1, 2]
NAMES = {0: "D2Q9", 1: "D3Q19", 2: "D3Q27"}


@pytest.fixture(scope="module")
def O(oracle_lib):
    return oracle_lib


# ---------------------------------------------------------------- lattice
def test_weights_match_textbook(O):
    """f0 = M^-1 m0 reduces to the lattice weights (Sec. 2.4)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "lattice_weights.txt"))
            if l.strip() and not l.startswith("#")]
    for st in STENCILS:
        xi, w, _ = O.lattice(st)
        for name, n2, frac in rows:
            if name != NAMES[st]:
                continue
            sel = (xi * xi).sum(1) == int(n2)
            assert sel.any()
            np.testing.assert_allclose(w[sel], float(Fraction(frac)), rtol=0, atol=1e-15)
        assert abs(w.sum() - 1.0) < 1e-15


@pytest.mark.parametrize("st", STENCILS)
def test_moment_matrix_inverse_and_velocity_order(O, st):
    xi, w, ex = O.lattice(st)
    q = len(w)
    mats = O.matrices(st)
    assert np.linalg.matrix_rank(mats["M"]) == q
    np.testing.assert_allclose(mats["M"] @ mats["Minv"], np.eye(q), atol=1e-13)
    # brute-force M from the definition m_e = sum_i f_i prod xi^e (Eq. 2.8)
    M = np.array([[np.prod([xi[i, d] ** ex[k, d] for d in range(3)]) for i in range(q)]
                  for k in range(q)], dtype=float)
    np.testing.assert_array_equal(M, mats["M"])
    # documented order: xi_0 = 0 and opposite pairs adjacent
    assert not xi[0].any()
    for i in range(1, q):
        ib = i + 1 if i % 2 else i - 1
        np.testing.assert_array_equal(xi[ib], -xi[i])
    # the exponent set is downward closed (needed by the Chimera passes)
    es = {tuple(e) for e in ex}
    for e in es:
        for d in range(3):
            if e[d]:
                lo = list(e)
                lo[d] -= 1
                assert tuple(lo) in es


@pytest.mark.parametrize("st", STENCILS)
def test_orthogonal_raw_basis_filtration(O, st):
    """O-MRT basis: rows orthogonal under the unweighted inner product; the
    rows of degree <= k span exactly the monomials of degree <= k."""
    xi, w, ex = O.lattice(st)
    mats = O.matrices(st)
    V = mats["Praw"] @ mats["M"]
    G = V @ V.T
    assert np.abs(G - np.diag(np.diag(G))).max() < 1e-12
    deg = ex.sum(1)
    g = mats["group"]
    row_deg = np.where(g < 0, np.where(np.arange(len(g)) == 0, 0, 1),
                       np.where(g <= 1, 2, g + 1))
    for k in range(int(deg.max()) + 1):
        A = mats["Praw"][row_deg <= k]
        B = np.eye(len(w))[deg <= k]
        assert np.linalg.matrix_rank(np.vstack([A, B]), tol=1e-9) == (deg <= k).sum()
        assert np.linalg.matrix_rank(A, tol=1e-9) == (deg <= k).sum()


def _tensor_raw_relax(xi, df, feq, rates):
    """Independent closed form of O-MRT on tensor-product stencils (D2Q9,
    D3Q27): the unweighted orthogonal polynomials are products of
    (1, x, x^2 - 2/3) per axis; each is relaxed with the rate of its order,
    with the order-2 diagonal split into trace (bulk) and traceless (shear)."""
    q, dim = df.shape[0], (3 if xi[:, 2].any() else 2)
    one_d = [lambda s: np.ones_like(s, dtype=float), lambda s: s.astype(float),
             lambda s: s.astype(float) ** 2 - 2.0 / 3.0]
    polys, orders = [], []
    for e in itertools.product(range(3), repeat=dim):
        v = np.ones(q)
        for d in range(dim):
            v = v * one_d[e[d]](xi[:, d])
        polys.append(v)
        orders.append(e)
    out = df.copy()
    neq = df - feq
    diag = []
    for v, e in zip(polys, orders):
        o = sum(e)
        c = (v @ neq) / (v @ v)
        if o <= 1:
            continue
        if o == 2 and max(e) == 2:
            diag.append((v, c))
            continue
        om = rates[0] if o == 2 else rates[o - 1]
        out -= om * c * v
    # diagonal order 2: equal norms -> trace / traceless split of coefficients
    cs = np.array([c for _, c in diag])
    mean = cs.mean()
    for (v, c) in diag:
        out -= (rates[1] * mean + rates[0] * (c - mean)) * v
    return out


@pytest.mark.parametrize("st", [0, 2])
def test_raw_mrt_equals_tensor_closed_form(O, st):
    xi, w, _ = O.lattice(st)
    rng = np.random.default_rng(7)
    rates = [1.73, 1.21, 1.37, 0.93, 1.55, 1.11]
    m = O.method(st, O.SPACE_RAW, O.EQ_DELTA, rates)
    for _ in range(5):
        rho = 1 + 0.02 * rng.standard_normal()
        u = 0.06 * rng.standard_normal(3)
        if st == 0:
            u[2] = 0
        feq = O.equilibrium(m, rho, u)[0]
        df = feq + 2e-3 * rng.standard_normal(len(w))
        # equilibrium of the perturbed state
        rho2 = 1 + df.sum()
        u2 = (df @ xi) / rho2
        feq2 = O.equilibrium(m, rho2, u2)[0]
        ref = _tensor_raw_relax(xi, df, feq2, rates)
        np.testing.assert_allclose(O.collide(m, df), ref, rtol=0, atol=1e-15)


# ------------------------------------------------------------ equilibria
def _discrete_feq(xi, w, rho, u):
    cu = xi @ u
    return w * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (u @ u))


@pytest.mark.parametrize("st", STENCILS)
def test_raw_equilibrium_vs_discrete_maxwellian(O, st):
    """Raw equilibrium moments (Maxwellian, truncated at O(u^2), Sec. 4.2)
    equal the moments of the discrete 2nd-order polynomial Maxwellian, except
    on D3Q19 where the x^2y^2-type moments differ by exactly -rho u_k^2 / 6."""
    xi, w, ex = O.lattice(st)
    mats = O.matrices(st)
    m = O.method(st, O.SPACE_RAW, O.EQ_DELTA, [1.0] * 6)
    rng = np.random.default_rng(3)
    for _ in range(6):
        rho = 1 + 0.05 * rng.standard_normal()
        u = 0.1 * rng.standard_normal(3)
        if st == 0:
            u[2] = 0
        m_or = mats["M"] @ (O.equilibrium(m, rho, u)[0] + w)
        m_disc = mats["M"] @ _discrete_feq(xi, w, rho, u)
        expect = m_disc.copy()
        if st == 1:
            for k, e in enumerate(ex):
                if sorted(e) == [0, 2, 2]:
                    kk = int(np.where(np.asarray(e) == 0)[0][0])
                    expect[k] = m_disc[k] + rho * u[kk] ** 2 / 6.0
        np.testing.assert_allclose(m_or, expect, rtol=0, atol=2e-15)


@pytest.mark.parametrize("st", STENCILS)
def test_central_matrix_equals_binomial_chimera_route(O, st):
    """K(u) f (direct definition, Sec. 2.3.2) equals the binomial expansion of
    the raw moments M f (Eq. 4.3)."""
    xi, w, ex = O.lattice(st)
    mats = O.matrices(st)
    idx = {tuple(e): k for k, e in enumerate(ex)}
    rng = np.random.default_rng(11)
    for _ in range(4):
        f = w + 0.01 * rng.standard_normal(len(w))
        u = 0.1 * rng.standard_normal(3)
        if st == 0:
            u[2] = 0
        kappa = O.central_matrix(st, u) @ f
        mraw = mats["M"] @ f
        for k, e in enumerate(ex):
            s = 0.0
            for a in range(e[0] + 1):
                for b in range(e[1] + 1):
                    for c in range(e[2] + 1):
                        s += (math.comb(e[0], a) * math.comb(e[1], b) * math.comb(e[2], c)
                              * (-u[0]) ** (e[0] - a) * (-u[1]) ** (e[1] - b)
                              * (-u[2]) ** (e[2] - c) * mraw[idx[(a, b, c)]])
            assert abs(kappa[k] - s) < 1e-15


# ------------------------------------------------------------- cumulants
def _poly_mul(p, q, dim):
    out = {}
    for ea, ca in p.items():
        for eb, cb in q.items():
            e = tuple(x + y for x, y in zip(ea, eb))
            if max(e) > 2:
                continue
            out[e] = out.get(e, 0) + ca * cb
    return out


def _cumulants_by_log_series(xi, f, dim):
    """Rescaled cumulants C = rho * c from the coefficients of log M(Xi)
    (Eq. 2.11) computed exactly with rational arithmetic.  Truncating each
    variable at degree 2 is exact for the derivatives needed here."""
    f = [Fraction(x) for x in f]
    rho = sum(f)
    h = {}
    for e in itertools.product(range(3), repeat=dim):
        if sum(e) == 0:
            continue
        mom = sum(fi * np.prod([int(xi[i][d]) ** e[d] for d in range(dim)])
                  for i, fi in enumerate(f))
        h[e] = Fraction(mom) / rho / math.prod(math.factorial(k) for k in e)
    logm = {}
    power = {tuple([0] * dim): Fraction(1)}
    for k in range(1, 2 * dim + 1):
        power = _poly_mul(power, h, dim)
        for e, c in power.items():
            logm[e] = logm.get(e, 0) + Fraction((-1) ** (k + 1), k) * c
    out = {}
    for e, c in logm.items():
        val = c * math.prod(math.factorial(k) for k in e)
        out[e] = val if sum(e) == 1 else rho * val
    out[tuple([0] * dim)] = rho
    return out


@pytest.mark.parametrize("st", STENCILS)
def test_cumulants_match_log_generating_function(O, st):
    xi, w, ex = O.lattice(st)
    dim = 2 if st == 0 else 3
    rng = np.random.default_rng(5)
    for trial in range(2):
        # exactly representable random populations (multiples of 2^-20)
        f = np.round((w + 0.02 * rng.standard_normal(len(w))) * 2 ** 20) / 2 ** 20
        ref = _cumulants_by_log_series(xi.tolist(), f.tolist(), dim)
        got = O.cumulants(st, f)
        for k, e in enumerate(ex):
            r = float(ref[tuple(e[:dim])])
            assert abs(got[k] - r) <= 1e-14 * max(1.0, abs(r)), (e, got[k], r)


def test_cumulant_partition_formula_textbook_cases(O):
    rng = np.random.default_rng(2)
    # independent coordinates: every mixed cumulant vanishes
    px = rng.random(4); px /= px.sum(); vx = rng.standard_normal(4)
    py = rng.random(3); py /= py.sum(); vy = rng.standard_normal(3)
    pz = rng.random(5); pz /= pz.sum(); vz = rng.standard_normal(5)
    mu = np.zeros((3, 3, 3))
    for a, b, c in itertools.product(range(3), repeat=3):
        mu[a, b, c] = (px @ vx ** a) * (py @ vy ** b) * (pz @ vz ** c)
    for a, b, c in itertools.product(range(3), repeat=3):
        if sum(x > 0 for x in (a, b, c)) >= 2:
            assert abs(O.cumulant_of(mu, a, b, c)) < 1e-14
    # univariate textbook: k2 = variance, Gaussian-vector cumulants of order > 2 vanish
    assert abs(O.cumulant_of(mu, 2, 0, 0) - (px @ vx ** 2 - (px @ vx) ** 2)) < 1e-15
    mean = rng.standard_normal(3) * 0.3
    S = rng.standard_normal((3, 3)); S = S @ S.T * 0.1
    # Gaussian raw moments up to exponent 2 per axis via Isserlis on X = mean + Y
    def gmom(e):
        labels = [d for d in range(3) for _ in range(e[d])]
        tot = 0.0
        for mask in itertools.product([0, 1], repeat=len(labels)):
            cen = [labels[i] for i in range(len(labels)) if mask[i]]
            fixed = np.prod([mean[labels[i]] for i in range(len(labels)) if not mask[i]])
            tot += fixed * _isserlis(cen, S)
        return tot
    for a, b, c in itertools.product(range(3), repeat=3):
        mu[a, b, c] = gmom((a, b, c))
    for a, b, c in itertools.product(range(3), repeat=3):
        o = a + b + c
        k = O.cumulant_of(mu, a, b, c)
        if o == 1:
            assert abs(k - mean[[a, b, c].index(1)]) < 1e-14
        elif o == 2:
            i = [d for d in range(3) for _ in range((a, b, c)[d])]
            assert abs(k - S[i[0], i[1]]) < 1e-14
        elif o > 2:
            assert abs(k) < 1e-13


def _isserlis(labels, S):
    if not labels:
        return 1.0
    if len(labels) % 2:
        return 0.0
    first, rest = labels[0], labels[1:]
    return sum(S[first, rest[j]] * _isserlis(rest[:j] + rest[j + 1:], S)
               for j in range(len(rest)))


@pytest.mark.parametrize("st", STENCILS)
def test_cumulant_round_trip(O, st):
    xi, w, ex = O.lattice(st)
    mats = O.matrices(st)
    rng = np.random.default_rng(9)
    f = w + 0.01 * rng.standard_normal(len(w))
    c = O.cumulants(st, f)
    np.testing.assert_allclose(O.moments_from_cumulants(st, c), mats["M"] @ f, atol=1e-15)


# ------------------------------------------------------------- collision
def _methods(st):
    out = []
    for sp, eq in [(1, 0), (1, 1), (2, 0), (2, 1), (3, 1)]:
        out.append((sp, eq))
    return out


@pytest.mark.parametrize("st", STENCILS)
def test_collision_fixed_point_conservation_and_unit_rates(O, st):
    xi, w, _ = O.lattice(st)
    rng = np.random.default_rng(13)
    for sp, eq in _methods(st):
        m = O.method(st, sp, eq, [1.7, 1.2, 1.3, 1.4, 1.5, 1.6])
        rho = 1 + 0.02 * rng.standard_normal(4)
        u = 0.06 * rng.standard_normal((4, 3))
        if st == 0:
            u[:, 2] = 0
        feq = O.equilibrium(m, rho, u)
        assert np.abs(O.collide(m, feq) - feq).max() < 2e-15
        df = feq + 1e-3 * rng.standard_normal(feq.shape)
        out = O.collide(m, df)
        assert np.abs(out.sum(1) - df.sum(1)).max() < 1e-15
        assert np.abs(out @ xi - df @ xi).max() < 1e-15
        m1 = O.method(st, sp, eq, [1.0] * 6)
        r2 = 1 + df.sum(1)
        eq2 = O.equilibrium(m1, r2, (df @ xi) / r2[:, None])
        assert np.abs(O.collide(m1, df) - eq2).max() < 2e-15


@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("sp", [1, 2])
def test_mrt_with_equal_rates_is_bgk(O, st, sp):
    """Raw and central MRT with every rate = omega reproduce BGK against the
    method's own equilibrium (T linear at fixed u)."""
    xi, w, _ = O.lattice(st)
    rng = np.random.default_rng(17)
    om = 1.63
    m = O.method(st, sp, 0, [om] * 6)
    df = 1e-3 * rng.standard_normal((6, len(w)))
    r = 1 + df.sum(1)
    u = (df @ xi) / r[:, None]
    feq = O.equilibrium(m, r, u)
    np.testing.assert_allclose(O.collide(m, df), df + om * (feq - df), rtol=0, atol=1e-15)
    srt = O.method(st, O.SPACE_POPULATIONS, 0, [om] * 6)
    if sp == 1:
        np.testing.assert_allclose(O.collide(srt, df), df + om * (feq - df), rtol=0, atol=1e-15)


@pytest.mark.parametrize("st", STENCILS)
def test_cumulant_collision_against_log_series(O, st):
    """Post-collision cumulants (computed by the independent log-series route)
    are the relaxed pre-collision ones: order-2 off-diagonal scaled by
    (1 - w_shear), order >= 3 by (1 - w_order)."""
    xi, w, ex = O.lattice(st)
    dim = 2 if st == 0 else 3
    rates = [1.6, 1.0, 1.3, 1.4, 1.5, 1.7]
    m = O.method(st, O.SPACE_CUMULANT, O.EQ_ABSOLUTE, rates)
    rng = np.random.default_rng(19)
    df = np.round(1e-2 * rng.standard_normal(len(w)) * 2 ** 24) / 2 ** 24
    out = O.collide(m, df)
    pre = _cumulants_by_log_series(xi.tolist(), (df + w).tolist(), dim)
    post = _cumulants_by_log_series(xi.tolist(), (out + w).tolist(), dim)
    for e in ex:
        e = tuple(e[:dim])
        o = sum(e)
        if o < 2 or (o == 2 and max(e) == 2):
            continue
        fac = 1 - (rates[0] if o == 2 else rates[o - 1])
        assert abs(float(post[e]) - fac * float(pre[e])) < 1e-14


# ------------------------------------------------------------- streaming
@pytest.mark.parametrize("st", STENCILS)
def test_pure_streaming_is_circular_shift(O, st):
    xi, w, _ = O.lattice(st)
    dims = (5, 4, 1) if st == 0 else (5, 4, 3)
    rng = np.random.default_rng(23)
    df = rng.standard_normal((len(w), dims[2], dims[1], dims[0]))
    m = O.method(st, O.SPACE_NONE, 0, [1.0] * 6)
    n = 7
    out = O.step(m, dims, df, n)
    for i in range(len(w)):
        ref = np.roll(df[i], shift=(n * xi[i, 2], n * xi[i, 1], n * xi[i, 0]), axis=(0, 1, 2))
        np.testing.assert_array_equal(out[i], ref)


def test_brute_force_srt_step_d2q9(O):
    """One full step on a 4x3 lattice by hand: BGK against the discrete
    Maxwellian (identical to the truncated moments on D2Q9), then push."""
    xi, w, _ = O.lattice(0)
    dims = (4, 3, 1)
    rng = np.random.default_rng(29)
    df = 1e-2 * rng.standard_normal((9, 1, 3, 4))
    om = 1.4
    m = O.method(0, O.SPACE_POPULATIONS, 0, [om] * 6)
    out = O.step(m, dims, df, 1)
    post = np.empty_like(df)
    for y in range(3):
        for x in range(4):
            f = df[:, 0, y, x] + w
            rho = f.sum()
            u = (f @ xi) / rho
            post[:, 0, y, x] = f + om * (_discrete_feq(xi, w, rho, u) - f) - w
    for i in range(9):
        ref = np.roll(post[i], shift=(xi[i, 2], xi[i, 1], xi[i, 0]), axis=(0, 1, 2))
        np.testing.assert_allclose(out[i], ref, rtol=0, atol=1e-15)


def test_inadmissible_delta_cumulant(O):
    m = O.method(2, O.SPACE_CUMULANT, O.EQ_DELTA, [1.0] * 6)
    with pytest.raises(O.OracleError):
        O.collide(m, np.zeros(27))


# --------------------------------------------------------- whole scheme
def test_taylor_green_decay_low_re(O):
    """D3Q19 O-MRT (R-) on the 32^3 Taylor-Green vortex: after the start-up
    transient of the equilibrium initialisation, the velocity amplitude decays
    at 2 nu kappa^2 and the energy at 4 nu kappa^2 (Eq. 5.1, 5.2)."""
    L, u0, nu, steps, fit0, tol = [float(x) for x in
                                   open(os.path.join(GOLDEN, "tgv_eq51.txt")).read()
                                   .split("\n")[-2].split()]
    L, steps, fit0 = int(L), int(steps), int(fit0)
    om = I.shear_viscosity_rate(nu)
    m = O.method(1, O.SPACE_RAW, O.EQ_DELTA, [om, 1, 1, 1, 1, 1])
    dims = (L, L, L)
    rho, u = I.taylor_green(dims, u0)
    df = O.init(m, dims, rho, u)
    k = 2 * np.pi / L
    x = np.arange(L)
    mode = np.cos(k * x)[None, None, :] * np.sin(k * x)[None, :, None]

    def amp_energy(state):
        r, uu = O.macroscopic(m, dims, state)
        return (uu[0] * mode).sum() / (mode * mode).sum(), 0.5 * (r * (uu ** 2).sum(0)).sum()

    df = O.step(m, dims, df, fit0)
    a1, e1 = amp_energy(df)
    df = O.step(m, dims, df, steps - fit0)
    a2, e2 = amp_energy(df)
    n = steps - fit0
    assert abs(-np.log(a2 / a1) / n / (2 * nu * k * k) - 1) < tol
    assert abs(-np.log(e2 / e1) / n / (4 * nu * k * k) - 1) < tol
