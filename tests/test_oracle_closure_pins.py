"""Pins of the oracle's learned-closure functions (features, MLP, closure
step, loss) against independent routes: eigenvalue invariants of directly
summed moments, symmetry of the lattice, closed-form networks, and the
already pinned fixed-rate collision."""
import itertools
import math

import numpy as np
import pytest

from paper_2211_02435_b300 import inputs as I

NP = 1444


@pytest.fixture(scope="module")
def O(oracle_lib):
    return oracle_lib


def _state(O, seed, st=2):
    xi, w, _ = O.lattice(st)
    rng = np.random.default_rng(seed)
    m = O.method(st, O.SPACE_CUMULANT, O.EQ_ABSOLUTE, [1.8] + [1.0] * 5)
    rho = 1 + 0.02 * rng.standard_normal()
    u = 0.06 * rng.standard_normal(3)
    return xi, w, O.equilibrium(m, rho, u)[0] + 3e-3 * w * rng.standard_normal(len(w))


def _features_direct(xi, w, df, om):
    f = df + w
    rho = f.sum()
    u = (f @ xi) / rho
    c = xi - u
    Pi = np.einsum("i,ia,ib->ab", f, c, c) / rho - np.eye(3) / 3
    S = -1.5 * om * Pi
    D = Pi - np.trace(Pi) / 3 * np.eye(3)

    def inv(A):
        # principal invariants and the Frobenius norm from the eigenvalues
        ev = np.linalg.eigvalsh(A)
        return (ev.sum(), ev[0] * ev[1] + ev[1] * ev[2] + ev[0] * ev[2], ev.prod(),
                np.sqrt((ev * ev).sum()))

    s1, s2, s3, ns = inv(S)
    _, d2, d3, nd = inv(D)
    return np.array([s1, s2 / ns, s3 / ns ** 2, d2 / nd, d3 / nd ** 2,
                     np.sqrt((Pi * Pi).sum()), rho - 1])


@pytest.mark.parametrize("st", [1, 2])
def test_features_equal_eigenvalue_invariants_of_summed_moments(O, st):
    for seed in range(5):
        xi, w, df = _state(O, seed, st)
        got = O.closure_features(st, df, 1.8)
        ref = _features_direct(xi, w, df, 1.8)
        np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-18)


def test_features_vanish_at_the_maxwellian_equilibrium(O):
    m = O.method(2, O.SPACE_CUMULANT, O.EQ_ABSOLUTE, [1.8] + [1.0] * 5)
    feq = O.equilibrium(m, 1.013, np.array([0.04, -0.03, 0.02]))[0]
    got = O.closure_features(2, feq, 1.8)
    assert np.abs(got[:6]).max() < 1e-15
    assert abs(got[6] - 0.013) < 1e-15


def _hermite2(O, st, A):
    """Zero-mass, zero-momentum populations whose second moment is exactly A:
    g_i = 9/2 w_i (xi_i xi_i - I/3) : A (fourth-order isotropy of the
    D3Q19 / D3Q27 weights, sum_i w_i xi xi xi xi = (delta delta + 2 perms)/9)."""
    xi, w, _ = O.lattice(st)
    return 4.5 * w * (np.einsum("ia,ib,ab->i", xi, xi, A) - np.trace(A) / 3)


@pytest.mark.parametrize("st", [1, 2])
def test_features_are_of_degree_one_in_the_second_moments(O, st):
    """At rest with f = w + lam g (g of second moment A) the normalised second
    central moments are Pi = lam A exactly, so every conditioned feature but
    the density is homogeneous of degree 1 in lam; under lam -> -lam the odd
    invariants (trace, determinants) change sign and the even ones do not."""
    rng = np.random.default_rng(7 + st)
    B = rng.standard_normal((3, 3))
    A = 1e-3 * (B + B.T)
    _, w, _ = O.lattice(st)
    g = _hermite2(O, st, A)
    base = O.closure_features(st, g, 1.7)
    # the oracle forms Pi from absolute moments (~1/3), so its rounding is
    # ~1e-16 absolute: amplitudes from 1e-4 keep it below the tolerance
    for lam in (0.1, 2.0, 10.0):
        got = O.closure_features(st, lam * g, 1.7)
        np.testing.assert_allclose(got[:6], lam * base[:6], rtol=1e-10, atol=1e-20)
        neg = O.closure_features(st, -lam * g, 1.7)
        sign = np.array([-1, 1, -1, 1, -1, 1])
        np.testing.assert_allclose(neg[:6], sign * lam * base[:6], rtol=1e-10, atol=1e-20)
        assert abs(got[6]) < 1e-16


def test_features_closed_forms(O):
    """Pi = eps diag(1, -1, 0): tr S = 0, I2(S)/|S| = -1.5 om eps/sqrt2, det S = 0,
    I2(D)/|D| = -eps/sqrt2, det D = 0, |Pi| = eps sqrt2.  Pi = eps diag(2, -1, -1):
    det S/|S|^2 = -om eps/2 and det D/|D|^2 = eps/3."""
    om, eps = 1.6, 2e-3
    g = _hermite2(O, 2, np.diag([eps, -eps, 0.0]))
    got = O.closure_features(2, g, om)
    r2 = np.sqrt(2.0)
    ref = [0.0, -1.5 * om * eps / r2, 0.0, -eps / r2, 0.0, eps * r2, 0.0]
    # zeros up to the rounding of absolute moments (~1e-16 times |S| ~ 1e-3)
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-14)
    g = _hermite2(O, 2, np.diag([2 * eps, -eps, -eps]))
    got = O.closure_features(2, g, om)
    assert abs(got[2] - (-0.5 * om * eps)) < 1e-10 * eps
    assert abs(got[4] - eps / 3) < 1e-10 * eps
    # a pure trace: S = s I, D = 0 (the D quotients are 0 by definition)
    g = _hermite2(O, 2, eps * np.eye(3))
    got = O.closure_features(2, g, om)
    s = -1.5 * om * eps
    np.testing.assert_allclose(got, [3 * s, 3 * s * s / (np.sqrt(3) * abs(s)),
                                     s ** 3 / (3 * s * s), 0, 0, eps * np.sqrt(3), 0],
                               rtol=1e-10, atol=1e-16)


def test_features_are_invariant_under_lattice_symmetries(O):
    xi, w, df = _state(O, 11)
    base = O.closure_features(2, df, 1.7)
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product([1, -1], repeat=3):
            P = np.zeros((3, 3))
            for a in range(3):
                P[a, perm[a]] = signs[a]
            mapped = (xi @ P.T).astype(int)
            idx = [int(np.where((xi == v).all(1))[0][0]) for v in mapped]
            df2 = np.empty_like(df)
            df2[idx] = df
            np.testing.assert_allclose(O.closure_features(2, df2, 1.7), base, rtol=1e-10,
                                       atol=1e-20)


def test_mlp_closed_form_cases(O):
    shift, scale = np.zeros(7), np.ones(7)
    raw = np.array([0.3, -0.2, 0.1, 0.05, -0.4, 0.2, 0.01])
    assert np.array_equal(O.closure_mlp(np.zeros(NP), shift, scale, raw), np.ones(4))
    p = np.zeros(NP)
    p[0] = 1.0  # W1[0][0]
    o2 = 32 * 7 + 32
    p[o2] = 1.0  # W2[0][0]
    o3 = o2 + 32 * 32 + 32
    c = np.array([0.7, -1.3, 2.0, -0.2])
    for k in range(4):
        p[o3 + k * 32] = c[k]  # W3[k][0]
    ref = 2.0 / (1.0 + np.exp(-c * math.tanh(math.tanh(raw[0]))))
    np.testing.assert_allclose(O.closure_mlp(p, shift, scale, raw), ref, rtol=1e-15)
    # normalisation, clamping and the non-finite fallback
    sh = np.array([0.1] + [0.0] * 6)
    sc = np.array([3.0] + [1.0] * 6)
    ref2 = 2.0 / (1.0 + np.exp(-c * math.tanh(math.tanh(3.0 * (raw[0] - 0.1)))))
    np.testing.assert_allclose(O.closure_mlp(p, sh, sc, raw), ref2, rtol=1e-15)
    big = p.copy()
    big[o3:o3 + 4 * 32] *= 1e4
    out = O.closure_mlp(big, shift, scale, raw)
    assert set(np.round(out, 6)) <= {1e-3, 1.999}
    bad = raw.copy()
    bad[3] = np.nan
    assert np.array_equal(O.closure_mlp(p, shift, scale, bad), np.ones(4))
    # a normalised input counts up to FP16's largest finite value, 65504
    # (the operand range of the GPU network), and falls back beyond it
    edge = raw.copy()
    edge[3] = -65504.0
    np.testing.assert_allclose(O.closure_mlp(p, shift, scale, edge), ref, rtol=1e-15)
    for v in (65504.5, -65505.0, np.inf):
        edge[3] = v
        assert np.array_equal(O.closure_mlp(p, shift, scale, edge), np.ones(4)), v


def _dims():
    return (6, 5, 4)


def _field(O, seed):
    dims = _dims()
    rho, u = I.taylor_green(dims, 0.05)
    u = I.add_uniform_noise(u, 5e-3, seed=seed)
    m = O.method(2, O.SPACE_CUMULANT, O.EQ_ABSOLUTE, [1.9] + [1.0] * 5)
    df = O.init(m, dims, rho, u)
    _, w, _ = O.lattice(2)
    pert = I.random_deviations(27, int(np.prod(dims)), 1e-3, seed=seed + 1)
    return dims, df + (w[:, None] * pert).reshape(df.shape)


def test_closure_step_with_constant_rates_is_the_plain_method(O):
    dims, df = _field(O, 3)
    shift, scale = np.zeros(7), np.ones(7)
    base = O.method(2, O.SPACE_CUMULANT, O.EQ_ABSOLUTE, [1.9, 1.0, 0.0, 0.0, 0.0, 0.0])
    p = np.zeros(NP)
    out = O.closure_step(base, dims, df, p, shift, scale)
    plain = O.step(O.method(2, O.SPACE_CUMULANT, O.EQ_ABSOLUTE, [1.9] + [1.0] * 5), dims, df, 1)
    np.testing.assert_allclose(out, plain, rtol=0, atol=1e-17)
    om = np.array([1.3, 0.7, 1.6, 1.1])
    o3 = 32 * 7 + 32 + 32 * 32 + 32 + 4 * 32
    p[o3:o3 + 4] = np.log(om / (2 - om))  # b3 = logit(omega / 2)
    out = O.closure_step(base, dims, df, p, shift, scale)
    plain = O.step(O.method(2, O.SPACE_CUMULANT, O.EQ_ABSOLUTE, [1.9, 1.0] + list(om)), dims, df, 1)
    np.testing.assert_allclose(out, plain, rtol=0, atol=1e-16)


def test_closure_loss_is_mean_squared_velocity_error_of_one_step(O):
    dims, df = _field(O, 5)
    _, target = _field(O, 9)
    base = O.method(2, O.SPACE_CUMULANT, O.EQ_ABSOLUTE, [1.9, 1.0, 0.0, 0.0, 0.0, 0.0])
    rng = np.random.default_rng(1)
    p = 0.3 * rng.standard_normal(NP)
    shift, scale = np.zeros(7), np.full(7, 50.0)
    loss = O.closure_loss(base, dims, df, target, p, shift, scale)
    stepped = O.closure_step(base, dims, df, p, shift, scale)
    _, u1 = O.macroscopic(base, dims, stepped)
    _, u2 = O.macroscopic(base, dims, target)
    assert abs(loss - ((u1 - u2) ** 2).sum() / np.prod(dims)) < 1e-18


def test_rollout_loss_is_zero_on_its_own_trajectory_and_matches_fixed_rate_steps(O):
    """K-step rollout loss: with targets taken from the plain method's own
    trajectory the zero network (rates 1) scores exactly 0; a network of
    constant rates scores the mean over the K steps of the squared velocity
    differences between two fixed-rate runs of the already pinned step."""
    dims, df = _field(O, 4)
    N = int(np.prod(dims))
    plain_m = O.method(2, O.SPACE_CUMULANT, O.EQ_ABSOLUTE, [1.9] + [1.0] * 5)
    base = O.method(2, O.SPACE_CUMULANT, O.EQ_ABSOLUTE, [1.9, 1.0, 0.0, 0.0, 0.0, 0.0])
    K = 3
    traj = [df]
    for _ in range(K):
        traj.append(O.step(plain_m, dims, traj[-1], 1))
    shift, scale = np.zeros(7), np.ones(7)
    p = np.zeros(NP)
    assert O.closure_rollout_loss(base, dims, traj, p, shift, scale) == 0.0
    om = np.array([0.4, 1.7, 1.2, 0.9])
    o3 = 32 * 7 + 32 + 32 * 32 + 32 + 4 * 32
    p[o3:o3 + 4] = np.log(om / (2 - om))
    fixed = O.method(2, O.SPACE_CUMULANT, O.EQ_ABSOLUTE, [1.9, 1.0] + list(om))
    ref, cur = 0.0, df
    for k in range(1, K + 1):
        cur = O.step(fixed, dims, cur, 1)
        _, u1 = O.macroscopic(plain_m, dims, cur)
        _, u2 = O.macroscopic(plain_m, dims, traj[k])
        ref += ((u1 - u2) ** 2).sum() / N
    got = O.closure_rollout_loss(base, dims, traj, p, shift, scale)
    assert ref > 0 and abs(got - ref / K) <= 1e-9 * ref / K
    # one step is the one-step loss
    one = O.closure_rollout_loss(base, dims, traj[:2], p, shift, scale)
    assert one == O.closure_loss(base, dims, traj[0], traj[1], p, shift, scale)
