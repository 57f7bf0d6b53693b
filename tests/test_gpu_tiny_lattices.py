"""GPU parity on degenerate lattices: boxes down to one cell, where one
thread applies the periodic wrap at both ends of an axis (Nx = 1, and Nx =
2 or 4 for the packed FP16 / BF16 kernels that take two or four cells per
thread), or a neighbour row or plane is the cell's own (Ny = 1, Nz = 1).
Every stencil, storage form and streaming pattern against the FP64 oracle
after an odd and an even number of steps (both AA parities), with the
tolerances of the other parity tests; and a batched ensemble of such boxes.
"""
import numpy as np
import pytest

import oracle as O
from paper_2211_02435_b300 import build as B
from paper_2211_02435_b300 import inputs as I
from paper_2211_02435_b300 import lbm as L

pytestmark = pytest.mark.gpu

TINY = {
    L.D2Q9: [(1, 1, 1), (2, 1, 1), (4, 1, 1), (3, 2, 1), (2, 3, 1), (8, 1, 1), (6, 5, 1)],
    L.D3Q19: [(1, 1, 1), (2, 1, 1), (4, 1, 1), (1, 1, 2), (2, 2, 2), (3, 1, 2), (4, 3, 1),
              (6, 2, 3)],
    L.D3Q27: [(1, 1, 1), (2, 1, 1), (4, 1, 1), (1, 1, 2), (2, 2, 2), (3, 1, 2), (4, 3, 1),
              (6, 2, 3)],
}
CASES = [(st, dims) for st, shapes in TINY.items() for dims in shapes]
# (storage, bound): the FP16 / BF16 bound is (n + 1) rounding units, as for
# the larger lattices
STORAGE = [(L.STORE_F64, lambda n: 1e-12), (L.STORE_F32, lambda n: 1e-5),
           (L.STORE_F16_DELTA, lambda n: (n + 1) * 2.0 ** -11),
           (L.STORE_BF16_DELTA, lambda n: (n + 1) * 2.0 ** -8)]
METHODS = [  # (space, equilibrium, rates): the regularised cumulant method and general raw MRT
    (L.SPACE_CUMULANT, L.EQ_ABSOLUTE, [1.9, 1.0, 1.0, 1.0, 1.0, 1.0]),
    (L.SPACE_RAW, L.EQ_DELTA, [1.7, 1.2, 1.3, 1.4, 1.5, 1.6]),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    O.build()


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def initial(st, space, eq, rates, dims, seed):
    """Unit density and a seeded velocity, uniform in +-0.05 per component
    (the Taylor-Green amplitude of the other parity tests), at the method's
    equilibrium, plus a random non-equilibrium part: a state that moves on
    any box size (a Taylor-Green field vanishes at Nx = 1)."""
    d = 2 if st == L.D2Q9 else 3
    N = int(np.prod(dims))
    rho = np.ones(N)
    u = np.random.default_rng(seed).uniform(-5e-2, 5e-2, d * N)
    m = O.method(st, space, eq, rates)
    df0 = O.init(m, dims, rho, u)
    _, w, _ = O.lattice(st)
    pert = I.random_deviations(len(w), N, 2e-3, seed=seed + 1)
    return m, df0 + (w[:, None] * pert).reshape(df0.shape)


@pytest.mark.parametrize("streaming", L.STREAMING_PATTERNS)
@pytest.mark.parametrize("storage,bound", STORAGE, ids=["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("method", METHODS, ids=["cumulant_reg", "raw_general"])
@pytest.mark.parametrize("st,dims", CASES, ids=[f"q{len(O.lattice(s)[1])}_{d[0]}x{d[1]}x{d[2]}"
                                               for s, d in CASES])
def test_tiny_box_matches_oracle(st, dims, method, storage, bound, streaming):
    space, eq, rates = method
    m, df0 = initial(st, space, eq, rates, dims, seed=21)
    with L.Lattice(st, space, eq, storage, streaming, rates, dims) as lat:
        lat.set_populations(df0)
        ref = df0
        done = 0
        for n in (3, 4):
            lat.step(n - done)
            ref = O.step(m, dims, ref, n - done)
            done = n
            got = lat.get_populations()
            assert rel_linf(got, ref) < bound(n), (n, rel_linf(got, ref))
            _, u_r = O.macroscopic(m, dims, ref)
            _, u_g = lat.macroscopic()
            assert np.abs(u_g - u_r).max() <= bound(n) * np.abs(u_r).max() + 1e-15, n


@pytest.mark.parametrize("storage,tol", [(L.STORE_F64, 1e-12), (L.STORE_F32, 1e-5)],
                         ids=["f64", "f32"])
def test_batched_ensemble_of_tiny_boxes(storage, tol):
    """One persistent launch over instances from one cell up: each instance
    against the oracle after 5 steps."""
    dims = [(1, 1, 1), (2, 1, 1), (4, 3, 2), (3, 1, 2), (1, 2, 1), (5, 1, 1), (2, 2, 2)]
    om = [1.2, 1.5, 0.9, 1.8, 1.1, 1.6, 1.3]
    rates = [1.0] * 6
    d = 3
    with L.Batch(L.D3Q19, L.SPACE_RAW, L.EQ_DELTA, storage, rates, dims, om) as b:
        fields = []
        for k, box in enumerate(dims):
            N = int(np.prod(box))
            rho = np.ones(N)
            u = np.random.default_rng(30 + k).uniform(-5e-2, 5e-2, d * N)
            fields.append((rho, u))
            b.init_velocity(k, rho, u)
        b.step(5)
        for k, box in enumerate(dims):
            m = O.method(O.D3Q19, L.SPACE_RAW, O.EQ_DELTA, [om[k]] + rates[1:])
            ref = O.step(m, box, O.init(m, box, *fields[k]), 5)
            assert rel_linf(b.get_populations(k), ref) < tol, (k, box)


@pytest.mark.parametrize("streaming", L.STREAMING_PATTERNS)
def test_zero_steps_leave_the_state_and_negative_counts_are_refused(streaming):
    dims = (6, 2, 3)
    space, eq, rates = METHODS[0]
    m, df0 = initial(L.D3Q27, space, eq, rates, dims, seed=5)
    with L.Lattice(L.D3Q27, space, eq, L.STORE_F32, streaming, rates, dims) as lat:
        lat.set_populations(df0)
        lat.step(1)  # an odd AA parity: the read-out gathers
        before, t0 = lat.get_populations(), lat.time()
        lat.step(0)
        assert np.array_equal(lat.get_populations(), before)
        assert L.lib().lbm_step(lat._h, -1) == -1
        assert np.array_equal(lat.get_populations(), before)
        assert lat.time() == t0
