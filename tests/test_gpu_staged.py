"""The shared-memory staged pull kernel (LBM_STEP_STAGED, bulk asynchronous
copies of whole source rows) against the direct pull kernel: the same
per-cell arithmetic, so the FP16 / BF16 states (explicit packed FMAs) must
be bitwise equal and the FP32 / FP64 states equal up to the compiler's
multiply-add contraction, and both within the parity tolerance of the
oracle.  Lattices have more rows than the
persistent grid has CTAs in some cases and fewer in others, small Ny / Nz
(periodic wrap of the source rows) and Nx a multiple of 8."""
import numpy as np
import pytest

import oracle as O
from paper_2211_02435_b300 import build as B
from paper_2211_02435_b300 import inputs as I
from paper_2211_02435_b300 import lbm as L

pytestmark = pytest.mark.gpu

RATES_GEN = [1.7, 1.2, 1.3, 1.4, 1.5, 1.6]
RATES_REG = [1.9, 1.0, 1.0, 1.0, 1.0, 1.0]


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    O.build()


def start(st, space, eq, rates, dims, seed):
    d = 2 if st == 0 else 3
    rho, u = I.taylor_green(dims, 0.05, d=d)
    u = I.add_uniform_noise(u, 1e-3, seed=seed)
    m = O.method(st, space, eq, rates)
    df = O.init(m, dims, rho, u)
    _, w, _ = O.lattice(st)
    pert = I.random_deviations(len(w), int(np.prod(dims)), 2e-3, seed=seed + 1)
    return m, df + (w[:, None] * pert).reshape(df.shape)


def run(st, space, eq, storage, rates, dims, df0, kernel, n):
    with L.Lattice(st, space, eq, storage, L.PULL, rates, dims) as lat:
        lat.set_step_kernel(kernel)
        lat.set_populations(df0)
        lat.step(n)
        out = lat.get_populations()
        inv = lat.invariants()
    return out, inv


CASES = [  # (stencil, space, eq, rates, dims)
    (2, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, RATES_REG, (64, 5, 4)),
    (2, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, RATES_GEN, (32, 3, 3)),
    (2, L.SPACE_CENTRAL, L.EQ_ABSOLUTE, RATES_REG, (48, 7, 2)),
    (1, L.SPACE_RAW, L.EQ_DELTA, RATES_GEN, (40, 6, 5)),
    (1, L.SPACE_CENTRAL, L.EQ_DELTA, RATES_REG, (64, 33, 31)),
    (0, L.SPACE_RAW, L.EQ_DELTA, RATES_REG, (256, 37, 1)),
    (0, L.SPACE_POPULATIONS, L.EQ_DELTA, [1.6] * 6, (24, 11, 1)),
    (2, L.SPACE_POPULATIONS, L.EQ_DELTA, [1.6] * 6, (16, 2, 3)),
    (1, L.SPACE_TRT, L.EQ_DELTA, [1.3, 1.0, 1.75, 1.0, 1.0, 1.0], (32, 5, 3)),
]


@pytest.mark.parametrize("storage", [L.STORE_F64, L.STORE_F32, L.STORE_F16_DELTA,
                                     L.STORE_BF16_DELTA])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_staged_equals_direct(case, storage):
    st, space, eq, rates, dims = CASES[case]
    m, df0 = start(st, space, eq, rates, dims, seed=40 + case)
    a, ia = run(st, space, eq, storage, rates, dims, df0, L.STEP_DIRECT, 5)
    b, ib = run(st, space, eq, storage, rates, dims, df0, L.STEP_STAGED, 5)
    if storage in (L.STORE_F16_DELTA, L.STORE_BF16_DELTA):
        # packed kernels spell out every fused multiply-add: bitwise equal
        assert np.array_equal(a, b)
        assert ia == ib
    else:
        # scalar kernels leave the multiply-add contraction to the compiler,
        # which may contract a few products differently in the two kernels
        tol = 1e-13 if storage == L.STORE_F64 else 1e-6
        assert np.abs(a - b).max() / np.abs(a).max() < tol
    if storage in (L.STORE_F64, L.STORE_F32):
        ref = O.step(m, dims, df0, 5)
        tol = 1e-12 if storage == L.STORE_F64 else 1e-5
        assert np.abs(b - ref).max() / np.abs(ref).max() < tol


def test_staged_large_rows_and_many_rows():
    """Nx = 512 (the largest FP32 D3Q27 row the stage buffers take) and more
    rows than the persistent grid has CTAs."""
    st, space, eq, rates = 2, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, RATES_REG
    dims = (512, 40, 30)
    rho, u = I.taylor_green(dims, 0.05)
    u = I.add_uniform_noise(u, 1e-3, seed=7)
    out = {}
    for storage in (L.STORE_F32, L.STORE_F16_DELTA):
        for kernel in (L.STEP_DIRECT, L.STEP_STAGED):
            with L.Lattice(st, space, eq, storage, L.PULL, rates, dims) as lat:
                lat.set_step_kernel(kernel)
                lat.init_velocity(rho.reshape(-1), u.reshape(-1))
                lat.step(3)
                out[storage, kernel] = lat.get_populations()
        a, b = out[storage, L.STEP_DIRECT], out[storage, L.STEP_STAGED]
        if storage == L.STORE_F16_DELTA:
            assert np.array_equal(a, b)
        else:
            assert np.abs(a - b).max() / np.abs(a).max() < 1e-6


def test_staged_rejects_what_it_cannot_run():
    bad = [  # (storage, streaming, dims, arithmetic)
        (L.STORE_F32, L.AA, (64, 4, 4), 0),
        (L.STORE_F16_DELTA, L.PULL, (36, 4, 4), 0),     # row 72 B, not a multiple of 16
        (L.STORE_F32, L.PULL, (1024, 2, 2), 0),         # 2 x 27 x 4 KiB > 110 KiB
        (L.STORE_F64, L.PULL, (64, 4, 4), L.ARITH_AS_WRITTEN),
        (L.STORE_F64_ABSOLUTE, L.PULL, (64, 4, 4), 0),
    ]
    for storage, streaming, dims, arith in bad:
        with L.Lattice(2, L.SPACE_CENTRAL, L.EQ_ABSOLUTE, storage, streaming, RATES_REG, dims,
                       arithmetic=arith) as lat:
            with pytest.raises(L.LBMError) as e:
                lat.set_step_kernel(L.STEP_STAGED)
            assert e.value.code == -2
            lat.set_step_kernel(L.STEP_DIRECT)
            lat.set_step_kernel(L.STEP_AUTO)
            with pytest.raises(L.LBMError) as e:
                lat.set_step_kernel(3)
            assert e.value.code == -1


@pytest.mark.parametrize("storage,tol", [(L.STORE_F32, 1e-5), (L.STORE_F16_DELTA, 4 * 2.0 ** -11)])
def test_bounded_wait_that_runs_out_reports_timeout_and_the_context_recovers(storage, tol):
    """Failure detection without a fault: with a wait bound of 0 cycles the
    staged kernel's first wait for its rows' bulk copies gives up, the CTA
    lets the copies already issued land and returns, and the next
    synchronising call reports LBM_ERR_TIMEOUT once.  With the default bound
    restored and the state set again, the same context steps to oracle
    parity."""
    rates = RATES_REG
    dims = (64, 6, 5)
    m, df0 = start(2, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, rates, dims, 71)
    ref = O.step(m, dims, df0, 2)
    with L.Lattice(2, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, storage, L.PULL, rates, dims) as lat:
        lat.set_step_kernel(L.STEP_STAGED)
        lat.set_populations(df0)
        lat.set_wait_limit(0)
        lat.step(1)
        with pytest.raises(L.LBMError) as e:
            lat.get_populations()
        assert e.value.code == -8  # LBM_ERR_TIMEOUT
        lat.set_wait_limit(2 ** 31)
        lat.set_populations(df0)
        lat.step(2)
        got = lat.get_populations()  # reported once: no error now
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= tol * scale
    with pytest.raises(L.LBMError):
        with L.Lattice(2, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, storage, L.PULL, rates, dims) as lat:
            lat.set_wait_limit(-1)
