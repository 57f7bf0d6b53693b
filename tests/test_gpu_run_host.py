"""The pipelined host job (lbm_run_host): set-up from host fields, n steps
and read-out to host with the copies and the steps of different slabs of
z-planes overlapping.  Every result equals lbm_init_velocity + lbm_step +
lbm_macroscopic bit for bit: 3 to many slabs (one plane per slab
included), uneven slabs, n = 0, 1, 2 and more steps, FP32 / FP16 / BF16
(packed and, for odd Nx, scalar) / FP64 storage, the discrete equilibrium,
with and without rho; the unsupported cases run the sequence."""
import numpy as np
import pytest

from paper_2211_02435_b300 import build as B
from paper_2211_02435_b300 import inputs as I
from paper_2211_02435_b300 import lbm as L

pytestmark = pytest.mark.gpu

RATES = [1.7] + [1.0] * 5


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def fields(dims, d=3):
    rho, u = I.taylor_green(dims, 0.05, d=d)
    u = I.add_uniform_noise(u, 1e-3, seed=3)
    return np.ascontiguousarray(rho.reshape(-1)), np.ascontiguousarray(u.reshape(-1))


def sequential(args, dims, rho, u, n, d=3):
    with L.Lattice(*args, dims) as lat:
        lat.init_velocity(rho, u)
        lat.step(n)
        r, v = lat.macroscopic()
        return r.reshape(-1), v.reshape(-1), lat.get_populations()


CASES = [
    ((L.D3Q27, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, L.STORE_F32, L.PULL, RATES), (40, 12, 23)),
    ((L.D3Q19, L.SPACE_RAW, L.EQ_DELTA, L.STORE_F16_DELTA, L.PULL, RATES), (34, 10, 17)),
    ((L.D3Q27, L.SPACE_CENTRAL, L.EQ_ABSOLUTE, L.STORE_F64, L.PULL, RATES), (19, 7, 9)),
    ((L.D3Q19, L.SPACE_TRT, L.EQ_DELTA, L.STORE_F32, L.PULL, [1.3, 1, 1.75, 1, 1, 1]), (21, 9, 11)),
    ((L.D3Q19, L.SPACE_CUMULANT, L.EQ_DISCRETE2, L.STORE_F64, L.PULL, RATES), (23, 8, 10)),
    ((L.D3Q27, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, L.STORE_BF16_DELTA, L.PULL, RATES), (33, 8, 12)),
]


@pytest.mark.parametrize("n", [0, 1, 2, 7])
@pytest.mark.parametrize("case", CASES, ids=["d3q27-k-f32", "d3q19-raw-f16", "d3q27-cm-f64",
                                             "d3q19-trt-f32", "d3q19-k-disc-f64",
                                             "d3q27-k-bf16-odd-nx"])
def test_run_host_equals_the_sequence(case, n):
    args, dims = case
    rho, u = fields(dims)
    r_ref, u_ref, f_ref = sequential(args, dims, rho, u, n)
    for slabs in (3, 4, 5, dims[2]):
        with L.Lattice(*args, dims) as lat:
            ro = np.empty_like(rho)
            uo = np.empty_like(u)
            lat.run_host(rho, u, n, ro, uo, slabs=slabs)
            assert lat.time() == (n, 0)
            assert np.array_equal(ro, r_ref), slabs
            assert np.array_equal(uo, u_ref), slabs
            # the context holds f(n): stepping on continues the same run
            assert np.array_equal(lat.get_populations(), f_ref), slabs


def test_run_host_without_rho_and_partial_outputs():
    args, dims = CASES[0]
    rho, u = fields(dims)
    ones = np.ones_like(rho)
    r_ref, u_ref, _ = sequential(args, dims, ones, u, 3)
    with L.Lattice(*args, dims) as lat:
        uo = np.empty_like(u)
        lat.run_host(None, u, 3, None, uo, slabs=6)
        assert np.array_equal(uo, u_ref)
    with L.Lattice(*args, dims) as lat:
        ro = np.empty_like(rho)
        lat.run_host(None, u, 3, ro, None, slabs=6)
        assert np.array_equal(ro, r_ref)


@pytest.mark.parametrize("args,dims", [
    ((L.D3Q27, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, L.STORE_F32, L.AA, RATES), (20, 6, 8)),
    ((L.D2Q9, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, L.STORE_F32, L.PULL, RATES), (40, 30, 1)),
    ((L.D3Q27, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, L.STORE_F32, L.PULL, RATES), (20, 6, 2)),
])
def test_run_host_sequential_cases(args, dims):
    d = 2 if args[0] == L.D2Q9 else 3
    rho, u = fields(dims, d)
    r_ref, u_ref, _ = sequential(args, dims, rho, u, 4, d)
    with L.Lattice(*args, dims) as lat:
        ro, uo = np.empty_like(rho), np.empty_like(u)
        lat.run_host(rho, u, 4, ro, uo)
        assert np.array_equal(ro, r_ref) and np.array_equal(uo, u_ref)


def test_run_host_with_a_force_runs_the_sequence():
    args, dims = CASES[0]
    rho, u = fields(dims)
    with L.Lattice(*args, dims) as a, L.Lattice(*args, dims) as b:
        for lat in (a, b):
            lat.set_force([1e-5, 0.0, 0.0])
        a.init_velocity(rho, u)
        a.step(3)
        r_ref, u_ref = a.macroscopic()
        ro, uo = np.empty_like(rho), np.empty_like(u)
        b.run_host(rho, u, 3, ro, uo, slabs=5)
        assert np.array_equal(ro, r_ref.reshape(-1)) and np.array_equal(uo, u_ref.reshape(-1))
