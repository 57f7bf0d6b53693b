"""GPU parity of the discrete second-order equilibrium (LBM_EQ_DISCRETE2:
q_eq = T(f_eq) with the polynomial f_eq prescribed as populations, Sec. 2.4)
against the FP64 oracle in every collision space, FP64 and FP32 storage,
general and regularised rates; the set-up is f_eq and a collision fixed
point; the combinations the library does not serve are refused."""
import numpy as np
import pytest

import oracle as O
from paper_2211_02435_b300 import build as B
from paper_2211_02435_b300 import inputs as I
from paper_2211_02435_b300 import lbm as L

pytestmark = pytest.mark.gpu

TOL = {L.STORE_F64: 1e-12, L.STORE_F32: 1e-5}
DIMS = {0: (133, 37, 1), 1: (133, 6, 5), 2: (133, 6, 5)}
RATES = {"gen": [1.7, 1.2, 1.3, 1.4, 1.5, 1.6], "reg": [1.9, 1.0, 1.0, 1.0, 1.0, 1.0],
         "srt": [1.6] * 6, "trt": [1.3, 1.0, 1.75, 1.0, 1.0, 1.0]}
SPACES = [(L.SPACE_POPULATIONS, "srt"), (L.SPACE_TRT, "trt"), (L.SPACE_RAW, "gen"),
          (L.SPACE_RAW, "reg"), (L.SPACE_RAW_WEIGHTED, "gen"), (L.SPACE_CENTRAL, "gen"),
          (L.SPACE_CENTRAL, "reg"), (L.SPACE_CUMULANT, "gen"), (L.SPACE_CUMULANT, "reg")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    O.build()


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def fields(st):
    dims = DIMS[st]
    rho, u = I.taylor_green(dims, 0.05, d=2 if st == 0 else 3)
    return dims, rho, I.add_uniform_noise(u, 1e-3, seed=11)


@pytest.mark.parametrize("storage", [L.STORE_F64, L.STORE_F32], ids=["f64", "f32"])
@pytest.mark.parametrize("sp", SPACES, ids=[f"sp{s}{r}" for s, r in SPACES])
@pytest.mark.parametrize("st", [0, 1, 2], ids=["D2Q9", "D3Q19", "D3Q27"])
def test_discrete_equilibrium_step_parity(st, sp, storage):
    space, rk = sp
    dims, rho, u = fields(st)
    m = O.method(st, space, O.EQ_DISCRETE2, RATES[rk])
    _, w, _ = O.lattice(st)
    df0 = O.init(m, dims, rho, u)
    pert = I.random_deviations(len(w), int(np.prod(dims)), 2e-3, seed=12)
    df0 = df0 + (w[:, None] * pert).reshape(df0.shape)
    with L.Lattice(st, space, L.EQ_DISCRETE2, storage, L.PULL, RATES[rk], dims) as lat:
        lat.set_populations(df0)
        done = 0
        for n in (3, 4):
            lat.step(n - done)
            done = n
            ref = O.step(m, dims, df0, n)
            assert rel_linf(lat.get_populations(), ref) < TOL[storage], n
            _, u_r = O.macroscopic(m, dims, ref)
            _, u_g = lat.macroscopic()
            assert rel_linf(u_g, u_r) < TOL[storage]


@pytest.mark.parametrize("space", [L.SPACE_RAW, L.SPACE_CENTRAL, L.SPACE_CUMULANT,
                                   L.SPACE_POPULATIONS])
@pytest.mark.parametrize("st", [0, 1, 2])
def test_set_up_is_feq_and_a_fixed_point(st, space):
    dims, rho, u = fields(st)
    rates = RATES["gen"] if space != L.SPACE_POPULATIONS else RATES["srt"]
    m = O.method(st, space, O.EQ_DISCRETE2, rates)
    ref = O.init(m, dims, rho, u)
    with L.Lattice(st, space, L.EQ_DISCRETE2, L.STORE_F64, L.PULL, rates, dims) as lat:
        lat.init_velocity(rho.reshape(-1), u.reshape(-1))
        assert rel_linf(lat.get_populations(), ref) < 1e-13
        lat.step(1)  # f_eq is a fixed point: one step is pure streaming
        shifted = O.step(O.method(st, O.SPACE_NONE, 0, [1.0] * 6), dims, ref, 1)
        assert rel_linf(lat.get_populations(), shifted) < 1e-12


def test_d3q19_equal_rate_mrt_is_bgk():
    """Raw-moment MRT with every rate equal, on D3Q19 with the discrete
    equilibrium, steps like SRT (the textbook BGK); with the truncated
    Maxwellian it does not."""
    st, om = 1, 1.45
    dims, rho, u = fields(st)
    m = O.method(st, O.SPACE_POPULATIONS, O.EQ_DISCRETE2, [om] * 6)
    df0 = O.init(m, dims, rho, u)
    _, w, _ = O.lattice(st)
    df0 = df0 + (w[:, None] * I.random_deviations(19, int(np.prod(dims)), 2e-3, 4)).reshape(df0.shape)
    out = {}
    for name, space, eq in (("mrt", L.SPACE_RAW, L.EQ_DISCRETE2),
                            ("bgk", L.SPACE_POPULATIONS, L.EQ_DISCRETE2),
                            ("mrt_max", L.SPACE_RAW, L.EQ_ABSOLUTE)):
        with L.Lattice(st, space, eq, L.STORE_F64, L.PULL, [om] * 6, dims) as lat:
            lat.set_populations(df0)
            lat.step(4)
            out[name] = lat.get_populations()
    assert rel_linf(out["mrt"], out["bgk"]) < 1e-13
    assert rel_linf(out["mrt_max"], out["bgk"]) > 1e-9


def test_refusals():
    base = dict(stencil=L.D3Q27, space=L.SPACE_CUMULANT, equilibrium=L.EQ_DISCRETE2,
                storage=L.STORE_F32, streaming=L.PULL, rates=[1.6] + [1.0] * 5, dims=(8, 8, 8))

    def make(**kw):
        p = dict(base, **kw)
        return L.Lattice(p["stencil"], p["space"], p["equilibrium"], p["storage"],
                         p["streaming"], p["rates"], p["dims"])

    for kw in (dict(storage=L.STORE_F16_DELTA), dict(storage=L.STORE_BF16_DELTA),
               dict(streaming=L.AA), dict(streaming=L.ESOTERIC_TWIST),
               dict(storage=L.STORE_F64_ABSOLUTE)):
        with pytest.raises(L.LBMError) as e:
            make(**kw)
        assert e.value.code == -2, kw
    with make() as lat:
        with pytest.raises(L.LBMError) as e:
            lat.set_force([1e-5, 0.0, 0.0])
        assert e.value.code == -2
        with pytest.raises(L.LBMError) as e:
            lat.set_step_kernel(L.STEP_STAGED)
        assert e.value.code == -2
    with pytest.raises(L.LBMError) as e:
        L.Batch(L.D3Q19, L.SPACE_RAW, L.EQ_DISCRETE2, L.STORE_F32, [1.0] * 6,
                [(8, 8, 8)], [1.5])
    assert e.value.code == -2
