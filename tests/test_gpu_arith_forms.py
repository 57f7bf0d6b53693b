"""GPU parity of the paper's arithmetic forms (Sec. 2.3, Table 3) against
the FP64 oracle: the absolute-equilibrium collision Eq. 2.6 in absolute
arithmetic on zero-centered FP64 storage (LBM_ARITH_AS_WRITTEN: background
moments added to and removed from the raw moments), and absolute FP64
storage of f itself with the standard collision Eq. 2.4
(LBM_STORE_F64_ABSOLUTE).  All forms compute the oracle's EQ_ABSOLUTE
collision up to rounding and are held to 1e-12 relative L-inf over the
zero-centered populations."""
import functools

import numpy as np
import pytest

import oracle as O
from paper_2211_02435_b300 import build as B
from paper_2211_02435_b300 import inputs as I
from paper_2211_02435_b300 import lbm as L

pytestmark = pytest.mark.gpu

DIMS = {0: (133, 37, 1), 1: (133, 6, 5), 2: (133, 6, 5)}
RATES_GEN = [1.7, 1.2, 1.3, 1.4, 1.5, 1.6]
RATES_REG = [1.9, 1.0, 1.0, 1.0, 1.0, 1.0]
METHODS = [  # (space, regularised); equilibrium always absolute
    (L.SPACE_POPULATIONS, False), (L.SPACE_RAW, False), (L.SPACE_RAW, True),
    (L.SPACE_CENTRAL, False), (L.SPACE_CENTRAL, True),
    (L.SPACE_CUMULANT, False), (L.SPACE_CUMULANT, True),
    (L.SPACE_RAW_WEIGHTED, False), (L.SPACE_RAW_WEIGHTED, True),
]
FORMS = {  # name: (storage, arithmetic)
    "zc_feq": (L.STORE_F64, L.ARITH_AS_WRITTEN),
    "absolute": (L.STORE_F64_ABSOLUTE, L.ARITH_DEVIATION),
    "absolute_as_written": (L.STORE_F64_ABSOLUTE, L.ARITH_AS_WRITTEN),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    O.build()


def rates_of(space, reg):
    if space == L.SPACE_POPULATIONS:
        return [1.6] * 6
    return RATES_REG if reg else RATES_GEN


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@functools.lru_cache(maxsize=None)
def case(st, space, reg):
    dims = DIMS[st]
    d = 2 if st == 0 else 3
    rho, u = I.taylor_green(dims, 0.05, d=d)
    u = I.add_uniform_noise(u, 1e-3, seed=21)
    m = O.method(st, space, O.EQ_ABSOLUTE, rates_of(space, reg))
    df = O.init(m, dims, rho, u)
    _, w, _ = O.lattice(st)
    pert = I.random_deviations(len(w), int(np.prod(dims)), 2e-3, seed=22)
    df0 = df + (w[:, None] * pert).reshape(df.shape)
    return m, dims, df0, {n: O.step(m, dims, df0, n) for n in (3, 4)}


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("method", METHODS, ids=lambda m: f"sp{m[0]}reg{int(m[1])}")
@pytest.mark.parametrize("st", [0, 1, 2], ids=["D2Q9", "D3Q19", "D3Q27"])
def test_form_parity(st, method, form):
    space, reg = method
    storage, arith = FORMS[form]
    m, dims, df0, ref = case(st, space, reg)
    with L.Lattice(st, space, L.EQ_ABSOLUTE, storage, L.PULL, rates_of(space, reg), dims,
                   arithmetic=arith) as lat:
        lat.set_populations(df0)
        # absolute storage adds w_i on the way in and removes it on the way out
        assert rel_linf(lat.get_populations(), df0) < 1e-13
        done = 0
        for n in (3, 4):
            lat.step(n - done)
            done = n
            got = lat.get_populations()
            assert rel_linf(got, ref[n]) < 1e-12, n
            rho_r, u_r = O.macroscopic(m, dims, ref[n])
            rho_g, u_g = lat.macroscopic()
            assert rel_linf(u_g, u_r) < 1e-12
            assert rel_linf(rho_g - 1, rho_r - 1) < 1e-11


def test_absolute_storage_holds_f_itself():
    st, space, reg = 2, L.SPACE_RAW, False
    m, dims, df0, _ = case(st, space, reg)
    _, w, _ = O.lattice(st)
    with L.Lattice(st, space, L.EQ_ABSOLUTE, L.STORE_F64_ABSOLUTE, L.PULL, rates_of(space, reg),
                   dims) as lat:
        lat.set_populations(df0)
        n = df0.size
        f = lat.get_state()[-8 * n:].view(np.float64).reshape(df0.shape)
    # the pull set-up writes f_i(x) at x - xi_i: compare each plane as a set
    flat = np.sort(f.reshape(len(w), -1), axis=1)
    want = np.sort(df0.reshape(len(w), -1) + w[:, None], axis=1)
    assert np.abs(flat - want).max() <= 2e-16
    assert abs(flat.sum() / flat.shape[1] - 1.0) < 1e-3  # mean density ~ 1


def test_as_written_arithmetic_rounds_differently():
    """Eq. 2.6 as written and its deviation form agree to rounding but not
    bitwise: the selector changes the arithmetic, not the method."""
    st, space, reg = 2, L.SPACE_CENTRAL, False
    m, dims, df0, ref = case(st, space, reg)
    out = []
    for arith in (L.ARITH_DEVIATION, L.ARITH_AS_WRITTEN):
        with L.Lattice(st, space, L.EQ_ABSOLUTE, L.STORE_F64, L.PULL, rates_of(space, reg), dims,
                       arithmetic=arith) as lat:
            lat.set_populations(df0)
            lat.step(4)
            out.append(lat.get_populations())
    assert not np.array_equal(out[0], out[1])
    assert rel_linf(out[0], out[1]) < 1e-12


def test_unsupported_form_combinations():
    dims = (8, 8, 8)
    bad = [  # (space, eq, storage, streaming, arithmetic, code)
        (L.SPACE_RAW, L.EQ_DELTA, L.STORE_F64_ABSOLUTE, L.PULL, 0, -3),
        (L.SPACE_RAW, L.EQ_ABSOLUTE, L.STORE_F64_ABSOLUTE, L.AA, 0, -2),
        (L.SPACE_CENTRAL, L.EQ_ABSOLUTE, L.STORE_F32, L.PULL, L.ARITH_AS_WRITTEN, -2),
    ]
    for space, eq, storage, streaming, arith, code in bad:
        with pytest.raises(L.LBMError) as e:
            L.Lattice(2, space, eq, storage, streaming, RATES_GEN, dims, arithmetic=arith)
        assert e.value.code == code
    with pytest.raises(L.LBMError) as e:
        L.Batch(2, L.SPACE_RAW, L.EQ_ABSOLUTE, L.STORE_F64_ABSOLUTE, RATES_GEN, [dims])
    assert e.value.code == -2
