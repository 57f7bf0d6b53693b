"""Parity at the full benchmark sizes, in the launch configurations bench.py
times, on sampled outputs the FP64 oracle computes one by one.

* D3Q27 cumulant (R-) on the 512^3 Taylor-Green vortex u0 = 0.05 with 1e-3
  noise: FP32 storage with pull streaming (the headline kernel) and the four
  in-place patterns, and FP16 / BF16 delta storage (the packed kernels),
  pull and in place.
* D3Q27 central moments (R-) on the 512^3 8-mode Fourier flow, FP16 / BF16
  delta storage.
* The 4096-domain D3Q19 O-MRT ensemble with the autotuned launch shape.

The oracle value of a sampled cell comes from the periodic (2n + 1)^3 cube
centred on it (tests/sampling.py, pinned against whole-lattice runs on the
CPU).  Samples include the lattice's corners and faces, where the GPU
gather wraps.
"""
import gc

import numpy as np
import pytest

import oracle as O
from paper_2211_02435_b300 import build as B
from paper_2211_02435_b300 import inputs as I
from paper_2211_02435_b300 import lbm as L
from sampling import cube_oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

EDGE = 512
DIMS = (EDGE, EDGE, EDGE)
NCELL = EDGE ** 3
STEPS = 3
RATES = [I.shear_viscosity_rate(1e-3)] + [1.0] * 5


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    O.build()
    yield
    gc.collect()
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def tgv_fields():
    rho, u = I.taylor_green(DIMS, 0.05)
    return rho, I.add_uniform_noise(u, 1e-3, seed=1)


@pytest.fixture(scope="module")
def fourier_fields():
    return I.fourier_modes(DIMS, n_modes=8, umax=0.08, seed=3)


def sample_cells(count=14, seed=11):
    e = EDGE - 1
    cells = [(0, 0, 0), (e, e, e), (0, e, 7), (e, 0, 300), (255, 0, e), (1, 256, 0)]
    rng = np.random.default_rng(seed)
    cells += [tuple(int(v) for v in rng.integers(0, EDGE, 3)) for _ in range(count - len(cells))]
    return cells


def gpu_samples(lat, cells):
    """Populations [q, S] and velocity [3, S] of the sampled cells, read out
    through the library into device buffers."""
    idx = torch.tensor([(z * EDGE + y) * EDGE + x for x, y, z in cells], device="cuda")
    out = torch.empty(lat.q * NCELL, dtype=torch.float64, device="cuda")
    lat.get_populations(out)
    df = out.view(lat.q, NCELL)[:, idx].cpu().numpy()
    del out
    rho = torch.empty(NCELL, dtype=torch.float64, device="cuda")
    u = torch.empty(3 * NCELL, dtype=torch.float64, device="cuda")
    lat.macroscopic(rho, u)
    uu = u.view(3, NCELL)[:, idx].cpu().numpy()
    del rho, u
    torch.cuda.empty_cache()
    return df, uu


def run_case(space, storage, streaming, rho, u, cells):
    rho_d = torch.from_numpy(np.ascontiguousarray(rho.reshape(-1))).cuda()
    u_d = torch.from_numpy(np.ascontiguousarray(u.reshape(-1))).cuda()
    with L.Lattice(L.D3Q27, space, L.EQ_ABSOLUTE, storage, streaming, RATES, DIMS) as lat:
        lat.init_velocity(rho_d, u_d)
        del rho_d, u_d
        lat.step(STEPS)
        assert lat.time()[0] == STEPS
        got = gpu_samples(lat, cells)
    gc.collect()
    torch.cuda.empty_cache()
    return got


def reference(space, rho, u, cells):
    m = O.method(O.D3Q27, space, O.EQ_ABSOLUTE, RATES)
    refs = [cube_oracle(m, DIMS, rho, u, c, STEPS) for c in cells]
    return np.stack([r[0] for r in refs], 1), np.stack([r[1] for r in refs], 1)


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


_ref_cache = {}
_fp32_pull = {}


def tgv_reference(tgv_fields, cells):
    if "tgv" not in _ref_cache:
        _ref_cache["tgv"] = reference(O.SPACE_CUMULANT, *tgv_fields, cells)
    return _ref_cache["tgv"]


@pytest.mark.parametrize("streaming", L.STREAMING_PATTERNS,
                         ids=["pull", "aa", "et", "epull", "epush"])
def test_fp32_cumulant_512_sampled(tgv_fields, streaming):
    cells = sample_cells()
    df, uu = run_case(L.SPACE_CUMULANT, L.STORE_F32, streaming, *tgv_fields, cells)
    ref_df, ref_u = tgv_reference(tgv_fields, cells)
    assert rel_linf(df, ref_df) < 1e-5
    assert rel_linf(uu, ref_u) < 1e-5
    # every pattern runs the pull kernel's per-cell arithmetic
    if streaming == L.PULL:
        _fp32_pull["df"] = df
    elif "df" in _fp32_pull:
        assert np.array_equal(df, _fp32_pull["df"])


_half_pull = {}


@pytest.mark.parametrize("streaming", L.STREAMING_PATTERNS,
                         ids=["pull", "aa", "et", "epull", "epush"])
@pytest.mark.parametrize("storage,p", [(L.STORE_F16_DELTA, 10), (L.STORE_BF16_DELTA, 7)],
                         ids=["f16", "bf16"])
def test_half_cumulant_512_sampled(tgv_fields, storage, p, streaming):
    """Packed FP16 / BF16 kernels (pull and in place): within (n + 1)
    2^-(p+1) of max |df| (one rounding of each scaled deviation per store,
    the initial encode included); the in-place patterns equal pull bit for
    bit."""
    cells = sample_cells()
    df, uu = run_case(L.SPACE_CUMULANT, storage, streaming, *tgv_fields, cells)
    ref_df, ref_u = tgv_reference(tgv_fields, cells)
    bound = (STEPS + 1) * 2.0 ** -(p + 1)
    assert rel_linf(df, ref_df) < bound
    assert rel_linf(uu, ref_u) < 4 * bound
    if streaming == L.PULL:
        _half_pull[storage] = df
    elif storage in _half_pull:
        assert np.array_equal(df, _half_pull[storage])


@pytest.mark.parametrize("storage,p", [(L.STORE_F16_DELTA, 10), (L.STORE_BF16_DELTA, 7)],
                         ids=["f16", "bf16"])
def test_half_central_fourier_512_sampled(fourier_fields, storage, p):
    cells = sample_cells(seed=12)
    df, uu = run_case(L.SPACE_CENTRAL, storage, L.PULL, *fourier_fields, cells)
    if "fourier" not in _ref_cache:
        _ref_cache["fourier"] = reference(O.SPACE_CENTRAL, *fourier_fields, cells)
    ref_df, ref_u = _ref_cache["fourier"]
    bound = (STEPS + 1) * 2.0 ** -(p + 1)
    assert rel_linf(df, ref_df) < bound
    assert rel_linf(uu, ref_u) < 4 * bound


def test_batched_ensemble_4096_sampled():
    """The bench's ensemble (4096 D3Q19 O-MRT R- Taylor-Green domains, edges
    16..96, per-instance viscosity, FP32) with the autotuned persistent
    launch; sampled instances of every edge length against the oracle."""
    gc.collect()
    torch.cuda.empty_cache()
    dims, nu, u0 = I.batch_ensemble(4096, seed=4)
    dims = [tuple(int(v) for v in d) for d in dims]
    om = [I.shear_viscosity_rate(v) for v in nu]
    with L.Batch(L.D3Q19, L.SPACE_RAW, L.EQ_DELTA, L.STORE_F32, [1.0] * 6, dims, om) as b:
        b.autotune(trial_steps=2)
        b.init_tgv(u0)
        b.step(STEPS)
        picks = {}
        for k, d in enumerate(dims):
            picks.setdefault(d[0], []).append(k)
        sample = [ks[0] for ks in picks.values()] + [len(dims) - 1]
        for k in sample:
            m = O.method(O.D3Q19, O.SPACE_RAW, O.EQ_DELTA, [om[k]] + [1.0] * 5)
            rho, u = I.taylor_green(dims[k], u0[k])
            ref = O.step(m, dims[k], O.init(m, dims[k], rho, u), STEPS)
            assert rel_linf(b.get_populations(k), ref) < 1e-5, k
            _, u_r = O.macroscopic(m, dims[k], ref)
            _, u_g = b.macroscopic(k)
            assert rel_linf(u_g, u_r) < 1e-5, k
    gc.collect()
    torch.cuda.empty_cache()
