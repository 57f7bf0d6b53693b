"""GPU tests of the batched ensemble (include/lbm_batch.h): per-instance
parity with the FP64 oracle, persistent vs per-instance launches vs the
single-domain path (bitwise), graph replay vs single launches, the device
Taylor-Green set-up and the autotuner."""
import numpy as np
import pytest

import oracle as O
from paper_2211_02435_b300 import build as B
from paper_2211_02435_b300 import inputs as I
from paper_2211_02435_b300 import lbm as L

pytestmark = pytest.mark.gpu

ST = L.D3Q19
RATES = [1.0] * 6  # bulk and higher orders at rate 1 (R-); shear per instance


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    O.build()


def ensemble(n=24, seed=4):
    dims, nu, u0 = I.batch_ensemble(n, edges=(16, 24, 32), seed=seed)
    dims = [tuple(d) for d in dims]
    # a few non-cubic, ragged boxes as well
    dims[1] = (17, 9, 5)
    dims[2] = (133, 3, 4)
    dims[3] = (5, 7, 11)
    return dims, [I.shear_viscosity_rate(v) for v in nu], u0


def host_fields(dims, u0):
    rho, u = I.taylor_green(dims, u0)
    return rho.reshape(-1), u.reshape(-1)


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("space", [L.SPACE_RAW, L.SPACE_TRT])
@pytest.mark.parametrize("storage,tol", [(L.STORE_F64, 1e-12), (L.STORE_F32, 1e-5)])
def test_instances_match_oracle(storage, tol, space):
    dims, om, u0 = ensemble()
    nsteps = 5
    rates = RATES if space == L.SPACE_RAW else [1.0, 1.0, 1.75, 1.0, 1.0, 1.0]
    with L.Batch(ST, space, L.EQ_DELTA, storage, rates, dims, om) as b:
        for k in range(len(dims)):
            b.init_velocity(k, *host_fields(dims[k], u0[k]))
        b.step(nsteps)
        assert b.time() == nsteps
        rng = np.random.default_rng(8)
        for k in sorted(set([1, 2, 3] + list(rng.choice(len(dims), 5, replace=False)))):
            m = O.method(O.D3Q19, space, O.EQ_DELTA, [om[k]] + rates[1:])
            rho, u = I.taylor_green(dims[k], u0[k])
            ref = O.step(m, dims[k], O.init(m, dims[k], rho, u), nsteps)
            assert rel_linf(b.get_populations(k), ref) < tol, k
            _, u_r = O.macroscopic(m, dims[k], ref)
            _, u_g = b.macroscopic(k)
            assert rel_linf(u_g, u_r) < tol, k


def test_persistent_per_instance_and_single_domain_agree_bitwise():
    dims, om, u0 = ensemble()
    out = {}
    for mode in (0, 1):
        with L.Batch(ST, L.SPACE_RAW, L.EQ_DELTA, L.STORE_F32, RATES, dims, om) as b:
            b.set_tuning(128, 2, 4, per_instance=mode)
            for k in range(len(dims)):
                b.init_velocity(k, *host_fields(dims[k], u0[k]))
            b.step(3)
            out[mode] = [b.get_populations(k) for k in range(len(dims))]
    for k in range(len(dims)):
        assert np.array_equal(out[0][k], out[1][k])
    for k in (0, 2):
        with L.Lattice(ST, L.SPACE_RAW, L.EQ_DELTA, L.STORE_F32, L.PULL, [om[k]] + [1.0] * 5,
                       dims[k]) as lat:
            lat.init_velocity(*host_fields(dims[k], u0[k]))
            lat.step(3)
            assert np.array_equal(lat.get_populations(), out[0][k])


def test_graph_replay_equals_single_launches_and_retuning():
    dims, om, u0 = ensemble(12, seed=7)
    res = []
    for split in ((7,), (1,) * 7, (2, 3, 2)):
        with L.Batch(ST, L.SPACE_RAW, L.EQ_DELTA, L.STORE_F32, RATES, dims, om) as b:
            for k in range(len(dims)):
                b.init_velocity(k, *host_fields(dims[k], u0[k]))
            for j, n in enumerate(split):
                if len(split) == 3:  # change the launch shape between replays
                    b.set_tuning(*[(64, 1, 16), (256, 8, 4), (128, 4, 8)][j])
                b.step(n)
            res.append([b.get_populations(k) for k in range(len(dims))])
    for r in res[1:]:
        for k in range(len(dims)):
            assert np.array_equal(r[k], res[0][k])


def test_device_taylor_green_setup_matches_host_fields():
    dims, om, u0 = ensemble(10, seed=9)
    with L.Batch(ST, L.SPACE_RAW, L.EQ_DELTA, L.STORE_F64, RATES, dims, om) as b:
        b.init_tgv(u0)
        for k in range(len(dims)):
            m = O.method(O.D3Q19, O.SPACE_RAW, O.EQ_DELTA, [om[k]] + [1.0] * 5)
            rho, u = I.taylor_green(dims[k], u0[k])
            ref = O.init(m, dims[k], rho, u)
            assert rel_linf(b.get_populations(k), ref) < 1e-13


def test_autotune_returns_a_valid_shape_and_keeps_results():
    dims, om, u0 = ensemble(16, seed=5)
    with L.Batch(ST, L.SPACE_RAW, L.EQ_DELTA, L.STORE_F32, RATES, dims, om) as b:
        t, mlups = b.autotune(trial_steps=2)
        assert t["threads"] in (64, 128, 256) and t["cells_per_thread"] in (1, 2, 4, 8)
        assert mlups > 0
        assert b.get_tuning() == t
        for k in range(len(dims)):
            b.init_velocity(k, *host_fields(dims[k], u0[k]))
        b.step(4)
        got = b.get_populations(0)
    with L.Lattice(ST, L.SPACE_RAW, L.EQ_DELTA, L.STORE_F32, L.PULL, [om[0]] + [1.0] * 5,
                   dims[0]) as lat:
        lat.init_velocity(*host_fields(dims[0], u0[0]))
        lat.step(4)
        assert np.array_equal(lat.get_populations(), got)


def test_batch_rejects_bad_arguments():
    with pytest.raises(L.LBMError) as e:
        L.Batch(ST, L.SPACE_RAW, L.EQ_DELTA, L.STORE_F32, RATES, [(8, 8, 8), (0, 4, 4)])
    assert e.value.code == -1
    with pytest.raises(L.LBMError) as e:
        L.Batch(ST, L.SPACE_RAW, L.EQ_DELTA, L.STORE_F32, RATES, [(8, 8, 8)], [2.5])
    assert e.value.code == -1
    with L.Batch(ST, L.SPACE_RAW, L.EQ_DELTA, L.STORE_F32, RATES, [(8, 8, 8)]) as b:
        with pytest.raises(L.LBMError):
            b.set_tuning(100, 1, 1)
        assert L.lib().lbm_batch_get_populations(b._h, 3, None, 0) == -1
        assert L.lib().lbm_batch_step(b._h, -1) == -1
