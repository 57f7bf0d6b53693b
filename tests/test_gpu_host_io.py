"""Host-pointer set-up and read-out on lattices large enough to move in
slabs (the copy of slab k overlapping the kernel of slab k - 1, with a
ragged last slab): every result equals the device-pointer path bit for
bit, for planes (3-D) and rows (2-D), pull and in-place layouts."""
import numpy as np
import pytest

from paper_2211_02435_b300 import build as B
from paper_2211_02435_b300 import inputs as I
from paper_2211_02435_b300 import lbm as L

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

CASES = [
    # stencil, space, eq, storage, streaming, dims (rho/u and df both in slabs)
    (L.D3Q27, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, L.STORE_F32, L.PULL, (208, 208, 208)),
    (L.D3Q19, L.SPACE_RAW, L.EQ_DELTA, L.STORE_F16_DELTA, L.AA, (211, 205, 203)),
    (L.D2Q9, L.SPACE_CENTRAL, L.EQ_ABSOLUTE, L.STORE_F64, L.ESOTERIC_TWIST, (4099, 3001, 1)),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


@pytest.mark.parametrize("case", CASES, ids=["d3q27-f32-pull", "d3q19-f16-aa", "d2q9-f64-et"])
def test_host_slab_path_equals_device_path(case):
    st, space, eq, storage, streaming, dims = case
    d = 2 if st == L.D2Q9 else 3
    rho, u = I.taylor_green(dims, 0.05, d=d)
    u = I.add_uniform_noise(u, 1e-3, seed=2)
    rho_h = np.ascontiguousarray(rho.reshape(-1))
    u_h = np.ascontiguousarray(u.reshape(-1))
    rates = [1.7] + [1.0] * 5
    mk = lambda: L.Lattice(st, space, eq, storage, streaming, rates, dims)
    with mk() as a, mk() as b:
        q, N = a.q, a.N
        a.init_velocity(rho_h, u_h)
        b.init_velocity(torch.from_numpy(rho_h).cuda(), torch.from_numpy(u_h).cuda())
        fa = torch.empty(q * N, dtype=torch.float64, device="cuda")
        fb = torch.empty(q * N, dtype=torch.float64, device="cuda")
        a.get_populations(fa)
        b.get_populations(fb)
        assert torch.equal(fa, fb)
        a.step(3)
        b.step(3)
        host = a.get_populations()  # host read-out in slabs
        b.get_populations(fb)
        assert np.array_equal(host.reshape(-1), fb.cpu().numpy())
        rh, uh = a.macroscopic()
        rd = torch.empty(N, dtype=torch.float64, device="cuda")
        ud = torch.empty(d * N, dtype=torch.float64, device="cuda")
        b.macroscopic(rd, ud)
        assert np.array_equal(rh.reshape(-1), rd.cpu().numpy())
        assert np.array_equal(uh.reshape(-1), ud.cpu().numpy())
        # velocity only, density only
        u_only = np.empty(d * N)
        a.macroscopic(None, u_only)
        assert np.array_equal(u_only, ud.cpu().numpy())
        r_only = np.empty(N)
        a.macroscopic(r_only, None)
        assert np.array_equal(r_only, rd.cpu().numpy())
        # host set-up of populations in slabs
        a.set_populations(host)
        a.get_populations(fa)
        b.set_populations(fb)
        b.get_populations(fb)
        assert torch.equal(fa, fb)
