"""GPU parity at the largest boxes the library accepts.  The step kernels form
cell index + periodic wrap correction in 32-bit integers, and lbm_create
refuses a box unless N + Nx*Ny + 2*Nx + 4096 < 2^31 (D2Q9: N + 2*Nx +
4096).  Boxes at that bound, with FP16 delta storage (one buffer in place,
two for pull), take 3 steps, and the velocity of sampled cells (the corners,
the faces where the wraps apply, the cell of the largest index) is compared
with the FP64 oracle's, computed on the periodic (2n + 1)-cell patch around
each cell (a cell's state after n steps depends only on the initial state
within n cells).

The initial velocity is a seeded table field u_d(x, y, z) = A_d[x mod 64] +
B_d[y mod 64] + C_d[z mod 64] at unit density, built on the device (the FP64
fields of 2^31 cells are 17 GB per component) and evaluated on the host for
the patches only.
"""
import gc

import numpy as np
import pytest

import oracle as O
from paper_2211_02435_b300 import build as B
from paper_2211_02435_b300 import lbm as L

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

STEPS = 3
GiB = 1 << 30
CASES = [  # (stencil, dims, space, streaming); Nx even: the packed two-cell kernels
    (L.D2Q9, (46338, 46339, 1), L.SPACE_CUMULANT, L.AA),
    (L.D2Q9, (46338, 46339, 1), L.SPACE_CUMULANT, L.PULL),
    (L.D3Q19, (1024, 1024, 2046), L.SPACE_CENTRAL, L.AA),
]
RATES = [1.8] + [1.0] * 5


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    O.build()
    yield
    gc.collect()
    torch.cuda.empty_cache()


def tables(d, seed=17):
    rng = np.random.default_rng(seed)
    return rng.uniform(-0.015, 0.015, size=(d, 3, 64))


def field_host(tab, X, Y, Z):
    """u[d, ...] at integer coordinates (broadcast arrays)."""
    return np.stack([tab[k, 0][X % 64] + tab[k, 1][Y % 64] + tab[k, 2][Z % 64]
                     for k in range(tab.shape[0])])


def field_device(tab, dims):
    nx, ny, nz = dims
    d = tab.shape[0]
    u = torch.empty((d, nz, ny, nx), dtype=torch.float64, device="cuda")
    t = torch.from_numpy(tab).cuda()
    xs = torch.arange(nx, device="cuda") % 64
    ys = torch.arange(ny, device="cuda") % 64
    zs = torch.arange(nz, device="cuda") % 64
    for k in range(d):  # written in place: no full-size temporary
        torch.add(t[k, 2][zs][:, None, None] + t[k, 1][ys][None, :, None],
                  t[k, 0][xs][None, None, :], out=u[k])
    return u.view(-1)


def patch_oracle(m, st, dims, tab, cell, n):
    """Oracle velocity of `cell` after n steps, stepped on the periodic
    (2n + 1)-cell patch centred on it (2-D patches for D2Q9)."""
    d3 = st != L.D2Q9
    idx = [np.arange(c - n, c + n + 1) % N for c, N in zip(cell, dims)]
    if not d3:
        idx[2] = np.array([0])
    Z, Y, X = np.meshgrid(idx[2], idx[1], idx[0], indexing="ij")
    pd = (2 * n + 1, 2 * n + 1, (2 * n + 1) if d3 else 1)
    u = field_host(tab, X, Y, Z)
    rho = np.ones(Z.shape)
    df = O.step(m, pd, O.init(m, pd, rho, u), n)
    _, uu = O.macroscopic(m, pd, df)
    return uu[:, 0 if not d3 else n, n, n]


def sample_cells(dims, seed=5):
    nx, ny, nz = dims
    cells = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (0, ny - 1, 0), (nx - 1, 0, nz - 1),
             (nx // 2, 0, nz // 2), (1, ny - 2, nz - 1)]
    rng = np.random.default_rng(seed)
    cells += [(int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz)))
              for _ in range(6)]
    return cells


@pytest.mark.parametrize("st,dims,space,streaming", CASES,
                         ids=["d2q9-aa", "d2q9-pull", "d3q19-aa"])
def test_largest_accepted_box_matches_oracle(st, dims, space, streaming):
    nx, ny, nz = dims
    N = nx * ny * nz
    d = 2 if st == L.D2Q9 else 3
    q = 9 if st == L.D2Q9 else 19
    # the box sits just under the index bound
    plane = nx * ny if d == 3 else 0
    assert 2 ** 31 - 2 ** 21 < N + plane + 2 * nx + 4096 < 2 ** 31
    buffers = 1 if streaming != L.PULL else 2
    need = (buffers * q * 2 + d * 8) * N + 4 * GiB
    free, _ = torch.cuda.mem_get_info()
    if free < need:
        pytest.skip(f"needs {need / GiB:.0f} GiB of free device memory, {free / GiB:.0f} free")
    tab = tables(d)
    cells = sample_cells(dims)
    m = O.method(st, space, O.EQ_ABSOLUTE, RATES)
    ref = np.stack([patch_oracle(m, st, dims, tab, c, STEPS) for c in cells], 1)
    with L.Lattice(st, space, L.EQ_ABSOLUTE, L.STORE_F16_DELTA, streaming, RATES, dims) as lat:
        u = field_device(tab, dims)
        lat.init_velocity(None, u)
        lat.step(STEPS)
        lat.macroscopic(None, u)  # the device buffer is reused for the read-out
        idx = torch.tensor([(z * ny + y) * nx + x for x, y, z in cells], device="cuda")
        got = u.view(d, N)[:, idx].cpu().numpy()
        del u
        gc.collect()
        torch.cuda.empty_cache()
    # FP16 delta storage: (n + 1) roundings to 11 bits of the scaled deviations
    bound = 4 * (STEPS + 1) * 2.0 ** -11
    err = float(np.abs(got - ref).max() / np.abs(ref).max())
    assert err < bound, (err, bound)
