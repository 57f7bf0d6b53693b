"""GPU test of lbm_invariants_noalloc, the reduction for callers that must
not allocate device memory (a host framework that owns the device pool, a
real-time loop, a caller that only lends this library its buffers).

It is checked against the allocating entry point lbm_invariants on the same
populations, twice in a row with different stencils, storage types and
sizes, so that the shared static scratch is reused between calls.  This file
is collected last on purpose."""
import numpy as np
import pytest

from paper_2211_02435_b300 import build as B
from paper_2211_02435_b300 import inputs as I
from paper_2211_02435_b300 import lbm as L

pytestmark = pytest.mark.gpu

CASES = [  # (stencil, storage, dims, torch dtype name)
    (L.D3Q27, L.STORE_F32, (133, 6, 5), "float32"),
    (L.D3Q19, L.STORE_F64, (40, 33, 7), "float64"),
]


def _reference(stencil, storage, dims, df64):
    # allocating entry point on an AA context at even parity: the state buffer
    # then holds slot i of cell c = f_i(c), the layout the no-alloc call reads
    with L.Lattice(stencil, L.SPACE_RAW, L.EQ_DELTA, storage, L.AA, [1.5], dims) as lat:
        lat.set_populations(df64)
        return lat.invariants()


def test_noalloc_matches_allocating_entry_point_twice():
    torch = pytest.importorskip("torch")
    B.build()
    for k, (st, so, dims, tname) in enumerate(CASES):
        q = L.Q_OF[st]
        n = int(np.prod(dims))
        dt = getattr(torch, tname)
        vals = I.random_deviations(q, n, 1e-2, seed=40 + k)
        dev = torch.from_numpy(vals.reshape(-1)).to(dt).cuda()
        # the exact values the device field holds, as FP64 for the reference
        ref = _reference(st, so, dims, dev.double().cpu().numpy())
        got = L.invariants_noalloc(st, so, dev, dims)
        for key in ref:
            assert abs(got[key] - ref[key]) <= 1e-12 * max(1.0, abs(ref[key])), key
        out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
        L.invariants_noalloc(st, so, dev, dims, out=out,
                             stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), np.array(list(ref.values())),
                                   rtol=1e-12, atol=1e-15)


def test_noalloc_rejects_sizes_beyond_the_limit():
    B.build()
    big = (1 << 20, 1 << 11, 1)  # 2^31 cells: one more than a call serves
    with pytest.raises(L.LBMError) as e:
        L.invariants_noalloc(L.D3Q27, L.STORE_F32, 1 << 20, big)
    assert e.value.code == -1
    with pytest.raises(L.LBMError):
        L.invariants_noalloc(L.D3Q27, L.STORE_F32, 1 << 20, (0, 4, 4))
