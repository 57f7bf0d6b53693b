"""The single-cell cube evaluation used by the full-size GPU tests equals
the oracle run on the whole periodic lattice, bit for bit, at the corners,
faces and interior, for every collision space."""
import numpy as np
import pytest

import oracle as O
from paper_2211_02435_b300 import inputs as I
from sampling import cube_oracle


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


@pytest.mark.parametrize("space,eq", [(O.SPACE_RAW, O.EQ_DELTA), (O.SPACE_CENTRAL, O.EQ_ABSOLUTE),
                                      (O.SPACE_CUMULANT, O.EQ_ABSOLUTE)])
@pytest.mark.parametrize("st", [O.D3Q19, O.D3Q27])
def test_cube_equals_whole_lattice(st, space, eq):
    dims, n = (11, 9, 8), 3
    rho, u = I.taylor_green(dims, 0.05)
    u = I.add_uniform_noise(u, 1e-2, seed=5)
    m = O.method(st, space, eq, [1.6, 1.0, 1.3, 1.0, 1.0, 1.0])
    full = O.step(m, dims, O.init(m, dims, rho, u), n)
    _, uf = O.macroscopic(m, dims, full)
    for cell in [(0, 0, 0), (10, 8, 7), (0, 8, 3), (5, 4, 0), (6, 2, 5)]:
        df, uu = cube_oracle(m, dims, rho, u, cell, n)
        x, y, z = cell
        assert np.array_equal(df, full[:, z, y, x]), cell
        assert np.array_equal(uu, uf[:, z, y, x]), cell
