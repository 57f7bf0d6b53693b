"""Oracle values of single cells of a large periodic lattice.

After n steps a cell's populations depend only on the initial state within n
cells of it (one lattice link per step), so the oracle can step the periodic
(2n + 1)^3 cube centred on the cell instead of the whole lattice: values
that wrap at the cube's faces are wrong, but the error starts at distance n
from the centre and moves one cell per step, so it reaches the centre only
after more than n steps.
"""
import numpy as np

import oracle as O


def cube_oracle(m, dims, rho, u, cell, n):
    """Oracle populations df[q] and velocity u[3] of `cell` = (x, y, z) after
    n steps of method m from the fields rho[Nz, Ny, Nx], u[3, Nz, Ny, Nx] on
    the periodic lattice dims = (Nx, Ny, Nz); every edge must be >= 2n + 1."""
    ix, iy, iz = (np.arange(c - n, c + n + 1) % N for c, N in zip(cell, dims))
    rho_c = rho[np.ix_(iz, iy, ix)]
    u_c = u[(slice(None),) + np.ix_(iz, iy, ix)]
    dc = (2 * n + 1,) * 3
    df = O.step(m, dc, O.init(m, dc, rho_c, u_c), n)
    _, uu = O.macroscopic(m, dc, df)
    return df[:, n, n, n], uu[:, n, n, n]
