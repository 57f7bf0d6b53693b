"""Circular dam break with the shallow-water methods (Sec. 5.2), all steps in
the library's kernels (include/lbm.h, lbm_set_shallow_water).

Set-up of the paper's Sec. 5.2: a 40 m x 40 m periodic basin on 100 x 100
cells (dx = 0.4 m), dt = 0.05 s, a water column of radius 2.5 m and height
2.5 m in the centre, 0.5 m of water elsewhere, kinematic viscosity 1 m^2/s
(omega_s = 1 / (3 nu dt / dx^2 + 1/2) = 0.696), all other rates 1.  Lattice
units: g = 9.81 dt^2 / dx, depths h / dx.  Returns the depth profile along
the row through the centre (y = 20 m) after 1, 2 and 3 s.
"""
from __future__ import annotations

import numpy as np

from . import lbm as L

DX, DT, G_SI, NU_SI = 0.4, 0.05, 9.81, 1.0


def dam_break_fields(n=100, length=40.0, r=2.5, h_in=2.5, h_out=0.5):
    """Depth (lattice units) and zero velocity of the circular dam break."""
    dx = length / n
    c = (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(c, c, indexing="xy")
    h = np.where((X - length / 2) ** 2 + (Y - length / 2) ** 2 <= r * r, h_in, h_out) / dx
    return h.reshape(1, n, n), np.zeros((2, 1, n, n))


def lattice_parameters(n=100, length=40.0):
    dx = length / n
    g = G_SI * DT * DT / dx
    nu = NU_SI * DT / (dx * dx)
    omega = 1.0 / (3.0 * nu + 0.5)
    return g, omega


def dam_break(space, n=100, times_s=(1.0, 2.0, 3.0), stream=None):
    g, omega = lattice_parameters(n)
    h, u = dam_break_fields(n)
    out = {"g_lattice": g, "omega_s": omega, "profiles_m": {}, "mass": []}
    with L.Lattice(L.D2Q9, space, L.EQ_ABSOLUTE, L.STORE_F64_ABSOLUTE, L.PULL,
                   [omega, 1.0, 1.0, 1.0, 1.0, 1.0], (n, n, 1), stream=stream) as lat:
        lat.set_shallow_water(g)
        lat.init_velocity(h.reshape(-1), u.reshape(-1))
        done = 0
        for t in times_s:
            steps = int(round(t / DT))
            lat.step(steps - done)
            done = steps
            hh, _ = lat.macroscopic()
            hh = hh.reshape(n, n)
            out["mass"].append(float(hh.sum()))
            row = 0.5 * (hh[n // 2 - 1] + hh[n // 2])  # y = 20 m lies between two rows
            out["profiles_m"][t] = (row * (40.0 / n)).tolist()
            out.setdefault("fields", {})[t] = hh
    out["mass0"] = float(h.sum())
    return out


def main():
    import json
    res = {}
    for name, sp in (("CM", L.SPACE_CENTRAL), ("K", L.SPACE_CUMULANT)):
        r = dam_break(sp)
        r.pop("fields")
        res[name] = r
    print(json.dumps(res))


if __name__ == "__main__":
    main()
