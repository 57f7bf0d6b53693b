"""Long-run accuracy studies of the reduced-precision forms on the GPU.

* ``fp32_vs_fp64``: D3Q27 cumulant (R-) Taylor-Green vortex u0 = 0.05 with
  seeded uniform 1e-3 velocity noise, FP32 and FP64 storage, pull and AA,
  velocity error of FP32 against FP64 at fixed intervals, and whether pull
  and AA agree bitwise.
* ``half_storage``: D3Q27 central-moment (R-) method on the seeded 8-mode
  Fourier flow (max |u| = 0.08), FP16 / BF16 delta storage and FP32 storage
  against FP64 storage, velocity and density-deviation errors (relative L-inf
  and L2) at fixed intervals.

The FP64 GPU runs are tied to the CPU oracle by the parity tests (1e-12 per
step); these studies measure how the reduced forms drift from them over
thousands of steps.  All stepping runs in the library's kernels.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs as I
from . import lbm as L


def _errors(u, ut, r=None, rt=None):
    out = {"u_rel_linf": float(np.abs(u - ut).max() / np.abs(ut).max()),
           "u_rel_l2": float(np.sqrt(((u - ut) ** 2).sum() / (ut ** 2).sum()))}
    if r is not None:
        dr, drt = r - 1.0, rt - 1.0
        out["drho_rel_linf"] = float(np.abs(dr - drt).max() / np.abs(drt).max())
        out["drho_rel_l2"] = float(np.sqrt(((dr - drt) ** 2).sum() / (drt ** 2).sum()))
    return out


def fp32_vs_fp64(n=256, nu=1e-3, steps=1000, every=100, seed=1, stream=None):
    rho, u = I.taylor_green((n, n, n), 0.05)
    u = I.add_uniform_noise(u, 1e-3, seed=seed)
    rates = [I.shear_viscosity_rate(nu)] + [1.0] * 5
    lats = {}
    for name, st, sm in (("f64", L.STORE_F64, L.PULL), ("f32", L.STORE_F32, L.PULL),
                         ("f32_aa", L.STORE_F32, L.AA)):
        lats[name] = L.Lattice(L.D3Q27, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, st, sm, rates, (n, n, n),
                               stream=stream)
        lats[name].init_velocity(rho.reshape(-1), u.reshape(-1))
    rows, secs = [], {k: 0.0 for k in lats}
    done = 0
    try:
        while done < steps:
            k = min(every, steps - done)
            for name, lat in lats.items():
                t0 = time.perf_counter()
                lat.step(k)
                lat.macroscopic(np.empty(n ** 3), None)  # synchronises
                secs[name] += time.perf_counter() - t0
            done += k
            _, u64 = lats["f64"].macroscopic()
            _, u32 = lats["f32"].macroscopic()
            rows.append({"step": done, **_errors(u32, u64)})
        # pull and AA run the same per-cell arithmetic: identical states
        equal = bool(np.array_equal(lats["f32"].get_populations(),
                                    lats["f32_aa"].get_populations()))
    finally:
        for lat in lats.values():
            lat.close()
    return {"config": f"D3Q27 cumulant R-, {n}^3 TGV u0=0.05 + 1e-3 noise, nu={nu}",
            "steps": steps, "rows": rows, "pull_aa_bitwise_equal_at_end": equal,
            "mlups_incl_readout": {k: n ** 3 * steps / v / 1e6 for k, v in secs.items()}}


def half_storage(n=512, nu=1e-3, steps=5000, every=1000, seed=3, stream=None):
    rho, u = I.fourier_modes((n, n, n), n_modes=8, umax=0.08, seed=seed)
    rates = [I.shear_viscosity_rate(nu)] + [1.0] * 5
    forms = (("f64", L.STORE_F64), ("f32", L.STORE_F32), ("f16_delta", L.STORE_F16_DELTA),
             ("bf16_delta", L.STORE_BF16_DELTA))
    lats = {}
    rows = []
    try:
        for name, st in forms:
            lats[name] = L.Lattice(L.D3Q27, L.SPACE_CENTRAL, L.EQ_ABSOLUTE, st, L.PULL, rates,
                                   (n, n, n), stream=stream)
            lats[name].init_velocity(rho.reshape(-1), u.reshape(-1))
        del rho, u
        done = 0
        while done < steps:
            k = min(every, steps - done)
            for lat in lats.values():
                lat.step(k)
            done += k
            r64, u64 = lats["f64"].macroscopic()
            row = {"step": done}
            for name in ("f32", "f16_delta", "bf16_delta"):
                r, uu = lats[name].macroscopic()
                row[name] = _errors(uu, u64, r, r64)
                del r, uu
            rows.append(row)
    finally:
        for lat in lats.values():
            lat.close()
    return {"config": f"D3Q27 central moments R-, {n}^3 8-mode Fourier flow max|u|=0.08 "
                      f"(seed {seed}), nu={nu}", "steps": steps, "rows": rows}


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("study", choices=["fp32_vs_fp64", "half_storage"])
    ap.add_argument("--n", type=int)
    ap.add_argument("--steps", type=int)
    ap.add_argument("--every", type=int)
    ap.add_argument("--nu", type=float, default=1e-3)
    ap.add_argument("--out")
    a = ap.parse_args()
    kw = {k: v for k, v in (("n", a.n), ("steps", a.steps), ("every", a.every)) if v}
    fn = fp32_vs_fp64 if a.study == "fp32_vs_fp64" else half_storage
    res = fn(nu=a.nu, **kw)
    txt = json.dumps(res, indent=1)
    if a.out:
        with open(a.out, "w") as f:
            f.write(txt)
    print(txt)


if __name__ == "__main__":
    main()
