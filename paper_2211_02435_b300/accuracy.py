"""Long-run accuracy studies of the reduced-precision forms on the GPU.

* ``fp32_vs_fp64``: D3Q27 cumulant (R-) Taylor-Green vortex u0 = 0.05 with
  seeded uniform 1e-3 velocity noise, FP32 and FP64 storage, pull and AA,
  velocity error of FP32 against FP64 at fixed intervals, and whether pull
  and AA agree bitwise.
* ``half_storage``: D3Q27 central-moment (R-) method on the seeded 8-mode
  Fourier flow (max |u| = 0.08), FP16 / BF16 delta storage and FP32 storage
  against FP64 storage, velocity and density-deviation errors (relative L-inf
  and L2) at fixed intervals.
* ``storage_encoding``: what one FP16 encode of a state costs, with the
  library's per-direction power-of-two scale and without it (the deviations
  stored as they are): D3Q27 central-moment (R-) states after 100 FP64 steps
  of flows from max |u| = 0.08 down to 1e-4; relative L2 error of the
  decoded populations and of the velocity and density deviation computed
  from them, and the share of deviations that fall below FP16's smallest
  normal number (2^-14) unscaled.
* ``tgv_plateau``: the round-off plateau of the decaying Taylor-Green vortex
  (Sec. 5.1, Eq. 5.1/5.2, Table 3): D3Q27, L x L x 1 (the flow is
  z-invariant), u0 = 0.25, nu = 1/6 (every rate 1), FP64; the relative
  kinetic energy E(t)/E0 of SRT, R-WO-MRT, R-O-MRT, R-CM and R-K in each storage /
  equilibrium / arithmetic form, against the analytic exp(-4 nu kappa^2 t).

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


def storage_encoding(n=128, nu=1e-3, steps=100, stream=None):
    rates = [I.shear_viscosity_rate(nu)] + [1.0] * 5
    dims = (n, n, n)
    cases = [("fourier", 0.08)] + [("taylor_green", u0) for u0 in (1e-2, 1e-3, 1e-4)]
    rows = []
    for kind, u0 in cases:
        if kind == "fourier":
            rho, u = I.fourier_modes(dims, n_modes=8, umax=u0, seed=3)
        else:
            rho, u = I.taylor_green(dims, u0)
        with L.Lattice(L.D3Q27, L.SPACE_CENTRAL, L.EQ_ABSOLUTE, L.STORE_F64, L.PULL, rates, dims,
                       stream=stream) as ref:
            ref.init_velocity(rho.reshape(-1), u.reshape(-1))
            ref.step(steps)
            df = ref.get_populations()
            r64, u64 = ref.macroscopic()
            # unscaled: each deviation rounded to the nearest FP16 number as it is
            plain = df.astype(np.float16).astype(np.float64)
            ref.set_populations(plain)
            r_p, u_p = ref.macroscopic()
        with L.Lattice(L.D3Q27, L.SPACE_CENTRAL, L.EQ_ABSOLUTE, L.STORE_F16_DELTA, L.PULL, rates,
                       dims, stream=stream) as lat:
            lat.set_populations(df)
            scaled = lat.get_populations()
            r_s, u_s = lat.macroscopic()
        del rho, u
        norm = np.sqrt((df ** 2).sum())
        nz = df != 0
        row = {"flow": kind, "u0": u0,
               "unscaled_subnormal_share": float((np.abs(df[nz]) < 2.0 ** -14).mean()),
               "scaled": {"pop_rel_l2": float(np.sqrt(((scaled - df) ** 2).sum()) / norm),
                          **_errors(u_s, u64, r_s, r64)},
               "unscaled": {"pop_rel_l2": float(np.sqrt(((plain - df) ** 2).sum()) / norm),
                            **_errors(u_p, u64, r_p, r64)}}
        rows.append(row)
        del df, plain, scaled
    return {"config": f"D3Q27 central moments R-, {n}^3, {steps} FP64 steps, nu={nu}",
            "rows": rows}


PLATEAU_METHODS = (("SRT", L.SPACE_POPULATIONS), ("R-WO-MRT", L.SPACE_RAW_WEIGHTED),
                   ("R-O-MRT", L.SPACE_RAW), ("R-CM", L.SPACE_CENTRAL),
                   ("R-K", L.SPACE_CUMULANT))
# (name, storage, equilibrium, arithmetic): the three forms of Table 3 and
# this library's default (absolute equilibrium in deviation arithmetic)
PLATEAU_FORMS = (
    ("absolute", L.STORE_F64_ABSOLUTE, L.EQ_ABSOLUTE, L.ARITH_AS_WRITTEN),
    ("zc_feq", L.STORE_F64, L.EQ_ABSOLUTE, L.ARITH_AS_WRITTEN),
    ("zc_dfeq", L.STORE_F64, L.EQ_DELTA, L.ARITH_DEVIATION),
    ("zc_feq_deviation", L.STORE_F64, L.EQ_ABSOLUTE, L.ARITH_DEVIATION),
)


def tgv_plateau(n=256, steps=200_000, every=10_000, u0=0.25, methods=None, forms=None,
                stream=None):
    """E(t)/E0 every `every` steps for each admissible (method, form) pair.

    E is the lattice sum of rho |u|^2 / 2 (lbm_invariants, a deterministic
    FP64 reduction); E0 is its value at t = 0, the equilibrium of Eq. 5.1.
    With nu = 1/6 the shear rate is 1 and every higher rate is 1 as well,
    so the weighted (WO-MRT) and unweighted (O-MRT) raw-moment methods are
    the same method (all non-conserved moments are set to equilibrium) and
    differ only in rounding."""
    nu = 1.0 / 6.0
    kappa = 2 * np.pi / n
    rho, u = I.taylor_green((n, n, 1), u0)
    rates = [1.0] * 6
    methods = methods or [m for m, _ in PLATEAU_METHODS]
    forms = forms or [f for f, *_ in PLATEAU_FORMS]
    times = list(range(0, steps + 1, every))
    if times[-1] != steps:
        times.append(steps)
    out = {"config": f"D3Q27 {n}x{n}x1 TGV u0={u0} nu=1/6 (all rates 1), FP64, {steps} steps",
           "steps": times, "analytic": [float(np.exp(-4 * nu * kappa * kappa * t)) for t in times],
           "runs": {}, "seconds": {}}
    for mname, space in PLATEAU_METHODS:
        if mname not in methods:
            continue
        for fname, storage, eq, arith in PLATEAU_FORMS:
            if fname not in forms or (space == L.SPACE_CUMULANT and eq == L.EQ_DELTA):
                continue  # no zero-centered cumulants (Sec. 3)
            t0 = time.perf_counter()
            with L.Lattice(L.D3Q27, space, eq, storage, L.PULL, rates, (n, n, 1), stream=stream,
                           arithmetic=arith) as lat:
                lat.init_velocity(rho.reshape(-1), u.reshape(-1))
                e0 = lat.invariants()["energy"]
                series, done = [1.0], 0
                for t in times[1:]:
                    lat.step(t - done)
                    done = t
                    series.append(lat.invariants()["energy"] / e0)
            out["runs"][f"{mname}/{fname}"] = series
            out["seconds"][f"{mname}/{fname}"] = time.perf_counter() - t0
    return out


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("study", choices=["fp32_vs_fp64", "half_storage", "storage_encoding",
                                      "tgv_plateau"])
    ap.add_argument("--n", type=int)
    ap.add_argument("--steps", type=int)
    ap.add_argument("--every", type=int)
    ap.add_argument("--nu", type=float, default=1e-3)
    ap.add_argument("--out")
    a = ap.parse_args()
    kw = {k: v for k, v in (("n", a.n), ("steps", a.steps), ("every", a.every)) if v}
    if a.study == "tgv_plateau":
        res = tgv_plateau(**kw)
    elif a.study == "storage_encoding":
        res = storage_encoding(nu=a.nu, **{k: v for k, v in kw.items() if k != "every"})
    else:
        fn = fp32_vs_fp64 if a.study == "fp32_vs_fp64" else half_storage
        res = fn(nu=a.nu, **kw)
    txt = json.dumps(res, indent=1)
    if a.out:
        with open(a.out, "w") as f:
            f.write(txt)
    print(txt)


if __name__ == "__main__":
    main()
