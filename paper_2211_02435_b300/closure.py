"""Training driver of the learned closure (include/lbm_closure.h).

Data: a fine D3Q27 run of the plain regularised cumulant method on the
seeded random-Fourier-mode flow, restricted by 4^3 block averages to the
coarse lattice (acoustic scaling: one coarse step = four fine steps, equal
lattice velocities, nu_coarse = nu_fine / 4).  The run spans `span` coarse
steps; its first 80 % supplies the training windows (K + 1 consecutive
coarse snapshots each), the last 20 % is held out.

Training: Adam on the K-step rollout loss of the windows, all in the
library's GPU kernels (forward, adjoint through the K steps, network
backward, Adam).  Evaluation, held out: the K-step loss of a window that
starts the held-out part, and a-posteriori rollouts of the coarse method
from the first held-out snapshot (`rollout` steps and a shorter one),
learned rates against the plain method (higher-order rates 1), both judged
by the restricted fine solution.

Host-side code here only orders the calls and computes summary statistics.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs as I
from . import lbm as L


def schedule(span, unroll, windows, rollout, short):
    """Coarse times to snapshot, sorted and distinct: `windows` training
    windows of unroll + 1 consecutive times spread over the first 80 % of the
    span, the held-out window at 80 %, and the held-out rollout targets.
    Consecutive integer times sit at consecutive snapshot indices, so a
    window starting at index s holds its targets at s + 1 .. s + unroll.
    Returns (times, training window indices, held-out window index,
    {"t0", "short", "long": index})."""
    t_held = int(round(0.8 * span))
    last = max(t_held - unroll - 1, 0)
    starts = np.unique(np.linspace(0, last, windows).round().astype(int))
    need = set()
    for s in list(starts) + [t_held]:
        need.update(range(int(s), int(s) + unroll + 1))
    need.update((t_held + short, t_held + rollout))
    times = sorted(need)
    at = {t: k for k, t in enumerate(times)}
    anchors = {"t0": at[t_held], "short": at[t_held + short], "long": at[t_held + rollout]}
    return times, [at[int(s)] for s in starts], at[t_held], anchors


def make_snapshots(trainer, fine_edge, times, nu_fine, seed, umax=0.08, stream=None):
    """Run the fine plain cumulant method (FP32, pull) and append one
    restricted snapshot at each coarse time of `times` (non-decreasing).
    Returns the fine MLUPS."""
    n = fine_edge
    rates = [I.shear_viscosity_rate(nu_fine)] + [1.0] * 5
    rho, u = I.fourier_modes((n, n, n), n_modes=8, umax=umax, seed=seed)
    with L.Lattice(L.D3Q27, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, L.STORE_F32, L.PULL, rates,
                   (n, n, n), stream=stream) as fine:
        fine.init_velocity(rho.reshape(-1), u.reshape(-1))
        del rho, u
        t0 = time.perf_counter()
        t = 0
        for T in times:
            fine.step(4 * (T - t))
            t = T
            trainer.add_restricted(fine)
        dt = time.perf_counter() - t0
    return n ** 3 * 4 * times[-1] / dt / 1e6


def feature_normalisation(trainer, snaps):
    """Per-input shift and scale (mean and 1/std over the cells of the given
    snapshots) so that the network sees O(1) inputs."""
    f = np.concatenate([trainer.features(s) for s in snaps], axis=1)
    mu = f.mean(1)
    sd = f.std(1)
    sc = np.where(sd > 0, 1.0 / np.where(sd > 0, sd, 1.0), 1.0)
    return mu, sc


def init_params(seed, scale=0.2):
    """Small random hidden layers and a zero output layer: the untrained
    network gives rates 1 everywhere, i.e. exactly the plain method."""
    rng = np.random.default_rng(seed)
    p = scale * rng.standard_normal(L.CLOSURE_NPARAM)
    p[1312:] = 0.0  # W3, b3
    return p


def mean_loss(trainer, windows):
    return float(np.mean([trainer.loss_grad(s)[0] for s in windows]))


def rollout_error(trainer, s0, steps, s1, omega_c, weights, stream=None):
    """Relative L2 and L-infinity velocity errors of `steps` coarse steps
    from snapshot s0 against snapshot s1 (the restricted fine state `steps`
    coarse steps later)."""
    dims = trainer.dims
    with L.Lattice(L.D3Q27, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, L.STORE_F32, L.PULL,
                   [omega_c] + [1.0] * 5, dims, stream=stream) as lat:
        if weights is not None:
            lat.set_closure(weights)
        lat.set_populations(trainer.snapshot(s0))
        lat.step(steps)
        _, u = lat.macroscopic()
    with L.Lattice(L.D3Q27, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, L.STORE_F64, L.PULL,
                   [omega_c] + [1.0] * 5, dims) as ref:
        ref.set_populations(trainer.snapshot(s1))
        _, ut = ref.macroscopic()
    return float(np.sqrt(((u - ut) ** 2).sum() / (ut ** 2).sum())), \
        float(np.abs(u - ut).max() / np.abs(ut).max())


def train_and_evaluate(fine_edge=512, span=1280, unroll=8, windows=24, epochs=6, lr=3e-3,
                       rollout=256, short=64, nu_fine=2e-4, seed=5, stream=None, log=None):
    """Fine run, restriction, training on the first 80 % of the span, and the
    held-out evaluation.  Times (span, rollout, short) are coarse steps."""
    coarse = fine_edge // 4
    omega_c = I.shear_viscosity_rate(nu_fine / 4)
    times, win_idx, held_idx, anchors = schedule(span, unroll, windows, rollout, short)
    out = {"fine": f"{fine_edge}^3", "coarse": f"{coarse}^3", "nu_fine": nu_fine,
           "span_coarse_steps": span, "unroll": unroll, "train_windows": len(win_idx),
           "heldout_from_step": times[held_idx], "snapshots": len(times)}
    with L.Trainer((coarse,) * 3, omega_c, 1.0, len(times), stream=stream) as tr:
        out["fine_mlups"] = make_snapshots(tr, fine_edge, times, nu_fine, seed, stream=stream)
        tr.set_unroll(unroll)
        shift, scale = feature_normalisation(tr, win_idx[::max(1, len(win_idx) // 4)])
        tr.set_params(np.zeros(L.CLOSURE_NPARAM), shift, scale)
        out["heldout_loss_plain"] = mean_loss(tr, [held_idx])
        out["train_loss_initial"] = mean_loss(tr, win_idx)
        tr.set_params(init_params(seed), shift, scale)
        rng = np.random.default_rng(seed)
        t0 = time.perf_counter()
        steps = 0
        for ep in range(epochs):
            losses = [tr.adam_step(int(s), lr) for s in rng.permutation(win_idx)]
            steps += len(losses)
            if log:
                log(f"epoch {ep}: mean train loss {np.mean(losses):.4e}")
        out["train_seconds"] = time.perf_counter() - t0
        out["adam_steps"] = steps
        out["train_loss_final"] = mean_loss(tr, win_idx)
        out["heldout_loss_learned"] = mean_loss(tr, [held_idx])
        w = tr.export()
        s0 = anchors["t0"]
        for key, length in (("short", short), ("long", rollout)):
            e_l = rollout_error(tr, s0, length, anchors[key], omega_c, w, stream)
            e_p = rollout_error(tr, s0, length, anchors[key], omega_c, None, stream)
            out[f"rollout{length}_err_learned"], out[f"rollout{length}_linf_learned"] = e_l
            out[f"rollout{length}_err_plain"], out[f"rollout{length}_linf_plain"] = e_p
        out["weights"] = w
    return out


RATE_SWEEP = [("plain", [1.0, 1.0, 1.0, 1.0])] + [
    (f"w3={w}", [w, 1.0, 1.0, 1.0]) for w in (0.01, 0.03, 0.1, 0.3, 0.5, 1.5)] + [
    (f"w4={w}", [1.0, w, 1.0, 1.0]) for w in (0.3, 1.9)] + [
    ("w5=0.3", [1.0, 1.0, 0.3, 1.0]), ("w6=0.3", [1.0, 1.0, 1.0, 0.3]),
    ("w3=0.1,w4=1.9", [0.1, 1.9, 1.0, 1.0]), ("w3=0.03,w4=1.5", [0.03, 1.5, 1.0, 1.0])]


def constant_rate_sweep(fine_edge=512, nu_fine=2e-4, seed=5, unroll=8, stream=None):
    """What constant rates of orders 3..6 gain over the plain method on the
    learned-closure data: rollout errors of the coarse method from the
    restricted state at coarse steps 0 and 1024 (times scaled by fine_edge /
    512) after 64 and 256 steps, and the mean one-step and `unroll`-step
    losses over windows at steps 64, 512 and 896."""
    sc = fine_edge / 512
    T = [int(round(v * sc)) for v in (0, 64, 256, 512, 896, 1024, 1088, 1280)]
    wins = [T[1], T[3], T[4]]
    times = sorted({T[0], T[2], T[5], T[6], T[7]} | {w + k for w in wins for k in range(unroll + 1)})
    at = {t: k for k, t in enumerate(times)}
    coarse = fine_edge // 4
    omega_c = I.shear_viscosity_rate(nu_fine / 4)
    rows = []
    with L.Trainer((coarse,) * 3, omega_c, 1.0, len(times), stream=stream) as tr:
        make_snapshots(tr, fine_edge, times, nu_fine, seed, stream=stream)
        for name, r4 in RATE_SWEEP:
            # constant rates: a network whose output biases give them everywhere
            p = np.zeros(L.CLOSURE_NPARAM)
            p[1440:1444] = np.log(np.array(r4) / (2.0 - np.array(r4)))
            tr.set_params(p, np.zeros(7), np.ones(7))
            w = tr.export()
            row = {"name": name, "rates_3_6": r4}
            for t0, lengths in ((T[0], (T[1], T[2])), (T[5], (T[1], T[2]))):
                for n in lengths:
                    row[f"rollout_{t0}_{n}"] = rollout_error(tr, at[t0], n, at[t0 + n], omega_c,
                                                             w, stream)[0]
            for K in (1, unroll):
                tr.set_unroll(K)
                row[f"loss_k{K}"] = mean_loss(tr, [at[wt] for wt in wins])
            tr.set_unroll(1)
            rows.append(row)
    return {"fine": f"{fine_edge}^3", "coarse": f"{coarse}^3", "nu_fine": nu_fine,
            "rows": rows}


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["sweep", "train"])
    ap.add_argument("--fine", type=int, default=512)
    a = ap.parse_args()
    if a.what == "sweep":
        print(json.dumps(constant_rate_sweep(a.fine)))
    else:
        sc = a.fine / 512
        res = train_and_evaluate(fine_edge=a.fine, span=int(round(1280 * sc)),
                                 rollout=int(round(256 * sc)), short=int(round(64 * sc)),
                                 log=print)
        res.pop("weights")
        print(json.dumps(res))
