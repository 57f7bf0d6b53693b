"""Training driver of the learned closure (include/lbm_closure.h).

Data: a fine D3Q27 run of the plain regularised cumulant method on the
seeded random-Fourier-mode flow, restricted by 4^3 block averages to the
coarse lattice every 4 fine steps (acoustic scaling: one coarse step = four
fine steps, equal lattice velocities, nu_coarse = nu_fine / 4).  Training:
Adam on the one-step velocity loss of consecutive coarse snapshots, all in
the library's GPU kernels.  Evaluation: one-step loss on held-out pairs and
an a-posteriori rollout of the coarse method from a held-out snapshot,
learned rates against the plain method (higher-order rates 1), both judged
by the restricted fine solution.

Host-side code here only orders the calls and computes summary statistics.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs as I
from . import lbm as L


def make_snapshots(trainer, fine_edge, nsnap, nu_fine, seed, umax=0.08, stream=None):
    """Run the fine plain cumulant method (FP32, pull) and append nsnap
    restricted snapshots, one every 4 fine steps.  Returns the fine MLUPS."""
    n = fine_edge
    rates = [I.shear_viscosity_rate(nu_fine)] + [1.0] * 5
    rho, u = I.fourier_modes((n, n, n), n_modes=8, umax=umax, seed=seed)
    with L.Lattice(L.D3Q27, L.SPACE_CUMULANT, L.EQ_ABSOLUTE, L.STORE_F32, L.PULL, rates,
                   (n, n, n), stream=stream) as fine:
        fine.init_velocity(rho.reshape(-1), u.reshape(-1))
        trainer.add_restricted(fine)
        t0 = time.perf_counter()
        for _ in range(nsnap - 1):
            fine.step(4)
            trainer.add_restricted(fine)
        dt = time.perf_counter() - t0
    return n ** 3 * 4 * (nsnap - 1) / dt / 1e6


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


def mean_loss(trainer, pairs):
    return float(np.mean([trainer.loss_grad(s)[0] for s in pairs]))


def rollout_error(trainer, s0, steps, omega_c, weights, stream=None):
    """Relative L2 velocity error of `steps` coarse steps from snapshot s0
    against the restricted fine snapshot s0 + steps."""
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
        ref.set_populations(trainer.snapshot(s0 + steps))
        _, ut = ref.macroscopic()
    return float(np.sqrt(((u - ut) ** 2).sum() / (ut ** 2).sum())), \
        float(np.abs(u - ut).max() / np.abs(ut).max())


def train_and_evaluate(fine_edge=512, nsnap=160, ntrain=128, epochs=8, lr=3e-3, rollout=32,
                       nu_fine=2e-4, seed=5, stream=None, log=None):
    coarse = fine_edge // 4
    omega_c = I.shear_viscosity_rate(nu_fine / 4)
    out = {"fine": f"{fine_edge}^3", "coarse": f"{coarse}^3", "nu_fine": nu_fine,
           "snapshots": nsnap, "train_pairs": ntrain - 1}
    with L.Trainer((coarse,) * 3, omega_c, 1.0, nsnap, stream=stream) as tr:
        out["fine_mlups"] = make_snapshots(tr, fine_edge, nsnap, nu_fine, seed, stream=stream)
        shift, scale = feature_normalisation(tr, list(range(0, ntrain, max(1, ntrain // 4))))
        train_pairs = list(range(ntrain - 1))
        held = list(range(ntrain, nsnap - 1))
        tr.set_params(np.zeros(L.CLOSURE_NPARAM), shift, scale)
        out["heldout_loss_plain"] = mean_loss(tr, held)
        out["train_loss_initial"] = mean_loss(tr, train_pairs)
        tr.set_params(init_params(seed), shift, scale)
        rng = np.random.default_rng(seed)
        t0 = time.perf_counter()
        steps = 0
        for ep in range(epochs):
            losses = [tr.adam_step(int(s), lr) for s in rng.permutation(train_pairs)]
            steps += len(losses)
            if log:
                log(f"epoch {ep}: mean train loss {np.mean(losses):.4e}")
        out["train_seconds"] = time.perf_counter() - t0
        out["adam_steps"] = steps
        out["train_loss_final"] = mean_loss(tr, train_pairs)
        out["heldout_loss_learned"] = mean_loss(tr, held)
        w = tr.export()
        s0 = ntrain
        steps_r = min(rollout, nsnap - 1 - s0)
        out["rollout_steps"] = steps_r
        e_l = rollout_error(tr, s0, steps_r, omega_c, w, stream)
        e_p = rollout_error(tr, s0, steps_r, omega_c, None, stream)
        out["rollout_err_learned"], out["rollout_linf_learned"] = e_l
        out["rollout_err_plain"], out["rollout_linf_plain"] = e_p
        out["weights"] = w
    return out
