"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds input recipes only (parameter grids, seeds, random site
tensors, job lists).  It contains none of the method's arithmetic.

Recipes:
  * Ising lattices are fully described by (beta, h, L, chi).
  * The generic-tensor test mode uses a random D x D x D x D site tensor with
    i.i.d. entries 1 + 0.5 * N(0,1) (mostly positive, as Boltzmann weights are,
    but with generic, almost surely non-degenerate singular spectra).
  * Base seeds: workload c uses 0x4D435452 + c; trajectory i uses counter i.
"""
import numpy as np

BASE_SEED = 0x4D435452


def seed_for(config_index):
    return BASE_SEED + int(config_index)


def generic_tensor(D, seed):
    rng = np.random.default_rng(int(seed))
    return 1.0 + 0.5 * rng.standard_normal((D, D, D, D))


def beta_grid():
    """The 16 inverse temperatures 0.30, 0.32, ..., 0.60 of the beta sweep."""
    return [0.30 + 0.02 * i for i in range(16)]


def uneven_jobs(n_jobs, seed, chis=(4, 8, 16), Ls=(8, 16, 32), traj_range=(64, 512)):
    """Random job list for the uneven-batch workload: (beta, h, L, chi, n_traj)."""
    rng = np.random.default_rng(int(seed))
    jobs = []
    for _ in range(n_jobs):
        jobs.append(dict(beta=float(rng.uniform(0.3, 0.6)), h=float(rng.uniform(0.0, 0.1)),
                         L=int(rng.choice(Ls)), chi=int(rng.choice(chis)),
                         n_traj=int(rng.integers(traj_range[0], traj_range[1] + 1))))
    return jobs
