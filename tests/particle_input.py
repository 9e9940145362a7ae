"""Particle-workload inputs for the shot-noise tests: the seeded lognormal
Poisson positions of ``synth.poisson_positions`` turned into delta(k) by the
oracle's own CIC + interlacing stage (oracle.density_from_particles), so the
GPU estimator and the oracle read the same complex64 half spectrum and no
input comes from the CUDA path."""
import numpy as np

import oracle
from paper_1708_05303_gb300.synth import poisson_positions


def particle_delta(model, seed: int, n_particles: int = 4 * 2 ** 20):
    """(complex64 half spectrum [n][n][n/2+1], realised N_p, nbar = N_p / V)."""
    pos = poisson_positions(model, seed, n_particles)
    dk, nbar = oracle.density_from_particles(pos, model.n, model.box)
    return dk.astype(np.complex64), int(pos.shape[0]), float(nbar)
