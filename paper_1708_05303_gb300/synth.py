"""Seeded synthetic inputs: redshift-space density fields delta(k).

This module only draws inputs.  It holds none of the estimator's arithmetic
(no shells, Legendre weights, inverse transforms of filtered fields or
contractions), so both the CUDA path and the FP64 oracle can be fed from it.

Field model (the paper measures on no dataset; these stand in for survey
grids):
  1. w_x ~ N(0, 1) on the n^3 grid, numpy PCG64(seed), C order.
  2. g(k) = sqrt(P(k) V) DFT(w)(k) / sqrt(n^3), P(k) = A k^{n_s} (k in h/Mpc,
     P(0) = 0); optionally rescaled so that the grid std of g_x is sigma_g.
  3. Local quadratic term: delta_x = g_x + (g_x^2 - <g^2>)/2, <.> the grid mean.
  4. Kaiser redshift-space factor along z (the last axis):
     delta_s(k) = (1 + f mu^2) delta(k), mu = k_z/|k|, factor 1 at k = 0
     (the linear limit of Sec. 1, Eq. Delta2Deltas).
  Optionally (the 256^3 particle workload): positions of a lognormal Poisson
  sample of delta_s with a fixed expected particle count (the deposit onto a
  grid is the estimator's input stage, not done here).

delta(k) is continuum normalised, delta(k) = (V/n^3) sum_x delta_x e^{-ik.x},
and returned as the complex64 half spectrum [n][n][n/2+1].
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class FieldModel:
    n: int = 64
    box: float = 1000.0         # Mpc/h
    amp: float = 2.0e4          # A in P(k) = A k^{n_s}
    n_s: float = -1.5
    f: float = 0.7              # Kaiser growth rate
    sigma_g: float | None = None  # rescale g to this grid std (None: keep A)
    quad: float = 0.5           # coefficient of (g^2 - <g^2>)
    g_sign: float = 1.0         # +1 or -1: draws the mirrored Gaussian field -g


def kf(box: float) -> float:
    return 2.0 * math.pi / box


def _freqs(n: int):
    j = np.arange(n)
    return np.where(j < n // 2, j, j - n).astype(np.float64)


def _kgrid_half(n: int, box: float):
    fx = _freqs(n)
    fz = np.arange(n // 2 + 1, dtype=np.float64)
    fz[n // 2] = -(n // 2)
    n2 = fx[:, None, None] ** 2 + fx[None, :, None] ** 2 + fz[None, None, :] ** 2
    k = kf(box) * np.sqrt(n2)
    with np.errstate(invalid="ignore", divide="ignore"):
        mu = np.where(n2 > 0, fz[None, None, :] / np.sqrt(n2), 0.0)
    return k, mu


def gaussian_real(model: FieldModel, seed: int):
    """g_x (float64 [n][n][n]) and the effective amplitude A after rescaling."""
    n, box = model.n, model.box
    V = box ** 3
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((n, n, n))
    k, _ = _kgrid_half(n, box)
    with np.errstate(divide="ignore"):
        P = np.where(k > 0, model.amp * np.power(np.where(k > 0, k, 1.0), model.n_s), 0.0)
    gk = np.sqrt(P * V) * np.fft.rfftn(w) / math.sqrt(n ** 3)
    g = np.fft.irfftn(gk * (n ** 3 / V), s=(n, n, n), axes=(0, 1, 2))
    amp = model.amp
    if model.sigma_g is not None:
        s = float(g.std())
        g *= model.sigma_g / s
        amp = model.amp * (model.sigma_g / s) ** 2
    return model.g_sign * g, amp


def delta_k_from_real(delta_x: np.ndarray, box: float) -> np.ndarray:
    """Continuum-normalised half spectrum (V/n^3) rfftn(delta_x), complex128."""
    n = delta_x.shape[0]
    return np.fft.rfftn(delta_x) * (box ** 3 / n ** 3)


def make_field(model: FieldModel, seed: int, dtype=np.complex64):
    """delta_s(k) half spectrum [n][n][n/2+1] and the effective P(k) amplitude."""
    g, amp = gaussian_real(model, seed)
    d = g + model.quad * (g * g - (g * g).mean())
    dk = delta_k_from_real(d, model.box)
    _, mu = _kgrid_half(model.n, model.box)
    dk *= 1.0 + model.f * mu ** 2
    return dk.astype(dtype), amp


def poisson_positions(model: FieldModel, seed: int, n_particles: int = 4 * 2 ** 20) -> np.ndarray:
    """Particle positions (float32 [N_p][3], box units in [0, box)) of the
    particle workload: delta_s(x) from ``make_field`` -> lognormal rate
    lambda_x proportional to exp(delta_s) with sum lambda = n_particles ->
    Poisson counts per cell -> positions uniform within the cell."""
    n, box = model.n, model.box
    dk, _ = make_field(model, seed, dtype=np.complex128)
    ds = np.fft.irfftn(dk * (n ** 3 / box ** 3), s=(n, n, n), axes=(0, 1, 2))
    lam = np.exp(ds - ds.max())
    lam *= n_particles / lam.sum()
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    cnt = rng.poisson(lam).ravel()
    cell = np.repeat(np.arange(n ** 3), cnt)
    cx, cy, cz = np.unravel_index(cell, (n, n, n))
    pos = np.stack([cx, cy, cz], axis=1).astype(np.float64)
    pos += rng.random((pos.shape[0], 3))
    pos *= box / n
    return np.minimum(pos, np.nextafter(box, 0)).astype(np.float32) % np.float32(box)


def linear_edges(n_shells: int, width: float = 2.0, start: float = 1.0):
    """Shell edges in k_f units: start + width*i, i = 0..n_shells."""
    return [start + width * i for i in range(n_shells + 1)]


def mock_model(m: int, sizes=(96, 128, 160), box: float = 1000.0) -> tuple[FieldModel, int]:
    """The m-th mock of the uneven-grid ensemble: n cycles through ``sizes``,
    n_s ~ U[-2, -1], f ~ U[0.5, 0.9] from its own seed, sigma_g = 0.3."""
    seed = 1708 * 1000 + m
    rng = np.random.Generator(np.random.PCG64(seed + 104729))
    ns = float(rng.uniform(-2.0, -1.0))
    f = float(rng.uniform(0.5, 0.9))
    return FieldModel(n=sizes[m % len(sizes)], box=box, amp=2.0e4, n_s=ns, f=f, sigma_g=0.3), seed
