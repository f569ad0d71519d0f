"""Seeded synthetic inputs: analytic initial conditions and random states.

This module holds no arithmetic of the discretisation: every function maps
node coordinates (computed by the caller with its own LGL rule) or a seed to
plain arrays.  It is the one module that both the CUDA path's callers and the
oracle's tests use, so that the same inputs reach both.

Initial conditions (Sec. 7 of the paper, with the readings stated per function):
* ``sine``: u0 = sin(2 pi x) for 1D linear advection.
* ``isentropic_vortex``: the 2D Euler vortex of Sec. 7.3 (S = 5, M = 0.5,
  gamma = 1.4, f = 1 - x0^2 - x1^2).  The total energy is read as
  E = p/(gamma-1) + rho (v1^2 + v2^2)/2 (the printed 0.5 (v1^2+v2^2)/rho is
  dimensionally inconsistent with v being a velocity); the centre is a
  parameter (x0 = x - cx, x1 = y - cy).  The exact solution is the initial
  field translated by (t, 0), periodically.
* ``density_wave``: rho = 1 + 0.2 sin(2 pi (x+y+z)), v = (1,1,1), p = 1 (in d
  dimensions: v = (1,..,1)); exact solution rho(x - t v).
* ``burgers_fourier``: 8 random Fourier modes with amplitudes summing to 0.5.
* ``burgers_instance``: the parameters of one instance of the batched viscous
  Burgers workload (grid side, N, s, viscosity, data seed) drawn from its seed.
"""
import math

import numpy as np


def sine(x, t=0.0, a=1.0):
    """u(x, t) = sin(2 pi (x - a t)), shape (..., 1)."""
    return np.sin(2.0 * np.pi * (np.asarray(x) - a * t))[..., None]


def isentropic_vortex(x, y, t=0.0, gamma=1.4, S=5.0, M=0.5, center=(5.0, 5.0), period=None):
    """Conservative state (rho, rho v1, rho v2, E) of the vortex, shape (..., 4).

    ``period`` = (Lx, Ly) wraps the translated coordinates into the periodic box
    centred on ``center`` (exact solution at time t on a periodic domain)."""
    x0 = np.asarray(x) - t - center[0]
    x1 = np.asarray(y) - center[1]
    if period is not None:
        x0 = (x0 + 0.5 * period[0]) % period[0] - 0.5 * period[0]
        x1 = (x1 + 0.5 * period[1]) % period[1] - 0.5 * period[1]
    f = 1.0 - x0 ** 2 - x1 ** 2
    rho = (1.0 - S ** 2 * (gamma - 1.0) * M ** 2 * np.exp(f) / (8.0 * np.pi ** 2)) ** (1.0 / (gamma - 1.0))
    v1 = 1.0 - S * x1 * np.exp(0.5 * f) / (2.0 * np.pi)
    v2 = S * x0 * np.exp(0.5 * f) / (2.0 * np.pi)
    p = rho ** gamma / (gamma * M ** 2)
    E = p / (gamma - 1.0) + 0.5 * rho * (v1 ** 2 + v2 ** 2)
    return np.stack([rho, rho * v1, rho * v2, E], axis=-1)


def density_wave(*coords, t=0.0, gamma=1.4, amp=0.2, p=1.0):
    """Conservative Euler state of the advected density wave in d = len(coords) dimensions."""
    d = len(coords)
    phase = sum(np.asarray(c) for c in coords) - d * t
    rho = 1.0 + amp * np.sin(2.0 * np.pi * phase)
    comps = [rho] + [rho * 1.0 for _ in range(d)]
    E = p / (gamma - 1.0) + 0.5 * rho * d
    comps.append(E * np.ones_like(rho))
    return np.stack(comps, axis=-1)


def burgers_fourier(x, y, seed, n_modes=8, amplitude=0.5, kmax=4):
    """u0 = sum_k a_k sin(2 pi (p_k x + q_k y) + phi_k), integer (p_k, q_k) in [-kmax, kmax]^2 \\ 0,
    a_k ~ U(-1, 1) rescaled so that sum |a_k| = amplitude, phi_k ~ U(0, 2 pi); shape (..., 1)."""
    rng = np.random.default_rng(seed)
    modes = []
    while len(modes) < n_modes:
        pq = rng.integers(-kmax, kmax + 1, size=2)
        if pq[0] != 0 or pq[1] != 0:
            modes.append(pq)
    a = rng.uniform(-1.0, 1.0, size=n_modes)
    a *= amplitude / np.sum(np.abs(a))
    phi = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    u = np.zeros(np.broadcast(np.asarray(x), np.asarray(y)).shape)
    for k in range(n_modes):
        u = u + a[k] * np.sin(2.0 * np.pi * (modes[k][0] * np.asarray(x) + modes[k][1] * np.asarray(y)) + phi[k])
    return u[..., None]


def random_array(shape, seed, scale=1.0):
    """Standard-normal array (FP64) with a fixed seed."""
    return scale * np.random.default_rng(seed).standard_normal(shape)


def perturbed(state, seed, rel=1e-2):
    """state * (1 + rel * N(0,1)) elementwise: a nearby non-smooth state that keeps the
    sign of every component (used to keep Euler density and pressure positive)."""
    return state * (1.0 + rel * np.random.default_rng(seed).standard_normal(state.shape))


def vortex_period_center(lo, hi):
    """Centre of the box [lo, hi]^2 (placement of the vortex in a periodic box)."""
    return (0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1]))


def log_uniform(rng, lo, hi):
    return math.exp(rng.uniform(math.log(lo), math.log(hi)))


def burgers_instance(i, sides=(8, 16, 32, 64), N_range=(2, 6), s_range=(2, 5), nu_range=(1e-3, 1e-1)):
    """Instance i of the batched 2D viscous Burgers workload on the periodic unit square:
    seed 1000 + i draws the grid side (uniform over ``sides``), N and s (uniform integers in
    the closed ranges), the viscosity (log-uniform) and the Fourier data seed."""
    rng = np.random.default_rng(1000 + i)
    side = int(sides[rng.integers(0, len(sides))])
    N = int(rng.integers(N_range[0], N_range[1] + 1))
    s = int(rng.integers(s_range[0], s_range[1] + 1))
    nu = log_uniform(rng, *nu_range)
    return {"side": side, "N": N, "s": s, "nu": nu, "seed": 1000 + i}
