"""Convective fluxes and the Rusanov (local Lax-Friedrichs) numerical flux.

Oracle (test infrastructure only).  FP64 NumPy, written so that every function
also accepts complex arrays: the exact Jacobian-vector products of
``oracle.stdg`` use the complex step, so |x| and max(a, b) are taken on the
real part (x * sign(Re x), branch chosen by Re) instead of np.abs / np.maximum.

* Euler equations, Eqs. eulereq/defu and the flux f_i printed after them
  (Sec. 7.3): u = (rho, rho v_1..rho v_d, E), p = (gamma-1)(E - |m|^2/(2 rho)),
  f_i = (m_i, m_i m_1/rho + delta_{i1} p, ..., m_i m_d/rho + delta_{id} p,
  (E + p) m_i/rho).
* Linear advection f_i = a_i u (Sec. 7.1 test problems, config of 1D advection).
* Inviscid Burgers f_i = u^2/2 (convective part of the viscous Burgers problem).
* Rusanov flux, Eq. flux:llf: H.n = {F_c}.n + lambda/2 [[u]], written for the
  face between a left state uL and a right state uR with normal +e_a:
  H_a = (f_a(uL) + f_a(uR))/2 - lambda/2 (uR - uL),
  lambda = max(|v_a(uL)| + c(uL), |v_a(uR)| + c(uR)) pointwise on the face.
  For advection lambda = |a_a|, which makes H the exact upwind flux.
"""
import numpy as np

ADVECTION, EULER, BURGERS = "advection", "euler", "burgers"


def re_abs(x):
    """|x| evaluated on the real part, complex-step safe.  At Re x = 0 the derivative is
    taken from the x >= 0 branch (|x| is not differentiable there; the paper is silent,
    this reading matches the tie rule of re_max)."""
    return np.where(np.real(x) >= 0, x, -x)


def re_max(a, b):
    """max(a, b) with the branch chosen on the real parts (ties take a)."""
    return np.where(np.real(a) >= np.real(b), a, b)


def num_components(eq, dim):
    return dim + 2 if eq == EULER else 1


def pressure(u, gamma):
    d = u.shape[-1] - 2
    rho = u[..., 0]
    ke = sum(u[..., 1 + k] ** 2 for k in range(d)) / (2.0 * rho)
    return (gamma - 1.0) * (u[..., -1] - ke)


def euler_flux(u, a, gamma):
    """f_a(u) for the Euler equations, direction a in 0..d-1."""
    d = u.shape[-1] - 2
    rho = u[..., 0]
    m_a = u[..., 1 + a]
    v_a = m_a / rho
    p = pressure(u, gamma)
    f = np.empty_like(u)
    f[..., 0] = m_a
    for k in range(d):
        f[..., 1 + k] = u[..., 1 + k] * v_a + (p if k == a else 0.0)
    f[..., -1] = (u[..., -1] + p) * v_a
    return f


def euler_wave_speed(u, a, gamma):
    """|v_a| + c with the speed of sound c = sqrt(gamma p / rho)."""
    rho = u[..., 0]
    c = np.sqrt(gamma * pressure(u, gamma) / rho)
    return re_abs(u[..., 1 + a] / rho) + c


def flux(eq, u, a, params):
    """Convective flux f_a(u) for equation ``eq``; u has components on the last axis."""
    if eq == ADVECTION:
        return params["adv_vel"][a] * u
    if eq == EULER:
        return euler_flux(u, a, params["gamma"])
    if eq == BURGERS:
        return 0.5 * u * u
    raise ValueError(eq)


def wave_speed(eq, u, a, params):
    """Largest characteristic speed in direction a (no component axis)."""
    if eq == ADVECTION:
        return abs(params["adv_vel"][a]) * np.ones(u.shape[:-1])
    if eq == EULER:
        return euler_wave_speed(u, a, params["gamma"])
    if eq == BURGERS:
        return re_abs(u[..., 0])
    raise ValueError(eq)


def rusanov(eq, uL, uR, a, params):
    """Numerical flux in direction a on a face with uL on the -e_a side, uR on the +e_a side."""
    lam = re_max(wave_speed(eq, uL, a, params), wave_speed(eq, uR, a, params))
    return 0.5 * (flux(eq, uL, a, params) + flux(eq, uR, a, params)) - 0.5 * lam[..., None] * (uR - uL)
