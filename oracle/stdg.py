"""Space-time DG-SEM (STDG) and Lobatto IIIC (LoDG) slab systems and their solvers.

Oracle (test infrastructure only).  FP64 NumPy.

Slab arrays are held time-major, U[m] = U^{m+1} for the temporal LGL nodes
m = 0..s-1 (Eq. StCoeff); ``to_external`` / ``from_external`` convert to the
library's layout U[e][m][node][c] (element-major, time node, spatial node,
component).

Residuals (F is any spatial operator u -> F(u), e.g. dgsem.spatial_operator):

* STDG, Eq. DG_vs_RK:DG moved to one side with the sign that makes its
  Jacobian exactly Eq. Jacobian_ST:
    R_ST(U) = (D_tau^T M_tau (x) I) U - (B_tau (x) I) U* + dt/2 (M_tau (x) I) F(U),
  with the upwind temporal flux U* = (u^n, 0, ..., 0, U^s) of Eq. upwind_flux.
* LoDG, Eq. DG_vs_RK:RK:  R_RK(U) = U - 1 (x) u^n - dt (A (x) I) F(U), with A from
  Eq. SBP_to_RK (lgl.lobatto_iiic_from_dgsem).
* New solution u^{n+1} = U^s (Eq. un).

Exact Jacobian-vector products use the complex step
J v = Im R(U + i h v) / h (no subtractive cancellation); physics is written to
be complex safe for this.

Solvers: dense Newton with LU (Jacobian assembled column by column from exact
J e_k) for small systems, and Newton + GMRES(m) (modified Gram-Schmidt,
Givens rotations) for larger ones; both FP64.
"""
import numpy as np

from . import lgl, dgsem


# --------------------------------------------------------------------------- layout

def to_external(U, grid):
    """Time-major (s, *K_rev, *n_rev, r) -> external (*K_rev, s, *n_rev, r)."""
    d = grid.dim
    return np.moveaxis(U, 0, d)


def from_external(U_ext, grid):
    d = grid.dim
    return np.moveaxis(U_ext, d, 0)


# --------------------------------------------------------------------------- residuals

def stdg_residual(F, U, u_n, dt):
    """R_ST(U) for the slab U (time-major, shape (s, ...)), previous slab trace u_n."""
    s = U.shape[0]
    B, M, D, _ = lgl.temporal_matrices(s)
    omega = np.diag(M)
    R = np.zeros_like(U)
    for i in range(s):
        # ((D^T M) (x) I) U, row i:  sum_j D[j, i] omega_j U_j
        for j in range(s):
            R[i] += D[j, i] * omega[j] * U[j]
        R[i] += 0.5 * dt * omega[i] * F(U[i])
    # -(B (x) I) U*  with U* = (u_n, 0, ..., 0, U_s) and B = diag(-1, 0, ..., 0, 1)
    Ustar = [u_n] + [None] * (s - 2) + [U[s - 1]]
    for i in (0, s - 1):
        R[i] -= B[i, i] * Ustar[i]
    return R


def lodg_residual(F, U, u_n, dt):
    """R_RK(U) = U - 1 (x) u_n - dt (A (x) I) F(U) (stage equations, Lobatto IIIC)."""
    s = U.shape[0]
    A, _, _ = lgl.lobatto_iiic_from_dgsem(s)
    FU = [F(U[j]) for j in range(s)]
    R = np.empty_like(U)
    for i in range(s):
        R[i] = U[i] - u_n
        for j in range(s):
            R[i] -= dt * A[i, j] * FU[j]
    return R


def lodg_step(F, U, u_n, dt):
    """u^{n+1} = u^n + dt (b^T (x) I) F(U) (Eq. RK_solution)."""
    s = U.shape[0]
    _, b, _ = lgl.lobatto_iiic_from_dgsem(s)
    return u_n + dt * sum(b[j] * F(U[j]) for j in range(s))


def residual(form, F, U, u_n, dt):
    return stdg_residual(F, U, u_n, dt) if form == "stdg" else lodg_residual(F, U, u_n, dt)


def jv_exact(form, F, U, u_n, dt, v):
    """J(U) v = Im R(U + i h v) / h, the complex-step derivative of the residual.

    h is chosen so small that every product of two perturbations (order h^2)
    underflows to exactly 0: the real part of every intermediate is then
    bitwise the real evaluation, so branch decisions (|x|, max) are taken on
    the exact real values, as in forward-mode differentiation."""
    vmax = float(np.max(np.abs(v))) if v.size else 0.0
    if vmax == 0.0:
        return np.zeros_like(U)
    h = 1e-200 / vmax
    Rc = residual(form, F, U.astype(np.complex128) + 1j * h * v, u_n.astype(np.complex128), dt)
    return np.imag(Rc) / h


def jacobian_dense(form, F, U, u_n, dt):
    """Dense Jacobian dR/dU (rows/cols over the flattened time-major slab)."""
    n = U.size
    J = np.empty((n, n))
    e = np.zeros(n)
    for k in range(n):
        e[k] = 1.0
        J[:, k] = jv_exact(form, F, U, u_n, dt, e.reshape(U.shape)).ravel()
        e[k] = 0.0
    return J


# --------------------------------------------------------------------------- solvers

def gmres(matvec, b, tol, m, maxit):
    """Restarted GMRES(m) from x0 = 0 with modified Gram-Schmidt and Givens rotations.

    Stops when ||b - A x|| <= tol * ||b|| (estimated by the rotated right-hand side).
    Returns (x, iterations, relative residual estimate)."""
    n = b.size
    x = np.zeros(n)
    beta0 = np.linalg.norm(b)
    if beta0 == 0.0:
        return x, 0, 0.0
    its = 0
    rel = 1.0
    while its < maxit:
        r = b - matvec(x) if its > 0 else b.copy()
        beta = np.linalg.norm(r)
        rel = beta / beta0
        if rel <= tol:
            break
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            w = matvec(V[j])
            for i in range(j + 1):
                H[i, j] = np.dot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            rel = abs(g[j + 1]) / beta0
            if rel <= tol or its >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + V[:k].T @ y
        if rel <= tol:
            break
    return x, its, rel


def solve_slab_direct(form, F, u_n, dt, s, U0=None, rtol=1e-14, maxit=20):
    """Newton with the exact dense Jacobian and LU.  Returns (U, newton_its)."""
    U = np.stack([u_n] * s) if U0 is None else U0.copy()
    R = residual(form, F, U, u_n, dt)
    r0 = np.linalg.norm(R)
    its = 0
    while its < maxit and np.linalg.norm(R) > rtol * max(r0, 1.0):
        J = jacobian_dense(form, F, U, u_n, dt)
        U = U - np.linalg.solve(J, R.ravel()).reshape(U.shape)
        R = residual(form, F, U, u_n, dt)
        its += 1
    return U, its


def solve_slab_newton_gmres(form, F, u_n, dt, s, rtol=1e-10, atol=0.0, maxit=20,
                            gmres_m=30, gmres_tol=1e-3, gmres_maxit=1000, stats=None, scaling=None):
    """Newton-Krylov: U0 = 1 (x) u_n; J dU = -R by GMRES(m) with exact J v; U += dU.

    Stops when ||R(U_k)||_2 <= max(rtol ||R(U_0)||_2, atol) or after maxit steps.
    scaling="temporal_mass" solves the left-scaled system (W^-1 J) dU = -W^-1 R with
    W = M_tau (x) I instead (every row of temporal node m divided by omega_m): the same
    Newton step, in fewer GMRES iterations; the GMRES tolerance then applies to the
    scaled residual."""
    U = np.stack([u_n] * s)
    R = residual(form, F, U, u_n, dt)
    r0 = np.linalg.norm(R)
    history = [r0]
    lin_its = 0
    k = 0
    if scaling == "temporal_mass":
        _, omega = lgl.lgl_nodes_weights(s)
        winv = (1.0 / omega).reshape((s,) + (1,) * (U.ndim - 1))
    elif scaling is None:
        winv = 1.0
    else:
        raise ValueError(scaling)
    while k < maxit and np.linalg.norm(R) > max(rtol * r0, atol):
        Uk = U
        mv = lambda x: (winv * jv_exact(form, F, Uk, u_n, dt, x.reshape(U.shape))).ravel()
        dU, its, _ = gmres(mv, -(winv * R).ravel(), gmres_tol, gmres_m, gmres_maxit)
        lin_its += its
        U = U + dU.reshape(U.shape)
        R = residual(form, F, U, u_n, dt)
        history.append(np.linalg.norm(R))
        k += 1
    if stats is not None:
        stats.update(newton_its=k, gmres_its=lin_its, history=history)
    return U


def march(form, F, u0, dt, s, nslabs, solver="direct", **kw):
    """Advance nslabs slabs; returns the list of final-node states u^1..u^nslabs."""
    out = []
    u = u0
    for _ in range(nslabs):
        if solver == "direct":
            U, _ = solve_slab_direct(form, F, u, dt, s)
        else:
            U = solve_slab_newton_gmres(form, F, u, dt, s, **kw)
        u = U[s - 1]
        out.append(u)
    return out


# --------------------------------------------------------------------------- norms

def lgl_weighted_norm(grid, U):
    """Space-time LGL-weighted L2 norm (Eq. DG_norm, read as the square root of the
    summed quadratic forms) of a time-major slab or of a single time level."""
    W = grid.node_weights()[..., None] * grid.jacobian()
    if U.ndim == len(grid.state_shape):
        return float(np.sqrt(np.sum(W * np.abs(U) ** 2)))
    s = U.shape[0]
    _, omega = lgl.lgl_nodes_weights(s)
    tot = sum(omega[m] * np.sum(W * np.abs(U[m]) ** 2) for m in range(s))
    return float(np.sqrt(tot))


def l2_error_overintegrated(grid, u, exact, nq=None):
    """||u_h - u_exact||_{L2} of one time level with (n+2)-point Gauss-Legendre per direction.

    exact(*coords) -> array (..., r).  Over-integration because LGL quadrature
    is not exact for the degree-2N integrand."""
    d, n = grid.dim, grid.n
    nq = nq or n + 2
    xg, wg = np.polynomial.legendre.leggauss(nq)
    P = lgl.lagrange_interpolation_matrix(grid.xi, xg)  # (nq, n)
    uq = u
    for a in range(d):
        ax = grid.node_axis(a)
        uq = np.moveaxis(np.tensordot(uq, P, axes=([ax], [1])), -1, ax)
    coords = []
    full = tuple(reversed(grid.cells)) + (nq,) * d
    for a in range(d):
        e_shape = [1] * (2 * d)
        e_shape[grid.elem_axis(a)] = grid.cells[a]
        q_shape = [1] * (2 * d)
        q_shape[grid.node_axis(a)] = nq
        x = grid.lo[a] + grid.h[a] * np.arange(grid.cells[a]).reshape(e_shape) \
            + 0.5 * grid.h[a] * (1.0 + xg.reshape(q_shape))
        coords.append(np.broadcast_to(x, full))
    Wq = np.ones((nq,) * d)
    for a in range(d):
        shape = [1] * d
        shape[d - 1 - a] = nq
        Wq = Wq * wg.reshape(shape)
    err = uq - exact(*coords)
    return float(np.sqrt(np.sum(grid.jacobian() * Wq[..., None] * err ** 2)))
