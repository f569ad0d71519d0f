"""Spatial DG-SEM operator F(u) = M^-1 L_h(u) in weak form on a periodic Cartesian grid.

Oracle (test infrastructure only).  FP64 NumPy (complex-step safe).

Follows Sec. 3.1: Eq. elementint (element integrals with F_v = 0, S = 0),
Eq. surfaceint (surface integrals with the numerical flux H_c of Eq. flux:llf),
collocated flux interpolation F_h = sum_i F(u_i) psi_i, LGL quadrature on the
LGL nodes (diagonal mass matrix), and Eq. ode (F = M^-1 L_h).  The weak form
is evaluated as printed: for every test function psi_I (tensor LGL node I of an
element E with Jacobian J = prod_a h_a/2 of the affine map from [-1,1]^d),

  (J w_I) F_I =  sum_a sum_{nodes K} J w_K f_a(u_K) d psi_I/dx_a (x_K)
               - sum_{faces e of E} int_e (H . n) psi_I dS,

with d psi_I/dx_a (x_K) = (2/h_a) D[k_a, i_a] prod_{b != a} delta(k_b, i_b),
D[j, i] = l_i'(xi_j), and the face integral by the LGL rule of the face
(Jacobian J / (h_a/2), weights prod_{b != a} w_{i_b}).  H is single valued per
face; it enters the element on the -e_a side with n = +e_a and the element on
the +e_a side with n = -e_a.

Readings (where the paper is silent or garbled):
* Reference element [-1, 1]^d with Jacobian h/2 per direction (the paper's
  DUNE code uses [0, 1]^d, Sec. 3.1; the scheme is the same).
* The printed UFL surface code adds the H_c term while Eq. surfaceint subtracts
  it and has unbalanced parentheses; the standard conservative weak form
  int F.grad(psi) - oint (H.n) psi, consistent with d_t u = -div F (Eq. general),
  is taken.

Array layout: a state of one time level has shape (*K_rev, *n_rev, r) where
K_rev = (K_z, K_y, K_x)[-d:] are the element counts (x fastest) and
n_rev = (n,)*d the LGL node counts (x fastest); the component axis is last.
Spatial direction a (0 = x) has element axis d-1-a and node axis 2d-1-a.
"""
import numpy as np

from . import lgl, physics


class Grid:
    """Uniform periodic Cartesian grid on the box [lo, hi] with K_a elements per direction."""

    def __init__(self, dim, cells, lo, hi, N, eq, params):
        self.dim = dim
        self.cells = tuple(int(k) for k in cells[:dim])
        self.lo = tuple(float(v) for v in lo[:dim])
        self.hi = tuple(float(v) for v in hi[:dim])
        self.N = N
        self.n = N + 1
        self.eq = eq
        self.params = params
        self.r = physics.num_components(eq, dim)
        self.h = tuple((self.hi[a] - self.lo[a]) / self.cells[a] for a in range(dim))
        self.xi, self.w = lgl.lgl_nodes_weights(self.n)
        self.D = lgl.lagrange_derivative_matrix(self.xi)

    @property
    def state_shape(self):
        return tuple(reversed(self.cells)) + (self.n,) * self.dim + (self.r,)

    def elem_axis(self, a):
        return self.dim - 1 - a

    def node_axis(self, a):
        return 2 * self.dim - 1 - a

    def jacobian(self):
        return float(np.prod([h / 2.0 for h in self.h]))

    def node_weights(self):
        """Tensor-product LGL weights W_I, shape (*n_rev)."""
        W = np.ones((self.n,) * self.dim)
        for a in range(self.dim):
            shape = [1] * self.dim
            shape[self.dim - 1 - a] = self.n
            W = W * self.w.reshape(shape)
        return W

    def coordinates(self):
        """Physical coordinates of every node: list of d arrays of shape (*K_rev, *n_rev)."""
        d = self.dim
        coords = []
        full = tuple(reversed(self.cells)) + (self.n,) * d
        for a in range(d):
            e_shape = [1] * (2 * d)
            e_shape[self.elem_axis(a)] = self.cells[a]
            n_shape = [1] * (2 * d)
            n_shape[self.node_axis(a)] = self.n
            left = self.lo[a] + self.h[a] * np.arange(self.cells[a]).reshape(e_shape)
            x = left + 0.5 * self.h[a] * (1.0 + self.xi.reshape(n_shape))
            coords.append(np.broadcast_to(x, full).copy())
        return coords


def _take(arr, axis, index):
    sl = [slice(None)] * arr.ndim
    sl[axis] = index
    return arr[tuple(sl)]


def spatial_operator(grid, u):
    """F(u) = M^-1 L_h(u) for one time level u of shape grid.state_shape."""
    d, n = grid.dim, grid.n
    J = grid.jacobian()
    W = grid.node_weights()[..., None]  # (*n_rev, 1)
    L = np.zeros_like(u)
    for a in range(d):
        ax_e, ax_n = grid.elem_axis(a), grid.node_axis(a)
        # element integral: sum_K J w_K f_a(u_K) (2/h_a) D[k_a, i_a]
        Wf = J * W * physics.flux(grid.eq, u, a, grid.params)
        vol = np.tensordot(Wf, grid.D, axes=([ax_n], [0]))  # new last axis = i_a
        L += (2.0 / grid.h[a]) * np.moveaxis(vol, -1, ax_n)
        # surface integral over the faces normal to e_a
        uL = _take(u, ax_n, n - 1)  # trace of each element on its +e_a face
        uR = np.roll(_take(u, ax_n, 0), -1, axis=ax_e)  # trace of the +e_a neighbour
        H = physics.rusanov(grid.eq, uL, uR, a, grid.params)
        W_face = _face_weights(grid, a)
        HS = (J / (grid.h[a] / 2.0)) * W_face * H
        sl_hi = [slice(None)] * u.ndim
        sl_hi[ax_n] = n - 1
        L[tuple(sl_hi)] -= HS  # n = +e_a on the element's upper face
        sl_lo = [slice(None)] * u.ndim
        sl_lo[ax_n] = 0
        L[tuple(sl_lo)] += np.roll(HS, 1, axis=ax_e)  # n = -e_a on the neighbour's lower face
    nu = grid.params.get("viscosity", 0.0)
    if nu:
        L -= sipg_form(grid, u, nu)
    return L / (J * W)


def penalty(grid):
    """Interior-penalty parameter eta = 10 p^2 of the paper's UFL code (Sec. 4), p = N."""
    return grid.params.get("penalty", 10.0 * grid.N ** 2)


def sipg_form(grid, u, nu):
    """B(u, psi_I) for every test function psi_I: the symmetric interior penalty form of
    -nu Laplace(u) (F_v = nu grad u, Eq. general; H_v^IP of Sec. 3.1 with eta = 10 p^2 and
    h_e = |E| / |e| = h_a on a face normal to e_a), LGL quadrature on volume and faces:

      B(u, psi) = sum_E int_E nu grad u . grad psi
                - sum_F int_F ( {nu grad u} . [[psi]] + {nu grad psi} . [[u]] )
                + sum_F int_F sigma [[u]] . [[psi]],       sigma = nu eta / h_e,

    with [[v]] = v_L - v_R and {v} = (v_L + v_R)/2 on the face between the element
    below (L) and above (R) it in direction a.  Reading: the paper's printed surface
    terms disagree in sign between Eq. surfaceint and the UFL listing; this is the
    standard symmetric form, consistent with d_t u = nu Laplace(u)."""
    d, n = grid.dim, grid.n
    J = grid.jacobian()
    W = grid.node_weights()[..., None]
    eta = penalty(grid)
    B = np.zeros_like(u)
    for a in range(d):
        ax_e, ax_n = grid.elem_axis(a), grid.node_axis(a)
        ga = 2.0 / grid.h[a]
        # gradient component a at every node: (2/h_a) sum_j D[k, j] u_j along the line
        g = ga * np.moveaxis(np.tensordot(u, grid.D, axes=([ax_n], [1])), -1, ax_n)
        # volume: sum_K J w_K nu g_K (2/h_a) D[k_a, i_a]
        B += ga * np.moveaxis(np.tensordot(J * W * nu * g, grid.D, axes=([ax_n], [0])), -1, ax_n)
        # faces normal to e_a
        uL = _take(u, ax_n, n - 1)
        uR = np.roll(_take(u, ax_n, 0), -1, axis=ax_e)
        gL = _take(g, ax_n, n - 1)
        gR = np.roll(_take(g, ax_n, 0), -1, axis=ax_e)
        jump = uL - uR
        avg = 0.5 * (gL + gR)
        sigma = nu * eta / grid.h[a]
        JWf = (J / (grid.h[a] / 2.0)) * _face_weights(grid, a)
        sl_hi = [slice(None)] * u.ndim
        sl_hi[ax_n] = n - 1
        sl_lo = [slice(None)] * u.ndim
        sl_lo[ax_n] = 0
        # psi of the element below the face: [[psi]] = psi at its node n-1,
        # {grad_a psi} = (1/2)(2/h_a) D[n-1, i_a]
        B[tuple(sl_hi)] += JWf * (-nu * avg + sigma * jump)
        line = [1] * u.ndim
        line[ax_n] = n
        B -= np.expand_dims(JWf * nu * 0.5 * ga * jump, ax_n) * grid.D[n - 1].reshape(line)
        # psi of the element above the face: [[psi]] = -psi at its node 0,
        # {grad_a psi} = (1/2)(2/h_a) D[0, i_a]
        B[tuple(sl_lo)] += np.roll(JWf * (nu * avg - sigma * jump), 1, axis=ax_e)
        B -= np.roll(np.expand_dims(JWf * nu * 0.5 * ga * jump, ax_n), 1, axis=ax_e) * grid.D[0].reshape(line)
    return B


def _face_weights(grid, a):
    """prod_{b != a} w_{i_b} on a face normal to e_a, shape of a face trace (with comp axis)."""
    d = grid.dim
    Wf = np.ones((grid.n,) * (d - 1))
    others = [b for b in range(d) if b != a]  # ascending directions
    # face trace axes (after removing node axis of a) keep the reversed order
    for pos, b in enumerate(reversed(others)):
        shape = [1] * (d - 1)
        shape[pos] = grid.n
        Wf = Wf * grid.w.reshape(shape)
    return Wf[..., None]


def integrate(grid, u):
    """Cell-summed conserved quantities sum_E J sum_I w_I u_I per component (shape (r,))."""
    J = grid.jacobian()
    W = grid.node_weights()[..., None]
    axes = tuple(range(2 * grid.dim))
    return np.sum(J * W * u, axis=axes)
