"""Test helpers: one problem specification -> matched oracle grid and library config.

Inputs reach both sides from here: node coordinates come from the oracle's
grid and initial data from paper_2201_05800_gb300.inputs; nothing here reads
a value produced by the CUDA path.

Tolerance of FP64 operator parity (derived from the arithmetic): the kernel
(strong form, Eq. SBP applied) and the oracle (weak form as printed) compute
each output as a differently associated sum of at most T = d(n+2) + s + 2
products.  Each side's rounding error is bounded by ~T * u * S_I with u =
2^-53 and S_I the sum of absolute values of the terms of output I (bounded by
``term_scale``).  For T <= 40, 2 * 40 * 1.1e-16 < 1e-14; the tests use
1e-12 * S (a 100x margin for the reciprocal, square root and division steps).
"""
import numpy as np

from oracle import dgsem, lgl, physics, stdg
from paper_2201_05800_gb300 import inputs

EQ = {"advection": 0, "euler": 1, "burgers": 2}


class Problem:
    def __init__(self, dim, cells, N, s, eq, dt, lo=None, hi=None, adv=(1.0, 0.5, -0.75), gamma=1.4, nu=0.0):
        self.dim, self.cells, self.N, self.s, self.eq, self.dt = dim, tuple(cells), N, s, eq, dt
        self.lo = tuple(lo or (0.0,) * dim)
        self.hi = tuple(hi or (1.0,) * dim)
        self.adv, self.gamma, self.nu = tuple(adv), gamma, nu
        params = {"adv_vel": self.adv, "gamma": gamma}
        if nu:
            params["viscosity"] = nu
        self.grid = dgsem.Grid(dim, cells, self.lo, self.hi, N, eq, params)

    def F(self, u):
        return dgsem.spatial_operator(self.grid, u)

    def config(self, **kw):
        from paper_2201_05800_gb300 import stdg as S
        base = dict(dim=self.dim, cells=list(self.cells) + [1] * (3 - self.dim), lo=list(self.lo) + [0.0] * (3 - self.dim),
                    hi=list(self.hi) + [1.0] * (3 - self.dim), N=self.N, s=self.s, equation=EQ[self.eq],
                    adv_vel=list(self.adv) + [0.0] * (3 - len(self.adv)), gamma=self.gamma, dt=self.dt,
                    viscosity=self.nu)
        base.update(kw)
        return S.make_config(**base)

    # ---- states (oracle layouts)
    def smooth_state(self):
        X = self.grid.coordinates()
        if self.eq == "euler":
            return inputs.density_wave(*X, gamma=self.gamma)
        return np.sin(2 * np.pi * sum(X))[..., None]

    def rough_state(self, seed, rel=0.05):
        u = self.smooth_state()
        if self.eq == "euler":
            return inputs.perturbed(u, seed, rel)
        return u + inputs.random_array(u.shape, seed, 0.3)

    def rough_slab(self, u_n, seed, rel=0.02):
        """Time-major slab near 1 (x) u_n (oracle layout (s, ...))."""
        out = []
        for m in range(self.s):
            if self.eq == "euler":
                out.append(inputs.perturbed(u_n, seed + 17 * m, rel))
            else:
                out.append(u_n + inputs.random_array(u_n.shape, seed + 17 * m, 0.1))
        return np.stack(out)

    def ext(self, U):
        """time-major oracle slab -> flat external layout [e][m][node][c]"""
        return np.ascontiguousarray(stdg.to_external(U, self.grid)).ravel()

    def from_ext(self, flat):
        shp = list(self.grid.state_shape)
        d = self.dim
        ext_shape = shp[:d] + [self.s] + shp[d:]
        return stdg.from_external(flat.reshape(ext_shape), self.grid)

    def term_scale(self, U, u_n, with_time=True):
        """Bound on the sum of absolute values of the terms of any residual entry."""
        g = self.grid
        _, M, D, _ = lgl.temporal_matrices(self.s)
        C = np.abs(D * np.diag(M)[:, None])
        umax = max(np.max(np.abs(U)), np.max(np.abs(u_n)))
        fmax = 0.0
        for m in range(self.s):
            for a in range(self.dim):
                fmax = max(fmax, np.max(np.abs(physics.flux(self.eq, U[m], a, g.params))))
        lam = 0.0
        if self.eq != "advection" or True:
            for m in range(self.s):
                for a in range(self.dim):
                    lam = max(lam, np.max(np.abs(physics.wave_speed(self.eq, U[m], a, g.params))))
        Dmax = np.max(np.abs(g.D))
        spatial = sum((2.0 / g.h[a]) * (g.n * Dmax * fmax + (2 * fmax + lam * 2 * umax) / g.w[0])
                      for a in range(self.dim))
        if self.nu:
            # interior penalty terms: second differences, averaged gradients, penalised jumps
            eta = 10.0 * self.N ** 2
            wmin = np.min(g.w)
            spatial += sum(self.nu * (2.0 / g.h[a]) ** 2 * (g.n * Dmax) ** 2 * umax * (1.0 + 2.0 / wmin)
                           + (2.0 / g.h[a]) / wmin * (self.nu * eta / g.h[a]) * 2 * umax
                           for a in range(self.dim))
        return (np.max(C.sum(axis=0)) + 2.0) * umax + 0.5 * self.dt * np.max(np.diag(M)) * spatial


def rel_lgl(prob, A, B):
    """Relative space-time LGL-weighted L2 difference ||A - B|| / ||B|| (time-major slabs)."""
    return stdg.lgl_weighted_norm(prob.grid, A - B) / stdg.lgl_weighted_norm(prob.grid, B)
