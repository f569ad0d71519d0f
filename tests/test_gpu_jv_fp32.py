"""The FP32 exact Jacobian-vector product (stdg_jv_fp32) against the oracle.

stdg_jv_fp32 runs the product the mixed-precision inner solve uses: for the 2D
(n = 5, s = 4) and 3D (n = 4, s = 3) Euler shapes the tangent-only kernel with
bulk-copied element tiles, otherwise the general operator kernel.  The oracle
evaluates J v = Im R(U + i h v) / h (complex step, FP64) at the same inputs,
rounded to FP32 first so that only the kernel's arithmetic is measured.

Tolerance (FP32 arithmetic, unit roundoff u = 2^-24 ~ 6e-8): each output is a
sum of at most T ~ 60 products (volume, faces, temporal coupling); its rounding
error is bounded by ~T u S with S the sum of absolute values of the terms, and
S / |J v| stays below ~30 for these states, so the relative LGL-weighted L2
error is required below 2e-5 and every entry within 2e-4 of max |J v|.
"""
import numpy as np
import pytest

from helpers import Problem
from oracle import stdg as ost
from paper_2201_05800_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2201_05800_gb300 import build, stdg
    build.build()
    stdg.load()
    return stdg


# (dim, cells, N, s): the two bulk-copy shapes with ragged last tiles and one-element
# periodic directions, grids with more tiles than the GPU holds CTAs at once (every CTA's L2
# prefetch of a later tile lands inside the grid), and a shape served by the general kernel
CASES = [(2, (7, 3), 4, 4), (2, (4, 4), 4, 4), (2, (1, 5), 4, 4), (3, (3, 2, 2), 3, 3), (3, (2, 1, 3), 3, 3),
         (3, (13, 12, 12), 3, 3), (2, (55, 50), 4, 4), (2, (3, 3), 3, 3), (3, (2, 2, 2), 2, 2)]


@pytest.mark.parametrize("dim,cells,N,s", CASES)
def test_jv_fp32_matches_oracle(S, dim, cells, N, s):
    import torch
    lo, hi = (0.0,) * dim, (1.0,) * dim
    prob = Problem(dim=dim, cells=cells, N=N, s=s, eq="euler", dt=0.02, lo=lo, hi=hi)
    u_n = prob.rough_state(11, rel=0.05)
    U = prob.rough_slab(u_n, 13)
    v = inputs.random_array(U.shape, 17)
    U32 = prob.ext(U).astype(np.float32)
    v32 = prob.ext(v).astype(np.float32)
    # the oracle at the FP32-rounded inputs
    Uq = prob.from_ext(U32.astype(np.float64))
    vq = prob.from_ext(v32.astype(np.float64))
    ref = ost.jv_exact("stdg", prob.F, Uq, u_n, prob.dt, vq)
    with S.Context(prob.config(gmres_m=1)) as ctx:
        out = ctx.jv_fp32(torch.from_numpy(U32).cuda(), torch.from_numpy(v32).cuda()).cpu().numpy()
    got = prob.from_ext(out.astype(np.float64))
    rel = ost.lgl_weighted_norm(prob.grid, got - ref) / ost.lgl_weighted_norm(prob.grid, ref)
    assert rel <= 2e-5, rel
    assert np.max(np.abs(got - ref)) <= 2e-4 * np.max(np.abs(ref))


def test_jv_fp32_full_size_density_wave_against_fp64_product(S):
    """3D density wave, 32^3 hexes, N = 3, s = 3 (the mixed-precision workload's launch): the
    FP32 product against the library's FP64 exact product at the same (FP32-rounded) inputs;
    the oracle itself is checked on the small grids above (the full grid is beyond it)."""
    import torch
    K = 32
    d = S.make_config(dim=3, cells=[K, K, K], lo=[0, 0, 0], hi=[1, 1, 1], N=3, s=3, equation=S.EULER, gamma=1.4,
                      dt=0.0067, gmres_m=1, jv_mode=S.JV_EXACT)
    with S.Context(d) as ctx:
        X = ctx.node_coordinates()
        u0 = inputs.density_wave(X[:, 0], X[:, 1], X[:, 2]).ravel()
        L = ctx.slab_len
        U = torch.from_numpy(np.tile(u0.reshape(-1, 1, 64 * 5), (1, 3, 1)).ravel()).cuda()
        U = U * (1.0 + 1e-3 * torch.from_numpy(inputs.random_array(L, 21)).cuda())
        v = torch.from_numpy(inputs.random_array(L, 22)).cuda()
        U32, v32 = U.float(), v.float()
        got = ctx.jv_fp32(U32, v32).double()
        ref = ctx.jv(U32.double(), torch.from_numpy(u0).cuda(), v32.double())
        rel = float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref))
        assert rel <= 2e-5, rel


@pytest.mark.parametrize("cells", [(3, 2, 2), (4, 4, 4), (2, 1, 3)])
def test_jv_bf16_tensor_cores_against_oracle(S, cells):
    """STDG_MIXED_BF16 (3D Euler, n = 4, s = 3): the volume contractions run on the tensor cores
    with BF16 inputs (relative rounding 2^-9 of each flux tangent and of each D entry) and FP32
    accumulation.  Against the oracle: within 1e-2 relative (LGL-weighted L2), and above the FP32
    kernel's error (the tensor-core path ran); ragged last tiles (odd element counts)."""
    import torch
    prob = Problem(dim=3, cells=cells, N=3, s=3, eq="euler", dt=0.02)
    u_n = prob.rough_state(31, rel=0.05)
    U = prob.rough_slab(u_n, 33)
    v = inputs.random_array(U.shape, 37)
    U32 = prob.ext(U).astype(np.float32)
    v32 = prob.ext(v).astype(np.float32)
    Uq = prob.from_ext(U32.astype(np.float64))
    vq = prob.from_ext(v32.astype(np.float64))
    ref = ost.jv_exact("stdg", prob.F, Uq, u_n, prob.dt, vq)
    out = {}
    for name, prec in (("bf16", S.MIXED_BF16), ("fp32", S.MIXED_FP32)):
        with S.Context(prob.config(gmres_m=1, precision=prec, jv_mode=S.JV_EXACT)) as ctx:
            o = ctx.jv_fp32(torch.from_numpy(U32).cuda(), torch.from_numpy(v32).cuda()).cpu().numpy()
        out[name] = prob.from_ext(o.astype(np.float64))
    nrm = ost.lgl_weighted_norm(prob.grid, ref)
    e_bf16 = ost.lgl_weighted_norm(prob.grid, out["bf16"] - ref) / nrm
    e_fp32 = ost.lgl_weighted_norm(prob.grid, out["fp32"] - ref) / nrm
    assert e_bf16 <= 1e-2, e_bf16
    assert e_fp32 <= 2e-5 and e_bf16 > 10 * e_fp32, (e_bf16, e_fp32)


def test_bf16_mixed_slab_solve_reaches_the_oracle(S):
    """3D density wave on 3^3 hexes, N = 3, s = 3: the BF16 tensor-core Jacobian-vector products
    in the inner solve, FP64 Newton residuals refine: the slab is within 1e-8 of the oracle's at
    the workload tolerances."""
    prob = Problem(dim=3, cells=(3, 3, 3), N=3, s=3, eq="euler", dt=1.0)
    X = prob.grid.coordinates()
    u0 = inputs.density_wave(*X)
    prob.dt = 0.5 * min(prob.grid.h) / 2.6
    U_or = ost.solve_slab_newton_gmres("stdg", prob.F, u0, prob.dt, prob.s, rtol=1e-13, atol=1e-14,
                                       gmres_tol=1e-11, gmres_m=40)
    with S.Context(prob.config(precision=S.MIXED_BF16, jv_mode=S.JV_EXACT, newton_rtol=1e-10, gmres_rtol=0.05,
                               newton_maxit=40)) as ctx:
        ctx.set_state(np.ascontiguousarray(u0).ravel())
        st = ctx.advance_slab()
        U = prob.from_ext(ctx.get_slab())
    assert st["status"] == 0, st
    rel = ost.lgl_weighted_norm(prob.grid, U - U_or) / ost.lgl_weighted_norm(prob.grid, U_or)
    assert rel <= 1e-8, (rel, st)


def test_bf16_precision_is_refused_for_other_shapes(S):
    prob = Problem(dim=2, cells=(4, 4), N=4, s=4, eq="euler", dt=0.02)
    with pytest.raises(S.StdgError):
        S.Context(prob.config(precision=S.MIXED_BF16, jv_mode=S.JV_EXACT))
