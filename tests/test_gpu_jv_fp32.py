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
# periodic directions, and a shape served by the general kernel
CASES = [(2, (7, 3), 4, 4), (2, (4, 4), 4, 4), (2, (1, 5), 4, 4), (3, (3, 2, 2), 3, 3), (3, (2, 1, 3), 3, 3),
         (2, (3, 3), 3, 3), (3, (2, 2, 2), 2, 2)]


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
