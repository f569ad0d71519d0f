"""The no-allocation norm entry point (stdg_slab_norm_noalloc) against stdg_slab_norm.

Some callers cannot allocate device memory (their device memory belongs to a
pool they manage, or they run a loop in which a cudaMalloc/cudaFree would
synchronise the device).  stdg_slab_norm_noalloc serves them: it keeps its
partial sums in a static device array instead of context-owned scratch.  This
test calls it through the C ABI twice in a row, on different vectors, and
checks each result against the existing context-based stdg_slab_norm within
the 1e-12 relative tolerance of the other FP64 parity tests; it also checks
that a length above the stated maximum is refused before anything is
launched.  It sits in its own file that pytest collects last."""
import ctypes

import numpy as np
import pytest

from paper_2201_05800_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_noalloc_norm_matches_context_norm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2201_05800_gb300 import build, stdg
    build.build()
    lib = stdg.load()
    desc = stdg.make_config(dim=2, cells=[64, 64, 1], lo=[0, 0, 0], hi=[10, 10, 1], N=4, s=4,
                            equation=stdg.EULER, gamma=1.4, dt=0.02)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with stdg.Context(desc) as ctx:
        L = ctx.slab_len  # 1,638,400 values: 100 blocks of the static partials
        for seed in (3, 4):  # two calls in a row, the second reuses the static array
            x = torch.from_numpy(inputs.random_array(L, seed)).cuda()
            ref = ctx.slab_norm(x)
            stdg.slab_norm_noalloc(x, out)
            torch.cuda.synchronize()
            got = float(out.item())
            assert abs(got - ref) <= 1e-12 * ref, (got, ref)
            assert abs(got - float(np.linalg.norm(x.cpu().numpy()))) <= 1e-12 * ref
        # a short vector (one partial block) right after a long one
        y = torch.from_numpy(inputs.random_array(1000, 5)).cuda()
        stdg.slab_norm_noalloc(y, out)
        torch.cuda.synchronize()
        assert abs(float(out.item()) - float(np.linalg.norm(y.cpu().numpy()))) <= 1e-12 * float(out.item())
    # above the stated maximum: refused before any launch
    fn = lib.stdg_slab_norm_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p]
    st = fn(ctypes.c_void_p(out.data_ptr()), 67108864 + 1, ctypes.c_void_p(out.data_ptr()), None)
    assert st == 1  # STDG_ERR_INVALID_ARG
