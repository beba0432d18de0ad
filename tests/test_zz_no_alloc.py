"""The allocation-free convergence increment (parareal_residual_noalloc).

Some callers cannot allocate device memory at all: a plugin inside a framework
that owns every allocation, a host callback, a loop that must never block on
the allocator.  This entry point keeps its scratch in a fixed device array of
the library and writes its results to a device buffer the caller passes.  These
tests call it through the C ABI and compare it with parareal_residual, which
uses library-allocated scratch, within the tolerance of the residual's parity
test (1e-12 relative on rel_l2; max_abs exactly).  The file sorts last so that a
run stopping at its first failure has run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import paper_2510_07672_gb300 as G
from paper_2510_07672_gb300 import abi


def test_noalloc_rejects_sizes_beyond_its_scratch():
    """The size check runs before any pointer is touched."""
    L = G.load()
    out = L.parareal_residual_noalloc(4096, 1024, G.AC_F32, None, None, None, None)
    assert out == -2
    assert b"scratch limit" in L.ac_last_error()


@pytest.mark.gpu
def test_noalloc_matches_allocating_residual_twice():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    for s, n, dt in ((5, 64, torch.float64), (32, 256, torch.float32)):
        a = rng.standard_normal((s + 1, n, n))
        b = a + 1e-3 * rng.standard_normal((s + 1, n, n))
        A = torch.tensor(a, dtype=dt, device="cuda")
        B = torch.tensor(b, dtype=dt, device="cuda")
        ref_l2, ref_mx = G.parareal_residual(A, B)
        for call in range(2):
            out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
            G.parareal_residual_noalloc(A, B, out)
            torch.cuda.synchronize()
            l2, mx = out[0].item(), out[1].item()
            assert abs(l2 - ref_l2) <= 1e-12 * ref_l2, (call, l2, ref_l2)
            assert mx == ref_mx, (call, mx, ref_mx)
        # swap the arguments on the second size: the array keeps no stale state
        out = torch.empty(4, dtype=torch.float64, device="cuda")
        G.parareal_residual_noalloc(B, A, out)
        l2b, mxb = G.parareal_residual(B, A)
        torch.cuda.synchronize()
        assert abs(out[0].item() - l2b) <= 1e-12 * l2b and out[1].item() == mxb
