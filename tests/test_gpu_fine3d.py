"""GPU parity of the fine step on the periodic cube (ac_fine3d_propagate, the 3D
experiments of Sec. 4) against the float64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import acpr_inputs as I
import oracle as O
import paper_2510_07672_gb300 as G

pytestmark = pytest.mark.gpu


def _cube(n, seed, zero_mean=False):
    u = -0.9 + 1.8 * I.uniform01(seed, I.STREAM_IC, n ** 3).reshape(n, n, n)
    return u - u.mean() if zero_mean else u


@pytest.mark.parametrize("variant", [0, 1])
def test_f64_matches_oracle(variant):
    """Three fields (the last pair has no partner) of 32^3, 5 steps: 1e-12."""
    n, steps = 32, 5
    u = np.stack([_cube(n, 10 + f, zero_mean=bool(variant)) for f in range(3)])
    fp = G.FineParams(n, 0.05, 2.0, 2e-3, variant=variant, precision=G.AC_F64)
    got = G.ac_fine3d_propagate(fp, steps, torch.tensor(u, device="cuda")).cpu().numpy()
    p = O.params(n, 0.05, 2.0, 2e-3, variant)
    for f in range(3):
        ref = O.fine3d_propagate(p, steps, u[f])
        assert np.abs(got[f] - ref).max() < 1e-12


@pytest.mark.parametrize("n", [64, 128])
def test_f32_matches_oracle(n):
    """float32, mass-conserving, two fields (one complex pair), 4 steps:
    2e-5 sqrt(steps) max-abs; the mean is held."""
    steps = 4
    u = np.stack([_cube(n, 20 + f, zero_mean=True) for f in range(2)])
    fp = G.FineParams(n, 0.02, 2.0, 1e-3, variant=1, precision=G.AC_F32)
    ut = torch.tensor(u, dtype=torch.float32, device="cuda")
    got = G.ac_fine3d_propagate(fp, steps, ut).double().cpu().numpy()
    p = O.params(n, 0.02, 2.0, 1e-3, 1)
    ref = O.fine3d_propagate(p, steps, ut[1].double().cpu().numpy())
    assert np.abs(got[1] - ref).max() < 2e-5 * np.sqrt(steps)
    assert abs(got[0].mean() - ut[0].double().mean().item()) < 1e-6


def test_constant_along_k_matches_gpu_2d_step_and_in_place():
    """A 128^3 field constant along the last axis evolves as the 2D step of its
    slice (the GPU's 2D kernel, float32, to rounding), also in place."""
    n, steps = 128, 10
    w = I.random_field(n, seed=30)
    fp2 = G.FineParams(n, 0.02, 2.0, 1e-3, variant=0, precision=G.AC_F32)
    w_t = torch.tensor(w, dtype=torch.float32, device="cuda")[None]
    ref2 = G.ac_fine_propagate_slices(fp2, steps, w_t)[0]
    u = w_t[0][:, :, None].expand(n, n, n).contiguous()[None]
    got = G.ac_fine3d_propagate(fp2, steps, u, u_out=u)  # in place
    assert got.data_ptr() == u.data_ptr()
    assert (got[0] - ref2[:, :, None]).abs().max().item() < 2e-5 * np.sqrt(steps)
    assert (got[0] - got[0][:, :, :1]).abs().max().item() < 1e-6
