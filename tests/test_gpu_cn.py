"""GPU parity of the Crank-Nicolson + Picard fine scheme of Sec. 3.1
(ac_cn_propagate_slices) against the float64 oracle (or_cn_propagate).

Tolerances as for the stabilised scheme: float64 1e-10 max-abs end to end
(Picard to 1e-13 on both sides); float32 2e-5 * sqrt(steps) (Picard to 1e-6
on the GPU, to 1e-13 in the oracle: the Picard map contracts by about
dt max|f'| / 2 per iteration, so the stopping gap is far below float32
rounding)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import acpr_inputs as I
import oracle as O
import paper_2510_07672_gb300 as G

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", [0, 1])
def test_cn_f64_64(variant):
    n, eps, dt, steps = 64, 0.025, 1e-4, 20
    u = np.stack([I.random_field(n, seed=s, zero_mean=bool(variant)) for s in range(3)])
    fp = G.FineParams(n, eps, 2.0, dt, variant=variant, precision=G.AC_F64)
    iters = torch.zeros(3, dtype=torch.int32, device="cuda")
    got = G.ac_cn_propagate_slices(fp, steps, torch.tensor(u, device="cuda"), tol=1e-13, max_iters=50,
                                   iters=iters).cpu().numpy()
    p = O.params(n, eps, 2.0, dt, variant)
    for i in range(3):
        ref, it = O.cn_propagate(p, steps, u[i], tol=1e-13, maxit=50)
        assert np.abs(got[i] - ref).max() < 1e-10
        assert abs(int(iters[i]) - it) <= steps     # the stopping test may flip by one near the threshold
    assert int(iters.min()) >= steps


@pytest.mark.parametrize("n,variant", [(64, 0), (128, 1), (256, 0), (256, 1)])
def test_cn_f32(n, variant):
    eps, dt, steps = 2.5 / n, 5e-5, 10
    u = np.stack([I.random_field(n, seed=10 + s, zero_mean=bool(variant)) for s in range(3)]).astype(np.float32)
    fp = G.FineParams(n, eps, 2.0, dt, variant=variant, precision=G.AC_F32)
    got = G.ac_cn_propagate_slices(fp, steps, torch.tensor(u, device="cuda"), tol=1e-6).double().cpu().numpy()
    p = O.params(n, eps, 2.0, dt, variant)
    ref, _ = O.cn_propagate(p, steps, u[1].astype(np.float64), tol=1e-13, maxit=50)
    assert np.abs(got[1] - ref).max() < 2e-5 * np.sqrt(steps)
    if variant:
        for i in range(3):
            assert abs(got[i].mean() - u[i].astype(np.float64).mean()) < 1e-7


def test_cn_mass_long_run_and_zero_steps():
    n = 256
    u = (I.random_field(n, seed=7) + 0.1).astype(np.float32)
    m0 = u.astype(np.float64).mean()
    fp = G.FineParams(n, 0.01, 2.0, 5e-5, variant=G.AC_MASS_CONSERVING, precision=G.AC_F32)
    ut = torch.tensor(u[None], device="cuda")
    out = G.ac_cn_propagate_slices(fp, 400, ut, tol=1e-6)
    assert abs(out.double().mean().item() - m0) < 1e-7
    assert torch.equal(G.ac_cn_propagate_slices(fp, 0, ut), ut)


def test_cn_unsupported_size_is_reported():
    fp = G.FineParams(512, 0.005, 2.0, 5e-5, precision=G.AC_F32)
    u = torch.zeros((1, 512, 512), device="cuda")
    with pytest.raises(G.AcprError):
        G.ac_cn_propagate_slices(fp, 1, u)


@pytest.mark.parametrize("graphs", [False, True])
def test_parareal_with_the_cn_fine_scheme_is_exact_at_k_equals_s(graphs):
    """Parareal whose F is the Crank-Nicolson step (ac_parareal_set_fine_scheme):
    at k = s the trajectory is the sequential Crank-Nicolson solve bit for bit
    (Sec. 3.3 exactness), with and without graph capture."""
    n, s, c = 64, 4, 20
    fp = G.FineParams(n, 2.5 / n, 2.0, 5e-5, variant=G.AC_MASS_CONSERVING, precision=G.AC_F32)
    wt, bs = I.cnn_weights(3, 16, seed=0)
    net = G.CoarseNet(3, 16, wt.astype(np.float32), bs.astype(np.float32), act=1, precision=G.AC_F32)
    u0 = torch.tensor(np.stack([I.random_field(n, seed=p, zero_mean=True) for p in range(3)]).astype(np.float32),
                      device="cuda")
    pr = G.Parareal(fp, net, u0, s, c)
    pr.enable_graphs(graphs)
    pr.set_fine_scheme(1, tol=1e-6, max_iters=50)
    its, _ = pr.solve(tol=0.0, kmax=s)
    assert its == [s] * 3
    seq = [u0]
    for _ in range(s):
        seq.append(G.ac_cn_propagate_slices(fp, c, seq[-1], tol=1e-6, max_iters=50))
    assert torch.equal(pr.trajectory(), torch.stack(seq, dim=1))
