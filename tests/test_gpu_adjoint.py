"""GPU parity of the adjoint path (ac_fine_trajectory, ac_fine_adjoint,
ac_energy, ac_energy_grad, ac_energy_gradient_ic) against the oracle, and the
checkpointed energy gradient of the 256^2 workload against central finite
differences (h = 1e-6, float64)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import acpr_inputs as I
import oracle as O
import paper_2510_07672_gb300 as G

pytestmark = pytest.mark.gpu


def dev(a, dt=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dt, device="cuda")


@pytest.mark.parametrize("n,variant", [(32, 0), (32, 1), (64, 1), (128, 0)])
def test_trajectory_and_adjoint_step(n, variant):
    eps, dt = 2.5 / n, 1e-3
    fp = G.FineParams(n, eps, 2.0, dt, variant=variant, precision=G.AC_F64)
    p = O.params(n, eps, 2.0, dt, variant)
    u = I.random_field(n, seed=3)
    traj = G.ac_fine_trajectory(fp, 3, dev(u[None])).cpu().numpy()
    ref = [u]
    for _ in range(3):
        ref.append(O.fine_step(p, ref[-1]))
    assert np.abs(traj[:, 0] - np.stack(ref)).max() < 1e-12
    lam = np.random.default_rng(2).standard_normal((n, n))
    got = G.ac_fine_adjoint(fp, 1, dev(u[None][None]), dev(lam[None])).cpu().numpy()[0]
    assert np.abs(got - O.fine_adjoint_step(p, u, lam)).max() < 1e-12


def test_energy_and_energy_grad():
    n = 64
    p = O.params(n, 0.03, 2.0, 1e-3, 0)
    fp = G.FineParams(n, 0.03, 2.0, 1e-3, precision=G.AC_F64)
    u = np.stack([I.random_field(n, seed=s) for s in range(3)])
    e = G.ac_energy(fp, dev(u)).cpu().numpy()
    g = G.ac_energy_grad(fp, dev(u)).cpu().numpy()
    for i in range(3):
        assert abs(e[i] - O.energy(p, u[i])) < 1e-13 * abs(e[i])
        assert np.abs(g[i] - O.energy_grad(p, u[i])).max() < 1e-14


@pytest.mark.parametrize("variant,K", [(0, 16), (1, 7)])
def test_checkpointed_gradient_matches_oracle(variant, K):
    """Segments of K steps recomputed from checkpoints give the oracle's
    store-everything adjoint gradient (K = 7 leaves a ragged last segment)."""
    n, steps = 32, 60
    fp = G.FineParams(n, 0.05, 2.0, 2e-3, variant=variant, precision=G.AC_F64)
    u0 = I.random_field(n, seed=9)
    g = G.ac_energy_gradient_ic(fp, steps, dev(u0), checkpoint_every=K).cpu().numpy()
    ref = O.energy_gradient_through_solve(O.params(n, 0.05, 2.0, 2e-3, variant), steps, u0)
    assert np.abs(g - ref).max() < 1e-10 * np.abs(ref).max()


def test_energy_gradient_full_size_finite_differences():
    """256^2, eps = 0.01, dt = 5e-5, E_h at step 2000, checkpoints every 32
    steps, float64: <grad, d> against central differences with h = 1e-6 in
    three random directions (the differences use the GPU's own float64 fine
    solver and energy)."""
    n, steps = 256, 2000
    fp = G.FineParams(n, 0.01, 2.0, 5e-5, variant=G.AC_CLASSIC, precision=G.AC_F64)
    u0 = dev(I.random_field(n, seed=0))
    g = G.ac_energy_gradient_ic(fp, steps, u0, checkpoint_every=32)

    def E(u):
        return G.ac_energy(fp, G.ac_fine_propagate_slices(fp, steps, u[None].contiguous()))[0].item()

    rng = np.random.default_rng(0)
    hh = 1e-6
    for _ in range(3):
        d = dev(rng.standard_normal((n, n)))
        fd = (E(u0 + hh * d) - E(u0 - hh * d)) / (2 * hh)
        ad = torch.vdot(g.flatten(), d.flatten()).item()
        assert abs(fd - ad) <= 1e-6 * abs(fd), (fd, ad)


def test_energy_gradient_float32_close_to_float64():
    """The float32 gradient follows the float64 one to float32 accuracy: each
    of the 2 x 400 steps (forward recomputation and adjoint) adds ~eps_32 *
    log2(n^2) ~ 1e-6 relative round-off, accumulating like a random walk
    (~3e-5), and the terminal condition h^2 eps^2 Lap_h u weights the
    high-frequency part of that round-off by up to 8 eps^2 / h^2 ~ 5 relative
    to the smooth part: a bound of 5e-4."""
    n, steps = 256, 400
    u0 = I.random_field(n, seed=1)
    g64 = G.ac_energy_gradient_ic(G.FineParams(n, 0.01, 2.0, 5e-5, precision=G.AC_F64), steps, dev(u0))
    g32 = G.ac_energy_gradient_ic(G.FineParams(n, 0.01, 2.0, 5e-5, precision=G.AC_F32), steps,
                                  dev(u0, torch.float32))
    rel = (torch.linalg.norm(g32.double() - g64) / torch.linalg.norm(g64)).item()
    assert rel < 5e-4


def _energy_torch(u, eps, h):
    """E_h(u) = h^2 sum eps^2/2 (|D+x u|^2 + |D+y u|^2) + (u^2 - 1)^2 / 4 on the
    periodic grid (Sec. 2, Eq. energy, forward differences), in torch so that
    autograd differentiates it."""
    dx = (torch.roll(u, -1, dims=-2) - u) / h
    dy = (torch.roll(u, -1, dims=-1) - u) / h
    return h * h * (0.5 * eps * eps * (dx * dx + dy * dy) + 0.25 * (u * u - 1.0) ** 2).sum()


@pytest.mark.parametrize("variant", [0, 1])
def test_fine_solve_autograd_function(variant):
    """torch.autograd.Function over 100 fine steps with a checkpoint every 32
    (segments 32, 32, 32, 4, each recomputed in the backward pass), float64:
    (1) an arbitrary scalar loss of u^N, sum w u^N + 0.5 |u^N|^2, against
    central differences (h = 1e-6) along random directions, 1e-7 relative;
    (2) the energy loss E_h(u^N) against the oracle's gradient through the
    solve (every state stored, no checkpoints), 1e-10 relative."""
    n, steps, every, eps, dt = 32, 100, 32, 0.05, 1e-3
    fp = G.FineParams(n, eps, 2.0, dt, variant=variant, precision=G.AC_F64)
    u0 = I.random_field(n, seed=11, zero_mean=bool(variant))[None]
    w = dev(np.random.default_rng(12).standard_normal((1, n, n)))

    def loss(x):
        uN = G.fine_solve(x, fp, steps, every)
        return (w * uN).sum() + 0.5 * (uN * uN).sum()

    x = dev(u0).requires_grad_(True)
    loss(x).backward()
    g = x.grad.detach()
    hh = 1e-6
    for k in range(3):
        d = dev(np.random.default_rng(20 + k).standard_normal((1, n, n)))
        with torch.no_grad():
            fd = (loss(dev(u0) + hh * d) - loss(dev(u0) - hh * d)).item() / (2 * hh)
        assert abs(fd - (g * d).sum().item()) < 1e-7 * max(1.0, abs(fd))
    x = dev(u0).requires_grad_(True)
    _energy_torch(G.fine_solve(x, fp, steps, every), eps, 1.0 / n).backward()
    ref = O.energy_gradient_through_solve(O.params(n, eps, 2.0, dt, variant), steps, u0[0])
    assert np.abs(x.grad[0].cpu().numpy() - ref).max() < 1e-10 * np.abs(ref).max()
