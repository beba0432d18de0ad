"""GPU parity of the fine propagator (ac_fine_step, ac_fine_propagate_slices)
against the float64 oracle, through the C ABI.

Tolerances: float64 mode 1e-10 max-abs end to end; float32 mode 2e-5 max-abs
per fine step (the FFT round-off of an N^2-point float32 transform is about
eps_32 * log2(N^2) * |u| ~ 1e-6), and 2e-5 * sqrt(steps) over a slice, whose
errors add like a random walk while the scheme damps them.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import acpr_inputs as I
import oracle as O
import paper_2510_07672_gb300 as G

pytestmark = pytest.mark.gpu


def dev(a, dtype):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


CASES_F64 = [(8, 0), (16, 1), (32, 0), (64, 0), (64, 1), (128, 1)]
CASES_F32 = [(16, 0), (64, 1), (128, 0), (128, 1), (256, 0), (256, 1), (512, 0), (512, 1), (1024, 0), (1024, 1)]


@pytest.mark.parametrize("n,variant", CASES_F64)
def test_fine_step_f64(n, variant):
    eps = 2.5 / n
    batch = 3  # odd: the last pair carries one field
    u = np.stack([I.random_field(n, seed=10 + i, zero_mean=bool(variant)) for i in range(batch)])
    fp = G.FineParams(n, eps, 2.0, 1e-4, variant=variant, precision=G.AC_F64)
    got = G.ac_fine_step(fp, dev(u, torch.float64)).cpu().numpy()
    p = O.params(n, eps, 2.0, 1e-4, variant)
    for i in range(batch):
        assert np.abs(got[i] - O.fine_step(p, u[i])).max() < 1e-12


@pytest.mark.parametrize("n,variant", CASES_F32)
def test_fine_step_f32(n, variant):
    eps = 2.5 / n
    batch = 5
    u = np.stack([I.random_field(n, seed=20 + i, zero_mean=bool(variant)) for i in range(batch)])
    u32 = u.astype(np.float32)
    fp = G.FineParams(n, eps, 2.0, 5e-5, variant=variant, precision=G.AC_F32)
    got = G.ac_fine_step(fp, dev(u32, torch.float32)).cpu().numpy()
    p = O.params(n, eps, 2.0, 5e-5, variant)
    for i in range(batch):
        ref = O.fine_step(p, u32[i].astype(np.float64))
        assert np.abs(got[i] - ref).max() < 2e-5


@pytest.mark.parametrize("n,variant,steps", [(64, 0, 100), (64, 1, 60), (128, 1, 20)])
def test_propagate_f64(n, variant, steps):
    eps = 0.025 if n == 64 else 2.5 / n
    u = np.stack([I.random_field(n, seed=i, zero_mean=bool(variant)) for i in range(2)])
    fp = G.FineParams(n, eps, 2.0, 1e-4, variant=variant, precision=G.AC_F64)
    got = G.ac_fine_propagate_slices(fp, steps, dev(u, torch.float64)).cpu().numpy()
    p = O.params(n, eps, 2.0, 1e-4, variant)
    for i in range(2):
        assert np.abs(got[i] - O.fine_propagate(p, steps, u[i])).max() < 1e-10


@pytest.mark.parametrize("n,variant,steps", [(128, 0, 50), (256, 1, 200)])
def test_propagate_f32(n, variant, steps):
    eps = 0.01 if n == 256 else 2.5 / n
    u = np.stack([I.random_field(n, seed=40 + i, zero_mean=bool(variant)) for i in range(3)]).astype(np.float32)
    fp = G.FineParams(n, eps, 2.0, 5e-5, variant=variant, precision=G.AC_F32)
    got = G.ac_fine_propagate_slices(fp, steps, dev(u, torch.float32)).double().cpu().numpy()
    p = O.params(n, eps, 2.0, 5e-5, variant)
    ref = O.fine_propagate(p, steps, u[1].astype(np.float64))
    assert np.abs(got[1] - ref).max() < 2e-5 * np.sqrt(steps)
    if variant:
        # mass held at its float64 entry value to float32 rounding
        for i in range(3):
            assert abs(got[i].mean() - u[i].astype(np.float64).mean()) < 1e-7


def test_propagate_zero_steps_and_empty():
    n = 64
    u = dev(I.random_field(n, 1)[None].repeat(3, 0), torch.float32)
    fp = G.FineParams(n, 0.04, 2.0, 1e-4, precision=G.AC_F32)
    out = G.ac_fine_propagate_slices(fp, 0, u)
    assert torch.equal(out, u)
    empty = torch.empty(0, n, n, device="cuda")
    assert G.ac_fine_propagate_slices(fp, 10, empty).numel() == 0


def test_mass_conservation_long_run_f32():
    """Mass stays at its entry value over 2000 steps (the mean mode is held)."""
    n = 256
    u = I.random_field(n, seed=3)
    u = (u - u.mean() + 0.1).astype(np.float32)
    m0 = u.astype(np.float64).mean()
    fp = G.FineParams(n, 0.01, 2.0, 5e-5, variant=G.AC_MASS_CONSERVING, precision=G.AC_F32)
    out = G.ac_fine_propagate_slices(fp, 2000, dev(u[None], torch.float32))
    assert abs(out.double().mean().item() - m0) < 1e-7
    assert out.abs().max().item() <= 2 / np.sqrt(3) + 1e-4


def test_maximum_bound_principle_f32():
    n = 128
    u = I.random_field(n, seed=4, amp=1.0).astype(np.float32)
    fp = G.FineParams(n, 2.5 / n, 2.0, 1e-2, variant=G.AC_CLASSIC, precision=G.AC_F32)
    out = G.ac_fine_propagate_slices(fp, 300, dev(u[None], torch.float32))
    assert out.abs().max().item() <= 1.0 + 1e-5


def test_full_size_sampled():
    """The 256^2 mass-conserving workload in the bench's launch shape (512
    fields, 200 steps); sampled fields are checked against the oracle."""
    n, steps = 256, 200
    w = I.MASS_F32_256
    ics = np.stack([I.random_field(n, seed=s, zero_mean=True) for s in range(512)]).astype(np.float32)
    fp = G.FineParams(n, w.eps, w.S, w.dt, variant=w.variant, precision=G.AC_F32)
    out = G.ac_fine_propagate_slices(fp, steps, dev(ics, torch.float32)).double().cpu().numpy()
    p = O.params(n, w.eps, w.S, w.dt, w.variant)
    for f in (0, 311, 511):
        ref = O.fine_propagate(p, steps, ics[f].astype(np.float64))
        assert np.abs(out[f] - ref).max() < 2e-5 * np.sqrt(steps)
    assert np.isfinite(out).all()


@pytest.mark.parametrize("n,prec", [(64, G.AC_F32), (128, G.AC_F32), (256, G.AC_F32), (128, G.AC_F64),
                                    (256, G.AC_F64)])
def test_every_launch_shape_computes_the_same(n, prec):
    """The launch shapes only re-partition the field over CTAs.  Rows travel in
    pairs (rows l and l + R/2 of a CTA's R rows), so the pairing, and with it
    the rounding, follows the partition: every shape agrees with the default to
    round-off (float32: 1e-5 after 7 steps; float64: 1e-12), and each shape is
    bitwise reproducible on its own."""
    dt = torch.float64 if prec == G.AC_F64 else torch.float32
    names = G.ac_fine_variants(n, prec)
    assert names
    u = dev(np.stack([I.random_field(n, seed=s) for s in range(5)]), dt)
    outs = {}
    for variant in (0, 1):
        fp = G.FineParams(n, 2.5 / n, 2.0, 5e-5, variant=variant, precision=prec)
        for i in range(len(names)):
            G.ac_fine_set_variant(n, prec, i)
            outs[(variant, i)] = G.ac_fine_propagate_slices(fp, 7, u)
        tol = 1e-12 if prec == G.AC_F64 else 1e-5
        for i in range(1, len(names)):
            assert (outs[(variant, i)] - outs[(variant, 0)]).abs().max().item() < tol, names[i]
            G.ac_fine_set_variant(n, prec, i)
            assert torch.equal(G.ac_fine_propagate_slices(fp, 7, u), outs[(variant, i)]), names[i]
        # shapes with the same cluster split (occupancy, exchange by cluster
        # barriers or by asynchronous copies, with or without a separate
        # exchange buffer) move the same values: bitwise equal
        split = lambda nm: "_".join(nm.split("_")[:3])  # noqa: E731
        for i, name in enumerate(names):
            first = next(k for k, nm in enumerate(names) if split(nm) == split(name))
            assert torch.equal(outs[(variant, i)], outs[(variant, first)]), (name, names[first])
    G.ac_fine_set_variant(n, prec, 0)


@pytest.mark.parametrize("n,prec", [(256, G.AC_F32), (128, G.AC_F64)])
def test_async_exchange_trajectory_and_adjoint(n, prec):
    """With an asynchronous-exchange shape selected, the trajectory mode gives
    the barrier kernel's states bit for bit, and the adjoint (whose mean
    broadcast needs the cluster barriers) falls back to the barrier kernel."""
    dt = torch.float64 if prec == G.AC_F64 else torch.float32
    names = G.ac_fine_variants(n, prec)
    split = lambda nm: "_".join(nm.split("_")[:3])  # noqa: E731
    fp = G.FineParams(n, 2.5 / n, 2.0, 5e-5, variant=1, precision=prec)
    u = dev(np.stack([I.random_field(n, seed=s, zero_mean=True) for s in range(3)]), dt)
    for ia in [i for i, nm in enumerate(names) if "_async" in nm]:
        ib = next(i for i, nm in enumerate(names) if "_async" not in nm and split(nm) == split(names[ia]))
        res = {}
        for i in (ib, ia):
            G.ac_fine_set_variant(n, prec, i)
            traj = G.ac_fine_trajectory(fp, 5, u)
            lam = G.ac_fine_adjoint(fp, 5, traj[:5].contiguous(), traj[5].contiguous())
            res[i] = (traj, lam)
        assert torch.equal(res[ia][0], res[ib][0]), names[ia]
        assert torch.equal(res[ia][1], res[ib][1]), names[ia]
    G.ac_fine_set_variant(n, prec, 0)


def test_autotune_picks_a_shape():
    n = 256
    fp = G.FineParams(n, 0.01, 2.0, 5e-5, variant=1, precision=G.AC_F32)
    u = dev(np.stack([I.random_field(n, seed=s, zero_mean=True) for s in range(64)]), torch.float32)
    out = torch.empty_like(u)
    times, idx = G.ac_fine_autotune(fp, 10, u, out)
    assert len(times) == len(G.ac_fine_variants(n, G.AC_F32))
    assert all(t > 0 for t in times.values())
    assert times[G.ac_fine_variants(n, G.AC_F32)[idx]] == min(times.values())
    G.ac_fine_set_variant(n, G.AC_F32, 0)


@pytest.mark.parametrize("variant", [0, 1])
def test_propagate_1024_two_pass(variant):
    """1024^2 fields run the two-pass path through L2/HBM; three fields (mapped
    launch), 6 steps, against the oracle, plus mass conservation."""
    n, steps = 1024, 6
    u = np.stack([I.random_field(n, seed=60 + i, zero_mean=bool(variant)) for i in range(3)]).astype(np.float32)
    fp = G.FineParams(n, 0.004, 2.0, 2e-5, variant=variant, precision=G.AC_F32)
    got = G.ac_fine_propagate_slices(fp, steps, dev(u, torch.float32)).double().cpu().numpy()
    p = O.params(n, 0.004, 2.0, 2e-5, variant)
    ref = O.fine_propagate(p, steps, u[2].astype(np.float64))
    assert np.abs(got[2] - ref).max() < 2e-5 * np.sqrt(steps)
    if variant:
        assert abs(got[0].mean() - u[0].astype(np.float64).mean()) < 1e-7
    zero = G.ac_fine_propagate_slices(fp, 0, dev(u, torch.float32)).cpu().numpy()
    assert np.array_equal(zero, u)


def test_propagate_1024_with_caller_workspace():
    """ac_fine_propagate_slices_ws: the 1024^2 path with the caller's
    workspace gives the same bits as with the library's own, and a workspace
    one byte too small is rejected before any launch."""
    n, steps = 1024, 3
    u = dev(np.stack([I.random_field(n, seed=70 + i) for i in range(2)]).astype(np.float32), torch.float32)
    fp = G.FineParams(n, 0.004, 2.0, 2e-5, variant=G.AC_CLASSIC, precision=G.AC_F32)
    ref = G.ac_fine_propagate_slices(fp, steps, u)
    nbytes = G.ac_fine_workspace_bytes(n, 2, G.AC_F32)
    assert nbytes > 0 and G.ac_fine_workspace_bytes(256, 2, G.AC_F32) == 0
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    out = torch.empty_like(u)
    G.ac_fine_propagate_slices_ws(fp, steps, u, out, ws)
    assert torch.equal(out, ref)
    with pytest.raises(G.AcprError, match="AC_ERR_ARG"):
        G.ac_fine_propagate_slices_ws(fp, steps, u, out, ws[: nbytes - 1])
