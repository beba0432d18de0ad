"""GPU parity of the Parareal driver (parareal_iterate / ac_parareal_solve) and
the convergence increment (parareal_residual) against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import acpr_inputs as I
import oracle as O
import paper_2510_07672_gb300 as G

pytestmark = pytest.mark.gpu


def test_residual_matches_oracle():
    s, n = 5, 64
    a = np.random.default_rng(0).standard_normal((s + 1, n, n))
    b = a + 1e-3 * np.random.default_rng(1).standard_normal((s + 1, n, n))
    for dt in (torch.float64, torch.float32):
        A = torch.tensor(a, dtype=dt, device="cuda")
        B = torch.tensor(b, dtype=dt, device="cuda")
        l2, mx = G.parareal_residual(A, B)
        rl2, rmx = O.residual(A.double().cpu().numpy(), B.double().cpu().numpy())
        assert abs(l2 - rl2) <= 1e-12 * rl2
        assert mx == rmx


def test_residual_nonfinite_is_reported():
    s, n = 2, 16
    A = torch.zeros(s + 1, n, n, device="cuda")
    B = torch.zeros(s + 1, n, n, device="cuda")
    A[2, 3, 4] = float("nan")
    with pytest.raises(G.AcprError, match="NONFINITE"):
        G.parareal_residual(A, B)


def test_plain_f64_workload_end_to_end():
    """64^2 classic AC in float64, 8 slices x 100 steps, tanh conv 1-16-16-16-1
    with N(0, 0.01^2) weights: every iteration's increment and the final
    trajectory match the oracle to 1e-10."""
    w = I.PLAIN_F64_64
    u0 = w.ics()
    wt, bs = w.weights()
    fp = G.FineParams(w.n, w.eps, w.S, w.dt, variant=w.variant, precision=G.AC_F64)
    net = G.CoarseNet(w.layers, w.channels, wt, bs, act=w.act, precision=G.AC_F64)
    pr = G.Parareal(fp, net, torch.tensor(u0, device="cuda"), w.slices, w.steps)
    pr.iterate()  # k = 0
    incs = []
    for k in range(1, w.kmax + 1):
        l2, mx = pr.iterate()
        incs.append(l2[0])
    U = pr.trajectory()[0].cpu().numpy()
    ref = O.parareal(O.params(w.n, w.eps, w.S, w.dt, w.variant), O.CnnSpec(w.layers, w.channels, wt, bs, act=w.act),
                     w.slices, w.steps, kmax=w.kmax, tol=0.0, u0=u0[0])
    assert np.abs(U - ref["U"]).max() < 1e-10
    assert np.allclose(incs, ref["res_l2"], rtol=1e-6, atol=1e-14)


@pytest.mark.parametrize("m", [2, 3])
def test_coarse_composition_matches_oracle_f64(m):
    """G composed m times per slice (the remark after Algorithm 2), float64:
    the k = 0 sweep and every later iterate match the oracle's Algorithm 2
    with the same composition to 1e-10, and the handle counts m coarse
    applications per evaluation."""
    w = I.PLAIN_F64_64
    u0 = w.ics()
    wt, bs = w.weights()
    fp = G.FineParams(w.n, w.eps, w.S, w.dt, variant=w.variant, precision=G.AC_F64)
    net = G.CoarseNet(w.layers, w.channels, wt, bs, act=w.act, precision=G.AC_F64)
    s, c, kmax = 6, 40, 3
    pr = G.Parareal(fp, net, torch.tensor(u0, device="cuda"), s, c)
    pr.set_coarse_substeps(m)
    pr.iterate()  # k = 0
    ref0 = O.parareal(O.params(w.n, w.eps, w.S, w.dt, w.variant), O.CnnSpec(w.layers, w.channels, wt, bs, act=w.act),
                      s, c, kmax=0, tol=0.0, u0=u0[0], coarse_repeat=m)
    assert np.abs(pr.trajectory()[0].cpu().numpy() - ref0["U"]).max() < 1e-10
    incs = [pr.iterate()[0][0] for _ in range(kmax)]
    ref = O.parareal(O.params(w.n, w.eps, w.S, w.dt, w.variant), O.CnnSpec(w.layers, w.channels, wt, bs, act=w.act),
                     s, c, kmax=kmax, tol=0.0, u0=u0[0], coarse_repeat=m)
    assert np.abs(pr.trajectory()[0].cpu().numpy() - ref["U"]).max() < 1e-10
    assert np.allclose(incs, ref["res_l2"], rtol=1e-6, atol=1e-14)
    st = pr.stats()
    assert st["coarse_calls"] % m == 0 and st["coarse_calls"] > 0


def test_coarse_composition_exactness_f32():
    """With G composed three times, slices 0..k are still the sequential fine
    solve bit for bit after k iterations (Sec. 3.3), in float32 with the bf16
    conv; switching back to m = 1 restores the plain-G iterates."""
    n, s, c = 64, 5, 30
    fp = G.FineParams(n, 0.04, 2.0, 1e-4, variant=G.AC_MASS_CONSERVING, precision=G.AC_F32)
    wt, bs = I.cnn_weights(6, 32, seed=0)
    net = G.CoarseNet(6, 32, wt.astype(np.float32), bs.astype(np.float32), act=1, precision=G.AC_F32)
    u0 = torch.tensor(np.stack([I.random_field(n, 7, zero_mean=True), I.random_field(n, 8, zero_mean=True)]),
                      dtype=torch.float32, device="cuda")
    seq = [u0]
    for j in range(s):
        seq.append(G.ac_fine_propagate_slices(fp, c, seq[-1]))
    seq = torch.stack(seq, 1)
    pr = G.Parareal(fp, net, u0, s, c)
    pr.set_coarse_substeps(3)
    pr.enable_graphs(True)
    pr.iterate()
    g3 = u0
    for _ in range(3):
        g3 = G.cnn_coarse_step(net, g3)
    assert torch.equal(pr.trajectory()[:, 1], g3)
    for k in range(1, s + 1):
        pr.iterate()
        assert torch.equal(pr.trajectory()[:, : k + 1], seq[:, : k + 1]), k
    plain = G.Parareal(fp, net, u0, s, c)
    plain.iterate()
    pr.set_coarse_substeps(1)
    pr.reset(u0)
    pr.iterate()
    assert torch.equal(pr.trajectory(), plain.trajectory())


def test_exactness_on_gpu_f32():
    """After k iterations slices 0..k equal the GPU's own sequential fine solve
    bitwise (Sec. 3.3), in float32 with the bf16 conv."""
    n, s, c = 64, 6, 30
    fp = G.FineParams(n, 0.04, 2.0, 1e-4, variant=G.AC_MASS_CONSERVING, precision=G.AC_F32)
    wt, bs = I.cnn_weights(6, 32, seed=0)
    net = G.CoarseNet(6, 32, wt.astype(np.float32), bs.astype(np.float32), act=1, precision=G.AC_F32)
    u0 = torch.tensor(np.stack([I.random_field(n, 7, zero_mean=True), I.random_field(n, 8, zero_mean=True)]),
                      dtype=torch.float32, device="cuda")
    seq = [u0]
    for j in range(s):
        seq.append(G.ac_fine_propagate_slices(fp, c, seq[-1]))
    seq = torch.stack(seq, 1)  # [problems][s+1][n][n]
    pr = G.Parareal(fp, net, u0, s, c)
    pr.iterate()
    for k in range(1, s + 1):
        pr.iterate()
        U = pr.trajectory()
        assert torch.equal(U[:, : k + 1], seq[:, : k + 1]), k
    assert torch.equal(U, seq)


def test_mass_f32_solve_matches_oracle_iterates():
    """A reduced mass-conserving float32 problem (64^2, 8 slices of 50 steps,
    bf16 conv 1-16-16-16-1).  The solve stops once the increment is below
    1e-6 (or at k = s, where it is exact).  Its trajectory then matches the
    oracle's Parareal iterate at the same k (float64 arithmetic, conv with the
    same bf16 rounding) to the float32 accuracy of the fine solves,
    2e-5 * sqrt(steps) max-abs per slice."""
    n, s, c = 64, 8, 50
    eps, S, dt = 0.04, 2.0, 5e-5
    wt, bs = I.cnn_weights(4, 16, seed=0)
    wt, bs = wt.astype(np.float32), bs.astype(np.float32)
    u0 = np.stack([I.random_field(n, seed=p, zero_mean=True) for p in range(2)]).astype(np.float32)
    fp = G.FineParams(n, eps, S, dt, variant=1, precision=G.AC_F32)
    net = G.CoarseNet(4, 16, wt, bs, act=1, precision=G.AC_F32)
    pr = G.Parareal(fp, net, torch.tensor(u0, device="cuda"), s, c)
    its, l2 = pr.solve(tol=1e-6, kmax=s)
    U = pr.trajectory().double().cpu().numpy()
    spec = O.CnnSpec(4, 16, wt.astype(np.float64), bs.astype(np.float64), act=1, bf16=1)
    for p in range(2):
        assert l2[p] < 1e-6 or its[p] == s
        ref = O.parareal(O.params(n, eps, S, dt, 1), spec, s, c, kmax=its[p], tol=0.0,
                         u0=u0[p].astype(np.float64))
        assert ref["iters"] == its[p]
        assert np.abs(U[p] - ref["U"]).max() < 2e-5 * np.sqrt(c)
        assert l2[p] < 2 * ref["res_l2"][-1] + 2e-6


def test_full_size_mass256_in_the_bench_configuration():
    """The benchmarked workload at full size, configured as bench.py times it
    (16 mass-conserving 256^2 problems, 32 slices x 200 steps, the committed
    trained G with the mass shift, every iteration a CUDA graph).  Every
    problem stops below the 1e-6 increment or at k = s; at k = s the
    trajectory is the sequential fine solve bit for bit (Sec. 3.3 exactness:
    the fine kernel computes each field alone, so the batched sequential
    solve is the same function); sampled slices are checked against the
    float64 oracle's fine propagation, 2e-5 * sqrt(steps) per slice."""
    import os
    W = I.MASS_F32_256
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    z = np.load(os.path.join(root, "paper_2510_07672_gb300", "weights", "mass256_c32l6_gelu.npz"))
    net = G.CoarseNet(W.layers, W.channels, z["w"].astype(np.float32), z["b"].astype(np.float32), act=W.act,
                      precision=G.AC_F32, mass_fix=W.mass_fix)
    fp = G.FineParams(W.n, W.eps, W.S, W.dt, variant=W.variant, precision=G.AC_F32)
    ics = W.ics().astype(np.float32)
    u0 = torch.tensor(ics, device="cuda")
    pr = G.Parareal(fp, net, u0, W.slices, W.steps)
    pr.enable_graphs(True)
    its, l2 = pr.solve(tol=W.tol, kmax=W.kmax)
    U = pr.trajectory()
    assert all(r < W.tol or k == W.slices for k, r in zip(its, l2))
    # sequential fine solve of all problems, slice after slice
    seq = [u0]
    for _ in range(W.slices):
        seq.append(G.ac_fine_propagate_slices(fp, W.steps, seq[-1]))
    seq = torch.stack(seq, dim=1)
    for p, k in enumerate(its):
        if k == W.slices:
            assert torch.equal(U[p], seq[p])
        else:
            assert torch.equal(U[p, :k + 1], seq[p, :k + 1])  # U^k_j is exact for j <= k
    # sampled slices against the oracle (one slice of 200 float64 steps each)
    p_o = O.params(W.n, W.eps, W.S, W.dt, W.variant)
    for p, j in ((0, 0), (7, 13), (15, 31)):
        ref = O.fine_propagate(p_o, W.steps, U[p, j].double().cpu().numpy())
        assert np.abs(U[p, j + 1].double().cpu().numpy() - ref).max() < 2e-5 * np.sqrt(W.steps)


def test_full_size_unconverged_iterates_match_oracle():
    """Unconverged Parareal iterates at the benchmark's full size (256^2,
    32 slices x 200 steps, mass-conserving, the committed trained bf16 G with
    the mass shift) for one problem, at k = 1 and k = 2, against the oracle's
    Algorithm 2 run to the same k from the same initial field (float64 fine
    solves, conv with the same bf16 roundings).  Every slice n > k carries
    the correction F(U^{k-1}_n) + G(U^k_n) - G(U^{k-1}_n) (Sec. 3.3), so a
    wrong sign or slice index fails by O(|F - G|) ~ 1e-2.  The bound allows
    the float32 fine error (2e-5 sqrt(c) per slice) and bf16 rounding flips
    of G (up to 2e-2 of the stack's contribution per application) carried
    along the sweep.  Measured on GB300: max-abs 1.6e-3, relative L2 6.4e-4
    and 7.4e-4, increments within 1.5%; the bounds below leave a factor 3."""
    import os
    W = I.MASS_F32_256
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    z = np.load(os.path.join(root, "paper_2510_07672_gb300", "weights", "mass256_c32l6_gelu.npz"))
    w32, b32 = z["w"].astype(np.float32), z["b"].astype(np.float32)
    net = G.CoarseNet(W.layers, W.channels, w32, b32, act=W.act, precision=G.AC_F32, mass_fix=W.mass_fix)
    fp = G.FineParams(W.n, W.eps, W.S, W.dt, variant=W.variant, precision=G.AC_F32)
    u0 = W.ics()[:1].astype(np.float32)
    pr = G.Parareal(fp, net, torch.tensor(u0, device="cuda"), W.slices, W.steps)
    pr.iterate()  # k = 0
    got, incs = {}, {}
    for k in (1, 2):
        l2, _ = pr.iterate()
        incs[k] = l2[0]
        got[k] = pr.trajectory()[0].double().cpu().numpy()
    spec = O.CnnSpec(W.layers, W.channels, w32.astype(np.float64), b32.astype(np.float64), act=W.act,
                     mass_fix=W.mass_fix, bf16=1)
    p_o = O.params(W.n, W.eps, W.S, W.dt, W.variant)
    with O.threads(os.cpu_count() or 1):
        for k in (1, 2):
            ref = O.parareal(p_o, spec, W.slices, W.steps, kmax=k, tol=0.0, u0=u0[0].astype(np.float64))
            assert ref["iters"] == k
            err = np.abs(got[k] - ref["U"]).max(axis=(1, 2))
            rel = np.linalg.norm(got[k] - ref["U"]) / np.linalg.norm(ref["U"])
            print(f"k={k}: max-abs per slice (first, mid, last) {err[1]:.2e} {err[16]:.2e} {err[-1]:.2e}; "
                  f"max {err.max():.2e}; rel-L2 {rel:.2e}; increment gpu {incs[k]:.6e} oracle {ref['res_l2'][-1]:.6e}")
            assert err[: k + 1].max() < 2e-5 * np.sqrt(W.steps * k)   # the exact prefix: fine solves only
            assert err.max() < 5e-3
            assert rel < 2e-3
            assert abs(incs[k] - ref["res_l2"][-1]) < 5e-2 * ref["res_l2"][-1]


@pytest.mark.parametrize("prec", [G.AC_F32, G.AC_F64])
def test_fused_increment_equals_standalone_residual(prec):
    """The corrections leave the increment's partial sums of the slices they
    write; slices frozen at iteration k contribute only sum U^2.  After every
    iteration the driver's increments must equal parareal_residual (a
    separate float64 pass over both trajectories) on the same trajectories:
    relative L2 to 1e-12 and the sup norm exactly (float32 fields: the
    differences are split exactly into float pairs)."""
    n, s, c = 64, 6, 30
    dt_ = torch.float64 if prec == G.AC_F64 else torch.float32
    fp = G.FineParams(n, 0.04, 2.0, 1e-4, variant=G.AC_MASS_CONSERVING, precision=prec)
    wt, bs = I.cnn_weights(4, 16, seed=0)
    net = G.CoarseNet(4, 16, wt, bs, act=1, precision=prec)
    u0 = torch.tensor(np.stack([I.random_field(n, 7 + p, zero_mean=True) for p in range(3)]), dtype=dt_,
                      device="cuda")
    pr = G.Parareal(fp, net, u0, s, c)
    pr.enable_graphs(True)
    pr.iterate()  # k = 0
    for k in range(1, 5):
        prev = pr.trajectory().clone()
        l2, mx = pr.iterate()
        cur = pr.trajectory()
        for p in range(3):
            rl2, rmx = G.parareal_residual(cur[p].contiguous(), prev[p].contiguous())
            assert abs(l2[p] - rl2) <= 1e-12 * rl2, (k, p)
            assert mx[p] == rmx, (k, p)
