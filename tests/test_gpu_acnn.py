"""GPU parity of the ResBlock ACNN / mACNN (Sec. 3.2), the scheme-residual
loss (Eq. loss_ACN), Adam and Algorithm 1 against the float64 oracle, and the
Parareal driver with the ACNN as G."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import acpr_inputs as I
import oracle as O
import paper_2510_07672_gb300 as G

pytestmark = pytest.mark.gpu

F64, F32 = G.AC_F64, G.AC_F32


def _fields(n, batch, seed, zero_mean=False):
    return np.stack([I.random_field(n, seed=seed + p, zero_mean=zero_mean) for p in range(batch)])


def _dt(prec):
    return torch.float64 if prec == F64 else torch.float32


@pytest.mark.parametrize("C,R", [(4, 0), (4, 1), (4, 2), (4, 3), (4, 4), (16, 1)])
@pytest.mark.parametrize("prec", [F64, F32])
def test_forward_matches_oracle(C, R, prec):
    """Fused kernel (C = 4, R <= 3) and per-layer path (R = 4, C = 16), with the
    mass shift and an active limiter, several 32 x 32 tiles per field: float64 to
    1e-12, float32 to 3e-5 (float32 arithmetic and the exponential-form tanh)."""
    n, batch = 64, 3
    w, b = I.acnn_weights(C, R, seed=C + R)
    w, b = 1.5 * w, 1.5 * b
    u = _fields(n, batch, 100)
    net = G.Acnn(C, R, w, b, mass_fix=1, limiter=1, lo=-0.9, hi=0.9, precision=prec)
    got = net(torch.tensor(u, dtype=_dt(prec), device="cuda")).double().cpu().numpy()
    ref = O.acnn_forward(O.AcnnSpec(C, R, w, b, mass_fix=1, limiter=1, lo=-0.9, hi=0.9), u)
    tol = 1e-12 if prec == F64 else 3e-5
    assert np.abs(got - ref).max() < tol
    assert (np.abs(ref) == 0.9).any()  # the limiter acted somewhere


@pytest.mark.parametrize("n", [32, 128])
def test_fused_equals_layered_f64_and_mapping(n):
    """The fused kernel and the per-layer kernels agree to rounding (float64);
    the plain-G path with no mass shift or limiter matches the oracle too."""
    C, R, batch = 4, 2, 2
    w, b = I.acnn_weights(C, R, seed=3)
    u = torch.tensor(_fields(n, batch, 200), device="cuda")
    net = G.Acnn(C, R, w, b, precision=F64)
    fused = net(u)
    ws = net.new_workspace(n, batch)
    layered = net.forward_train(u, ws)
    assert (fused - layered).abs().max().item() < 1e-13
    ref = O.acnn_forward(O.AcnnSpec(C, R, w, b), u.cpu().numpy())
    assert np.abs(fused.cpu().numpy() - ref).max() < 1e-12


@pytest.mark.parametrize("C,R,mass_fix", [(4, 2, 1), (4, 0, 0), (16, 1, 1)])
def test_backward_matches_oracle_f64(C, R, mass_fix):
    """Parameter gradients (sums over the batch, limiter clamping some values)
    match the oracle's to 1e-10 relative to the largest entry."""
    n, batch = 32, 2
    w, b = I.acnn_weights(C, R, seed=7 + C)
    w, b = 1.5 * w, 1.5 * b
    u = _fields(n, batch, 300)
    gout = np.random.default_rng(4).standard_normal(u.shape)
    kw = dict(mass_fix=mass_fix, limiter=1, lo=-0.8, hi=0.8)
    net = G.Acnn(C, R, w, b, precision=F64, **kw)
    ut = torch.tensor(u, device="cuda")
    ws = net.new_workspace(n, batch)
    net.forward_train(ut, ws)
    gw, gb = net.backward(ut, torch.tensor(gout, device="cuda"), ws)
    rw, rb = O.acnn_backward(O.AcnnSpec(C, R, w, b, **kw), u, gout)
    scale = max(np.abs(rw).max(), np.abs(rb).max())
    assert np.abs(gw.cpu().numpy() - rw).max() < 1e-10 * scale
    assert np.abs(gb.cpu().numpy() - rb).max() < 1e-10 * scale


def test_backward_f32_close_to_oracle():
    C, R, n, batch = 4, 2, 64, 4
    w, b = I.acnn_weights(C, R, seed=9)
    u = _fields(n, batch, 400, zero_mean=True)
    gout = np.random.default_rng(5).standard_normal(u.shape)
    net = G.Acnn(C, R, w, b, mass_fix=1, precision=F32)
    ut = torch.tensor(u, dtype=torch.float32, device="cuda")
    ws = net.new_workspace(n, batch)
    net.forward_train(ut, ws)
    gw, gb = net.backward(ut, torch.tensor(gout, dtype=torch.float32, device="cuda"), ws)
    rw, rb = O.acnn_backward(O.AcnnSpec(C, R, w, b, mass_fix=1), u, gout)
    scale = max(np.abs(rw).max(), np.abs(rb).max())
    assert np.abs(gw.double().cpu().numpy() - rw).max() < 1e-4 * scale
    assert np.abs(gb.double().cpu().numpy() - rb).max() < 1e-4 * scale


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("prec", [F64, F32])
def test_loss_acn_matches_oracle(variant, prec):
    """Loss and dL/dU1 over a batch of pairs (n = 64, several blocks per field)."""
    n, batch = 64, 3
    p = G.FineParams(n, 0.02, 0.0, 1e-2, variant=variant, precision=prec)
    U0 = _fields(n, batch, 500)
    U1 = U0 + 0.05 * np.random.default_rng(6).standard_normal(U0.shape)
    dt = _dt(prec)
    loss, g = G.loss_acn(p, torch.tensor(U0, dtype=dt, device="cuda"), torch.tensor(U1, dtype=dt, device="cuda"))
    po = O.params(n, 0.02, 0.0, 1e-2, variant)
    U0c = torch.tensor(U0, dtype=dt).double().numpy()
    U1c = torch.tensor(U1, dtype=dt).double().numpy()
    rl, rg = O.loss_acn(po, U0c, U1c)
    tol = 1e-12 if prec == F64 else 2e-5
    assert abs(loss.item() - rl) <= tol * rl
    assert np.abs(g.double().cpu().numpy() - rg).max() <= tol * np.abs(rg).max() * (1 if prec == F64 else 10)


def test_adam_matches_oracle_f64():
    rng = np.random.default_rng(7)
    w = rng.standard_normal(1000)
    m, v = np.zeros(1000), np.zeros(1000)
    wt = torch.tensor(w, device="cuda")
    mt, vt = torch.zeros(1000, dtype=torch.float64, device="cuda"), torch.zeros(1000, dtype=torch.float64,
                                                                                device="cuda")
    lib = G.load()
    import ctypes as C
    for t in range(1, 4):
        g = rng.standard_normal(1000)
        gt = torch.tensor(g, device="cuda")
        rc = lib.acnn_adam_step(F64, C.c_void_p(wt.data_ptr()), C.c_void_p(gt.data_ptr()), C.c_void_p(mt.data_ptr()),
                                C.c_void_p(vt.data_ptr()), 1000, 1e-2, 0.9, 0.999, 1e-8, t,
                                C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0
        O.adam(w, g, m, v, 1e-2, 0.9, 0.999, 1e-8, t)
    assert np.abs(wt.cpu().numpy() - w).max() < 1e-14


def test_algorithm1_matches_oracle_f64():
    """Algorithm 1 (two epochs, two subsets of two fields, two time steps, two
    inner updates): every loss and the final parameters match the oracle's run
    of the same algorithm to 1e-9."""
    C, R, n = 4, 2, 32
    w, b = I.acnn_weights(C, R, seed=11)
    U0s = _fields(n, 4, 600, zero_mean=True)
    perm = np.array([[2, 0, 3, 1], [1, 3, 0, 2]])
    p = G.FineParams(n, 0.03, 0.0, 5e-3, variant=1, precision=F64)
    net = G.Acnn(C, R, w, b, mass_fix=1, precision=F64)
    losses = net.train_alg1(p, torch.tensor(U0s, device="cuda"), perm, q=2, steps=2, b_inner=2, lr=2e-3)
    spec = O.AcnnSpec(C, R, w, b, mass_fix=1)
    rl, st = O.acnn_train(O.params(n, 0.03, 0.0, 5e-3, 1), spec, U0s, perm, 2, 2, 2, lr=2e-3)
    assert np.allclose(losses.cpu().numpy(), rl, rtol=1e-9, atol=0)
    assert np.abs(net.w.cpu().numpy() - spec.w).max() < 1e-9
    assert np.abs(net.b.cpu().numpy() - spec.b).max() < 1e-9
    assert net.t == st["t"] == 16


def test_algorithm1_f32_lowers_the_loss():
    """float32 training at 64^2: the scheme loss of the last updates is below
    that of the first ones."""
    C, R, n = 4, 2, 64
    w, b = I.acnn_weights(C, R, seed=12)
    U0s = torch.tensor(_fields(n, 8, 700, zero_mean=True), dtype=torch.float32, device="cuda")
    perm = np.stack([np.random.default_rng(e).permutation(8) for e in range(3)])
    p = G.FineParams(n, 0.03, 0.0, 5e-3, variant=1, precision=F32)
    net = G.Acnn(C, R, w, b, mass_fix=1, precision=F32)
    losses = net.train_alg1(p, U0s, perm, q=4, steps=3, b_inner=4, lr=3e-3).cpu().numpy()
    assert np.isfinite(losses).all()
    assert losses[-8:].mean() < 0.5 * losses[:8].mean()


def test_parareal_with_acnn_matches_oracle_f64():
    """Algorithm 2 with the ACNN as G (mACNN, 64^2, 6 slices of 40 steps): the
    k = 0 sweep and three iterations match the oracle's to 1e-10; at k = s the
    trajectory is the GPU's sequential fine solve bit for bit."""
    C, R, n, s, c = 4, 2, 64, 6, 40
    w, b = I.acnn_weights(C, R, seed=13)
    w, b = 0.3 * w, 0.3 * b
    fp = G.FineParams(n, 0.04, 2.0, 1e-4, variant=1, precision=F64)
    u0 = _fields(n, 2, 800, zero_mean=True)
    net = G.Acnn(C, R, w, b, mass_fix=1, precision=F64)
    pr = G.Parareal(fp, net, torch.tensor(u0, device="cuda"), s, c)
    pr.iterate()
    spec = O.AcnnSpec(C, R, w, b, mass_fix=1)
    po = O.params(n, 0.04, 2.0, 1e-4, 1)
    ref0 = O.parareal(po, spec, s, c, kmax=0, tol=0.0, u0=u0[1])
    assert np.abs(pr.trajectory()[1].cpu().numpy() - ref0["U"]).max() < 1e-10
    for _ in range(3):
        pr.iterate()
    ref = O.parareal(po, spec, s, c, kmax=3, tol=0.0, u0=u0[1])
    assert np.abs(pr.trajectory()[1].cpu().numpy() - ref["U"]).max() < 1e-10
    for _ in range(s - 3):
        pr.iterate()
    seq = [torch.tensor(u0, device="cuda")]
    for _ in range(s):
        seq.append(G.ac_fine_propagate_slices(fp, c, seq[-1]))
    assert torch.equal(pr.trajectory(), torch.stack(seq, 1))


def test_parareal_with_acnn_f32_graphs_and_switching():
    """float32 with CUDA graphs: the k = 0 sweep is the net's rollout bit for
    bit, exactness at k = s holds, and a handle created with the conv stack can
    switch to the ACNN and back."""
    n, s, c = 128, 4, 20
    fp = G.FineParams(n, 0.04, 2.0, 1e-4, variant=1, precision=F32)
    w, b = I.acnn_weights(4, 2, seed=14)
    net = G.Acnn(4, 2, 0.3 * w, 0.3 * b, mass_fix=1, precision=F32)
    u0 = torch.tensor(_fields(n, 3, 900, zero_mean=True), dtype=torch.float32, device="cuda")
    pr = G.Parareal(fp, net, u0, s, c)
    pr.enable_graphs(True)
    pr.iterate()
    roll = u0
    for j in range(s):
        roll = net(roll)
        assert torch.equal(pr.trajectory()[:, j + 1], roll)
    its, _ = pr.solve(tol=0.0, kmax=s)
    seq = [u0]
    for _ in range(s):
        seq.append(G.ac_fine_propagate_slices(fp, c, seq[-1]))
    assert torch.equal(pr.trajectory(), torch.stack(seq, 1))
    cw, cb = I.cnn_weights(4, 16, seed=0)
    cnet = G.CoarseNet(4, 16, cw.astype(np.float32), cb.astype(np.float32), act=0, precision=F32)
    pc = G.Parareal(fp, cnet, u0, s, c)
    pc.set_coarse_acnn(net)
    pc.iterate()
    assert torch.equal(pc.trajectory()[:, 1], net(u0))
    pc.set_coarse_acnn(None)
    pc.reset(u0)
    pc.iterate()
    assert torch.equal(pc.trajectory()[:, 1], G.cnn_coarse_step(cnet, u0))
