"""GPU parity of the coarse-propagator training path (cnn_forward_train,
cnn_backward, cnn_adam_step, mse_loss_grad) against the oracle.

The oracle's backward in bf16 mode uses the forward's rounded weights and
layer inputs (straight-through); the kernels additionally round each layer's
pre-activation gradient to bf16 before it enters a product (relative error
2^-9 per value) and accumulate in float32.  Over a few layers that gives
gradients within about 1e-2 of the oracle in relative L2 norm, the tolerance
used here.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import acpr_inputs as I
import oracle as O
import paper_2510_07672_gb300 as G

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("n,L,C,act,mass_fix", [(32, 4, 16, 1, 0), (16, 3, 32, 0, 0), (64, 5, 32, 1, 0),
                                                (32, 4, 16, 1, 1), (128, 4, 64, 1, 1)])
def test_backward_matches_oracle(n, L, C, act, mass_fix):
    w, b = I.cnn_weights(L, C, seed=7, sigma=0.25)
    w, b = w.astype(np.float32), b.astype(np.float32)
    batch = 2
    u = np.stack([I.random_field(n, seed=s) for s in range(batch)]).astype(np.float32)
    g = np.random.default_rng(1).standard_normal((batch, n, n)).astype(np.float32)
    net = G.TrainableCoarseNet(L, C, w, b, act=act, mass_fix=mass_fix)
    ws = net.new_workspace(n, batch)
    U = torch.tensor(u, device="cuda")
    out = net.forward_train(U, ws)
    # forward_train is the inference forward, bit for bit
    assert torch.equal(out, G.cnn_coarse_step(net, U))
    du = torch.empty_like(U)
    net.backward(U, torch.tensor(g, device="cuda"), ws, grad_in=du)
    spec = O.CnnSpec(L, C, w.astype(np.float64), b.astype(np.float64), act=act, bf16=1, mass_fix=mass_fix)
    gw_ref = np.zeros(w.size)
    gb_ref = np.zeros(b.size)
    du_ref = np.zeros((batch, n, n))
    for i in range(batch):
        gi, gw, gb = O.cnn_backward(spec, u[i].astype(np.float64), g[i].astype(np.float64))
        du_ref[i] = gi
        gw_ref += gw
        gb_ref += gb
    assert rel(du.double().cpu().numpy() - g, du_ref - g) < 1e-2
    assert rel(net.gw.double().cpu().numpy(), gw_ref) < 1e-2
    assert rel(net.gb.double().cpu().numpy(), gb_ref) < 1e-2


def test_backward_accumulates_and_is_deterministic():
    n, L, C = 32, 4, 16
    w, b = I.cnn_weights(L, C, seed=3, sigma=0.2)
    net = G.TrainableCoarseNet(L, C, w.astype(np.float32), b.astype(np.float32), act=1)
    U = torch.tensor(I.random_field(n, 2)[None], dtype=torch.float32, device="cuda")
    g = torch.ones_like(U)
    ws = net.new_workspace(n, 1)
    net.forward_train(U, ws)
    net.backward(U, g, ws)
    gw1 = net.gw.clone()
    net.backward(U, g, ws)
    assert torch.equal(net.gw, gw1)
    net.backward(U, g, ws, accumulate=True)
    assert torch.equal(net.gw, 2 * gw1)


def test_adam_step_matches_formula():
    rng = np.random.default_rng(0)
    w0 = rng.standard_normal(1000).astype(np.float32)
    g = rng.standard_normal(1000).astype(np.float32)
    net = G.TrainableCoarseNet(3, 16, np.zeros(16 * 9 * 2 + 16 * 16 * 9, np.float32), np.zeros(33, np.float32))
    W = torch.tensor(w0, device="cuda")
    Gr = torch.tensor(g, device="cuda")
    m = torch.zeros_like(W)
    v = torch.zeros_like(W)
    L = G.load()
    from paper_2510_07672_gb300.abi import _dev, _stream
    wr, mr, vr = w0.astype(np.float64), np.zeros(1000), np.zeros(1000)
    for t in (1, 2, 3):
        assert L.cnn_adam_step(_dev(W), _dev(Gr), _dev(m), _dev(v), 1000, 1e-3, 0.9, 0.999, 1e-8, t, _stream(None)) == 0
        mr = 0.9 * mr + 0.1 * g
        vr = 0.999 * vr + 0.001 * g.astype(np.float64) ** 2
        wr = wr - 1e-3 * (mr / (1 - 0.9 ** t)) / (np.sqrt(vr / (1 - 0.999 ** t)) + 1e-8)
    assert np.abs(W.double().cpu().numpy() - wr).max() < 1e-5
    del net


def test_mse_loss_grad():
    rng = np.random.default_rng(4)
    p = rng.standard_normal(5000).astype(np.float32)
    t = rng.standard_normal(5000).astype(np.float32)
    P, T = torch.tensor(p, device="cuda"), torch.tensor(t, device="cuda")
    grad = torch.empty_like(P)
    loss = G.mse_loss_grad(P, T, 0.5, grad=grad)
    d = p.astype(np.float64) - t
    assert abs(loss.item() - 0.5 * (d ** 2).sum()) < 1e-9 * (d ** 2).sum()
    assert np.abs(grad.cpu().numpy() - (2 * 0.5 * d)).max() < 1e-6


def test_autograd_function_matches_manual_backward():
    n, L, C = 32, 4, 16
    w, b = I.cnn_weights(L, C, seed=5, sigma=0.2)
    net = G.TrainableCoarseNet(L, C, w.astype(np.float32), b.astype(np.float32), act=1)
    Fn = G.coarse_step_function()
    U = torch.tensor(I.random_field(n, 1)[None], dtype=torch.float32, device="cuda", requires_grad=True)
    Wt = net.w.clone().requires_grad_(True)
    Bt = net.b.clone().requires_grad_(True)
    out = Fn.apply(U, Wt, Bt, net)
    gout = torch.randn_like(out)
    out.backward(gout)
    ws = net.new_workspace(n, 1)
    net.forward_train(U.detach(), ws)
    du = torch.empty_like(U)
    net.backward(U.detach(), gout, ws, grad_in=du)
    assert torch.equal(U.grad, du)
    assert torch.equal(Wt.grad, net.gw)
    assert torch.equal(Bt.grad, net.gb)


def test_training_reduces_one_slice_error():
    """A short run on 64^2 mass-conserving trajectories: the trained G's
    one-slice error falls well below the untrained G's (which is about the
    identity), on held-out initial data."""
    from paper_2510_07672_gb300.train import make_trajectories, train_coarse
    n, S, c = 64, 8, 100
    fp = G.FineParams(n, 0.04, 2.0, 5e-5, variant=1, precision=G.AC_F32)
    mk = lambda seeds: torch.tensor(np.stack([I.random_field(n, seed=s, zero_mean=True) for s in seeds]),
                                    dtype=torch.float32, device="cuda")
    traj = make_trajectories(fp, mk(range(100, 116)), S, c)
    test = make_trajectories(fp, mk(range(200, 204)), S, c)
    w, b = I.cnn_weights(4, 16, seed=0)
    net = G.TrainableCoarseNet(4, 16, w.astype(np.float32), b.astype(np.float32), act=1)

    def err():
        x = test[:, :-1].reshape(-1, n, n).contiguous()
        y = test[:, 1:].reshape(-1, n, n)
        return (torch.linalg.norm(G.cnn_coarse_step(net, x) - y) / torch.linalg.norm(y)).item()

    e0 = err()
    losses = train_coarse(net, traj, iters=300, batch=8, unroll=2, lr=3e-3, seed=1)
    e1 = err()
    assert losses[-1] < 0.5 * losses[0]
    assert e1 < 0.5 * e0, (e0, e1)


def test_weight_gradient_tensor_cores_match_cuda_cores():
    """The hidden layers' weight gradient on the tensor cores (C = 64, n a
    multiple of 128: per-tap 64 x 64 x 16 MMAs over 16-pixel groups, float32
    sums in TMEM, per-chunk partials) equals the CUDA-core one up to the order
    of the float32 sums, is bitwise repeatable, and leaves every other
    gradient unchanged."""
    n, L, C, batch = 256, 4, 64, 3
    w, b = I.cnn_weights(L, C, seed=11, sigma=0.05)
    u = np.stack([I.random_field(n, seed=s) for s in range(batch)]).astype(np.float32)
    g = np.random.default_rng(2).standard_normal((batch, n, n)).astype(np.float32)
    U, Gt = torch.tensor(u, device="cuda"), torch.tensor(g, device="cuda")
    res = {}
    try:
        for tc in (True, False, True):
            G.cnn_train_set_wgrad_tc(tc)
            net = G.TrainableCoarseNet(L, C, w.astype(np.float32), b.astype(np.float32), act=1, mass_fix=0)
            ws = net.new_workspace(n, batch)
            net.forward_train(U, ws)
            du = torch.empty_like(U)
            net.backward(U, Gt, ws, grad_in=du)
            key = "tc" if tc else "cc"
            if key in res:
                assert torch.equal(res[key][0], net.gw) and torch.equal(res[key][1], net.gb)
            res[key] = (net.gw.clone(), net.gb.clone(), du.clone())
    finally:
        G.cnn_train_set_wgrad_tc(True)
    gw_tc, gb_tc, du_tc = res["tc"]
    gw_cc, gb_cc, du_cc = res["cc"]
    assert torch.equal(du_tc, du_cc)  # the input gradient does not involve the weight gradient
    # first and last layers stay on the CUDA cores: identical
    first = 9 * C
    last = C * 9
    assert torch.equal(gw_tc[:first], gw_cc[:first]) and torch.equal(gw_tc[-last:], gw_cc[-last:])
    rel = ((gw_tc - gw_cc).norm() / gw_cc.norm()).item()
    assert rel < 1e-4, rel
    relb = ((gb_tc - gb_cc).norm() / gb_cc.norm()).item()
    assert relb < 1e-4, relb
