"""Pins of the oracle's ResBlock ACNN / mACNN, the scheme-residual loss
(Eq. loss_ACN), Adam and Algorithm 1 (Sec. 3.2) against facts fixed by the
paper and by mathematics.  None of these call the CUDA path."""
import numpy as np
import pytest

import acpr_inputs as I
import oracle as O


def rng(seed):
    return np.random.default_rng(seed)


def _split(C, R, w, b):
    """Per-conv views of the concatenated parameters."""
    out, ow, ob = [], 0, 0
    for ci, co in I.acnn_layer_dims(C, R):
        out.append((w[ow:ow + ci * co * 9], b[ob:ob + co]))
        ow += ci * co * 9
        ob += co
    return out


def test_param_counts():
    """C = 4, two blocks (the paper's light model): 36 + 4*144 + 36 weights, 4 + 4*4 + 1 biases."""
    assert O.acnn_param_counts(4, 2) == (36 + 4 * 144 + 36, 4 + 16 + 1)
    w, b = I.acnn_weights(4, 2, seed=0)
    assert (w.size, b.size) == O.acnn_param_counts(4, 2)


def test_identity_blocks_reduce_to_plain_stack():
    """Blocks with zero conv2 weights and biases add tanh(0) = 0: the ACNN is then
    the two-conv stack tanh(conv_in) -> conv_out without global residual, which
    the (separately pinned) plain conv-stack oracle computes."""
    C, R, n = 4, 2, 12
    w, b = I.acnn_weights(C, R, seed=1)
    parts = _split(C, R, w, b)
    for r in range(R):
        parts[2 + 2 * r][0][:] = 0.0
        parts[2 + 2 * r][1][:] = 0.0
    spec = O.AcnnSpec(C, R, w, b)
    plain = O.CnnSpec(2, C, np.concatenate([parts[0][0], parts[-1][0]]),
                      np.concatenate([parts[0][1], parts[-1][1]]), act=0, residual=0)
    u = I.random_field(n, seed=3)
    assert np.abs(O.acnn_forward(spec, u) - O.cnn_forward(plain, u)).max() < 1e-14


def test_skip_connection_adds_block_output():
    """With conv2 weights zero and bias beta, a block adds the constant
    tanh(beta_c) to channel c; the output conv then sees a0 + sum_r tanh(beta_r),
    the plain stack with output bias b_out + sum_c (sum_r tanh(beta_rc)) sum_taps W_out[c]."""
    C, R, n = 4, 2, 10
    w, b = I.acnn_weights(C, R, seed=2)
    parts = _split(C, R, w, b)
    shift = np.zeros(C)
    for r in range(R):
        parts[2 + 2 * r][0][:] = 0.0
        parts[2 + 2 * r][1][:] = 0.3 * (r + 1) * np.arange(1, C + 1) / C
        shift += np.tanh(parts[2 + 2 * r][1])
    spec = O.AcnnSpec(C, R, w, b)
    wout = parts[-1][0].reshape(C, 9)
    bout = parts[-1][1] + (shift * wout.sum(axis=1)).sum()
    plain = O.CnnSpec(2, C, np.concatenate([parts[0][0], parts[-1][0]]),
                      np.concatenate([parts[0][1], bout]), act=0, residual=0)
    u = I.random_field(n, seed=4)
    assert np.abs(O.acnn_forward(spec, u) - O.cnn_forward(plain, u)).max() < 1e-13


def test_translation_equivariance_mass_shift_and_limiter():
    """Circular convolutions commute with periodic shifts; the mACNN shift makes
    mean(out) = mean(u); the limiter keeps out in [lo, hi]."""
    C, R, n = 4, 2, 16
    w, b = I.acnn_weights(C, R, seed=5)
    u = I.random_field(n, seed=6)
    spec = O.AcnnSpec(C, R, w, b, mass_fix=1)
    out = O.acnn_forward(spec, u)
    assert abs(out.mean() - u.mean()) < 1e-15
    sh = O.acnn_forward(spec, np.roll(u, (3, -5), axis=(0, 1)))
    assert np.abs(sh - np.roll(out, (3, -5), axis=(0, 1))).max() < 1e-14
    lim = O.AcnnSpec(C, R, w * 3, b * 3, mass_fix=1, limiter=1, lo=-0.2, hi=0.25)
    o2 = O.acnn_forward(lim, u)
    assert o2.min() >= -0.2 and o2.max() <= 0.25 and (o2 == 0.25).any()


@pytest.mark.parametrize("mass_fix", [0, 1])
def test_backward_finite_differences(mass_fix):
    """dJ/dW and dJ/db for J = <gout, ACNN(u)> against central differences in
    random directions (limiter on, but inactive at these values)."""
    C, R, n, batch = 4, 2, 8, 2
    w, b = I.acnn_weights(C, R, seed=7)
    u = np.stack([I.random_field(n, seed=8 + p) for p in range(batch)])
    gout = rng(1).standard_normal(u.shape)

    def J(ww, bb):
        return np.vdot(gout, O.acnn_forward(O.AcnnSpec(C, R, ww, bb, mass_fix=mass_fix, limiter=1,
                                                       lo=-50.0, hi=50.0), u))

    gw, gb = O.acnn_backward(O.AcnnSpec(C, R, w, b, mass_fix=mass_fix, limiter=1, lo=-50.0, hi=50.0), u, gout)
    hh = 1e-6
    for seed in range(3):
        dw = rng(10 + seed).standard_normal(w.shape)
        db = rng(20 + seed).standard_normal(b.shape)
        fd = (J(w + hh * dw, b) - J(w - hh * dw, b)) / (2 * hh)
        assert abs(fd - np.vdot(gw, dw)) < 1e-7 * max(1.0, abs(fd))
        fd = (J(w, b + hh * db) - J(w, b - hh * db)) / (2 * hh)
        assert abs(fd - np.vdot(gb, db)) < 1e-7 * max(1.0, abs(fd))


def test_backward_limiter_blocks_clamped_entries():
    """Where the limiter clamps, the output does not depend on the parameters:
    a gradient placed only on clamped entries gives zero parameter gradient."""
    C, R, n = 4, 1, 8
    w, b = I.acnn_weights(C, R, seed=11)
    u = I.random_field(n, seed=12)
    spec = O.AcnnSpec(C, R, w * 4, b * 4, limiter=1, lo=-0.05, hi=0.05)
    out = O.acnn_forward(spec, u)
    gout = np.where(np.abs(out) >= 0.05, 1.0, 0.0)
    assert gout.sum() > 0
    gw, gb = O.acnn_backward(spec, u, gout)
    assert np.abs(gw).max() == 0.0 and np.abs(gb).max() == 0.0


@pytest.mark.parametrize("variant", [0, 1])
def test_loss_vanishes_on_the_crank_nicolson_step(variant):
    """Eq. loss_ACN is the squared residual of the fully discrete scheme
    (Eq. fully-discrete, Sec. 3.1): it vanishes at the scheme's own solution
    U1 = F(U0) (the separately pinned Crank-Nicolson + Picard oracle, iterated
    to 1e-14), and not at U1 = U0."""
    n = 16
    p = O.params(n, eps=0.05, S=0.0, dt=2e-3, variant=variant)
    U0 = np.stack([I.random_field(n, seed=s, zero_mean=bool(variant)) for s in (30, 31)])
    U1 = np.stack([O.cn_step(p, u, tol=1e-15, maxit=200)[0] for u in U0])
    loss, _ = O.loss_acn(p, U0, U1)
    assert loss < 1e-27
    far, _ = O.loss_acn(p, U0, U0)
    assert far > 1e-8


@pytest.mark.parametrize("variant", [0, 1])
def test_loss_gradient_finite_differences(variant):
    n = 8
    p = O.params(n, eps=0.08, S=0.0, dt=5e-3, variant=variant)
    U0 = np.stack([I.random_field(n, seed=s) for s in (40, 41)])
    U1 = U0 + 0.1 * rng(2).standard_normal(U0.shape)
    _, g = O.loss_acn(p, U0, U1)
    hh = 1e-6
    for seed in range(3):
        d = rng(50 + seed).standard_normal(U1.shape)
        fd = (O.loss_acn(p, U0, U1 + hh * d, grad=False)[0] - O.loss_acn(p, U0, U1 - hh * d, grad=False)[0]) / (2 * hh)
        assert abs(fd - np.vdot(g, d)) < 1e-7 * max(1e-3, abs(fd))


def test_adam_first_step_closed_form():
    """From zero moments, step 1 moves every parameter by -lr g / (|g| + eps)
    (the bias corrections cancel), and step 2 with the same g again by the same amount."""
    w = np.array([0.5, -1.0, 2.0])
    g = np.array([0.3, -2e-3, 0.0])
    m, v = np.zeros(3), np.zeros(3)
    w0 = w.copy()
    O.adam(w, g, m, v, 1e-2, 0.9, 0.999, 1e-8, 1)
    assert np.allclose(w - w0, -1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    w1 = w.copy()
    O.adam(w, g, m, v, 1e-2, 0.9, 0.999, 1e-8, 2)
    assert np.allclose(w - w1, -1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-10, atol=0)


def test_algorithm1_data_flow_with_zero_learning_rate():
    """lr = 0 leaves G fixed, so Algorithm 1's updates walk each subset along G's
    own rollout: the loss of update (step j, inner k) is the loss of the pair
    (G^j(U0), G^{j+1}(U0)) for that subset, the same for every k."""
    C, R, n = 4, 1, 8
    w, b = I.acnn_weights(C, R, seed=13)
    spec = O.AcnnSpec(C, R, w, b, mass_fix=1)
    p = O.params(n, eps=0.08, S=0.0, dt=1e-2, variant=1)
    U0s = np.stack([I.random_field(n, seed=60 + i, zero_mean=True) for i in range(4)])
    perm = np.array([[2, 0, 3, 1]])
    q, steps, b_in = 2, 3, 2
    losses, st = O.acnn_train(p, spec, U0s, perm, q, steps, b_in, lr=0.0)
    assert st["t"] == 2 * steps * b_in
    li = 0
    for sub in range(2):
        U = U0s[perm[0, sub * q:(sub + 1) * q]]
        for j in range(steps):
            U1 = O.acnn_forward(spec, U)
            ref, _ = O.loss_acn(p, U, U1, grad=False)
            for k in range(b_in):
                assert losses[li] == ref
                li += 1
            U = U1


def test_algorithm1_lowers_the_scheme_loss():
    """A short run of Algorithm 1 lowers the loss of a fixed held-out pair."""
    C, R, n = 4, 2, 8
    w, b = I.acnn_weights(C, R, seed=14)
    spec = O.AcnnSpec(C, R, w, b, mass_fix=1)
    p = O.params(n, eps=0.08, S=0.0, dt=1e-2, variant=1)
    U0s = np.stack([I.random_field(n, seed=70 + i, zero_mean=True) for i in range(4)])
    test = I.random_field(n, seed=99, zero_mean=True)
    before = O.loss_acn(p, test, O.acnn_forward(spec, test), grad=False)[0]
    perm = np.array([[0, 1, 2, 3], [3, 2, 1, 0], [1, 3, 0, 2]])
    losses, _ = O.acnn_train(p, spec, U0s, perm, 2, 2, 3, lr=3e-3)
    after = O.loss_acn(p, test, O.acnn_forward(spec, test), grad=False)[0]
    assert after < 0.5 * before
    assert losses[-6:].mean() < losses[:6].mean()


def test_parareal_with_acnn_first_sweep_and_exactness():
    """Algorithm 2 with the ACNN as G: the k = 0 sweep is the network's rollout,
    and at k = s the trajectory is the sequential fine solve (Sec. 3.3)."""
    C, R, n, s, c = 4, 2, 16, 5, 4
    w, b = I.acnn_weights(C, R, seed=15)
    spec = O.AcnnSpec(C, R, w, b, mass_fix=1)
    p = O.params(n, eps=0.05, S=2.0, dt=2e-3, variant=1)
    u0 = I.random_field(n, seed=16, zero_mean=True)
    r0 = O.parareal(p, spec, s, c, kmax=0, tol=0.0, u0=u0)
    u = u0
    for j in range(s):
        u = O.acnn_forward(spec, u)
        assert np.array_equal(r0["U"][j + 1], u)
    r = O.parareal(p, spec, s, c, kmax=s, tol=0.0, u0=u0)
    seq = [u0]
    for j in range(s):
        seq.append(O.fine_propagate(p, c, seq[-1]))
    assert np.array_equal(r["U"], np.stack(seq))
    assert r["g_calls"] == (2 * s - s) * (s + 1) // 2
