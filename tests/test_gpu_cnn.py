"""GPU parity of the coarse propagator (cnn_coarse_step) against the oracle.

float64 mode: 1e-12 max-abs (the same arithmetic up to summation order and
libm vs CUDA tanh/erf ulps).
bf16 mode: compared with the oracle's bf16-emulating mode (weights, conv input
and hidden activations rounded to bf16, everything else float64).  The kernel
accumulates in float32 and so may round an activation to the neighbouring bf16
value (a relative change of 2^-8 in that activation); with weights of size
sigma the effect on the output is of order 2^-8 * sigma * |activation| per
flip, so the test allows 2e-3 * sigma-scaled max-abs and checks that the
median error is at float32 level.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import acpr_inputs as I
import oracle as O
import paper_2510_07672_gb300 as G

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,L,C,act", [(64, 4, 16, 0), (32, 3, 5, 1), (16, 2, 1, 0)])
def test_cnn_f64(n, L, C, act):
    w, b = I.cnn_weights(L, C, seed=1, sigma=0.3)
    u = np.stack([I.random_field(n, seed=s) for s in range(3)])
    net = G.CoarseNet(L, C, w, b, act=act, precision=G.AC_F64)
    got = G.cnn_coarse_step(net, torch.tensor(u, device="cuda")).cpu().numpy()
    spec = O.CnnSpec(L, C, w, b, act=act)
    ref = O.cnn_forward(spec, u)
    assert np.abs(got - ref).max() < 1e-12


@pytest.mark.parametrize("n,L,C,act,sigma", [(64, 6, 32, 1, 0.1), (32, 4, 16, 0, 0.2), (16, 8, 64, 1, 0.05),
                                             (256, 6, 32, 1, 0.01)])
def test_cnn_bf16(n, L, C, act, sigma):
    w, b = I.cnn_weights(L, C, seed=2, sigma=sigma)
    u = np.stack([I.random_field(n, seed=s) for s in range(2)]).astype(np.float32)
    w32, b32 = w.astype(np.float32), b.astype(np.float32)
    net = G.CoarseNet(L, C, w32, b32, act=act, precision=G.AC_F32)
    got = G.cnn_coarse_step(net, torch.tensor(u, device="cuda")).double().cpu().numpy()
    spec = O.CnnSpec(L, C, w32.astype(np.float64), b32.astype(np.float64), act=act, bf16=1)
    ref = O.cnn_forward(spec, u.astype(np.float64))
    err = np.abs(got - ref)
    scale = max(np.abs(ref - u).max(), 1e-3)  # size of the stack's contribution
    assert err.max() < 2e-2 * scale + 1e-6
    assert np.median(err) < 1e-3 * scale + 1e-7


def test_cnn_mass_fix_and_limiter_f64():
    n, L, C = 32, 3, 4
    w, b = I.cnn_weights(L, C, seed=5, sigma=0.5)
    u = I.random_field(n, seed=1)[None]
    net = G.CoarseNet(L, C, w, b, act=0, precision=G.AC_F64, mass_fix=1, limiter=1, lo=-0.6, hi=0.6)
    got = G.cnn_coarse_step(net, torch.tensor(u, device="cuda")).cpu().numpy()
    ref = O.cnn_forward(O.CnnSpec(L, C, w, b, act=0, mass_fix=1, limiter=1, lo=-0.6, hi=0.6), u[0])
    assert np.abs(got[0] - ref).max() < 1e-12


def test_cnn_deterministic():
    """Same input, same output bits (no atomics): needed for the exactness of
    Parareal (U^k_k equals the fine result bitwise)."""
    n, L, C = 64, 6, 32
    w, b = I.cnn_weights(L, C, seed=3, sigma=0.05)
    net = G.CoarseNet(L, C, w.astype(np.float32), b.astype(np.float32), act=1, precision=G.AC_F32)
    u = torch.tensor(I.random_field(n, 0)[None].repeat(4, 0), dtype=torch.float32, device="cuda")
    a = G.cnn_coarse_step(net, u)
    bb = G.cnn_coarse_step(net, u)
    assert torch.equal(a, bb)
    assert torch.equal(a[0], a[3])


def test_cnn_bf16_partition_independent():
    """The persistent tensor-core kernel (n >= 128) splits row blocks over
    CTAs by the batch size; a field's result must not depend on the split."""
    n, L, C = 256, 6, 32
    w, b = I.cnn_weights(L, C, seed=4, sigma=0.05)
    net = G.CoarseNet(L, C, w.astype(np.float32), b.astype(np.float32), act=1, precision=G.AC_F32)
    u = torch.tensor(np.stack([I.random_field(n, seed=s) for s in range(5)]), dtype=torch.float32, device="cuda")
    many = G.cnn_coarse_step(net, u)
    for i in (0, 3):
        assert torch.equal(G.cnn_coarse_step(net, u[i:i + 1].contiguous())[0], many[i])


@pytest.mark.parametrize("n,L,C", [(128, 4, 32), (128, 3, 64), (512, 4, 16), (256, 3, 64), (256, 4, 32)])
def test_cnn_bf16_persistent_shapes(n, L, C):
    """The persistent row-streaming kernel for every channel count (TMEM slots
    of 64, 128 and 256 columns), one, two or four 128-column blocks, with and
    without the fused last layer, against the oracle's bf16-emulating mode,
    with weights large enough (sigma 0.05) that the stack's output depends on
    its input."""
    w, b = I.cnn_weights(L, C, seed=6, sigma=0.05)
    u = np.stack([I.random_field(n, seed=s) for s in range(2)]).astype(np.float32)
    w32, b32 = w.astype(np.float32), b.astype(np.float32)
    net = G.CoarseNet(L, C, w32, b32, act=1, precision=G.AC_F32)
    got = G.cnn_coarse_step(net, torch.tensor(u, device="cuda")).double().cpu().numpy()
    ref = O.cnn_forward(O.CnnSpec(L, C, w32.astype(np.float64), b32.astype(np.float64), act=1, bf16=1),
                        u.astype(np.float64))
    err = np.abs(got - ref)
    scale = max(np.abs(ref - u).max(), 1e-3)
    assert err.max() < 2e-2 * scale + 1e-6
    assert np.median(err) < 1e-3 * scale + 1e-7


def test_gelu_activation_error_bound():
    """float32 GELU x Phi(x) with Phi from Abramowitz & Stegun 7.1.26 (error
    <= 1.5e-7 in erfc).  A 1 -> 16 -> 1 stack without residual whose first
    layer copies bf16(u) into channel 0 and whose last layer reads channel 0
    back gives out = bf16(GELU(bf16(u))).  It must be the correctly rounded
    bf16 of the exact GELU, or a neighbouring bf16 value where the exact value
    lies within the approximation's error of a rounding midpoint."""
    from math import erf, sqrt
    n, L, C = 64, 2, 16
    w = np.zeros(C * 9 + C * 9)
    w[4] = 1.0                      # layer 1, out channel 0, centre tap
    w[C * 9 + 4] = 1.0              # layer 2, in channel 0, centre tap
    b = np.zeros(C + 1)
    net = G.CoarseNet(L, C, w.astype(np.float32), b.astype(np.float32), act=1, precision=G.AC_F32, residual=0)
    u = np.linspace(-7.0, 5.0, n * n).reshape(1, n, n).astype(np.float32)
    got = G.cnn_coarse_step(net, torch.tensor(u, device="cuda")).cpu().numpy().astype(np.float64)
    ub = torch.tensor(u).to(torch.bfloat16).double().numpy()
    exact = np.vectorize(lambda x: 0.5 * x * (1.0 + erf(x / sqrt(2.0))))(ub)
    ref = torch.tensor(exact).to(torch.bfloat16).double().numpy()
    ulp = np.maximum(np.abs(ref), 1e-30) * 2.0 ** -7
    err = np.abs(got - ref)
    exact_hit = err <= 1e-7 + 1e-6 * np.abs(ref)
    assert np.all(exact_hit | (err <= ulp * 1.01))
    # one-step flips are rare (about 1% of this ramp, measured)
    assert np.mean(exact_hit) > 0.98


def test_gelu_activation_error_bound_hidden_layer():
    """The paired-instruction GELU of the hidden tensor-core layer (the same
    Abramowitz & Stegun 7.1.26 form, written as max(x, 0) - |x| Phi(-|x|)):
    a 1 -> 32 -> 32 -> 1 stack at 128^2 whose first layer copies bf16(u) into
    channel 0, whose hidden layer copies channel 0 (centre tap) and whose
    fused last layer reads channel 0 back gives
    out = bf16(GELU(bf16(GELU(bf16(u))))).  Each stage must be the correctly
    rounded bf16 of the exact GELU or, where the exact value lies within the
    approximation's error of a rounding midpoint, a neighbouring bf16 value."""
    from math import erf, sqrt
    n, L, C = 128, 3, 32
    w = np.zeros(C * 9 + C * C * 9 + C * 9)
    w[4] = 1.0                              # first layer, out channel 0, centre tap
    w[C * 9 + 4] = 1.0                      # hidden layer, out 0 <- in 0, centre tap
    w[C * 9 + C * C * 9 + 4] = 1.0          # last layer, in channel 0, centre tap
    b = np.zeros(C + C + 1)
    net = G.CoarseNet(L, C, w.astype(np.float32), b.astype(np.float32), act=1, precision=G.AC_F32, residual=0)
    u = np.linspace(-7.0, 5.0, n * n).reshape(1, n, n).astype(np.float32)
    got = G.cnn_coarse_step(net, torch.tensor(u, device="cuda")).cpu().numpy().astype(np.float64)
    gelu = np.vectorize(lambda x: 0.5 * x * (1.0 + erf(x / sqrt(2.0))))
    bf = lambda x: torch.tensor(x).to(torch.bfloat16).double().numpy()
    ref = bf(gelu(bf(gelu(bf(u)))))
    ulp = np.maximum(np.abs(ref), 1e-30) * 2.0 ** -7
    err = np.abs(got - ref)
    exact_hit = err <= 1e-7 + 1e-6 * np.abs(ref)
    # a flip in the first stage moves the second by about one ulp as well
    assert np.all(exact_hit | (err <= ulp * 1.2))
    assert np.mean(exact_hit) > 0.96


def test_cnn_bf16_mass_shift_trained_256():
    """The coarse net exactly as the benchmark runs it: the committed trained
    1 -> 32 x 6 GELU stack, bf16 with float32 accumulation and the mACNN mass
    shift (Sec. 3.2), on 256^2 zero-mean fields.  Against the oracle's
    bf16-emulating mode with the same shift: the tolerance of the bf16 tests
    above (bf16 rounding flips bounded by 2e-2 of the stack's contribution,
    median at float32 level); the shift keeps the output's mean equal to the
    input's, up to float32 summation over 65536 values."""
    import os
    W = I.MASS_F32_256
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    z = np.load(os.path.join(root, "paper_2510_07672_gb300", "weights", "mass256_c32l6_gelu.npz"))
    w32, b32 = z["w"].astype(np.float32), z["b"].astype(np.float32)
    net = G.CoarseNet(W.layers, W.channels, w32, b32, act=W.act, precision=G.AC_F32, mass_fix=1)
    u = W.ics()[:2].astype(np.float32)
    got = G.cnn_coarse_step(net, torch.tensor(u, device="cuda")).double().cpu().numpy()
    spec = O.CnnSpec(W.layers, W.channels, w32.astype(np.float64), b32.astype(np.float64), act=W.act,
                     mass_fix=1, bf16=1)
    with O.threads(os.cpu_count() or 1):
        ref = O.cnn_forward(spec, u.astype(np.float64))
    err = np.abs(got - ref)
    scale = max(np.abs(ref - u).max(), 1e-3)
    assert err.max() < 2e-2 * scale + 1e-6
    assert np.median(err) < 1e-3 * scale + 1e-7
    for p in range(2):
        assert abs(got[p].mean() - u[p].astype(np.float64).mean()) < 1e-6


def test_bounded_wait_timeout_is_reported_and_cleared():
    """Failure detection without a fault: the test hook makes the persistent
    tensor-core kernel's MMA issuer wait on an mbarrier that nothing arrives
    on, with a short poll limit.  The kernel gives up, drains its copies,
    frees its tensor memory and stores the code in the workspace status word;
    cnn_coarse_step reports AC_ERR_TIMEOUT and clears the word, and the next
    call (hook off) is correct again: equal to a fresh net's output."""
    n, L, C = 256, 4, 32
    w, b = I.cnn_weights(L, C, seed=7, sigma=0.05)
    w32, b32 = w.astype(np.float32), b.astype(np.float32)
    net = G.CoarseNet(L, C, w32, b32, act=1, precision=G.AC_F32)
    u = torch.tensor(np.stack([I.random_field(n, seed=s) for s in range(2)]), dtype=torch.float32, device="cuda")
    G.ac_test_conv_stall(2000)
    try:
        with pytest.raises(G.AcprError, match="AC_ERR_TIMEOUT"):
            G.cnn_coarse_step(net, u)
    finally:
        G.ac_test_conv_stall(0)
    G.ac_conv_status(net._work)  # cleared: no error now
    got = G.cnn_coarse_step(net, u)
    ref = G.cnn_coarse_step(G.CoarseNet(L, C, w32, b32, act=1, precision=G.AC_F32), u)
    assert torch.equal(got, ref)


@pytest.mark.parametrize("n,C", [(256, 32), (128, 64)])
def test_conv_tile_shapes_identical_and_autotune(n, C):
    """Every shape of the persistent row-streaming tensor-core kernel (input
    ring depth, TMEM slots) forms each output with the same sums in the same
    order, so G is bitwise the same under every shape; cnn_autotune times them
    all and keeps the fastest."""
    L = 6
    w, b = I.cnn_weights(L, C, seed=9, sigma=0.05)
    net = G.CoarseNet(L, C, w.astype(np.float32), b.astype(np.float32), act=1, precision=G.AC_F32, mass_fix=1)
    u = torch.tensor(np.stack([I.random_field(n, seed=s) for s in range(3)]), dtype=torch.float32, device="cuda")
    shapes = G.cnn_conv_variants(n, C)
    assert len(shapes) >= 2
    outs = []
    for i in range(len(shapes)):
        G.cnn_conv_set_variant(n, C, i)
        outs.append(G.cnn_coarse_step(net, u))
    G.cnn_conv_set_variant(n, C, -1)
    for i in range(1, len(shapes)):
        assert torch.equal(outs[i], outs[0]), shapes[i]
    times, best = G.cnn_autotune(net, u)
    assert len(times) == len(shapes) and all(t > 0 for t in times.values())
    assert times[shapes[best]] == min(times.values())
    assert torch.equal(G.cnn_coarse_step(net, u), outs[0])
    G.cnn_conv_set_variant(n, C, -1)
