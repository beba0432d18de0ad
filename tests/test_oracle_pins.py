"""Pins of the float64 oracle against facts fixed by the paper and by mathematics.

None of these call the CUDA path.  Each test names the passage or identity it
checks; together they are chosen so that a dropped term, a wrong sign or index,
or a transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.signal
import scipy.special

import acpr_inputs as I
import oracle as O


def rng(seed):
    return np.random.default_rng(seed)


# --------------------------------------------------------------------- FFT
@pytest.mark.parametrize("n", [2, 4, 8, 16])
def test_fft_matches_naive_dft(n):
    """Radix-2 recursion equals the DFT definition, both signs."""
    x = rng(n).standard_normal((n, n)) + 1j * rng(n + 1).standard_normal((n, n))
    for sign in (-1, 1):
        a = O.fft2(x, sign)
        b = O.dft2_naive(x, sign)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("n", [32, 64, 256])
def test_fft_matches_library(n):
    """numpy's pocketfft is an independent implementation of the same DFT."""
    x = rng(3).standard_normal((n, n)) + 1j * rng(4).standard_normal((n, n))
    assert np.abs(O.fft2(x, -1) - np.fft.fft2(x)).max() <= 1e-12 * n * n
    assert np.abs(O.fft2(x, 1) - np.fft.ifft2(x) * n * n).max() <= 1e-12 * n * n


def test_fft_single_mode_is_delta():
    n, k, l = 16, 3, 5
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x = np.exp(2j * np.pi * (k * i + l * j) / n)
    X = O.fft2(x, -1)
    ref = np.zeros((n, n), complex)
    ref[k, l] = n * n
    assert np.abs(X - ref).max() < 1e-10


# ------------------------------------------------------------ linear solve
def dense_laplacian(n, h):
    """Periodic 5-point Laplacian as an explicit n^2 x n^2 matrix."""
    m = n * n
    L = np.zeros((m, m))
    for i in range(n):
        for j in range(n):
            r = i * n + j
            L[r, r] = -4.0 / h ** 2
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                L[r, ((i + di) % n) * n + (j + dj) % n] += 1.0 / h ** 2
    return L


@pytest.mark.parametrize("n", [4, 8])
def test_solve_matches_dense_gaussian_elimination(n):
    """The DFT solve of ((1+S dt) I - dt eps^2 Lap_h) v = r equals a dense solve."""
    p = O.params(n, eps=0.07, S=2.0, dt=3e-3, length=1.0)
    r = rng(n).standard_normal((n, n))
    A = (1 + p.S * p.dt) * np.eye(n * n) - p.dt * p.eps ** 2 * dense_laplacian(n, 1.0 / n)
    v = np.linalg.solve(A, r.ravel()).reshape(n, n)
    assert np.abs(O.solve_A(p, r) - v).max() <= 1e-13 * max(1.0, np.abs(v).max())


@pytest.mark.parametrize("n", [4, 8])
@pytest.mark.parametrize("variant", [0, 1])
def test_step_matches_dense_step(n, variant):
    """Full step against Gaussian elimination, with the mean of f subtracted in
    the mass-conserving variant (Eq. mass_AC_eq, explicit at u^n)."""
    p = O.params(n, eps=0.05, S=2.0, dt=1e-2, variant=variant, length=2.0)
    u = rng(10 + n).uniform(-0.9, 0.9, (n, n))
    f = u - u ** 3
    if variant:
        f = f - f.mean()
    A = (1 + p.S * p.dt) * np.eye(n * n) - p.dt * p.eps ** 2 * dense_laplacian(n, p.length / n)
    v = np.linalg.solve(A, ((1 + p.S * p.dt) * u + p.dt * f).ravel()).reshape(n, n)
    assert np.abs(O.fine_step(p, u) - v).max() <= 1e-13


# ------------------------------------------------------------- closed forms
@pytest.mark.parametrize("a", [-0.7, 0.3, 0.95])
def test_constant_field(a):
    """u = a: Lap_h u = 0, so the classic step gives a + dt f(a)/(1+S dt) and the
    mass-conserving step leaves a unchanged."""
    n = 8
    u = np.full((n, n), a)
    pc = O.params(n, 0.03, 2.0, 0.01, 0)
    pm = O.params(n, 0.03, 2.0, 0.01, 1)
    exp_c = a + pc.dt * (a - a ** 3) / (1 + pc.S * pc.dt)
    assert np.abs(O.fine_step(pc, u) - exp_c).max() < 1e-15
    assert np.abs(O.fine_step(pm, u) - a).max() < 1e-15


def _D(p, k, n):
    h = p.length / n
    return 1 + p.S * p.dt + p.dt * p.eps ** 2 * (4 / h ** 2) * math.sin(math.pi * k / n) ** 2


@pytest.mark.parametrize("variant", [0, 1])
def test_offset_cosine_mode_closed_form(variant):
    """u = a + b cos(theta_i), theta_i = 2 pi k i / n.  By the power-reduction
    identities u^3 splits into modes 0, k, 2k, 3k, each of which the linear
    solve divides by its own symbol D; the mass variant removes the mode-0 part
    of f (its mean), the classic one keeps it."""
    n, k, a, b = 32, 2, 0.2, 0.5
    p = O.params(n, eps=0.04, S=2.0, dt=5e-3, variant=variant)
    i = np.arange(n)
    th = 2 * np.pi * k * i / n
    u = np.repeat((a + b * np.cos(th))[:, None], n, axis=1)
    f0 = a - a ** 3 - 1.5 * a * b ** 2
    f1 = b - 3 * a ** 2 * b - 0.75 * b ** 3
    f2 = -1.5 * a * b ** 2
    f3 = -0.25 * b ** 3
    if variant:
        f0 = 0.0
    c = 1 + p.S * p.dt
    m0 = (c * a + p.dt * f0) / _D(p, 0, n)
    m1 = (c * b + p.dt * f1) / _D(p, k, n)
    m2 = p.dt * f2 / _D(p, 2 * k, n)
    m3 = p.dt * f3 / _D(p, 3 * k, n)
    exp = m0 + m1 * np.cos(th) + m2 * np.cos(2 * th) + m3 * np.cos(3 * th)
    got = O.fine_step(p, u)
    assert np.abs(got - exp[:, None]).max() < 1e-14
    # the field is constant along the second index (no transposition)
    assert np.abs(got - got[:, :1]).max() < 1e-15


def test_orientation_second_axis():
    """The same mode along the second index gives the transposed result."""
    n = 16
    p = O.params(n, 0.05, 2.0, 4e-3, 0)
    u = 0.6 * np.cos(2 * np.pi * 3 * np.arange(n) / n)
    a = O.fine_step(p, np.repeat(u[:, None], n, 1))
    b = O.fine_step(p, np.repeat(u[None, :], n, 0))
    assert np.abs(a - b.T).max() < 1e-15


# ---------------------------------------------------------------- invariants
def test_energy_decreases_classic_and_mass():
    """Both models dissipate E (Sec. 2, Eq. energy); the stabilised scheme with
    S = 2 inherits this step by step (S >= L/2 with |f'| <= 2 on [-1,1])."""
    n = 32
    u0 = I.random_field(n, seed=7)
    for variant in (0, 1):
        p = O.params(n, eps=0.02, S=2.0, dt=1e-3, variant=variant)
        u, e_prev = u0.copy(), O.energy(p, u0)
        for _ in range(40):
            u = O.fine_step(p, u)
            e = O.energy(p, u)
            assert e <= e_prev + 1e-14
            e_prev = e


def test_maximum_bound_principle_classic():
    """|u0| <= 1 implies |u^n| <= 1 for the classic model (Sec. 2, MBP) when
    1 + (S - 2) dt >= 0."""
    n = 32
    p = O.params(n, eps=0.01, S=2.0, dt=0.05, variant=0)
    u = I.random_field(n, seed=3, amp=1.0)
    for _ in range(30):
        u = O.fine_step(p, u)
        assert np.abs(u).max() <= 1.0 + 1e-12


def test_mass_conservation():
    """M(t) = M(0) for the mass-conserving model (Sec. 2)."""
    n = 32
    p = O.params(n, eps=0.02, S=2.0, dt=1e-3, variant=1)
    u = I.random_field(n, seed=5) + 0.1
    m0 = O.mass(p, u)
    u = O.fine_propagate(p, 50, u)
    assert abs(O.mass(p, u) - m0) <= 1e-13 * n * n * 1e-3 + 1e-14
    pc = O.params(n, eps=0.02, S=2.0, dt=1e-3, variant=0)
    assert abs(O.mass(pc, O.fine_propagate(pc, 50, I.random_field(n, seed=5) + 0.1)) - m0) > 1e-4


def test_solve_is_symmetric():
    """A is symmetric, so <A^-1 x, y> = <x, A^-1 y> (used by the adjoint)."""
    n = 16
    p = O.params(n, 0.05, 2.0, 1e-2)
    x, y = rng(1).standard_normal((n, n)), rng(2).standard_normal((n, n))
    assert abs(np.vdot(O.solve_A(p, x), y) - np.vdot(x, O.solve_A(p, y))) < 1e-12


# --------------------------------------------------------------- adjoint
@pytest.mark.parametrize("variant", [0, 1])
def test_energy_gradient_finite_differences(variant):
    """dE_h(u^M)/du^0 by the adjoint recursion equals central differences."""
    n, steps = 8, 12
    p = O.params(n, eps=0.08, S=2.0, dt=5e-3, variant=variant)
    u0 = I.random_field(n, seed=11)
    g = O.energy_gradient_through_solve(p, steps, u0)
    for t in range(3):
        d = rng(100 + t).standard_normal((n, n))
        hh = 1e-6
        ep = O.energy(p, O.fine_propagate(p, steps, u0 + hh * d))
        em = O.energy(p, O.fine_propagate(p, steps, u0 - hh * d))
        fd = (ep - em) / (2 * hh)
        assert abs(fd - np.vdot(g, d)) <= 1e-7 * max(1.0, abs(fd))


def test_energy_grad_matches_fd():
    n = 8
    p = O.params(n, eps=0.1, S=2.0, dt=1e-3)
    u = I.random_field(n, seed=2)
    g = O.energy_grad(p, u)
    d = rng(5).standard_normal((n, n))
    hh = 1e-6
    fd = (O.energy(p, u + hh * d) - O.energy(p, u - hh * d)) / (2 * hh)
    assert abs(fd - np.vdot(g, d)) < 1e-8


# ------------------------------------------------------------------ CNN
def test_bf16_rounding_values():
    assert O.round_bf16(1.0 + 2 ** -8) == 1.0                 # tie -> even
    assert O.round_bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6    # tie -> even (up)
    assert O.round_bf16(0.1) == 0.10009765625
    assert O.round_bf16(-3.0) == -3.0
    assert O.round_bf16(1.0 + 2 ** -8 + 2 ** -20) == 1.0 + 2 ** -7


def _one_layer(w3x3, bias=0.0):
    return O.CnnSpec(layers=1, channels=1, w=np.asarray(w3x3, float).ravel(), b=[bias], residual=0)


def test_conv_identity_and_shift():
    """Centre tap -> identity; tap (a, e) -> out[i,j] = in[i+a-1, j+e-1] (mod n):
    pins the cross-correlation orientation and the circular wrap (Sec. 3.2)."""
    n = 8
    u = rng(0).standard_normal((n, n))
    w = np.zeros((3, 3)); w[1, 1] = 1.0
    assert np.array_equal(O.cnn_forward(_one_layer(w, 0.0), u), u)
    for a in range(3):
        for e in range(3):
            w = np.zeros((3, 3)); w[a, e] = 1.0
            exp = np.roll(np.roll(u, -(a - 1), axis=0), -(e - 1), axis=1)
            assert np.array_equal(O.cnn_forward(_one_layer(w, 0.25), u), exp + 0.25)


def _gelu(x):
    return 0.5 * x * (1 + scipy.special.erf(x / math.sqrt(2)))


def _stack_scipy(u, w, b, layers, C, act):
    """Independent conv stack built from scipy.signal.correlate2d(wrap)."""
    dims = I.cnn_layer_dims(layers, C)
    a = [u]
    wo = bo = 0
    for l, (ci, co) in enumerate(dims):
        W = w[wo:wo + ci * co * 9].reshape(co, ci, 3, 3)
        out = []
        for o in range(co):
            z = np.full_like(u, b[bo + o])
            for c in range(ci):
                z = z + scipy.signal.correlate2d(a[c], W[o, c], mode="same", boundary="wrap")
            out.append(z)
        wo += ci * co * 9
        bo += co
        if l < layers - 1:
            out = [np.tanh(z) if act == 0 else _gelu(z) for z in out]
        a = out
    return u + a[0]


@pytest.mark.parametrize("act", [0, 1])
def test_conv_stack_matches_scipy(act):
    n, L, C = 8, 4, 5
    w, b = I.cnn_weights(L, C, seed=3, sigma=0.3)
    u = I.random_field(n, seed=1)
    spec = O.CnnSpec(L, C, w, b, act=act)
    assert np.abs(O.cnn_forward(spec, u) - _stack_scipy(u, w, b, L, C, act)).max() < 1e-13


def _bf16_library(x):
    """Round to bfloat16 (nearest even) with torch's float32 -> bfloat16 cast;
    exact for inputs that are float32 values."""
    torch = pytest.importorskip("torch")
    t = torch.tensor(np.asarray(x, dtype=np.float32))
    return t.to(torch.bfloat16).to(torch.float64).numpy()


def test_bf16_rounding_matches_the_library_cast():
    """The oracle's bf16 rounding equals torch's float32 -> bfloat16 cast on
    float32 inputs of every scale, ties included."""
    x = np.concatenate([rng(11).standard_normal(4000) * 10.0 ** rng(12).integers(-6, 6, 4000),
                        1.0 + np.arange(0, 2 ** 9) * 2.0 ** -9])   # every tie pattern just above 1
    x = x.astype(np.float32).astype(np.float64)
    mine = np.array([O.round_bf16(v) for v in x])
    assert np.array_equal(mine, _bf16_library(x))


def _bf16_bits(x):
    """Round float64 values to 8 significant bits, nearest even, on the bit
    pattern: add half an ulp of the kept part (minus one, plus the kept LSB)
    and clear the 45 dropped mantissa bits."""
    bits = np.ascontiguousarray(x, dtype=np.float64).view(np.uint64)
    lsb = (bits >> np.uint64(45)) & np.uint64(1)
    bits = (bits + (np.uint64((1 << 44) - 1) + lsb)) & ~np.uint64((1 << 45) - 1)
    return bits.view(np.float64)


@pytest.mark.parametrize("act", [0, 1])
def test_bf16_stack_matches_library_rounding(act):
    """The bf16 mode of the conv stack (reading 5: input, weights and hidden
    activations rounded to bf16; biases, sums and activations exact; the
    residual adds the unrounded input) against the scipy stack with torch's
    bf16 cast of the float32-valued input and weights and a bit-level
    round-to-nearest-even of the float64 hidden activations."""
    n, L, C = 8, 3, 4
    w, b = I.cnn_weights(L, C, seed=13, sigma=0.3)
    w = w.astype(np.float32).astype(np.float64)
    b = b.astype(np.float32).astype(np.float64)
    u = I.random_field(n, seed=14).astype(np.float32).astype(np.float64)
    spec = O.CnnSpec(L, C, w, b, act=act, bf16=1)
    dims = I.cnn_layer_dims(L, C)
    wr = _bf16_library(w)
    a = [_bf16_library(u)]
    wo = bo = 0
    for l, (ci, co) in enumerate(dims):
        W = wr[wo:wo + ci * co * 9].reshape(co, ci, 3, 3)
        out = []
        for o in range(co):
            z = np.full_like(u, b[bo + o])
            for c in range(ci):
                z = z + scipy.signal.correlate2d(a[c], W[o, c], mode="same", boundary="wrap")
            out.append(z)
        wo += ci * co * 9
        bo += co
        if l < L - 1:
            out = [np.tanh(z) if act == 0 else _gelu(z) for z in out]
            out = [_bf16_bits(z) for z in out]
        a = out
    ref = u + a[0]
    assert np.abs(O.cnn_forward(spec, u) - ref).max() < 1e-13


def test_conv_constant_input_closed_form():
    """A constant input stays constant through every layer: z = b + x * sum W."""
    n, L, C = 8, 3, 4
    w, b = I.cnn_weights(L, C, seed=9, sigma=0.4)
    x = 0.37
    dims = I.cnn_layer_dims(L, C)
    a = np.array([x])
    wo = bo = 0
    for l, (ci, co) in enumerate(dims):
        W = w[wo:wo + ci * co * 9].reshape(co, ci, 9)
        z = b[bo:bo + co] + W.sum(axis=2) @ a
        a = np.tanh(z) if l < L - 1 else z
        wo += ci * co * 9
        bo += co
    out = O.cnn_forward(O.CnnSpec(L, C, w, b, act=0), np.full((n, n), x))
    assert np.abs(out - (x + a[0])).max() < 1e-15


def test_mass_fix_and_limiter():
    """mACNN shift (mean preserved) applied before the bound limiter (Sec. 3.2)."""
    n, L, C = 8, 3, 4
    w, b = I.cnn_weights(L, C, seed=2, sigma=0.5)
    u = I.random_field(n, seed=4)
    base = O.cnn_forward(O.CnnSpec(L, C, w, b, act=0), u)
    fixed = O.cnn_forward(O.CnnSpec(L, C, w, b, act=0, mass_fix=1), u)
    assert abs(fixed.mean() - u.mean()) < 1e-15
    assert np.abs((fixed - base) - (fixed - base).mean()).max() < 1e-15
    lim = O.cnn_forward(O.CnnSpec(L, C, w, b, act=0, mass_fix=1, limiter=1, lo=-0.5, hi=0.5), u)
    assert np.array_equal(lim, np.clip(fixed, -0.5, 0.5))


def test_bf16_mode_rounds_inputs_and_weights():
    """With bf16 on, a one-layer identity-like stack sees bf16(u) and bf16(w)."""
    n = 8
    u = I.random_field(n, seed=8)
    w = np.zeros((3, 3)); w[1, 1] = 1.0 + 2 ** -10
    spec = O.CnnSpec(1, 1, w.ravel(), [0.0], residual=0, bf16=1)
    rb = np.vectorize(O.round_bf16)
    assert np.array_equal(O.cnn_forward(spec, u), rb(u) * rb(1.0 + 2 ** -10))


@pytest.mark.parametrize("act,mass_fix", [(0, 0), (1, 0), (1, 1)])
def test_conv_backward_finite_differences(act, mass_fix):
    n, L, C = 6, 3, 3
    w, b = I.cnn_weights(L, C, seed=5, sigma=0.4)
    u = I.random_field(n, seed=6)
    gout = rng(7).standard_normal((n, n))
    spec = O.CnnSpec(L, C, w, b, act=act, mass_fix=mass_fix)
    gin, gw, gb = O.cnn_backward(spec, u, gout)
    hh = 1e-6

    def J(uu, ww, bb):
        return np.vdot(gout, O.cnn_forward(O.CnnSpec(L, C, ww, bb, act=act, mass_fix=mass_fix), uu))

    d = rng(8).standard_normal((n, n))
    fd = (J(u + hh * d, w, b) - J(u - hh * d, w, b)) / (2 * hh)
    assert abs(fd - np.vdot(gin, d)) < 1e-7 * max(1, abs(fd))
    dw = rng(9).standard_normal(w.shape)
    fd = (J(u, w + hh * dw, b) - J(u, w - hh * dw, b)) / (2 * hh)
    assert abs(fd - np.vdot(gw, dw)) < 1e-7 * max(1, abs(fd))
    db = rng(10).standard_normal(b.shape)
    fd = (J(u, w, b + hh * db) - J(u, w, b - hh * db)) / (2 * hh)
    assert abs(fd - np.vdot(gb, db)) < 1e-7 * max(1, abs(fd))


def _stack_frozen_rounding(u, w, b, layers, C, act, mass_fix, r_u, r_w, r_a):
    """The conv stack with every bf16 rounding replaced by the addition of a
    constant offset (r_u to the input, r_w to the weights, r_a[l] to the
    activations of hidden layer l); scipy correlate2d(wrap) convolutions."""
    dims = I.cnn_layer_dims(layers, C)
    a = [u + r_u]
    wr = w + r_w
    wo = bo = 0
    for l, (ci, co) in enumerate(dims):
        W = wr[wo:wo + ci * co * 9].reshape(co, ci, 3, 3)
        out = []
        for o in range(co):
            z = np.full_like(u, b[bo + o])
            for c in range(ci):
                z = z + scipy.signal.correlate2d(a[c], W[o, c], mode="same", boundary="wrap")
            out.append(z)
        wo += ci * co * 9
        bo += co
        if l < layers - 1:
            out = [(np.tanh(z) if act == 0 else _gelu(z)) + r_a[l][o] for o, z in enumerate(out)]
        a = out
    res = u + a[0]
    if mass_fix:
        res = res + (u.mean() - res.mean())
    return res


@pytest.mark.parametrize("act,mass_fix", [(0, 0), (1, 0), (1, 1)])
def test_bf16_backward_is_the_gradient_with_frozen_rounding(act, mass_fix):
    """The straight-through backward of the bf16 mode (reading 5) is the exact
    gradient of the stack in which each bf16 rounding is frozen into a
    constant offset taken at the evaluation point: that stack equals the bf16
    forward there, and it is smooth, so central differences of it in random
    directions of u, W and b must match the backward's inner products."""
    n, L, C = 6, 3, 3
    w, b = I.cnn_weights(L, C, seed=15, sigma=0.4)
    w = w.astype(np.float32).astype(np.float64)
    b = b.astype(np.float32).astype(np.float64)
    u = I.random_field(n, seed=16).astype(np.float32).astype(np.float64)
    gout = rng(17).standard_normal((n, n))
    spec = O.CnnSpec(L, C, w, b, act=act, mass_fix=mass_fix, bf16=1)
    # the rounding offsets at the evaluation point, from an independent forward
    r_u = _bf16_bits(u) - u
    r_w = _bf16_bits(w) - w
    dims = I.cnn_layer_dims(L, C)
    a = [u + r_u]
    wr = w + r_w
    r_a = []
    wo = bo = 0
    for l, (ci, co) in enumerate(dims[:-1]):
        W = wr[wo:wo + ci * co * 9].reshape(co, ci, 3, 3)
        acts = []
        for o in range(co):
            z = np.full_like(u, b[bo + o])
            for c in range(ci):
                z = z + scipy.signal.correlate2d(a[c], W[o, c], mode="same", boundary="wrap")
            acts.append(np.tanh(z) if act == 0 else _gelu(z))
        r_a.append([_bf16_bits(v) - v for v in acts])
        a = [v + r for v, r in zip(acts, r_a[-1])]
        wo += ci * co * 9
        bo += co
    frozen = lambda uu, ww, bb: _stack_frozen_rounding(uu, ww, bb, L, C, act, mass_fix, r_u, r_w, r_a)
    # at the evaluation point the frozen stack is the bf16 forward
    assert np.abs(frozen(u, w, b) - O.cnn_forward(spec, u)).max() < 1e-13
    gin, gw, gb = O.cnn_backward(spec, u, gout)
    hh = 1e-6
    J = lambda uu, ww, bb: np.vdot(gout, frozen(uu, ww, bb))
    d = rng(18).standard_normal((n, n))
    fd = (J(u + hh * d, w, b) - J(u - hh * d, w, b)) / (2 * hh)
    assert abs(fd - np.vdot(gin, d)) < 1e-7 * max(1, abs(fd))
    dw = rng(19).standard_normal(w.shape)
    fd = (J(u, w + hh * dw, b) - J(u, w - hh * dw, b)) / (2 * hh)
    assert abs(fd - np.vdot(gw, dw)) < 1e-7 * max(1, abs(fd))
    db = rng(20).standard_normal(b.shape)
    fd = (J(u, w, b + hh * db) - J(u, w, b - hh * db)) / (2 * hh)
    assert abs(fd - np.vdot(gb, db)) < 1e-7 * max(1, abs(fd))


# -------------------------------------------------------------- Parareal
def _small_problem(variant=0):
    n, s, c = 16, 6, 5
    p = O.params(n, eps=0.05, S=2.0, dt=2e-3, variant=variant)
    w, b = I.cnn_weights(3, 4, seed=1)
    return p, O.CnnSpec(3, 4, w, b, act=0), n, s, c, I.random_field(n, seed=2)


@pytest.mark.parametrize("variant", [0, 1])
def test_parareal_exactness(variant):
    """After k iterations the first k slices equal the sequential fine solve,
    bitwise (Sec. 3.3); at k = s the whole trajectory does."""
    p, G, n, s, c, u0 = _small_problem(variant)
    seq = [u0]
    for j in range(s):
        seq.append(O.fine_propagate(p, c, seq[-1]))
    for k in range(1, s + 1):
        r = O.parareal(p, G, s, c, kmax=k, tol=0.0, u0=u0)
        assert r["iters"] == k
        for j in range(k + 1):
            assert np.array_equal(r["U"][j], seq[j]), (k, j)
    assert np.array_equal(r["U"], np.stack(seq))


def test_parareal_with_fine_as_coarse_converges_at_once():
    """G = F makes U^0 the fine trajectory, so the first increment is zero."""
    p, _, n, s, c, u0 = _small_problem()
    r = O.parareal(p, None, s, c, kmax=s, tol=1e-300, u0=u0, coarse_steps=c)
    assert r["res_l2"][0] == 0.0 and r["iters"] == 1


def test_parareal_cost_model_count():
    """G evaluations: s + (s-1) + ... + (s-k) = (2s-k)(k+1)/2 (Sec. 3.4)."""
    p, G, n, s, c, u0 = _small_problem()
    for k in (1, 2, 4, s):
        r = O.parareal(p, G, s, c, kmax=k, tol=0.0, u0=u0)
        assert r["g_calls"] == (2 * s - k) * (k + 1) // 2


def test_parareal_reuse_equals_literal_algorithm():
    """Reusing stored G(U^{k-1}_n) gives bitwise the iterates of the literal
    Algorithm 2, which evaluates both G terms afresh."""
    p, G, n, s, c, u0 = _small_problem(1)
    for k in (1, 3):
        a = O.parareal(p, G, s, c, kmax=k, tol=0.0, u0=u0)
        b = O.parareal(p, G, s, c, kmax=k, tol=0.0, u0=u0, literal=True)
        assert np.array_equal(a["U"], b["U"])
        assert np.array_equal(a["res_l2"], b["res_l2"])


def test_parareal_coarse_composition_of_fine_is_longer_fine():
    """Composing G = F over c0 steps m times is F over m*c0 steps (the coarse
    composition of the remark after Algorithm 2), so the iterates are
    identical to those with coarse_steps = m*c0, and each evaluation counts m
    applications."""
    p, _, n, s, c, u0 = _small_problem(1)
    for m in (2, 3):
        a = O.parareal(p, None, s, c, kmax=3, tol=0.0, u0=u0, coarse_steps=2, coarse_repeat=m)
        b = O.parareal(p, None, s, c, kmax=3, tol=0.0, u0=u0, coarse_steps=2 * m)
        assert np.array_equal(a["U"], b["U"])
        assert np.array_equal(a["res_l2"], b["res_l2"])
        assert a["g_calls"] == m * b["g_calls"]


def test_parareal_coarse_composition_first_sweep_and_exactness():
    """With G composed twice the k = 0 sweep is U_{j+1} = G(G(U_j)) (brute force
    with the network), and after k = s iterations the trajectory is still the
    sequential fine solve (Sec. 3.3: exactness does not depend on G)."""
    p, G, n, s, c, u0 = _small_problem(0)
    r = O.parareal(p, G, s, c, kmax=0, tol=0.0, u0=u0, coarse_repeat=2)
    u = u0.copy()
    for j in range(s):
        u = O.cnn_forward(G, O.cnn_forward(G, u))
        assert np.array_equal(r["U"][j + 1], u)
    r = O.parareal(p, G, s, c, kmax=s, tol=0.0, u0=u0, coarse_repeat=2)
    seq = [u0]
    for j in range(s):
        seq.append(O.fine_propagate(p, c, seq[-1]))
    assert np.array_equal(r["U"], np.stack(seq))


def test_residual_definition():
    """Relative L2 over slices 1..s and the sup norm (slice 0 is the fixed IC)."""
    Un = np.zeros((3, 2, 2)); Uo = np.zeros((3, 2, 2))
    Un[0] = 5.0                 # ignored
    Un[1, 0, 0] = 3.0; Uo[1, 0, 0] = 1.0
    Un[2, 1, 1] = 4.0; Uo[2, 1, 1] = 4.0
    l2, mx = O.residual(Un, Uo)
    assert mx == 2.0
    assert abs(l2 - 2.0 / 5.0) < 1e-16


def _linear_modes_problem(variant):
    """Two small-amplitude Fourier modes (one along each axis) on a 16^2 grid.
    At amplitude 1e-9 the cubic term u^3 is ~1e-27, far below float64
    rounding of u, so one fine step multiplies each mode by the scalar
    r(m) = (1 + S dt + dt) / D(m), D(m) = 1 + S dt + dt eps^2 (4/h^2) sin^2(pi m/N)
    (Sec. 3.1 scheme with f(u) = u - u^3 linearised at 0; for the mass variant
    beta = mean f(u) = -mean u^3 vanishes to the same order)."""
    n, eps, S, dt = 16, 0.05, 2.0, 2e-3
    p = O.params(n, eps=eps, S=S, dt=dt, variant=variant)
    h = 1.0 / n
    i = np.arange(n)
    modes = ((1, 1.0e-9, 0), (5, 0.7e-9, 1))   # (wavenumber, amplitude, axis)
    fields, ratios = [], []
    for m, amp, axis in modes:
        line = amp * np.cos(2 * np.pi * m * i / n)
        fields.append(np.tile(line[:, None], (1, n)) if axis == 0 else np.tile(line[None, :], (n, 1)))
        D = 1 + S * dt + dt * eps ** 2 * (4 / h ** 2) * math.sin(math.pi * m / n) ** 2
        ratios.append((1 + S * dt + dt) / D)
    return p, fields, ratios


@pytest.mark.parametrize("variant", [0, 1])
def test_parareal_linear_closed_form(variant):
    """Parareal on a linear scalar problem has a closed form (Gander &
    Vandewalle, SIAM J. Sci. Comput. 29 (2007)): with propagators F = rF,
    G = rG and U^0_n = rG^n u0, the correction of Sec. 3.3 / Algorithm 2,
    U^k_{n+1} = G U^k_n + F U^{k-1}_n - G U^{k-1}_n, gives
        U^k_n = sum_{j=0..min(k,n)} C(n, j) (rF - rG)^j rG^(n-j) u0.
    Here F is c fine steps and G = F over c' != c steps, both scalar on each
    Fourier mode of a small-amplitude field.  Slices n > k (not yet exact)
    pin the sign and the indices of the correction: a flipped (G_new - G_old)
    changes the j = 1 term by ~1e-2 relative, the tolerance is 1e-12."""
    p, fields, ratios = _linear_modes_problem(variant)
    s, c, cg = 6, 5, 2
    u0 = fields[0] + fields[1]
    scale = max(np.abs(f).max() for f in fields)
    for k in (1, 2, 3):
        r = O.parareal(p, None, s, c, kmax=k, tol=0.0, u0=u0, coarse_steps=cg)
        assert r["iters"] == k
        for n_ in range(s + 1):
            ref = np.zeros_like(u0)
            for f, rr in zip(fields, ratios):
                rF, rG = rr ** c, rr ** cg
                ref += sum(math.comb(n_, j) * (rF - rG) ** j * rG ** (n_ - j)
                           for j in range(min(k, n_) + 1)) * f
            assert np.abs(r["U"][n_] - ref).max() < 1e-12 * scale, (k, n_)
    # the closed form really separates the iterates from the fine solve at n > k
    rF, rG = ratios[0] ** c, ratios[0] ** cg
    assert abs(sum(math.comb(4, j) * (rF - rG) ** j * rG ** (4 - j) for j in range(2)) - rF ** 4) > 1e-6


def test_oracle_threads_do_not_change_results():
    """The oracle's optional threads split conv output rows and independent
    fine solves only, so every value is bit-identical for any thread count."""
    p, G, n, s, c, u0 = _small_problem(1)
    a = O.parareal(p, G, s, c, kmax=3, tol=0.0, u0=u0)
    with O.threads(3):
        b = O.parareal(p, G, s, c, kmax=3, tol=0.0, u0=u0)
        y = O.cnn_forward(G, u0)
    assert np.array_equal(a["U"], b["U"]) and np.array_equal(a["res_l2"], b["res_l2"])
    assert np.array_equal(y, O.cnn_forward(G, u0))
