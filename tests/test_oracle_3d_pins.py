"""Pins of the oracle's 3D fine step (the model on the periodic cube, d = 3;
the 3D experiments of Sec. 4) against facts fixed by mathematics and by the
separately pinned 2D oracle.  None of these call the CUDA path."""
import numpy as np
import pytest

import acpr_inputs as I
import oracle as O


def rng(seed):
    return np.random.default_rng(seed)


@pytest.mark.parametrize("n", [4, 8])
def test_fft3_matches_library(n):
    x = rng(n).standard_normal((n, n, n)) + 1j * rng(n + 1).standard_normal((n, n, n))
    assert np.abs(O.fft3(x, -1) - np.fft.fftn(x)).max() < 1e-12 * n ** 3
    assert np.abs(O.fft3(x, +1) - np.fft.ifftn(x) * n ** 3).max() < 1e-12 * n ** 3


def test_seven_point_symbol():
    """The direct 7-point stencil applied to a Fourier mode multiplies it by
    -(4/h^2)(sin^2(pi a/N) + sin^2(pi b/N) + sin^2(pi c/N)); the solve uses that symbol."""
    n, h = 8, 1.0 / 8
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    for a, b, c in ((1, 0, 0), (0, 2, 0), (0, 0, 3), (1, 2, 3)):
        phase = 2 * np.pi * (a * i + b * j + c * k) / n
        lam = -(4 / h ** 2) * (np.sin(np.pi * a / n) ** 2 + np.sin(np.pi * b / n) ** 2 + np.sin(np.pi * c / n) ** 2)
        for u in (np.cos(phase), np.sin(phase)):
            assert np.abs(O.lap3(u, h) - lam * u).max() < 1e-10 * abs(lam)


def test_solve_matches_dense_elimination():
    """((1 + S dt) I - dt eps^2 Lap_h) v = r for N = 4 against Gaussian
    elimination of the 64 x 64 system built from the 7-point stencil."""
    n = 4
    p = O.params(n, eps=0.1, S=2.0, dt=0.05)
    h = p.length / n
    m = n ** 3
    A = np.zeros((m, m))
    for col in range(m):
        e = np.zeros(m)
        e[col] = 1.0
        A[:, col] = (1 + p.S * p.dt) * e - p.dt * p.eps ** 2 * O.lap3(e.reshape(n, n, n), h).ravel()
    r = rng(3).standard_normal((n, n, n))
    assert np.abs(O.solve_A3(p, r).ravel() - np.linalg.solve(A, r.ravel())).max() < 1e-12


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_constant_along_an_axis_reduces_to_2d(variant, axis):
    """A field constant along one axis stays so, and its 3D step is the
    (separately pinned) 2D step of the remaining two axes."""
    n = 8
    w = I.random_field(n, seed=10 + axis, zero_mean=bool(variant))
    u = np.repeat(np.expand_dims(w, axis), n, axis=axis)
    p = O.params(n, eps=0.05, S=2.0, dt=1e-3, variant=variant)
    out3 = O.fine3d_propagate(p, 3, u)
    out2 = O.fine_propagate(p, 3, w)
    ref = np.repeat(np.expand_dims(out2, axis), n, axis=axis)
    assert np.abs(out3 - ref).max() < 1e-13


def test_mass_conservation_and_maximum_principle():
    """The mass variant keeps the mean; the classic step with S = 2 keeps
    |u| <= 1 from data in [-0.9, 0.9]."""
    n = 8
    u = rng(5).uniform(-0.9, 0.9, (n, n, n))
    p = O.params(n, eps=0.05, S=2.0, dt=5e-3, variant=1)
    out = O.fine3d_propagate(p, 20, u)
    assert abs(out.mean() - u.mean()) < 1e-14
    p0 = O.params(n, eps=0.05, S=2.0, dt=5e-3, variant=0)
    out0 = O.fine3d_propagate(p0, 20, u)
    assert np.abs(out0).max() <= 1.0
    assert abs(out0.mean() - u.mean()) > 1e-6  # the classic model does not conserve mass


# ---------------------------------------------- ResBlock ACNN on the cube --
def _acnn3(C, R, seed, mass_fix=0):
    w, b = I.acnn3d_weights(C, R, seed=seed)
    return w, b, O.Acnn3dSpec(C, R, w, b, mass_fix=mass_fix)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_acnn3d_on_a_field_constant_along_an_axis_is_the_2d_network(axis):
    """A field constant along one axis stays so through every layer; the 3D
    network then equals the (pinned) 2D network on the other two axes whose
    3 x 3 weights are the 3 x 3 x 3 weights summed over that axis's tap index
    (which fixes the orientation of the other two tap indices)."""
    C, R, n = 4, 2, 8
    w3, b3, spec3 = _acnn3(C, R, seed=1 + axis, mass_fix=1)
    w2 = w3.reshape(-1, 3, 3, 3).sum(axis=1 + axis).ravel()
    spec2 = O.AcnnSpec(C, R, w2, b3, mass_fix=1)
    u2 = I.random_field(n, seed=2)
    u3 = np.repeat(np.expand_dims(u2, axis), n, axis=axis)
    out3 = O.acnn3d_forward(spec3, u3)
    out2 = O.acnn_forward(spec2, u2)
    assert np.abs(out3 - np.expand_dims(out2, axis)).max() < 1e-13


def test_acnn3d_translation_and_mass():
    C, R, n = 4, 1, 8
    _, _, spec = _acnn3(C, R, seed=3, mass_fix=1)
    u = rng(4).uniform(-0.9, 0.9, (n, n, n))
    out = O.acnn3d_forward(spec, u)
    sh = O.acnn3d_forward(spec, np.roll(u, (1, -2, 3), axis=(0, 1, 2)))
    assert np.abs(sh - np.roll(out, (1, -2, 3), axis=(0, 1, 2))).max() < 1e-13
    assert abs(out.mean() - u.mean()) < 1e-15


def test_parareal3d_sweep_exactness_and_g_equals_f():
    """Algorithm 2 on the cube: the k = 0 sweep is the 3D network's rollout;
    at k = s the trajectory is the sequential 3D fine solve (Sec. 3.3); with
    G = F the first increment is zero."""
    C, R, n, s, c = 4, 1, 8, 3, 2
    _, _, spec = _acnn3(C, R, seed=5, mass_fix=1)
    p = O.params(n, eps=0.05, S=2.0, dt=2e-3, variant=1)
    u0 = rng(6).uniform(-0.9, 0.9, (n, n, n))
    u0 -= u0.mean()
    r0 = O.parareal3d(p, spec, s, c, kmax=0, tol=0.0, u0=u0)
    u = u0
    for j in range(s):
        u = O.acnn3d_forward(spec, u)
        assert np.array_equal(r0["U"][j + 1], u)
    r = O.parareal3d(p, spec, s, c, kmax=s, tol=0.0, u0=u0)
    seq = [u0]
    for j in range(s):
        seq.append(O.fine3d_propagate(p, c, seq[-1]))
    assert np.array_equal(r["U"], np.stack(seq))
    rf = O.parareal3d(p, None, s, c, kmax=s, tol=1e-300, u0=u0, coarse_steps=c)
    assert rf["res_l2"][0] == 0.0 and rf["iters"] == 1
