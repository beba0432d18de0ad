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
