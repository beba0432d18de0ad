"""Pins of the oracle's Crank-Nicolson + Picard fine step (Sec. 3.1) against
facts the scheme fixes, independent of its DFT solve and of its Picard loop:
the defining equation evaluated with a direct 5-point stencil, the scalar
closed form for constant fields, exact mass conservation in the conservative
variant, and second-order accuracy in time."""
import numpy as np
import pytest

import acpr_inputs as I
import oracle as O


def lap5(u, h):
    return (np.roll(u, 1, 0) + np.roll(u, -1, 0) + np.roll(u, 1, 1) + np.roll(u, -1, 1) - 4 * u) / h ** 2


def f(u):
    return u - u ** 3


def cn_residual(u, up, eps, dt, h, mass):
    """(U' - U)/dt - eps^2 Lap (U' + U)/2 - (f(U') + f(U))/2 + g, g the mean of
    (f(U') + f(U))/2 in the conservative variant (Sec. 3.1, first form)."""
    g = np.mean(0.5 * (f(up) + f(u))) if mass else 0.0
    return (up - u) / dt - eps ** 2 * lap5(up + u, h) / 2 - (f(up) + f(u)) / 2 + g


@pytest.mark.parametrize("variant", [0, 1])
def test_converged_step_satisfies_the_scheme(variant):
    n, eps, dt = 32, 0.05, 1e-3
    u = I.random_field(n, seed=3, zero_mean=bool(variant))
    p = O.params(n, eps, 2.0, dt, variant)
    up, it = O.cn_step(p, u, tol=1e-14, maxit=60)
    assert it < 60
    r = cn_residual(u, up, eps, dt, 1.0 / n, variant == 1)
    assert np.abs(r).max() < 1e-9          # residual per unit time; U' moves O(1e-2) per step


@pytest.mark.parametrize("a", [-0.7, 0.2, 0.95])
def test_constant_field_closed_form(a):
    """u = a everywhere: Lap u = 0, so a' solves a' = a + dt/2 (f(a) + f(a'))
    (classic; scalar Newton here) and a' = a (conservative: g cancels)."""
    n, dt = 8, 0.05
    u = np.full((n, n), a)
    x = a
    for _ in range(50):
        F = x - a - dt / 2 * (f(a) + f(x))
        x -= F / (1 - dt / 2 * (1 - 3 * x * x))
    up, _ = O.cn_step(O.params(n, 0.1, 2.0, dt, 0), u, tol=1e-15, maxit=200)
    assert np.abs(up - x).max() < 1e-13
    upm, _ = O.cn_step(O.params(n, 0.1, 2.0, dt, 1), u, tol=1e-15, maxit=200)
    assert np.abs(upm - a).max() < 1e-14


def test_mass_is_conserved_exactly():
    n = 32
    u = I.random_field(n, seed=5, zero_mean=False)
    p = O.params(n, 0.05, 2.0, 2e-3, 1)
    up, _ = O.cn_propagate(p, 20, u, tol=1e-14, maxit=60)
    assert abs(up.sum() - u.sum()) < 1e-11 * n * n


def test_second_order_in_time():
    """A smooth initial state; errors at T against a run with a 16 times
    smaller step fall by about 4 when the step halves."""
    n, eps, T = 16, 0.1, 0.02
    x = np.arange(n) / n
    u0 = 0.5 * np.cos(2 * np.pi * x)[:, None] + 0.3 * np.sin(4 * np.pi * x)[None, :]
    def run(dt):
        out, _ = O.cn_propagate(O.params(n, eps, 2.0, dt, 0), int(round(T / dt)), u0, tol=1e-15, maxit=100)
        return out
    ref = run(T / 320)
    e1 = np.abs(run(T / 10) - ref).max()
    e2 = np.abs(run(T / 20) - ref).max()
    assert 3.5 < e1 / e2 < 4.5


def test_picard_contracts_fast_for_small_steps():
    """The Picard map's contraction factor is about dt/2 max|f'| / (1 + ...): at
    dt = 5e-5 a few iterations reach 1e-12."""
    n = 32
    u = I.random_field(n, seed=2)
    _, it = O.cn_step(O.params(n, 0.01, 2.0, 5e-5, 0), u, tol=1e-12, maxit=50)
    assert it <= 5
