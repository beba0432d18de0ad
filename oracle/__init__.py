"""Float64 CPU oracle for the Allen-Cahn Parareal hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference legs may import this package; the library
in ``paper_2510_07672_gb300`` never does, and shares no code with it.

The arithmetic lives in ``acpr_oracle.c`` (plain C, float64, no blocking or
fusion), compiled with gcc on first use into ``oracle/_build/`` and loaded with
ctypes.  This module only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "acpr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class Params(C.Structure):
    _fields_ = [("n", C.c_int), ("length", C.c_double), ("eps", C.c_double),
                ("S", C.c_double), ("dt", C.c_double), ("variant", C.c_int)]


class Cnn(C.Structure):
    _fields_ = [("layers", C.c_int), ("channels", C.c_int), ("act", C.c_int),
                ("residual", C.c_int), ("mass_fix", C.c_int), ("limiter", C.c_int),
                ("bf16", C.c_int), ("lo", C.c_double), ("hi", C.c_double),
                ("w", C.POINTER(C.c_double)), ("b", C.POINTER(C.c_double))]


class Acnn(C.Structure):
    _fields_ = [("channels", C.c_int), ("blocks", C.c_int), ("mass_fix", C.c_int), ("limiter", C.c_int),
                ("lo", C.c_double), ("hi", C.c_double),
                ("w", C.POINTER(C.c_double)), ("b", C.POINTER(C.c_double))]


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, no FMA contraction so x86 and Arm agree)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            L.or_set_threads.argtypes = [C.c_int]
            L.or_get_threads.restype = C.c_int
            L.or_fft2d_ri.argtypes = [dp, C.c_int, C.c_int]
            L.or_dft2d_naive_ri.argtypes = [dp, dp, C.c_int, C.c_int]
            L.or_fine_step.argtypes = [C.POINTER(Params), dp, dp]
            L.or_fine_propagate.argtypes = [C.POINTER(Params), C.c_int, dp, dp]
            L.or_cn_step.argtypes = [C.POINTER(Params), dp, dp, C.c_double, C.c_int]
            L.or_cn_step.restype = C.c_int
            L.or_cn_propagate.argtypes = [C.POINTER(Params), C.c_int, dp, dp, C.c_double, C.c_int]
            L.or_cn_propagate.restype = C.c_long
            L.or_solve_A.argtypes = [C.POINTER(Params), dp, dp]
            L.or_energy.argtypes = [C.POINTER(Params), dp]
            L.or_energy.restype = C.c_double
            L.or_mass.argtypes = [C.POINTER(Params), dp]
            L.or_mass.restype = C.c_double
            L.or_energy_grad.argtypes = [C.POINTER(Params), dp, dp]
            L.or_fine_adjoint_step.argtypes = [C.POINTER(Params), dp, dp, dp]
            L.or_energy_gradient_through_solve.argtypes = [C.POINTER(Params), C.c_int, dp, dp]
            L.or_round_bf16.argtypes = [C.c_double]
            L.or_round_bf16.restype = C.c_double
            L.or_cnn_forward.argtypes = [C.POINTER(Cnn), C.c_int, dp, dp]
            L.or_cnn_forward_batch.argtypes = [C.POINTER(Cnn), C.c_int, C.c_int, dp, dp]
            L.or_cnn_backward.argtypes = [C.POINTER(Cnn), C.c_int, dp, dp, dp, dp, dp]
            L.or_residual.argtypes = [C.c_int, C.c_int, dp, dp, dp, dp]
            L.or_parareal.argtypes = [C.POINTER(Params), C.POINTER(Cnn), C.c_int, C.c_int, C.c_int,
                                      C.c_int, C.c_double, C.c_int, dp, dp, dp, dp,
                                      C.POINTER(C.c_int)]
            L.or_parareal.restype = C.c_long
            L.or_parareal_rep.argtypes = [C.POINTER(Params), C.POINTER(Cnn), C.c_int, C.c_int, C.c_int, C.c_int,
                                          C.c_int, C.c_double, C.c_int, dp, dp, dp, dp, C.POINTER(C.c_int)]
            L.or_parareal_rep.restype = C.c_long
            L.or_fft3d_ri.argtypes = [dp, C.c_int, C.c_int]
            L.or_solve_A3.argtypes = [C.POINTER(Params), dp, dp]
            L.or_fine3d_step.argtypes = [C.POINTER(Params), dp, dp]
            L.or_fine3d_propagate.argtypes = [C.POINTER(Params), C.c_int, dp, dp]
            L.or_lap3.argtypes = [C.c_int, C.c_double, dp, dp]
            L.or_acnn3d_param_counts.argtypes = [C.POINTER(Acnn), C.POINTER(C.c_long)]
            L.or_acnn3d_param_counts.restype = C.c_long
            L.or_acnn3d_forward.argtypes = [C.POINTER(Acnn), C.c_int, C.c_int, dp, dp]
            L.or_parareal3d.argtypes = [C.POINTER(Params), C.POINTER(Acnn), C.c_int, C.c_int, C.c_int, C.c_int,
                                        C.c_int, C.c_double, dp, dp, dp, dp, C.POINTER(C.c_int)]
            L.or_parareal3d.restype = C.c_long
            L.or_parareal_acnn.argtypes = [C.POINTER(Params), C.POINTER(Acnn), C.c_int, C.c_int, C.c_int, C.c_int,
                                           C.c_double, dp, dp, dp, dp, C.POINTER(C.c_int)]
            L.or_parareal_acnn.restype = C.c_long
            L.or_acnn_param_counts.argtypes = [C.POINTER(Acnn), C.POINTER(C.c_long)]
            L.or_acnn_param_counts.restype = C.c_long
            L.or_acnn_forward.argtypes = [C.POINTER(Acnn), C.c_int, C.c_int, dp, dp]
            L.or_acnn_backward.argtypes = [C.POINTER(Acnn), C.c_int, C.c_int, dp, dp, dp, dp]
            L.or_loss_acn.argtypes = [C.POINTER(Params), C.c_int, dp, dp, dp]
            L.or_loss_acn.restype = C.c_double
            L.or_adam.argtypes = [dp, dp, dp, dp, C.c_long, C.c_double, C.c_double, C.c_double, C.c_double,
                                  C.c_int]
            L.or_acnn_train.argtypes = [C.POINTER(Params), C.POINTER(Acnn), dp, dp, C.c_int, dp,
                                        C.POINTER(C.c_int), C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                        C.c_double, C.c_double, C.c_double, dp, dp, C.POINTER(C.c_int), dp]
            _lib = L
    return _lib


class threads:
    """Context manager: run the oracle's conv layers (split by output rows)
    and Algorithm 2's independent fine solves on `t` threads.  Results are
    identical for every t; only the wall time changes."""

    def __init__(self, t: int):
        self.t = int(t)

    def __enter__(self):
        self.old = lib().or_get_threads()
        lib().or_set_threads(self.t)
        return self

    def __exit__(self, *exc):
        lib().or_set_threads(self.old)
        return False


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def params(n, eps, S, dt, variant=0, length=1.0) -> Params:
    return Params(int(n), float(length), float(eps), float(S), float(dt), int(variant))


class CnnSpec:
    """Conv-stack description holding float64 copies of the parameters."""

    def __init__(self, layers, channels, w, b, act=0, residual=1, mass_fix=0, limiter=0,
                 bf16=0, lo=-1.0, hi=1.0):
        self.w = _f64(w).ravel().copy()
        self.b = _f64(b).ravel().copy()
        self.s = Cnn(int(layers), int(channels), int(act), int(residual), int(mass_fix),
                     int(limiter), int(bf16), float(lo), float(hi), _dp(self.w), _dp(self.b))


class AcnnSpec:
    """The paper's ResBlock ACNN / mACNN (Sec. 3.2) with float64 copies of its
    parameters: input conv 1 -> C, `blocks` blocks x -> x + tanh(conv(tanh(conv(x)))),
    output conv C -> 1, then the mass shift and the bound limiter."""

    def __init__(self, channels, blocks, w, b, mass_fix=0, limiter=0, lo=-1.0, hi=1.0):
        self.w = _f64(w).ravel().copy()
        self.b = _f64(b).ravel().copy()
        self.s = Acnn(int(channels), int(blocks), int(mass_fix), int(limiter), float(lo), float(hi),
                      _dp(self.w), _dp(self.b))
        nb = C.c_long()
        nw = lib().or_acnn_param_counts(C.byref(self.s), C.byref(nb))
        if self.w.size != nw or self.b.size != nb.value:
            raise ValueError(f"ACNN C={channels} blocks={blocks} takes {nw} weights and {nb.value} biases")


def acnn_param_counts(channels: int, blocks: int):
    """(number of weights, number of biases) of the ResBlock ACNN."""
    d = Acnn(int(channels), int(blocks), 0, 0, 0.0, 0.0, None, None)
    nb = C.c_long()
    nw = lib().or_acnn_param_counts(C.byref(d), C.byref(nb))
    return int(nw), int(nb.value)


def acnn_forward(spec: AcnnSpec, u) -> np.ndarray:
    u = _f64(u)
    out = np.empty_like(u)
    batch = 1 if u.ndim == 2 else u.shape[0]
    lib().or_acnn_forward(C.byref(spec.s), u.shape[-1], batch, _dp(u), _dp(out))
    return out


def acnn_backward(spec: AcnnSpec, u, gout):
    """(dL/dW, dL/db) summed over the batch for gout = dL/d(output)."""
    u, gout = _f64(u), _f64(gout)
    batch = 1 if u.ndim == 2 else u.shape[0]
    gw = np.empty_like(spec.w)
    gb = np.empty_like(spec.b)
    lib().or_acnn_backward(C.byref(spec.s), u.shape[-1], batch, _dp(u), _dp(gout), _dp(gw), _dp(gb))
    return gw, gb


def loss_acn(p: Params, U0, U1, grad: bool = True):
    """Eq. loss_ACN with time step p.dt: (loss, dL/dU1 or None)."""
    U0, U1 = _f64(U0), _f64(U1)
    batch = 1 if U0.ndim == 2 else U0.shape[0]
    g = np.empty_like(U1) if grad else None
    loss = lib().or_loss_acn(C.byref(p), batch, _dp(U0), _dp(U1), _dp(g) if grad else None)
    return loss, g


def adam(w, g, m, v, lr, b1, b2, eps, t):
    """One Adam step in place on float64 arrays w, m, v."""
    for a in (w, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _f64(g)
    lib().or_adam(_dp(w), _dp(g), _dp(m), _dp(v), w.size, lr, b1, b2, eps, int(t))


def acnn_train(p: Params, spec: AcnnSpec, U0s, perm, q, steps, b_inner, lr=1e-3, b1=0.9, b2=0.999, aeps=1e-8,
               state=None):
    """Algorithm 1 on `spec` (parameters updated in place).  perm: [epochs][R]
    visiting order.  state: dict(m, v, t) carried between calls.  Returns
    (losses per update, state)."""
    U0s = _f64(U0s)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    epochs, R = perm.shape
    nw, nb = spec.w.size, spec.b.size
    if state is None:
        state = {"m": np.zeros(nw + nb), "v": np.zeros(nw + nb), "t": 0}
    t = C.c_int(state["t"])
    losses = np.zeros(epochs * (R // q) * steps * b_inner)
    lib().or_acnn_train(C.byref(p), C.byref(spec.s), _dp(spec.w), _dp(spec.b), R, _dp(U0s),
                        perm.ctypes.data_as(C.POINTER(C.c_int)), int(q), int(steps), int(b_inner), epochs,
                        lr, b1, b2, aeps, _dp(state["m"]), _dp(state["v"]), C.byref(t), _dp(losses))
    state["t"] = t.value
    return losses, state


# ------------------------------------------------------------------- 3D --
def fft3(x: np.ndarray, sign: int = -1) -> np.ndarray:
    z = np.ascontiguousarray(np.asarray(x, dtype=np.complex128)).copy()
    lib().or_fft3d_ri(_dp(z.view(np.float64)), z.shape[0], sign)
    return z


def solve_A3(p: Params, r) -> np.ndarray:
    r = _f64(r)
    v = np.empty_like(r)
    lib().or_solve_A3(C.byref(p), _dp(r), _dp(v))
    return v


def fine3d_step(p: Params, u) -> np.ndarray:
    """One stabilised semi-implicit step on the periodic cube (u: [n][n][n])."""
    u = _f64(u)
    out = np.empty_like(u)
    lib().or_fine3d_step(C.byref(p), _dp(u), _dp(out))
    return out


def fine3d_propagate(p: Params, steps: int, u) -> np.ndarray:
    u = _f64(u)
    out = np.empty_like(u)
    lib().or_fine3d_propagate(C.byref(p), int(steps), _dp(u), _dp(out))
    return out


class Acnn3dSpec:
    """The ResBlock ACNN with 3 x 3 x 3 convolutions (parameters
    W_l[cout][cin][3][3][3] in the 2D network's layer order)."""

    def __init__(self, channels, blocks, w, b, mass_fix=0, limiter=0, lo=-1.0, hi=1.0):
        self.w = _f64(w).ravel().copy()
        self.b = _f64(b).ravel().copy()
        self.s = Acnn(int(channels), int(blocks), int(mass_fix), int(limiter), float(lo), float(hi),
                      _dp(self.w), _dp(self.b))
        nb = C.c_long()
        nw = lib().or_acnn3d_param_counts(C.byref(self.s), C.byref(nb))
        if self.w.size != nw or self.b.size != nb.value:
            raise ValueError(f"3D ACNN C={channels} blocks={blocks} takes {nw} weights and {nb.value} biases")


def acnn3d_forward(spec: Acnn3dSpec, u) -> np.ndarray:
    u = _f64(u)
    out = np.empty_like(u)
    batch = 1 if u.ndim == 3 else u.shape[0]
    lib().or_acnn3d_forward(C.byref(spec.s), u.shape[-1], batch, _dp(u), _dp(out))
    return out


def parareal3d(p: Params, coarse, s: int, c: int, kmax: int, tol: float, u0, coarse_steps: int = 0,
               coarse_repeat: int = 1):
    """Algorithm 2 on the periodic cube: F = the 3D fine step; G = the 3D
    ACNN (coarse: Acnn3dSpec) or the 3D fine step over coarse_steps steps
    (coarse None)."""
    u0 = _f64(u0)
    n = u0.shape[-1]
    U = np.empty((s + 1, n, n, n))
    rl2 = np.zeros(kmax + 2)
    rmx = np.zeros(kmax + 2)
    it = C.c_int()
    cptr = C.byref(coarse.s) if coarse is not None else None
    g = lib().or_parareal3d(C.byref(p), cptr, int(coarse_steps), int(coarse_repeat), int(s), int(c), int(kmax),
                            float(tol), _dp(u0), _dp(U), _dp(rl2), _dp(rmx), C.byref(it))
    k = it.value
    return dict(U=U, res_l2=rl2[1:k + 1].copy(), res_max=rmx[1:k + 1].copy(), iters=k, g_calls=g)


def lap3(u, h: float) -> np.ndarray:
    u = _f64(u)
    out = np.empty_like(u)
    lib().or_lap3(u.shape[0], float(h), _dp(u), _dp(out))
    return out


# ------------------------------------------------------------------ FFT --
def fft2(x: np.ndarray, sign: int = -1) -> np.ndarray:
    z = np.ascontiguousarray(np.asarray(x, dtype=np.complex128)).copy()
    ri = z.view(np.float64)
    lib().or_fft2d_ri(_dp(ri), z.shape[0], sign)
    return z


def dft2_naive(x: np.ndarray, sign: int = -1) -> np.ndarray:
    z = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
    y = np.empty_like(z)
    lib().or_dft2d_naive_ri(_dp(z.view(np.float64)), _dp(y.view(np.float64)), z.shape[0], sign)
    return y


# ---------------------------------------------------------------- model --
def fine_step(p: Params, u) -> np.ndarray:
    u = _f64(u)
    out = np.empty_like(u)
    lib().or_fine_step(C.byref(p), _dp(u), _dp(out))
    return out


def fine_propagate(p: Params, steps: int, u) -> np.ndarray:
    u = _f64(u)
    if u.ndim == 3:
        return np.stack([fine_propagate(p, steps, x) for x in u])
    out = np.empty_like(u)
    lib().or_fine_propagate(C.byref(p), int(steps), _dp(u), _dp(out))
    return out


def cn_step(p: Params, u, tol: float = 1e-13, maxit: int = 50):
    """One Crank-Nicolson step with Picard iteration (Sec. 3.1); returns
    (U', iterations).  S in p is unused by this scheme."""
    u = _f64(u)
    out = np.empty_like(u)
    it = lib().or_cn_step(C.byref(p), _dp(u), _dp(out), float(tol), int(maxit))
    return out, int(it)


def cn_propagate(p: Params, steps: int, u, tol: float = 1e-13, maxit: int = 50):
    """`steps` Crank-Nicolson steps; returns (U, total Picard iterations)."""
    u = _f64(u)
    out = np.empty_like(u)
    it = lib().or_cn_propagate(C.byref(p), int(steps), _dp(u), _dp(out), float(tol), int(maxit))
    return out, int(it)


def solve_A(p: Params, r) -> np.ndarray:
    r = _f64(r)
    out = np.empty_like(r)
    lib().or_solve_A(C.byref(p), _dp(r), _dp(out))
    return out


def energy(p: Params, u) -> float:
    return lib().or_energy(C.byref(p), _dp(_f64(u)))


def mass(p: Params, u) -> float:
    return lib().or_mass(C.byref(p), _dp(_f64(u)))


def energy_grad(p: Params, u) -> np.ndarray:
    u = _f64(u)
    g = np.empty_like(u)
    lib().or_energy_grad(C.byref(p), _dp(u), _dp(g))
    return g


def fine_adjoint_step(p: Params, u, lam) -> np.ndarray:
    u, lam = _f64(u), _f64(lam)
    out = np.empty_like(u)
    lib().or_fine_adjoint_step(C.byref(p), _dp(u), _dp(lam), _dp(out))
    return out


def energy_gradient_through_solve(p: Params, steps: int, u0) -> np.ndarray:
    u0 = _f64(u0)
    g = np.empty_like(u0)
    lib().or_energy_gradient_through_solve(C.byref(p), int(steps), _dp(u0), _dp(g))
    return g


def round_bf16(x: float) -> float:
    return lib().or_round_bf16(float(x))


# ------------------------------------------------------------------ CNN --
def cnn_forward(spec: CnnSpec, u) -> np.ndarray:
    u = _f64(u)
    out = np.empty_like(u)
    if u.ndim == 2:
        lib().or_cnn_forward(C.byref(spec.s), u.shape[-1], _dp(u), _dp(out))
    else:
        lib().or_cnn_forward_batch(C.byref(spec.s), u.shape[-1], u.shape[0], _dp(u), _dp(out))
    return out


def cnn_backward(spec: CnnSpec, u, gout):
    u, gout = _f64(u), _f64(gout)
    gin = np.empty_like(u)
    gw = np.zeros_like(spec.w)
    gb = np.zeros_like(spec.b)
    lib().or_cnn_backward(C.byref(spec.s), u.shape[-1], _dp(u), _dp(gout), _dp(gin), _dp(gw), _dp(gb))
    return gin, gw, gb


# ------------------------------------------------------------- Parareal --
def residual(Unew, Uold):
    Unew, Uold = _f64(Unew), _f64(Uold)
    l2, mx = C.c_double(), C.c_double()
    lib().or_residual(Unew.shape[0] - 1, Unew.shape[-1], _dp(Unew), _dp(Uold), C.byref(l2), C.byref(mx))
    return l2.value, mx.value


def parareal(p: Params, coarse, s: int, c: int, kmax: int, tol: float, u0,
             coarse_steps: int = 0, literal: bool = False, coarse_repeat: int = 1):
    """Algorithm 2.  coarse: CnnSpec, AcnnSpec (the ResBlock ACNN), or None for
    G = F over coarse_steps fine steps.
    coarse_repeat > 1 composes that propagator with itself per slice (the
    remark after Algorithm 2).

    Returns dict(U=[s+1,n,n], res_l2=[...], res_max=[...], iters=k, g_calls=...).
    """
    u0 = _f64(u0)
    n = u0.shape[-1]
    U = np.empty((s + 1, n, n))
    rl2 = np.zeros(kmax + 2)
    rmx = np.zeros(kmax + 2)
    it = C.c_int()
    if isinstance(coarse, AcnnSpec):
        if literal:
            raise ValueError("the literal form is built for the conv stack only")
        g = lib().or_parareal_acnn(C.byref(p), C.byref(coarse.s), int(coarse_repeat), int(s), int(c), int(kmax),
                                   float(tol), _dp(u0), _dp(U), _dp(rl2), _dp(rmx), C.byref(it))
        k = it.value
        return dict(U=U, res_l2=rl2[1:k + 1].copy(), res_max=rmx[1:k + 1].copy(), iters=k, g_calls=g)
    cptr = C.byref(coarse.s) if coarse is not None else None
    g = lib().or_parareal_rep(C.byref(p), cptr, int(coarse_steps), int(coarse_repeat), int(s), int(c), int(kmax),
                              float(tol), int(literal), _dp(u0), _dp(U), _dp(rl2), _dp(rmx),
                              C.byref(it))
    k = it.value
    return dict(U=U, res_l2=rl2[1:k + 1].copy(), res_max=rmx[1:k + 1].copy(), iters=k, g_calls=g)
