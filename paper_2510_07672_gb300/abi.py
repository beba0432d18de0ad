"""ctypes binding of include/acpr.h: same entry-point names, argument marshalling only.

Device buffers are torch CUDA tensors (contiguous, the dtype of the call's
precision); the stream is torch's current stream unless one is passed.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

AC_OK = 0
AC_CLASSIC, AC_MASS_CONSERVING = 0, 1
AC_F64, AC_F32 = 0, 1
AC_ACT_TANH, AC_ACT_GELU = 0, 1
_ERRS = {-1: "AC_ERR_ARG", -2: "AC_ERR_UNSUPPORTED", -3: "AC_ERR_CUDA", -4: "AC_ERR_TIMEOUT",
         -5: "AC_ERR_NONFINITE", -6: "AC_ERR_NOT_CONVERGED", -7: "AC_ERR_NOMEM"}

_lock = threading.Lock()
_lib = None


class AcprError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRS.get(code, code)}: {msg}")
        self.code = code


class ac_params(C.Structure):
    _fields_ = [("n", C.c_int), ("length", C.c_double), ("eps", C.c_double), ("S", C.c_double),
                ("dt", C.c_double), ("variant", C.c_int), ("precision", C.c_int)]


class cnn_desc(C.Structure):
    _fields_ = [("layers", C.c_int), ("channels", C.c_int), ("act", C.c_int), ("residual", C.c_int),
                ("mass_fix", C.c_int), ("limiter", C.c_int), ("lo", C.c_double), ("hi", C.c_double),
                ("precision", C.c_int), ("w", C.c_void_p), ("b", C.c_void_p), ("packed", C.c_void_p),
                ("work", C.c_void_p), ("work_bytes", C.c_size_t)]


class acnn_desc(C.Structure):
    _fields_ = [("channels", C.c_int), ("blocks", C.c_int), ("mass_fix", C.c_int), ("limiter", C.c_int),
                ("lo", C.c_double), ("hi", C.c_double), ("precision", C.c_int), ("w", C.c_void_p),
                ("b", C.c_void_p)]


class ac_parareal_stats(C.Structure):
    _fields_ = [("fine_ms", C.c_double), ("coarse_ms", C.c_double), ("increment_ms", C.c_double),
                ("fine_launches", C.c_longlong), ("fine_cell_steps", C.c_longlong),
                ("coarse_calls", C.c_longlong), ("coarse_cells", C.c_longlong),
                ("iterations", C.c_longlong)]


EXPORTS = ["ac_last_error", "ac_fine_supported", "ac_fine_step", "ac_fine_propagate_slices", "ac_cn_propagate_slices",
           "cnn_packed_bytes", "cnn_work_bytes", "cnn_pack_weights", "cnn_coarse_step",
           "parareal_residual", "parareal_residual_noalloc", "ac_parareal_create", "parareal_iterate", "ac_parareal_set_active",
           "ac_parareal_trajectory", "ac_parareal_copy_trajectory", "ac_parareal_solve", "ac_parareal_create_uneven", "ac_parareal_enable_graphs",
           "ac_parareal_solve_many", "ac_parareal_reset", "ac_parareal_enable_timing", "ac_parareal_set_fine_scheme", "ac_parareal_set_coarse_substeps",
           "ac_parareal_get_stats", "ac_parareal_reset_stats", "ac_launch_count", "ac_parareal_destroy",
           "ac_fine_variant_count", "ac_fine_variant_name", "ac_fine_get_variant", "ac_fine_set_variant",
           "ac_fine_autotune", "ac_fine_propagate_work", "ac_fine_workspace_bytes", "ac_fine_propagate_slices_ws", "ac_fine_trajectory", "ac_fine_adjoint", "ac_energy", "ac_energy_grad",
           "ac_energy_gradient_workspace", "ac_energy_gradient_ic",
           "ac_conv_status", "ac_test_conv_stall", "cnn_conv_variant_count", "cnn_conv_variant_shape",
           "cnn_conv_set_variant", "cnn_conv_get_variant", "cnn_autotune", "cnn_train_bytes", "cnn_forward_train", "cnn_backward", "cnn_train_set_wgrad_tc", "cnn_adam_step", "mse_loss_grad",
           "acnn_param_count", "acnn_create", "acnn_destroy", "acnn_work_bytes", "acnn_forward", "acnn_train_bytes",
           "acnn_forward_train", "acnn_backward", "loss_acn_work_bytes", "loss_acn", "acnn_adam_step",
           "acnn_train_alg1", "acnn_train_alg1_bytes", "ac_parareal_set_coarse_acnn",
           "ac_fine3d_supported", "ac_fine3d_work_bytes", "ac_fine3d_propagate"]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libacpr.so (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"acpr library not built: {path}")
        L = C.CDLL(path)
        P, I, D, S = C.POINTER, C.c_int, C.c_double, C.c_void_p
        L.ac_last_error.restype = C.c_char_p
        L.ac_fine_supported.argtypes = [I, I]
        L.ac_fine_step.argtypes = [P(ac_params), I, S, S, S]
        L.ac_fine_propagate_slices.argtypes = [P(ac_params), I, I, S, S, S]
        L.ac_fine_workspace_bytes.argtypes = [I, I, I]
        L.ac_fine_workspace_bytes.restype = C.c_size_t
        L.ac_fine_propagate_slices_ws.argtypes = [P(ac_params), I, I, S, S, S, C.c_size_t, S]
        L.ac_cn_propagate_slices.argtypes = [P(ac_params), I, I, S, S, D, I, S, S]
        L.cnn_packed_bytes.argtypes = [P(cnn_desc)]
        L.cnn_packed_bytes.restype = C.c_size_t
        L.cnn_work_bytes.argtypes = [P(cnn_desc), I, I]
        L.cnn_work_bytes.restype = C.c_size_t
        L.cnn_pack_weights.argtypes = [P(cnn_desc), S]
        L.cnn_coarse_step.argtypes = [P(cnn_desc), I, I, S, S, S]
        L.parareal_residual.argtypes = [I, I, I, S, S, P(D), P(D), S]
        L.parareal_residual_noalloc.argtypes = [I, I, I, S, S, S, S]
        L.ac_parareal_create.argtypes = [P(ac_params), P(cnn_desc), I, I, I, S, P(S)]
        L.parareal_iterate.argtypes = [S, P(I), P(D), P(D), S]
        L.ac_parareal_set_active.argtypes = [S, I, I]
        L.ac_parareal_trajectory.argtypes = [S]
        L.ac_parareal_trajectory.restype = S
        L.ac_parareal_copy_trajectory.argtypes = [S, S, S]
        L.ac_parareal_solve.argtypes = [S, D, I, P(I), P(D), S]
        L.ac_parareal_set_fine_scheme.argtypes = [S, I, D, I]
        L.ac_parareal_set_coarse_substeps.argtypes = [S, I]
        L.ac_parareal_create_uneven.argtypes = [P(ac_params), P(cnn_desc), I, P(I), P(I), S, P(S)]
        L.ac_parareal_enable_graphs.argtypes = [S, I]
        L.ac_parareal_solve_many.argtypes = [P(S), I, P(S), D, I, P(I), P(D)]
        L.ac_parareal_reset.argtypes = [S, S, S]
        L.ac_parareal_enable_timing.argtypes = [S, I]
        L.ac_parareal_get_stats.argtypes = [S, P(ac_parareal_stats)]
        L.ac_parareal_reset_stats.argtypes = [S]
        L.ac_launch_count.restype = C.c_longlong
        L.ac_fine_variant_count.argtypes = [I, I]
        L.ac_fine_variant_name.argtypes = [I, I, I]
        L.ac_fine_variant_name.restype = C.c_char_p
        L.ac_fine_get_variant.argtypes = [I, I]
        L.ac_fine_set_variant.argtypes = [I, I, I]
        L.ac_fine_autotune.argtypes = [P(ac_params), I, I, S, S, P(C.c_float), S]
        L.ac_fine_trajectory.argtypes = [P(ac_params), I, I, S, S, S]
        L.ac_fine_propagate_work.argtypes = [P(ac_params), I, S, S, S, S]
        L.ac_fine_adjoint.argtypes = [P(ac_params), I, I, S, S, S, S]
        L.ac_energy.argtypes = [P(ac_params), I, S, S, S]
        L.ac_energy_grad.argtypes = [P(ac_params), I, S, S, S]
        L.ac_energy_gradient_workspace.argtypes = [P(ac_params), I, I]
        L.ac_energy_gradient_workspace.restype = C.c_size_t
        L.ac_energy_gradient_ic.argtypes = [P(ac_params), I, I, S, S, S, C.c_size_t, S]
        L.ac_conv_status.argtypes = [S, S]
        L.cnn_conv_variant_count.argtypes = [I, I]
        L.cnn_conv_variant_shape.argtypes = [I, I, I, P(I), P(I)]
        L.cnn_conv_set_variant.argtypes = [I, I, I]
        L.cnn_conv_get_variant.argtypes = [I, I]
        L.cnn_autotune.argtypes = [P(cnn_desc), I, I, S, S, P(C.c_float), S]
        L.ac_test_conv_stall.argtypes = [I]
        L.cnn_train_bytes.argtypes = [P(cnn_desc), I, I]
        L.cnn_train_bytes.restype = C.c_size_t
        L.cnn_forward_train.argtypes = [P(cnn_desc), I, I, S, S, S, S]
        L.cnn_backward.argtypes = [P(cnn_desc), I, I, S, S, S, S, S, I, S, S]
        L.cnn_adam_step.argtypes = [S, S, S, S, C.c_longlong, D, D, D, D, I, S]
        L.cnn_train_set_wgrad_tc.argtypes = [I]
        L.mse_loss_grad.argtypes = [S, S, C.c_longlong, D, S, I, S, S, I, S]
        L.ac_parareal_destroy.argtypes = [S]
        L.ac_parareal_destroy.restype = None
        L.acnn_param_count.argtypes = [I, I, P(C.c_longlong)]
        L.acnn_param_count.restype = C.c_longlong
        L.acnn_create.argtypes = [P(acnn_desc), P(S)]
        L.acnn_destroy.argtypes = [S]
        L.acnn_destroy.restype = None
        L.acnn_work_bytes.argtypes = [S, I, I]
        L.acnn_work_bytes.restype = C.c_size_t
        L.acnn_forward.argtypes = [S, I, I, S, S, S, C.c_size_t, S]
        L.acnn_train_bytes.argtypes = [P(acnn_desc), I, I]
        L.acnn_train_bytes.restype = C.c_size_t
        L.acnn_forward_train.argtypes = [P(acnn_desc), I, I, S, S, S, S]
        L.acnn_backward.argtypes = [P(acnn_desc), I, I, S, S, S, S, S, S]
        L.loss_acn_work_bytes.argtypes = [I, I]
        L.loss_acn_work_bytes.restype = C.c_size_t
        L.loss_acn.argtypes = [P(ac_params), I, S, S, S, S, S, S]
        L.acnn_adam_step.argtypes = [I, S, S, S, S, C.c_longlong, D, D, D, D, I, S]
        L.acnn_train_alg1.argtypes = [P(ac_params), P(acnn_desc), I, S, P(I), I, I, I, I, D, D, D, D, S, S, P(I),
                                      S, S, C.c_size_t, S]
        L.acnn_train_alg1_bytes.argtypes = [P(acnn_desc), I, I]
        L.acnn_train_alg1_bytes.restype = C.c_size_t
        L.ac_parareal_set_coarse_acnn.argtypes = [S, S]
        L.ac_fine3d_supported.argtypes = [I, I]
        L.ac_fine3d_work_bytes.argtypes = [I, I, I]
        L.ac_fine3d_work_bytes.restype = C.c_size_t
        L.ac_fine3d_propagate.argtypes = [P(ac_params), I, I, S, S, S, C.c_size_t, S]
        _lib = L
        return L


def _check(rc: int):
    if rc != AC_OK:
        raise AcprError(rc, load().ac_last_error().decode())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dtype(precision):
    import torch
    return torch.float64 if precision == AC_F64 else torch.float32


def _dev(t, dtype=None, name="tensor"):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (no CPU path exists)")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


class FineParams:
    """Python view of ac_params (Sec. 3.1 problem statement)."""

    def __init__(self, n, eps, S, dt, variant=AC_CLASSIC, precision=AC_F32, length=1.0):
        self.n, self.eps, self.S, self.dt = int(n), float(eps), float(S), float(dt)
        self.variant, self.precision, self.length = int(variant), int(precision), float(length)

    def c(self) -> ac_params:
        return ac_params(self.n, self.length, self.eps, self.S, self.dt, self.variant, self.precision)

    @property
    def dtype(self):
        return _dtype(self.precision)


def ac_fine_supported(n: int, precision: int) -> bool:
    return bool(load().ac_fine_supported(int(n), int(precision)))


def ac_fine_step(params: FineParams, u_in, u_out=None, stream=None):
    u_out = u_out if u_out is not None else u_in.new_empty(u_in.shape)
    batch = u_in.numel() // (params.n * params.n)
    p = params.c()
    _check(load().ac_fine_step(C.byref(p), batch, _dev(u_in, params.dtype, "u_in"),
                               _dev(u_out, params.dtype, "u_out"), _stream(stream)))
    return u_out


def ac_cn_propagate_slices(params: FineParams, steps: int, u_in, u_out=None, tol: float = 1e-6,
                           max_iters: int = 50, iters=None, stream=None):
    """Crank-Nicolson steps with Picard iteration (Sec. 3.1) for every field of
    u_in.  iters: optional device int32 tensor [fields] for the total Picard
    iterations per field."""
    import torch
    u_out = u_out if u_out is not None else u_in.new_empty(u_in.shape)
    fields = u_in.numel() // (params.n * params.n)
    p = params.c()
    it_ptr = None
    if iters is not None:
        it_ptr = _dev(iters, torch.int32, "iters")
    _check(load().ac_cn_propagate_slices(C.byref(p), fields, int(steps), _dev(u_in, params.dtype, "u_in"),
                                         _dev(u_out, params.dtype, "u_out"), float(tol), int(max_iters), it_ptr,
                                         _stream(stream)))
    return u_out


def ac_fine_propagate_slices(params: FineParams, steps: int, u_in, u_out=None, stream=None):
    u_out = u_out if u_out is not None else u_in.new_empty(u_in.shape)
    fields = u_in.numel() // (params.n * params.n)
    p = params.c()
    _check(load().ac_fine_propagate_slices(C.byref(p), fields, int(steps), _dev(u_in, params.dtype, "u_in"),
                                           _dev(u_out, params.dtype, "u_out"), _stream(stream)))
    return u_out


def ac_fine_workspace_bytes(n: int, num_fields: int, precision: int) -> int:
    return int(load().ac_fine_workspace_bytes(int(n), int(num_fields), int(precision)))


def ac_fine_propagate_slices_ws(params: FineParams, steps: int, u_in, u_out, workspace, stream=None):
    """ac_fine_propagate_slices with a caller-owned workspace (uint8 device
    tensor of ac_fine_workspace_bytes bytes; the call allocates nothing)."""
    fields = u_in.numel() // (params.n * params.n)
    p = params.c()
    ws = _dev(workspace, None, "workspace") if workspace is not None else None
    nbytes = workspace.numel() if workspace is not None else 0
    _check(load().ac_fine_propagate_slices_ws(C.byref(p), fields, int(steps), _dev(u_in, params.dtype, "u_in"),
                                              _dev(u_out, params.dtype, "u_out"), ws, nbytes, _stream(stream)))
    return u_out


def ac_fine_variants(n: int, precision: int):
    L = load()
    return [L.ac_fine_variant_name(int(n), int(precision), i).decode()
            for i in range(L.ac_fine_variant_count(int(n), int(precision)))]


def ac_fine_set_variant(n: int, precision: int, index: int):
    _check(load().ac_fine_set_variant(int(n), int(precision), int(index)))


def ac_fine_get_variant(n: int, precision: int) -> int:
    return int(load().ac_fine_get_variant(int(n), int(precision)))


def ac_fine_autotune(params: FineParams, steps: int, u_in, u_out, stream=None):
    """Time every launch shape on this problem, keep the fastest; returns
    {name: ms per call} and the chosen index."""
    L = load()
    cnt = L.ac_fine_variant_count(params.n, params.precision)
    ms = (C.c_float * max(cnt, 1))()
    fields = u_in.numel() // (params.n * params.n)
    p = params.c()
    _check(L.ac_fine_autotune(C.byref(p), fields, int(steps), _dev(u_in, params.dtype, "u_in"),
                              _dev(u_out, params.dtype, "u_out"), ms, _stream(stream)))
    names = ac_fine_variants(params.n, params.precision)
    return {names[i]: ms[i] for i in range(cnt)}, ac_fine_get_variant(params.n, params.precision)


def ac_fine_propagate_work(params: FineParams, work, u_in, u_out, stream=None):
    """work: int32 CUDA tensor [count][4] = (in field, out field, steps, 0)."""
    import torch
    count = work.shape[0]
    p = params.c()
    _check(load().ac_fine_propagate_work(C.byref(p), count, _dev(work, torch.int32, "work"),
                                         _dev(u_in, params.dtype, "u_in"), _dev(u_out, params.dtype, "u_out"),
                                         _stream(stream)))
    return u_out


def ac_fine_trajectory(params: FineParams, steps: int, u0, traj=None, stream=None):
    """traj[s][f] = u^s, s = 0..steps (device tensor [steps+1][fields][n][n])."""
    import torch
    n = params.n
    fields = u0.numel() // (n * n)
    if traj is None:
        traj = torch.empty((steps + 1, fields, n, n), dtype=params.dtype, device=u0.device)
    p = params.c()
    _check(load().ac_fine_trajectory(C.byref(p), fields, int(steps), _dev(u0, params.dtype, "u0"),
                                     _dev(traj, params.dtype, "traj"), _stream(stream)))
    return traj


def ac_fine_adjoint(params: FineParams, steps: int, states, lam_end, lam_start=None, stream=None):
    n = params.n
    fields = lam_end.numel() // (n * n)
    lam_start = lam_start if lam_start is not None else lam_end.new_empty(lam_end.shape)
    p = params.c()
    _check(load().ac_fine_adjoint(C.byref(p), fields, int(steps), _dev(states, params.dtype, "states"),
                                  _dev(lam_end, params.dtype, "lam_end"), _dev(lam_start, params.dtype, "lam_start"),
                                  _stream(stream)))
    return lam_start


def ac_energy(params: FineParams, u, stream=None):
    import torch
    n = params.n
    fields = u.numel() // (n * n)
    e = torch.empty(fields, dtype=torch.float64, device=u.device)
    p = params.c()
    _check(load().ac_energy(C.byref(p), fields, _dev(u, params.dtype, "u"), _dev(e, torch.float64, "e"),
                            _stream(stream)))
    return e


def ac_energy_grad(params: FineParams, u, g=None, stream=None):
    n = params.n
    fields = u.numel() // (n * n)
    g = g if g is not None else u.new_empty(u.shape)
    p = params.c()
    _check(load().ac_energy_grad(C.byref(p), fields, _dev(u, params.dtype, "u"), _dev(g, params.dtype, "g"),
                                 _stream(stream)))
    return g


def ac_energy_gradient_ic(params: FineParams, steps: int, u0, checkpoint_every=32, stream=None):
    """dE_h(u^steps)/du0 for one field by the checkpointed adjoint."""
    import torch
    p = params.c()
    nbytes = load().ac_energy_gradient_workspace(C.byref(p), int(steps), int(checkpoint_every))
    ws = torch.empty(nbytes, dtype=torch.uint8, device=u0.device)
    g = u0.new_empty(u0.shape)
    _check(load().ac_energy_gradient_ic(C.byref(p), int(steps), int(checkpoint_every), _dev(u0, params.dtype, "u0"),
                                        _dev(g, params.dtype, "grad"), _dev(ws, None, "ws"), nbytes, _stream(stream)))
    return g


class CoarseNet:
    """Device-side conv stack G (Sec. 3.2): owns torch buffers for the weights,
    the packed bf16 copy and the activation workspace."""

    def __init__(self, layers, channels, w, b, act=AC_ACT_TANH, precision=AC_F32, residual=1,
                 mass_fix=0, limiter=0, lo=-1.0, hi=1.0, device="cuda"):
        import torch
        dt = _dtype(precision)
        self.layers, self.channels, self.act, self.precision = int(layers), int(channels), int(act), int(precision)
        self.residual, self.mass_fix, self.limiter, self.lo, self.hi = int(residual), int(mass_fix), int(limiter), float(lo), float(hi)
        self.w = torch.as_tensor(w, dtype=dt).to(device).contiguous()
        self.b = torch.as_tensor(b, dtype=dt).to(device).contiguous()
        self._packed = None
        self._work = None
        d = self.desc()
        nb = load().cnn_packed_bytes(C.byref(d))
        if nb:
            self._packed = torch.empty(nb, dtype=torch.uint8, device=device)
        self.repack()

    def desc(self) -> cnn_desc:
        return cnn_desc(self.layers, self.channels, self.act, self.residual, self.mass_fix, self.limiter,
                        self.lo, self.hi, self.precision, self.w.data_ptr(), self.b.data_ptr(),
                        self._packed.data_ptr() if self._packed is not None else None,
                        self._work.data_ptr() if self._work is not None else None,
                        self._work.numel() if self._work is not None else 0)

    def repack(self, stream=None):
        if self._packed is not None:
            d = self.desc()
            _check(load().cnn_pack_weights(C.byref(d), _stream(stream)))

    def ensure_work(self, n, batch):
        import torch
        d = self.desc()
        need = load().cnn_work_bytes(C.byref(d), int(n), int(batch))
        if self._work is None or self._work.numel() < need:
            # zeros: the workspace header holds the conv kernels' status word
            self._work = torch.zeros(max(need, 256), dtype=torch.uint8, device=self.w.device)


class TrainableCoarseNet(CoarseNet):
    """CoarseNet (AC_F32) with float32 gradient buffers and Adam moments, for
    training G to step the fine operator (Sec. 3.2)."""

    def __init__(self, layers, channels, w, b, act=AC_ACT_GELU, mass_fix=0, device="cuda"):
        import torch
        super().__init__(layers, channels, w, b, act=act, precision=AC_F32, mass_fix=mass_fix, device=device)
        self.gw = torch.zeros_like(self.w)
        self.gb = torch.zeros_like(self.b)
        self.mw, self.vw = torch.zeros_like(self.w), torch.zeros_like(self.w)
        self.mb, self.vb = torch.zeros_like(self.b), torch.zeros_like(self.b)
        self.t = 0

    def train_bytes(self, n, batch):
        d = self.desc()
        return load().cnn_train_bytes(C.byref(d), int(n), int(batch))

    def new_workspace(self, n, batch):
        import torch
        # zeros: the workspace header holds the conv kernels' status word
        return torch.zeros(self.train_bytes(n, batch), dtype=torch.uint8, device=self.w.device)

    def forward_train(self, u, ws, out=None, stream=None):
        n = u.shape[-1]
        batch = u.numel() // (n * n)
        out = out if out is not None else torch_empty_like(u)
        d = self.desc()
        _check(load().cnn_forward_train(C.byref(d), n, batch, _dev(u, None, "u"), _dev(out, None, "out"),
                                        _dev(ws, None, "ws"), _stream(stream)))
        return out

    def backward(self, u, grad_out, ws, grad_in=None, accumulate=False, stream=None):
        n = u.shape[-1]
        batch = u.numel() // (n * n)
        d = self.desc()
        gi = _dev(grad_in, None, "grad_in") if grad_in is not None else None
        _check(load().cnn_backward(C.byref(d), n, batch, _dev(u, None, "u"), _dev(grad_out, None, "grad_out"), gi,
                                   _dev(self.gw, None, "gw"), _dev(self.gb, None, "gb"), int(accumulate),
                                   _dev(ws, None, "ws"), _stream(stream)))
        return grad_in

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        self.t += 1
        for w, g, m, v in ((self.w, self.gw, self.mw, self.vw), (self.b, self.gb, self.mb, self.vb)):
            _check(load().cnn_adam_step(_dev(w), _dev(g), _dev(m), _dev(v), w.numel(), lr, beta1, beta2, eps,
                                        self.t, _stream(stream)))
        self.repack(stream)


def torch_empty_like(t):
    import torch
    return torch.empty_like(t)


def mse_loss_grad(pred, target, scale, grad=None, grad_accumulate=False, loss=None, scratch=None,
                  accumulate=False, stream=None):
    """scale * sum (pred - target)^2 into loss[0] (float64 device tensor) and
    its gradient into grad (float32), both with our kernels."""
    import torch
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float64, device=pred.device)
    if scratch is None:
        scratch = torch.empty(64, dtype=torch.float64, device=pred.device)
    g = _dev(grad, torch.float32, "grad") if grad is not None else None
    _check(load().mse_loss_grad(_dev(pred, torch.float32, "pred"), _dev(target, torch.float32, "target"),
                                pred.numel(), float(scale), g, int(grad_accumulate), _dev(loss, torch.float64, "loss"),
                                _dev(scratch, torch.float64, "scratch"), int(accumulate), _stream(stream)))
    return loss


def ac_fine3d_propagate(params: FineParams, steps: int, u_in, u_out=None, work=None, stream=None):
    """`steps` fine steps of the fields u_in [F][n][n][n] on the periodic cube."""
    import torch
    n = params.n
    if u_in.shape[-3:] != (n, n, n):
        raise ValueError(f"fields must be [F][{n}][{n}][{n}]")
    F = u_in.numel() // (n ** 3)
    u_out = u_out if u_out is not None else torch.empty_like(u_in)
    need = load().ac_fine3d_work_bytes(n, F, params.precision)
    if need == 0:
        raise AcprError(-2, f"3D fine step not built for n={n}")
    if work is None or work.numel() < need:
        work = torch.empty(need, dtype=torch.uint8, device=u_in.device)
    p = params.c()
    _check(load().ac_fine3d_propagate(C.byref(p), int(steps), F, _dev(u_in, params.dtype, "u_in"),
                                      _dev(u_out, params.dtype, "u_out"), _dev(work, None, "work"), need,
                                      _stream(stream)))
    return u_out


def acnn_param_count(channels: int, blocks: int):
    """(number of weights, number of biases) of the ResBlock ACNN."""
    nb = C.c_longlong()
    nw = load().acnn_param_count(int(channels), int(blocks), C.byref(nb))
    if nw < 0:
        raise AcprError(-2, f"ACNN C={channels} blocks={blocks} not built")
    return int(nw), int(nb.value)


class Acnn:
    """The paper's ResBlock ACNN / mACNN coarse network (Sec. 3.2).

    Parameters live on the device (w, b, in the layouts of include/acpr.h) and
    train in place; `handle()` builds the inference handle (parameters baked
    into the kernel argument) and is rebuilt after every update."""

    def __init__(self, channels, blocks, w, b, mass_fix=0, limiter=0, lo=-1.0, hi=1.0, precision=AC_F32,
                 device="cuda"):
        import torch
        self.channels, self.blocks = int(channels), int(blocks)
        self.mass_fix, self.limiter, self.lo, self.hi = int(mass_fix), int(limiter), float(lo), float(hi)
        self.precision = int(precision)
        dt = _dtype(self.precision)
        nw, nb = acnn_param_count(self.channels, self.blocks)
        self.w = torch.as_tensor(w, dtype=dt).reshape(-1).to(device).contiguous()
        self.b = torch.as_tensor(b, dtype=dt).reshape(-1).to(device).contiguous()
        if self.w.numel() != nw or self.b.numel() != nb:
            raise ValueError(f"ACNN C={channels} blocks={blocks} takes {nw} weights and {nb} biases")
        self.nw, self.nb = nw, nb
        self._h = None
        self._retired = []   # earlier handles: a Parareal handle may still point at one
        self._work = {}
        self.m = self.v = None
        self.t = 0

    def desc(self) -> acnn_desc:
        return acnn_desc(self.channels, self.blocks, self.mass_fix, self.limiter, self.lo, self.hi, self.precision,
                         self.w.data_ptr(), self.b.data_ptr())

    def handle(self):
        if self._h is None:
            h = C.c_void_p()
            d = self.desc()
            _check(load().acnn_create(C.byref(d), C.byref(h)))
            self._h = h
        return self._h

    def invalidate(self):
        """Retire the inference handle (call after changing w or b in place);
        the next use builds a new one.  Retired handles are freed with the
        object, since a Parareal handle may still point at one until it
        re-attaches (it does so before every iteration)."""
        if self._h is not None:
            self._retired.append(self._h)
            self._h = None

    def _free_handles(self):
        L = load()
        for h in self._retired + ([self._h] if self._h is not None else []):
            L.acnn_destroy(h)
        self._retired, self._h = [], None

    def __call__(self, u, out=None, stream=None):
        """G(u) for u [batch][n][n] (or [n][n]) through the inference handle."""
        import torch
        n = u.shape[-1]
        batch = u.numel() // (n * n)
        h = self.handle()
        need = load().acnn_work_bytes(h, n, batch)
        key = (n, batch)
        if key not in self._work or self._work[key].numel() < need:
            self._work[key] = torch.empty(max(need, 1), dtype=torch.uint8, device=u.device)
        out = out if out is not None else torch.empty_like(u)
        dt = _dtype(self.precision)
        _check(load().acnn_forward(h, n, batch, _dev(u, dt, "u"), _dev(out, dt, "out"),
                                   _dev(self._work[key], None, "work"), need, _stream(stream)))
        return out

    def new_workspace(self, n, batch):
        import torch
        d = self.desc()
        nb = load().acnn_train_bytes(C.byref(d), int(n), int(batch))
        return torch.empty(max(nb, 1), dtype=torch.uint8, device=self.w.device)

    def forward_train(self, u, ws, out=None, stream=None):
        import torch
        n = u.shape[-1]
        batch = u.numel() // (n * n)
        out = out if out is not None else torch.empty_like(u)
        d = self.desc()
        dt = _dtype(self.precision)
        _check(load().acnn_forward_train(C.byref(d), n, batch, _dev(u, dt, "u"), _dev(out, dt, "out"),
                                         _dev(ws, None, "ws"), _stream(stream)))
        return out

    def backward(self, u, grad_out, ws, gw=None, gb=None, stream=None):
        """(dL/dw, dL/db) of the last forward_train for grad_out = dL/d(output)."""
        import torch
        n = u.shape[-1]
        batch = u.numel() // (n * n)
        gw = gw if gw is not None else torch.empty_like(self.w)
        gb = gb if gb is not None else torch.empty_like(self.b)
        d = self.desc()
        dt = _dtype(self.precision)
        _check(load().acnn_backward(C.byref(d), n, batch, _dev(u, dt, "u"), _dev(grad_out, dt, "grad_out"),
                                    _dev(gw, dt, "gw"), _dev(gb, dt, "gb"), _dev(ws, None, "ws"), _stream(stream)))
        return gw, gb

    def _moments(self):
        import torch
        if self.m is None:
            self.m = torch.zeros(self.nw + self.nb, dtype=self.w.dtype, device=self.w.device)
            self.v = torch.zeros_like(self.m)

    def adam(self, gw, gb, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        """One Adam step on w and b (moments held by the object)."""
        self._moments()
        self.t += 1
        dt = _dtype(self.precision)
        for par, g, off in ((self.w, gw, 0), (self.b, gb, self.nw)):
            _check(load().acnn_adam_step(self.precision, _dev(par, dt, "w"), _dev(g, dt, "grad"),
                                         C.c_void_p(self.m.data_ptr() + off * self.m.element_size()),
                                         C.c_void_p(self.v.data_ptr() + off * self.v.element_size()),
                                         par.numel(), lr, beta1, beta2, eps, self.t, _stream(stream)))
        self.invalidate()

    def train_alg1(self, params: FineParams, U0s, perm, q, steps, b_inner, lr=1e-3, beta1=0.9, beta2=0.999,
                   eps=1e-8, stream=None):
        """Algorithm 1 with the scheme-residual loss at time step params.dt.
        perm: int array [epochs][R].  Returns the losses (float64 device
        tensor, one per update)."""
        import numpy as np
        import torch
        self._moments()
        perm = np.ascontiguousarray(perm, dtype=np.int32)
        epochs, R = perm.shape
        losses = torch.zeros(max(epochs * (R // q) * steps * b_inner, 1), dtype=torch.float64, device=self.w.device)
        p = params.c()
        d = self.desc()
        t = C.c_int(self.t)
        nbytes = load().acnn_train_alg1_bytes(C.byref(d), int(params.n), int(q))
        if getattr(self, "_alg1_ws", None) is None or self._alg1_ws.numel() < nbytes:
            self._alg1_ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.w.device)
        _check(load().acnn_train_alg1(C.byref(p), C.byref(d), R, _dev(U0s, _dtype(self.precision), "U0s"),
                                      perm.ctypes.data_as(C.POINTER(C.c_int)), epochs, int(q), int(steps),
                                      int(b_inner), lr, beta1, beta2, eps, C.c_void_p(self.m.data_ptr()),
                                      C.c_void_p(self.v.data_ptr()), C.byref(t),
                                      _dev(losses, torch.float64, "losses"), _dev(self._alg1_ws, None, "ws"),
                                      self._alg1_ws.numel(), _stream(stream)))
        self.t = t.value
        self.invalidate()
        return losses[: epochs * (R // q) * steps * b_inner]

    def __del__(self):
        try:
            self._free_handles()
        except Exception:
            pass


def loss_acn(params: FineParams, U0, U1, grad=True, stream=None):
    """Eq. loss_ACN at time step params.dt: (loss as a float64 device tensor
    of one element, dL/dU1 or None), computed by the library's kernels."""
    import torch
    n = U0.shape[-1]
    batch = U0.numel() // (n * n)
    dt = params.dtype
    work = torch.empty(load().loss_acn_work_bytes(n, batch), dtype=torch.uint8, device=U0.device)
    loss = torch.zeros(1, dtype=torch.float64, device=U0.device)
    g = torch.empty_like(U1) if grad else None
    p = params.c()
    _check(load().loss_acn(C.byref(p), batch, _dev(U0, dt, "U0"), _dev(U1, dt, "U1"),
                           _dev(loss, torch.float64, "loss"), _dev(g, dt, "grad") if grad else None,
                           _dev(work, None, "work"), _stream(stream)))
    return loss, g


def coarse_step_function():
    """torch.autograd.Function over the conv stack: forward = cnn_forward_train,
    backward = cnn_backward (gradients for u, w and b)."""
    import torch

    class CoarseStep(torch.autograd.Function):
        @staticmethod
        def forward(ctx, u, w, b, net):
            n = u.shape[-1]
            batch = u.numel() // (n * n)
            ws = net.new_workspace(n, batch)
            out = net.forward_train(u.contiguous(), ws)
            ctx.save_for_backward(u)
            ctx.ws, ctx.net = ws, net
            return out

        @staticmethod
        def backward(ctx, gout):
            (u,) = ctx.saved_tensors
            net = ctx.net
            du = torch.empty_like(u)
            net.backward(u.contiguous(), gout.contiguous(), ctx.ws, grad_in=du, accumulate=False)
            return du, net.gw.clone(), net.gb.clone(), None

    return CoarseStep


def fine_solve_function():
    """torch.autograd.Function over `steps` fine steps of a batch of fields
    (the stabilised scheme of ac_params, Sec. 3.1), for gradients of any
    scalar loss of the final fields through long rollouts.

    forward(u0, params, steps, checkpoint_every): u^steps from u0 [.., n, n],
    keeping only the fields at every `checkpoint_every`-th step (one segment
    start each).  backward: for each segment, last first, the library
    recomputes the segment's states from its checkpoint (ac_fine_trajectory)
    and runs the transposed steps through them (ac_fine_adjoint), so memory is
    (steps / checkpoint_every + checkpoint_every) fields per field.  Every
    step of both passes runs in the library's kernels."""
    import torch

    class FineSolve(torch.autograd.Function):
        @staticmethod
        def forward(ctx, u0, params, steps, checkpoint_every=32):
            if steps < 0 or checkpoint_every < 1:
                raise ValueError("need steps >= 0 and checkpoint_every >= 1")
            u = u0.contiguous()
            ckpts, lens = [], []
            done = 0
            while done < steps:
                seg = min(checkpoint_every, steps - done)
                ckpts.append(u)
                lens.append(seg)
                u = ac_fine_propagate_slices(params, seg, u)
                done += seg
            ctx.params, ctx.lens = params, lens
            ctx.save_for_backward(*ckpts)
            return u if steps else u.clone()

        @staticmethod
        def backward(ctx, gout):
            params, lens = ctx.params, ctx.lens
            ckpts = ctx.saved_tensors
            lam = gout.contiguous()
            for u_start, seg in zip(reversed(ckpts), reversed(lens)):
                traj = ac_fine_trajectory(params, seg, u_start)
                lam = ac_fine_adjoint(params, seg, traj[:seg].contiguous(), lam)
            return lam, None, None, None

    return FineSolve


def fine_solve(u0, params: FineParams, steps: int, checkpoint_every: int = 32):
    """u^steps = F_1^steps(u0), differentiable with respect to u0 (see
    fine_solve_function)."""
    return fine_solve_function().apply(u0, params, int(steps), int(checkpoint_every))


def cnn_packed_bytes(net: CoarseNet) -> int:
    d = net.desc()
    return load().cnn_packed_bytes(C.byref(d))


def cnn_work_bytes(net: CoarseNet, n: int, batch: int) -> int:
    d = net.desc()
    return load().cnn_work_bytes(C.byref(d), int(n), int(batch))


def cnn_pack_weights(net: CoarseNet, stream=None):
    net.repack(stream)


def cnn_coarse_step(net: CoarseNet, u_in, u_out=None, stream=None):
    n = u_in.shape[-1]
    batch = u_in.numel() // (n * n)
    net.ensure_work(n, batch)
    u_out = u_out if u_out is not None else u_in.new_empty(u_in.shape)
    d = net.desc()
    dt = _dtype(net.precision)
    _check(load().cnn_coarse_step(C.byref(d), n, batch, _dev(u_in, dt, "u_in"), _dev(u_out, dt, "u_out"),
                                  _stream(stream)))
    return u_out


def cnn_conv_variants(n: int, channels: int):
    """[(input-ring depth, TMEM slots)] of the persistent row-streaming
    tensor-core conv for (n, channels)."""
    L = load()
    out = []
    for i in range(L.cnn_conv_variant_count(int(n), int(channels))):
        a, b = C.c_int(), C.c_int()
        _check(L.cnn_conv_variant_shape(int(n), int(channels), i, C.byref(a), C.byref(b)))
        out.append((a.value, b.value))
    return out


def cnn_conv_set_variant(n: int, channels: int, index: int):
    _check(load().cnn_conv_set_variant(int(n), int(channels), int(index)))


def cnn_autotune(net, u_in, u_out=None, stream=None):
    """Time every shape of the persistent conv kernel on this problem, keep the fastest; returns
    {shape: ms per call} and the chosen index."""
    n = u_in.shape[-1]
    batch = u_in.numel() // (n * n)
    net.ensure_work(n, batch)
    u_out = u_out if u_out is not None else u_in.new_empty(u_in.shape)
    shapes = cnn_conv_variants(n, net.channels)
    ms = (C.c_float * max(len(shapes), 1))()
    d = net.desc()
    _check(load().cnn_autotune(C.byref(d), n, batch, _dev(u_in, None, "u_in"), _dev(u_out, None, "u_out"), ms,
                               _stream(stream)))
    return {shapes[i]: ms[i] for i in range(len(shapes))}, int(load().cnn_conv_get_variant(n, net.channels))


def ac_conv_status(workspace, stream=None):
    """Raise AC_ERR_TIMEOUT if a tensor-core conv kernel that used this
    workspace (CoarseNet work or a training workspace) gave up a bounded wait
    since the last check; clears the status word."""
    _check(load().ac_conv_status(_dev(workspace, None, "workspace"), _stream(stream)))


def ac_test_conv_stall(polls: int):
    """Test hook: polls > 0 makes the persistent tensor-core conv kernels wait,
    for that many polls, on an mbarrier nothing arrives on (0 turns it off)."""
    _check(load().ac_test_conv_stall(int(polls)))


def cnn_train_set_wgrad_tc(on: bool):
    """Hidden-layer weight gradients of cnn_backward on the tensor cores (True,
    default; C = 64, n a multiple of 128) or on the CUDA cores (False)."""
    _check(load().cnn_train_set_wgrad_tc(int(bool(on))))


def parareal_solve_many(handles, streams, tol, kmax, allow_unconverged=False):
    """ac_parareal_solve_many over Parareal handles (one stream each)."""
    L = load()
    for h in handles:
        h._sync_acnn()
    total = sum(h.problems for h in handles)
    hs = (C.c_void_p * len(handles))(*[h._h.value for h in handles])
    ss = (C.c_void_p * len(handles))(*[s.cuda_stream for s in streams])
    it = (C.c_int * total)()
    l2 = (C.c_double * total)()
    rc = L.ac_parareal_solve_many(hs, len(handles), ss, float(tol), int(kmax), it, l2)
    if rc != AC_OK and not (allow_unconverged and rc == -6):
        _check(rc)
    out, i = [], 0
    for h in handles:
        out.append((list(it[i:i + h.problems]), list(l2[i:i + h.problems])))
        h.k = max(h.k, max(it[i:i + h.problems]) + 1)
        i += h.problems
    return out


def ac_launch_count() -> int:
    return int(load().ac_launch_count())


def parareal_residual(U_new, U_old, precision=None, stream=None):
    """(rel_l2, max_abs) between two [s+1][n][n] trajectories (slices 1..s)."""
    import torch
    precision = precision if precision is not None else (AC_F64 if U_new.dtype == torch.float64 else AC_F32)
    s = U_new.shape[0] - 1
    n = U_new.shape[-1]
    l2, mx = C.c_double(), C.c_double()
    dt = _dtype(precision)
    _check(load().parareal_residual(s, n, precision, _dev(U_new, dt, "U_new"), _dev(U_old, dt, "U_old"),
                                    C.byref(l2), C.byref(mx), _stream(stream)))
    return l2.value, mx.value


def parareal_residual_noalloc(U_new, U_old, out, precision=None, stream=None):
    """Allocation-free variant: writes (rel_l2, max_abs, sum d^2, sum U_new^2)
    into the float64 CUDA tensor `out` (4 elements) without a host read-back."""
    import torch
    precision = precision if precision is not None else (AC_F64 if U_new.dtype == torch.float64 else AC_F32)
    s = U_new.shape[0] - 1
    n = U_new.shape[-1]
    dt = _dtype(precision)
    _check(load().parareal_residual_noalloc(s, n, precision, _dev(U_new, dt, "U_new"), _dev(U_old, dt, "U_old"),
                                            _dev(out, torch.float64, "out"), _stream(stream)))
    return out


class Parareal:
    """Handle on ac_parareal: Algorithm 2 for `problems` independent problems.
    `slices` / `steps` may be per-problem sequences (ac_parareal_create_uneven)."""

    def __init__(self, params: FineParams, net, u0, slices, steps):
        """net: a CoarseNet (the conv stack) or an Acnn (the paper's ResBlock
        network, Sec. 3.2)."""
        self.params, self.net = params, net
        self.problems = u0.shape[0] if u0.dim() == 3 else 1
        self._u0 = u0.contiguous()
        p = params.c()
        acnn = net if isinstance(net, Acnn) else None
        d = None if acnn is not None else net.desc()
        dref = C.byref(d) if d is not None else None
        h = C.c_void_p()
        if isinstance(slices, int) and isinstance(steps, int):
            self.s, self.c = int(slices), int(steps)
            _check(load().ac_parareal_create(C.byref(p), dref, self.problems, self.s, self.c,
                                             _dev(self._u0, params.dtype, "u0"), C.byref(h)))
        else:
            sl = [int(x) for x in (slices if not isinstance(slices, int) else [slices] * self.problems)]
            st = [int(x) for x in (steps if not isinstance(steps, int) else [steps] * self.problems)]
            self.s, self.c = max(sl), st
            _check(load().ac_parareal_create_uneven(C.byref(p), dref, self.problems, (C.c_int * len(sl))(*sl),
                                                    (C.c_int * len(st))(*st), _dev(self._u0, params.dtype, "u0"),
                                                    C.byref(h)))
        self._h = h
        self.k = 0
        self._acnn = None
        self._acnn_h = None
        if acnn is not None:
            self.set_coarse_acnn(acnn)

    def set_coarse_acnn(self, acnn):
        """Use the ResBlock ACNN as G (None: back to the conv stack the handle
        was created with).  The net's current parameters are used: after an
        update of the net the next iteration re-attaches its new handle."""
        h = acnn.handle() if acnn is not None else None
        _check(load().ac_parareal_set_coarse_acnn(self._h, h))
        self._acnn, self._acnn_h = acnn, h

    def _sync_acnn(self):
        if self._acnn is not None and self._acnn._h is not self._acnn_h:
            self.set_coarse_acnn(self._acnn)

    def enable_graphs(self, on=True):
        _check(load().ac_parareal_enable_graphs(self._h, int(on)))

    def set_coarse_substeps(self, substeps: int):
        """Each coarse evaluation applies G `substeps` times (the remark after
        Algorithm 2)."""
        _check(load().ac_parareal_set_coarse_substeps(self._h, int(substeps)))

    def set_fine_scheme(self, scheme: int, tol: float = 1e-6, max_iters: int = 50):
        """0: the stabilised semi-implicit step; 1: Crank-Nicolson with Picard
        iteration (Sec. 3.1)."""
        _check(load().ac_parareal_set_fine_scheme(self._h, int(scheme), float(tol), int(max_iters)))

    def iterate(self, stream=None):
        self._sync_acnn()
        kk = C.c_int(self.k)
        l2 = (C.c_double * self.problems)()
        mx = (C.c_double * self.problems)()
        _check(load().parareal_iterate(self._h, C.byref(kk), l2, mx, _stream(stream)))
        self.k = kk.value
        return list(l2), list(mx)

    def set_active(self, p: int, active: bool):
        _check(load().ac_parareal_set_active(self._h, int(p), int(active)))

    def solve(self, tol: float, kmax: int, stream=None, allow_unconverged=False):
        self._sync_acnn()
        it = (C.c_int * self.problems)()
        l2 = (C.c_double * self.problems)()
        rc = load().ac_parareal_solve(self._h, float(tol), int(kmax), it, l2, _stream(stream))
        if rc != AC_OK and not (allow_unconverged and rc == -6):
            _check(rc)
        self.k = max(self.k, max(list(it)) + 1)
        return list(it), list(l2)

    def trajectory(self, out=None, stream=None):
        """Copy of U[problems][s+1][n][n] (the last iterate) into a torch tensor."""
        import torch
        n = self.params.n
        if out is None:
            out = torch.empty((self.problems, self.s + 1, n, n), dtype=self.params.dtype, device="cuda")
        _check(load().ac_parareal_copy_trajectory(self._h, _dev(out, self.params.dtype, "out"), _stream(stream)))
        return out

    def reset(self, u0, stream=None):
        self._u0 = u0.contiguous()
        _check(load().ac_parareal_reset(self._h, _dev(self._u0, self.params.dtype, "u0"), _stream(stream)))
        self.k = 0

    def enable_timing(self, on=True):
        _check(load().ac_parareal_enable_timing(self._h, int(on)))

    def stats(self) -> dict:
        st = ac_parareal_stats()
        _check(load().ac_parareal_get_stats(self._h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in ac_parareal_stats._fields_}

    def reset_stats(self):
        _check(load().ac_parareal_reset_stats(self._h))

    def close(self):
        if getattr(self, "_h", None):
            load().ac_parareal_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


