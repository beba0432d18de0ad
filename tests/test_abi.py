"""Host-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every function include/acpr.h declares; argument validation runs on the
host and never touches a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_2510_07672_gb300 as G
from paper_2510_07672_gb300 import abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"^\s*#.*$", "", src, flags=re.M)
        src = re.sub(r"typedef[^;]*\{[^}]*\}[^;]*;", "", src, flags=re.S)
        src = re.sub(r"enum\s*\{[^}]*\}\s*;", "", src, flags=re.S)
        for stmt in src.split(";"):
            if "typedef" in stmt or "extern" in stmt:
                continue
            m = re.search(r"([a-z_][a-z_0-9]*)\s*\(", stmt)
            if m:
                names.append(m.group(1))
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = G.load()
    decl = declared_functions()
    assert len(decl) >= 15
    missing = [n for n in decl if not hasattr(L, n)]
    assert not missing, missing
    assert set(abi.EXPORTS) <= set(decl)


def test_supported_sizes():
    assert G.ac_fine_supported(256, G.AC_F32)
    assert G.ac_fine_supported(64, G.AC_F64)
    assert not G.ac_fine_supported(48, G.AC_F32)
    assert not G.ac_fine_supported(4096, G.AC_F32)


def test_argument_errors_are_reported_on_the_host():
    L = G.load()
    assert L.ac_fine_step(None, 1, None, None, None) == -1
    assert b"NULL" in L.ac_last_error()
    p = abi.ac_params(48, 1.0, 0.01, 2.0, 1e-4, 0, 1)
    assert L.ac_fine_step(C.byref(p), 1, None, None, None) == -2      # unsupported size
    p = abi.ac_params(64, 1.0, 0.01, 2.0, -1.0, 0, 1)
    assert L.ac_fine_step(C.byref(p), 1, None, None, None) == -1      # dt <= 0
    p = abi.ac_params(64, 1.0, 0.01, 2.0, 1e-4, 0, 1)
    assert L.ac_fine_step(C.byref(p), 0, None, None, None) == 0       # empty batch is a no-op
    assert L.ac_fine_step(C.byref(p), 2, None, None, None) == -1      # null fields
    d = abi.cnn_desc(4, 24, 0, 1, 0, 0, -1.0, 1.0, 1, None, None, None, None, 0)
    assert L.cnn_coarse_step(C.byref(d), 64, 1, None, None, None) == -1   # null weights first
    d = abi.cnn_desc(4, 24, 0, 1, 0, 0, -1.0, 1.0, 1, 16, 16, None, None, 0)
    assert L.cnn_coarse_step(C.byref(d), 64, 1, None, None, None) == -2   # C=24 not built for bf16
    h = C.c_void_p()
    assert L.ac_parareal_create(None, None, 1, 1, 1, None, C.byref(h)) == -1
    assert L.parareal_iterate(None, None, None, None, None) == -1


def test_binding_refuses_cpu_tensors():
    torch = pytest.importorskip("torch")
    fp = G.FineParams(64, 0.01, 2.0, 1e-4)
    with pytest.raises(ValueError, match="CUDA tensor"):
        G.ac_fine_step(fp, torch.zeros(1, 64, 64))


def test_acnn_and_3d_host_queries_and_argument_errors():
    """Host-only entry points of the ResBlock ACNN (Sec. 3.2) and the 3D step:
    sizes and argument validation, no GPU touched."""
    L = G.load()
    nb = C.c_longlong()
    assert L.acnn_param_count(4, 2, C.byref(nb)) == 36 + 4 * 144 + 36 and nb.value == 21
    assert L.acnn_param_count(16, 3, None) == 9 * 16 + 6 * 9 * 256 + 9 * 16
    assert L.acnn_param_count(8, 2, None) == -1          # C = 8 not built
    assert L.acnn_param_count(4, 5, None) == -1          # at most 4 blocks
    assert L.loss_acn_work_bytes(256, 4) >= 8 * 256 * 256 * 4
    assert L.loss_acn_work_bytes(48, 4) == 0
    d = abi.acnn_desc(8, 2, 0, 0, -1.0, 1.0, 1, 16, 16)
    h = C.c_void_p()
    assert L.acnn_create(C.byref(d), C.byref(h)) == -2   # unsupported width
    d = abi.acnn_desc(4, 2, 0, 1, 1.0, -1.0, 1, 16, 16)
    assert L.acnn_create(C.byref(d), C.byref(h)) == -1   # limiter lo >= hi
    d = abi.acnn_desc(4, 2, 0, 0, -1.0, 1.0, 1, None, None)
    assert L.acnn_forward_train(C.byref(d), 64, 1, None, None, None, None) == -1
    assert L.acnn_train_bytes(C.byref(d), 64, 1) == 0    # null parameters
    assert L.acnn_adam_step(1, None, None, None, None, 10, 1e-3, 0.9, 0.999, 1e-8, 1, None) == -1
    assert L.acnn_adam_step(1, 16, 16, 16, 16, 10, 1e-3, 0.9, 0.999, 1e-8, 0, None) == -1   # t >= 1
    p = abi.ac_params(64, 1.0, 0.01, 2.0, 1e-2, 1, 1)
    assert L.loss_acn(C.byref(p), 0, None, None, None, None, None, None) == -1
    assert L.ac_fine3d_supported(128, G.AC_F32) == 1
    assert L.ac_fine3d_supported(256, G.AC_F32) == 0
    assert L.ac_fine3d_work_bytes(128, 3, G.AC_F32) >= 2 * 8 * 128 ** 3   # two complex pairs
    p3 = abi.ac_params(256, 1.0, 0.02, 2.0, 1e-4, 0, 1)
    assert L.ac_fine3d_propagate(C.byref(p3), 1, 1, None, None, None, 0, None) == -2
    p3 = abi.ac_params(64, 1.0, 0.02, 2.0, 1e-4, 0, 1)
    assert L.ac_fine3d_propagate(C.byref(p3), 1, 0, None, None, None, 0, None) == 0     # no fields
    assert L.ac_fine3d_propagate(C.byref(p3), 1, 2, None, None, None, 0, None) == -1    # null fields
    assert L.ac_parareal_set_coarse_acnn(None, None) == -1
    assert L.ac_parareal_set_coarse_substeps(None, 2) == -1


def test_acnn_handle_lifetime_with_a_parareal_handle(monkeypatch):
    """Host logic of the binding, with a stand-in library: updating an Acnn
    attached to a Parareal handle retires (does not free) its inference
    handle, the Parareal handle re-attaches the new one before the next
    iteration, and every handle is freed with the Acnn object."""
    torch = pytest.importorskip("torch")

    class FakeLib:
        def __init__(self):
            self.created, self.destroyed, self.attached, self.next = [], [], [], 100

        def acnn_param_count(self, c, b, nb):
            nb._obj.value = 21
            return 648

        def acnn_create(self, d, out):
            out._obj.value = self.next
            self.created.append(self.next)
            self.next += 1
            return 0

        def acnn_destroy(self, h):
            self.destroyed.append(h.value)

        def ac_parareal_set_coarse_acnn(self, st, h):
            self.attached.append(None if h is None else h.value)
            return 0

        def parareal_iterate(self, st, kk, l2, mx, s):
            return 0

    fake = FakeLib()
    monkeypatch.setattr(abi, "load", lambda build_if_missing=True: fake)
    monkeypatch.setattr(abi, "_stream", lambda s: None)
    net = abi.Acnn(4, 2, np.zeros(648), np.zeros(21), device="cpu")
    pr = abi.Parareal.__new__(abi.Parareal)
    pr._h, pr.k, pr.problems, pr._acnn, pr._acnn_h = C.c_void_p(1), 0, 1, None, None
    pr.set_coarse_acnn(net)
    assert fake.attached == [100]
    pr.iterate()
    assert fake.attached == [100]            # unchanged net: no re-attach
    net.invalidate()                         # as after an Adam step
    assert fake.destroyed == []              # the attached handle stays alive
    pr.iterate()
    assert fake.attached == [100, 101]       # re-attached to the new handle
    net._free_handles()
    assert sorted(fake.destroyed) == [100, 101]


def test_conv_shape_queries_on_the_host():
    """The persistent conv kernel's shape table (ring depth, TMEM slots) is
    host logic: every (n, C) with n a multiple of 128 has at least one shape,
    the shapes are distinct, the ring holds at most 24 rows, the slots of
    3C columns (rounded up to a power of two) fit the 512 TMEM columns, and
    selecting, reading back and resetting a shape works without a GPU; the
    weight-gradient switch is host state too."""
    L = G.load()
    for C_ in (16, 32, 64):
        width = 64 if C_ <= 16 else (128 if C_ <= 32 else 256)
        for n in (128, 256, 512, 1024):
            shapes = G.cnn_conv_variants(n, C_)
            assert shapes, (n, C_)
            assert len(set(shapes)) == len(shapes)
            for ring, slots in shapes:
                assert 2 <= ring <= 24 and 2 <= slots and slots * width <= 512, (n, C_, ring, slots)
        assert G.cnn_conv_variants(64, C_) == []  # below 128 the one-shot kernel runs
    assert L.cnn_conv_variant_count(256, 24) == 0
    n_sh = len(G.cnn_conv_variants(256, 32))
    G.cnn_conv_set_variant(256, 32, n_sh - 1)
    assert L.cnn_conv_get_variant(256, 32) == n_sh - 1
    G.cnn_conv_set_variant(256, 32, -1)
    assert L.cnn_conv_get_variant(256, 32) == -1
    with pytest.raises(G.AcprError):
        G.cnn_conv_set_variant(256, 32, n_sh)
    r, s = C.c_int(), C.c_int()
    assert L.cnn_conv_variant_shape(256, 32, n_sh, C.byref(r), C.byref(s)) != 0
    G.cnn_train_set_wgrad_tc(False)
    G.cnn_train_set_wgrad_tc(True)
