"""Host-side checks of the C ABI: the library loads, exports every entry point
declared in include/fewha.h, and rejects invalid arguments before touching a
GPU (no compute call is made here)."""

import ctypes

import pytest

from paper_2009_00946_b300 import configs, fewha


def test_library_exports_every_declared_symbol():
    L = fewha.lib()
    names = fewha.declared_symbols()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    L = fewha.lib()
    for n in fewha.declared_symbols():
        assert getattr(L, n).restype is not None or n in ("fewha_destroy",), n


def _create(g, p):
    L = fewha.lib()
    h = ctypes.c_void_p()
    st = L.fewha_create(ctypes.byref(g), ctypes.byref(p), None, ctypes.byref(h))
    return st, h, L.fewha_last_error(None).decode()


@pytest.mark.parametrize("mutate,code", [
    (lambda g, p: setattr(g, "D", -1.0), 1),
    (lambda g, p: setattr(g, "n_wfs", 0), 1),
    (lambda g, p: setattr(g, "n_wfs", 17), 1),
    (lambda g, p: setattr(g, "precision", 5), 1),
    (lambda g, p: setattr(p, "alpha", 0.0), 1),
    (lambda g, p: p.n_side.__setitem__(0, 48), 1),          # not a power of two
    (lambda g, p: p.levels.__setitem__(0, 5), 1),            # 32 >> 5 < 2
    (lambda g, p: p.cn2.__setitem__(1, 0.0), 1),
    (lambda g, p: g.noise_sigma.__setitem__(0, 0.0), 1),
    (lambda g, p: setattr(g, "obstruction", 1.0), 1),
])
def test_create_rejects_invalid_arguments_on_host(mutate, code):
    g, p = fewha.structs_from_config(configs.c1_plain())
    mutate(g, p)
    st, h, msg = _create(g, p)
    assert st == code and not h.value and msg


def test_create_rejects_layer_above_lgs():
    cfg = configs.c5_autograd()
    cfg["layers"][-1]["height"] = 95000.0
    g, p = fewha.structs_from_config(cfg)
    st, h, msg = _create(g, p)
    assert st == 3 and "guide star" in msg


def test_null_pointers_rejected():
    L = fewha.lib()
    assert L.fewha_create(None, None, None, None) == 1
    assert L.fewha_destroy(None) == 1
    assert L.fewha_solve(None, 4, 1) == 1
    assert L.fewha_sync(None) == 1
    assert L.fewha_launch_count(None) == -1
    assert L.fewha_set_host_transfer(None, 1) == 1
    assert L.fewha_frame_arm(None, None, 4, 1, None, 1.0) == 1
    assert L.fewha_frame_fire(None) == 1
    assert L.fewha_tape_bytes_batch(None, 4, 32) == -1
    assert L.fewha_solve_taped_batch(None, 32, None, 4, None, None) == 1
    assert L.fewha_backward_batch(None, 32, None, 4, None, None, None, None, None, None) == 1


def test_header_documents_every_entry_point():
    import os
    import re
    hdr = open(fewha.HEADER).read()
    for n in fewha.declared_symbols():
        # every declaration is preceded by a comment block
        m = re.search(r"\*/\s*\n(?:[^\n]*\n){0,4}[^\n;]*\b" + n + r"\s*\(", hdr)
        assert m, n


def test_batch_rejects_invalid_arguments_on_host():
    """Batch creation checks its arguments before touching the device."""
    L = fewha.lib()
    b = ctypes.c_void_p()
    assert L.fewha_batch_create(0, None, None, None, 0, 0, ctypes.byref(b)) == 1 and not b.value
    assert "count" in L.fewha_batch_last_error(None).decode()
    cfgs = [configs.c5_autograd(), configs.c1_plain()]
    geoms = (fewha.Geometry * 2)()
    profs = (fewha.Profile * 2)()
    for i, c in enumerate(cfgs):
        geoms[i], profs[i] = fewha.structs_from_config(c, fewha.FP32)
    assert L.fewha_batch_create(2, geoms, profs, None, 0, 3, ctypes.byref(b)) == 1 and not b.value
    assert "cluster_size" in L.fewha_batch_last_error(None).decode()
    geoms[1].precision = fewha.FP64
    assert L.fewha_batch_create(2, geoms, profs, None, 0, 0, ctypes.byref(b)) == 1 and not b.value
    assert "instance 1" in L.fewha_batch_last_error(None).decode()
    geoms[1].precision = fewha.FP32
    profs[0].alpha = -1.0
    st = L.fewha_batch_create(2, geoms, profs, None, 0, 0, ctypes.byref(b))
    assert st == 1 and "instance 0" in L.fewha_batch_last_error(None).decode()
    assert L.fewha_batch_destroy(None) == 1 and L.fewha_batch_frame(None, None, 4, 1, None, 0) == 1
    assert L.fewha_batch_launch_count(None) == -1
    assert L.fewha_batch_set_groups(None, None, 0) == 1
    assert L.fewha_batch_set_max_launches(None, 1) == 1


def test_debug_library_exports_every_declared_symbol():
    """libfewha_debug.so (the bounds-checked build of the same sources) loads
    beside the release library and exports the same entry points."""
    import os
    path = os.path.join(os.path.dirname(fewha.LIB_PATH), "libfewha_debug.so")
    assert os.path.exists(path)
    D = ctypes.CDLL(path)
    missing = [n for n in fewha.declared_symbols() if not hasattr(D, n)]
    assert not missing, missing


def test_release_build_reports_no_bounds_checks():
    """The release library compiles every check out: fewha_debug_bounds says
    so (0) without touching a device."""
    L = fewha.lib()
    first, count = ctypes.c_ulonglong(7), ctypes.c_ulonglong(7)
    if fewha.LIB_PATH.endswith("libfewha.so"):
        assert L.fewha_debug_bounds(ctypes.byref(first), ctypes.byref(count)) == 0
        assert first.value == 0 and count.value == 0
    assert L.fewha_debug_bounds(None, ctypes.byref(count)) == 1   # FEWHA_ERR_ARG


def test_debug_site_numbers_agree():
    """The check sites are numbered alike in include/fewha.h (FEWHA_DBG_*),
    in the device code's enum and in the binding's names."""
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    hdr = open(os.path.join(root, "include", "fewha.h")).read()
    dev = open(os.path.join(root, "paper_2009_00946_b300", "csrc", "debug.cuh")).read()
    h = sorted(int(v) for v in re.findall(r"FEWHA_DBG_[A-Z_]+ = (\d+)", hdr))
    d = sorted(int(v) for v in re.findall(r"kDbg[A-Za-z]+ = (\d+)", dev) if int(v) > 0)
    assert h == d == sorted(fewha.DEBUG_SITES) == list(range(1, len(h) + 1))
