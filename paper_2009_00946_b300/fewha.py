"""Python binding of libfewha.so (ctypes): argument marshalling only.

Every step of the reconstruction runs in the library's CUDA kernels.  The
binding loads the in-tree ``libfewha.so`` and raises if it is missing: there is
no CPU fallback.  Arrays may be numpy arrays (host) or torch CUDA tensors
(device, ordered on the solver's stream).
"""

from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfewha.so")
# FEWHA_DEBUG=1: the debug build (bounds checks at every gather and scatter,
# reported by fewha_debug_bounds) in place of the release library
if os.environ.get("FEWHA_DEBUG") == "1":
    LIB_PATH = os.path.join(HERE, "libfewha_debug.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "fewha.h")

MAX_WFS, MAX_LAYERS, MAX_DMS, MAX_FIT_DIRS, MAX_JACOBI_LEVELS = 16, 64, 8, 64, 16
FP32, FP64 = 0, 1
PATH_PLAIN, PATH_FUSED = 0, 1
FIT_MCAO, FIT_MOAO = 0, 1
ERRORS = {0: "OK", 1: "ARG", 2: "INPUT", 3: "GEOMETRY", 4: "BREAKDOWN", 5: "TIMEOUT", 6: "LAUNCH", 7: "CUDA",
          8: "STATE"}
VEC_C, VEC_R, VEC_B, VEC_JACOBI, VEC_ALPHA_D = 0, 1, 2, 3, 4
OP_W, OP_WT, OP_P, OP_PT, OP_GAMMA, OP_GAMMA_T = 0, 1, 2, 3, 4, 5


class FewhaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("FEWHA_ERR_%s: %s" % (ERRORS.get(code, code), msg))
        self.code = code
        self.name = ERRORS.get(code, str(code))


class Geometry(ctypes.Structure):
    _fields_ = [("D", ctypes.c_double), ("obstruction", ctypes.c_double), ("n_wfs", ctypes.c_int),
                ("n_sub", ctypes.c_int * MAX_WFS), ("theta_x", ctypes.c_double * MAX_WFS),
                ("theta_y", ctypes.c_double * MAX_WFS), ("gs_height", ctypes.c_double * MAX_WFS),
                ("noise_sigma", ctypes.c_double * MAX_WFS), ("n_dm", ctypes.c_int),
                ("dm_height", ctypes.c_double * MAX_DMS), ("dm_pitch", ctypes.c_double * MAX_DMS),
                ("n_fit_dir", ctypes.c_int), ("fit_theta_x", ctypes.c_double * MAX_FIT_DIRS),
                ("fit_theta_y", ctypes.c_double * MAX_FIT_DIRS), ("fit_n_sub", ctypes.c_int),
                ("precision", ctypes.c_int), ("lgs_tt_filter", ctypes.c_int), ("fit_mode", ctypes.c_int)]


class Profile(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int), ("height", ctypes.c_double * MAX_LAYERS),
                ("cn2", ctypes.c_double * MAX_LAYERS), ("n_side", ctypes.c_int * MAX_LAYERS),
                ("levels", ctypes.c_int * MAX_LAYERS), ("r0", ctypes.c_double), ("alpha", ctypes.c_double),
                ("jacobi_level_weight", ctypes.c_double * MAX_JACOBI_LEVELS)]


_lib = None


def declared_symbols() -> list[str]:
    """Entry points declared in include/fewha.h."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fewha_[a-z0-9_]+)\s*\(", text)))


def lib():
    """Load libfewha.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise OSError("%s not built: run python -m paper_2009_00946_b300.build" % os.path.basename(LIB_PATH))
    L = ctypes.CDLL(LIB_PATH)
    vp, ci, cd, cl, cll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_long, ctypes.c_longlong
    sig = {
        "fewha_create": (ci, [ctypes.POINTER(Geometry), ctypes.POINTER(Profile), vp, ctypes.POINTER(vp)]),
        "fewha_destroy": (ci, [vp]),
        "fewha_last_error": (ctypes.c_char_p, [vp]),
        "fewha_sizes": (ci, [vp, ctypes.POINTER(cl), ctypes.POINTER(cl), ctypes.POINTER(cl)]),
        "fewha_set_path": (ci, [vp, ci]),
        "fewha_set_residual_replacement": (ci, [vp, ci]),
        "fewha_set_frame": (ci, [vp, vp, ci]),
        "fewha_solve": (ci, [vp, ci, ci]),
        "fewha_fit_dm": (ci, [vp, cd, ci, vp, ci]),
        "fewha_get_layers": (ci, [vp, vp, ci]),
        "fewha_get_vector": (ci, [vp, ci, vp, ci]),
        "fewha_get_state": (ci, [vp, vp, vp, vp, ci]),
        "fewha_set_state": (ci, [vp, vp, vp, vp, ci, cl]),
        "fewha_apply_M": (ci, [vp, vp, vp, ci]),
        "fewha_frame": (ci, [vp, vp, ci, ci, cd, ci, vp, vp, ci]),
        "fewha_sync": (ci, [vp]),
        "fewha_set_barrier_budget": (ci, [vp, cll]),
        "fewha_launch_count": (cll, [vp]),
        "fewha_describe": (ci, [vp, ctypes.c_char_p, ci]),
        "fewha_set_trace": (ci, [vp, ci]),
        "fewha_get_trace": (ci, [vp, ctypes.POINTER(ctypes.c_ulonglong), ci, ctypes.POINTER(ci),
                                 ctypes.POINTER(ci)]),
        "fewha_layers_noalloc": (ci, [vp, vp, ci, ctypes.POINTER(ci), ctypes.POINTER(ci), vp, ctypes.c_char_p,
                                      ci]),
        "fewha_get_fine_trace": (ci, [vp, ctypes.POINTER(ctypes.c_ulonglong), ci, ctypes.POINTER(ci),
                                      ctypes.POINTER(ci)]),
        "fewha_set_cluster_size": (ci, [vp, ci]),
        "fewha_set_layer_transform": (ci, [vp, ci]),
        "fewha_set_host_transfer": (ci, [vp, ci]),
        "fewha_frame_arm": (ci, [vp, vp, ci, ci, vp, cd]),
        "fewha_frame_fire": (ci, [vp]),
        "fewha_get_frame_timing": (ci, [vp, ctypes.POINTER(cd)]),
        "fewha_autotune": (ci, [vp, ci, ci, ctypes.c_char_p, ci]),
        "fewha_set_loop": (ci, [vp, ci]),
        "fewha_operator_dims": (ci, [vp, ci, ctypes.POINTER(cl), ctypes.POINTER(cl)]),
        "fewha_apply_operator": (ci, [vp, ci, vp, vp, ci]),
        "fewha_time_operator": (ci, [vp, ci, ci, ctypes.POINTER(cd)]),
        "fewha_set_params": (ci, [vp, ctypes.POINTER(cd), cd, ctypes.POINTER(cd)]),
        "fewha_tape_bytes": (cl, [vp, ci]),
        "fewha_solve_taped": (ci, [vp, vp, ci, vp, vp]),
        "fewha_backward": (ci, [vp, vp, ci, vp, vp, vp, vp, vp, vp]),
        "fewha_tape_bytes_batch": (cl, [vp, ci, ci]),
        "fewha_solve_taped_batch": (ci, [vp, ci, vp, ci, vp, vp]),
        "fewha_backward_batch": (ci, [vp, ci, vp, ci, vp, vp, vp, vp, vp, vp]),
        "fewha_batch_create": (ci, [ci, ctypes.POINTER(Geometry), ctypes.POINTER(Profile), vp, ci, ci,
                                    ctypes.POINTER(vp)]),
        "fewha_batch_destroy": (ci, [vp]),
        "fewha_batch_last_error": (ctypes.c_char_p, [vp]),
        "fewha_batch_sizes": (ci, [vp, ctypes.POINTER(ci), ctypes.POINTER(cl), ctypes.POINTER(cl)]),
        "fewha_batch_set_residual_replacement": (ci, [vp, ci]),
        "fewha_batch_frame": (ci, [vp, vp, ci, ci, vp, ci]),
        "fewha_batch_get_state": (ci, [vp, ci, vp, vp, vp, ci]),
        "fewha_batch_sync": (ci, [vp]),
        "fewha_batch_describe": (ci, [vp, ctypes.c_char_p, ci]),
        "fewha_batch_launch_count": (cll, [vp]),
        "fewha_batch_autotune": (ci, [vp, ci, ci, ctypes.c_char_p, ci]),
        "fewha_batch_set_groups": (ci, [vp, ctypes.POINTER(ci), ci]),
        "fewha_batch_set_max_launches": (ci, [vp, ci]),
        "fewha_batch_set_trace": (ci, [vp, ci]),
        "fewha_batch_get_fine_trace": (ci, [vp, ctypes.POINTER(ctypes.c_ulonglong), ci, ctypes.POINTER(ci),
                                            ctypes.POINTER(ci)]),
        "fewha_measure_l2": (ci, [cl, ci, ci, ctypes.POINTER(cd), ctypes.POINTER(cd), ctypes.c_char_p, ci]),
        "fewha_debug_bounds": (ci, [ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_ulonglong)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def structs_from_config(cfg: dict, precision: int | None = None):
    """fewha_geometry / fewha_profile from a configuration dict."""
    g = Geometry()
    g.D = cfg["D"]
    g.obstruction = cfg.get("obstruction", 0.0)
    wfs = cfg["wfs"]
    if len(wfs) > MAX_WFS:
        raise ValueError("too many sensors")
    g.n_wfs = len(wfs)
    for i, w in enumerate(wfs):
        g.n_sub[i] = int(w["n_sub"])
        g.theta_x[i] = w["theta_x"]
        g.theta_y[i] = w["theta_y"]
        g.gs_height[i] = w["gs_height"]
        g.noise_sigma[i] = w["sigma"]
    dms = cfg.get("dms", [])
    g.n_dm = len(dms)
    for i, d in enumerate(dms):
        g.dm_height[i] = d["height"]
        g.dm_pitch[i] = d["pitch"]
    fd = cfg.get("fit_dirs", [])
    g.n_fit_dir = len(fd)
    for i, (tx, ty) in enumerate(fd):
        g.fit_theta_x[i] = tx
        g.fit_theta_y[i] = ty
    g.fit_n_sub = int(cfg.get("fit_n_sub", 0))
    if precision is None:
        precision = FP64 if cfg.get("precision", "fp32") == "fp64" else FP32
    g.precision = precision
    g.lgs_tt_filter = 1 if cfg.get("lgs_tip_tilt_filter", False) else 0
    mode = str(cfg.get("fit_mode", "mcao")).lower()
    if mode not in ("mcao", "moao"):
        raise ValueError("fit_mode must be 'mcao' or 'moao'")
    g.fit_mode = FIT_MOAO if mode == "moao" else FIT_MCAO
    p = Profile()
    lay = cfg["layers"]
    if len(lay) > MAX_LAYERS:
        raise ValueError("too many layers")
    p.n_layers = len(lay)
    for i, l in enumerate(lay):
        p.height[i] = l["height"]
        p.cn2[i] = l["cn2"]
        p.n_side[i] = int(l["n"])
        p.levels[i] = int(l["levels"])
    p.r0 = cfg["r0"]
    p.alpha = cfg["alpha"]
    jw = [float(x) for x in cfg.get("jacobi_level_weights", [])]
    if len(jw) > MAX_JACOBI_LEVELS or any(not (x > 0.0) for x in jw):
        raise ValueError("jacobi_level_weights: at most %d weights, each > 0" % MAX_JACOBI_LEVELS)
    for j, x in enumerate(jw):
        p.jacobi_level_weight[j] = x
    return g, p


def _ptr(a, dtype, count, on_device):
    """Pointer of a numpy array (host) or torch CUDA tensor (device)."""
    if hasattr(a, "data_ptr"):
        if a.dtype != dtype[1] or a.numel() != count or not a.is_contiguous():
            raise ValueError("tensor must be contiguous %s with %d elements" % (dtype[1], count))
        return ctypes.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    arr = a
    if arr.dtype != dtype[0] or arr.size != count or not arr.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous %s with %d elements" % (dtype[0], count))
    return ctypes.c_void_p(arr.__array_interface__["data"][0]), 0


def _marks(rows):
    """Per CTA a list of (tag, ns) from the packed fine-trace words."""
    marks = []
    for r in rows:
        r = r[r != 0]
        marks.append([(int(v >> np.uint64(56)), int(v & np.uint64(0x00FFFFFFFFFFFFFF))) for v in r])
    return marks


class Solver:
    """One FEWHA instance on the current CUDA device (a fewha_handle)."""

    def __init__(self, cfg: dict, precision: int | None = None, stream=None, path: int | None = None,
                 k_rr: int | None = None):
        import torch
        L = lib()
        g, p = structs_from_config(cfg, precision)
        self.precision = g.precision
        self.np_dtype = np.float64 if self.precision == FP64 else np.float32
        self.torch_dtype = torch.float64 if self.precision == FP64 else torch.float32
        if stream is None:
            self._stream_obj = torch.cuda.Stream()
        else:
            self._stream_obj = stream
        self.stream = self._stream_obj
        h = ctypes.c_void_p()
        st = L.fewha_create(ctypes.byref(g), ctypes.byref(p), ctypes.c_void_p(self._stream_obj.cuda_stream),
                            ctypes.byref(h))
        if st != 0:
            raise FewhaError(st, L.fewha_last_error(None).decode())
        self.h = h
        n, s, a = ctypes.c_long(), ctypes.c_long(), ctypes.c_long()
        L.fewha_sizes(h, ctypes.byref(n), ctypes.byref(s), ctypes.byref(a))
        self.N, self.S, self.NA = n.value, s.value, a.value
        self.cfg = cfg
        if path is not None:
            self.set_path(path)
        if k_rr is not None:
            self._check(L.fewha_set_residual_replacement(self.h, int(k_rr)))

    # -- plumbing --
    def _check(self, st):
        if st != 0:
            raise FewhaError(st, lib().fewha_last_error(self.h).decode())

    def _dt(self):
        return (self.np_dtype, self.torch_dtype)

    def close(self):
        if getattr(self, "h", None):
            lib().fewha_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- API --
    def set_path(self, path: int):
        self._check(lib().fewha_set_path(self.h, int(path)))

    def set_residual_replacement(self, k_rr: int):
        self._check(lib().fewha_set_residual_replacement(self.h, int(k_rr)))

    def operator_dims(self, op: int):
        ni, no = ctypes.c_long(), ctypes.c_long()
        self._check(lib().fewha_operator_dims(self.h, int(op), ctypes.byref(ni), ctypes.byref(no)))
        return ni.value, no.value

    def apply_operator(self, op: int, x):
        """One of W, W^T, P, P^T, Gamma, Gamma^T on a host array (numpy)."""
        ni, no = self.operator_dims(op)
        x = np.ascontiguousarray(x, dtype=self.np_dtype)
        if x.size != ni:
            raise ValueError("operator %d takes %d values" % (op, ni))
        out = np.empty(no, self.np_dtype)
        self._check(lib().fewha_apply_operator(self.h, int(op), ctypes.c_void_p(x.ctypes.data),
                                               ctypes.c_void_p(out.ctypes.data), 0))
        return out

    def time_operator(self, op: int, reps: int = 50) -> float:
        us = ctypes.c_double()
        self._check(lib().fewha_time_operator(self.h, int(op), int(reps), ctypes.byref(us)))
        return us.value

    def set_loop(self, closed: bool):
        """Alg. 1 closed loop (pseudo-open-loop slopes, closed-loop gain) or open loop."""
        self._check(lib().fewha_set_loop(self.h, 1 if closed else 0))

    def set_barrier_budget(self, cycles: int):
        self._check(lib().fewha_set_barrier_budget(self.h, int(cycles)))

    def set_frame(self, slopes):
        ptr, dev = _ptr(slopes, self._dt(), self.S, None)
        self._check(lib().fewha_set_frame(self.h, ptr, dev))

    def solve(self, n_iter: int, warm: bool = True):
        self._check(lib().fewha_solve(self.h, int(n_iter), 1 if warm else 0))

    def sync(self):
        self._check(lib().fewha_sync(self.h))

    def fit_dm(self, gain: float = 1.0, n_fit: int = 8, out=None):
        if out is None:
            out = np.empty(self.NA, self.np_dtype)
        ptr, dev = _ptr(out, self._dt(), self.NA, None)
        self._check(lib().fewha_fit_dm(self.h, float(gain), int(n_fit), ptr, dev))
        return out

    def layers(self, out=None):
        if out is None:
            out = np.empty(self.N, self.np_dtype)
        ptr, dev = _ptr(out, self._dt(), self.N, None)
        self._check(lib().fewha_get_layers(self.h, ptr, dev))
        return out

    def vector(self, which: int, out=None):
        if out is None:
            out = np.empty(self.N, self.np_dtype)
        ptr, dev = _ptr(out, self._dt(), self.N, None)
        self._check(lib().fewha_get_vector(self.h, int(which), ptr, dev))
        return out

    def get_state(self):
        c, b, r = (np.empty(self.N, self.np_dtype) for _ in range(3))
        self._check(lib().fewha_get_state(self.h, ctypes.c_void_p(c.ctypes.data), ctypes.c_void_p(b.ctypes.data),
                                          ctypes.c_void_p(r.ctypes.data), 0))
        return c, b, r

    def set_state(self, c, b, r, frame_count: int):
        c, b, r = (np.ascontiguousarray(v, dtype=self.np_dtype) for v in (c, b, r))
        self._check(lib().fewha_set_state(self.h, ctypes.c_void_p(c.ctypes.data), ctypes.c_void_p(b.ctypes.data),
                                          ctypes.c_void_p(r.ctypes.data), 0, int(frame_count)))

    def apply_M(self, x, out=None):
        if out is None:
            out = np.empty(self.N, self.np_dtype) if not hasattr(x, "data_ptr") else x.new_empty(self.N)
        px, dx = _ptr(x, self._dt(), self.N, None)
        py, dy = _ptr(out, self._dt(), self.N, None)
        if dx != dy:
            raise ValueError("x and out must both be host or both be device")
        self._check(lib().fewha_apply_M(self.h, px, py, dx))
        return out

    def frame(self, slopes, n_iter: int, warm: bool = True, gain: float = 1.0, n_fit: int = 8,
              layers_out=None, dm_out=None):
        """One whole frame through the captured CUDA graph.  All arrays host
        (numpy; the call synchronises) or all device (torch CUDA tensors; the
        call only enqueues on the solver's stream)."""
        ps, ds = _ptr(slopes, self._dt(), self.S, None)
        pl = pd = None
        if layers_out is not None:
            pl, dl = _ptr(layers_out, self._dt(), self.N, None)
            if dl != ds:
                raise ValueError("slopes and layers_out must both be host or both be device")
        if dm_out is not None:
            pd, dd = _ptr(dm_out, self._dt(), self.NA, None)
            if dd != ds:
                raise ValueError("slopes and dm_out must both be host or both be device")
        self._check(lib().fewha_frame(self.h, ps, int(n_iter), 1 if warm else 0, float(gain), int(n_fit), pl, pd,
                                      ds))

    def bind_frame(self, slopes, n_iter: int, warm: bool = True, gain: float = 1.0, n_fit: int = 8,
                   layers_out=None, dm_out=None):
        """frame() bound to fixed buffers, for a real-time loop: the arguments
        are checked and converted once, and each call of the returned function
        runs one frame on what the buffers hold then (the caller refills the
        slopes array in place).  Host arrays: the call returns with the
        results in layers_out / dm_out; device tensors: it only enqueues."""
        ps, ds = _ptr(slopes, self._dt(), self.S, None)
        pl = pd = None
        if layers_out is not None:
            pl, dl = _ptr(layers_out, self._dt(), self.N, None)
            if dl != ds:
                raise ValueError("slopes and layers_out must both be host or both be device")
        if dm_out is not None:
            pd, dd = _ptr(dm_out, self._dt(), self.NA, None)
            if dd != ds:
                raise ValueError("slopes and dm_out must both be host or both be device")
        fn = lib().fewha_frame
        args = (self.h, ps, ctypes.c_int(int(n_iter)), ctypes.c_int(1 if warm else 0), ctypes.c_double(float(gain)),
                ctypes.c_int(int(n_fit)), pl, pd, ctypes.c_int(ds))
        check = self._check

        def run():
            st = fn(*args)
            if st:
                check(st)

        run.buffers = (slopes, layers_out, dm_out)   # kept alive with the function
        return run

    def arm_frame(self, slopes, n_iter: int, warm: bool = True, layers_out=None, wait_s: float = 1.0):
        """Launch a host frame ahead of its slopes (fewha_frame_arm): fill
        `slopes` in place, then fire_frame().  Pinned host arrays only."""
        ps, ds = _ptr(slopes, self._dt(), self.S, None)
        pl, dl = _ptr(layers_out, self._dt(), self.N, None)
        if ds or dl:
            raise ValueError("armed frames take pinned host arrays")
        self._armed_buffers = (slopes, layers_out)
        self._check(lib().fewha_frame_arm(self.h, ps, int(n_iter), 1 if warm else 0, pl, float(wait_s)))

    def fire_frame(self):
        """Let the armed frame run and wait for its layers (fewha_frame_fire)."""
        try:
            self._check(lib().fewha_frame_fire(self.h))
        finally:
            self._armed_buffers = None

    def launch_count(self) -> int:
        return int(lib().fewha_launch_count(self.h))

    def frame_timing(self) -> dict:
        """Host-side timing of the last frame() (us): prep, launch, wait, total."""
        t = (ctypes.c_double * 6)()
        self._check(lib().fewha_get_frame_timing(self.h, t))
        return {"prep_us": t[0], "launch_us": t[1], "wait_us": t[2], "total_us": t[3],
                "repointed": bool(t[4]), "captured": bool(t[5])}

    def set_cluster_size(self, cluster_size: int):
        self._check(lib().fewha_set_cluster_size(self.h, int(cluster_size)))

    def set_host_transfer(self, slopes_by_copy: bool):
        """Host frames on the fused path: slopes by one copy-engine transfer
        (True, default) or read by the kernel through the pinned mapping."""
        self._check(lib().fewha_set_host_transfer(self.h, 1 if slopes_by_copy else 0))

    def set_layer_transform(self, form: int):
        """Fused layer phase: 0 row stripes (a cluster barrier per DWT level),
        1 level-stacked (one exchange per transform), -1 automatic."""
        self._check(lib().fewha_set_layer_transform(self.h, int(form)))

    def autotune(self, n_iter: int = 4, reps: int = 5) -> str:
        """Time the feasible fused-kernel shapes on the current frame, keep the fastest."""
        buf = ctypes.create_string_buffer(512)
        self._check(lib().fewha_autotune(self.h, int(n_iter), int(reps), buf, 512))
        return buf.value.decode()

    def describe(self) -> str:
        buf = ctypes.create_string_buffer(512)
        self._check(lib().fewha_describe(self.h, buf, 512))
        return buf.value.decode()

    # -- differentiation (device tensors only) --
    @property
    def n_layers(self) -> int:
        return len(self.cfg["layers"])

    @property
    def n_wfs(self) -> int:
        return len(self.cfg["wfs"])

    def set_params(self, cn2, alpha: float, w):
        """New Cn^2 fractions, alpha and sensor weights for M and b (the
        Jacobi preconditioner keeps its create-time value)."""
        cn2 = np.ascontiguousarray(np.asarray(cn2, np.float64).ravel())
        w = np.ascontiguousarray(np.asarray(w, np.float64).ravel())
        if cn2.size != self.n_layers or w.size != self.n_wfs:
            raise ValueError("need %d Cn^2 fractions and %d sensor weights" % (self.n_layers, self.n_wfs))
        dp = ctypes.POINTER(ctypes.c_double)
        self._check(lib().fewha_set_params(self.h, cn2.ctypes.data_as(dp), float(alpha), w.ctypes.data_as(dp)))

    def tape_bytes(self, n_iter: int) -> int:
        return int(lib().fewha_tape_bytes(self.h, int(n_iter)))

    def solve_taped(self, slopes, n_iter: int, tape, layers_out=None):
        ps, ds = _ptr(slopes, self._dt(), self.S, None)
        if not ds or not tape.is_cuda or tape.numel() < self.tape_bytes(n_iter) or tape.data_ptr() % 8:
            raise ValueError("device slopes and an 8-byte aligned device tape of tape_bytes(n_iter) bytes needed")
        pl = None
        if layers_out is not None:
            pl, dl = _ptr(layers_out, self._dt(), self.N, None)
            if not dl:
                raise ValueError("layers_out must be a device tensor")
        self._check(lib().fewha_solve_taped(self.h, ps, int(n_iter), ctypes.c_void_p(tape.data_ptr()), pl))

    def backward(self, slopes, n_iter: int, tape, layers_bar, g_cn2, g_alpha, g_w, g_slopes=None):
        import torch
        ps, ds = _ptr(slopes, self._dt(), self.S, None)
        pb, db = _ptr(layers_bar, self._dt(), self.N, None)
        for t, n in ((g_cn2, self.n_layers), (g_alpha, 1), (g_w, self.n_wfs)):
            if not (t.is_cuda and t.dtype == torch.float64 and t.numel() == n and t.is_contiguous()):
                raise ValueError("gradients must be contiguous float64 device tensors")
        pg = None
        if g_slopes is not None:
            pg, dg = _ptr(g_slopes, self._dt(), self.S, None)
        if not (ds and db):
            raise ValueError("device tensors needed")
        self._check(lib().fewha_backward(self.h, ps, int(n_iter), ctypes.c_void_p(tape.data_ptr()), pb,
                                         ctypes.c_void_p(g_cn2.data_ptr()), ctypes.c_void_p(g_alpha.data_ptr()),
                                         ctypes.c_void_p(g_w.data_ptr()), pg))

    def tape_bytes_batch(self, n_iter: int, n_frames: int) -> int:
        return int(lib().fewha_tape_bytes_batch(self.h, int(n_iter), int(n_frames)))

    def solve_taped_batch(self, slopes, n_iter: int, tape, layers_out=None):
        """Taped solves of every frame of slopes ([B, S] device tensor) in one
        launch sequence; layers_out [B, N] or None."""
        if not (slopes.is_cuda and slopes.dtype == self.torch_dtype and slopes.dim() == 2 and
                slopes.shape[1] == self.S and slopes.is_contiguous()):
            raise ValueError("slopes must be a contiguous [frames, S] device tensor of the solver's dtype")
        B = int(slopes.shape[0])
        if not (tape.is_cuda and tape.numel() >= self.tape_bytes_batch(n_iter, B) and tape.data_ptr() % 8 == 0):
            raise ValueError("an 8-byte aligned device tape of tape_bytes_batch(n_iter, frames) bytes needed")
        pl = None
        if layers_out is not None:
            if not (layers_out.is_cuda and layers_out.dtype == self.torch_dtype and
                    tuple(layers_out.shape) == (B, self.N) and layers_out.is_contiguous()):
                raise ValueError("layers_out must be a contiguous [frames, N] device tensor")
            pl = ctypes.c_void_p(layers_out.data_ptr())
        self._check(lib().fewha_solve_taped_batch(self.h, B, ctypes.c_void_p(slopes.data_ptr()), int(n_iter),
                                                  ctypes.c_void_p(tape.data_ptr()), pl))

    def backward_batch(self, slopes, n_iter: int, tape, layers_bar, g_cn2, g_alpha, g_w, g_slopes=None):
        """Reverse mode of solve_taped_batch: per-frame gradients g_cn2 [B, L],
        g_alpha [B], g_w [B, G] (float64) and g_slopes [B, S] (or None)."""
        import torch
        B = int(slopes.shape[0])
        for t, shp, dt in ((layers_bar, (B, self.N), self.torch_dtype), (g_cn2, (B, self.n_layers), torch.float64),
                           (g_alpha, (B,), torch.float64), (g_w, (B, self.n_wfs), torch.float64)):
            if not (t.is_cuda and t.dtype == dt and tuple(t.shape) == shp and t.is_contiguous()):
                raise ValueError("layers_bar and the gradients: contiguous device tensors of shape %s" % (shp,))
        pg = None
        if g_slopes is not None:
            if not (g_slopes.is_cuda and g_slopes.dtype == self.torch_dtype and tuple(g_slopes.shape) == (B, self.S)
                    and g_slopes.is_contiguous()):
                raise ValueError("g_slopes must be a contiguous [frames, S] device tensor")
            pg = ctypes.c_void_p(g_slopes.data_ptr())
        vp = ctypes.c_void_p
        self._check(lib().fewha_backward_batch(self.h, B, vp(slopes.data_ptr()), int(n_iter), vp(tape.data_ptr()),
                                               vp(layers_bar.data_ptr()), vp(g_cn2.data_ptr()),
                                               vp(g_alpha.data_ptr()), vp(g_w.data_ptr()), pg))

    def set_trace(self, on: bool = True):
        self._check(lib().fewha_set_trace(self.h, 1 if on else 0))

    def trace(self):
        """Last fused launch: array [slot, cta, (arrive, depart)] of globaltimer ns."""
        slots, grid = ctypes.c_int(), ctypes.c_int()
        self._check(lib().fewha_get_trace(self.h, None, 0, ctypes.byref(slots), ctypes.byref(grid)))
        n = slots.value * grid.value * 2
        out = np.zeros(max(n, 1), np.uint64)
        self._check(lib().fewha_get_trace(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_ulonglong)), n,
                                          ctypes.byref(slots), ctypes.byref(grid)))
        return out[:n].reshape(slots.value, grid.value, 2)

    def fine_trace(self):
        """Last fused launch: per CTA a list of (tag, ns) marks inside the phases."""
        per, grid = ctypes.c_int(), ctypes.c_int()
        self._check(lib().fewha_get_fine_trace(self.h, None, 0, ctypes.byref(per), ctypes.byref(grid)))
        n = per.value * grid.value
        out = np.zeros(max(n, 1), np.uint64)
        self._check(lib().fewha_get_fine_trace(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_ulonglong)), n,
                                               ctypes.byref(per), ctypes.byref(grid)))
        return _marks(out[:n].reshape(grid.value, per.value))


class Batch:
    """Many independent FP32 instances advanced together, one fused launch per
    frame or one per group of instances (a fewha_batch).  Slopes and layers
    are concatenated in instance order; `slope_off` / `coeff_off` give each
    instance's slice."""

    def __init__(self, cfgs: list, stream=None, max_tile_side: int = 24, cluster_size: int = 0,
                 k_rr: int | None = None):
        import torch
        L = lib()
        n = len(cfgs)
        if n < 1:
            raise ValueError("empty batch")
        geoms = (Geometry * n)()
        profs = (Profile * n)()
        for i, cfg in enumerate(cfgs):
            geoms[i], profs[i] = structs_from_config(cfg, FP32)
        self._stream_obj = torch.cuda.Stream() if stream is None else stream
        self.stream = self._stream_obj
        b = ctypes.c_void_p()
        st = L.fewha_batch_create(n, geoms, profs, ctypes.c_void_p(self._stream_obj.cuda_stream),
                                  int(max_tile_side), int(cluster_size), ctypes.byref(b))
        if st != 0:
            raise FewhaError(st, L.fewha_batch_last_error(None).decode())
        self.h = b
        cnt = ctypes.c_int()
        co = (ctypes.c_long * (n + 1))()
        so = (ctypes.c_long * (n + 1))()
        L.fewha_batch_sizes(b, ctypes.byref(cnt), co, so)
        self.count = cnt.value
        self.coeff_off = np.array(co[:], np.int64)
        self.slope_off = np.array(so[:], np.int64)
        self.N, self.S = int(self.coeff_off[-1]), int(self.slope_off[-1])
        self.cfgs = cfgs
        if k_rr is not None:
            self._check(L.fewha_batch_set_residual_replacement(self.h, int(k_rr)))

    def _check(self, st):
        if st != 0:
            raise FewhaError(st, lib().fewha_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().fewha_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def concat_slopes(self, per_instance) -> np.ndarray:
        """One host slope vector from a list of per-instance slope vectors."""
        return np.concatenate([np.asarray(v, np.float32).ravel() for v in per_instance])

    def split_layers(self, layers) -> list:
        return [layers[self.coeff_off[i]:self.coeff_off[i + 1]] for i in range(self.count)]

    def frame(self, slopes, n_iter: int, warm: bool = True, layers_out=None):
        """One frame of every instance.  Host arrays (numpy; the call
        synchronises) or device tensors (the call only enqueues)."""
        import torch
        dt = (np.float32, torch.float32)
        ps, ds = _ptr(slopes, dt, self.S, None)
        pl = None
        if layers_out is not None:
            pl, dl = _ptr(layers_out, dt, self.N, None)
            if dl != ds:
                raise ValueError("slopes and layers_out must both be host or both be device")
        self._check(lib().fewha_batch_frame(self.h, ps, int(n_iter), 1 if warm else 0, pl, ds))

    def get_state(self, i: int):
        nn = int(self.coeff_off[i + 1] - self.coeff_off[i])
        c, b, r = (np.empty(nn, np.float32) for _ in range(3))
        self._check(lib().fewha_batch_get_state(self.h, int(i), ctypes.c_void_p(c.ctypes.data),
                                                ctypes.c_void_p(b.ctypes.data), ctypes.c_void_p(r.ctypes.data), 0))
        return c, b, r

    def sync(self):
        self._check(lib().fewha_batch_sync(self.h))

    def set_trace(self, on: bool = True):
        self._check(lib().fewha_batch_set_trace(self.h, 1 if on else 0))

    def fine_trace(self):
        """Last traced frame: per CTA a list of (tag, ns) marks inside the
        phases (the CTAs of every launch of the frame, in launch order)."""
        per, grid = ctypes.c_int(), ctypes.c_int()
        self._check(lib().fewha_batch_get_fine_trace(self.h, None, 0, ctypes.byref(per), ctypes.byref(grid)))
        n = per.value * grid.value
        out = np.zeros(max(n, 1), np.uint64)
        self._check(lib().fewha_batch_get_fine_trace(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_ulonglong)),
                                                     n, ctypes.byref(per), ctypes.byref(grid)))
        return _marks(out[:n].reshape(grid.value, per.value))

    def describe(self) -> str:
        buf = ctypes.create_string_buffer(1024)
        self._check(lib().fewha_batch_describe(self.h, buf, 1024))
        return buf.value.decode()

    def launch_count(self) -> int:
        return int(lib().fewha_batch_launch_count(self.h))

    def autotune(self, n_iter: int = 4, reps: int = 3) -> str:
        """Time the groupings of the instances by layer size and, per group,
        the feasible cluster shapes and sensor-tile bounds on the current
        slopes (after a frame); keep the fastest."""
        buf = ctypes.create_string_buffer(2048)
        self._check(lib().fewha_batch_autotune(self.h, int(n_iter), int(reps), buf, 2048))
        return buf.value.decode()

    def set_max_launches(self, m: int):
        """Bound on the launches per frame the autotuner may choose (0: none)."""
        self._check(lib().fewha_batch_set_max_launches(self.h, int(m)))

    def set_groups(self, group):
        """group[i]: the launch (0 .. G - 1) that advances instance i."""
        g = np.ascontiguousarray(group, np.int32)
        if g.shape != (self.count,):
            raise ValueError("one launch index per instance")
        self._check(lib().fewha_batch_set_groups(self.h, g.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                                 self.count))


def measure_l2(nbytes: int = 48 << 20, passes: int = 40, reps: int = 5) -> dict:
    """Achievable L2 bandwidth of the current GPU (fewha_measure_l2): a buffer
    of nbytes resident in L2 read, and copied half to half, passes times per
    launch; the fastest of reps launches, GB/s (read, and read + write)."""
    rd, cp = ctypes.c_double(), ctypes.c_double()
    msg = ctypes.create_string_buffer(256)
    st = lib().fewha_measure_l2(int(nbytes), int(passes), int(reps), ctypes.byref(rd), ctypes.byref(cp), msg, 256)
    if st:
        raise FewhaError(st, msg.value.decode())
    return {"read_gbs": rd.value, "copy_gbs": cp.value, "bytes": int(nbytes), "passes": int(passes),
            "reps": int(reps)}


# bounds-check sites of the debug build (include/fewha.h, FEWHA_DBG_*)
DEBUG_SITES = {1: "sensor bilinear read of the layers", 2: "reserved", 3: "reserved",
               4: "slope index", 5: "Gamma^T output", 6: "field staging source", 7: "field staging",
               8: "P^T gather read", 9: "DWT store into a row owner", 10: "DWT store into a column owner",
               11: "coefficient index", 12: "tip-tilt correction", 13: "layer output",
               14: "row-stripe DWT peer read", 15: "table staging", 16: "plain P", 17: "plain P^T",
               18: "plain Gamma / Gamma^T", 19: "fit", 20: "no-allocation transform"}


def debug_bounds() -> dict:
    """Violations recorded by the debug build's bounds checks since the last
    call (and clears them): {"debug_build", "count", "site", "index"}.  The
    release build checks nothing and reports debug_build False."""
    first, count = ctypes.c_ulonglong(), ctypes.c_ulonglong()
    st = lib().fewha_debug_bounds(ctypes.byref(first), ctypes.byref(count))
    if st < 0:
        raise FewhaError(st, "reading the bounds-check records failed")
    site = int(first.value >> 48)
    idx = int(first.value & ((1 << 48) - 1))
    if idx >= 1 << 47:
        idx -= 1 << 48
    return {"debug_build": st == 1, "count": int(count.value), "site": DEBUG_SITES.get(site, site) if site else None,
            "index": idx if site else None}
