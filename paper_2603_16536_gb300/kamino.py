"""Python binding of the kamino C ABI (``include/kamino.h``): argument marshalling only.

Every computation of the step runs in the library's CUDA kernels.  PyTorch provides the device
memory of the state (one ``uint8`` buffer, carved by the library) and the CUDA stream; the views
returned here are zero-copy tensors over that buffer.  There is no CPU fallback: loading fails
loudly when the shared library has not been built, and stepping fails when no GPU is present.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from dataclasses import dataclass

import numpy as np

from . import build as _build

FP32, FP64, MIXED = 0, 1, 2
WARM_COLD, WARM_CACHED, WARM_EXTERNAL = 0, 1, 2
BUF_BODY_Q, BUF_BODY_U, BUF_CACHE, BUF_WARM, BUF_RESIDUAL, BUF_TAU = 0, 1, 2, 3, 4, 5
WORLD_NOT_CONVERGED, WORLD_NONFINITE, WORLD_TIMEOUT, WORLD_STALLED = 1, 2, 4, 8
STATUS = {0: "KAMINO_OK", 1: "KAMINO_E_INVALID_ARG", 2: "KAMINO_E_TOPOLOGY", 3: "KAMINO_E_NOMEM",
          4: "KAMINO_E_CUDA", 5: "KAMINO_E_NONFINITE", 6: "KAMINO_E_TIMEOUT", 7: "KAMINO_E_UNSUPPORTED"}


class KaminoError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class SolverParams(C.Structure):
    _fields_ = [("eta", C.c_double), ("rho", C.c_double), ("beta", C.c_double), ("margin", C.c_double),
                ("nesterov", C.c_int32), ("precond", C.c_int32), ("warm_mode", C.c_int32), ("refine64", C.c_int32),
                ("integrator", C.c_int32), ("cr_iters", C.c_int32), ("ncp_stop", C.c_int32),
                ("stall_window", C.c_int32), ("schedule", C.c_int32), ("residual_every", C.c_int32)]


INTEGRATOR_EULER, INTEGRATOR_MIDPOINT = 0, 1


def make_params(eta=1e-6, rho=0.1, beta=0.2, margin=0.005, nesterov=True, precond=True, warm_mode=WARM_COLD,
                refine64=True, integrator=INTEGRATOR_EULER, cr_iters=0, ncp_stop=False, stall_window=0,
                schedule=1, residual_every=8):
    """Solver parameters (kamino_solver_params); ``schedule`` 1 = KAMINO_SCHEDULE_LONGEST_FIRST;
    ``residual_every`` 8 = the dense x-step's refinement residual evaluated every 8th iteration."""
    return SolverParams(eta, rho, beta, margin, int(nesterov), int(precond), int(warm_mode), int(refine64),
                        int(integrator), int(cr_iters), int(ncp_stop), int(stall_window), int(schedule),
                        int(residual_every))


_P = C.c_void_p


class ModelDesc(C.Structure):
    _fields_ = [("num_worlds", C.c_int32), ("precision", C.c_int32),
                ("world_body_offset", _P), ("world_joint_offset", _P), ("world_contact_offset", _P),
                ("world_num_actuators", _P), ("world_mu", _P), ("body_mass", _P), ("body_inertia", _P),
                ("joint_type", _P), ("joint_parent", _P), ("joint_child", _P), ("joint_actuator", _P),
                ("joint_frame_parent", _P), ("joint_frame_child", _P), ("contact_body", _P),
                ("contact_point", _P), ("gravity", C.c_double * 3), ("terrain_kind", C.c_int32),
                ("hf_nx", C.c_int32), ("hf_ny", C.c_int32), ("hf_origin", C.c_double * 2), ("hf_cell", C.c_double),
                ("hf_heights", _P), ("body_q0", _P), ("body_u0", _P), ("params", SolverParams),
                ("joint_drive", _P), ("joint_limit", _P)]

DRIVE_TORQUE, DRIVE_PD = 0, 1


class ModelInfo(C.Structure):
    _fields_ = [("num_worlds", C.c_int32), ("num_bodies", C.c_int32), ("max_bodies", C.c_int32),
                ("max_rows", C.c_int32), ("n_act_max", C.c_int32), ("cache_len", C.c_int32),
                ("precision", C.c_int32), ("threads_per_world", C.c_int32), ("smem_bytes", C.c_int64)]


LAUNCH_SINGLE, LAUNCH_PERSISTENT = 0, 1


class BucketInfo(C.Structure):
    _fields_ = [("rows_pad", C.c_int32), ("num_worlds", C.c_int32), ("group_threads", C.c_int32),
                ("panel", C.c_int32), ("grid", C.c_int32), ("worlds_per_cta", C.c_int32),
                ("tuned_ms", C.c_float), ("reserved", C.c_float)]


class MlpInfo(C.Structure):
    _fields_ = [("num_worlds", C.c_int32), ("d_in", C.c_int32), ("d_hidden", C.c_int32),
                ("hidden_layers", C.c_int32), ("d_out", C.c_int32), ("max_batch", C.c_int32),
                ("num_params", C.c_int64)]


RESIDUAL_DTYPE = np.dtype([("iterations", np.int32), ("status", np.int32), ("num_rows", np.int32),
                           ("num_contacts", np.int32), ("r_primal", np.float32), ("r_dual", np.float32),
                           ("r_compl", np.float32), ("r_ncp", np.float32)])

_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(path: str | None = None):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"kamino CUDA library not built ({path} missing); run paper_2603_16536_gb300.build.build()")
    lib = C.CDLL(path)
    vp, i32, i64, dbl, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_size_t
    sig = {
        "kamino_model_create": ([C.POINTER(ModelDesc), C.POINTER(vp)], i32),
        "kamino_model_destroy": ([vp], i32),
        "kamino_model_get_info": ([vp, C.POINTER(ModelInfo)], i32),
        "kamino_model_set_params": ([vp, C.POINTER(SolverParams)], i32),
        "kamino_state_bytes": ([vp, C.POINTER(sz)], i32),
        "kamino_state_alloc": ([vp, vp, sz, C.POINTER(vp)], i32),
        "kamino_state_free": ([vp], i32),
        "kamino_state_get": ([vp, i32, C.POINTER(vp), C.POINTER(i64)], i32),
        "kamino_state_upload": ([vp, i32, vp, i64, vp], i32),
        "kamino_state_download": ([vp, i32, vp, i64, vp], i32),
        "kamino_step": ([vp, dbl, i32, dbl, vp, vp], i32),
        "kamino_residuals": ([vp, vp, vp], i32),
        "kamino_fk": ([vp, vp, vp, vp, i32, dbl, vp], i32),
        "kamino_last_error": ([], C.c_char_p),
        "kamino_plan_get": ([vp, C.POINTER(BucketInfo), i32, C.POINTER(i32), C.POINTER(i32)], i32),
        "kamino_plan_set_mode": ([vp, i32], i32),
        "kamino_autotune": ([vp, dbl, i32, dbl, vp, vp], i32),
        "kamino_graph_create": ([vp, dbl, i32, dbl, vp, vp, C.POINTER(vp)], i32),
        "kamino_graph_launch": ([vp, vp], i32),
        "kamino_graph_destroy": ([vp], i32),
        "kamino_mlp_create": ([vp, vp, i32, i32, i32, C.c_uint64, C.POINTER(vp)], i32),
        "kamino_mlp_destroy": ([vp], i32),
        "kamino_mlp_get_info": ([vp, C.POINTER(MlpInfo)], i32),
        "kamino_mlp_features": ([vp, vp, vp, vp, vp], i32),
        "kamino_mlp_targets": ([vp, vp, vp, vp], i32),
        "kamino_mlp_fit_normalization": ([vp, vp, vp, i64, vp], i32),
        "kamino_mlp_train_step": ([vp, vp, vp, vp, i32, C.c_float, vp, vp], i32),
        "kamino_mlp_gradients": ([vp, vp, vp, vp, i32, vp, vp, vp], i32),
        "kamino_mlp_predict": ([vp, vp, i32, vp, vp], i32),
        "kamino_mlp_warm_start": ([vp, vp, vp, vp], i32),
        "kamino_mlp_get_params": ([vp, vp, i64], i32),
        "kamino_mlp_set_params": ([vp, vp, i64], i32),
        "kamino_mlp_get_normalization": ([vp, vp], i32),
        "kamino_mlp_set_normalization": ([vp, vp], i32),
        "kamino_mlp_predict_static": ([vp, vp, i32, vp, vp], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def header_functions(header: str | None = None) -> list[str]:
    """Names of the functions declared in include/kamino.h."""
    header = header or os.path.join(_build.ROOT, "include", "kamino.h")
    text = open(header).read()
    return sorted(set(re.findall(r"\b(kamino_[a-z_0-9]+)\s*\(", text)))


def _check(status):
    if status != 0:
        msg = load_library().kamino_last_error().decode()
        raise KaminoError(status, msg)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None and a.size else None


def _tau_ptr(tau, dtype, need):
    """Device pointer of an actuation tensor, after checking what the library cannot: a contiguous
    CUDA tensor of the state's element type with at least `need` elements (None passes through)."""
    if tau is None:
        return None
    if not (tau.is_cuda and tau.dtype == dtype and tau.is_contiguous() and tau.numel() >= need):
        raise ValueError(f"actuation must be a contiguous CUDA {dtype} tensor of >= {need} elements "
                         f"(got {tau.dtype}, {tau.numel()} elements, cuda={tau.is_cuda}, contiguous={tau.is_contiguous()})")
    return C.c_void_p(tau.data_ptr())


def _host_ptr(which, host, elem_dtype):
    """Pointer and element count of a host array for upload/download: the library copies `count`
    elements of the buffer's own type, so the array must be C-contiguous and of exactly that type
    (kamino_residual records for BUF_RESIDUAL) or it would read or write past the array."""
    want = RESIDUAL_DTYPE if which == BUF_RESIDUAL else np.dtype(elem_dtype)
    if not isinstance(host, np.ndarray) or host.dtype != want or not host.flags.c_contiguous:
        raise ValueError(f"host array must be a C-contiguous numpy array of {want}")
    return host.ctypes.data_as(C.c_void_p), host.size


class Model:
    """A set of worlds on the device (kamino_model_create)."""

    def __init__(self, ws, precision: str = "fp32", params: SolverParams | None = None):
        lib = load_library()
        self.precision = {"fp32": FP32, "fp64": FP64, "mixed": MIXED, FP32: FP32, FP64: FP64, MIXED: MIXED}[precision]
        self.ws = ws
        keep = {
            "bo": np.ascontiguousarray(ws.world_body_offset, np.int32),
            "jo": np.ascontiguousarray(ws.world_joint_offset, np.int32),
            "co": np.ascontiguousarray(ws.world_contact_offset, np.int32),
            "na": np.ascontiguousarray(ws.world_num_actuators, np.int32),
            "mu": np.ascontiguousarray(ws.world_mu, np.float64),
            "mass": np.ascontiguousarray(ws.body_mass, np.float64),
            "inert": np.ascontiguousarray(ws.body_inertia, np.float64).reshape(-1),
            "jt": np.ascontiguousarray(ws.joint_type, np.int32),
            "jp": np.ascontiguousarray(ws.joint_parent, np.int32),
            "jc": np.ascontiguousarray(ws.joint_child, np.int32),
            "ja": np.ascontiguousarray(ws.joint_actuator, np.int32),
            "fp": np.ascontiguousarray(ws.joint_frame_parent, np.float64).reshape(-1),
            "fc": np.ascontiguousarray(ws.joint_frame_child, np.float64).reshape(-1),
            "cb": np.ascontiguousarray(ws.contact_body, np.int32),
            "cp": np.ascontiguousarray(ws.contact_point, np.float64).reshape(-1),
            "hh": np.ascontiguousarray(ws.hf_heights, np.float64).reshape(-1),
            "q0": np.ascontiguousarray(ws.body_q0, np.float64).reshape(-1),
            "u0": np.ascontiguousarray(ws.body_u0, np.float64).reshape(-1),
        }
        drive, limit = getattr(ws, "joint_drive", None), getattr(ws, "joint_limit", None)
        if drive is not None:
            keep["drv"] = np.ascontiguousarray(drive, np.float64).reshape(-1)
            if keep["drv"].size != 5 * len(ws.joint_type):
                raise ValueError("joint_drive must hold 5 values per joint")
        if limit is not None:
            keep["lim"] = np.ascontiguousarray(limit, np.float64).reshape(-1)
            if keep["lim"].size != 2 * len(ws.joint_type):
                raise ValueError("joint_limit must hold 2 values per joint")
        d = ModelDesc()
        d.num_worlds = ws.num_worlds
        d.precision = self.precision
        d.world_body_offset, d.world_joint_offset = _ptr(keep["bo"]), _ptr(keep["jo"])
        d.world_contact_offset, d.world_num_actuators = _ptr(keep["co"]), _ptr(keep["na"])
        d.world_mu, d.body_mass, d.body_inertia = _ptr(keep["mu"]), _ptr(keep["mass"]), _ptr(keep["inert"])
        d.joint_type, d.joint_parent, d.joint_child = _ptr(keep["jt"]), _ptr(keep["jp"]), _ptr(keep["jc"])
        d.joint_actuator, d.joint_frame_parent, d.joint_frame_child = _ptr(keep["ja"]), _ptr(keep["fp"]), _ptr(keep["fc"])
        d.contact_body, d.contact_point = _ptr(keep["cb"]), _ptr(keep["cp"])
        d.gravity = (C.c_double * 3)(*[float(g) for g in ws.gravity])
        d.terrain_kind = int(ws.terrain_kind)
        d.hf_nx, d.hf_ny = int(ws.hf_nx), int(ws.hf_ny)
        d.hf_origin = (C.c_double * 2)(*[float(v) for v in ws.hf_origin])
        d.hf_cell = float(ws.hf_cell)
        d.hf_heights = _ptr(keep["hh"])
        d.body_q0, d.body_u0 = _ptr(keep["q0"]), _ptr(keep["u0"])
        d.joint_drive = _ptr(keep["drv"]) if "drv" in keep else None
        d.joint_limit = _ptr(keep["lim"]) if "lim" in keep else None
        d.params = params if params is not None else make_params()
        self.handle = C.c_void_p()
        _check(lib.kamino_model_create(C.byref(d), C.byref(self.handle)))
        info = ModelInfo()
        _check(lib.kamino_model_get_info(self.handle, C.byref(info)))
        self.info = info
        self.params = d.params

    def set_params(self, params: SolverParams):
        _check(load_library().kamino_model_set_params(self.handle, C.byref(params)))
        self.params = params

    def plan(self):
        """(mode, [bucket dicts]) of the current launch plan."""
        cap = 64
        arr = (BucketInfo * cap)()
        n, mode = C.c_int32(), C.c_int32()
        _check(load_library().kamino_plan_get(self.handle, arr, cap, C.byref(n), C.byref(mode)))
        out = [{f: getattr(arr[i], f) for f, _ in BucketInfo._fields_ if f != "reserved"} for i in range(n.value)]
        return mode.value, out

    def set_launch_mode(self, mode: int):
        _check(load_library().kamino_plan_set_mode(self.handle, int(mode)))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.kamino_model_destroy(self.handle)
            self.handle = None


class State:
    """Device state of a model over one PyTorch-allocated buffer (kamino_state_alloc)."""

    def __init__(self, model: Model, device="cuda"):
        import torch
        lib = load_library()
        self.model = model
        nbytes = C.c_size_t()
        _check(lib.kamino_state_bytes(model.handle, C.byref(nbytes)))
        self._raw = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=device)
        base = self._raw.data_ptr()
        self._off = (-base) % 256
        self.handle = C.c_void_p()
        _check(lib.kamino_state_alloc(model.handle, C.c_void_p(base + self._off), nbytes.value, C.byref(self.handle)))
        self.dtype = torch.float64 if model.precision == FP64 else torch.float32
        self._np_dtype = np.float64 if model.precision == FP64 else np.float32
        self._tau_len = model.ws.num_worlds * max(model.info.n_act_max, 0)
        self.body_q = self._view(BUF_BODY_Q, self.dtype).view(-1, 7)
        self.body_u = self._view(BUF_BODY_U, self.dtype).view(-1, 6)
        self.cache = self._view(BUF_CACHE, self.dtype)
        self.warm = self._view(BUF_WARM, self.dtype)
        self.residual_raw = self._view(BUF_RESIDUAL, torch.int32).view(-1, 8)
        self.tau = self._view(BUF_TAU, self.dtype)

    def _view(self, which, dtype):
        import torch
        ptr, count = C.c_void_p(), C.c_int64()
        _check(load_library().kamino_state_get(self.handle, which, C.byref(ptr), C.byref(count)))
        esz = torch.empty(0, dtype=dtype).element_size() if which != BUF_RESIDUAL else 4
        n = count.value * (8 if which == BUF_RESIDUAL else 1)
        start = (ptr.value or 0) - self._raw.data_ptr()
        return self._raw[start:start + n * esz].view(dtype)

    def step(self, dt: float, iters: int, tol: float, tau=None, stream=None):
        """One step of every world (kamino_step).  ``tau``: device tensor [W, n_act_max] or None."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        tptr = _tau_ptr(tau, self.dtype, self._tau_len)
        _check(load_library().kamino_step(self.handle, float(dt), int(iters), float(tol), tptr,
                                          C.c_void_p(stream.cuda_stream)))

    def fk(self, targets, select=None, fixed=None, max_iters: int = 50, tol: float = 1e-12, stream=None):
        """Gauss-Newton forward kinematics for resets (kamino_fk): ``targets`` device float64 [J] joint
        coordinates, ``select`` device int32 [J] (None: the actuated joints), ``fixed`` device int32
        [B] bodies that keep their poses (None: none).  Poses are updated in place; the per-world
        report (iterations, status, max |F| in r_primal) is in residuals()."""
        import torch
        stream = stream or torch.cuda.current_stream()
        nj, nb = len(self.model.ws.joint_type), int(self.model.ws.world_body_offset[-1])
        tp = _dev(targets, torch.float64, "targets", min_numel=nj)
        sp = None if select is None else _dev(select, torch.int32, "select", min_numel=nj)
        fp = None if fixed is None else _dev(fixed, torch.int32, "fixed", min_numel=nb)
        _check(load_library().kamino_fk(self.handle, tp, sp, fp, int(max_iters), float(tol),
                                        C.c_void_p(stream.cuda_stream)))

    def autotune(self, dt: float, iters: int, tol: float, tau=None, stream=None):
        """Time every feasible per-bucket configuration on this state's worlds (state unchanged)."""
        import torch
        stream = stream or torch.cuda.current_stream()
        tptr = _tau_ptr(tau, self.dtype, self._tau_len)
        _check(load_library().kamino_autotune(self.handle, float(dt), int(iters), float(tol), tptr,
                                              C.c_void_p(stream.cuda_stream)))

    def graph(self, dt: float, iters: int, tol: float, tau=None, stream=None):
        """Capture one step into a CUDA graph (returns a StepGraph)."""
        import torch
        stream = stream or torch.cuda.current_stream()
        tptr = _tau_ptr(tau, self.dtype, self._tau_len)
        h = C.c_void_p()
        _check(load_library().kamino_graph_create(self.handle, float(dt), int(iters), float(tol), tptr,
                                                  C.c_void_p(stream.cuda_stream), C.byref(h)))
        return StepGraph(h, self)

    def upload(self, which, host: np.ndarray, stream=None):
        import torch
        s = (stream or torch.cuda.current_stream()).cuda_stream
        ptr, n = _host_ptr(which, host, self._np_dtype)
        _check(load_library().kamino_state_upload(self.handle, which, ptr, n, C.c_void_p(s)))

    def download(self, which, host: np.ndarray, stream=None):
        import torch
        s = (stream or torch.cuda.current_stream()).cuda_stream
        ptr, n = _host_ptr(which, host, self._np_dtype)
        _check(load_library().kamino_state_download(self.handle, which, ptr, n, C.c_void_p(s)))

    def residuals(self) -> np.ndarray:
        """Per-world reports as a numpy structured array (synchronises the current stream)."""
        raw = self.residual_raw.cpu().numpy()
        return raw.view(RESIDUAL_DTYPE).reshape(-1)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.kamino_state_free(self.handle)
            self.handle = None


class StepGraph:
    """A captured step (kamino_graph_create); launch() replays it on a stream."""

    def __init__(self, handle, state):
        self.handle = handle
        self.state = state     # keeps the state alive while the graph exists

    def launch(self, stream=None):
        import torch
        stream = stream or torch.cuda.current_stream()
        _check(load_library().kamino_graph_launch(self.handle, C.c_void_p(stream.cuda_stream)))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.kamino_graph_destroy(self.handle)
            self.handle = None


def _dptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _dev(t, dtype, name, cols=None, min_numel=0):
    """Device pointer of a tensor the library will read or write through a raw pointer, after the
    checks it cannot make: a contiguous CUDA tensor of `dtype`, `cols` columns when given, and at
    least `min_numel` elements (None passes through; the library rejects it where it is required)."""
    if t is None:
        return None
    ok = t.is_cuda and t.dtype == dtype and t.is_contiguous() and t.numel() >= min_numel
    if ok and cols is not None:
        ok = t.dim() == 2 and t.shape[1] == cols
    if not ok:
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor"
                         + (f" with {cols} columns" if cols is not None else "")
                         + f" and >= {min_numel} elements (got {t.dtype}, shape {tuple(t.shape)})")
    return C.c_void_p(t.data_ptr())


def _sptr(stream):
    import torch
    return C.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)


class Mlp:
    """Warm-start network for the worlds `worlds` of one type (kamino_mlp_create)."""

    def __init__(self, model: Model, worlds, hidden: int = 256, max_batch: int = 4096, seed: int = 0):
        self.model = model
        w = np.ascontiguousarray(worlds, np.int32)
        self.worlds = w
        self.handle = C.c_void_p()
        _check(load_library().kamino_mlp_create(model.handle, w.ctypes.data_as(C.c_void_p), len(w), int(hidden),
                                                int(max_batch), C.c_uint64(seed), C.byref(self.handle)))
        info = MlpInfo()
        _check(load_library().kamino_mlp_get_info(self.handle, C.byref(info)))
        self.info = info

    def _xy(self, X, Y):
        import torch
        xp = _dev(X, torch.float32, "X", cols=self.info.d_in)
        yp = _dev(Y, torch.float32, "Y", cols=self.info.d_out)
        if X is not None and Y is not None and X.shape[0] != Y.shape[0]:
            raise ValueError(f"X and Y must have the same rows (got {X.shape[0]} and {Y.shape[0]})")
        return xp, yp

    def features(self, state: State, tau=None, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.info.num_worlds, self.info.d_in), dtype=torch.float32, device=state._raw.device)
        op = _dev(out, torch.float32, "out", min_numel=self.info.num_worlds * self.info.d_in)
        _check(load_library().kamino_mlp_features(self.handle, state.handle, _tau_ptr(tau, state.dtype, state._tau_len),
                                                  op, _sptr(stream)))
        return out

    def targets(self, state: State, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.info.num_worlds, self.info.d_out), dtype=torch.float32, device=state._raw.device)
        op = _dev(out, torch.float32, "out", min_numel=self.info.num_worlds * self.info.d_out)
        _check(load_library().kamino_mlp_targets(self.handle, state.handle, op, _sptr(stream)))
        return out

    def fit_normalization(self, X, Y, stream=None):
        xp, yp = self._xy(X, Y)
        _check(load_library().kamino_mlp_fit_normalization(self.handle, xp, yp, X.shape[0], _sptr(stream)))

    def train_step(self, X, Y, rows=None, lr=1e-3, loss=None, stream=None):
        import torch
        xp, yp = self._xy(X, Y)
        batch = self.info.num_worlds if rows is None and X is None else (rows.numel() if rows is not None else X.shape[0])
        _check(load_library().kamino_mlp_train_step(self.handle, xp, yp, _dev(rows, torch.int32, "rows"), int(batch),
                                                    float(lr), _dev(loss, torch.float32, "loss", min_numel=1),
                                                    _sptr(stream)))

    def gradients(self, X, Y, rows=None, stream=None):
        import torch
        xp, yp = self._xy(X, Y)
        batch = rows.numel() if rows is not None else X.shape[0]
        g = torch.empty(self.info.num_params, dtype=torch.float32, device=X.device)
        loss = torch.zeros(1, dtype=torch.float32, device=X.device)
        _check(load_library().kamino_mlp_gradients(self.handle, xp, yp, _dev(rows, torch.int32, "rows"), int(batch),
                                                   _dptr(g), _dptr(loss), _sptr(stream)))
        return g, loss

    def predict(self, X, stream=None):
        import torch
        xp = _dev(X, torch.float32, "X", cols=self.info.d_in)
        y = torch.empty((X.shape[0], self.info.d_out), dtype=torch.float32, device=X.device)
        _check(load_library().kamino_mlp_predict(self.handle, xp, X.shape[0], _dptr(y), _sptr(stream)))
        return y

    def predict_static(self, X, out=None, stream=None):
        """kamino_mlp_predict without allocation: activations in the library's static scratch."""
        import torch
        xp = _dev(X, torch.float32, "X", cols=self.info.d_in)
        y = out if out is not None else torch.empty((X.shape[0], self.info.d_out), dtype=torch.float32,
                                                    device=X.device)
        yp = _dev(y, torch.float32, "out", min_numel=X.shape[0] * self.info.d_out)
        _check(load_library().kamino_mlp_predict_static(self.handle, xp, X.shape[0], yp, _sptr(stream)))
        return y

    def warm_start(self, state: State, tau=None, stream=None):
        _check(load_library().kamino_mlp_warm_start(self.handle, state.handle, _tau_ptr(tau, state.dtype, state._tau_len),
                                                    _sptr(stream)))

    def get_params(self) -> np.ndarray:
        out = np.empty(self.info.num_params, np.float32)
        _check(load_library().kamino_mlp_get_params(self.handle, out.ctypes.data_as(C.c_void_p), out.size))
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, np.float32)
        _check(load_library().kamino_mlp_set_params(self.handle, p.ctypes.data_as(C.c_void_p), p.size))

    def get_normalization(self) -> np.ndarray:
        out = np.empty(2 * (self.info.d_in + self.info.d_out), np.float32)
        _check(load_library().kamino_mlp_get_normalization(self.handle, out.ctypes.data_as(C.c_void_p)))
        return out

    def set_normalization(self, v: np.ndarray):
        v = np.ascontiguousarray(v, np.float32)
        if v.size != 2 * (self.info.d_in + self.info.d_out):
            raise ValueError(f"normalisation vector must have 2 (d_in + d_out) = "
                             f"{2 * (self.info.d_in + self.info.d_out)} entries (got {v.size})")
        _check(load_library().kamino_mlp_set_normalization(self.handle, v.ctypes.data_as(C.c_void_p)))

    def layer_params(self, p: np.ndarray | None = None):
        """Split a flat parameter vector into ([W0..WL], [b0..bL]) with W_l of shape (out, in)."""
        p = self.get_params() if p is None else p
        dims = [self.info.d_in] + [self.info.d_hidden] * self.info.hidden_layers + [self.info.d_out]
        Ws, bs, o = [], [], 0
        for fin, fout in zip(dims[:-1], dims[1:]):
            Ws.append(p[o:o + fout * fin].reshape(fout, fin)); o += fout * fin
            bs.append(p[o:o + fout]); o += fout
        return Ws, bs

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.kamino_mlp_destroy(self.handle)
            self.handle = None
