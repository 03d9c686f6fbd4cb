"""Thin Python binding of libtt (include/tt.h).

Argument marshalling only: every step of the gradient-residual path runs in
libtt's CUDA kernels.  PyTorch supplies device memory and the current CUDA
stream.  There is no CPU fallback: if libtt.so is missing or fails to load,
every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtt.so")

TT_OK, TT_INVALID_ARG, TT_UNSUPPORTED, TT_OUT_OF_MEMORY, TT_NONFINITE, TT_LINESEARCH_FAILED, TT_CUDA_ERROR = range(7)
TT_F32, TT_F64, TT_BF16, TT_F16 = 0, 1, 2, 3
PRECISIONS = {"f32": TT_F32, "f64": TT_F64, "bf16": TT_BF16, "f16": TT_F16}
KSLOTS = ["pack", "forward", "backcontract", "adjoint", "unpack", "reduce", "basis", "vector"]

_lock = threading.Lock()
_lib = None


class TTError(RuntimeError):
    def __init__(self, status: int, what: str, msg: str):
        super().__init__(f"{what}: status {status} ({_status_name(status)}): {msg}")
        self.status = status


def _status_name(s):
    names = ["TT_OK", "TT_INVALID_ARG", "TT_UNSUPPORTED", "TT_OUT_OF_MEMORY", "TT_NONFINITE",
             "TT_LINESEARCH_FAILED", "TT_CUDA_ERROR"]
    return names[s] if 0 <= s < len(names) else "TT_UNKNOWN"


class _Frame(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double * 3) for n in ("p", "j", "k", "q0", "q90", "inner_axis", "outer_axis")]


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("nj", ctypes.c_int), ("nk", ctypes.c_int), ("n_proj", ctypes.c_int),
        ("ell_max", ctypes.c_int), ("n_seg", ctypes.c_int),
        ("inner_angle", ctypes.POINTER(ctypes.c_double)), ("outer_angle", ctypes.POINTER(ctypes.c_double)),
        ("j_offset", ctypes.POINTER(ctypes.c_double)), ("k_offset", ctypes.POINTER(ctypes.c_double)),
        ("seg_start", ctypes.POINTER(ctypes.c_double)), ("seg_end", ctypes.POINTER(ctypes.c_double)),
        ("two_theta", ctypes.c_double), ("voxel_size", ctypes.c_double), ("step_size", ctypes.c_double),
        ("frame", _Frame),
    ]


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); the C-ABI declared in include/tt.h
SIGNATURES = {
    "tt_num_coeffs": (ctypes.c_int, [ctypes.c_int]),
    "tt_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "tt_last_error": (ctypes.c_char_p, []),
    "tt_create": (ctypes.c_int, [ctypes.POINTER(_Problem), ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "tt_destroy": (ctypes.c_int, [_P]),
    "tt_set_stream": (ctypes.c_int, [_P, _P]),
    "tt_set_forward_kernel": (ctypes.c_int, [_P, ctypes.c_int]),
    "tt_get_sizes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    "tt_basis_matrix": (ctypes.c_int, [_P, _P]),
    "tt_basis_matrix_noalloc": (ctypes.c_int, [ctypes.POINTER(_Problem), _P, _P]),
    "tt_project": (ctypes.c_int, [_P, _P, _P]),
    "tt_project_f64": (ctypes.c_int, [_P, _P, _P]),
    "tt_adjoint": (ctypes.c_int, [_P, _P, _P]),
    "tt_adjoint_f64": (ctypes.c_int, [_P, _P, _P]),
    "tt_gradient_residual": (ctypes.c_int, [_P, _P, _P, _P, _P, _D]),
    "tt_gradient_residual_f64": (ctypes.c_int, [_P, _P, _P, _P, _P, _D]),
    "tt_gradient_residual_host": (ctypes.c_int, [_P, _P, _P, _P, _P, _D]),
    "tt_l2_norm": (ctypes.c_int, [_P, _P, _P, _D]),
    "tt_l2_norm_f64": (ctypes.c_int, [_P, _P, _P, _D]),
    "tt_tv_huber": (ctypes.c_int, [_P, _P, ctypes.c_double, _P, _D]),
    "tt_tv_huber_f64": (ctypes.c_int, [_P, _P, ctypes.c_double, _P, _D]),
    "tt_lbfgs_create": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, ctypes.POINTER(_P)]),
    "tt_lbfgs_create_ray": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_double, _P, _P, _D,
                                           ctypes.POINTER(_P)]),
    "tt_lbfgs_step": (ctypes.c_int, [_P, _P, _P, _D, ctypes.POINTER(ctypes.c_int)]),
    "tt_lbfgs_get": (ctypes.c_int, [_P, _P, _P, _P, _D]),
    "tt_lbfgs_destroy": (ctypes.c_int, [_P]),
    "tt_lbfgs_checkpoint_bytes": (ctypes.c_longlong, [_P]),
    "tt_lbfgs_stats": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong), _D]),
    "tt_lbfgs_save": (ctypes.c_int, [_P, _P, _P, ctypes.c_longlong]),
    "tt_lbfgs_restore": (ctypes.c_int, [_P, _P, ctypes.c_longlong, _P, _P, ctypes.POINTER(_P)]),
    "tt_sirt_weights": (ctypes.c_int, [_P, _P, _P, _P]),
    "tt_sirt_weights_f64": (ctypes.c_int, [_P, _P, _P, _P]),
    "tt_mitra_create": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_double, ctypes.c_double, ctypes.POINTER(_P)]),
    "tt_mitra_step": (ctypes.c_int, [_P, _D]),
    "tt_mitra_get": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_int)]),
    "tt_mitra_destroy": (ctypes.c_int, [_P]),
    "tt_wsnet_num_weights": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    "tt_wsnet_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, ctypes.POINTER(_P)]),
    "tt_wsnet_destroy": (ctypes.c_int, [_P]),
    "tt_wsnet_set_stream": (ctypes.c_int, [_P, _P]),
    "tt_wsnet_forward": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, ctypes.c_double,
                                        ctypes.c_double, _P]),
    "tt_wsnet_gradient": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_double,
                                         ctypes.c_double, _P, _D]),
    "tt_wsnet_train_step": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, _D]),
    "tt_wsnet_get_weights": (ctypes.c_int, [_P, _P]),
    "tt_conv3d_bf16": (ctypes.c_int, [ctypes.c_int] * 5 + [_P, _P, ctypes.c_int, _P, _P]),
    "tt_conv3d_bf16_act": (ctypes.c_int, [ctypes.c_int] * 5 + [_P, _P, ctypes.c_int, _P, _P]),
    "tt_conv3d_wgrad_bf16": (ctypes.c_int, [ctypes.c_int] * 5 + [_P, _P, _P, _P]),
    "tt_umma_gemm_bf16": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, _P, _P]),
    "tt_zonal_to_sh": (ctypes.c_int, [ctypes.c_int, ctypes.c_longlong, _P, _P, _P, _P]),
    "tt_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "tt_profile_read": (ctypes.c_int, [_P, ctypes.c_int, _D, ctypes.POINTER(ctypes.c_longlong)]),
    "tt_profile_reset": (ctypes.c_int, [_P]),
    "tt_kernel_slot_name": (ctypes.c_char_p, [ctypes.c_int]),
    "tt_launch_count": (ctypes.c_longlong, [_P]),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libtt.so (built by paper_2504_16446_gb300.build).  Raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"libtt.so not found at {path}: build it with "
                                   "`python -m paper_2504_16446_gb300.build` (there is no CPU fallback)")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int, what: str):
    if status != TT_OK:
        raise TTError(status, what, load().tt_last_error().decode())


def num_coeffs(ell_max: int) -> int:
    return (ell_max + 1) * (ell_max + 2) // 2


def _stream_ptr(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t: torch.Tensor, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


STANDARD_FRAME = dict(
    p=(0.0, 0.0, 1.0), j=(0.0, 1.0, 0.0), k=(1.0, 0.0, 0.0),
    q0=(1.0, 0.0, 0.0), q90=(0.0, 1.0, 0.0),
    inner_axis=(0.0, 1.0, 0.0), outer_axis=(1.0, 0.0, 0.0),
)


class Handle:
    """A tt_handle for one problem (geometry + sizes) on the current CUDA device.

    ``setup`` is any object with the fields of ``synth.Setup`` (shape, nj, nk,
    ell_max, inner_angle, outer_angle, seg_start, seg_end, j_offset, k_offset,
    two_theta, a, b).  precision: "f32", "f64", or "bf16" / "f16" (float API,
    2-byte storage of the volume and of the back-contracted residual).
    """

    def __init__(self, setup, precision: str = "f32", stream=None, frame=None):
        self.lib = load()
        self.setup = setup
        self.precision = precision
        self.dtype = torch.float64 if precision == "f64" else torch.float32
        self._arrays = [np.ascontiguousarray(a, dtype=np.float64) for a in (
            setup.inner_angle, setup.outer_angle, setup.j_offset, setup.k_offset, setup.seg_start, setup.seg_end)]
        P = _Problem()
        P.nx, P.ny, P.nz = (int(v) for v in setup.shape)
        P.nj, P.nk = int(setup.nj), int(setup.nk)
        P.n_proj = int(self._arrays[0].size)
        P.ell_max = int(setup.ell_max)
        P.n_seg = int(self._arrays[4].size)
        ptrs = [a.ctypes.data_as(_D) for a in self._arrays]
        P.inner_angle, P.outer_angle, P.j_offset, P.k_offset, P.seg_start, P.seg_end = ptrs
        P.two_theta, P.voxel_size, P.step_size = float(setup.two_theta), float(setup.a), float(setup.b)
        fr = STANDARD_FRAME if frame is None else frame
        for name in ("p", "j", "k", "q0", "q90", "inner_axis", "outer_axis"):
            setattr(P.frame, name, (ctypes.c_double * 3)(*[float(x) for x in fr[name]]))
        self._prob = P
        h = _P()
        _check(self.lib.tt_create(ctypes.byref(P), PRECISIONS[precision],
                                  _stream_ptr(stream), ctypes.byref(h)), "tt_create")
        self._h = h
        self.K = num_coeffs(setup.ell_max)
        self.S, self.C = P.n_proj, P.n_seg
        self.volume_shape = (P.nx, P.ny, P.nz, self.K)
        self.data_shape = (self.S, P.nj, P.nk, self.C)

    def close(self):
        if getattr(self, "_h", None):
            self.lib.tt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _sync_stream(self):
        _check(self.lib.tt_set_stream(self._h, _stream_ptr()), "tt_set_stream")

    FORWARD_KERNELS = {"auto": 0, "l1": 1, "staged": 2}

    def set_forward_kernel(self, kind: str) -> None:
        """Forward-projection kernel for the calls that follow: "auto", "l1" (taps read
        from the L1/L2-resident volume) or "staged" (taps staged in shared memory)."""
        _check(self.lib.tt_set_forward_kernel(self._h, self.FORWARD_KERNELS[kind]), "tt_set_forward_kernel")

    @property
    def _sfx(self):
        return "_f64" if self.precision == "f64" else ""

    def basis_matrix(self) -> torch.Tensor:
        self._sync_stream()
        B = torch.empty((self.S, self.C, self.K), dtype=torch.float64, device="cuda")
        _check(self.lib.tt_basis_matrix(self._h, ctypes.c_void_p(B.data_ptr())), "tt_basis_matrix")
        return B

    def project(self, c: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        self._sync_stream()
        out = torch.empty(self.data_shape, dtype=self.dtype, device=c.device) if out is None else out
        fn = getattr(self.lib, "tt_project" + self._sfx)
        _check(fn(self._h, _dptr(c, self.dtype, self.volume_shape, "c"),
                  _dptr(out, self.dtype, self.data_shape, "I")), "tt_project")
        return out

    def adjoint(self, R: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        self._sync_stream()
        out = torch.empty(self.volume_shape, dtype=self.dtype, device=R.device) if out is None else out
        fn = getattr(self.lib, "tt_adjoint" + self._sfx)
        _check(fn(self._h, _dptr(R, self.dtype, self.data_shape, "R"),
                  _dptr(out, self.dtype, self.volume_shape, "g")), "tt_adjoint")
        return out

    def gradient_residual(self, c, I, W=None, want_grad=True, out=None, check=True):
        """(loss, grad): loss = sum W (A c - I)^2, grad = 2 A^T (W (A c - I)).
        c = None means c = 0 (the back-projection of the data, without a
        forward projection)."""
        self._sync_stream()
        g = None
        if want_grad:
            g = torch.empty(self.volume_shape, dtype=self.dtype, device=I.device) if out is None else out
        loss = ctypes.c_double(0.0)
        fn = getattr(self.lib, "tt_gradient_residual" + self._sfx)
        st = fn(self._h, None if c is None else _dptr(c, self.dtype, self.volume_shape, "c"),
                _dptr(I, self.dtype, self.data_shape, "I"),
                None if W is None else _dptr(W, self.dtype, self.data_shape, "W"),
                None if g is None else _dptr(g, self.dtype, self.volume_shape, "g"),
                ctypes.byref(loss))
        if check:
            _check(st, "tt_gradient_residual")
        return loss.value, g

    def gradient_residual_host(self, c: np.ndarray, I: np.ndarray, W=None, g_out=None):
        """End-to-end call on HOST arrays (float32); returns (loss, g)."""
        self._sync_stream()
        if self.precision == "f64":
            raise TypeError("the host entry point takes float arrays")
        g = np.empty(self.volume_shape, np.float32) if g_out is None else g_out
        checks = [("c", c, self.volume_shape), ("I", I, self.data_shape), ("g_out", g, self.volume_shape)]
        if W is not None:
            checks.append(("W", W, self.data_shape))
        for name, a, shp in checks:
            if a.dtype != np.float32 or a.shape != shp or not a.flags["C_CONTIGUOUS"]:
                raise ValueError(f"{name} must be C-contiguous float32 of shape {shp}")
        if not g.flags["WRITEABLE"]:
            raise ValueError("g_out must be writeable")
        loss = ctypes.c_double(0.0)
        _check(self.lib.tt_gradient_residual_host(
            self._h, c.ctypes.data_as(_P), I.ctypes.data_as(_P),
            None if W is None else W.ctypes.data_as(_P), g.ctypes.data_as(_P), ctypes.byref(loss)),
            "tt_gradient_residual_host")
        return loss.value, g

    def l2_norm(self, c, want_grad=True):
        """(sum c^2, 2c)."""
        self._sync_stream()
        g = torch.empty(self.volume_shape, dtype=self.dtype, device=c.device) if want_grad else None
        v = ctypes.c_double(0.0)
        fn = getattr(self.lib, "tt_l2_norm" + self._sfx)
        _check(fn(self._h, _dptr(c, self.dtype, self.volume_shape, "c"),
                  None if g is None else ctypes.c_void_p(g.data_ptr()), ctypes.byref(v)), "tt_l2_norm")
        return v.value, g

    def tv_huber(self, c, delta, want_grad=True):
        """(Huber total variation, gradient); see tt_tv_huber in include/tt.h."""
        self._sync_stream()
        g = torch.empty(self.volume_shape, dtype=self.dtype, device=c.device) if want_grad else None
        v = ctypes.c_double(0.0)
        fn = getattr(self.lib, "tt_tv_huber" + self._sfx)
        _check(fn(self._h, _dptr(c, self.dtype, self.volume_shape, "c"), float(delta),
                  None if g is None else ctypes.c_void_p(g.data_ptr()), ctypes.byref(v)), "tt_tv_huber")
        return v.value, g

    def sirt_weights(self, W=None):
        """(R, D): SIRT data weights [S, nj, nk, C] and preconditioner [nx, ny, nz, K]
        (inverse row / column sums of |A|; see tt_sirt_weights in include/tt.h)."""
        self._sync_stream()
        R = torch.empty(self.data_shape, dtype=self.dtype, device="cuda")
        D = torch.empty(self.volume_shape, dtype=self.dtype, device="cuda")
        fn = getattr(self.lib, "tt_sirt_weights" + self._sfx)
        _check(fn(self._h, None if W is None else _dptr(W, self.dtype, self.data_shape, "W"),
                  ctypes.c_void_p(R.data_ptr()), ctypes.c_void_p(D.data_ptr())), "tt_sirt_weights")
        return R, D

    # ------------------------------------------------------------ profiling
    def profile(self, enable: bool = True):
        _check(self.lib.tt_profile_enable(self._h, int(enable)), "tt_profile_enable")

    def profile_reset(self):
        _check(self.lib.tt_profile_reset(self._h), "tt_profile_reset")

    def profile_read(self) -> dict:
        out = {}
        for slot, name in enumerate(KSLOTS):
            ms = ctypes.c_double(0.0)
            n = ctypes.c_longlong(0)
            _check(self.lib.tt_profile_read(self._h, slot, ctypes.byref(ms), ctypes.byref(n)), "tt_profile_read")
            out[name] = (ms.value, n.value)
        return out

    def launch_count(self) -> int:
        return int(self.lib.tt_launch_count(self._h))


class LBFGS:
    """Device-resident L-BFGS on a Handle (tt_lbfgs_*)."""

    def __init__(self, handle: Handle, c0: torch.Tensor | None, I: torch.Tensor, W: torch.Tensor | None = None,
                 m: int = 10, log: bool = True):
        """c0 = None starts at zero (its evaluation skips the forward projection)."""
        self.h = handle
        handle._sync_stream()
        self._keep = (c0, I, W)
        st = _P()
        dt, vs, ds = handle.dtype, handle.volume_shape, handle.data_shape
        _check(handle.lib.tt_lbfgs_create(handle._h, int(m), None if c0 is None else _dptr(c0, dt, vs, "c0"),
                                          _dptr(I, dt, ds, "I"),
                                          None if W is None else _dptr(W, dt, ds, "W"), ctypes.byref(st)),
               "tt_lbfgs_create")
        self._st = st
        self.loss = self.get()[2]
        self._start_log(I, W, log)

    def _start_log(self, I, W, log):
        """Per-iteration log (log=True): loss, gradient evaluations, line-search
        step and the relative data residual sqrt(L / sum W I^2)."""
        self.history = []
        self._data_norm2 = None
        if log:
            Id = I.double()
            self._data_norm2 = float(torch.sum(Id * Id if W is None else W.double() * Id * Id))

    def stats(self) -> dict:
        """Accepted iterations, gradient evaluations (creation's included) and
        the line-search step of the last iteration (tt_lbfgs_stats)."""
        it, ev, a = ctypes.c_longlong(0), ctypes.c_longlong(0), ctypes.c_double(0.0)
        _check(self.h.lib.tt_lbfgs_stats(self._st, ctypes.byref(it), ctypes.byref(ev), ctypes.byref(a)),
               "tt_lbfgs_stats")
        return {"iterations": it.value, "evaluations": ev.value, "last_step": a.value}

    def save(self) -> np.ndarray:
        """Checkpoint of the state (iterate, gradient, stored pairs, Gram
        matrix, counters, loss) as a host byte array (tt_lbfgs_save)."""
        self.h._sync_stream()
        n = int(self.h.lib.tt_lbfgs_checkpoint_bytes(self._st))
        buf = np.empty(n, dtype=np.uint8)
        _check(self.h.lib.tt_lbfgs_save(self.h._h, self._st, buf.ctypes.data_as(_P), n), "tt_lbfgs_save")
        return buf

    @classmethod
    def restore(cls, handle: "Handle", buf: np.ndarray, I: torch.Tensor, W: torch.Tensor | None = None,
                log: bool = True) -> "LBFGS":
        """A state from a checkpoint of save() (tt_lbfgs_restore); I and W as
        for the constructor."""
        handle._sync_stream()
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        dt, ds = handle.dtype, handle.data_shape
        st = _P()
        _check(handle.lib.tt_lbfgs_restore(handle._h, buf.ctypes.data_as(_P), int(buf.size), _dptr(I, dt, ds, "I"),
                                           None if W is None else _dptr(W, dt, ds, "W"), ctypes.byref(st)),
               "tt_lbfgs_restore")
        self = cls.__new__(cls)
        self.h = handle
        self._keep = (None, I, W)
        self._st = st
        self.loss = self.get()[2]
        self._start_log(I, W, log)
        return self

    @classmethod
    def from_ray(cls, handle: "Handle", u: torch.Tensor, g0: torch.Tensor, loss0: float, I: torch.Tensor,
                 W: torch.Tensor | None = None, m: int = 10, log: bool = True) -> "LBFGS":
        """A state started at the loss minimiser along the ray {a u}, given the
        gradient g0 and loss loss0 at zero (tt_lbfgs_create_ray: one gradient
        evaluation, at u).  The chosen a is in .alpha (0: started at zero)."""
        handle._sync_stream()
        dt, vs, ds = handle.dtype, handle.volume_shape, handle.data_shape
        st = _P()
        alpha = ctypes.c_double(0.0)
        _check(handle.lib.tt_lbfgs_create_ray(handle._h, int(m), _dptr(u, dt, vs, "u"), _dptr(g0, dt, vs, "g0"),
                                              float(loss0), _dptr(I, dt, ds, "I"),
                                              None if W is None else _dptr(W, dt, ds, "W"), ctypes.byref(alpha),
                                              ctypes.byref(st)), "tt_lbfgs_create_ray")
        self = cls.__new__(cls)
        self.h = handle
        self._keep = (u, I, W)
        self._st = st
        self.alpha = alpha.value
        self.loss = self.get()[2]
        self._start_log(I, W, log)
        return self

    def step(self):
        """One iteration -> (loss, n_evals, status); raises on errors other than line-search failure."""
        self.h._sync_stream()
        loss = ctypes.c_double(0.0)
        ne = ctypes.c_int(0)
        st = self.h.lib.tt_lbfgs_step(self.h._h, self._st, None, ctypes.byref(loss), ctypes.byref(ne))
        if st not in (TT_OK, TT_LINESEARCH_FAILED):
            _check(st, "tt_lbfgs_step")
        self.loss = loss.value
        if self._data_norm2 is not None:
            self.history.append({"loss": loss.value, "evals": ne.value, "step": self.stats()["last_step"],
                                 "relative_residual": (loss.value / self._data_norm2) ** 0.5
                                 if self._data_norm2 > 0 else float("nan"), "status": st})
        return loss.value, ne.value, st

    def get(self):
        self.h._sync_stream()
        x = torch.empty(self.h.volume_shape, dtype=self.h.dtype, device="cuda")
        g = torch.empty_like(x)
        loss = ctypes.c_double(0.0)
        _check(self.h.lib.tt_lbfgs_get(self.h._h, self._st, ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(g.data_ptr()), ctypes.byref(loss)), "tt_lbfgs_get")
        return x, g, loss.value

    def close(self):
        if getattr(self, "_st", None):
            self.h.lib.tt_lbfgs_destroy(self._st)
            self._st = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MITRA:
    """SIRT-preconditioned gradient descent with Nesterov momentum (tt_mitra_*)."""

    def __init__(self, handle: Handle, c0: torch.Tensor, I: torch.Tensor, W: torch.Tensor | None = None,
                 eta: float = 1.0, momentum: float = -1.0):
        self.h = handle
        handle._sync_stream()
        self._keep = I
        st = _P()
        dt, vs, ds = handle.dtype, handle.volume_shape, handle.data_shape
        _check(handle.lib.tt_mitra_create(handle._h, _dptr(c0, dt, vs, "c0"), _dptr(I, dt, ds, "I"),
                                          None if W is None else _dptr(W, dt, ds, "W"), float(eta),
                                          float(momentum), ctypes.byref(st)), "tt_mitra_create")
        self._st = st

    def step(self, want_loss: bool = True):
        """One iteration; returns L_R at the extrapolated point (None if not wanted:
        then nothing synchronises with the host)."""
        self.h._sync_stream()
        loss = ctypes.c_double(0.0)
        _check(self.h.lib.tt_mitra_step(self._st, ctypes.byref(loss) if want_loss else None), "tt_mitra_step")
        return loss.value if want_loss else None

    def get(self):
        """(x, R, D, iterations)."""
        self.h._sync_stream()
        x = torch.empty(self.h.volume_shape, dtype=self.h.dtype, device="cuda")
        R = torch.empty(self.h.data_shape, dtype=self.h.dtype, device="cuda")
        D = torch.empty_like(x)
        it = ctypes.c_int(0)
        _check(self.h.lib.tt_mitra_get(self._st, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(R.data_ptr()),
                                       ctypes.c_void_p(D.data_ptr()), ctypes.byref(it)), "tt_mitra_get")
        return x, R, D, it.value

    def close(self):
        if getattr(self, "_st", None):
            self.h.lib.tt_mitra_destroy(self._st)
            self._st = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def umma_gemm_bf16(A: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
    """C = A B^T for A [128][K], B [N][K] bfloat16 on the tcgen05 tensor cores
    (one tile); raises if the kernel's wait for the tensor cores gave up."""
    lib = load()
    N, K = B.shape
    A = A.contiguous()
    B = B.contiguous()
    C = torch.empty((128, N), dtype=torch.float32, device=A.device)
    status = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(lib.tt_umma_gemm_bf16(_dptr(A, torch.bfloat16, (128, K), "A"), _dptr(B, torch.bfloat16, (N, K), "B"),
                                 ctypes.c_void_p(C.data_ptr()), int(N), int(K), ctypes.c_void_p(status.data_ptr()),
                                 _stream_ptr()), "tt_umma_gemm_bf16")
    if int(status.item()) != 0:
        raise TTError(TT_CUDA_ERROR, "tt_umma_gemm_bf16", "tensor-core wait gave up")
    return C


def zonal_to_sh(ell_max: int, dirs: torch.Tensor, amps: torch.Tensor) -> torch.Tensor:
    """SH coefficients [n, K] (FP32, on the GPU) of zonal functions rotated to dirs."""
    lib = load()
    n = dirs.shape[0]
    d = dirs.reshape(n, 3).contiguous()
    a = amps.reshape(n, ell_max // 2 + 1).contiguous()
    c = torch.empty((n, num_coeffs(ell_max)), dtype=torch.float32, device=d.device)
    _check(lib.tt_zonal_to_sh(int(ell_max), int(n), _dptr(d, torch.float32, (n, 3), "dirs"),
                              _dptr(a, torch.float32, (n, ell_max // 2 + 1), "amps"),
                              ctypes.c_void_p(c.data_ptr()), _stream_ptr()), "tt_zonal_to_sh")
    return c


class WarmStartNet:
    """The learned warm start (tt_wsnet_*): 4 layers of 3x3x3 convolutions,
    k_in -> 32 -> 32 -> 32 -> k_out, ReLU between layers, no biases."""

    HIDDEN = 32

    def __init__(self, k_in: int, k_out: int, weights: np.ndarray | None = None, seed: int = 0):
        self.lib = load()
        self.k_in, self.k_out = int(k_in), int(k_out)
        n = self.lib.tt_wsnet_num_weights(self.k_in, self.k_out)
        if n <= 0:
            raise ValueError("k_in, k_out must be in [1, 16]")
        if weights is None:
            weights = self.he_init(self.k_in, self.k_out, seed)
        w = np.ascontiguousarray(weights, dtype=np.float32).ravel()
        if w.size != n:
            raise ValueError(f"expected {n} weights, got {w.size}")
        h = _P()
        _check(self.lib.tt_wsnet_create(self.k_in, self.k_out, w.ctypes.data_as(_P), _stream_ptr(),
                                        ctypes.byref(h)), "tt_wsnet_create")
        self._h = h

    @staticmethod
    def layer_shapes(k_in, k_out):
        H = WarmStartNet.HIDDEN
        return [(3, 3, 3, H, k_in), (3, 3, 3, H, H), (3, 3, 3, H, H), (3, 3, 3, k_out, H)]

    @staticmethod
    def he_init(k_in, k_out, seed):
        """He-normal initial weights (seeded), flattened layer by layer."""
        rng = np.random.default_rng(seed)
        parts = [rng.normal(0.0, np.sqrt(2.0 / (27 * shp[4])), shp).astype(np.float32)
                 for shp in WarmStartNet.layer_shapes(k_in, k_out)]
        return np.concatenate([p.ravel() for p in parts])

    def _sync(self):
        _check(self.lib.tt_wsnet_set_stream(self._h, _stream_ptr()), "tt_wsnet_set_stream")

    def forward(self, x: torch.Tensor, in_scale: float, out_scale: float | None = None) -> torch.Tensor:
        """out_scale * net(x / in_scale) (out_scale defaults to in_scale)."""
        self._sync()
        nx, ny, nz, _ = x.shape
        y = torch.empty((nx, ny, nz, self.k_out), dtype=torch.float32, device=x.device)
        _check(self.lib.tt_wsnet_forward(self._h, nx, ny, nz, _dptr(x, torch.float32, (nx, ny, nz, self.k_in), "x"),
                                         float(in_scale), float(in_scale if out_scale is None else out_scale),
                                         ctypes.c_void_p(y.data_ptr())), "tt_wsnet_forward")
        return y

    def gradient(self, x, target, in_scale, out_scale=None):
        self._sync()
        nx, ny, nz, _ = x.shape
        g = np.empty(self.lib.tt_wsnet_num_weights(self.k_in, self.k_out), np.float32)
        loss = ctypes.c_double(0.0)
        _check(self.lib.tt_wsnet_gradient(self._h, nx, ny, nz, _dptr(x, torch.float32, (nx, ny, nz, self.k_in), "x"),
                                          _dptr(target, torch.float32, (nx, ny, nz, self.k_out), "target"),
                                          float(in_scale), float(in_scale if out_scale is None else out_scale),
                                          g.ctypes.data_as(_P), ctypes.byref(loss)), "tt_wsnet_gradient")
        return loss.value, g

    def train_step(self, x, target, in_scale, lr, out_scale=None):
        self._sync()
        nx, ny, nz, _ = x.shape
        loss = ctypes.c_double(0.0)
        _check(self.lib.tt_wsnet_train_step(self._h, nx, ny, nz, _dptr(x, torch.float32, (nx, ny, nz, self.k_in), "x"),
                                            _dptr(target, torch.float32, (nx, ny, nz, self.k_out), "target"),
                                            float(in_scale), float(in_scale if out_scale is None else out_scale),
                                            float(lr), ctypes.byref(loss)), "tt_wsnet_train_step")
        return loss.value

    def weights(self) -> np.ndarray:
        w = np.empty(self.lib.tt_wsnet_num_weights(self.k_in, self.k_out), np.float32)
        _check(self.lib.tt_wsnet_get_weights(self._h, w.ctypes.data_as(_P)), "tt_wsnet_get_weights")
        return w

    def close(self):
        if getattr(self, "_h", None):
            self.lib.tt_wsnet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
