"""FP64 CPU oracle for the tensor-tomography gradient-residual path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library in
``paper_2504_16446_gb300/csrc`` and never calls it.

The arithmetic lives in ``tt_oracle.c`` (plain C, double precision,
single-threaded) and in ``lbfgs.py`` (numpy).  This module compiles the C file
with gcc on first use and wraps it with ctypes.  Citations are to the sections
and equations of Mumott (arXiv 2504.16446).

Parity pins: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, textbook special cases, brute force or identities; none
is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tt_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile tt_oracle.c into oracle/_build/liboracle.so (gcc, -O2)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Problem(ctypes.Structure):
    """Mirror of ``or_problem`` in tt_oracle.c."""
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("nj", ctypes.c_int), ("nk", ctypes.c_int),
        ("n_proj", ctypes.c_int), ("ell_max", ctypes.c_int), ("n_seg", ctypes.c_int),
        ("inner_angle", ctypes.POINTER(ctypes.c_double)),
        ("outer_angle", ctypes.POINTER(ctypes.c_double)),
        ("j_offset", ctypes.POINTER(ctypes.c_double)),
        ("k_offset", ctypes.POINTER(ctypes.c_double)),
        ("seg_start", ctypes.POINTER(ctypes.c_double)),
        ("seg_end", ctypes.POINTER(ctypes.c_double)),
        ("two_theta", ctypes.c_double), ("a", ctypes.c_double), ("b", ctypes.c_double),
        ("p", ctypes.c_double * 3), ("j", ctypes.c_double * 3), ("k", ctypes.c_double * 3),
        ("q0", ctypes.c_double * 3), ("q90", ctypes.c_double * 3),
        ("alpha_axis", ctypes.c_double * 3), ("beta_axis", ctypes.c_double * 3),
    ]


_DP = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(Problem)
            lib.or_num_coeffs.argtypes = [ctypes.c_int]
            lib.or_num_coeffs.restype = ctypes.c_int
            lib.or_sh_eval.argtypes = [ctypes.c_int, ctypes.c_int, _DP, _DP]
            lib.or_gauss_legendre.argtypes = [ctypes.c_int, _DP, _DP]
            lib.or_rotation.argtypes = [_DP, ctypes.c_double, _DP]
            lib.or_projection_rotation.argtypes = [P, ctypes.c_int, _DP]
            lib.or_projection_frame.argtypes = [P, ctypes.c_int, _DP]
            lib.or_main_axis.argtypes = [_DP]
            lib.or_main_axis.restype = ctypes.c_int
            lib.or_basis_matrix.argtypes = [P, ctypes.c_int, _DP]
            lib.or_john_forward.argtypes = [P, ctypes.c_int, _DP, _DP]
            lib.or_john_adjoint.argtypes = [P, ctypes.c_int, _DP, _DP]
            lib.or_forward.argtypes = [P, _DP, _DP, _DP]
            lib.or_adjoint.argtypes = [P, _DP, _DP, _DP]
            lib.or_gradient_residual.argtypes = [P, _DP, _DP, _DP, _DP, _DP]
            lib.or_gradient_residual.restype = ctypes.c_double
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


def num_coeffs(ell_max: int) -> int:
    return (ell_max + 1) * (ell_max + 2) // 2


# Standard geometry, Table "geometry_vectors": p=+z, j=+y, k=+x, q0=+x,
# q90=+y, inner axis alpha=+y, outer axis beta=+x.
STANDARD_FRAME = dict(
    p=(0.0, 0.0, 1.0), j=(0.0, 1.0, 0.0), k=(1.0, 0.0, 0.0),
    q0=(1.0, 0.0, 0.0), q90=(0.0, 1.0, 0.0),
    alpha_axis=(0.0, 1.0, 0.0), beta_axis=(1.0, 0.0, 0.0),
)


class Geometry:
    """Holds the problem description and keeps its arrays alive."""

    def __init__(self, shape, nj, nk, ell_max, inner_angle, outer_angle,
                 seg_start, seg_end, j_offset=None, k_offset=None,
                 two_theta=0.0, a=1.0, b=1.0, frame=None):
        self.shape = tuple(int(v) for v in shape)
        self.nj, self.nk = int(nj), int(nk)
        self.ell_max = int(ell_max)
        self.K = num_coeffs(self.ell_max)
        self.inner_angle = np.ascontiguousarray(inner_angle, dtype=np.float64)
        self.outer_angle = np.ascontiguousarray(outer_angle, dtype=np.float64)
        S = self.inner_angle.size
        self.S = S
        self.j_offset = np.zeros(S) if j_offset is None else np.ascontiguousarray(j_offset, dtype=np.float64)
        self.k_offset = np.zeros(S) if k_offset is None else np.ascontiguousarray(k_offset, dtype=np.float64)
        self.seg_start = np.ascontiguousarray(seg_start, dtype=np.float64)
        self.seg_end = np.ascontiguousarray(seg_end, dtype=np.float64)
        self.C = self.seg_start.size
        self.two_theta, self.a, self.b = float(two_theta), float(a), float(b)
        self.frame = dict(STANDARD_FRAME if frame is None else frame)
        P = Problem()
        P.nx, P.ny, P.nz = self.shape
        P.nj, P.nk, P.n_proj, P.ell_max, P.n_seg = self.nj, self.nk, S, self.ell_max, self.C
        P.inner_angle = _ptr(self.inner_angle)
        P.outer_angle = _ptr(self.outer_angle)
        P.j_offset = _ptr(self.j_offset)
        P.k_offset = _ptr(self.k_offset)
        P.seg_start = _ptr(self.seg_start)
        P.seg_end = _ptr(self.seg_end)
        P.two_theta, P.a, P.b = self.two_theta, self.a, self.b
        for name in ("p", "j", "k", "q0", "q90", "alpha_axis", "beta_axis"):
            setattr(P, name, (ctypes.c_double * 3)(*[float(x) for x in self.frame[name]]))
        self._P = P

    @property
    def n_vox(self) -> int:
        return self.shape[0] * self.shape[1] * self.shape[2]

    @property
    def data_shape(self):
        return (self.S, self.nj, self.nk, self.C)

    @property
    def volume_shape(self):
        return (*self.shape, self.K)


# ---------------------------------------------------------------- wrappers


def sh_eval(ell_max: int, dirs) -> np.ndarray:
    """Real even-l SH Y_i at unit directions dirs[n,3] -> [n, K]."""
    lib = _load()
    d = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((d.shape[0], num_coeffs(ell_max)))
    lib.or_sh_eval(ell_max, d.shape[0], _ptr(d), _ptr(out))
    return out


def gauss_legendre(n: int):
    lib = _load()
    x, w = np.zeros(n), np.zeros(n)
    lib.or_gauss_legendre(n, _ptr(x), _ptr(w))
    return x, w


def rotation(axis, angle) -> np.ndarray:
    lib = _load()
    ax = np.ascontiguousarray(axis, dtype=np.float64)
    R = np.zeros(9)
    lib.or_rotation(_ptr(ax), float(angle), _ptr(R))
    return R.reshape(3, 3)


def projection_frame(g: Geometry, s: int) -> dict:
    lib = _load()
    F = np.zeros(15)
    lib.or_projection_frame(ctypes.byref(g._P), s, _ptr(F))
    F = F.reshape(5, 3)
    return dict(p=F[0], j=F[1], k=F[2], q0=F[3], q90=F[4])


def main_axis(d) -> int:
    lib = _load()
    dd = np.ascontiguousarray(d, dtype=np.float64)
    return lib.or_main_axis(_ptr(dd))


def basis_matrix(g: Geometry, n_nodes: int = 32) -> np.ndarray:
    """B[s, c, i], Eq. (projection_matrix)."""
    lib = _load()
    B = np.zeros((g.S, g.C, g.K))
    lib.or_basis_matrix(ctypes.byref(g._P), n_nodes, _ptr(B))
    return B


def john_forward(g: Geometry, c: np.ndarray) -> np.ndarray:
    """Per-channel John transform: c[nx,ny,nz,K'] -> Y[S,nj,nk,K']."""
    lib = _load()
    c = np.ascontiguousarray(c, dtype=np.float64)
    Kc = c.shape[-1]
    assert c.shape[:3] == g.shape
    Y = np.zeros((g.S, g.nj, g.nk, Kc))
    lib.or_john_forward(ctypes.byref(g._P), Kc, _ptr(c), _ptr(Y))
    return Y


def john_adjoint(g: Geometry, Y: np.ndarray) -> np.ndarray:
    lib = _load()
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    Kc = Y.shape[-1]
    assert Y.shape[:3] == (g.S, g.nj, g.nk)
    c = np.zeros((*g.shape, Kc))
    lib.or_john_adjoint(ctypes.byref(g._P), Kc, _ptr(Y), _ptr(c))
    return c


def forward(g: Geometry, c: np.ndarray, B: np.ndarray | None = None) -> np.ndarray:
    """I = A c, Eq. (forward_model): c[nx,ny,nz,K] -> I[S,nj,nk,C]."""
    lib = _load()
    B = basis_matrix(g) if B is None else np.ascontiguousarray(B, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    assert c.shape == g.volume_shape
    I = np.zeros(g.data_shape)
    lib.or_forward(ctypes.byref(g._P), _ptr(B), _ptr(c), _ptr(I))
    return I


def adjoint(g: Geometry, R: np.ndarray, B: np.ndarray | None = None) -> np.ndarray:
    """g = A^T R: R[S,nj,nk,C] -> [nx,ny,nz,K]."""
    lib = _load()
    B = basis_matrix(g) if B is None else np.ascontiguousarray(B, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    assert R.shape == g.data_shape
    out = np.zeros(g.volume_shape)
    lib.or_adjoint(ctypes.byref(g._P), _ptr(B), _ptr(R), _ptr(out))
    return out


def gradient_residual(g: Geometry, c, I, W=None, B=None, want_grad=True):
    """(loss, grad): loss = sum W (A c - I)^2, grad = 2 A^T (W (A c - I))."""
    lib = _load()
    B = basis_matrix(g) if B is None else np.ascontiguousarray(B, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    I = np.ascontiguousarray(I, dtype=np.float64)
    assert c.shape == g.volume_shape and I.shape == g.data_shape
    Wp = None
    if W is not None:
        W = np.ascontiguousarray(W, dtype=np.float64)
        assert W.shape == g.data_shape
        Wp = _ptr(W)
    grad = np.zeros(g.volume_shape) if want_grad else None
    loss = lib.or_gradient_residual(ctypes.byref(g._P), _ptr(B), _ptr(c), _ptr(I), Wp,
                                    _ptr(grad) if want_grad else None)
    return loss, grad


def zonal_to_sh(ell_max: int, dirs, amps) -> np.ndarray:
    """SH coefficients of a zonal function rotated to axis n.

    For f(q) = sum_l a_l sqrt((2l+1)/(4 pi)) P_l(q . n) the addition theorem
    gives c_lm = a_l sqrt(4 pi/(2l+1)) Y_lm(n).  dirs[n,3], amps[n, L/2+1]
    (a_0, a_2, ...) -> c[n, K].
    """
    Y = sh_eval(ell_max, dirs)
    amps = np.asarray(amps, dtype=np.float64).reshape(Y.shape[0], -1)
    c = np.zeros_like(Y)
    i = 0
    for li, l in enumerate(range(0, ell_max + 1, 2)):
        scale = np.sqrt(4.0 * np.pi / (2 * l + 1))
        for _m in range(-l, l + 1):
            c[:, i] = amps[:, li] * scale * Y[:, i]
            i += 1
    return c


from .lbfgs import LBFGS  # noqa: E402  (numpy two-loop L-BFGS on top of the above)
from .sirt import MITRA, sirt_weights  # noqa: E402  (SIRT-preconditioned solver)
