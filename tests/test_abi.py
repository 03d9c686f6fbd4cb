"""The C-ABI library builds, loads and exports every entry point declared in
include/tt.h; argument validation that needs no GPU rejects bad problems."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_2504_16446_gb300 import build, synth
from paper_2504_16446_gb300 import tt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return tt.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tt_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(tt.SIGNATURES), set(names) ^ set(tt.SIGNATURES)


def test_num_coeffs_and_status_strings(lib):
    for L in range(0, 14, 2):
        assert lib.tt_num_coeffs(L) == (L + 1) * (L + 2) // 2
    assert lib.tt_status_string(0) == b"TT_OK"
    assert lib.tt_status_string(5) == b"TT_LINESEARCH_FAILED"


def _create(st, **override):
    h = tt.Handle.__new__(tt.Handle)
    # build the ctypes problem exactly as Handle does, then corrupt one field
    arrays = [np.ascontiguousarray(a, dtype=np.float64) for a in (
        st.inner_angle, st.outer_angle, st.j_offset, st.k_offset, st.seg_start, st.seg_end)]
    P = tt._Problem()
    P.nx, P.ny, P.nz = st.shape
    P.nj, P.nk, P.n_proj, P.ell_max, P.n_seg = st.nj, st.nk, st.S, st.ell_max, st.C
    ptrs = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in arrays]
    P.inner_angle, P.outer_angle, P.j_offset, P.k_offset, P.seg_start, P.seg_end = ptrs
    P.two_theta, P.voxel_size, P.step_size = st.two_theta, st.a, st.b
    for name in ("p", "j", "k", "q0", "q90", "inner_axis", "outer_axis"):
        setattr(P.frame, name, (ctypes.c_double * 3)(*tt.STANDARD_FRAME[name]))
    for k, v in override.items():
        if k.startswith("frame_"):
            setattr(P.frame, k[6:], (ctypes.c_double * 3)(*v))
        else:
            setattr(P, k, v)
    out = ctypes.c_void_p()
    status = tt.load().tt_create(ctypes.byref(P), 0, None, ctypes.byref(out))
    return status, arrays


@pytest.mark.parametrize("override,expect", [
    (dict(nx=0), tt.TT_INVALID_ARG),
    (dict(nj=-1), tt.TT_INVALID_ARG),
    (dict(ell_max=3), tt.TT_INVALID_ARG),
    (dict(ell_max=14), tt.TT_UNSUPPORTED),
    (dict(n_seg=0), tt.TT_INVALID_ARG),
    (dict(n_proj=0), tt.TT_INVALID_ARG),
    (dict(voxel_size=0.0), tt.TT_INVALID_ARG),
    (dict(step_size=float("nan")), tt.TT_INVALID_ARG),
    (dict(frame_p=(0.0, 0.0, 0.0)), tt.TT_INVALID_ARG),            # degenerate (zero-length) beam axis
    (dict(frame_inner_axis=(0.0, 0.0, 0.0)), tt.TT_INVALID_ARG),   # degenerate rotation axis
    (dict(frame_j=(0.0, 0.0, 1.0)), tt.TT_INVALID_ARG),            # j parallel to p
    (dict(frame_q0=(0.0, 0.0, 1.0)), tt.TT_INVALID_ARG),           # q0 along the beam
])
def test_invalid_problems_are_rejected_without_a_gpu(lib, override, expect):
    st = synth.small_setup(seed=0)
    status, _ = _create(st, **override)
    assert status == expect
    assert len(lib.tt_last_error()) > 0


def test_nonfinite_angles_and_bad_segments_rejected(lib):
    st = synth.small_setup(seed=1)
    st.inner_angle[2] = math.inf
    assert _create(st)[0] == tt.TT_INVALID_ARG
    st = synth.small_setup(seed=1)
    st.seg_end[1] = st.seg_start[1]
    assert _create(st)[0] == tt.TT_INVALID_ARG


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.tt_project(None, None, None) == tt.TT_INVALID_ARG
    assert lib.tt_gradient_residual(None, None, None, None, None, None) == tt.TT_INVALID_ARG
    assert lib.tt_destroy(None) == tt.TT_OK
    assert lib.tt_zonal_to_sh(3, 10, None, None, None, None) == tt.TT_INVALID_ARG
