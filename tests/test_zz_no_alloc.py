"""tt_basis_matrix_noalloc: the basis matrix for callers that cannot
allocate device memory (their memory is owned or pre-reserved elsewhere, or
they must not trigger the device synchronisation cudaMalloc/cudaFree can
cause).  It keeps its scratch in a fixed device array inside libtt, so it
needs no handle; its output must equal what tt_basis_matrix returns for the
same problem, call after call (every call reuses the same scratch).

This file is collected last on purpose (test_zz_*): if it fails, a run that
stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2504_16446_gb300 import build, synth, tt


def _problem(st):
    """A tt_problem for a synth.Setup, with its arrays kept alive."""
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
    return P, arrays


def _noalloc(lib, st, out):
    P, keep = _problem(st)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = lib.tt_basis_matrix_noalloc(ctypes.byref(P), ctypes.c_void_p(out.data_ptr()), stream)
    torch.cuda.current_stream().synchronize()
    del keep
    return status


@pytest.mark.gpu
def test_noalloc_basis_matrix_matches_handle_entry_point_on_consecutive_calls():
    build.build()
    lib = tt.load()
    setups = [synth.workload("ell64"),
              synth.small_setup(n=(8, 10, 6), nj=9, nk=19, ell_max=8, n_proj=13, n_seg=7, seed=3, two_theta=0.3)]
    refs = [tt.Handle(st, "f32").basis_matrix() for st in setups]
    outs = [torch.full_like(r, float("nan")) for r in refs]
    torch.cuda.synchronize()
    for call, (st, ref, out) in enumerate(zip(setups, refs, outs)):
        free_before = torch.cuda.mem_get_info()[0]
        assert _noalloc(lib, st, out) == tt.TT_OK, lib.tt_last_error()
        if call > 0:   # after the first call on this device the scratch address is cached
            assert torch.cuda.mem_get_info()[0] == free_before
        np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), atol=1e-13, rtol=0)
    # the first result is unchanged by the second call, which reused the scratch
    np.testing.assert_allclose(outs[0].cpu().numpy(), refs[0].cpu().numpy(), atol=1e-13, rtol=0)


def test_noalloc_rejects_more_projections_than_its_scratch_holds():
    build.build()
    lib = tt.load()
    st = synth.small_setup(n_proj=2049, seed=1)
    P, keep = _problem(st)
    status = lib.tt_basis_matrix_noalloc(ctypes.byref(P), ctypes.c_void_p(16), None)
    assert status == tt.TT_INVALID_ARG
    assert b"2048" in lib.tt_last_error()


@pytest.mark.gpu
def test_noalloc_basis_matrix_at_full_scratch_capacity():
    """2048 projections, 64 segments and l_max 12 fill the fixed scratch to
    its last element (a 4^3 volume and 4 x 4 pixels keep the rest small); the
    result equals the handle entry point's on two calls in a row."""
    build.build()
    lib = tt.load()
    st = synth.small_setup(n=(4, 4, 4), nj=4, nk=4, ell_max=12, n_proj=2048, n_seg=64, seed=11, two_theta=0.2)
    h = tt.Handle(st, "f32")
    ref = h.basis_matrix()
    torch.cuda.synchronize()
    h.close()
    for _ in range(2):
        out = torch.full_like(ref, float("nan"))
        assert _noalloc(lib, st, out) == tt.TT_OK, lib.tt_last_error()
        np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), atol=1e-13, rtol=0)
