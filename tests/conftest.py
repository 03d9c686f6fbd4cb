import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def oracle_geometry(setup):
    """oracle.Geometry from a synth.Setup."""
    import oracle
    return oracle.Geometry(setup.shape, setup.nj, setup.nk, setup.ell_max,
                           setup.inner_angle, setup.outer_angle,
                           setup.seg_start, setup.seg_end,
                           j_offset=setup.j_offset, k_offset=setup.k_offset,
                           two_theta=setup.two_theta, a=setup.a, b=setup.b)
