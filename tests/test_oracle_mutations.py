"""The oracle's pins catch planted mistakes.  Each case copies the oracle,
the pin tests and the input generators into a scratch directory, plants one
plausible mistake in the copy of tt_oracle.c (a sign, an order, a dropped
factor, a transposed index), and runs the pin suite there in a child
process: it must fail.  Nothing outside the scratch copy is touched."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, original text, planted mistake) -- each original occurs exactly once
MUTATIONS = [
    ("rotation_sign", "R[3 * r + q] = (r == q ? 1.0 : 0.0) + s * K[3 * r + q] + (1.0 - c) * kk;",
     "R[3 * r + q] = (r == q ? 1.0 : 0.0) - s * K[3 * r + q] + (1.0 - c) * kk;"),
    ("rotation_order", "v += Rb[3 * r + t] * Ra[3 * t + q];", "v += Ra[3 * r + t] * Rb[3 * t + q];"),
    ("step_length", "double step = P->a / fabs(d[m]);", "double step = P->a;"),
    ("offset_sign", "double tj = P->b * (j - 0.5 * (P->nj - 1) - P->j_offset[s]);",
     "double tj = P->b * (j - 0.5 * (P->nj - 1) + P->j_offset[s]);"),
    ("sh_phase", "if (m < 0) v *= sqrt(2.0) * sin(am * phi);", "if (m < 0) v *= -sqrt(2.0) * sin(am * phi);"),
    ("azimuth_axes", "double phi = atan2(q[1], q[0]);", "double phi = atan2(q[0], q[1]);"),
    ("voxel_centring", "double Xm = P->a * (p - 0.5 * (N[m] - 1));", "double Xm = P->a * (p - 0.5 * N[m]);"),
    ("half_angle", "double th = 0.5 * P->two_theta;", "double th = P->two_theta;"),
    ("voxel_strides", "return ((size_t)xyz[0] * P->ny + xyz[1]) * P->nz + xyz[2];",
     "return ((size_t)xyz[2] * P->ny + xyz[1]) * P->nx + xyz[0];"),
    ("bilinear_weight", "double w = (du ? wu : 1.0 - wu) * (dv ? wv : 1.0 - wv);",
     "double w = (du ? 1.0 - wu : wu) * (dv ? wv : 1.0 - wv);"),
]


def _scratch_copy(dst):
    def ignore(_dir, names):
        return [n for n in names if n in ("_build", "__pycache__", "csrc") or n.endswith((".so", ".o"))]
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"), ignore=ignore)
    shutil.copytree(os.path.join(ROOT, "paper_2504_16446_gb300"), os.path.join(dst, "paper_2504_16446_gb300"),
                    ignore=ignore)
    tdst = os.path.join(dst, "tests")
    os.makedirs(tdst)
    for f in os.listdir(os.path.join(ROOT, "tests")):
        if f == "conftest.py" or (f.startswith("test_oracle_") and f.endswith(".py") and f != os.path.basename(__file__)):
            shutil.copy(os.path.join(ROOT, "tests", f), tdst)
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(tdst, "golden"))


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_a_planted_mistake(tmp_path, name, old, new):
    src_path = os.path.join(ROOT, "oracle", "tt_oracle.c")
    src = open(src_path).read()
    assert src.count(old) == 1, name
    _scratch_copy(str(tmp_path))
    with open(os.path.join(tmp_path, "oracle", "tt_oracle.c"), "w") as fh:
        fh.write(src.replace(old, new))
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        "tests"], cwd=tmp_path, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"planted mistake {name!r} passed every pin:\n{r.stdout[-2000:]}"


def test_the_unmodified_copy_passes(tmp_path):
    """Control: the same scratch copy without a planted mistake passes, so the
    failures above come from the mistakes, not from the copy."""
    _scratch_copy(str(tmp_path))
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        "tests"], cwd=tmp_path, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:]
    assert " passed" in r.stdout
