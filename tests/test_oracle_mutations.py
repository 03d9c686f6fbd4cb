"""The oracle's pins catch planted mistakes.  Each case copies the oracle,
the pin tests and the input generators into a scratch directory, plants one
plausible mistake in the copy of one oracle source (a sign, an order, a
dropped factor, a transposed index), and runs the pin suite there in a child
process: it must fail.  Nothing outside the scratch copy is touched."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, original text, planted mistake) in tt_oracle.c -- each original occurs exactly once
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
    ("gradient_factor_two", "r[q] *= 2.0 * w;", "r[q] *= w;"),
    ("weights_on_residual_not_square", "loss += w * r[q] * r[q];", "loss += r[q] * r[q];"),
    ("segment_mean", "Bsc[i] += 0.5 * w[t] * y[i];", "Bsc[i] += half * w[t] * y[i];"),
    ("legendre_recurrence", "plm = ((2.0 * ll - 1.0) * x * pm1m - (ll + m - 1.0) * pmm) / (ll - m);",
     "plm = ((2.0 * ll - 1.0) * x * pm1m - (ll + m) * pmm) / (ll - m);"),
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


# the same in the numpy parts of the oracle: (name, file, original, mistake)
PY_MUTATIONS = [
    ("lbfgs_initial_scaling", "lbfgs.py", "r = gamma * q", "r = q"),
    ("lbfgs_store_every_pair", "lbfgs.py", "if sy > 1e-10 * np.linalg.norm(s) * np.linalg.norm(y):",
     "if sy > -1e300:"),
    ("lbfgs_curvature_threshold", "lbfgs.py", "if sy > 1e-10 * np.linalg.norm(s)", "if sy > 1e-12 * np.linalg.norm(s)"),
    ("lbfgs_no_descent_check", "lbfgs.py", "if gd >= 0.0:", "if gd > 1e300:"),
    ("lbfgs_restart_keeps_memory", "lbfgs.py", "self.S.clear(); self.Y.clear(); self.rho.clear()", "pass"),
    ("lbfgs_restart_unit_step", "lbfgs.py", "alpha = 1.0 / np.linalg.norm(self.g)", "alpha = 1.0"),
    ("lbfgs_armijo_c1", "lbfgs.py", "c1: float = 1e-4", "c1: float = 1e-3"),
    ("lbfgs_armijo_plain_decrease", "lbfgs.py", "if f_t <= self.f + self.c1 * alpha * gd:", "if f_t <= self.f:"),
    ("lbfgs_halving", "lbfgs.py", "alpha *= 0.5", "alpha *= 0.25"),
    ("lbfgs_max_evals", "lbfgs.py", "max_evals: int = 20", "max_evals: int = 21"),
    ("lbfgs_failed_search_moves", "lbfgs.py", "        self.total_evals += self.max_evals\n",
     "        self.total_evals += self.max_evals\n        self.x = x_t\n"),
    ("huber_quadratic_branch", "regularizers.py", "t * t / (2.0 * delta)", "t * t / delta"),
    ("nesterov_momentum", "sirt.py", "(t - 1.0) / (t + 2.0)", "t / (t + 2.0)"),
    ("relu_dropped", "convnet.py", "y = rnd(np.maximum(y, 0.0))", "y = rnd(y)"),
]
CASES = [(n, "tt_oracle.c", o, w) for n, o, w in MUTATIONS] + PY_MUTATIONS


@pytest.mark.parametrize("name,fname,old,new", CASES, ids=[m[0] for m in CASES])
def test_pins_catch_a_planted_mistake(tmp_path, name, fname, old, new):
    src_path = os.path.join(ROOT, "oracle", fname)
    src = open(src_path).read()
    assert src.count(old) == 1, name
    _scratch_copy(str(tmp_path))
    with open(os.path.join(tmp_path, "oracle", fname), "w") as fh:
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
