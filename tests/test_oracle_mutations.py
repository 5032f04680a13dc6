"""The oracle's pins catch plausible mistakes.

Each case copies the oracle (and the tests) into a temporary directory, plants
one mistake in the copy's source (the C path code, the numpy MLP or the
whole-program tape), and runs the pins that must catch it against the copy:
they must fail.  The unmodified copy passes the same pins, so the failures come
from the planted mistakes.  Nothing here touches the oracle in the repository.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = "mcaad_oracle.c"
PINS = "tests/test_oracle_pins.py::"
MLP_FD = "tests/test_oracle_mlp.py::test_loss_grad_fd[0.7]"

# (mistake, oracle file, text in it, replacement, pins that must fail)
MUTATIONS = [
    ("GBM drift term dropped",
     SRC,
     "s1[0] = s[0] + (r - 0.5 * vol * vol) * dt + vol * sdt * z[n];",
     "s1[0] = s[0] + r * dt + vol * sdt * z[n];",
     [PINS + "test_gbm_matches_black_scholes"]),
    ("Heston correlation: wrong sign of the independent part",
     SRC,
     "double w = rho * z1 + sqrt(1.0 - rho * rho) * z2;\n            s1[0] = x + (r - 0.5 * vp) * dt + sq * z1;",
     "double w = rho * z1 - sqrt(1.0 - rho * rho) * z2;\n            s1[0] = x + (r - 0.5 * vp) * dt + sq * z1;",
     [PINS + "test_two_step_equals_full_tape_fries[heston]"]),
    ("Heston adjoint: kappa term dropped",
     SRC,
     "double w = rho * z1 + rhob * z2;\n            g[0] += vb * (th - vp) * dt;",
     "double w = rho * z1 + rhob * z2;\n            g[0] += 0.0;",
     [PINS + "test_two_step_equals_full_tape_fries[heston]"]),
    ("local vol adjoint: d sigma / dx term dropped",
     SRC,
     "xb = xb + sb * e.dsdx;",
     "xb = xb;",
     [PINS + "test_two_step_equals_full_tape_fries[lv]"]),
    ("local vol: wrong bilinear node weight",
     SRC,
     "e.wgt[1] = (1.0 - a) * b;",
     "e.wgt[1] = a * b;",
     [PINS + "test_two_step_equals_full_tape_fries[lv]"]),
    ("local vol: sigma at the step's end instead of its start",
     SRC,
     "double ut = ((double)n * pb->dt) / ht;",
     "double ut = ((double)(n + 1) * pb->dt) / ht;",
     [PINS + "test_two_step_equals_full_tape_fries[lv]"]),
    ("GBM: a bucket's end step counted in the bucket",
     SRC,
     "while (n >= pb->bucket_end[b]) ++b;",
     "while (n > pb->bucket_end[b]) ++b;",
     [PINS + "test_two_step_equals_full_tape_fries[gbm]"]),
    ("Philox: wrong key increment",
     SRC,
     "k0 += 0x9E3779B9u;",
     "k0 += 0x9E3779B7u;",
     ["tests/test_oracle_philox.py::test_philox_matches_curand_host"]),
    ("payoff discount dropped",
     SRC,
     "y[i] = disc * (S > pb->K[i] ? S - pb->K[i] : 0.0);",
     "y[i] = (S > pb->K[i] ? S - pb->K[i] : 0.0);",
     [PINS + "test_gbm_matches_black_scholes"]),
    ("Heston adjoint: xi term of the variance adjoint dropped",
     SRC,
     "if (vp > 0.0) vpb += (xb * z1 + vb * xi * w) * dt / (2.0 * sq);",
     "if (vp > 0.0) vpb += (xb * z1) * dt / (2.0 * sq);",
     [PINS + "test_two_step_equals_full_tape_fries[heston]"]),
    ("SLV adjoint: leverage drift term dropped",
     SRC,
     "double levb = xb * (-lev * vp * dt + sq * z1);",
     "double levb = xb * (sq * z1);",
     [PINS + "test_slv_two_step_equals_full_tape"]),
    ("Box-Muller: cosine and sine swapped",
     SRC,
     "return (j & 1) ? rad * sin(ORC_TWO_PI * ub) : rad * cos(ORC_TWO_PI * ub);",
     "return (j & 1) ? rad * cos(ORC_TWO_PI * ub) : rad * sin(ORC_TWO_PI * ub);",
     ["tests/test_oracle_philox.py::test_box_muller_structure"]),
    ("MLP double backward: silu'' term dropped",
     "mlp.py",
     "zbar_t[l] = pbar * g[l] * d2silu(z[l])",
     "zbar_t[l] = 0.0 * pbar",
     [MLP_FD]),
    ("MLP double backward: w5 tangent term dropped",
     "mlp.py",
     'grads["w5"] += gbar.sum(axis=0)\n',
     "\n",
     [MLP_FD]),
    ("MLP double backward: tangent weight gradient dropped",
     "mlp.py",
     'grads["W%d" % l] += _mm(pl[l].T, gbar, bf16)\n',
     "\n",
     [MLP_FD]),
    ("tape oracle: expectation adjoint not averaged over the paths",
     "tape.py",
     "D[j] = D[j] + np.mean(D[m])",
     "D[j] = D[j] + D[m]",
     ["tests/test_tape_host.py::test_oracle_tape_product_of_expectations"]),
    ("tape oracle: product partials swapped",
     "tape.py",
     "[(self.idx, o.v), (o.idx, self.v)]",
     "[(self.idx, self.v), (o.idx, o.v)]",
     [PINS + "test_two_step_equals_full_tape_fries[heston]"]),
]


TAPE = "tape.py"
MOMENTS = PINS + "test_one_step_conditional_moments"
CF = PINS + "test_heston_matches_characteristic_function_price"
CONSISTENCY = [PINS + "test_two_step_equals_full_tape_fries[heston]", PINS + "test_slv_two_step_equals_full_tape",
               PINS + "test_fd_common_random_numbers[heston]"]

# Mistakes in the model itself, made the same way in the C forward sweep, the C adjoint and the
# whole-program tape: the pins that compare the oracle with itself (two-step against the tape,
# finite differences) still pass, so only the pins of the dynamics against the mathematics can
# catch them.  (mistake, [(file, text, replacement, occurrences)], pins that must fail)
CONSISTENT_MUTATIONS = [
    ("Heston and SLV: rho and sqrt(1 - rho^2) swapped",
     [(SRC, "double w = rho * z1 + sqrt(1.0 - rho * rho) * z2;",
       "double w = sqrt(1.0 - rho * rho) * z1 + rho * z2;", 2),
      (SRC, "double w = rho * z1 + rhob * z2;", "double w = rhob * z1 + rho * z2;", 2),
      (SRC, "g[3] += vb * xi * sq * (z1 - rho / rhob * z2);",
       "g[3] += vb * xi * sq * (-rho / rhob * z1 + z2);", 2),
      (TAPE, "w = rho * z1 + rhob * z2", "w = rhob * z1 + rho * z2", 2)],
     [MOMENTS, CF]),
    ("Heston and SLV: xi v+ dt in place of xi sqrt(v+ dt)",
     [(SRC, "s1[1] = v + kappa * (th - vp) * dt + xi * sq * w;",
       "s1[1] = v + kappa * (th - vp) * dt + xi * vp * dt * w;", 2),
      (SRC, "g[2] += vb * sq * w;", "g[2] += vb * vp * dt * w;", 2),
      (SRC, "g[3] += vb * xi * sq * (z1 - rho / rhob * z2);",
       "g[3] += vb * xi * vp * dt * (z1 - rho / rhob * z2);", 2),
      (SRC, "double vpb = xb * (-0.5 * dt) + vb * (-kappa * dt);",
       "double vpb = xb * (-0.5 * dt) + vb * (-kappa * dt) + vb * xi * w * dt;", 1),
      (SRC, "if (vp > 0.0) vpb += (xb * z1 + vb * xi * w) * dt / (2.0 * sq);",
       "if (vp > 0.0) vpb += (xb * z1) * dt / (2.0 * sq);", 1),
      (SRC, "double vpb = xb * (-0.5 * lev * lev * dt) + vb * (-kappa * dt);",
       "double vpb = xb * (-0.5 * lev * lev * dt) + vb * (-kappa * dt) + vb * xi * w * dt;", 1),
      (SRC, "if (vp > 0.0) vpb += (xb * lev * z1 + vb * xi * w) * dt / (2.0 * sq);",
       "if (vp > 0.0) vpb += (xb * lev * z1) * dt / (2.0 * sq);", 1),
      (TAPE, "v = v + kappa * (thh - vp) * dt + xi * sq * w", "v = v + kappa * (thh - vp) * dt + xi * vp * dt * w", 2)],
     [MOMENTS, CF]),
]


def _copy(dst):
    """Oracle and tests copied (the copy builds its own library), the package linked."""
    skip = shutil.ignore_patterns("*.so", "*.tmp", "__pycache__", ".pytest_cache")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"), ignore=skip)
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(dst, "tests"), ignore=skip)
    os.symlink(os.path.join(ROOT, "paper_1901_04200_gb300"), os.path.join(dst, "paper_1901_04200_gb300"))
    os.symlink(os.path.join(ROOT, "include"), os.path.join(dst, "include"))


def _run_pins(cwd, nodes):
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    cmd = [sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", "-m", "not gpu"] + nodes
    return subprocess.run(cmd, cwd=cwd, env=env, capture_output=True, text=True, timeout=600)


def test_unmodified_copy_passes_the_pins(tmp_path):
    _copy(str(tmp_path))
    nodes = sorted({n for m in MUTATIONS for n in m[4]} | {n for m in CONSISTENT_MUTATIONS for n in m[2]}
                   | set(CONSISTENCY))
    res = _run_pins(str(tmp_path), nodes)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-2000:]


@pytest.mark.parametrize("mistake,fname,old,new,nodes", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, mistake, fname, old, new, nodes):
    _copy(str(tmp_path))
    path = os.path.join(str(tmp_path), "oracle", fname)
    with open(path) as f:
        src = f.read()
    assert src.count(old) == 1, "the oracle's source changed: update this mutation (%s)" % mistake
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    res = _run_pins(str(tmp_path), nodes)
    # pytest exits 1 when tests ran and some failed
    assert res.returncode == 1 and " failed" in res.stdout, (mistake, res.stdout[-2000:] + res.stderr[-2000:])


def _plant(root, edits):
    for fname, old, new, count in edits:
        path = os.path.join(root, "oracle", fname)
        with open(path) as f:
            src = f.read()
        assert src.count(old) == count, "the oracle's source changed: update this mutation (%s)" % old
        with open(path, "w") as f:
            f.write(src.replace(old, new))


@pytest.mark.slow
@pytest.mark.parametrize("mistake,edits,nodes", CONSISTENT_MUTATIONS, ids=[m[0] for m in CONSISTENT_MUTATIONS])
def test_consistent_model_mistake_fails_a_dynamics_pin(tmp_path, mistake, edits, nodes):
    _copy(str(tmp_path))
    _plant(str(tmp_path), edits)
    res = _run_pins(str(tmp_path), CONSISTENCY)
    assert res.returncode == 0, ("the mistake is not consistent", mistake, res.stdout[-2000:] + res.stderr[-2000:])
    for node in nodes:
        res = _run_pins(str(tmp_path), [node])
        assert res.returncode == 1 and " failed" in res.stdout, (mistake, node, res.stdout[-2000:] + res.stderr[-2000:])
