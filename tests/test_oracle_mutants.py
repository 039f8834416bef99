"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a dropped
term, a wrong sign, a transposed operand, a wrong index, a wrong constant,
a wrong operand order) and runs the pin suites (test_oracle_pins.py,
test_oracle_srht.py) against that copy in a subprocess: at least one pin
must fail.  A control run of the unchanged copy must pass, and the copy must
be the module the subprocess imports.  CPU only; nothing here touches the
product library.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = [os.path.join(ROOT, "tests", "test_oracle_pins.py"),
        os.path.join(ROOT, "tests", "test_oracle_srht.py")]

# (name, original text, planted mistake); each original occurs exactly once
MUTANTS = [
    ("gram_drops_last_row",
     "for (int64_t i = 0; i < m; ++i)\n                acc += xk[i] * xj[i];",
     "for (int64_t i = 0; i + 1 < m; ++i)\n                acc += xk[i] * xj[i];"),
    ("cholesky_radicand_sign",
     "d -= IDX(R, ldr, k, j) * IDX(R, ldr, k, j);",
     "d += IDX(R, ldr, k, j) * IDX(R, ldr, k, j);"),
    ("cholesky_offdiagonal_index",
     "acc -= IDX(R, ldr, k, i) * IDX(R, ldr, k, j);",
     "acc -= IDX(R, ldr, i, k) * IDX(R, ldr, k, j);"),
    ("trsm_transposed_factor",
     "acc -= row[k] * IDX(R, ldr, k, j);",
     "acc -= row[k] * IDX(R, ldr, j, k);"),
    ("trmm_drops_last_term",
     "for (int64_t k = i; k <= j; ++k)\n                    acc += IDX(A, lda, i, k) * IDX(B, ldb, k, j);",
     "for (int64_t k = i; k < j; ++k)\n                    acc += IDX(A, lda, i, k) * IDX(B, ldb, k, j);"),
    ("gepp_ties_to_the_last_row",
     "            if (v > best) {\n                best = v;\n                p = i;",
     "            if (v >= best) {\n                best = v;\n                p = i;"),
    ("householder_beta_sign",
     "double beta = alpha >= 0.0 ? -norm : norm;",
     "double beta = alpha >= 0.0 ? norm : -norm;"),
    ("sign_normalisation_dropped",
     "        if (IDX(R, ldr, i, i) < 0.0)\n            for (int64_t j = i; j < n; ++j)",
     "        if (IDX(R, ldr, i, i) < -HUGE_VAL)\n            for (int64_t j = i; j < n; ++j)"),
    ("final_product_order",
     "orc_trmm_upper(n, R4, n, R3, n, R, ldr);",
     "orc_trmm_upper(n, R3, n, R4, n, R, ldr);"),
    ("r3_product_order",
     "orc_trmm_upper(n, R2, n, R1, n, R3, n);",
     "orc_trmm_upper(n, R1, n, R2, n, R3, n);"),
    ("sketch_skips_first_row",
     "        for (int64_t i = 0; i < m; ++i) {\n            const double x = xj[i];",
     "        for (int64_t i = 1; i < m; ++i) {\n            const double x = xj[i];"),
    ("rcluppr_sketches_x_not_m",
     "orc_apply_sketch(kind, s, m, n, zeta, S, lds, rows, signs, M, m, Ms, s);",
     "orc_apply_sketch(kind, s, m, n, zeta, S, lds, rows, signs, X, ldx, Ms, s);"),
    ("philox_multiplier",
     "uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;",
     "uint64_t p0 = (uint64_t)0xD2511F55u * (uint64_t)c0;"),
    ("philox_key_increment",
     "k0 += 0x9E3779B9u;",
     "k0 += 0x9E3779BBu;"),
    ("gauss_cosine_for_both_lanes",
     "return (lane & 1) ? rho * s : rho * c;",
     "return rho * c;"),
    ("ln_series_coefficient",
     "p = p * t2 + 0x1.99999ap-3f;   /* 1/5  */",
     "p = p * t2 + 0x1.b33334p-3f;   /* 1/5  */"),
    ("cossin_quadrant",
     "case 1: c = -s0; s = c0; break;",
     "case 1: c = s0; s = -c0; break;"),
    ("givens_rotation_sign",
     "W[i + j * s] = c * y - sn * x;",
     "W[i + j * s] = c * y + sn * x;"),
    ("srht_or_instead_of_and",
     "__builtin_popcountll((uint64_t)p[r] & g)",
     "__builtin_popcountll((uint64_t)p[r] | g)"),
    ("scholqr3_shift_without_n",
     "11.0 * ((double)m * (double)n * u + (double)n * (double)(n + 1) * u) * g",
     "11.0 * ((double)m * (double)n * u + (double)(n + 1) * u) * g"),
]


def _source():
    with open(os.path.join(ROOT, "oracle", "rclupp_oracle.c")) as f:
        return f.read()


def _run_pins(tmp_path, src):
    """Run the pin suites against an oracle package built from `src`."""
    pkg = tmp_path / "oracle"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), pkg / "__init__.py")
    (pkg / "rclupp_oracle.c").write_text(src)
    # the copy comes first (the working directory); the repository root, after
    # it, supplies the input generators and the test configuration
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([ROOT] + [p for p in [os.environ.get("PYTHONPATH")] if p]))
    which = subprocess.run([sys.executable, "-c", "import oracle; print(oracle.__file__)"],
                           cwd=tmp_path, env=env, capture_output=True, text=True, timeout=120)
    assert which.returncode == 0 and which.stdout.strip().startswith(str(tmp_path)), which
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] + PINS,
                          cwd=tmp_path, env=env, capture_output=True, text=True, timeout=900)


@pytest.fixture(scope="module")
def source():
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    return _source()


def test_control_copy_passes_the_pins(tmp_path, source):
    r = _run_pins(tmp_path, source)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, source, name, old, new):
    assert source.count(old) == 1, name
    r = _run_pins(tmp_path, source.replace(old, new))
    # exit code 1: tests ran and at least one failed (not a build or collection error)
    assert r.returncode == 1, (name, r.returncode, r.stdout[-3000:], r.stderr[-2000:])
    assert " failed" in r.stdout, (name, r.stdout[-2000:])
