"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle, in its C source or
its Python layer (a dropped term, a wrong sign, a transposed operand, a
wrong index, a wrong constant, a wrong operand order), and runs the pin
suites (test_oracle_pins.py, test_oracle_srht.py) against that copy in a
subprocess: at least one pin must fail.  A control run of the unchanged copy
must pass, and the copy must be the module the subprocess imports.  CPU
only; nothing here touches the product library.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = [os.path.join(ROOT, "tests", "test_oracle_pins.py"),
        os.path.join(ROOT, "tests", "test_oracle_srht.py")]

# (name, original text, planted mistake[, "py" for the Python layer]); each
# original occurs exactly once.
# Mistakes that no output can show are left out (e.g. keeping the LU
# multipliers below N's diagonal: the triangular product reads only N's
# upper triangle).
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
    ("unit_lower_keeps_the_diagonal",
     "IDX(M, ldm, i, j) = i > j ? IDX(A, lda, i, j) : (i == j ? 1.0 : 0.0);",
     "IDX(M, ldm, i, j) = i >= j ? IDX(A, lda, i, j) : 0.0;"),
    ("lc2_gram_of_x_not_m",
     "orc_gram(m, n, M, m, G, n);",
     "orc_gram(m, n, X, ldx, G, n);"),
    ("rcholqr_sign_normalisation_dropped",
     "orc_r0(r0_method, s, n, K, s, R1, n);\n        orc_sign_fix_rows(n, R1, n);",
     "orc_r0(r0_method, s, n, K, s, R1, n);"),
    ("cholqr2_product_order",
     "            if (st == ORC_OK)\n                orc_trmm_upper(n, Z, n, R1, n, R, ldr);",
     "            if (st == ORC_OK)\n                orc_trmm_upper(n, R1, n, Z, n, R, ldr);"),
    ("sparse_duplicate_rows_allowed",
     "            if (dup)\n                continue;\n            rows[cnt] = row;",
     "            if (dup && 0)\n                continue;\n            rows[cnt] = row;"),
    ("sparse_sign_from_the_top_bit",
     "signs[cnt] = (w[t] & 1u) ? (int8_t)-1 : (int8_t)1;",
     "signs[cnt] = (w[t] >> 31) ? (int8_t)-1 : (int8_t)1;"),
    ("bf16_truncates",
     "if (rnd && (sticky || lsb))",
     "if (0)"),
    ("bf16_ties_away_from_zero",
     "if (rnd && (sticky || lsb))",
     "if (rnd)"),
    ("bf16_split_wrong_residual",
     "const double x3 = orc_round_bf16(r1 - x2);",
     "const double x3 = orc_round_bf16(x - x2);"),
    ("tier_levels_without_the_half",
     "orc_normal_quantile(((double)j + 0.5) / 4096.0)",
     "orc_normal_quantile(((double)j + 1.0) / 4097.0)"),
    ("tier_levels_truncated",
     "T[j] = nearbyint(32.0 * orc_normal_quantile(",
     "T[j] = trunc(32.0 * orc_normal_quantile("),
    ("digits_five_instead_of_six",
     "F[i] = (int64_t)round(ldexp(IDX(X, ldx, i, j), 47 - E));",
     "F[i] = (int64_t)round(ldexp(IDX(X, ldx, i, j), 39 - E)) * 256;"),
    ("digits_truncate_instead_of_round",
     "F[i] = (int64_t)round(ldexp(IDX(X, ldx, i, j), 47 - E));",
     "F[i] = (int64_t)trunc(ldexp(IDX(X, ldx, i, j), 47 - E));"),
    ("digits_exponent_off_by_one",
     "        const int E = bmax - 1022;",
     "        const int E = bmax - 1023;"),
    ("tier_quantile_symmetry_sign",
     "        return -orc_normal_quantile(1.0 - p);",
     "        return orc_normal_quantile(1.0 - p);"),
    ("tier_counter_words_swapped",
     "uint32_t ctr[4] = {(uint32_t)q, (uint32_t)(q >> 32), (uint32_t)(uint64_t)r, 0x53424631u};",
     "uint32_t ctr[4] = {(uint32_t)(uint64_t)r, (uint32_t)(q >> 32), (uint32_t)q, 0x53424631u};"),
    ("tier_entries_share_a_half",
     "const uint32_t h = (w[t >> 1] >> (16 * (t & 1))) & 0xffffu;",
     "const uint32_t h = (w[t >> 1] >> (16 * 0)) & 0xffffu;"),
    ("bf16_sketch_scaled_twice",
     "            IDX(Y, ldy, r, j) *= scale;",
     "            IDX(Y, ldy, r, j) *= scale * scale;"),
    ("feistel_widths_not_swapped",
     "        int t = wl;\n        wl = wr;\n        wr = t;",
     "        int t = wl;\n        wl = t;\n        wr = wr;"),
    ("srht_sign_bit_layout",
     "d[i] = ((w[k >> 5] >> (k & 31u)) & 1u)",
     "d[i] = ((w[k & 3u] >> (k >> 2)) & 1u)"),
    ("srht_missing_scale",
     "IDX(S, lds, r, i) = (d[i] < 0 ? -h : h) * scale;",
     "IDX(S, lds, r, i) = (d[i] < 0 ? -h : h);"),
    ("gaussian_sketch_missing_scale",
     "IDX(S, lds, r, i) = (double)orc_gauss_entry(seed, r, i) * scale;",
     "IDX(S, lds, r, i) = (double)orc_gauss_entry(seed, r, i);"),
    ("gepp_rows_not_swapped",
     "        if (p != k)\n            for (int64_t j = 0; j < n; ++j) {\n                double t = IDX(A, lda, k, j);",
     "        if (0)\n            for (int64_t j = 0; j < n; ++j) {\n                double t = IDX(A, lda, k, j);"),
    ("gepp_multiplier_times_pivot",
     "IDX(A, lda, i, k) = IDX(A, lda, i, k) / piv;",
     "IDX(A, lda, i, k) = IDX(A, lda, i, k) * piv;"),
    ("householder_tau_sign",
     "double tau = (beta - alpha) / beta;",
     "double tau = (alpha - beta) / beta;"),
    ("trsm_divides_by_the_first_diagonal",
     "row[j] = acc / IDX(R, ldr, j, j);",
     "row[j] = acc / IDX(R, ldr, 0, 0);"),
    ("gram_one_triangle_only",
     "            IDX(G, ldg, k, j) = acc;\n            IDX(G, ldg, j, k) = acc;",
     "            IDX(G, ldg, k, j) = acc;"),
    ("scholqr3_shift_first_diagonal_not_max",
     "        if (IDX(G, ldg, j, j) > g)\n            g = IDX(G, ldg, j, j);",
     "        if (j == 0)\n            g = IDX(G, ldg, j, j);"),
    ("sparse_apply_scale",
     "double val = 1.0 / sqrt((double)zeta);",
     "double val = 1.0 / (double)zeta;"),
    ("sparse_apply_ignores_signs",
     "double sv = signs[i * zeta + t] > 0 ? val : -val;",
     "double sv = val;"),
    ("sparse_apply_first_nonzero_only",
     "            for (int t = 0; t < zeta; ++t) {\n                int64_t r = rows[i * zeta + t];",
     "            for (int t = 0; t < 1; ++t) {\n                int64_t r = rows[i * zeta + t];"),
    ("cholqr2_second_pass_on_x",
     "st = orc_cholqr(m, n, Q1, m, Q, ldq, Z, n, info);",
     "st = orc_cholqr(m, n, X, ldx, Q, ldq, Z, n, info);"),
    ("givens_rotates_only_zeros",
     "            if (b == 0.0)\n                continue;",
     "            if (b != 0.0)\n                continue;"),
    ("sign_normalisation_of_the_diagonal_only",
     "            for (int64_t j = i; j < n; ++j)\n                IDX(R, ldr, i, j) = -IDX(R, ldr, i, j);",
     "            for (int64_t j = i; j < i + 1; ++j)\n                IDX(R, ldr, i, j) = -IDX(R, ldr, i, j);"),
    # the oracle's Python layer (numpy helpers the tests use as references)
    ("py_sparse_to_dense_scale",
     "val = 1.0 / np.sqrt(zeta)",
     "val = 1.0 / zeta", "py"),
    ("py_sparse_to_dense_sign",
     "np.where(np.asarray(signs) > 0, val, -val)",
     "np.where(np.asarray(signs) > 0, -val, val)", "py"),
    ("py_orthogonality_without_the_identity",
     "q.T @ q - np.eye(n)",
     "q.T @ q - 0.0 * np.eye(n)", "py"),
    ("py_residual_not_relative",
     '/ np.linalg.norm(x, "fro"))',
     ")", "py"),
    ("py_srht_order_off_by_one",
     "    while (1 << b) < m:",
     "    while (1 << b) <= m:", "py"),
    ("py_bf16_split_third_term",
     "x3 = r(x - x1 - x2)",
     "x3 = r(x - x2)", "py"),
]


def _sources():
    """(C source, Python layer) of the oracle."""
    with open(os.path.join(ROOT, "oracle", "rclupp_oracle.c")) as f:
        c = f.read()
    with open(os.path.join(ROOT, "oracle", "__init__.py")) as f:
        py = f.read()
    return c, py


def _run_pins(tmp_path, src, py, pins=PINS):
    """Run the pin suites against an oracle package made of `src` (C) and `py`."""
    pkg = tmp_path / "oracle"
    pkg.mkdir()
    (pkg / "__init__.py").write_text(py)
    (pkg / "rclupp_oracle.c").write_text(src)
    # the copy comes first (the working directory); the repository root, after
    # it, supplies the input generators and the test configuration; one
    # OpenMP thread per run, since several runs go at once
    env = dict(os.environ, OMP_NUM_THREADS="1",
               PYTHONPATH=os.pathsep.join([ROOT] + [p for p in [os.environ.get("PYTHONPATH")] if p]))
    which = subprocess.run([sys.executable, "-c", "import oracle; print(oracle.__file__)"],
                           cwd=tmp_path, env=env, capture_output=True, text=True, timeout=300)
    assert which.returncode == 0 and which.stdout.strip().startswith(str(tmp_path)), which
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] + list(pins),
                          cwd=tmp_path, env=env, capture_output=True, text=True, timeout=1200)


@pytest.fixture(scope="module")
def runs(tmp_path_factory):
    """The control and every mutant, run concurrently (each in its own
    directory and process); name -> CompletedProcess."""
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    c, py = _sources()
    jobs = {"control": (c, py, PINS)}
    for name, old, new, *target in MUTANTS:
        text = py if target == ["py"] else c
        assert text.count(old) == 1, name
        c_m, py_m = (c, py.replace(old, new)) if target == ["py"] else (c.replace(old, new), py)
        # the SRHT's own pins first for its mistakes (-x stops at the first failure)
        jobs[name] = (c_m, py_m, PINS[::-1] if "srht" in name or "feistel" in name else PINS)
    workers = max(1, min(8, os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {name: ex.submit(_run_pins, tmp_path_factory.mktemp(name), src, pysrc, pins)
                for name, (src, pysrc, pins) in jobs.items()}
        return {name: f.result() for name, f in futs.items()}


def test_control_copy_passes_the_pins(runs):
    r = runs["control"]
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(runs, name):
    r = runs[name]
    # exit code 1: tests ran and at least one failed (not a build or collection error)
    assert r.returncode == 1, (name, r.returncode, r.stdout[-3000:], r.stderr[-2000:])
    assert " failed" in r.stdout, (name, r.stdout[-2000:])
