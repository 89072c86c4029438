"""The oracle's pins are sensitive: each plausible mistake planted in a copy of
the oracle (a dropped term, a wrong sign, index, shift or bound) makes the pin
file named beside it fail.

Every mutant is applied to a temporary copy of ``oracle/`` and ``synth/``,
built there with gcc, and the named test file runs against it in a
subprocess.  The unmutated copy must pass the same files (the control).  The
repository's own oracle is never modified.  Each mutant's text must occur
exactly once in the source, so an edit to the oracle that moves a line shows
up here and the catalogue is brought up to date with it.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC_PATH = os.path.join(ROOT, "oracle", "gse_oracle.c")

F, S, T, V, P, L, O = ("test_oracle_format.py", "test_oracle_spmv.py", "test_oracle_table.py",
                       "test_oracle_table_variants.py", "test_oracle_policy.py", "test_oracle_lowp.py",
                       "test_oracle_solvers.py")

# (name, pin file that must fail, original text, planted text)
MUTANTS = [
    # encode / decode (Sec. III-B, Alg. 1, Alg. 2)
    ("group_exponent_without_plus_one", F, "int Eg = emax == 0 ? 0 : emax + 1;", "int Eg = emax == 0 ? 0 : emax;"),
    ("alignment_shift_off_by_one", F, "int shift = W - 52 - d;         /* M", "int shift = W - 53 - d;         /* M"),
    ("sign_dropped", F, "uint64_t sign = b >> 63;\n            int e = (int)((b >> 52) & 0x7FF);\n            uint64_t M = 0;",
     "uint64_t sign = 0;\n            int e = (int)((b >> 52) & 0x7FF);\n            uint64_t M = 0;"),
    ("hidden_one_for_subnormals", F,
     "            if (e != 0) {\n                uint64_t S = (1ULL << 52) | (b & ((1ULL << 52) - 1));\n                int d = Eg - e;",
     "            {\n                uint64_t S = (1ULL << 52) | (b & ((1ULL << 52) - 1));\n                int d = Eg - e;"),
    ("last_partial_group_short", F, "int64_t lo = g * G, hi = lo + G < nnz ? lo + G : nnz;",
     "int64_t lo = g * G, hi = lo + G < nnz ? lo + G : nnz - 1;"),
    ("nonfinite_accepted", F, "            if (e == 0x7FF) return ORC_NONFINITE;\n            if (e > emax) emax = e;",
     "            if (e > emax) emax = e;"),
    ("decode_bias", F, "double v = ldexp((double)M, Eg - 1023 - Wk);", "double v = ldexp((double)M, Eg - 1022 - Wk);"),
    ("decode_tail_widths_swapped", F, "if (k >= 2) M = (M << seg_bits[1]) | t1;", "if (k >= 2) M = (M << seg_bits[2]) | t1;"),
    ("decode_sign_bit", F, "uint64_t sign = (h >> (s1 - 1)) & 1;", "uint64_t sign = (h >> (s1 - 2)) & 1;"),
    ("level_width_stops_at_two", F, "    for (int i = 1; i < k; i++) w += seg_bits[i];",
     "    for (int i = 1; i < k && i < 2; i++) w += seg_bits[i];"),
    # table format (Sec. III-B extraction, Alg. 1 lookup, Sec. III-C index)
    ("table_entry_without_plus_one", T, "table[n++] = (int16_t)(best + 1);", "table[n++] = (int16_t)(best);"),
    ("table_max_in_first_slot", T, "else if (!taken[emax]) table[n - 1] = (int16_t)(emax + 1);",
     "else if (!taken[emax]) table[0] = (int16_t)(emax + 1);"),
    ("table_ties_to_smaller_exponent", V,
     "if (count[e] > 0 && !taken[e] && (best < 0 || count[e] > count[best])) best = e;",
     "if (count[e] > 0 && !taken[e] && (best < 0 || count[e] >= count[best])) best = e;"),
    ("lookup_accepts_equal_entry", T, "if (diff > 0 && diff < min_diff)", "if (diff >= 0 && diff < min_diff)"),
    ("table_decode_ignores_index", T,
     "out[i] = decode_one(head[i], k >= 2 ? tail1[i] : 0, k >= 3 ? tail2[i] : 0, table[idx[i]], seg_bits, k);",
     "out[i] = decode_one(head[i], k >= 2 ? tail1[i] : 0, k >= 3 ? tail2[i] : 0, table[0], seg_bits, k);"),
    ("sampled_row_counted_once", V, "if (e != 0) count[e] += rows_in_block;", "if (e != 0) count[e] += 1;"),
    ("sampled_last_block_full", V,
     "int64_t rows_in_block = first + block_rows <= n_rows ? block_rows : n_rows - first;",
     "int64_t rows_in_block = block_rows;"),
    ("index_in_head_misplaced", V,
     "head[i] = (uint16_t)((sign << (seg_bits[0] - 1)) | ((uint32_t)idx[i] << ws) | mag);",
     "head[i] = (uint16_t)((sign << (seg_bits[0] - 1)) | ((uint32_t)idx[i] << (ws - 1)) | mag);"),
    ("index_bits_one_too_many", V, "    while ((1 << b) < n_table) b++;", "    while ((1 << b) <= n_table) b++;"),
    # 16-bit baselines (Sec. IV-C)
    ("round_half_up", L, "double n = rint(ldexp(a, -qexp));", "double n = floor(ldexp(a, -qexp) + 0.5);"),
    ("no_carry_into_next_binade", L, "if (ni == (1u << (mbits + 1))) { ni >>= 1; E++; }", ""),
    ("subnormal_quantum", L, "int qexp = (E < emin ? emin : E) - mbits;", "int qexp = E - mbits;"),
    ("overflow_counts_infinite_inputs", L,
     "if (isfinite(val[i]) && ((out[i] >> mb) & ((1 << eb) - 1)) == (1 << eb) - 1) ov++;",
     "if (((out[i] >> mb) & ((1 << eb) - 1)) == (1 << eb) - 1) ov++;"),
    # SpMV (Sec. III-C) and the parity scale
    ("gse_spmv_group_of_the_row", S,
     "                              gexp[j / G], seg_bits, k);\n        s = s + v * x[col[j]];",
     "                              gexp[i / G], seg_bits, k);\n        s = s + v * x[col[j]];"),
    ("dot2_error_term_dropped", S, "        y[i] = p + s;", "        y[i] = p;"),
    ("dot2_twosum_sign", S, "double q = (p - (q0 - z)) + (h - z);", "double q = (p - (q0 - z)) - (h - z);"),
    ("row_scale_without_abs", S, "sa = sa + fabs(h);", "sa = sa + h;"),
    # CG and GMRES
    ("cg_beta_inverted", O,
     "        double beta = rho_new / rho;\n        for (int64_t i = 0; i < n; i++) p[i] = r[i] + beta * p[i];\n        rho = rho_new;\n    }\n    if (trace_n",
     "        double beta = rho / rho_new;\n        for (int64_t i = 0; i < n; i++) p[i] = r[i] + beta * p[i];\n        rho = rho_new;\n    }\n    if (trace_n"),
    ("cg_residual_update_with_p", O,
     "        for (int64_t i = 0; i < n; i++) r[i] = r[i] - alpha * q[i];\n        double rho_new = dot(n, r, r);\n        it++;",
     "        for (int64_t i = 0; i < n; i++) r[i] = r[i] - alpha * p[i];\n        double rho_new = dot(n, r, r);\n        it++;"),
    ("cg_breakdown_missed", O, "        if (pq <= 0.0) { status = ORC_BREAKDOWN; break; }",
     "        if (pq < -1e300) { status = ORC_BREAKDOWN; break; }"),
    ("cg_true_residual_not_recomputed", O, "        residual(n, row_ptr, col, a, b, x, q);\n        info->rel_res_true",
     "        info->rel_res_true"),
    ("givens_sign", O, "hr[j + 1] = -ws->sn[j] * hr[j] + ws->cs[j] * hr[j + 1];",
     "hr[j + 1] = ws->sn[j] * hr[j] + ws->cs[j] * hr[j + 1];"),
    ("back_substitution_transposed", O,
     "for (int c = j + 1; c < i; c++) s = s - ws->Hrot[(int64_t)c * (m + 1) + j] * ws->y[c];",
     "for (int c = j + 1; c < i; c++) s = s - ws->Hrot[(int64_t)j * (m + 1) + c] * ws->y[c];"),
    ("gmres_last_basis_vector_dropped", O,
     "    for (int j = 0; j < i; j++)\n        for (int64_t t = 0; t < n; t++) x[t] = x[t] + ws->y[j] * V[(int64_t)j * n + t];",
     "    for (int j = 0; j + 1 < i; j++)\n        for (int64_t t = 0; t < n; t++) x[t] = x[t] + ws->y[j] * V[(int64_t)j * n + t];"),
    # step metrics and conditions (Sec. III-D, Eqs. 3-6, Conditions 1-3)
    ("rsd_sample_variance", P, "*rsd = sqrt(var / t) / avg;", "*rsd = sqrt(var / (t - 1)) / avg;"),
    ("ndec_counts_ties", P, "if (resid[i] > resid[i + 1]) nd++;", "if (resid[i] >= resid[i + 1]) nd++;"),
    ("reldec_denominator", P, "*reldec = (resid[j - t] - resid[j - 1]) / resid[j - t];",
     "*reldec = (resid[j - t] - resid[j - 1]) / resid[j - 1];"),
    ("condition1_direction", P, "if (rsd > p->rsd_limit && (double)ndec < thr) c |= 1;",
     "if (rsd < p->rsd_limit && (double)ndec < thr) c |= 1;"),
    ("condition3_one_decrease", P, "if (ndec == 0) c |= 4;", "if (ndec <= 1) c |= 4;"),
    ("ndec_limit_ignored", P, "double thr = p->ndec_limit > 0 ? (double)p->ndec_limit : 0.5 * t;", "double thr = 0.5 * t;"),
    # stepped solvers (Alg. 3 and the readings where the paper is silent)
    ("first_check_after_l", O, "return j >= p->l && p->m > 0 && j % p->m == 0;",
     "return j > p->l && p->m > 0 && j % p->m == 0;"),
    ("history_kept_at_a_step", O, "            rho = dot(n, r, r);\n            wlen = 0;\n        }",
     "            rho = dot(n, r, r);\n        }"),
    ("jump_to_kmax", O,
     "                if (orc_step_decide(rsd, ndec, reldec, pol->t, pol)) {\n                    k++; sw[k - 1] = j; restart = 1;",
     "                if (orc_step_decide(rsd, ndec, reldec, pol->t, pol)) {\n                    k = kmax; sw[k - 1] = j; restart = 1;"),
    ("true_residual_at_current_level", O,
     "                residual(n, row_ptr, col, a_levels[kmax - 1], b, x, q);\n                double tr = nrm2(n, q) / nb;",
     "                residual(n, row_ptr, col, a_levels[k - 1], b, x, q);\n                double tr = nrm2(n, q) / nb;"),
    ("stop_on_recurrence_at_kmax", O,
     "                if (k < kmax) { k++; sw[k - 1] = j; }\n                restart = 1;",
     "                if (k < kmax) { k++; sw[k - 1] = j; }\n                else { status = ORC_OK; break; }\n                restart = 1;"),
    ("breakdown_below_kmax_reported", O,
     "            if (k < kmax) { k++; sw[k - 1] = j; restart = 1; }\n            else { status = ORC_BREAKDOWN; break; }",
     "            status = ORC_BREAKDOWN; break;"),
    ("floor_without_x_norm", O, "res <= eta[k] * nrm2(n, x) / nb", "res <= eta[k] / nb"),
    ("level_gap_summed_over_rows", O, "        if (s > eta) eta = s;", "        eta += s;"),
    ("gmres_check_only_on_multiples", O, "j >= pol->l && j / pol->m > j_before / pol->m && wlen >= pol->t + 1",
     "j >= pol->l && j % pol->m == 0 && wlen >= pol->t + 1"),
    ("gmres_history_not_returned", O,
     "        if (hist) for (int i = wlen_before; i < wlen && nh < hist_cap; i++) hist[nh++] = win[i];", ""),
]


def _run_copy(name, pin, old, new, base):
    src = open(SRC_PATH).read()
    if old is not None:
        if src.count(old) != 1:
            return name, f"text occurs {src.count(old)} times"
        src = src.replace(old, new)
    d = os.path.join(base, name)
    for sub in ("oracle", "synth"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub),
                        ignore=shutil.ignore_patterns("*.so", "*.so.tmp*", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(d, "tests"),
                    ignore=shutil.ignore_patterns("__pycache__", os.path.basename(__file__)))
    with open(os.path.join(d, "pytest.ini"), "w") as fh:
        fh.write("[pytest]\ntestpaths = tests\n")
    with open(os.path.join(d, "oracle", "gse_oracle.c"), "w") as fh:
        fh.write(src)
    env = {k: v for k, v in os.environ.items() if not k.startswith("PYTEST")}
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        os.path.join("tests", pin)], cwd=d, capture_output=True, text=True, timeout=600, env=env)
    tail = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else r.stderr[-200:]
    return name, (r.returncode, tail)


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    base = str(tmp_path_factory.mktemp("mutants"))
    jobs = [(m[0], m[1], m[2], m[3], base) for m in MUTANTS]
    jobs += [(f"control_{pin[:-3]}", pin, None, None, base) for pin in sorted({m[1] for m in MUTANTS})]
    with ThreadPoolExecutor(max(2, min(16, os.cpu_count() or 2))) as ex:
        return dict(ex.map(lambda j: _run_copy(*j), jobs))


@pytest.mark.parametrize("pin", sorted({m[1] for m in MUTANTS}))
def test_unmutated_copy_passes(outcomes, pin):
    rc, tail = outcomes[f"control_{pin[:-3]}"]
    assert rc == 0, tail


@pytest.mark.parametrize("name,pin", [(m[0], m[1]) for m in MUTANTS])
def test_planted_mistake_is_caught(outcomes, name, pin):
    res = outcomes[name]
    assert not isinstance(res, str), res
    rc, tail = res
    assert rc == 1 and "failed" in tail, f"{name} survived {pin}: {tail}"
