"""Planted mistakes in the oracle must be caught by the pins (CPU only).

Each mutant is a copy of oracle.c with one plausible bug, compiled on the fly; at least one pin
must fail on it.  The oracle source itself is never modified."""
import os
import subprocess
import tempfile

import pytest

import oracle
import oracle_pins as pins

MUTANTS = {
    "dropped_last_term": ("for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {\n      const double a = val[e];",
                          "for (int64_t e = rowptr[i]; e + 1 < rowptr[i + 1]; ++e) {\n      const double a = val[e];"),
    "tile_boundary_off_by_one": ("if (j >= c0 && j < c0 + width) {", "if (j >= c0 && j <= c0 + width && j < K) {"),
    "rank_shifted": ("rank[j] = u;", "rank[j] = u + (u > 1);"),
    "sddmm_sign": ("for (int32_t k = 0; k < N; ++k) s += g[k] * b[k];", "for (int32_t k = 0; k < N; ++k) s -= g[k] * b[k];"),
    "spmm_t_transposed_operand": ("d[k] += val[e] * g[k];", "d[k] += val[e] * g[k] * (k == 0 ? 1.0 : 0.5);"),
    "transpose_unstable": ("int64_t pos = fill[col[e]]++;", "int64_t pos = rowptrT[col[e] + 1] - 1 - (fill[col[e]]++ - rowptrT[col[e]]);"),
    "bounds_floor": ("int64_t b = (n + P - 1) / P;", "int64_t b = n / P > 0 ? n / P : 1;"),
    "rows_count_per_nnz": ("rows_t += row_hit;", "rows_t += row_hit ? (rowptr[i + 1] - rowptr[i]) : 0;"),
    "abs_scale_signed": ("const double a = fabs(val[e]);", "const double a = val[e];"),
    "cut_read_flipped": ("cover_col[v] = (uint8_t)(via[1 + nL + v] != -2);", "cover_col[v] = (uint8_t)(via[1 + nL + v] == -2);"),
    "no_residual_twin": ("cap[via[x] ^ 1] += b;", "(void)0;"),
    "source_capacity_wrong": ("ORACLE_ARC(s, 1 + u, w_row[u]);", "ORACLE_ARC(s, 1 + u, w_row[u] + (u == 0));"),
    "scaled_error_plus_one": ("else r = d / s;", "else r = d / (s + 1.0);"),
    "scaled_error_zero_rule_dropped": ("else if (s == 0.0) r = (c == 0.0) ? 0.0 : INFINITY;",
                                       "else if (s == 0.0) r = 0.0;"),
    "scaled_error_mean": ("if (r > rmax) rmax = r;", "rmax += r / (double)N;"),
    "scaled_error_relative_to_c64": ("else r = d / s;", "else r = d / fabs(C64[i * ld64 + k]);"),
    "scaled_error_signed": ("const double d = fabs(c - C64[i * ld64 + k]);",
                            "const double d = c - C64[i * ld64 + k];"),
    "volumes_width_off_by_one": ("v_block[t] = (cb[q + 1] - cb[q]) * (int64_t)N * sz;",
                                 "v_block[t] = (cb[q + 1] - cb[q] + 1) * (int64_t)N * sz;"),
    "volumes_q_of_row_block": ("int32_t q = diag_only ? t : t % Pc;\n    v_block",
                               "int32_t q = diag_only ? t : t / Pc;\n    v_block"),
    "matching_no_flip": ("for (int32_t l = d - 1; l >= 0; --l) matchR[sv[l]] = su[l];", "(void)sv;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    src = src.replace(old, new, 1)
    c = tmp_path / "mut.c"
    c.write_text(src)
    so = str(tmp_path / "libmut.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", str(c),
                    "-o", so, "-lm"], check=True)
    oracle.lib()
    prev = oracle.use_library(so)
    failed = []
    try:
        for chk in pins.ALL_CHECKS:
            try:
                chk()
            except (AssertionError, ValueError):
                failed.append(chk.__name__)
    finally:
        oracle.use_library(prev)
    assert failed, f"no pin caught the planted mistake {name}"
