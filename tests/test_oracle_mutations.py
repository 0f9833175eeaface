"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C sources (never in the real ones),
builds it, and runs the pin tests and the randomised properties against that build; they
must fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ftgemm_oracle.c")

MUTATIONS = {
    "delta_sign": ("dr[ii] = Cr_ref - Cr;", "dr[ii] = Cr - Cr_ref;"),
    "dropped_beta_term": ("if (p->beta != 0.0) Cr = Cr + p->beta * cin_sum;", ""),
    "transposed_operand": ("int64_t p = (trans == OR_TRANS) ? c : r;", "int64_t p = (trans == OR_NO_TRANS) ? c : r;"),
    "injection_point_off_by_one_tile": ("const int64_t kstar = p->bk * (nk / 2);", "const int64_t kstar = p->bk * ((nk + 1) / 2);"),
    "wrong_located_column": ("r.j = (fc >= 0) ? j0 + fc : -1;", "r.j = (fc >= 0) ? j0 + (fc + 1) % nJ : -1;"),
    "dropped_term_in_Be": ("for (int64_t j = j0; j < j0 + nJ; ++j) { double b = b_elem(p, k, j); s = s + b;",
                           "for (int64_t j = j0 + 1; j < j0 + nJ; ++j) { double b = b_elem(p, k, j); s = s + b;"),
    "missing_alpha_in_prediction": ("double Cc = p->alpha * dotp;", "double Cc = dotp;"),
    "online_recompute_over_all_of_K": ("for (int64_t k = 0; k < kh; ++k) {", "for (int64_t k = 0; k < K; ++k) {"),
    "column_prediction_from_magnitude_sums": ("dotp = dotp + Ac[k] * b;", "dotp = dotp + Ac_abs[k] * b;"),
    # binary32-accumulation model of the tensor-core forms
    "acc32_output_not_rounded": ("double v = round32(scale_out(p, acc, i, j));", "double v = scale_out(p, acc, i, j);"),
    "acc32_correction_keeps_faulty_element": ("if (jj != fcl) rest = rest + T[fr + jj * nI];",
                                              "rest = rest + T[fr + jj * nI];"),
    "acc32_accumulator_flip_in_binary64": ("acc = flip_bit32(acc, inj[q].bit);", "acc = flip_bit(acc, inj[q].bit);"),
    "acc32_row_recompute_with_beta": ("const int recompute_row = (nr == 1 && nc == 0 && p->beta == 0.0);",
                                      "const int recompute_row = (nr == 1 && nc == 0);"),
    "acc32_row_recompute_never_used": ("const int recompute_row = (nr == 1 && nc == 0 && p->beta == 0.0);",
                                       "const int recompute_row = 0;"),
    "acc32_row_threshold_without_the_prediction_term": ("P * (gK * (1.0 + piece_sum) +", "P * (gK * (1.0) +"),
    # sampled rows of the plain product
    "gemm_rows_without_beta": ("v = scale_out(p, dot_row_col(p, i, j, 0, -1), i, j);",
                               "v = p->alpha * dot_row_col(p, i, j, 0, -1);"),
    "gemm_rows_shifted_row": ("int64_t i = rows[r];", "int64_t i = rows[(r + 1) % nrows];"),
    # triangular solve
    "trsm_lower_sums_the_diagonal": ("for (int64_t c = 0; c < r; ++c) s = s + T[r + c * ldt] * w[c];",
                                     "for (int64_t c = 0; c <= r; ++c) s = s + T[r + c * ldt] * w[c];"),
    "trsm_upper_reads_the_diagonal": ("for (int64_t c = r + 1; c < n; ++c) s = s + T[r + c * ldt] * w[c];",
                                      "for (int64_t c = r; c < n; ++c) s = s + T[r + c * ldt] * w[c];"),
}


# the emulated FP64 product (emu_oracle.c)
EMU_MUTATIONS = {
    "emu_slices_truncated_not_rounded": ("double a = nearbyint(r);", "double a = floor(r);"),
    "emu_group_pairs_shifted": ("const int32_t* b = &bs[(jj * s + (g - pp)) * K];",
                                "const int32_t* b = &bs[(jj * s + (g - pp + 1) % s) * K];"),
    "emu_group_weight": ("S[jj] = S[jj] * 16 + gi;", "S[jj] = S[jj] * 8 + gi;"),
    "emu_scale_shift_off_by_one_slice": ("const int shift = -4 * (s + 1);", "const int shift = -4 * s;"),
    "emu_checksum_digit_weight": ("for (int t = 0; t < EO_DIGITS; ++t, w *= 16) {",
                                  "for (int t = 0; t < EO_DIGITS; ++t, w *= 8) {"),
    "emu_location_never_recorded": ("if (bits64(before) != bits64(after))", "if (0)"),
    "emu_conversion_drops_high_bits": ("return (double)x;", "return (double)(int64_t)x;"),
    "emu_binary64_stage_without_threshold": ("double tauC = 2.0 * gamma_u(", "double tauC = 0.0 * gamma_u("),
    "emu_more_flagged_rows_accepted": ("#define EO_MAX_FLAGGED_ROWS 4", "#define EO_MAX_FLAGGED_ROWS 5"),
}
EMU_SRC = os.path.join(ROOT, "oracle", "emu_oracle.c")


@pytest.mark.parametrize("name", sorted(MUTATIONS) + sorted(EMU_MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    target, (old, new) = (SRC, MUTATIONS[name]) if name in MUTATIONS else (EMU_SRC, EMU_MUTATIONS[name])
    srcs = []
    for path in (SRC, EMU_SRC):
        text = open(path).read()
        if path == target:
            assert text.count(old) >= 1, f"mutation anchor for {name} not found"
            text = text.replace(old, new)
        out = tmp_path / os.path.basename(path)
        out.write_text(text)
        srcs.append(str(out))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                    "-o", str(lib), *srcs, "-lm"], check=True, capture_output=True)
    env = dict(os.environ, ORACLE_LIB=str(lib))
    tests = [os.path.join(ROOT, "tests", "test_oracle_pins.py"), os.path.join(ROOT, "tests", "test_emu_oracle.py")]
    try:
        import hypothesis  # noqa: F401  (the randomised properties need it)
        tests.append(os.path.join(ROOT, "tests", "test_oracle_properties.py"))
    except ImportError:
        pass
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *tests],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch mutation {name}:\n{r.stdout[-2000:]}"
