"""Plants plausible mistakes in a copy of the oracle (on the CPU) and checks that the
pins of test_oracle.py catch every one of them."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "psl_oracle.c")

# (name, original text, planted text)
MUTATIONS = [
    ("flip_sign", "Cn[k] = C[k] - 2 *", "Cn[k] = C[k] + 2 *"),
    ("flip_minus_partner_index", "if (j >= k) partners += s[j - k];", "if (j > k) partners += s[j - k];"),
    ("autocorr_dropped_term", "for (uint32_t i = 0; i + k < L; i++)", "for (uint32_t i = 0; i + k + 1 < L; i++)"),
    ("psl_skips_k1", "int32_t p = 0;\n    for (uint32_t k = 1;", "int32_t p = 0;\n    for (uint32_t k = 2;"),
    ("fitness_includes_c0", "wide_set_u64(F, 0);\n    for (uint32_t k = 1;", "wide_set_u64(F, 0);\n    for (uint32_t k = 0;"),
    ("scan_keeps_last_minimum", "wide_cmp(&value_j, &value_step) < 0", "wide_cmp(&value_j, &value_step) <= 0"),
    ("psl_best_keeps_last", "if (psl_j < psl_best_new)", "if (psl_j <= psl_best_new)"),
    ("switch_threshold", "st->unimproved > p->ls_lmt", "st->unimproved >= p->ls_lmt"),
    ("alpha_not_toggled", "(st->alpha == p->alpha1) ? p->alpha2 : p->alpha1", "p->alpha2"),
    ("rng_constant", "0xBF58476D1CE4E5B9ULL", "0xBF58476D1CE4E5B8ULL"),
    ("local_best_not_stored", "memcpy(st->local_best, st->s, L);\n            memcpy(st->value_local",
     "memcpy(st->value_local"),
    ("rounding_not_to_even", "if (round && (sticky || (mant & 1u))) mant++;", "if (round) mant++;"),
    ("window_off_by_one", "((uint64_t)start + i) % L", "((uint64_t)start + i - 1) % L"),
    ("start_bits_inverted", "s[i] = ((d >> (i % 64)) & 1u) ? -1 : 1;", "s[i] = ((d >> (i % 64)) & 1u) ? 1 : -1;"),
    ("power_off_by_one", "for (uint32_t a = 0; a < alpha; a++)", "for (uint32_t a = 1; a < alpha; a++)"),
    ("fbest_ties_take_last", "if (wide_cmp(&f, &b) < 0) {", "if (wide_cmp(&f, &b) <= 0) {"),
    ("fbest_ignores_moves", "memcpy(st->F, value_step.w, sizeof st->F);\n        note_pivot(p, st);",
     "memcpy(st->F, value_step.w, sizeof st->F);"),
    ("fbest_kept_with_two_alphas", "if (p->alpha1 != p->alpha2) return;", "if (p->alpha1 == 0) return;"),
    ("eval_nb_power_table_no_headroom", "power_table(max_abs_sidelobe(C, L) + 4, alpha)",
     "power_table(max_abs_sidelobe(C, L), alpha)"),
    ("eval_nb_neighbour_index_offset", "orc_flip_autocorr(s, C, L, js[q], Cn);",
     "orc_flip_autocorr(s, C, L, (js[q] + 1) % L, Cn);"),
    ("eval_nb_psl_of_pivot", "if (psl_out) psl_out[q] = orc_psl(Cn, L);", "if (psl_out) psl_out[q] = orc_psl(C, L);"),
    ("eval_nb_limb_offset", "memcpy(limbs_out + (size_t)q * WL, v.w, sizeof v.w);",
     "memcpy(limbs_out + (size_t)q * WL + 1, v.w, sizeof v.w - 8);"),
    ("transposed_pair", "c += (int32_t)s[i] * (int32_t)s[i + k];", "c += (int32_t)s[i] * (int32_t)s[L - 1 - i];"),
]


@pytest.mark.slow
@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new):
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation anchor for {name} not unique"
    src = tmp_path / "mut.c"
    src.write_text(text.replace(old, new))
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fvisibility=hidden", "-o", str(lib),
                           str(src), "-lm"])
    env = dict(os.environ, PSL_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not slow", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle.py")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"planted mistake {name} was not caught:\n{r.stdout[-2000:]}"
