"""Plant plausible mistakes in copies of the oracle and check that the pins
catch every one. Each mutant is compiled from a patched copy of
``oracle/gmm_oracle.c`` into a temporary directory; the real oracle is never
modified."""
import ctypes
import inspect
import os
import subprocess
import textwrap

import pytest

import oracle as O
import oracle_pins as P

SRC = os.path.join(os.path.dirname(O.__file__), "gmm_oracle.c")

MUTANTS = {
    "distance_sign": ("double diff = x[c] - mu[i * D + c];", "double diff = x[c] + mu[i * D + c];"),
    "match_not_strict": ("if (d2 < lim)", "if (d2 <= lim)"),
    "k_not_squared": ("double lim = k * k * v[i];", "double lim = k * v[i];"),
    "no_renormalise": ("w[i] = w[i] / s;", "w[i] = w[i];"),
    "no_match_gain": ("w[j] = w[j] + alpha;", "w[j] = w[j];"),
    "no_decay": ("w[i] = (1.0 - alpha) * w[i];", "w[i] = w[i];"),
    "replace_best": ("j = M - 1;", "j = 0;"),
    "sort_ascending": ("key[perm[r - 1]] < key[p]", "key[perm[r - 1]] > key[p]"),
    "sort_unstable": ("key[perm[r - 1]] < key[p]", "key[perm[r - 1]] <= key[p]"),
    "key_w_over_v": ("return w / sqrt(v);", "return w / v;"),
    "payload_not_permuted": ("tmu[r * D + c] = mu[p * D + c];", "tmu[r * D + c] = mu[r * D + c];"),
    "B_not_strict": ("if (s > T)", "if (s >= T)"),
    "fg_rank_off_by_one": ("(rank_j >= B)", "(rank_j > B)"),
    "variance_old_mean": ("            double diff = x[c] - mu[j * D + c];\n            d2 += diff * diff;\n"
                          "        }\n        if (flags",
                          "            double diff = (x[c] - mu[j * D + c]) / (1.0 - rho);\n"
                          "            d2 += diff * diff;\n        }\n        if (flags"),
    "variance_no_decay": ("double vn = (1.0 - rho) * v[j] + rho * d2;", "double vn = v[j] + rho * d2;"),
    "mean_rate_fixed_alpha": ("mu[j * D + c] = (1.0 - rho) * mu[j * D + c] + rho * x[c];",
                              "mu[j * D + c] = (1.0 - alpha) * mu[j * D + c] + alpha * x[c];"),
    "init_weight_unnormalised": ("w[i] = 1.0 / (double)M;", "w[i] = 1.0;"),
    "list1_three_frames": ("if (*cpt == 3)", "if (*cpt == 2)"),
    "list1_plus3_to_depth": ("*F = f_rgb;", "*F = f_d;"),
    "list1_counter_direction": ("*cpt = *cpt + 1;", "*cpt = *cpt - 1;"),
    "invalid_depth_background": ("fdp = fc;", "fdp = 0;"),
    "morph_outside_one": ("int val = 0;", "int val = 1;"),
    "eta_power": ("pow(2.0 * kPi * s2, -0.5 * D)", "pow(2.0 * kPi * s2, -1.0 * D)"),
    "eta_exponent_halving": ("exp(-d2 / (2.0 * s2))", "exp(-d2 / s2)"),
    "eta_sigma_swapped": ("(flags & FLAG_VAR_PER_CHANNEL) ? v[j] : v[j] / D",
                          "(flags & FLAG_VAR_PER_CHANNEL) ? v[j] / D : v[j]"),
    "per_channel_no_divide": ("d2 = d2 / D;", "d2 = d2;"),
    "augmented_imputes_wrong_component": ("x[3] = first ? 0.0 : mn[3];",
                                          "x[3] = first ? 0.0 : mn[7];"),
    "augmented_depth_unscaled": ("depth_scale * (double)depth[n]};", "(double)depth[n]};"),
    # the near-threshold report and the margins, decisions beside it
    "near_match_absolute": ("if (fabs(d2 - lim) <= eps * lim)", "if (fabs(d2 - lim) <= eps)"),
    "near_match_exclusive": ("if (fabs(d2 - lim) <= eps * lim)", "if (fabs(d2 - lim) < eps * lim)"),
    "near_T_absolute": ("if (fabs(acc - T) <= eps * T)", "if (fabs(acc - T) <= eps)"),
    "near_T_exclusive": ("if (fabs(acc - T) <= eps * T)", "if (fabs(acc - T) < eps * T)"),
    "near_key_exclusive": ("if (!twins && fabs(ka - kb) <= eps * fmax(ka, kb))",
                           "if (!twins && fabs(ka - kb) < eps * fmax(ka, kb))"),
    "near_key_dropped": ("near |= NEAR_KEY;", "near |= 0;"),
    "near_key_flags_twins": ("if (!twins && fabs(ka - kb) <= eps * fmax(ka, kb))",
                             "if (fabs(ka - kb) <= eps * fmax(ka, kb))"),
    "near_key_skips_exact_ties": ("if (!twins && fabs(ka - kb) <= eps * fmax(ka, kb))",
                                  "if (ka != kb && fabs(ka - kb) <= eps * fmax(ka, kb))"),
    "twins_by_weight_only": ("const int twins = (w[a] == w[b] && v[a] == v[b]);",
                             "const int twins = (w[a] == w[b]);"),
    "near_depth_in_colour_bits": ("nbits |= info[3] << 4;", "nbits |= info[3];"),
    "margin_match_absolute": ("mrg = fmin(mrg, fabs(d2 - lim) / lim);",
                              "mrg = fmin(mrg, fabs(d2 - lim));"),
    "margin_T_dropped": ("mrg = fmin(mrg, fabs(acc - T) / T);", "mrg = mrg;"),
    "margin_key_dropped": ("mrg = fmin(mrg, fabs(ka - kb) / fmax(ka, kb));", "mrg = mrg;"),
    "margin_depth_from_colour": ("margin_d[n] = md;", "margin_d[n] = mc;"),
    "decision_depth_from_colour": ("dec[6 * n + 3 + k] = (int8_t)dd[k];",
                                   "dec[6 * n + 3 + k] = (int8_t)dc[k];"),
}

# Plausible mistakes in the F1 tooling (Eq. 1-3), planted in copies of
# oracle.f1_scores.
F1_MUTANTS = {
    "recall_over_fp": ("R = tp / (tp + fn)", "R = tp / (tp + fp)"),
    "precision_over_fn": ("P = tp / (tp + fp)", "P = tp / (tp + fn)"),
    "f1_without_two": ("F1 = 2 * P * R / (P + R)", "F1 = P * R / (P + R)"),
    "f1_arithmetic_mean": ("F1 = 2 * P * R / (P + R)", "F1 = (P + R) / 2"),
    "fn_counts_fp": ("fn = int(np.count_nonzero(~p & t))", "fn = int(np.count_nonzero(p & ~t))"),
    "tn_keeps_fn": ("tn = int(p.size - tp - fp - fn)", "tn = int(p.size - tp - fp)"),
    "empty_recall_one": ("R = tp / (tp + fn) if tp + fn else 0.0", "R = tp / (tp + fn) if tp + fn else 1.0"),
}


@pytest.fixture
def swap_oracle_lib():
    saved = O._lib

    def install(lib):
        O._declare(lib)
        O._lib = lib

    yield install
    O._lib = saved


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path, swap_oracle_lib):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found or not unique"
    mutated = src.replace(old, new, 1)
    c_path = tmp_path / "mutant.c"
    c_path.write_text(mutated)
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", str(so),
                    str(c_path), "-lm"], check=True)
    swap_oracle_lib(ctypes.CDLL(str(so)))
    failed = []
    for check in P.ALL_CHECKS:
        try:
            check()
        except AssertionError:
            failed.append(check.__name__)
            break
    assert failed, f"no pin caught mutant {name}"


@pytest.mark.parametrize("name", sorted(F1_MUTANTS))
def test_pins_catch_f1_mutant(name, monkeypatch):
    old, new = F1_MUTANTS[name]
    src = textwrap.dedent(inspect.getsource(O.f1_scores))
    assert src.count(old) == 1, f"mutation site for {name} not found or not unique"
    ns = {"np": O.np}
    exec(src.replace(old, new, 1), ns)
    monkeypatch.setattr(O, "f1_scores", ns["f1_scores"])
    failed = []
    for check in P.ALL_CHECKS:
        try:
            check()
        except AssertionError:
            failed.append(check.__name__)
            break
    assert failed, f"no pin caught F1 mutant {name}"
