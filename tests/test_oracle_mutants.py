"""Plant one plausible mistake at a time in a copy of the oracle source,
build it, and require that at least one pin check fails on it. This shows
that the pins constrain every part of the oracle: the f update, the alpha
step and its clipping, the kernel, the index sets, the tie-break, the
threshold, the objective and the shrink rule and schedule. Mutants are
built from a temporary copy; the oracle itself is never modified."""
import os
import subprocess
import sys

import pytest

sys.path.insert(0, os.path.dirname(__file__))
import oracle  # noqa: E402
import oracle_pins as P  # noqa: E402

SRC = os.path.join(os.path.dirname(oracle.__file__), "smo_oracle.c")

MUTANTS = {
    "fup_drops_low_term": ("f[i] = f[i] + du * ku + dl * kl;", "f[i] = f[i] + du * ku;"),
    "fup_wrong_sign": ("f[i] = f[i] + du * ku + dl * kl;", "f[i] = f[i] + du * ku - dl * kl;"),
    "step_wrong_sign": ("double t = al + slope / eta;", "double t = al - slope / eta;"),
    "step_wrong_operand": ("double kul = kern(X, nrm, gamma, u, l);\n        or_step st = alpha_step(C, y[u], y[l], alpha[u], alpha[l], f[u], f[l], kuu, kll, kul);\n        alpha[u] = st.au;\n        alpha[l] = st.al;\n        set[u] = (uint8_t)set_of(y[u], alpha[u], C);\n        set[l] = (uint8_t)set_of(y[l], alpha[l], C);\n        update_f(X, nrm, gamma, n, NULL",
                           "double kul = kern(X, nrm, gamma, u, u);\n        or_step st = alpha_step(C, y[u], y[l], alpha[u], alpha[l], f[u], f[l], kuu, kll, kul);\n        alpha[u] = st.au;\n        alpha[l] = st.al;\n        set[u] = (uint8_t)set_of(y[u], alpha[u], C);\n        set[l] = (uint8_t)set_of(y[l], alpha[l], C);\n        update_f(X, nrm, gamma, n, NULL"),
    "clip_upper_bound": ("H = fmin(C, C + al - au);", "H = fmin(C, al - au + C * 0.5);"),
    "clip_same_sign": ("L = fmax(0.0, al + au - C);", "L = fmax(0.0, al - au);"),
    "kernel_dot_factor": ("double d2 = nx + nz - 2.0 * dot;", "double d2 = nx + nz - dot;"),
    "set_up_includes_I3": ("static int in_up(int s) { return s == OR_SET_I0 || s == OR_SET_I1 || s == OR_SET_I2; }",
                           "static int in_up(int s) { return s == OR_SET_I0 || s == OR_SET_I1 || s == OR_SET_I3; }"),
    "set_swap_I2_I3": ("return y > 0 ? OR_SET_I3 : OR_SET_I2; /* a == C */", "return y > 0 ? OR_SET_I2 : OR_SET_I3; /* a == C */"),
    "tie_highest_index": ("(fi == s->b_up && (s->i_up < 0 || i < s->i_up))", "(fi == s->b_up && (s->i_up < 0 || i > s->i_up))"),
    "threshold_b_midpoint": ("return c ? s / (double)c : 0.5 * (b_up + b_low);", "return 0.5 * (b_up + b_low);"),
    "objective_sign": ("return s1 - 0.5 * s2;", "return s1 + 0.5 * s2;"),
    "stop_one_tau": ("while (s.b_low - s.b_up > 2.0 * tau) {", "while (s.b_low - s.b_up > 20.0 * tau) {"),
    "shrink_rule_inverted": ("&& f[i] < s.b_up) ||", "&& f[i] > s.b_up) ||"),
    "shrink_rule_wrong_sets": ("int drop = ((st_i == OR_SET_I3 || st_i == OR_SET_I4) && f[i] < s.b_up) ||\n                               ((st_i == OR_SET_I1 || st_i == OR_SET_I2) && f[i] > s.b_low);",
                               "int drop = ((st_i == OR_SET_I1 || st_i == OR_SET_I2) && f[i] < s.b_up) ||\n                               ((st_i == OR_SET_I3 || st_i == OR_SET_I4) && f[i] > s.b_low);"),
    "recon_skips_label": ("f[a] = acc - (double)y[a];", "f[a] = acc;"),
    "poly_power_off_by_one": ("for (int k = 1; k < g_degree; ++k) r *= b;", "for (int k = 2; k < g_degree; ++k) r *= b;"),
    "poly_drops_coef0": ("const double b = gamma * dot + g_coef0;", "const double b = gamma * dot;"),
    "linear_scaled": ("if (g_kind == 1) return dot;", "if (g_kind == 1) return dot * 0.5;"),
    "wss2_gain_not_squared": ("const double g = (b * b) / a;", "const double g = b / a;"),
    "wss2_shrink_first_order": ("l = select_low2(X, nrm, gamma, m, act, f, set, u, &gap2);",
                                "l = s.i_low; (void)gap2;"),
    "wss2_shrink_ignores_active": ("const int64_t t = act ? act[k] : k;", "const int64_t t = k;"),
    "shrink_counter_floor": ("h = (int64_t)ceil(value * (double)n);", "h = (int64_t)floor(value * (double)n);"),
    "shrink_reset_to_h": ("counter = h < m ? h : m;", "counter = h;"),
    "first_recon_at_2tau": ("double thr = shrinking ? first_factor * tau : 2.0 * tau;",
                            "double thr = 2.0 * tau;"),
    "multi_restart_stale_counter": ("        } else {\n            counter = h;\n        }\n        thr = 2.0 * tau;",
                                    "        } else {\n        }\n        thr = 2.0 * tau;"),
    "recon_never_resets": ("for (int64_t i = 0; i < n; ++i) { act[i] = i; live[i] = 1; }\n        m = n;",
                           "for (int64_t i = 0; i < n; ++i) { live[i] = 1; }"),
}

# cheapest first; stop at the first failing check
ORDER = [P.check_kernel_closed_form, P.check_dot_and_norm, P.check_two_point_closed_form,
         P.check_invariants, P.check_gradient_and_decision, P.check_bruteforce,
         P.check_shrink_none_is_plain, P.check_shrink_keeps_path, P.check_shrink_same_optimum,
         P.check_shrink_schedule,
         P.check_linear_two_point_closed_form, P.check_kernels_bruteforce,
         P.check_linear_decision_is_primal, P.check_kernels_invariants, P.check_wss2,
         P.check_wss2_shrink]


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mutated = src.replace(old, new)
    assert mutated != src
    c = tmp_path / f"{name}.c"
    c.write_text(mutated)
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                           "-std=c99", str(c), "-o", str(so), "-lm"])
    return oracle.load_variant(str(so))


@pytest.mark.timeout(300)
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(orc, tmp_path, name):
    old, new = MUTANTS[name]
    lib = _build(tmp_path, name, old, new)
    caught = []
    for check in ORDER:
        try:
            check(lib=lib)
        except Exception as e:  # noqa: BLE001 - any failure counts as caught
            caught.append((check.__name__, type(e).__name__))
            break
    assert caught, f"planted mistake {name} passed every pin"
