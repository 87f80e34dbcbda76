"""Planted mistakes: each one must make at least one oracle pin fail (CPU only).

Every mutant is a copy of the oracle source with one plausible mistake (a dropped
term, a wrong sign, a wrong index, the misprinted branch conditions of Eq. 5),
compiled into a temporary library.  The pins of ``test_oracle.py`` then run
against it; a mutant that passes them all would mean the pins leave that part of
the oracle unchecked.
"""
import os

import pytest

import oracle
from tests import test_oracle as T
from tests import test_oracle_penalty as Q
from tests import test_oracle_shrink as S

MUTANTS = [
    # Eq. 5 exactly as printed (conditions without the +/-1 terms)
    ("eq5_as_printed", "if (g + l1 <= h * w) return -(g + l1) / h;", "if (g <= h * w) return -(g + l1) / h;"),
    ("grad_sign", "g += (tau - 1.0) * y * x;", "g += (1.0 - tau) * y * x;"),
    ("hess_power", "h += tau * (1.0 - tau) * x * x;", "h += tau * (1.0 - tau) * x;"),
    ("svm_hess_factor", "h += 2.0 * x * x;", "h += x * x;"),
    ("svm_grad_label", "g += -2.0 * y * x * b;", "g += -2.0 * x * b;"),
    ("delta_drops_l1", "Delta = lin + ar->gamma * quad + l1;", "Delta = lin + ar->gamma * quad;"),
    ("armijo_drops_sigma", "if (dF <= ar->sigma * a * Delta) { accepted = 1; break; }",
     "if (dF <= a * Delta) { accepted = 1; break; }"),
    ("update_drops_alpha", "if (p->loss == OR_LOSS_LOGISTIC) mq[i] *= exp(alpha * dx[i]);",
     "if (p->loss == OR_LOSS_LOGISTIC) mq[i] *= exp(dx[i]);"),
    ("lr_label_term", "return log1p(expm1(-u) / (1.0 + E)) + (y_i < 0 ? u : 0.0);",
     "return log1p(expm1(-u) / (1.0 + E)) + (y_i > 0 ? u : 0.0);"),
    ("dx_overwrites", "dx[p->row_idx[e]] += d[k] * (double)p->val[e];", "dx[p->row_idx[e]] = d[k] * (double)p->val[e];"),
    ("kkt_branch_swap", "return fabs(g) > l1 ? (g > 0 ? g - l1 : g + l1) : 0.0;",
     "return fabs(g) > l1 ? (g > 0 ? g + l1 : g - l1) : 0.0;"),
    ("refresh_sign", "mq[i] = (p->loss == OR_LOSS_LOGISTIC) ? exp(z[i]) : 1.0 - (double)p->y[i] * z[i];",
     "mq[i] = (p->loss == OR_LOSS_LOGISTIC) ? exp(-z[i]) : 1.0 - (double)p->y[i] * z[i];"),
    ("perm_key_index", "return or_splitmix64_output(s_epoch, (uint64_t)j + 1);",
     "return or_splitmix64_output(s_epoch, (uint64_t)j);"),
    ("nu_ignored", "if (h <= 0.0) h = nu;", "if (h < 0.0) h = nu;"),
    # Eq. 10's log-ratio taken literally for every sample (cancels at large margins)
    ("eq10_literal", "      if (E <= 1.0) return log1p(E / (1.0 + E) * expm1(u)) - (y_i > 0 ? u : 0.0);\n", ""),
    # shrinking: the margin's sign, the w_j != 0 condition, the partition order of the active set
    ("shrink_margin_sign", "const double bound = p->l1 - M / (double)p->n;", "const double bound = p->l1 + M / (double)p->n;"),
    ("shrink_drops_nonzero_w", "active[j] = (w[j] != 0.0 || fabs(g[j]) >= bound) ? 1 : 0;",
     "active[j] = (fabs(g[j]) >= bound) ? 1 : 0;"),
    ("shrink_filter_index", "if (active[perm[t]]) perm[npos++] = perm[t];", "if (active[t]) perm[npos++] = perm[t];"),
    # the separable penalty: its L2 part left out of the line search, of the Hessian diagonal, its L1
    # weight left out of Delta
    ("pen_ls_drops_l2", "if (p->l2 != 0.0) r += 0.5 * p->l2 * ((wj + t) * (wj + t) - wj * wj);", ""),
    ("pen_hess_drops_l2", "    *h += p->l2;\n", ""),
    ("pen_delta_l1_weight", "l1 += p->l1 * (fabs(w[j] + d[k]) - fabs(w[j]));", "l1 += fabs(w[j] + d[k]) - fabs(w[j]);"),
]


def _pins():
    """(name, callable) for every pin in test_oracle.py, parameters expanded."""
    out = [
        ("splitmix", T.test_splitmix64_matches_independent_python),
        ("partition", lambda: T.test_partition_is_sorted_key_order(64)),
        ("dir_hand", lambda: [T.test_direction_hand_cases(*c) for c in
                              [(-3.0, 2.0, 0.0, 1.0), (3.0, 2.0, 0.0, -1.0), (0.5, 1.0, 0.0, 0.0),
                               (0.5, 1.0, 2.0, -1.5), (-0.5, 1.0, -2.0, 1.5), (0.2, 4.0, 0.1, -0.1)]]),
        ("dir_brute", T.test_direction_is_brute_force_argmin),
        ("lr_hess", T.test_logistic_hessian_matches_second_differences),
        ("svm_hess", T.test_svm_generalised_hessian_matches_second_differences),
        ("nu", T.test_nu_replaces_zero_hessian),
        ("loss_change", T.test_row_loss_change_against_the_definition),
        ("extreme", lambda: T.test_maintained_line_search_exact_at_extreme_margins(80.0)),
    ]
    for loss in ("logistic", "l2svm"):
        out += [
            (f"grad_{loss}", lambda l=loss: T.test_gradient_matches_finite_differences(l)),
            (f"ls_{loss}", lambda l=loss: T.test_maintained_line_search_equals_direct(l)),
            (f"p1_{loss}", lambda l=loss: T.test_p1_is_cdn(l)),
            (f"pm_{loss}", lambda l=loss: T.test_p_equals_m_is_diagonal_proximal_newton(l)),
            (f"kkt_{loss}", lambda l=loss: T.test_kkt_is_min_norm_subgradient(l)),
        ]
    out += [
        ("bound_lr", lambda: T.test_delta_bound_descent_and_step_lower_bound("logistic", 0.25)),
        ("bound_svm", lambda: T.test_delta_bound_descent_and_step_lower_bound("l2svm", 2.0)),
        ("fista_lr", lambda: T.test_converged_objective_matches_fista("logistic", 1.0, 3)),
        ("fista_svm", lambda: T.test_converged_objective_matches_fista("l2svm", 0.5, 4)),
        ("shrink_first", lambda: S.test_first_outer_iteration_visits_every_feature(*S.CASES[0])),
        ("shrink_active", lambda: S.test_active_set_from_an_independent_gradient(*S.CASES[0])),
        ("shrink_random", lambda: S.test_active_set_at_random_points(*S.CASES[0])),
        ("shrink_order", lambda: S.test_shrunk_outer_iteration_is_the_restricted_partition(*S.CASES[0])),
        ("pen_step", lambda: Q.test_full_bundle_step_is_the_penalised_proximal_newton_step("logistic", 0.3, 2.0)),
        ("pen_ls", lambda: Q.test_penalised_line_search_equals_direct("logistic", 1.0, 0.5)),
        ("pen_kkt", lambda: Q.test_kkt_is_the_penalised_min_norm_subgradient("l2svm", 0.3, 2.0)),
    ]
    return out


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, old, new):
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mpath = os.path.join(tmp_path, f"mut_{name}.c")
    with open(mpath, "w") as f:
        f.write(src.replace(old, new))
    lib = oracle.compile_source(mpath, os.path.join(tmp_path, f"libmut_{name}.so"))
    saved = oracle._libs.get("default")
    oracle._libs["default"] = oracle._load(lib)
    caught = []
    try:
        for pin_name, fn in _pins():
            try:
                fn()
            except (AssertionError, RuntimeError):
                caught.append(pin_name)
    finally:
        if saved is None:
            oracle._libs.pop("default", None)
        else:
            oracle._libs["default"] = saved
    assert caught, f"no pin caught the planted mistake {name}"
