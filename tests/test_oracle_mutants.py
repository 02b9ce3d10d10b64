"""Plants plausible mistakes in a copy of the oracle and checks that the pins
catch each one.  Every mutant is compiled from a text-substituted copy of
oracle/fbs_oracle.c in a temporary directory, on the CPU; the real oracle is
untouched."""
import os

import pytest

import oracle
from tests import test_oracle_all_slice as als
from tests import test_oracle_conditionals as cond
from tests import test_oracle_geweke as gew
from tests import test_oracle_slice_moments as sm
from tests import test_oracle_three_level as tl

MUTANTS = {
    "eps prior term dropped": (
        "return y * x - exp(eta) - x * x / (2.0 * st->gam[g]);",
        "return y * x - exp(eta);",
        [cond.test_density_differences_match_model_terms]),
    "gamma shape misses nu": (
        "double shape = 0.5 * ((double)N + nu);", "double shape = 0.5 * ((double)N);",
        [cond.test_gamma_step_matches_posterior]),
    "nu conditional as printed (nu / gamma_g)": (
        "0.5 * nu * (c->S1 + c->tau * c->S2);", "0.5 * nu * (c->S1 + nu * c->S2);",
        [cond.test_density_differences_match_model_terms]),
    "sigma^2 shape G/2 (Jacobian dropped)": (
        "double shape = 0.5 * ((double)m->G - 1.0);", "double shape = 0.5 * ((double)m->G);",
        [cond.test_sigma_step_matches_posterior_with_truncation]),
    "theta prior variance c instead of c^2": (
        "1.0 / (m->c[l] * m->c[l])", "1.0 / m->c[l]",
        [cond.test_theta_step_matches_posterior]),
    "shrinkage moves the wrong end": (
        "if (xs > x0) hi = xs; else lo = xs;", "if (xs > x0) lo = xs; else hi = xs;",
        [lambda: sm.test_slice_normal_target(40.0), sm.test_slice_gamma_target_and_far_start]),
    "beta density reads the wrong eps": (
        "rate += exp(m->h[n] + st->eps[(size_t)g * N + n] + xb);",
        "rate += exp(m->h[n] + st->eps[(size_t)g * N] + xb);",
        [lambda: cond.test_beta_step_preserves_conditional(0)]),
    "tau rate doubled": (
        "double rate = m->b + 0.5 * nu * S2;", "double rate = m->b + nu * S2;",
        [cond.test_tau_step_matches_posterior]),
    "gamma step sums |eps| instead of eps^2": (
        "ss += e * e;", "ss += fabs(e);",
        [gew.test_geweke_gene_level_steps]),
    "gamma slice density misses the +1 of the Inverse-Gamma": (
        "orc_gam_ctx c = {shape + 1.0, scale};", "orc_gam_ctx c = {shape, scale};",
        [als.test_gamma_slice_step_matches_posterior]),
    "tau slice density exponent shape instead of shape - 1": (
        "return (c->shape - 1.0) * log(x) - c->rate * x;", "return c->shape * log(x) - c->rate * x;",
        [als.test_tau_slice_step_matches_posterior]),
    "sigma slice density with the sigma^2 Jacobian": (
        "return -c->G * log(x) - c->hS / (x * x);",
        "return -(c->G - 1.0) * log(x) - c->hS / (x * x);",
        [als.test_sigma_slice_step_matches_posterior_with_truncation]),
    "sigma slice ignores the upper bound s_l": (
        "if (!(x > 0.0 && x < c->s)) return -INFINITY;", "if (!(x > 0.0)) return -INFINITY;",
        [als.test_sigma_slice_step_matches_posterior_with_truncation]),
    "psi: rate of b misses b_b": (
        "psi[0] = gv / (b_b + st);", "psi[0] = gv / st;",
        [tl.test_psi_step_matches_posterior]),
    "psi: shape of b counts datasets instead of summing a_k": (
        "sa += a[k];", "sa += 1.0;",
        [tl.test_psi_step_matches_posterior]),
    "psi: prior precision 1/e^2 of m_l dropped": (
        "double w = 1.0 / (prec + 1.0 / (e[l] * e[l]));", "double w = 1.0 / prec;",
        [tl.test_psi_step_matches_posterior]),
    "theta ignores the top-level prior mean": (
        "v * (B1 / sig2 + m->theta_mean[l] / (m->c[l] * m->c[l]))", "v * (B1 / sig2)",
        [tl.test_theta_and_tau_steps_use_the_top_level, tl.test_geweke_top_level_composition]),
    "stepping out never moves right": (
        "if (logu < f(hi, ctx)) hi += w; else break;", "break;",
        [lambda: sm.test_slice_normal_target(0.05)]),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path, monkeypatch):
    old, new, catchers = MUTANTS[name]
    with open(oracle._SRC) as f:
        src = f.read()
    assert src.count(old) == 1, name
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = oracle.build(src=str(path), out=str(tmp_path / "libmutant.so"))
    monkeypatch.setattr(oracle, "_lib", oracle.load(so))
    caught = []
    for fn in catchers:
        try:
            fn()
        except AssertionError:
            caught.append(fn)
    assert caught, f"mutant '{name}' passed every pin"
