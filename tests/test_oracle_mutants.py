"""Planted mistakes in the oracle must fail its pins (CPU only).

Each mutant below is one plausible slip in the oracle's C sources (a dropped
term, a wrong sign, index or operand, a missing conjugate update, a flipped
comparison) applied to a copy of the oracle package.  The oracle's pins
(closed forms, exact distributions, invariants and special cases:
tests/test_oracle_*.py and tests/test_closed_forms.py; not the regression
fixtures of tests/golden/, which the oracle wrote itself) run against every
copy in a child process and must fail; the unmodified copy must pass them.
The children run in parallel; each stops at its first failing pin.
"""
from __future__ import annotations

import os
import re
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

import pytest

HERE = Path(__file__).resolve().parent
ROOT = HERE.parent
ORACLE = ROOT / "oracle"
ORACLE_FILES = ("__init__.py", "smc_oracle.c", "smc_oracle.h", "smc_oracle_prec.inc")
C_SRC, P_SRC = "smc_oracle.c", "smc_oracle_prec.inc"

# (name, file, text, replacement, which occurrence of text)
MUTANTS = [
    # Philox4x32-10 (counter-based generator): a round mixes the wrong key word,
    # the key schedule bumps by the wrong Weyl constant
    ("philox_round_key_word", C_SRC, "c0 = hi1 ^ c1 ^ k0;", "c0 = hi1 ^ c1 ^ k1;", 0),
    ("philox_key_bump", C_SRC, "k1 += PHILOX_W1;", "k1 += PHILOX_W0;", 0),
    ("philox_multiplied_word", C_SRC, "uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;",
     "uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c3;", 0),
    ("key_ignores_run_id", C_SRC, "key[1] = (uint32_t)(seed >> 32) ^ run_id;",
     "key[1] = (uint32_t)(seed >> 32);", 0),
    ("fp32_uniform_bits", C_SRC, "return (float)((w[1] >> 8) | 1u) * 0x1p-24f; }",
     "return (float)((w[1] >> 9) | 1u) * 0x1p-24f; }", 0),
    # variate recipes
    ("box_muller_angle_from_u1", P_SRC, "return rad * COS2PIR(u2);",
     "return rad * COS2PIR(u1);", 0),
    ("box_muller_radius", P_SRC, "R rad = SQRTR((R)-2.0 * LOGR(u1));",
     "R rad = SQRTR((R)-1.0 * LOGR(u1));", 0),
    ("exponential_times_rate", P_SRC, "return -LOGR(u) / rate;", "return -LOGR(u) * rate;", 0),
    ("gamma1_scale_as_rate", P_SRC, "return theta * -LOGR(u);", "return -LOGR(u) / theta;", 0),
    ("uniform_ab_offset", P_SRC, "return FMAR(hi - lo, u, lo);", "return FMAR(hi - lo, u, hi);", 0),
    ("bernoulli_flipped", P_SRC, "return u < p;", "return u > p;", 0),
    ("lognormal_shift_not_scale", P_SRC, "return EXPR(sigma * SFX(normal01)(s));",
     "return EXPR(sigma + SFX(normal01)(s));", 0),
    ("poisson_inversion_term", P_SRC, "p = p * mean / (R)k;", "p = p * mean / (R)(k + 1);", 0),
    ("poisson_ptrs_log_factorial", P_SRC, "- LFACTR(kr))", "- LFACTR(kr - (R)1.0))", 0),
    # the FP32 mode's own elementary functions
    ("fp32_fn_log_series_coef", C_SRC, "R = fmaf(R, z, 0x1.99999ap-2f /* 2/5 */);",
     "R = fmaf(R, z, 0x1.24924ap-2f /* 2/5 */);", 0),
    ("fp32_fn_log_drops_ln2_lo", C_SRC, "const float lo = fmaf(fe, F_LN2_LO, l);",
     "const float lo = l;", 0),
    ("fp32_fn_log_no_halving", C_SRC, "    *e += 1;\n    return f_bits_to_float(frac | (126u << 23));",
     "    return f_bits_to_float(frac | (126u << 23));", 0),
    ("fp32_fn_exp_tail_coef", C_SRC, "q = fmaf(q, r, 0x1.555556p-3f);  /* 1/3! */",
     "q = fmaf(q, r, 0x1.555556p-5f);  /* 1/3! */", 0),
    ("fp32_fn_exp_scale", C_SRC, "  return y * f_pow2(n);", "  return y * f_pow2(n + 1);", 0),
    ("fp32_fn_cos2pi_quadrant_sign", C_SRC, "return quad == 1 ? -sv : sv;",
     "return quad == 1 ? sv : -sv;", 0),
    ("fp32_fn_cos2pi_series_coef", C_SRC, "c = fmaf(c, z, 0x1.03c1f0p-2f);",
     "c = fmaf(c, z, 0x1.03c1f0p-3f);", 0),
    ("fp32_fn_expm1_small_branch", C_SRC, "return x + f_exp_tail(x, 1);",
     "return f_exp_tail(x, 1);", 0),
    ("fp32_fn_lfact_half", C_SRC, "const float a = (x - 0.5f) * orc_logf(x);",
     "const float a = (x + 0.5f) * orc_logf(x);", 0),
    ("poisson_ptrs_shift", P_SRC, "U + mean + (R)0.43);", "U + mean + (R)1.43);", 0),
    ("gamma_mt_d", P_SRC, "const R d = shape - (R)1.0 / (R)3.0;",
     "const R d = shape - (R)1.0 / (R)2.0;", 0),
    ("gamma_mt_log_test_sign", P_SRC, "d * ((R)1.0 - v + LOGR(v))", "d * ((R)1.0 - v - LOGR(v))", 0),
    ("beta_swapped", P_SRC, "return x / (x + y);", "return y / (x + y);", 0),
    ("lomax_shape_times", P_SRC, "return beta * EXPM1R(-LOGR(u) / alpha);",
     "return beta * EXPM1R(-LOGR(u) * alpha);", 0),
    ("neg_binomial_p0_inverted", P_SRC, "R pk = EXPR(-alpha * LOG1PR(tau / beta));",
     "R pk = EXPR(-alpha * LOG1PR(beta / tau));", 0),
    ("neg_binomial_term_index", P_SRC, "pk = pk * (q * (alpha + (R)k) / (R)(k + 1));",
     "pk = pk * (q * (alpha + (R)k + (R)1.0) / (R)(k + 1));", 0),
    ("neg_binomial_mixture_rate", P_SRC, "R lam = SFX(gamma_mt)(s, alpha) / beta;",
     "R lam = SFX(gamma_mt)(s, alpha) * beta;", 0),
    ("binomial_inversion_term", P_SRC, "f = f * r * (R)(n - k) / (R)(k + 1);",
     "f = f * r * (R)(n - k + 1) / (R)(k + 1);", 0),
    ("binomial_no_flip_back", P_SRC, "return flip ? n - k : k;", "return k;", 0),
    ("binomial_btrs_mode_term", P_SRC, "const R h = (R)lfact_d(m) + (R)lfact_d(n - m);",
     "const R h = (R)lfact_d(m) + (R)lfact_d(n - m - 1);", 0),
    ("log_factorial_no_series", C_SRC, "return (x - 0.5) * log(x) - x + HALF_LOG_2PI_D + series;",
     "return (x - 0.5) * log(x) - x + HALF_LOG_2PI_D;", 0),
    ("binomial_logpmf_failure_term", P_SRC,
     "if (z - y > 0) lp = lp + (R)(z - y) * LOGR((R)1.0 - rho);",
     "if (z - y > 0) lp = lp + (R)(z - y) * LOGR(rho);", 0),
    # normaliser, systematic resampling, ESS (Algorithm 1, Section 3.3)
    ("log_z_increment_drops_log_n", C_SRC, "*incr = mx + (log(s) - log((double)N));",
     "*incr = mx + log(s);", 0),
    ("systematic_drops_offset_u", C_SRC, "double y = (double)i + u;", "double y = (double)i;", 0),
    ("systematic_scale", C_SRC, "double r = (double)N / S;", "double r = 1.0 / S;", 0),
    ("normaliser_max_flipped", C_SRC, "if (lw[i] > mx) mx = lw[i];", "if (lw[i] < mx) mx = lw[i];", 0),
    ("step_limit_off_by_one", P_SRC, "const int at_limit = !all_stop && k + 1 >= c->max_segments;",
     "const int at_limit = !all_stop && k >= c->max_segments;", 0),
    ("ess_not_squared", C_SRC, "return (S * S) / q;", "return S / q;", 0),
    ("ess_comparison_flipped", P_SRC, "resample_now = ess < target;", "resample_now = ess > target;", 0),
    ("log_z_closes_every_checkpoint", P_SRC, "const int close = all_stop || at_limit || resample_now;",
     "const int close = 1;", 0),
    ("kept_weights_reset", P_SRC, "nxt[i].logw = resample_now ? (R)0.0 : cur[anc[i]].logw;",
     "nxt[i].logw = (R)0.0;", 0),
    ("state_not_resampled", P_SRC, "SFX(copy_particle)(&nxt[i], &cur[anc[i]]);",
     "SFX(copy_particle)(&nxt[i], &cur[i]);", 0),
    # linear-Gaussian state-space model
    ("lg_drops_normal_constant", P_SRC, "R lp = (R)-0.5 * (dz * dz) - (R)mc->lg_lc;",
     "R lp = (R)-0.5 * (dz * dz);", 0),
    ("lg_observation_sd", P_SRC, "R dz = (y - P->x) / (R)m->r_sd;", "R dz = (y - P->x) / (R)m->q_sd;", 0),
    ("lg_transition_sd", P_SRC, "FMAR((R)m->q_sd, z, (R)m->b)", "FMAR((R)m->r_sd, z, (R)m->b)", 0),
    ("lg_initial_sd", P_SRC, "P->x = FMAR((R)m->x0_sd, z0, (R)m->x0_mean);",
     "P->x = FMAR((R)m->q_sd, z0, (R)m->x0_mean);", 0),
    ("lg_stops_a_step_early", P_SRC, "P->pc = ((int32_t)k + 1 == m->T) ? PC_STOP : 1;",
     "P->pc = ((int32_t)k + 2 >= m->T) ? PC_STOP : 1;", 0),
    # CRBD (Listing 1)
    ("crbd_correction_tips", C_SRC, "mc->corr = (double)(tips - 1) * LN2_D - lnfact;",
     "mc->corr = (double)(tips) * LN2_D - lnfact;", 0),
    ("crbd_survival_uses_lambda", P_SRC, "R lnp1 = -P->mu * dt;", "R lnp1 = -P->lam * dt;", 0),
    ("crbd_tip_drops_rho", P_SRC, ": (R)log(m->rho); /* log rho: a run constant */",
     ": (R)0.0;", 0),
    ("crbd_hidden_lifetime_rate", P_SRC, "R dur = SFX(exponential)(&c->s, c->mu);",
     "R dur = SFX(exponential)(&c->s, c->lam);", 0),
    ("crbd_hidden_detection_test", P_SRC, "if (dur > t) {", "if (dur < t) {", 0),
    ("crbd_branch_drops_ln2", P_SRC, "acc = acc + LN2R;", "acc = acc;", 0),
    ("crbd_branch_count_mean", P_SRC, "int32_t nev = SFX(poisson)(&s, lam * dt);",
     "int32_t nev = SFX(poisson)(&s, lam);", 0),
    ("crbd_hidden_count_length", P_SRC, "int32_t n = SFX(poisson)(&c->s, c->lam * bl);",
     "int32_t n = SFX(poisson)(&c->s, c->lam * t);", 0),
    ("crbd_hidden_event_window", P_SRC, "R lo = t - bl;", "R lo = (R)0.0;", 0),
    ("crbd_skips_last_node", P_SRC, "P->pc = ((int32_t)k + 1 == m->n_nodes) ? PC_STOP : 1;",
     "P->pc = ((int32_t)k + 2 >= m->n_nodes) ? PC_STOP : 1;", 0),
    ("crbd_lambda_prior_scale", P_SRC, "P->lam = SFX(gamma1)(&s, (R)m->lambda_scale);",
     "P->lam = SFX(gamma1)(&s, (R)m->mu_scale);", 0),
    ("crbd_hidden_detection_probability", P_SRC,
     "if (SFX(bernoulli)(&c->s, (R)c->m->rho)) return 0;",
     "if (SFX(bernoulli)(&c->s, (R)1.0 - (R)c->m->rho)) return 0;", 0),
    ("crbd_depth_cap_off_by_one", P_SRC, "if (depth > c->m->depth_cap) {",
     "if (depth >= c->m->depth_cap) {", 0),
    # clade-specific rate shifts
    ("rateshift_root_rate", P_SRC, "lam = lam_p * mult;", "lam = P->lam * mult;", 0),
    ("rateshift_left_child_rate", P_SRC, "lam_p = P->stack[P->sp - 1];", "lam_p = P->stack[0];", 0),
    ("rateshift_pushes_root_rate", P_SRC, "P->stack[P->sp] = lam;", "P->stack[P->sp] = P->lam;", 0),
    ("resampled_stack_short", P_SRC,
     "for (int32_t i = 0; i < src->sp; i++) dst->stack[i] = src->stack[i];",
     "for (int32_t i = 0; i + 1 < src->sp; i++) dst->stack[i] = src->stack[i];", 0),
    # delayed sampling (Section 6.3): missing conjugate updates, wrong predictives
    ("ds_branch_survival_update", P_SRC, "g[3] = g[3] + dt;", "", 0),
    ("ds_node_speciation_update", P_SRC, "g[0] = g[0] + (R)1.0;", "", 0),
    ("ds_branch_count_update", P_SRC, "g[0] = g[0] + (R)nev;", "", 0),
    ("ds_branch_exposure_update", P_SRC, "g[1] = g[1] + dt;", "", 0),
    ("ds_lifetime_exposure_update", P_SRC, "g[3] = g[3] + dur;", "", 0),
    ("ds_lifetime_shape_update", P_SRC, "g[2] = g[2] + (R)1.0;", "", 0),
    ("ds_hidden_count_update", P_SRC, "g[0] = g[0] + (R)n;", "", 0),
    ("ds_hidden_exposure_update", P_SRC, "g[1] = g[1] + bl;", "", 0),
    ("ds_lambda_prior_rate", P_SRC, "g[1] = (R)1.0 / (R)m->lambda_scale;",
     "g[1] = (R)m->lambda_scale;", 0),
    ("ds_mu_prior_rate", P_SRC, "g[3] = (R)1.0 / (R)m->mu_scale;", "g[3] = (R)m->mu_scale;", 0),
    ("ds_survival_predictive", P_SRC, "R lnp1 = -g[2] * LOG1PR(dt / g[3]);",
     "R lnp1 = -g[2] * LOG1PR(g[3] / dt);", 0),
    ("ds_node_factor_inverted", P_SRC, "lnp2 = LOGR(g[0] / g[1]);", "lnp2 = LOGR(g[1] / g[0]);", 0),
    ("ds_hidden_detection_test", P_SRC, "if (dur > t) {", "if (dur < t) {", 1),
    ("ds_branch_drops_ln2", P_SRC, "acc = acc + LN2R;", "acc = acc;", 1),
    ("ds_hidden_event_window", P_SRC, "R lo = t - bl;", "R lo = (R)0.0;", 1),
    ("ds_tip_drops_rho", P_SRC, "lnp2 = (R)log(m->rho);", "lnp2 = (R)0.0;", 0),
    ("ds_drops_correction", P_SRC, "P->logw = P->logw + (R)mc->corr;", "P->logw = P->logw;", 1),
    ("ds_skips_last_node", P_SRC, "P->pc = ((int32_t)k + 1 == m->n_nodes) ? PC_STOP : 1;",
     "P->pc = ((int32_t)k + 2 >= m->n_nodes) ? PC_STOP : 1;", 1),
    ("ds_hidden_detection_probability", P_SRC,
     "if (SFX(bernoulli)(&c->s, (R)c->m->rho)) return 0;",
     "if (SFX(bernoulli)(&c->s, (R)1.0 - (R)c->m->rho)) return 0;", 1),
    # SEIR (Listing 2)
    ("seir_incubation_rate", P_SRC, "hDeltaI = SFX(binomial)(&s, hEP, th[1]);",
     "hDeltaI = SFX(binomial)(&s, hEP, th[2]);", 0),
    ("seir_recovery_rate", P_SRC, "const int32_t hDeltaR = SFX(binomial)(&s, hIP, th[2]);",
     "const int32_t hDeltaR = SFX(binomial)(&s, hIP, th[1]);", 0),
    ("seir_infection_rate", P_SRC, "const int32_t hDeltaE = SFX(binomial)(&s, hTau, th[0]);",
     "const int32_t hDeltaE = SFX(binomial)(&s, hTau, th[3]);", 0),
    ("seir_force_of_infection", P_SRC, "EXPR(-((R)mIP / (R)hN))", "EXPR(-((R)hIP / (R)hN))", 0),
    ("seir_mosquito_birth_survival_swapped", P_SRC,
     "const R mMu = (R)6.0 / (R)7.0, mNu = (R)1.0 / (R)7.0;",
     "const R mMu = (R)1.0 / (R)7.0, mNu = (R)6.0 / (R)7.0;", 0),
    ("seir_mosquito_births", P_SRC, "mS = mS + SFX(binomial)(&s, mN, mNu);", "mS = mS;", 0),
    ("seir_report_probability", P_SRC, "SFX(binomial_logpmf)(y, C[8], th[5]);",
     "SFX(binomial_logpmf)(y, C[8], th[0]);", 0),
    ("seir_cases_not_reset", P_SRC, "SFX(binomial_logpmf)(y, C[8], th[5]);\n        C[8] = 0;",
     "SFX(binomial_logpmf)(y, C[8], th[5]);", 0),
    ("seir_initial_infectious", P_SRC, "const int32_t hI = 1 + SFX(poisson)(&s, (R)5.0);",
     "const int32_t hI = SFX(poisson)(&s, (R)5.0);", 0),
    ("seir_initial_exposed_mean", P_SRC, "const int32_t hE = SFX(poisson)(&s, (R)5.0);",
     "const int32_t hE = SFX(poisson)(&s, (R)4.0);", 0),
    ("seir_initial_susceptible", P_SRC, "C[0] = n - hE - hI - hR;", "C[0] = n - hE - hI;", 0),
    ("seir_mosquitoes_e_not_10", P_SRC,
     "C[4] = (int32_t)FLOORR((R)n * EXPR(u * (R)2.302585092994045684));",
     "C[4] = (int32_t)FLOORR((R)n * EXPR(u));", 0),
    ("seir_incubation_prior", P_SRC,
     "th[1] = SFX(beta)(&s, (R)1.0 + (R)2.0 / (R)4.4, (R)3.0 - (R)2.0 / (R)4.4);",
     "th[1] = SFX(beta)(&s, (R)1.0 + (R)2.0 / (R)4.4, (R)3.0 + (R)2.0 / (R)4.4);", 0),
    ("seir_reporting_prior", P_SRC, "th[5] = SFX(beta)(&s, (R)1.0, (R)1.0);",
     "th[5] = SFX(beta)(&s, (R)2.0, (R)1.0);", 0),
    ("seir_day0_cases", P_SRC, "hDeltaI = hI;", "hDeltaI = 0;", 0),
    ("seir_stops_a_day_early", P_SRC, "P->pc = ((int32_t)k + 1 == m->T) ? PC_STOP : 1;",
     "P->pc = ((int32_t)k + 2 >= m->T) ? PC_STOP : 1;", 1),
    # weighted geometric program (Fig. 2a)
    ("geometric_weight_sign", P_SRC, "P->logw = P->logw + (R)m->geo_logw;",
     "P->logw = P->logw - (R)m->geo_logw;", 0),
    ("geometric_count", P_SRC, "P->count += 1;", "P->count += 2;", 0),
    # follow mode and boundary flags (what every GPU parity test relies on)
    ("follow_adopts_nothing", P_SRC, "if (fa[i] >= 0 && fa[i] < N) anc[i] = fa[i];", ";", 0),
    ("follow_counts_swapped", P_SRC, "if (flag[i]) o->n_flag_mismatch += 1;",
     "if (!flag[i]) o->n_flag_mismatch += 1;", 0),
    ("follow_decision_ignored", P_SRC, "resample_now = c->follow_resampled[k] != 0;", ";", 0),
    ("flag_tolerance_not_scaled", C_SRC, "const double tol = BOUNDARY_EPS * (double)N;",
     "const double tol = BOUNDARY_EPS;", 0),
    ("flag_lower_boundary_ignored", C_SRC, "if (a > 0 && fabs(q[a - 1] - y) < tol) f = 1;", ";", 0),
    ("ess_near_band_absolute", P_SRC, "const int near = fabs(ess - target) <= 1e-9 * target;",
     "const int near = fabs(ess - target) <= 1e-9;", 0),
    # snapshot / resume: a field not restored, the step limit's closure kept in
    # the closed log Z, the snapshot's last segment run a second time
    ("resume_forgets_stack_pointer", P_SRC, "P->sp = in[N + i];", "P->sp = 0;", 0),
    ("resume_closed_log_z_includes_limit", P_SRC, "if (!at_limit) logz_closed = logz;",
     "logz_closed = logz;", 0),
    ("resume_reruns_last_segment", P_SRC, "    propagated = 1;\n", "    propagated = 0;\n", 0),
]

PIN_FILES = sorted(str(p) for p in HERE.glob("test_oracle_*.py") if p.name != Path(__file__).name)
PIN_FILES.append(str(HERE / "test_closed_forms.py"))

# The pins of a mutant's own area run first, as "file" or "file::test" (only
# to reach the failure sooner: every mutant still runs the whole pin suite
# until its first failure).
def _in(f: str, *tests: str) -> list[str]:
    return [str(HERE / f) + ("::" + s if s else "") for s in (tests or ("",))]


AREA_FIRST = [
    (("philox_", "box_muller_", "exponential_", "gamma1_", "uniform_ab_", "bernoulli_",
      "poisson_", "key_", "fp32_uniform_", "lognormal_"), _in("test_oracle_rng.py")),
    (("fp32_fn_",), _in("test_oracle_mathf.py")),
    (("gamma_mt_", "beta_", "binomial_"), _in("test_oracle_seir.py")),
    (("log_factorial_", "seir_"),
     _in("test_oracle_seir.py", "test_day_zero_draws", "test_one_day_transition_law",
         "test_full_run_invariants") + _in("test_oracle_seir.py")),
    (("lomax_", "neg_binomial_"), _in("test_oracle_crbd_ds.py")),
    (("ds_",), _in("test_oracle_crbd_ds.py", "test_crbd_ds_posterior_bookkeeping",
                   "test_crbd_ds_unbiased_vs_quadrature") + _in("test_oracle_crbd_ds.py")),
    (("log_z_increment_", "systematic_", "normaliser_"), _in("test_oracle_resample.py")),
    (("ess_", "log_z_closes_", "kept_weights_"), _in("test_oracle_ess.py")),
    (("lg_", "state_not_resampled"),
     _in("test_oracle_models.py", "test_lg_unbiased_vs_kalman", "test_eq2_ssm_unbiased_vs_kalman")),
    (("crbd_",), _in("test_oracle_models.py", "test_crbd_fixed_rates_unbiased",
                     "test_depth_cap_one_closed_form", "test_crbd_priors_unbiased_vs_quadrature")),
    (("rateshift_", "resampled_stack_"),
     _in("test_oracle_models.py", "test_rateshift_sigma_zero_is_crbd",
         "test_rateshift_fixed_multipliers_unbiased")),
    (("resume_",), _in("test_oracle_resume.py")),
    (("follow_",), _in("test_oracle_models.py", "test_ancestor_follow_mode_adopts")
     + _in("test_oracle_ess.py", "test_follow_mode_adopts_decisions")),
    (("ess_near_",), _in("test_oracle_ess.py", "test_ess_near_band_is_relative")),
    (("flag_",), _in("test_oracle_resample.py")),
    (("geometric_", "step_limit_"),
     _in("test_oracle_models.py", "test_geometric_z_equals_two_and_posterior", "test_step_limit")),
]


def _pin_order(name: str) -> list[str]:
    head = next((h for prefixes, h in AREA_FIRST if name.startswith(prefixes)), [])
    return head + PIN_FILES


def _apply(text: str, old: str, new: str, which: int) -> str:
    starts = [m.start() for m in re.finditer(re.escape(old), text)]
    if which >= len(starts):
        raise ValueError(f"occurrence {which} of {old!r} not found ({len(starts)} found)")
    i = starts[which]
    return text[:i] + new + text[i + len(old):]


def _copy_oracle(dst: Path, mutant=None) -> Path:
    pkg = dst / "oracle"
    pkg.mkdir(parents=True)
    for name in ORACLE_FILES:
        shutil.copy(ORACLE / name, pkg / name)
    if mutant is not None:
        _, fname, old, new, which = mutant
        f = pkg / fname
        f.write_text(_apply(f.read_text(), old, new, which))
    return dst


def _run_pins(root: Path, files: list[str]) -> tuple[int, str]:
    env = dict(os.environ, SMC_ORACLE_UNDER_TEST=str(root), PYTHONDONTWRITEBYTECODE="1")
    # --keep-duplicates keeps the area's tests in front of the files that hold them
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-rf", "-m", "not gpu",
           "-p", "no:cacheprovider", "--keep-duplicates", *files]
    try:
        r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    except subprocess.TimeoutExpired:
        return -1, "timed out"
    return r.returncode, r.stdout + r.stderr


def _first_failure(out: str) -> str:
    m = re.search(r"^FAILED (\S+)", out, re.M)
    return m.group(1) if m else "?"


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    base = tmp_path_factory.mktemp("oracle_mutants")
    jobs = {"(unmodified)": _copy_oracle(base / "unmodified")}
    for mt in MUTANTS:
        jobs[mt[0]] = _copy_oracle(base / mt[0], mt)
    workers = max(1, min(8, os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {name: ex.submit(_run_pins, root, PIN_FILES if name == "(unmodified)"
                                else _pin_order(name))
                for name, root in jobs.items()}
        res = {name: f.result() for name, f in futs.items()}
    return res, jobs


def test_mutant_names_unique_and_sites_found():
    names = [m[0] for m in MUTANTS]
    assert len(names) == len(set(names))
    for _, heads in AREA_FIRST:  # the ordering hints name existing tests
        for h in heads:
            f, _, test = h.partition("::")
            assert Path(f).exists() and (not test or f"def {test}(" in Path(f).read_text()), h
    for _, fname, old, _, which in MUTANTS:
        text = (ORACLE / fname).read_text()
        assert text.count(old) > which, (fname, old)


def test_unmodified_copy_passes_the_pins(outcomes):
    res, jobs = outcomes
    rc, out = res["(unmodified)"]
    assert rc == 0, out[-3000:]
    # the pins ran against the copy, which built its own library
    assert (jobs["(unmodified)"] / "oracle" / "liboracle.so").exists()


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(outcomes, name):
    res, jobs = outcomes
    rc, out = res[name]
    assert (jobs[name] / "oracle" / "liboracle.so").exists(), f"{name}: did not build\n{out[-3000:]}"
    assert rc != 0, f"{name}: survived every pin"
    assert rc == 1, f"{name}: pins did not run (exit {rc})\n{out[-3000:]}"
    assert _first_failure(out) != "?", out[-3000:]
