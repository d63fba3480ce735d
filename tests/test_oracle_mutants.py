"""The oracle pins catch plausible mistakes.

Each case plants one mistake in a temporary copy of the oracle's C source
(a dropped term, a wrong sign or scale, a wrong index, a frozen or misrouted
transmission, a wrong weight), builds it with gcc and runs the pins of
``test_oracle_pins`` against it until one fails.  A mutant that passes every
pin means the pins leave that part of the oracle unchecked.  CPU only.
"""
import os
import subprocess
import tempfile

import pytest

import oracle
from oracle import oracle as _oracle_mod
import test_oracle_pins as P
import test_oracle_bruteforce as B

SRC = os.path.join(os.path.dirname(_oracle_mod.__file__), "pma_oracle.c")

# pins in rough order of cost; each mutant stops at the first that fails
PINS = [
    ("monitor", P.test_monitor_closed_forms),
    ("first_step", lambda: [P.test_first_step_from_identity_in_closed_form(d, r)
                            for d in (1, 2, 3) for r in ("log", "root")]),
    ("l2_norm", lambda: [P.test_l2_increment_residual_is_the_trapezoid_norm_of_the_step(d)
                         for d in (1, 2, 3)]),
    ("bruteforce", B.check_all),
    ("alternating_order", P.test_alternating_transmission_takes_new_values_from_preceding_owners_only),
    ("quad1", lambda: P.test_operator_exact_on_quadratics(1)),
    ("quad2", lambda: P.test_operator_exact_on_quadratics(2)),
    ("quad3", lambda: P.test_operator_exact_on_quadratics(3)),
    ("mirror", P.test_neumann_mirror_keeps_boundary_nodes_on_boundary),
    ("mass1d", P.test_1d_trapezoid_sum_of_det_is_domain_length),
    ("extents", P.test_extents_overlap_and_cores),
    ("uniform2dd", lambda: P.test_uniform_density_keeps_identity(2, (2, 3, 1), 4)),
    ("uniform3dd", lambda: P.test_uniform_density_keeps_identity(3, (2, 2, 2), 3)),
    ("separable", P.test_separable_density_reduces_to_1d),
    ("symmetric", P.test_symmetric_density_gives_symmetric_mesh),
    ("stop", P.test_stop_rule_and_status),
    ("ma_steady", P.test_steady_state_satisfies_monge_ampere_config1),
    ("equidist1d", P.test_1d_steady_state_equidistributes),
    ("dd_steady", lambda: P.test_dd_steady_state_equals_single_domain(0)),
    ("overlap", P.test_dd_error_decreases_with_overlap),
    ("table", P.test_table_monitor_is_exact_on_multilinear_densities),
    ("alternating", lambda: P.test_dd_steady_state_equals_single_domain(1)),
    ("exchange1", P.test_exchange_every_one_is_the_parallel_method),
    ("frozen", P.test_frozen_interface_data_hold_between_exchanges),
]

MUTANTS = {
    "cross_term_sign": ("vget(s, v, pp[0], pp[1], pp[2]) - vget(s, v, pm[0], pm[1], pm[2]) -",
                        "vget(s, v, pp[0], pp[1], pp[2]) + vget(s, v, pm[0], pm[1], pm[2]) -"),
    "cross_term_scale": ("(4.0 * d->h[a] * d->h[b])", "(2.0 * d->h[a] * d->h[b])"),
    "gradient_scale": ("x[a] = xi + (vp - vm) / (2.0 * d->h[a]);",
                       "x[a] = xi + (vp - vm) / (d->h[a]);"),
    "diagonal_dropped_centre": ("(vp - 2.0 * vc + vm)", "(vp - vc + vm)"),
    "mirror_one_sided": ("if (i < 0) return -i;", "if (i < 0) return 0;"),
    "mirror_high_side": ("return 2 * (n - 1) - i;", "return n - 1;"),
    "det3_sign": ("H[0][1] * (H[1][0] * H[2][2] - H[1][2] * H[2][0]) +",
                  "H[0][1] * (H[1][0] * H[2][2] - H[1][2] * H[2][0]) -"),
    "xi_offset_local": ("xi = d->lo[a] + (double)(s->lo[a] + c[a]) * d->h[a];",
                        "xi = d->lo[a] + (double)(c[a]) * d->h[a];"),
    "frozen_transmission": ("u->vn[k] = (ddp->alternating && o < s) ? w->vn[ko] : w->v[ko];",
                            "u->vn[k] = u->v[k];"),
    "transmission_new_for_all": ("u->vn[k] = (ddp->alternating && o < s) ? w->vn[ko] : w->v[ko];",
                                 "u->vn[k] = w->vn[ko];"),
    "theta_all_nodes": ("if (is_owned(u, d.dim, gidx)) {", "if (1) {"),
    "trapezoid_weight": ("return (gi == 0 || gi == d->N[a] - 1) ? 0.5 * d->h[a] : d->h[a];",
                         "return d->h[a];"),
    "euler_sign": ("u->vn[k] = u->v[k] + p->dt * F;", "u->vn[k] = u->v[k] - p->dt * F;"),
    "log_dropped": ("F = log(u->R[k] * u->D[k]) - c;", "F = u->R[k] * u->D[k] - c;"),
    "ring_radius_sign": ("s = q - t->r2;", "s = q + t->r2;"),
    "sine_axes_swapped": ("double s = x[t->axis] - t->c[t->axis] - t->a * sin(2.0 * OR_PI * t->k * x[t->along]);",
                          "double s = x[t->along] - t->c[t->along] - t->a * sin(2.0 * OR_PI * t->k * x[t->axis]);"),
    "core_partition_floor": ("long b0 = (2 * (long)k * n + parts) / (2 * parts);",
                             "long b0 = ((long)k * n) / parts + 1;"),
    "owner_output_from_first": ("int o = owner_of(d, gidx);\n        const sub_t *s = &d->sub[o];",
                                "int o = 0;\n        const sub_t *s = &d->sub[o];"),
    "table_weights_swapped": ("w *= up ? frac[a] : 1.0 - frac[a];",
                              "w *= up ? 1.0 - frac[a] : frac[a];"),
    "table_not_clamped": ("if (s > (double)(m->tn[a] - 1)) s = (double)(m->tn[a] - 1);",
                          ""),
    "table_cell_stride": ("stride[1] = m->tn[0];", "stride[1] = m->tn[1];"),
    "l2_no_sqrt": ("if (p->stop_norm == OR_STOP_L2_INCREMENT) rs = sqrt(rs);", ""),
    "l2_weights_not_halved": ("w *= (c3[a] == 0 || c3[a] == u->n[a] - 1) ? 0.5 * d.h[a] : d.h[a];",
                              "w *= d.h[a];"),
    "root_exponent_half": ("1.0 / (double)d.dim) - 1.0;", "0.5) - 1.0;"),
    "root_theta_not_lagged": ("double th = (p->lag_theta ? theta_prev : theta);",
                              "double th = theta;"),
    "alternating_order": ("(ddp->alternating && o < s)", "(ddp->alternating && o > s)"),
    "any_rule_is_max": ("last_res = (p->stop_rule == OR_RULE_ANY) ? rmin : rmax;",
                        "last_res = rmax;"),
    "normalisation_always_on": ("if (p->normalize == OR_NORM_GLOBAL_THETA) c = log(theta / d.vol);",
                                "c = log(theta / d.vol);"),
    "exchange_every_step": ("exchange = (n % exchange_every) == 0;", "exchange = 1;"),
    "exchange_phase": ("exchange = (n % exchange_every) == 0;",
                       "exchange = ((n + 1) % exchange_every) == 0;"),
    "frozen_takes_owner": ("              u->vn[k] = u->v[k];\n              continue;",
                           "              u->vn[k] = d.sub[owner_of(&d, gidx)].v[0];\n              continue;"),
}


def _build_mutant(name, tmp):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation site for %s not found" % name
    src = src.replace(old, new, 1)
    cpath = os.path.join(tmp, "m_%s.c" % name)
    with open(cpath, "w") as f:
        f.write(src)
    hdr = os.path.join(os.path.dirname(SRC), "pma_oracle.h")
    so = os.path.join(tmp, "m_%s.so" % name)
    subprocess.run(["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                    "-I", os.path.dirname(hdr), "-o", so, cpath, "-lm"], check=True)
    return so


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name):
    with tempfile.TemporaryDirectory() as tmp:
        so = _build_mutant(name, tmp)
        caught = None
        with oracle.oracle.use_library(so):
            for pin, fn in PINS:
                try:
                    fn()
                except (AssertionError, ValueError, FloatingPointError):
                    caught = pin
                    break
        assert caught is not None, "no pin catches mutant %s" % name
