"""Plant plausible mistakes in a copy of the oracle (CPU only) and check that
the pins in test_oracle_pins catch every one of them."""
import ctypes
import os
import subprocess

import pytest

import oracle
import test_oracle_force as force_pins
import test_oracle_hmc as hmc_pins
import test_oracle_pins as pins
import test_oracle_shift as shift_pins
import test_oracle_staggered as stag_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "jqcd_oracle.c")

WILSON_W = "            cplx w = (dir == 0) ? link(L, U, mu, x, a, b) : cconj(link(L, U, mu, y, b, a));"

MUTATIONS = {
    "gamma_x_sign": ("{{0, 0, 0, 1}, {0, 0, 1, 0}, {0, -1, 0, 0}, {-1, 0, 0, 0}},",
                     "{{0, 0, 0, -1}, {0, 0, -1, 0}, {0, 1, 0, 0}, {1, 0, 0, 0}},"),
    # Wilson hop line (the staggered hop has a similar one, declared const)
    "backward_link_not_daggered": (WILSON_W, WILSON_W.replace("cconj(link(L, U, mu, y, b, a))",
                                                              "link(L, U, mu, y, a, b)")),
    "backward_link_transposed_only": (WILSON_W, WILSON_W.replace("cconj(link(L, U, mu, y, b, a))",
                                                                 "link(L, U, mu, y, b, a)")),
    "backward_link_wrong_site": (WILSON_W, WILSON_W.replace("cconj(link(L, U, mu, y, b, a))",
                                                            "cconj(link(L, U, mu, x, b, a))")),
    "forward_link_transposed": (WILSON_W, WILSON_W.replace("link(L, U, mu, x, a, b) :",
                                                           "link(L, U, mu, x, b, a) :")),
    "spin_projector_swapped": ("double s = (dir == 0) ? -(double)sgn : (double)sgn;",
                               "double s = (dir == 0) ? (double)sgn : -(double)sgn;"),
    "no_backward_bc_sign": ("nc[mu] = L->n[mu] - 1;\n          if (mu == 3 && L->tanti) bc = -1.0;",
                            "nc[mu] = L->n[mu] - 1;"),
    "bc_on_wrong_axis": ("if (mu == 3 && L->tanti) bc = -1.0;\n        }\n      } else",
                         "if (mu == 2 && L->tanti) bc = -1.0;\n        }\n      } else"),
    "schur_kappa_not_squared": ("-kappa * kappa); /* out_e", "-kappa); /* out_e"),
    "cg_beta_inverted": ("      double beta = rr_new / rr;", "      double beta = rr / rr_new;"),
    "eo_reconstruction_sign": ("hop_axpy(&L, U, x, t, 1, 1, 0.0, kappa);",
                               "hop_axpy(&L, U, x, t, 1, 1, 0.0, -kappa);"),
    "eo_source_sign": ("hop_axpy(&L, U, b, t, 1, 0, 0.0, kappa);",
                       "hop_axpy(&L, U, b, t, 1, 0, 0.0, -kappa);"),
    "eo_rhs_without_dagger": ("schur(&L, kappa, U, t, rhs, -1, t2);",
                              "schur(&L, kappa, U, t, rhs, 1, t2);"),
    "shift_sign": ("out[i] += A->shift * in[i];", "out[i] -= A->shift * in[i];"),
    "stag_eta_includes_mu": ("for (int nu = 0; nu < mu; ++nu) s += c[nu];",
                             "for (int nu = 0; nu <= mu; ++nu) s += c[nu];"),
    "stag_backward_not_subtracted": ("(dir == 0 ? 1.0 : -1.0) * sgn", "sgn"),
    "stag_half_dropped": ("const double f = 0.5 * eta", "const double f = eta"),
    "stag_backward_link_not_daggered": ("(dir == 0) ? link(L, U, mu, x, a, b) : cconj(link(L, U, mu, y, b, a));\n            acc = cadd(acc, cmul(w, ld(in, b + 3 * y)));",
                                        "(dir == 0) ? link(L, U, mu, x, a, b) : link(L, U, mu, y, a, b);\n            acc = cadd(acc, cmul(w, ld(in, b + 3 * y)));"),
    "gauge_force_no_lower_staple": ("cadd(up.m[a][b], dn.m[a][b])", "up.m[a][b]"),
    "gauge_force_sign": ("cscale(G.m[a][b], -beta / 3.0)", "cscale(G.m[a][b], beta / 3.0)"),
    "plaquette_trace_imaginary": ("sum += P.m[0][0].re + P.m[1][1].re + P.m[2][2].re;",
                                  "sum += P.m[0][0].im + P.m[1][1].re + P.m[2][2].re;"),
    "force_projectors_swapped": ("cm(d - GRE[mu][alpha][beta], -GIM[mu][alpha][beta]);  /* 1 - gamma */",
                                 "cm(d + GRE[mu][alpha][beta], GIM[mu][alpha][beta]);  /* 1 - gamma */"),
    "force_no_boundary_sign": ("if (mu == 3 && L->tanti) s = -1.0;", ""),
    "force_second_term_not_conjugated": ("acc = cadd(acc, cconj(cmul(gp,", "acc = cadd(acc, (cmul(gp,"),
    "force_factor_two_dropped": ("cscale(acc, 2.0 * kappa * s)", "cscale(acc, kappa * s)"),
    "force_link_on_the_right": ("cmul(link(L, U, mu, x, i, b), M[b][a])",
                                "cmul(M[i][b], link(L, U, mu, x, b, a))"),
}

PINS = [
    ("gamma_basis", lambda: pins.test_gamma_basis()),
    ("free_field", lambda: [pins.test_free_field_closed_form(t, d) for t in (True, False)
                            for d in (False, True)]),
    ("gauge_covariance", lambda: pins.test_gauge_covariance(True)),
    ("adjoint", lambda: pins.test_adjoint_and_gamma5_hermiticity()),
    ("dense", lambda: pins.test_dense_brute_force((2, 2, 2, 4), True)),
    ("cg_free", lambda: pins.test_cg_free_field_inverse()),
    ("shifted_cg", lambda: shift_pins.test_shifted_cg_against_dense(True)),
    ("staggered_dense", lambda: stag_pins.test_staggered_dense_brute_force((2, 2, 2, 4), True)),
    ("staggered_free", lambda: stag_pins.test_staggered_free_field(True)),
    ("cold_start", lambda: hmc_pins.test_cold_start_action()),
    ("gauge_force_derivative", lambda: hmc_pins.test_gauge_force_is_the_derivative()),
    ("force_derivative", lambda: force_pins.test_force_is_the_derivative_of_the_action(True)),
    ("force_covariance", lambda: force_pins.test_force_gauge_covariance()),
]


def _build_mutant(tmp_path, name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation {name} does not match the oracle source"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    lib = tmp_path / f"lib_{name}.so"
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-std=c11", str(path), "-o", str(lib),
                    "-lm"], check=True)
    return oracle._configure(ctypes.CDLL(str(lib)))


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name, tmp_path, monkeypatch):
    monkeypatch.setattr(oracle, "_lib", _build_mutant(tmp_path, name))
    caught = None
    for pin, fn in PINS:  # stop at the first pin that fails
        try:
            fn()
        except (AssertionError, RuntimeError, ValueError, FloatingPointError):
            caught = pin
            break
    assert caught, f"no pin detects mutation {name}"
