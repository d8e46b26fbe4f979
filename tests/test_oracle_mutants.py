"""The oracle's pins must catch plausible mistakes in the oracle itself.

Each case copies oracle/adpar_oracle.c to a temporary directory, plants one
mistake (a dropped term, a wrong sign, index or tie rule, a transposed
operand), builds it with the oracle's own flags and runs the pin suite
against that build in a subprocess.  The suite must fail for every mutant.
Nothing here touches the committed oracle or any GPU.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "adpar_oracle.c")

MUTANTS = {
    "max_tie_to_later": ("case O_MAX: return (t >= a) ? 1.0 : 0.0;",
                         "case O_MAX: return (t > a) ? 1.0 : 0.0;"),
    "min_tie_to_later": ("case O_MIN: return (t <= a) ? 1.0 : 0.0;",
                         "case O_MIN: return (t < a) ? 1.0 : 0.0;"),
    "mul_wrong_operand": ("case O_MUL: return t;\n", "case O_MUL: return a;\n"),
    "linrec_jright_transposed": ("Jr->v[1][0] = prev[1];", "Jr->v[0][1] = prev[1];"),
    "linrec_jleft_dropped_term": ("Jl->v[1][1] = x[0];", "Jl->v[1][1] = 1.0;"),
    "scan_first_element_dropped": ("for (int c = 0; c < w; ++c) asb[c][0] += rsbar[c];",
                                   "for (int c = 0; c < w; ++c) asb[c][0] += 0.0 * rsbar[c];"),
    "scan_overwrites_adjoint": ("rsbar[(i - 1) * w + c] += dl[c];\n            asb[c][i] += dr[c];",
                                "rsbar[(i - 1) * w + c] += dl[c];\n            asb[c][i] = dr[c];"),
    "reduce_general_overwrites_adjoint": ("asb[c][i] += dr[c];\n            g[c] = dl[c];",
                                          "asb[c][i] = dr[c];\n            g[c] = dl[c];"),
    "xd_exponent_dropped": ("r.e = a.e + b.e + e;", "r.e = a.e + b.e;"),
    "hist_chain_wrong_factor": ("g[b] = ft * g[b];", "g[b] = fa * g[b];"),
    "scatter_wrong_index": ("vsbar[j] += ysbar_inout[k];", "vsbar[j] += ysbar_inout[j];"),
    "sqdist_sign": ("asbar[i * width + k] += -2.0 * diff * xb;",
                    "asbar[i * width + k] += 2.0 * diff * xb;"),
    "kmeans_sign": ("ybar * (-2.0) * (X[i * d + j] - C[arg * d + j]);",
                    "ybar * (2.0) * (X[i * d + j] - C[arg * d + j]);"),
    "prod_zero_count_off": ("if (first < 0) first = i;\n            ++nz;",
                            "if (first < 0) first = i + 1;\n            ++nz;"),
    "jvp_right_jacobian_transposed": ("mat_vec(&Jr, xd, t2, w);", "mat_t_vec(&Jr, xd, t2, w);"),
    "jvp_left_term_dropped": ("rd[c] = t1[c] + t2[c];", "rd[c] = t2[c];"),
    "reduce_general_jacobians_swapped": ("mat_t_vec(&Jr, g, dr, w);\n        mat_t_vec(&Jl, g, dl, w);",
                                         "mat_t_vec(&Jl, g, dr, w);\n        mat_t_vec(&Jr, g, dl, w);"),
    "reduce_general_linrec_neutral": ("if (op == O_LINREC) { t[0] = 1.0; t[1] = 0.0; }",
                                      "if (op == O_LINREC) { t[0] = 1.0; t[1] = 1.0; }"),
    "reduce_general_chain_not_carried": ("            g[c] = dl[c];\n", "            g[c] = g[c] + 0.0 * dl[c];\n"),
    "hist_general_jacobians_swapped": ("mat_t_vec(&Jr, &gb[k * w], to_v, w);\n        mat_t_vec(&Jl, &gb[k * w], to_t, w);",
                                       "mat_t_vec(&Jl, &gb[k * w], to_v, w);\n        mat_t_vec(&Jr, &gb[k * w], to_t, w);"),
    "hist_general_chain_not_carried": ("gb[k * w + c] = to_t[c];", "gb[k * w + c] += 0.0 * to_t[c];"),
    "hist_general_operands_transposed": ("scan_combine(op, &tp[i * w], x, out);",
                                         "scan_combine(op, x, &tp[i * w], out);"),
    "hist_general_linrec_neutral": ("bins[k * 2 + 1] = 0.0;", "bins[k * 2 + 1] = 1.0;"),
    "wide_matrix_product_order": ("out[2 * j + k] = r[2 * j + 0] * l[0 + k] + r[2 * j + 1] * l[2 + k];",
                                  "out[2 * j + k] = l[2 * j + 0] * r[0 + k] + l[2 * j + 1] * r[2 + k];"),
    "wide_jleft_transposed": ("Jl->v[2 * j + k][2 * m + k] = x[2 * j + m];",
                              "Jl->v[2 * j + k][2 * m + k] = x[2 * m + j];"),
    "wide_jright_wrong_column": ("Jr->v[4 + j][2 * j + m] = prev[4 + m];", "Jr->v[4 + j][2 * m + j] = prev[4 + m];"),
    "wide_linrec_jright_transposed": ("{ { prev[0], 0.0 }, { prev[1], 1.0 } }", "{ { prev[0], prev[1] }, { 0.0, 1.0 } }"),
    "kmeans_hessdiag_factor": ("H[(int64_t)c * d + j] = 2.0 * ybar * (double)cnt[c];",
                               "H[(int64_t)c * d + j] = ybar * (double)cnt[c];"),
    "kmeans_tie_to_highest_k": ("if (s < best) { best = s; arg = c; }\n        }\n        if (argmin_out)",
                                "if (s <= best) { best = s; arg = c; }\n        }\n        if (argmin_out)"),
    "kmeans_hessdiag_tie_to_highest_k": ("if (s < best) { best = s; arg = c; }\n        }\n        if (arg >= 0) ++cnt[arg];",
                                         "if (s <= best) { best = s; arg = c; }\n        }\n        if (arg >= 0) ++cnt[arg];"),
    "prod_jvp_uses_updated_product": (
        "td = xd_add(xd_mul(ai, td), xd_mul(t, xd_make(adot[i])));\n        t = xd_mul(t, ai);",
        "t = xd_mul(t, ai);\n        td = xd_add(xd_mul(ai, td), xd_mul(t, xd_make(adot[i])));"),
    "xd_add_exponent_dropped": ("r.e = (r.m == 0.0) ? 0 : a.e + e;", "r.e = (r.m == 0.0) ? 0 : a.e;"),
    "hist_prod_jvp_wrong_factor": ("td[b] = xd_add(xd_mul(vi, td[b]), xd_mul(t[b], xd_make(vdot[i])));",
                                   "td[b] = xd_add(xd_mul(t[b], td[b]), xd_mul(t[b], xd_make(vdot[i])));"),
    "hist_jvp_chain_dropped": ("hd[b] = (ft != 0.0 ? ft * hd[b] : 0.0) + (fa != 0.0 ? fa * vdot[i] : 0.0);",
                               "hd[b] = (fa != 0.0 ? fa * vdot[i] : 0.0);"),
    "map_acc_jvp_scale_term_dropped": ("xsdot[j] = asdot[i] * ws[j] + (wsdot ? as[i] * wsdot[j] : 0.0);",
                                       "xsdot[j] = asdot[i] * ws[j];"),
    "map_acc_jvp_sqdist_sign": ("double dd = (wsdot ? wsdot[j * width + k] : 0.0) - asdot[i * width + k];",
                                "double dd = (wsdot ? wsdot[j * width + k] : 0.0) + asdot[i * width + k];"),
    "scatter_jvp_wrong_index": ("xsdot_inout[k] = vsdot[j];", "xsdot_inout[j] = vsdot[j];"),
    "kmeans_fwd_rev_sign": ("Cbardot[arg * d + j] += ybar * (-2.0) * (0.0 - Cdot[arg * d + j]);",
                            "Cbardot[arg * d + j] += ybar * (2.0) * (0.0 - Cdot[arg * d + j]);"),
    "kmeans_fwd_rev_distance_tangent_sign": ("sd += 2.0 * (-diff) * Cdot[(int64_t)c * d + j];",
                                             "sd += 2.0 * diff * Cdot[(int64_t)c * d + j];"),
    "wide_first_element_dropped": ("for (int c = 0; c < d; ++c) abar[c] += rsb[c];",
                                   "for (int c = 0; c < d; ++c) abar[c] += 0.0 * rsb[c];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not found exactly once: %s" % name
    msrc = tmp_path / "mutant.c"
    msrc.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           "-ffp-contract=off", "-fno-fast-math", "-o", str(lib),
                           str(msrc), "-lm"])
    env = dict(os.environ, ADPAR_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "pins did not catch mutant %s:\n%s" % (name, r.stdout[-2000:])
