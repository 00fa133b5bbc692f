"""Plant plausible mistakes in a copy of the oracle and check that a pin catches each.

Every mutation is a textual edit of oracle/fse_oracle.c compiled into a
temporary library (CPU only); the committed oracle is never touched.  A
mutation that no pin detects would mean the pins leave that part of the
oracle unchecked.
"""
import pytest

import oracle_pins as P

MUTATIONS = {
    # Eq. A1: sign of the cross term of the elliptical radius
    "R2_cross_sign": ("         - 4.0 * g2 * t1 * t2;", "         + 4.0 * g2 * t1 * t2;"),
    # Sec. 2: weight exp(-R^2/2 sigma_w^2) loses its factor 2
    "weight_width": ("double c = 1.0 / (2.0 * sw * sw);", "double c = 1.0 / (sw * sw);"),
    # Eqs. 5-6: gain k dropped from the centroid step
    "centroid_gain": ("s.dx = mx / (k_gain * N);", "s.dx = mx / N;"),
    # Sec. 2, k determined from the moments: sign of the g2 cross term of d<x>/dy_c
    "newton_J12_sign": ("double J12 = 2.0 * c * (B * Q12 - 2.0 * gw2 * Q11);",
                        "double J12 = 2.0 * c * (B * Q12 + 2.0 * gw2 * Q11);"),
    # Sec. 2, k determined from the moments: the -N of d<x>/dx_c dropped
    "newton_J11_N": ("double J11 = 2.0 * c * (A * Q11 - 2.0 * gw2 * Q12) - N;",
                     "double J11 = 2.0 * c * (A * Q11 - 2.0 * gw2 * Q12);"),
    # Sec. 2, k determined from the moments: the Newton solve with J transposed
    "newton_transpose": ("s.dx = -(J22 * mx - J12 * my) / dj;", "s.dx = -(J22 * mx - J21 * my) / dj;"),
    # Eq. A5: transposed operand in the X^SH_21 integrand
    "XSH21_operand": ("X21 += f * (4.0 * Wp * p12 * a1);", "X21 += f * (4.0 * Wp * p12 * a2);"),
    # Eq. B9: dropped W' term of P_1
    "P1_dropped_term": ("P1 += f * (4.0 * W * d1 + 2.0 * Wp * d1 * b1);", "P1 += f * (4.0 * W * d1);"),
    # Eq. A6: e^SH loses the factor 2 on e
    "eSH_factor": ("2.0 * e1 + 2.0 * eS1 / T", "e1 + 2.0 * eS1 / T"),
    # Eq. 8: wrong index in P^SH = X - e e^SH
    "PSH_index": ("X[0][1] - e1 * eSH[1]", "X[0][1] - e2 * eSH[1]"),
    # Eq. 9: e_w taken as g_w instead of 2 g_w/(1+g_w^2)
    "e_w_convention": ("double r1 = e1 - 2.0 * gw1 / (1.0 + gg);", "double r1 = e1 - gw1;"),
    # incomplete gamma series: off-by-one in the denominator
    "gamma_series": ("term *= x / (a + k);", "term *= x / (a + k + 1);"),
    # incomplete gamma continued fraction: sign inside a_n
    "gamma_cf": ("double an = -i * (i - a);", "double an = -i * (i + a);"),
    # b'(n): Richardson combination swapped
    "db_richardson": ("return (4.0 * d2 - d1) / 3.0;", "return (4.0 * d1 - d2) / 3.0;"),
    # flux closed form: dropped factor n
    "flux_n": ("return 2.0 * M_PI * n * exp(", "return 2.0 * M_PI * exp("),
    # flux closed form: axis ratio without the (1+|g|)
    "flux_q": ("double q = (1.0 - gabs) / (1.0 + gabs);\n    return", "double q = (1.0 - gabs);\n    return"),
    # Sérsic radius not divided by (1 - |g|)
    "sersic_radius": ("r[((i * w + j) * S + c) * S + a] = sqrt(R2 > 0.0 ? R2 : 0.0) / (1.0 - gabs);",
                      "r[((i * w + j) * S + c) * S + a] = sqrt(R2 > 0.0 ? R2 : 0.0);"),
    # dm/dr_e loses the 1/n
    "jac_re": ("J[1] += I0 * Ek * b * u / (n * re);", "J[1] += I0 * Ek * b * u / re;"),
    # dm/dn: sign of the b' term
    "jac_n_sign": ("(b * log(x) / (n * n) - db)", "(b * log(x) / (n * n) + db)"),
    # Eq. 13: amplitude normalised by sqrt
    "I0_closed_form": ("double I0 = sIf / sff;                                   /* Eq. 13 */",
                       "double I0 = sIf / sqrt(sff);                             /* Eq. 13 */"),
    # start-up: ties / argmax replaced by argmin
    "brightest_pixel": ("if (I[p] > I[best]) best = p;", "if (I[p] < I[best]) best = p;"),
    # start-up: r50 at a quarter of the total instead of half
    "r50_fraction": ("double half = 0.5 * total, prev = 0.0;", "double half = 0.25 * total, prev = 0.0;"),
    # adjoint: the (1 - |g|) part of dr/dg dropped
    "grad_abs_g_term": ("const double dr_g1 = dr_dR2 * dR2_g1 + r / (1.0 - gabs) * dabs1;",
                        "const double dr_g1 = dr_dR2 * dR2_g1;"),
    # adjoint: sign of the cross term in dR^2/dx0
    "grad_x0_cross_sign": ("const double dR2_x0 = -(2.0 * A * t1 - 4.0 * g2 * t2);",
                           "const double dR2_x0 = -(2.0 * A * t1 + 4.0 * g2 * t2);"),
    # adjoint: sign of the pixel gradient
    "grad_dpix_sign": ("if (dpix) dpix[k] = -c;", "if (dpix) dpix[k] = c;"),
    # star (Sec. 4.2): Moffat weight with exponent 2 instead of 3
    "star_moffat_weight": ("W = 1.0 / (t * t * t);", "W = 1.0 / (t * t);"),
    # star: the factor 2 of the Moffat beta
    "star_moffat_beta": ("double ratio = m[2] * m[0] / (2.0 * m[1] * m[1]);",
                         "double ratio = m[2] * m[0] / (m[1] * m[1]);"),
    # star: Gaussian I0 without the axis ratio of the elliptical pixel sums
    "star_gauss_I0_q": ("res->I0 = m[0] / (M_PI * size * size * q);", "res->I0 = m[0] / (M_PI * size * size);"),
    # star: Moffat r50 exponent
    "star_moffat_r50": ("pow(2.0, 1.0 / (beta - 1.0)) - 1.0", "pow(2.0, 1.0 / beta) - 1.0"),
    # implicit gradient: sign of the cross term in dR^2/dxc
    "mom_grad_dR2_cross": ("dR2[0] = -(2.0 * A * t1 - 4.0 * g2 * t2);", "dR2[0] = -(2.0 * A * t1 + 4.0 * g2 * t2);"),
    # implicit gradient: d e_w1 / d g1 with the signs of d e_w2 / d g2
    "mom_grad_dew": ("2.0 * (1.0 - g1 * g1 + g2 * g2) / q", "2.0 * (1.0 + g1 * g1 - g2 * g2) / q"),
    # implicit gradient: d W / d sigma_w loses a power of sigma_w
    "mom_grad_dW_sigma": ("dW[4] = W * R2 / (s * s * s);", "dW[4] = W * R2 / (s * s);"),
    # implicit gradient: sign of the e_w term of d m_3 / d yc
    "mom_grad_dm3": ("dm[2][1] = 2.0 * t2 + ew1 * 2.0 * t2;", "dm[2][1] = 2.0 * t2 - ew1 * 2.0 * t2;"),
    # implicit gradient: VJP solved with J instead of J^T
    "mom_grad_vjp_transpose": ("int n = moment_active_block(J, mode, 1, Ja, act);",
                               "int n = moment_active_block(J, mode, 0, Ja, act);"),
    # implicit gradient: growth-curve r50 derivative with the wrong disc
    "mom_grad_r50_disc": ("dr = ((0.5 - inP) * (S - P)", "dr = ((0.5 - inS) * (S - P)"),
    # implicit gradient: sign of the sigma_w coupling in the VJP
    "mom_grad_kappa_sign": ("for (int k = 0; k < 5; ++k) kappa -= lam[k] * J[k * 5 + 4];",
                            "for (int k = 0; k < 5; ++k) kappa += lam[k] * J[k * 5 + 4];"),
    # cut-out: the side truncated instead of rounded
    "cutout_side_round": ("long side = (long)floor(side_factor * r50 + 0.5);", "long side = (long)floor(side_factor * r50);"),
    # cut-out: the square starts one pixel late
    "cutout_origin": ("int r0 = pr - (int)(side / 2), c0 = pc - (int)(side / 2);",
                      "int r0 = pr - (int)(side / 2) + 1, c0 = pc - (int)(side / 2);"),
    # cut-out: the far edge not cut to the image
    "cutout_clip": ("if (c1 > W) c1 = W;", "if (c1 > W + 1) c1 = W + 1;"),
    # pixel-integrated model: the sub-grid not centred on the pixel
    "ss_subgrid": ("double oy = (c + 0.5) / S - 0.5, ox = (a + 0.5) / S - 0.5;",
                   "double oy = (c + 0.5) / S - 0.5, ox = (a + 0.5) / S;"),
    # pixel-integrated model: the amplitude's template averaged over one sample too few
    "ss_template_mean": ("        f /= d->ns;", "        f /= (d->ns > 1 ? d->ns - 1 : 1);"),
    # pixel-integrated model: dm/dn summed instead of averaged
    "ss_jac_n_mean": ("        J[2] /= d->ns;", ""),
    # non-finite input no longer flagged
    "nonfinite_check": ("if (!isfinite(I[p])) { *status |= ORC_NONFINITE; return 0; }", ""),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(oracle, tmp_path, name):
    old, new = MUTATIONS[name]
    src = oracle.source_text()
    assert old in src, f"mutation site for {name} no longer in the oracle source"
    variant = oracle.compile_variant(src.replace(old, new), str(tmp_path))
    failed = []
    for pin in P.ALL_PINS:
        try:
            pin(variant)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"no pin detects mutation {name}"
