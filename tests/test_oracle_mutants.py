"""The oracle pins catch plausible mistakes.

Each case copies oracle/ to a temporary directory, plants one mistake in the
C source or the Python diagnostics (a dropped term, a flipped sign, a wrong
index or a transposed operand), rebuilds it there and runs the pin suite against the copy, which
must then fail. The committed oracle is never modified.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "alpha_rotation_sign": ("- ax[r * 3 + s] + a[r] * a[s]", "+ ax[r * 3 + s] + a[r] * a[s]"),
    "alpha_drops_aaT": ("- ax[r * 3 + s] + a[r] * a[s])", "- ax[r * 3 + s])"),
    "jhat_drops_1_over_gamma": ("vJ[r] /= gbar;", ";"),
    "jhat_skips_alpha": ("vJ[r] += alpha[r * 3 + k] * u[k];", "vJ[r] += (r == k) * u[k];"),
    "mass_matrix_wrong_weight": ("cM * W[a] * W[b] * alpha[rs]", "cM * W[a] * W[a] * alpha[rs]"),
    "mass_matrix_drops_gamma": ("double cM = w[p] * q * beta / (gbar * dV);",
                                "double cM = w[p] * q * beta / dV;"),
    "pair_slot_no_unwrap": ("if (di > 1) di -= c->nx;", ";"),
    "curl_c_sign": ("out[nn + n00] = -DX(Ez);", "out[nn + n00] = DX(Ez);"),
    "curl_n_sign": ("out[2 * nn + c11] = DX(By) - DY(Bx);", "out[2 * nn + c11] = DX(By) + DY(Bx);"),
    "operator_drops_square": ("out[k] = v[k] + td * td * cn[k] + td * mv[k];",
                              "out[k] = v[k] + td * cn[k] + td * mv[k];"),
    "apply_M_wrong_node": ("acc[r] += blk[r * 3 + s] * v[s * nn + h];",
                           "acc[r] += blk[r * 3 + s] * v[s * nn + g];"),
    "rhs_current_sign": ("b[k] = E[k] + td * cn[k] - td * J[k];", "b[k] = E[k] + td * cn[k] + td * J[k];"),
    "faraday_sign": ("B[k] = B[k] - c->dt * cc[k];", "B[k] = B[k] + c->dt * cc[k];"),
    "E_update_drops_extrapolation": ("E[k] = (Etheta[k] - (1.0 - th) * E[k]) / th;", "E[k] = Etheta[k];"),
    "push_no_leapfrog": ("u1[k] = 2.0 * ub[k] - u0[k];", "u1[k] = ub[k];"),
    "push_alpha_transposed": ("ub[r] += alpha[r * 3 + k] * wv[k];", "ub[r] += alpha[k * 3 + r] * wv[k];"),
    "push_double_kick": ("wv[k] = u0[k] + beta * Ep[k];", "wv[k] = u0[k] + 2.0 * beta * Ep[k];"),
    "push_position_uses_u": ("x[p] = wrap_pos(x[p] + c->dt * u1[0] / g1, Lx);",
                             "x[p] = wrap_pos(x[p] + c->dt * u1[0], Lx);"),
    "gather_B_on_nodes": ("    centre_weights(c, x, y, g, W);\n", "    orc_node_weights(c, x, y, g, W);\n"),
    "node_offsets_transposed": ("locate(x, c->dx, c->nx, &i, &fx);\n    locate(y, c->dy, c->ny, &j, &fy);",
                                "locate(x, c->dx, c->nx, &i, &fy);\n    locate(y, c->dy, c->ny, &j, &fx);"),
    "gmres_update_half": ("x[k] += y[i] * V[(int64_t)i * n + k];", "x[k] += 0.5 * y[i] * V[(int64_t)i * n + k];"),
    "gmres_givens_sign": ("H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];",
                          "H[(i + 1) * m + j] = sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];"),
    "sort_unstable": ("perm[start[k] + cursor[k]++] = p;", "perm[start[k + 1] - 1 - cursor[k]++] = p;"),
    "field_energy_factor": ("out[0] = 0.5 * dV * dot(3 * nn, E, E);", "out[0] = dV * dot(3 * nn, E, E);"),
    "push_uses_new_E": ("orc_push(c, off, x, y, ux, uy, uz, w, Et, B0, E0, sums);",
                        "orc_push(c, off, x, y, ux, uy, uz, w, E, B0, E0, sums);"),
    "push_uses_new_B": ("orc_push(c, off, x, y, ux, uy, uz, w, Et, B0, E0, sums);",
                        "orc_push(c, off, x, y, ux, uy, uz, w, Et, B, E0, sums);"),
    "pred_gbar_ignores_E": ("return gamma_of(u[0] + beta * Ep[0], u[1] + beta * Ep[1], u[2] + beta * Ep[2]);",
                            "return gamma_of(u[0], u[1] + beta * Ep[1], u[2] + beta * Ep[2]);"),
    "pred_mismatch_uses_Etheta": ("if (c->gamma_pred) orc_gather_E(c, E, x[p], y[p], Ep0);",
                                  "if (c->gamma_pred) orc_gather_E(c, Etheta, x[p], y[p], Ep0);"),
    "pred_mismatch_sign": ("d1 += (us - u1[k]) * (us + u1[k]);", "d1 -= (us - u1[k]) * (us + u1[k]);"),
    "dissipation_sign": ("led->dissipation = (c->theta - 0.5) * dV * (dE2 + dB2);",
                         "led->dissipation = (0.5 - c->theta) * dV * (dE2 + dB2);"),
}


# mistakes planted in the Python part of the oracle (diagnostics)
PY_MUTANTS = {
    "modes_no_mirror_factor": ("cm = np.full(e.size, 2.0)", "cm = np.full(e.size, 1.0)"),
    "modes_nyquist_counted_twice": ("        cm[-1] = 1.0", "        cm[-1] = 2.0"),
    "modes_drops_cell_volume": ("return (0.5 * dV * cm * e / nx)[:nmodes]", "return (0.5 * cm * e / nx)[:nmodes]"),
    "modes_wrong_axis": ("F = np.fft.rfft(Bc, axis=1)", "F = np.fft.rfft(Bc.T, axis=1)"),
    "growth_fit_no_log": ("slope = np.polyfit(t, np.log(seg), 1)[0]", "slope = np.polyfit(t, seg, 1)[0]"),
    "growth_fit_smallest": ("if best is None or slope > best[0]:", "if best is None or slope < best[0]:"),
    "adjoint_untransposed": ("lam = np.linalg.solve(A.T, gEt)", "lam = np.linalg.solve(A, gEt)"),
    "adjoint_drops_E_extrapolation": ("gE0 = lam - (1.0 - th) / th * gE1", "gE0 = lam"),
    "adjoint_mass_pair_swapped": ("np.outer(L3[:, g], Et[:, h])", "np.outer(L3[:, h], Et[:, g])"),
    "push_adjoint_alpha_untransposed": ('gw = np.einsum("nji,jn->in", alpha, gub)',
                                        'gw = np.einsum("nij,jn->in", alpha, gub)'),
    "push_adjoint_drops_gbar": ("ggb = -beta * (ga * Bp).sum(axis=0) / gb ** 2\n        gu += _gbar_back(c, ggb, u, sv, gb, beta, gN, WN, WNx, WNy, En, gEn, gx0, gy0, a0, a1)\n",
                                "ggb = -beta * (ga * Bp).sum(axis=0) / gb ** 2\n"),
    "pred_adjoint_drops_En_path": ("    gEp = beta * gs\n", "    gEp = 0.0 * gs\n"),
    "pred_push_adjoint_gbar_of_u": ("sv = u + beta * sum(WN[k] * En[:, gN[k]] for k in range(4)) if c.gamma_pred else u\n"
                                    "        gb = np.sqrt(1.0 + (sv * sv).sum(axis=0))\n        a = beta * Bp / gb\n        n = a1 - a0",
                                    "sv = u\n"
                                    "        gb = np.sqrt(1.0 + (sv * sv).sum(axis=0))\n        a = beta * Bp / gb\n        n = a1 - a0"),
    "push_adjoint_B_on_nodes": ("gC, WC, WCx, WCy = _cic(c, x, y, 0.5)\n        Ep = sum(",
                                "gC, WC, WCx, WCy = _cic(c, x, y, 0.0)\n        Ep = sum("),
    "deposit_adjoint_drops_pair_gbar": ("                ggb -= cM * WN[k] * WN[l] * s2 / gb ** 2\n", "\n"),
    "deposit_adjoint_current_untransposed": ('gu += cJ * WN[k] / gb * np.einsum("nji,jn->in", alpha, gj)',
                                             'gu += cJ * WN[k] / gb * np.einsum("nij,jn->in", alpha, gj)'),
    "deposit_adjoint_one_sided_pairs": ("                gWn[l] += cM * WN[k] * s2 / gb\n", "\n"),
    "deposit_adjoint_w_drops_current": ("            gw0[a0:a1] += (q / dV) * WN[k] * sJ / gb\n", "\n"),
    "mode_rates_energy_slope": ("out[m] = 0.5 * np.polyfit(t, np.log(seg), 1)[0]",
                                "out[m] = np.polyfit(t, np.log(seg), 1)[0]"),
    "dispersion_fit_drops_cubic": ("g = xb * (1.0 - xb * xb)\n    A = (g @ r)", "g = xb * (1.0 - xb)\n    A = (g @ r)"),
    "deposit_adjoint_w_wrong_pair_weight": ("gw0[a0:a1] += (q * beta / dV) * WN[k] * WN[l] * s2 / gb",
                                            "gw0[a0:a1] += (q * beta / dV) * WN[k] * WN[k] * s2 / gb"),
}
# mistakes planted in the 3D oracle, caught by its own pins
MUTANTS3 = {
    "curl3_c_z_edge_wrong_row": ("sz += f[idx3(c, i + e1, j + e2, k + 1)] - f[idx3(c, i + e1, j + e2, k)];",
                                 "sz += f[idx3(c, i + e1, j + e2, k + 1)] - f[idx3(c, i + e1, j, k)];"),
    "deposit3_dk_sign": ("int dk = ((b >> 2) & 1) - ((a >> 2) & 1);", "int dk = ((a >> 2) & 1) - ((b >> 2) & 1);"),
    "weights3_z_from_y": ("(az ? f[2] : 1.0 - f[2])", "(az ? f[1] : 1.0 - f[1])"),
    "gather3_B_on_nodes": ("weights3(c, x, y, z, 0.5, cell, g, W);", "weights3(c, x, y, z, 0.0, cell, g, W);"),
    "apply_M3_z_neighbour_flipped": ("int64_t h = idx3(c, i + di, j + dj, k + dk);",
                                     "int64_t h = idx3(c, i + di, j + dj, k - dk);"),
    "push3_z_moves_with_uy": ("z[p] = wrap_pos3(z[p] + c->dt * u1[2] / g1, L[2]);",
                              "z[p] = wrap_pos3(z[p] + c->dt * u1[1] / g1, L[2]);"),
    "curl3_n_dz_uses_dy": ("sz += f[idx3(c, i + e1, j + e2, k)] - f[idx3(c, i + e1, j + e2, k - 1)];\n"
                           "                        }\n"
                           "                    d[0][comp] = sx / (4.0 * c->dx);\n"
                           "                    d[1][comp] = sy / (4.0 * c->dy);\n"
                           "                    d[2][comp] = sz / (4.0 * c->dz);",
                           "sz += f[idx3(c, i + e1, j + e2, k)] - f[idx3(c, i + e1, j + e2, k - 1)];\n"
                           "                        }\n"
                           "                    d[0][comp] = sx / (4.0 * c->dx);\n"
                           "                    d[1][comp] = sy / (4.0 * c->dy);\n"
                           "                    d[2][comp] = sz / (4.0 * c->dy);"),
}
# mistakes planted in the quadratic-shape oracle, caught by its own pins
MUTANTSQ = {
    "quad_outer_weights_swapped": ("    w[0] = 0.5 * (0.5 - d) * (0.5 - d);\n", "    w[0] = 0.5 * (0.5 + d) * (0.5 + d);\n"),
    "quad_centre_weight": ("    w[1] = 0.75 - d * d;\n", "    w[1] = 0.75 - 0.5 * d * d;\n"),
    "quadB_on_nodes": ("    weightsq(c, x, y, 0.5, g, W);\n", "    weightsq(c, x, y, 0.0, g, W);\n"),
    "quad_pair_offset_transposed": ("int o = (dj + 2) * 5 + (di + 2);\n                    double* blk",
                                    "int o = (di + 2) * 5 + (dj + 2);\n                    double* blk"),
    "quad_apply_M_wrong_neighbour": ("int64_t h = wrapq(j + dj, ny) * nx + wrapq(i + di, nx);",
                                     "int64_t h = wrapq(j - dj, ny) * nx + wrapq(i + di, nx);"),
    "quad_mass_matrix_drops_gamma": ("double cM = w[p] * q * beta / (gbar * dV);", "double cM = w[p] * q * beta / dV;"),
}
# sign mistakes in the curls that keep curl_n = curl_c^T, so the discrete
# energy identity still closes: caught by the linear tearing pin (the Harris
# sheet's force balance and its tearing dispersion), each run against that
# pin alone
MUTANTS_TEARING = {
    "tearing_curl_z_pair_sign": [("out[2 * nn + n00] = DX(Ey) - DY(Ex);", "out[2 * nn + n00] = DY(Ex) - DX(Ey);"),
                                 ("out[2 * nn + c11] = DX(By) - DY(Bx);", "out[2 * nn + c11] = DY(Bx) - DX(By);")],
    "tearing_curl_inplane_pair_sign": [("out[n00] = DY(Ez);", "out[n00] = -DY(Ez);"),
                                       ("out[nn + n00] = -DX(Ez);", "out[nn + n00] = DX(Ez);"),
                                       ("out[c11] = DY(Bz);", "out[c11] = -DY(Bz);"),
                                       ("out[nn + c11] = -DX(Bz);", "out[nn + c11] = DX(Bz);")],
}
PINS = "test_oracle_pins.py"
CASES = {**{k: ("relsim_oracle.c",) + v + (PINS,) for k, v in MUTANTS.items()},
         **{k: ("__init__.py",) + v + (PINS if not k.startswith(("mode_rates", "dispersion")) else
                                        "test_oracle_tearing.py",) for k, v in PY_MUTANTS.items()},
         **{k: ("relsim_oracle3.c",) + v + ("test_oracle3_pins.py",) for k, v in MUTANTS3.items()},
         **{k: ("relsim_oracle_q.c",) + v + ("test_oracle_q_pins.py",) for k, v in MUTANTSQ.items()},
         **{k: ("relsim_oracle.c", v, None, "test_oracle_tearing.py") for k, v in MUTANTS_TEARING.items()}}


@pytest.mark.parametrize("name", sorted(CASES))
def test_pins_catch_planted_mistake(name, tmp_path):
    fname, orig, repl, pins = CASES[name]
    src_dir = os.path.join(ROOT, "oracle")
    src = open(os.path.join(src_dir, fname)).read()
    # one replacement, or a list of (site, replacement) pairs planted together
    edits = orig if repl is None else [(orig, repl)]
    for o, rp in edits:
        assert src.count(o) == 1, f"mutation site {o!r} for {name} is not unique"
        src = src.replace(o, rp)
    dst = tmp_path / "oracle"
    shutil.copytree(src_dir, dst, ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    (dst / fname).write_text(src)
    env = dict(os.environ, RELSIM_ORACLE_MUTANT_DIR=str(tmp_path))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins)],
                       cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=600)
    # the copy really was the one under test
    assert (dst / "liboracle.so").exists()
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
