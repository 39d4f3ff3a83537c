"""Plant plausible mistakes in copies of the oracle source and check that the
pins catch every one of them (CPU only; nothing is planted in the real oracle)."""
import os
import tempfile

import pytest

import oracle
import oracle_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "ags_oracle.c")

# (name, original text, planted text, pins expected to catch it)
MUTANTS = [
    ("dropped_lowpass", "cc = jaddc(S2[3], 0.3);", "cc = S2[3];",
     ["pin_isotropic_on_axis"]),
    ("quat_sign", "Rq[1] = jscale(jsub(jmul(x, y), jmul(w, z)), 2.0);",
     "Rq[1] = jscale(jadd(jmul(x, y), jmul(w, z)), 2.0);", ["pin_rotation_conventions"]),
    ("camera_rotation_transposed", "acc = jadd(acc, jscale(J[a * 3 + k], cam->R[k * 3 + b]));",
     "acc = jadd(acc, jscale(J[a * 3 + k], cam->R[b * 3 + k]));", ["pin_rotation_conventions"]),
    ("dropped_offaxis_jacobian", "J[2] = jscale(jmul(tx, iz2), -cam->fx);", "J[2] = jc(0.0);",
     ["pin_off_axis_jacobian"]),
    ("no_frustum_clamp", "if (txtz.v > limx) { tx = jscale(t[2], limx); fclamp |= 8; }",
     "if (0) { tx = jscale(t[2], limx); fclamp |= 8; }", ["pin_off_axis_jacobian"]),
    ("eq10_det_not_sqrt", "double sd = sqrt(det.v);", "double sd = det.v;",
     ["pin_isotropic_on_axis", "pin_eq9_quadrature"]),
    ("eq10_missing_2pi", "th = par->K / (tup * 2.0 * M_PI * sd) + par->tau;",
     "th = par->K / (tup * sd) + par->tau;", ["pin_isotropic_on_axis", "pin_eq9_quadrature"]),
    ("radius_not_clamped_at_3", "rarg = sqrt(lam1) * fmin(3.0, sqrt(2.0 * log(opac.v / th)));",
     "rarg = sqrt(lam1) * sqrt(2.0 * log(opac.v / th));", ["pin_invariants"]),
    ("th_cull_inverted", "if (th > opac.v) { irec[I_EDGE] = edge; irec[I_CULL] = CULL_TH; return CULL_TH; }",
     "if (th < opac.v) { irec[I_EDGE] = edge; irec[I_CULL] = CULL_TH; return CULL_TH; }",
     ["pin_isotropic_on_axis"]),
    ("lut_bin_off_by_one", "int bin = (int)floor(fb);", "int bin = (int)floor(fb) + 1;",
     ["pin_isotropic_on_axis"]),
    ("colour_after_transmittance_update", "col[0] += g[F_R] * alpha * T;", "col[0] += g[F_R] * alpha * test_T;",
     ["pin_isotropic_on_axis"]),
    ("no_condon_shortley", "double s = sqrt(2.0) * K * ((m & 1) ? -1.0 : 1.0);", "double s = sqrt(2.0) * K;",
     ["pin_sh_basis"]),
    ("sh_cos_sin_swapped", "Y[l * l + l + m] = jscale(jmul(pz, re), s);", "Y[l * l + l + m] = jscale(jmul(pz, im), s);",
     ["pin_sh_basis"]),
    ("colour_no_offset", "jet acc = jc(0.5);", "jet acc = jc(0.0);", ["pin_isotropic_on_axis", "pin_sh_colour"]),
    ("depth_sort_descending", "if (x->depth < y->depth) return -1;", "if (x->depth < y->depth) return 1;",
     ["pin_ideal_render", "pin_max_T"]),
    ("rect_floor_not_ceil", "double plo = ceil(lo), phi = floor(hi);", "double plo = floor(lo), phi = floor(hi);",
     ["pin_rect_enumeration"]),
    ("max_T_after_update", "T = test_T;\n    last = (int32_t)(k + 1);",
     "T = test_T;\n    if (maxT) maxT[list[k]] = T;\n    last = (int32_t)(k + 1);", ["pin_max_T"]),
    ("backward_missing_behind_colour", "dLda += g[ch] * Ti[j] * (c[ch] - R[ch]);",
     "dLda += g[ch] * Ti[j] * c[ch];", ["pin_backward_fd"]),
    ("backward_mean_sign", "atomic_add_double(&G[who[j] * 9 + 0], dLdp * (-(f[F_A] * dx + f[F_B] * dy)));",
     "atomic_add_double(&G[who[j] * 9 + 0], dLdp * (f[F_A] * dx + f[F_B] * dy));", ["pin_backward_fd"]),
    ("backward_ignores_alpha_clamp", "if (clampa[j]) continue;", "", ["pin_backward_fd"]),
    ("ellipse_level_missing_2", "double Q = 2.0 * log(opac.v / th);", "double Q = log(opac.v / th);",
     ["pin_ellipse_tiles", "pin_ellipse_lossless_plain"]),
    ("ellipse_cross_term_sign", "best = fmin(best, A * x * x + 2.0 * B * x * y + C * y * y);\n    y = ys[k];",
     "best = fmin(best, A * x * x - 2.0 * B * x * y + C * y * y);\n    y = ys[k];",
     ["pin_ellipse_tiles", "pin_ellipse_lossless_plain"]),
    ("ellipse_tile_unclipped", "xh = fmin(OC_TILE * tx + OC_TILE - 1, width - 1) - g[F_U];",
     "xh = OC_TILE * tx + OC_TILE - 1 - g[F_U];", ["pin_ellipse_tiles"]),
    ("ps_after_transmittance_update", "double c = alpha * T;\n          if (alpha < level[i]) {",
     "double c = alpha * test_T;\n          if (alpha < level[i]) {",
     ["pin_peripheral_two_layers", "pin_peripheral_closed_form"]),
    ("ps_ignores_level", "if (alpha < level[i]) {", "if (alpha >= par->tau) {",
     ["pin_peripheral_two_layers", "pin_peripheral_closed_form", "pin_peripheral_invariants"]),
    ("skip_ranked_by_image_transmittance", "double c = rule == 0 ? alpha * T : weight[list[k]] * alpha;",
     "double c = rule == 0 ? alpha * Ts : weight[list[k]] * alpha;", ["pin_skip_render"]),
    ("skipped_blend_still_occludes", "            Ts *= 1.0 - alpha;\n          }\n",
     "          }\n          Ts *= 1.0 - alpha;\n", ["pin_skip_render"]),
    # edge classes: each band widened tenfold, narrowed to nothing, or missing a term
    ("edge_near_x10", "if (near_edge(t[2].v, cam->near_z, eps, fmax(fabs(t[2].v), cam->near_z))) edge |= EDGE_NEAR;",
     "if (near_edge(t[2].v, cam->near_z, 10 * eps, fmax(fabs(t[2].v), cam->near_z))) edge |= EDGE_NEAR;",
     ["pin_edge_near_plane"]),
    ("edge_near_camera_magnitude", "if (near_edge(t[2].v, cam->near_z, eps, fmax(fabs(t[2].v), cam->near_z))) edge |= EDGE_NEAR;",
     "if (near_edge(t[2].v, cam->near_z, eps, fmax(fabs(t[2].v) + fabs(cam->t[2]), cam->near_z))) edge |= EDGE_NEAR;",
     ["pin_edge_near_plane"]),
    ("edge_rect_magnitude_sum", "double uscale = fabs(cam->fx * t[0].v / t[2].v) + fabs(cam->cx);",
     "double uscale = fabs(cam->fx * t[0].v / t[2].v) + fabs(cam->cx) + cam->fx * fabs(cam->t[0]) / t[2].v;",
     ["pin_edge_rect"]),
    ("edge_det_x10", "if (near_edge(det.v, 0.0, eps, fabs(ca.v * cc.v) + cb.v * cb.v)) edge |= EDGE_DET;",
     "if (near_edge(det.v, 0.0, 10 * eps, fabs(ca.v * cc.v) + cb.v * cb.v)) edge |= EDGE_DET;",
     ["pin_edge_det_guard"]),
    ("edge_th_x10", "if (near_edge(th, opac.v, eps, fmax(th, opac.v))) edge |= EDGE_TH;",
     "if (near_edge(th, opac.v, 10 * eps, fmax(th, opac.v))) edge |= EDGE_TH;", ["pin_edge_th_vs_opacity"]),
    ("edge_ceil_x10", "rarg_hi = 3.0 * sqrt(lam1 * (1 + eps));", "rarg_hi = 3.0 * sqrt(lam1 * (1 + 10 * eps));",
     ["pin_edge_radius_ceil"]),
    ("edge_ceil_dropped", "if ((int)ceil(rarg_hi) != (int)ceil(rarg_lo)) edge |= EDGE_CEIL;", "",
     ["pin_edge_radius_ceil"]),
    ("edge_rect_no_slack", "double su = eps * uscale, sv = eps * vscale;", "double su = 0.0, sv = 0.0;",
     ["pin_edge_rect"]),
    ("edge_rect_x10", "double su = eps * uscale, sv = eps * vscale;",
     "double su = 10 * eps * uscale, sv = 10 * eps * vscale;", ["pin_edge_rect"]),
    ("edge_lut_x10", "near_edge(fb, fr, eps, fmax(fabs(fb), 1.0))", "near_edge(fb, fr, 10 * eps, fmax(fabs(fb), 1.0))",
     ["pin_edge_lut_bin"]),
    ("edge_lut_open_end_flagged", "if (fr >= 1.0 && fr <= par->lut_bins - 1 &&", "if (fr >= 1.0 && fr <= par->lut_bins &&",
     ["pin_edge_lut_bin"]),
    ("edge_ellipse_x10", "double tol = eps * fmax(Q, 1.0) +", "double tol = 10 * eps * fmax(Q, 1.0) +",
     ["pin_edge_ellipse"]),
    ("edge_ellipse_no_size_term", "sqrt((A.v + C.v) * fmax(fmax(Q, m), 0.0)) + 2e-6 * S;",
     "sqrt((A.v + C.v) * fmax(fmax(Q, m), 0.0));", ["pin_edge_ellipse"]),
    ("edge_ellipse_no_position_term", "double tol = eps * fmax(Q, 1.0) + 2.0 * par->pos_err *",
     "double tol = eps * fmax(Q, 1.0) + 0.0 * par->pos_err *", ["pin_edge_ellipse"]),
    ("edge_budget_alpha_tau_dropped",
     "if (araw > 0.0 && fabs(log(araw / par->tau)) <= tol) budget += 2.0 * par->tau * T * cmax;", "",
     ["pin_edge_pixel_budget"]),
    ("edge_budget_x10", "\n    double tol = par->edge_rel + par->pos_err * gl;\n",
     "\n    double tol = 10 * par->edge_rel + par->pos_err * gl;\n", ["pin_edge_pixel_budget"]),
    ("edge_budget_no_gradient_term", "\n    double tol = par->edge_rel + par->pos_err * gl;\n",
     "\n    double tol = par->edge_rel;\n", ["pin_edge_pixel_budget"]),
    ("edge_budget_p_term_dropped",
     "if (fabs(p) <= par->edge_rel && g[F_OPAC] >= par->tau) budget += 2.0 * g[F_OPAC] * T * cmax;", "",
     ["pin_edge_pixel_budget"]),
    ("eval_count_off_by_one", "if (test_T < par->t_min) { nev = (int32_t)(k + 1); break; }",
     "if (test_T < par->t_min) { nev = (int32_t)k; break; }", ["pin_eval_count"]),
    ("gedge_colour_dropped", "if (fabs(acc.v) <= eps * mag) irec[I_GEDGE] |= GEDGE_COLOUR;", "",
     ["pin_gradient_edges"]),
    ("gedge_frustum_x10", "if (near_edge(fabs(txtz.v), limx, eps, limx) || near_edge(fabs(tytz.v), limy, eps, limy))",
     "if (near_edge(fabs(txtz.v), limx, 10 * eps, limx) || near_edge(fabs(tytz.v), limy, eps, limy))",
     ["pin_gradient_edges"]),
    ("gedge_stop_dropped", "stopd = fabs(log(tt / par->t_min)) <=", "stopd = 0 * fabs(log(tt / par->t_min)) >",
     ["pin_gradient_edges"]),
    ("gbudget_no_colour_behind_term", "(rho * fabs(c[ch] - R[ch]) + dR)", "(rho * fabs(c[ch] - R[ch]))",
     ["pin_gradient_edges"]),
    ("gbudget_flip_not_recorded", "                  nflip++;\n", "",
     ["pin_gradient_edges"]),
    ("gbudget_front_behind_swapped", "if (fbl[q] ? fpos[q] < j : fpos[q] <= j) rho += frho[q];",
     "if (fpos[q] > j) rho += frho[q];", ["pin_gradient_edges"]),
]


@pytest.mark.parametrize("mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(mut):
    name, old, new, pins = mut
    src = open(SRC).read()
    assert src.count(old) == 1, name
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, name + ".c")
        open(path, "w").write(src.replace(old, new))
        lib = oracle.compile_library(path, os.path.join(d, "lib" + name + ".so"))
        orc = oracle.Oracle(lib)
        caught = []
        for pname in pins:
            pin = getattr(oracle_pins, pname)
            try:
                if pname == "pin_backward_fd":
                    pin(orc, n_check=120)
                else:
                    pin(orc)
            except AssertionError:
                caught.append(pname)
        assert caught, "planted mistake %s passed every pin" % name
