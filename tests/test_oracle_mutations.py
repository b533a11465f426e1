"""Planted mistakes in the oracle, each caught by its pins (CPU only).

Every case rewrites one spot of the oracle's source -- a flipped sign, a
dropped term or factor, a wrong index, a swapped operand -- loads the mutant in
place of the oracle (the C part rebuilt into a temporary library, a Python
function recompiled in its module), runs the pins named for that spot and
requires at least one of them to fail. A mutant that all its pins accept
would mark a part of the oracle that nothing independent checks.
"""
import inspect
import textwrap

import pytest

import oracle as O
import oracle.losses as OL
import oracle.visibility as OV
import test_oracle_autograd as PA
import test_oracle_forward_shading as PF
import test_oracle_grad as PG
import test_oracle_pins as PP
import test_oracle_visibility as PV

FD = [(PG.test_fd_scene_parameters_basic_mlp, (0,)), (PG.test_fd_scene_parameters_basic_mlp, (1,))]
AG = [(PA.test_oracle_gradients_equal_dense_autograd, (0, False)),
      (PA.test_oracle_gradients_equal_dense_autograd, (3, True))]

# (name, exact source text, replacement, pins that must catch it)
C_MUTANTS = [
    ("rotation entry sign", "R[1] = 2 * (x * y - w * z);", "R[1] = 2 * (x * y + w * z);",
     [(PP.test_covariance_is_rotation_conjugate_and_unnormalised_quaternion_ok, ())]),
    ("scale not squared", "acc += R[i * 3 + k] * s[k] * s[k] * R[j * 3 + k];", "acc += R[i * 3 + k] * s[k] * R[j * 3 + k];",
     [(PP.test_identity_quaternion_gives_diagonal_covariance, ())]),
    ("Jacobian sign", "0, fy / t[2], -fy * t[1] / (t[2] * t[2])};", "0, fy / t[2], fy * t[1] / (t[2] * t[2])};",
     [(PP.test_off_axis_projection_matches_monte_carlo, ([0.4, 0.9, 0.6], [0.004, 0.002, 0.02]))]),
    ("dilation dropped on one axis", "double a = S2[0] + dil, b = S2[1], c = S2[3] + dil;",
     "double a = S2[0] + dil, b = S2[1], c = S2[3];", [(PP.test_isotropic_gaussian_on_axis_closed_form, ())]),
    ("conic off-diagonal sign", "P[3] = -b / det;", "P[3] = b / det;",
     [(PP.test_anisotropic_alpha_follows_the_projected_covariance, ())] + FD),
    ("principal point swapped", "P[0] = fx * t[0] / t[2] + cx;", "P[0] = fx * t[0] / t[2] + cy;",
     [(PP.test_anisotropic_alpha_follows_the_projected_covariance, ())]),
    ("exponent halving dropped", "double p = 0.5 * (P[2] * dx * dx + P[4] * dy * dy) + P[3] * dx * dy;",
     "double p = (P[2] * dx * dx + P[4] * dy * dy) + P[3] * dx * dy;",
     [(PP.test_isotropic_alpha_falloff_closed_form, ()), (PP.test_anisotropic_alpha_follows_the_projected_covariance, ())]),
    ("alpha clamp dropped", "double alpha = fmin(a_max, araw);", "double alpha = araw;",
     [(PP.test_opaque_gaussian_alpha_clamps_at_alpha_max, ())]),
    ("stop rule skips instead of stopping", "if (Tn < T_min) break;", "if (Tn < T_min) continue;",
     [(PP.test_depth_order_and_stop_rule, ()), (PP.test_stop_rule_ends_the_walk, ())]),
    ("weight without transmittance", "double w = T * alpha;\n            const double* f = feat",
     "double w = alpha;\n            const double* f = feat", [(PP.test_weights_telescope_to_one_minus_T_everywhere, ())]),
    ("depth ties broken the other way", "return (i > j) - (i < j);\n}\n\n/*\n * Render",
     "return (i < j) - (i > j);\n}\n\n/*\n * Render", [(PP.test_equal_depth_ties_composite_in_storage_order, ())]),
    ("GGX normalisation dropped", "double D = a2 / (PI_D * den * den);\n    double V = 1.0 /",
     "double D = a2 / (den * den);\n    double V = 1.0 /", [(PP.test_brdf_normal_incidence_closed_form, ())]),
    ("Smith term of the wrong direction", "(ni + sqrt(a2 + (1 - a2) * ni * ni)));",
     "(no + sqrt(a2 + (1 - a2) * ni * ni)));", [(PP.test_brdf_rough_dielectric_at_sixty_degrees, ())]),
    ("shading F0 without metal weight", "F0[c] = 0.04 * (1 - mb) + bb[c] * mb;", "F0[c] = 0.04 * (1 - mb) + bb[c];",
     [(PP.test_deferred_position_and_blend_closed_forms, ())]),
    ("cosine term dropped", "Lc[c] = sb * Ls[c] + (1 - sb) * (fs[c] + fd[c]) * Li * ni;",
     "Lc[c] = sb * Ls[c] + (1 - sb) * (fs[c] + fd[c]) * Li;", [(PP.test_deferred_position_and_blend_closed_forms, ())]),
    ("coverage not applied", "out[c] = A * Lc[c];", "out[c] = Lc[c];",
     [(PP.test_deferred_position_and_blend_closed_forms, ())]),
    ("opacity gradient without G", "dg[5] += da * cb[i].G;", "dg[5] += da;", AG + FD),
    ("final-T gradient sign", "double da = -dT * T / (1 - a);", "double da = dT * T / (1 - a);", AG + FD),
    ("roughness chain factor", "dg[7] += da2 * 4 * rb * rb * rb;", "dg[7] += da2 * 2 * rb * rb * rb;", AG + FD),
    ("sigmoid derivative", "d_logit[g] += dg[5] * o * (1 - o);", "d_logit[g] += dg[5] * o;", AG + FD),
    ("quaternion gradient sign", "- y * G[6] + x * G[7]);", "+ y * G[6] + x * G[7]);", AG + FD),
    ("covariance gradient factor", "dM[i * 3 + j] = 2 * acc;", "dM[i * 3 + j] = acc;", AG + FD),
    ("depth gradient sign", "dt[2] += ddepth[g];", "dt[2] -= ddepth[g];", AG + FD),
    ("pixel rectangle too small", "double ex = sqrt(2.0 * L * a) * (1.0 + 1e-9);", "double ex = sqrt(L * a) * (1.0 + 1e-9);",
     [(PP.test_brute_force_equals_tiled_bitwise_and_tile_size_independent, ())]),
    ("mean gradient uses the wrong conic entry", "dg[0] += dp * (P[2] * dx + P[3] * dy);",
     "dg[0] += dp * (P[2] * dx + P[4] * dy);", AG + FD),
    ("per-Gaussian shading upstream sign", "dF[c] = dimg[3 * (size_t)q + c];", "dF[c] = -dimg[3 * (size_t)q + c];",
     [(PF.test_fd_of_the_per_gaussian_shaded_render, (0,))]),
    ("Smith derivative sign", "dni += dLi * (1 + (1 - a2) * ni / si);", "dni += dLi * (1 - (1 - a2) * ni / si);", AG + FD),
    ("SSS blend gradient term dropped", "dg[9] += gL[c] * (Ls[c] - (fs[c] + fd[c]) * Li * ni);",
     "dg[9] += gL[c] * Ls[c];", AG + FD),
    ("depth gradient of the deferred position", "dg[0] += dot3(dXc, ray);", "dg[0] -= dot3(dXc, ray);", AG + FD),
    ("projected-mean gradient without focal length", "dt[0] += dg[0] * fx / tz;", "dt[0] += dg[0] / tz;", AG + FD),
    ("alpha gradient of the later sum", "da += dF[c] * (Ti * f[c] - S[c] / (1 - a));",
     "da += dF[c] * (Ti * f[c] - S[c]);", AG + FD),
    ("bin order by item reversed", "return (x->item > y->item) - (x->item < y->item);",
     "return (x->item < y->item) - (x->item > y->item);", [(PP.test_bin_sort_equals_python_stable_sort, ())]),
]

# (module, function, exact source text, replacement, pins)
PY_MUTANTS = [
    (OV, "sh_basis", "_C3b * x * y * z", "_C3b * x * y * y", [(PV.test_sh_basis_equals_scipy_real_harmonics, ())]),
    (OV, "sh_basis_grad", "(zero, zero, _C2b * 6 * z)", "(zero, zero, _C2b * 3 * z)",
     [(PV.test_sh_gradient_equals_finite_differences, ())]),
    (OV, "vis_sh_backward", 'dV = (dw - np.einsum("nc,nc->n", w, dw)[:, None] * w) / r[:, None]', "dV = dw / r[:, None]",
     [(PV.test_vis_sh_backward_equals_finite_differences, ())]),
    (OV, "vis_sh_backward", "return dc, -dV", "return dc, dV", [(PV.test_vis_sh_backward_equals_finite_differences, ())]),
    (OV, "trace_visibility", "take = (t > 0.0) & (t < tL) & (a >= alpha_min)", "take = (t > 0.0) & (a >= alpha_min)",
     [(PV.test_trace_closed_forms, ())]),
    (OV, "trace_visibility", "q = np.einsum(\"ni,ni->n\", op, op) - od * od / dd",
     "q = np.einsum(\"ni,ni->n\", op, op) + od * od / dd", [(PV.test_trace_peak_response_equals_dense_ray_sampling, ())]),
    (OV, "vis_loss", "lam * np.sign(d) / d.size", "lam * np.sign(d)", [(PV.test_vis_loss_gradient, ())]),
    (OV, "vis_sh", "np.clip(u, 0.0, 1.0)", "np.clip(u, 0.0, 2.0)",
     [(PV.test_vis_sh_equals_clamped_expansion_in_scipy_harmonics, ())]),
    (OV, "rotation", "np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1)",
     "np.stack([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z + w * y)], -1)",
     [(PV.test_rotation_scale_reproduce_the_covariance, ())]),
    (OL, "ssim_map", "(sxx + syy + SSIM_C2)", "(sxx + syy + SSIM_C1)", [(PP.test_ssim_equals_brute_force_window_sums, ())]),
    (O, "input_grads", "dmu = dX[:, 0:3] + back_unit(wo, lo, dX[:, 3:6]) + back_unit(wi, li, dX[:, 6:9])",
     "dmu = dX[:, 0:3] + back_unit(wi, li, dX[:, 3:6]) + back_unit(wi, li, dX[:, 6:9])", FD),
    (OL, "gaussian_window", "return w / w.sum()", "return w", [(PP.test_ssim_closed_forms, ())]),
    (OL, "ssim_map", "sxy = window_mean(x * y) - mx * my", "sxy = window_mean(x * y)",
     [(PP.test_ssim_equals_brute_force_window_sums, ())]),
    (OL, "ssim", "d_sxy = dS_dA2 * 2", "d_sxy = dS_dA2",
     [(PP.test_ssim_and_image_loss_gradients_equal_conv2d_autograd, ()),
      (PP.test_image_and_incident_loss_gradients_match_finite_differences, ())]),
    (OL, "ssim", "g = window_mean(d_mx) + 2 * x * window_mean(d_sxx) + y * window_mean(d_sxy)",
     "g = window_mean(d_mx) + x * window_mean(d_sxx) + y * window_mean(d_sxy)",
     [(PP.test_ssim_and_image_loss_gradients_equal_conv2d_autograd, ())]),
    (OL, "image_loss", "- lam * gs", "+ lam * gs", [(PP.test_image_and_incident_loss_gradients_match_finite_differences, ())]),
    (OL, "incident_loss", "return loss, s * (L_in < 1.0), -s", "return loss, s, -s",
     [(PP.test_image_and_incident_loss_gradients_match_finite_differences, ())]),
    (O, "bf16_round", "np.rint(np.ldexp(m, 8))", "np.floor(np.ldexp(m, 8))", [(PP.test_bf16_rounding_matches_torch_bfloat16, ())]),
    (O, "mlp_forward", "h = rnd(np.maximum(z, 0.0))", "h = rnd(np.maximum(z, 0.01 * z))",
     [(PP.test_mlp_matches_torch_linear_chain_fp64, ())]),
    (O, "mlp_inputs", "feats.append(np.cos((2.0 ** k) * math.pi * mu))\n    X = np.concatenate(feats + [mu, wo, wi,",
     "feats.append(np.cos((2.0 ** k) * mu))\n    X = np.concatenate(feats + [mu, wo, wi,",
     [(PP.test_input_encoding_gradients_match_autograd, ()), (PG.test_fd_pe6_mlp_inputs_and_weights, ())]),
    (O, "input_grads", "dmu += dX[:, 48:49] * (-wi)", "dmu += dX[:, 48:49] * wi",
     [(PP.test_input_encoding_gradients_match_autograd, ()), (PG.test_fd_pe6_mlp_inputs_and_weights, ())]),
    (O, "mlp_inputs", "np.exp(log_s), wi, wo", "log_s, wi, wo",
     [(PP.test_paper_input_encoding_and_gradients_match_autograd, ())]),
    (O, "_paper_backward", "dzh = rnd((dzi @ W[4]) * _dlrelu(hid))", "dzh = rnd(dzi @ W[4])",
     [(PP.test_paper_mlp_matches_torch_modules_fp64, ()), (PG.test_fd_paper_mlp_inputs_and_weights, ())]),
    (O, "render_pair", "scene.normal, scene.base, scene.rough[:, None],", "scene.base, scene.normal, scene.rough[:, None],",
     [(PP.test_two_coincident_gaussians_closed_form, ())]),
    (O, "render_pair", 'g["metal"] += dfeat[:, 8]', 'g["metal"] += dfeat[:, 7]', FD),
    (O, "gaussian_colors", "F0 = 0.04 * (1 - m[:, None]) + b * m[:, None]", "F0 = 0.04 + b * m[:, None]",
     [(PF.test_colour_equals_deferred_shading_at_the_mean, ())]),
]


def _caught(pins):
    """Name of the first pin that fails (AssertionError), else None."""
    for fn, args in pins:
        try:
            fn(*args)
        except AssertionError:
            return fn.__name__
    return None


@pytest.fixture(scope="module")
def oracle_src():
    with open(O._build.SRC) as fh:
        return fh.read()


@pytest.mark.parametrize("name,old,new,pins", C_MUTANTS, ids=[m[0] for m in C_MUTANTS])
def test_c_mutant_is_caught(name, old, new, pins, oracle_src, tmp_path, monkeypatch):
    assert oracle_src.count(old) == 1, f"mutation site not unique: {old!r}"
    assert _caught(pins) is None, "the pins fail on the unmutated oracle"
    src = tmp_path / "mutant.c"
    src.write_text(oracle_src.replace(old, new))
    so = str(tmp_path / "libmutant.so")
    O._build.compile_library(str(src), so)
    monkeypatch.setattr(O._build, "build", lambda force=False: so)
    monkeypatch.setattr(O, "_LIB", None)
    assert _caught(pins) is not None, f"mutant '{name}' passes every pin named for it"


def _mutate(module, fname, old, new):
    func = getattr(module, fname)
    code = textwrap.dedent(inspect.getsource(func))
    assert code.count(old) == 1, f"mutation site not unique: {old!r}"
    scope = dict(func.__globals__)
    exec(compile(code.replace(old, new), f"<mutant of {fname}>", "exec"), scope)
    return scope[fname]


@pytest.mark.parametrize("module,fname,old,new,pins", PY_MUTANTS,
                         ids=[f"{m[1]}-{k}" for k, m in enumerate(PY_MUTANTS)])
def test_python_mutant_is_caught(module, fname, old, new, pins, monkeypatch):
    assert _caught(pins) is None, "the pins fail on the unmutated oracle"
    original = getattr(module, fname)
    mutant = _mutate(module, fname, old, new)
    monkeypatch.setattr(module, fname, mutant)
    if getattr(O, fname, None) is original:          # re-exported by the oracle package
        monkeypatch.setattr(O, fname, mutant)
    assert _caught(pins) is not None, f"mutant of {fname} passes every pin named for it"
