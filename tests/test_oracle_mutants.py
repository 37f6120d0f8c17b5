"""Planted mistakes in the FP64 oracle must fail its pins (no GPU).

Each case copies ``oracle/upslam_oracle.c``, plants one plausible mistake (a
flipped sign, a dropped term, a transposed operand, a wrong index or gate),
compiles the copy with the oracle's own flags and runs the pin tests against it
in a child process (``UPSLAM_ORACLE_LIB``).  The Python parts of the oracle
(a-trous smoothing, pose network, downsampling, the grid-search and consistency
glue) are mutated the same way in a copy of the source tree.  The pins pass on the real oracle; a
case passes here only when some pin fails on the broken copy.  This shows that
the pins are tied to the paper and the mathematics tightly enough to catch
mistakes of these kinds anywhere in the oracle.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "upslam_oracle.c")

PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_consistency_pins.py", "tests/test_oracle_grid_pins.py",
        "tests/test_oracle_irls_pins.py"]
# the two slow pins (a 10 s tracking run and a 7 s per-pixel re-assembly) are left to the main suite
SLOW = ["tests/test_oracle_pins.py::test_sequence_tracks_tunnel",
        "tests/test_oracle_irls_pins.py::test_weighted_normal_equations_match_per_pixel_definition"]

# each child runs single-threaded; the children run side by side
ONE_THREAD = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}

# (name, text in upslam_oracle.c, planted replacement)
MUTANTS = [
    # a1: binning (Sec. III-A)
    ("atan2_reflection_sign", "    if (x < 0.0f) a = ORC_PI_F - a;", "    if (x < 0.0f) a = ORC_PI_F + a;"),
    ("atan2_octant_sign", "    if (ay > ax) a = ORC_HALF_PI_F - a;", "    if (ay > ax) a = ORC_HALF_PI_F + a;"),
    ("elevation_sign", "    float fr = (pp->el_top - el) * pp->s_el;", "    float fr = (pp->el_top + el) * pp->s_el;"),
    ("azimuth_mirrored", "    float fc = (ORC_PI_F - az) * pp->s_az;", "    float fc = (ORC_PI_F + az) * pp->s_az;"),
    ("inverse_not_transposed",
     "    *qx = (r[0] * dx + r[4] * dy) + r[8] * dz;\n"
     "    *qy = (r[1] * dx + r[5] * dy) + r[9] * dz;\n"
     "    *qz = (r[2] * dx + r[6] * dy) + r[10] * dz;",
     "    *qx = (r[0] * dx + r[1] * dy) + r[2] * dz;\n"
     "    *qy = (r[4] * dx + r[5] * dy) + r[6] * dz;\n"
     "    *qz = (r[8] * dx + r[9] * dy) + r[10] * dz;"),
    ("zbuffer_first_come",
     "        int64_t k = (int64_t)v * pp->cols + u;\n        if (key < best[k]) best[k] = key;",
     "        int64_t k = (int64_t)v * pp->cols + u;\n        if (best[k] == UINT64_MAX) best[k] = key;"),
    # a2: normals (Sec. III-A)
    ("normal_cross_component",
     "double n[3] = { a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0] };",
     "double n[3] = { a[1] * b[2] - a[2] * b[1], a[0] * b[2] - a[2] * b[0], a[0] * b[1] - a[1] * b[0] };"),
    ("normal_orientation",
     "double s = (n[0] * P[0] + n[1] * P[1] + n[2] * P[2]) > 0.0 ? -1.0 / nn : 1.0 / nn;",
     "double s = (n[0] * P[0] + n[1] * P[1] + n[2] * P[2]) < 0.0 ? -1.0 / nn : 1.0 / nn;"),
    ("normal_jump_absolute_term", "    float lim = np->jump_rel * d + np->jump_abs;", "    float lim = np->jump_rel * d;"),
    # SE(3) and the 6x6 solve
    ("se3_rotation_transposed", "        R[i] = I + A * W[i] + B * W2[i];", "        R[i] = I - A * W[i] + B * W2[i];"),
    ("se3_v_coefficient", "        V[i] = I + B * W[i] + C * W2[i];", "        V[i] = I + A * W[i] + C * W2[i];"),
    ("solve_back_substitution_index", "        for (int k = i + 1; k < 6; ++k) s -= L[6 * k + i] * x[k];",
     "        for (int k = i + 1; k < 6; ++k) s -= L[6 * i + k] * x[k];"),
    # a3: Eq. 1, filter Omega, Gauss-Newton (Sec. III-B)
    ("jacobian_rotation_sign", "    J[0] = p[1] * n[2] - p[2] * n[1];", "    J[0] = p[2] * n[1] - p[1] * n[2];"),
    ("residual_dropped_term", "    *r_out = e[0] * n[0] + e[1] * n[1] + e[2] * n[2];", "    *r_out = e[0] * n[0] + e[1] * n[1];"),
    ("omega_normal_gate_dropped", "    if (!(cs >= (double)ip->cos_theta_max)) return 0;", "    (void)cs;"),
    ("omega_distance_gate_dropped", "    if (!(dist <= (double)ip->d_max)) return 0;", "    (void)dist;"),
    ("gauss_newton_rhs_sign", "    for (int i = 0; i < 6; ++i) nb[i] = -st->b[i];", "    for (int i = 0; i < 6; ++i) nb[i] = st->b[i];"),
    ("irls_weight_constant", "                w = 1.0 / (ar > (double)ip->loss_delta ? ar : (double)ip->loss_delta);",
     "                w = 1.0 / (double)ip->loss_delta;"),
    ("normal_equations_unweighted", "                for (int c = a; c < 6; ++c) st->A[p++] += w * J[a] * J[c];",
     "                for (int c = a; c < 6; ++c) st->A[p++] += J[a] * J[c];"),
    # a4: keyframe update (Sec. III-C)
    ("fusion_weights_swapped", "            kf_depth[k] = (w * kf_depth[k] + dm) / (w + 1.0);",
     "            kf_depth[k] = (kf_depth[k] + w * dm) / (w + 1.0);"),
    ("fusion_count_unsaturated", "            kf_w[k] = (w + 1.0 < (double)fp->w_max) ? w + 1.0 : (double)fp->w_max;",
     "            kf_w[k] = w + 1.0;"),
    ("fusion_distance_gate_dropped",
     "            if (!(sqrt(e0 * e0 + e1 * e1 + e2 * e2) <= (double)fp->d_max)) continue;",
     "            (void)e0; (void)e1; (void)e2;"),
    # motion prior (Sec. IV-F footnote)
    ("prior_product_order", "        pose_mul34(T_prev, M, t);", "        pose_mul34(M, T_prev, t);"),
    ("prior_not_orthonormalised", "        pose_mul34(T_prev, M, t);\n        orc_orthonormalise_rows(t);",
     "        pose_mul34(T_prev, M, t);"),
    ("prior_translation_dropped", "            if (j == 3) s += A[4 * i + 3];", "            (void)0;"),
    ("motion_inverse_translation_sign",
     "        inv[4 * i + 3] = -(T_prev[i] * T_prev[3] + T_prev[4 + i] * T_prev[7] + T_prev[8 + i] * T_prev[11]);",
     "        inv[4 * i + 3] = (T_prev[i] * T_prev[3] + T_prev[4 + i] * T_prev[7] + T_prev[8 + i] * T_prev[11]);"),
    ("motion_inverse_not_transposed", "        for (int j = 0; j < 3; ++j) inv[4 * i + j] = T_prev[4 * j + i];",
     "        for (int j = 0; j < 3; ++j) inv[4 * i + j] = T_prev[4 * i + j];"),
    ("gram_schmidt_projection_dropped", "    for (int i = 0; i < 3; ++i) r1[i] -= d * r0[i];", "    (void)d;"),
    ("gram_schmidt_third_row_reversed", "    r2[0] = r0[1] * r1[2] - r0[2] * r1[1];\n    r2[1] = r0[2] * r1[0] - r0[0] * r1[2];\n    r2[2] = r0[0] * r1[1] - r0[1] * r1[0];",
     "    r2[0] = r0[2] * r1[1] - r0[1] * r1[2];\n    r2[1] = r0[0] * r1[2] - r0[2] * r1[0];\n    r2[2] = r0[1] * r1[0] - r0[0] * r1[1];"),
    ("hole_fill_farthest",
     "        if (!was_empty[k]) continue;\n        uint32_t rb;\n        memcpy(&rb, &r, 4);\n"
     "        uint64_t key = ((uint64_t)rb << 32) | (uint32_t)j;\n        if (key < best[k]) best[k] = key;",
     "        if (!was_empty[k]) continue;\n        uint32_t rb;\n        memcpy(&rb, &r, 4);\n"
     "        uint64_t key = ((uint64_t)rb << 32) | (uint32_t)j;\n"
     "        if (best[k] == UINT64_MAX || key > best[k]) best[k] = key;"),
    # keyframe mutual consistency (Sec. III-C) and the fixed-order inverse
    ("consistency_test_inverted", "                    if (dn > 0.0f && !(dn > lim)) {",
     "                    if (dn > 0.0f && (dn > lim)) {"),
    ("pose_inverse_sign", "        out[4 * i + 3] = -((T[i] * T[3] + T[4 + i] * T[7]) + T[8 + i] * T[11]);",
     "        out[4 * i + 3] = ((T[i] * T[3] + T[4 + i] * T[7]) + T[8 + i] * T[11]);"),
    # second batch: thresholds, counts and the less-travelled branches
    ("se3_c_coefficient_power", "C = (th - sin(th)) / (th2 * th);", "C = (th - sin(th)) / th2;"),
    ("solve_pivot_threshold_dropped", "if (!(s > pivot_eps * dmax)) return 3;", "if (!(s > 0.0)) return 3;"),
    ("range_minimum_dropped", "if (!(r >= pp->r_min && r <= pp->r_max)) return 0;", "if (!(r <= pp->r_max)) return 0;"),
    ("normal_degeneracy_test_dropped", "if (!(nn >= (double)np->min_cross * na * nb) || nn == 0.0) continue;",
     "if (nn == 0.0) continue;"),
    ("keyframe_normal_validity_dropped",
     "if (!(nk[0] * nk[0] + nk[1] * nk[1] + nk[2] * nk[2] > 0.25f)) return 0;", "(void)nk;"),
    ("sse_not_squared", "st->sse += w * r * r;", "st->sse += w * r;"),
    ("valid_counts_every_pixel", "st->valid += sp4[4 * j + 3] != 0.0f;", "st->valid += 1;"),
    ("convergence_either_norm", "st->converged = (wn < ip->eps_rot && vn < ip->eps_trans) ? 1 : 0;",
     "st->converged = (wn < ip->eps_rot || vn < ip->eps_trans) ? 1 : 0;"),
    ("fusion_normal_weights_swapped", "double nn[3] = { w * n[0] + Rm[0], w * n[1] + Rm[1], w * n[2] + Rm[2] };",
     "double nn[3] = { n[0] + w * Rm[0], n[1] + w * Rm[1], n[2] + w * Rm[2] };"),
    ("fusion_range_in_sweep_frame", "double dm = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);",
     "double dm = sqrt((double)P[0] * P[0] + (double)P[1] * P[1] + (double)P[2] * P[2]);"),
    ("consistency_centre_row_only", "for (int dv = -1; dv <= 1 && seen_through; ++dv) {",
     "for (int dv = 0; dv <= 0 && seen_through; ++dv) {"),
    ("consistency_absolute_margin_dropped", "float lim = (rel * r + abs_m) + r;", "float lim = rel * r + r;"),
    ("irls_weight_sum", "                w = 1.0 / (ar > (double)ip->loss_delta ? ar : (double)ip->loss_delta);",
     "                w = 1.0 / (ar + (double)ip->loss_delta);"),
]


# (name, file under oracle/, text, planted replacement): the Python parts of the oracle
PY_PINS = ["tests/test_oracle_atrous_pins.py", "tests/test_oracle_cnn_pins.py"]
PY_MUTANTS = [
    # a-trous smoothing (Sec. III-A)
    ("atrous_linear_dilation", "atrous.py", "        s = 1 << lev", "        s = lev + 1"),
    ("atrous_tap_set", "atrous.py", "TAPS = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0",
     "TAPS = np.array([1.0, 2.0, 6.0, 2.0, 1.0]) / 12.0"),
    ("atrous_rows_wrap", "atrous.py", "    out = np.full_like(A, fill)\n    rolled = np.roll(A, -dc, axis=1)",
     "    return np.roll(np.roll(A, -dc, axis=1), -dr, axis=0)\n    rolled = np.roll(A, -dc, axis=1)"),
    ("atrous_plane_distance_sign", "atrous.py", "dpl = np.sum(N * (Pq - P), axis=-1)",
     "dpl = np.sum(N * (Pq + P), axis=-1)"),
    ("atrous_no_normalisation", "atrous.py",
     "        N = np.where(V[..., None], acc / np.where(norm > 0, norm, 1.0)[..., None], 0.0)",
     "        N = np.where(V[..., None], acc, 0.0)"),
    ("atrous_normal_weight_unscaled", "atrous.py", "np.exp(-dn2 * inv_sn2)", "np.exp(-dn2)"),
    # pose network (no counterpart in the paper)
    ("cnn_im2col_taps_swapped", "cnn.py", "cols[:, :, :, ky, kx, :] = xp[:, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2, :]",
     "cols[:, :, :, ky, kx, :] = xp[:, kx:kx + 2 * Ho:2, ky:ky + 2 * Wo:2, :]"),
    ("cnn_col2im_taps_swapped", "cnn.py", "+= d[:, :, :, ky, kx, :]", "+= d[:, :, :, kx, ky, :]"),
    ("cnn_relu_mask_dropped", "cnn.py", "        dy = da.reshape(-1, co) * (cache[f\"pre{l}\"] > 0)",
     "        dy = da.reshape(-1, co)"),
    ("cnn_pool_scale_dropped", "cnn.py", "dg[:, None, None, :] / (H * W)", "dg[:, None, None, :]"),
    ("cnn_loss_gradient_factor", "cnn.py", "    return L, 2.0 * weights * diff / B", "    return L, weights * diff / B"),
    ("cnn_bias_gradient_mean", "cnn.py", "\"bf\": dout.sum(axis=0)", "\"bf\": dout.mean(axis=0)"),
    ("adam_no_bias_correction", "cnn.py", "        mh = m[k] / (1 - b1 ** t)", "        mh = m[k]"),
    ("adam_no_second_moment_correction", "cnn.py", "        vh = v[k] / (1 - b2 ** t)", "        vh = v[k]"),
    ("adam_step_sign", "cnn.py", "        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)",
     "        p[k] = p[k] + lr * mh / (np.sqrt(vh) + eps)"),
    ("cnn_forward_relu_dropped", "cnn.py", "        a = np.maximum(y, 0.0).reshape(B, H // 2, W // 2, co)",
     "        a = y.reshape(B, H // 2, W // 2, co)"),
    ("cnn_pool_sum", "cnn.py", "    g = x.mean(axis=(1, 2))", "    g = x.sum(axis=(1, 2))"),
    ("cnn_head_bias_dropped", "cnn.py", "    out = g @ p[\"wf\"].T + p[\"bf\"]", "    out = g @ p[\"wf\"].T"),
    ("downsample_counts_empty_pixels", "cnn.py", "                out[r, c, 0] = d[m].mean() / depth_scale",
     "                out[r, c, 0] = d.mean() / depth_scale"),
    # the Python glue of the oracle: grid search (Sec. III-C) and the two-way consistency check
    ("grid_not_subsampled", "__init__.py", "    kd[::stride, ::stride] = np.asarray(kf_depth, np.float32)[::stride, ::stride]",
     "    kd[:, :] = np.asarray(kf_depth, np.float32)"),
    ("grid_last_best", "__init__.py", "    return scores, int(np.argmax(scores)) if len(scores) else -1",
     "    return scores, int(len(scores) - 1 - np.argmax(scores[::-1])) if len(scores) else -1"),
    ("consistency_second_pose_not_inverted", "__init__.py",
     "    Tba = np.ascontiguousarray(pose_inv_fixed(Tab).reshape(12))", "    Tba = Tab"),
    ("downsample_depth_test_dropped", "cnn.py",
     "            m = (d > 0) & (n[..., 3] != 0) & (np.abs(n[..., :3]).sum(-1) > 0)",
     "            m = (n[..., 3] != 0) & (np.abs(n[..., :3]).sum(-1) > 0)"),
]


def _survives_py(name, fname, old, new, workdir, oracle_lib):
    """True when every pin passes with this mistake planted in a copy of the oracle's Python source."""
    import shutil
    tree = os.path.join(workdir, name)
    ignore = shutil.ignore_patterns("__pycache__", "*.so", "*.o")
    for d in ("oracle", "synth", "tests"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(tree, d), ignore=ignore)
    path = os.path.join(tree, "oracle", fname)
    src = open(path).read()
    assert src.count(old) == 1, f"{name}: the text to mutate must occur exactly once"
    mutated = src.replace(old, new)
    compile(mutated, path, "exec")  # a planted mistake must still be a valid program
    with open(path, "w") as fh:
        fh.write(mutated)
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PY_PINS, *PINS]
    for s in SLOW:
        cmd += ["--deselect", s]
    env = dict(os.environ, UPSLAM_ORACLE_LIB=oracle_lib, **ONE_THREAD)
    r = subprocess.run(cmd, cwd=tree, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode in (0, 1), f"{name}: pytest ended with status {r.returncode}:\n{r.stdout[-1500:]}"
    # a mutant counts as caught only through a failing pin, never through an import or collection error
    summary = [ln for ln in r.stdout.splitlines() if ln.strip()][-1]
    assert r.returncode == 0 or ("failed" in summary and "error" not in summary), f"{name}: {summary}"
    return r.returncode == 0


def _survives(name, old, new, workdir):
    """True when every pin passes on the oracle with this mistake planted."""
    src = open(SRC).read()
    assert src.count(old) == 1, f"{name}: the text to mutate must occur exactly once"
    mutant_c = os.path.join(workdir, f"{name}.c")
    mutant_so = os.path.join(workdir, f"{name}.so")
    with open(mutant_c, "w") as fh:
        fh.write(src.replace(old, new))
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", mutant_c,
                           "-o", mutant_so, "-lm"])
    env = dict(os.environ, UPSLAM_ORACLE_LIB=mutant_so, **ONE_THREAD)
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS]
    for s in SLOW:
        cmd += ["--deselect", s]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode in (0, 1), f"{name}: pytest ended with status {r.returncode}:\n{r.stdout[-1500:]}"
    # a mutant counts as caught only through a failing pin, never through an import or collection error
    summary = [ln for ln in r.stdout.splitlines() if ln.strip()][-1]
    assert r.returncode == 0 or ("failed" in summary and "error" not in summary), f"{name}: {summary}"
    return r.returncode == 0


def test_pins_fail_on_every_planted_mistake(tmp_path):
    workers = max(1, min(len(MUTANTS), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        results = list(ex.map(lambda m: (m[0], _survives(*m, str(tmp_path))), MUTANTS))
    survivors = [name for name, alive in results if alive]
    assert not survivors, f"planted mistakes that passed every pin: {survivors}"


def test_numpy_oracle_pins_fail_on_every_planted_mistake(tmp_path):
    sys.path.insert(0, ROOT)
    import oracle
    lib = oracle.build()  # the unmodified C part, shared by every copy
    workers = max(1, min(len(PY_MUTANTS), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        results = list(ex.map(lambda m: (m[0], _survives_py(*m, str(tmp_path), lib)), PY_MUTANTS))
    survivors = [name for name, alive in results if alive]
    assert not survivors, f"planted mistakes that passed every pin: {survivors}"
