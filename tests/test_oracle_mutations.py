"""Planted mistakes: each mutation of the oracle (made here, on the CPU, with monkeypatch) must make
at least one pin fail.  This shows the pins are sensitive to the plausible errors they target."""
import numpy as np
import pytest

from oracle import constraints as C, padmm as PA, rigid, timestep as T
import tests.test_oracle_closed_forms as TF
import tests.test_oracle_constraints as TC
import tests.test_oracle_padmm as TP
import tests.test_oracle_rigid as TR


def _fails(fn, *a):
    try:
        fn(*a)
    except AssertionError:
        return True
    return False


def test_gyroscopic_sign_flip_is_caught(monkeypatch):
    orig = rigid.newton_euler_h

    def flipped(mass, inertia_diag, R, omega, gravity, force=None, torque=None):
        h = orig(mass, inertia_diag, R, omega, gravity, force, torque)
        Iw = R @ np.diag(inertia_diag) @ R.T
        h[3:] += 2 * np.cross(omega, Iw @ omega)
        return h

    monkeypatch.setattr(rigid, "newton_euler_h", flipped)
    import oracle.timestep as T
    monkeypatch.setattr(T, "newton_euler_h", flipped)
    assert _fails(TR.test_torque_free_symmetric_top_precession)


def test_dropped_lever_arm_is_caught(monkeypatch):
    orig = C.joint_rows

    def no_lever(jtype, parent, child, fp, fc, r, R):
        rows = orig(jtype, parent, child, fp, fc, r, R)
        out = []
        for k, (ba, Ja, bb, Jb, f) in enumerate(rows):
            if k < 3 and jtype != C.PRISMATIC:
                Jb = Jb.copy()
                Jb[3:] = 0.0
            out.append((ba, Ja, bb, Jb, f))
        return out

    monkeypatch.setattr(C, "joint_rows", no_lever)
    assert _fails(TC.test_joint_jacobian_is_derivative_of_error, C.REVOLUTE, False)


def test_wrong_cone_projection_is_caught(monkeypatch):
    def radial(x, n_bilateral, mu):            # scales onto the cone instead of projecting
        y = x.copy()
        for k, m in enumerate(mu):
            i = n_bilateral + 3 * k
            tn = np.hypot(x[i], x[i + 1])
            if tn > m * x[i + 2]:
                n = max(x[i + 2], 0.0)
                y[i:i + 2] = x[i:i + 2] * (m * n / tn if tn > 0 else 0.0)
                y[i + 2] = n
        return y

    monkeypatch.setattr(PA, "project_cone", radial)
    assert _fails(TP.test_cone_projection_kkt_and_brute_force, 0.3)


def test_transposed_desaxce_is_caught(monkeypatch):
    def on_tangent(v, n_bilateral, mu):        # correction put on a tangential row
        s = np.zeros_like(v)
        for k, m in enumerate(mu):
            i = n_bilateral + 3 * k
            s[i] = m * np.hypot(v[i], v[i + 1])
        return s

    monkeypatch.setattr(PA, "desaxce", on_tangent)
    assert _fails(TP.test_desaxce_operator)


def test_baumgarte_sign_flip_is_caught(monkeypatch):
    orig = C.joint_rows

    def flipped(jtype, parent, child, fp, fc, r, R):      # bias +(beta/dt) f instead of -(...)
        return [(ba, Ja, bb, Jb, -f) for ba, Ja, bb, Jb, f in orig(jtype, parent, child, fp, fc, r, R)]

    monkeypatch.setattr(C, "joint_rows", flipped)
    assert _fails(TF.test_baumgarte_shrinks_joint_error_by_one_minus_beta_per_step)


def test_body_frame_rotation_update_is_caught(monkeypatch):
    def right_product(r, q, v_plus, w_plus, dt):          # world-frame omega applied on the right
        q_new = rigid.quat_mul(q, rigid.quat_exp(dt * w_plus))
        return r + dt * v_plus, q_new / np.linalg.norm(q_new)

    monkeypatch.setattr(T, "integrate_pose", right_product)
    assert _fails(TR.test_torque_free_symmetric_top_precession)


def test_explicit_euler_position_update_is_caught(monkeypatch):
    orig_step = T.step

    def explicit(ws, state, tau, dt, params, worlds=None):  # r+ = r + dt u- instead of dt u+
        new, infos = orig_step(ws, state, tau, dt, params, worlds)
        new.q[:, :3] += dt * (state.u[:, :3] - new.u[:, :3])
        return new, infos

    monkeypatch.setattr(T, "step", explicit)
    assert _fails(TR.test_free_body_momentum_and_ballistics)


def test_delassus_without_inverse_mass_is_caught(monkeypatch):
    monkeypatch.setattr(PA, "delassus", lambda J, Minv, R=None: J @ J.T)
    assert _fails(TP.test_box_resting_on_plane_carries_its_weight)


def test_unshared_tangential_scaling_is_caught(monkeypatch):
    def own_scale(D, n_bilateral, n_contacts, precond=True):   # scaled cone no longer circular
        return 1.0 / np.sqrt(np.diag(D)) if precond else np.ones(D.shape[0])

    monkeypatch.setattr(PA, "jacobi_scaling", own_scale)
    assert _fails(TP.test_sliding_box_decelerates_at_mu_g_and_stops, 1)


def test_dropped_dual_residual_is_caught(monkeypatch):
    orig = PA.residuals

    def no_dual(*a):                                        # stops as soon as x = y
        r_p, _, r_c = orig(*a)
        return r_p, 0.0, r_c

    monkeypatch.setattr(PA, "residuals", no_dual)
    assert _fails(TP.test_padmm_matches_direct_kkt, TP.wg.make_fourbar, 1e-3)


def test_baumgarte_on_speculative_contacts_is_caught(monkeypatch):
    def always_beta(phi, beta, dt):                        # beta phi/dt on gaps too
        return [0.0, 0.0, beta * phi / dt]

    monkeypatch.setattr(C, "contact_bias", always_beta)
    assert _fails(TP.test_approaching_box_lands_on_the_surface_and_stops)


def test_contact_bias_without_beta_is_caught(monkeypatch):
    def full_depth(phi, beta, dt):                         # whole depth removed in one step
        return [0.0, 0.0, phi / dt]

    monkeypatch.setattr(C, "contact_bias", full_depth)
    assert _fails(TP.test_penetrating_box_rises_at_beta_depth_over_dt)


def test_conjugate_gradient_steps_in_cr_are_caught(monkeypatch):
    import tests.test_oracle_cr as TCR

    def cg(apply_A, c, x0, iters):                          # (r, r) and (p, A p): CG, not CR
        x = np.array(x0, dtype=np.float64)
        r = c - apply_A(x)
        p = r.copy()
        for _ in range(iters):
            Ap = apply_A(p)
            rr = float(r @ r)
            if rr == 0.0:
                break
            alpha = rr / float(p @ Ap)
            x = x + alpha * p
            r = r - alpha * Ap
            p = r + (float(r @ r) / rr) * p
        return x

    monkeypatch.setattr(PA, "conjugate_residual", cg)
    assert _fails(TCR.test_cr_iterate_minimises_residual_over_krylov_space, 3)


def test_stopping_test_blind_to_the_cr_residual_is_caught(monkeypatch):
    import tests.test_oracle_cr as TCR
    orig = PA.residuals

    def blind(*a):                                          # drops lin_res
        return orig(*a[:9])

    monkeypatch.setattr(PA, "residuals", blind)
    assert _fails(TCR.test_cr_padmm_matches_direct_kkt, TCR.wg.make_excavator, 2e-3, 1)


def test_one_sided_scaling_in_matrix_free_delassus_is_caught(monkeypatch):
    import tests.test_oracle_cr as TCR

    def one_sided(J, Minv, p, R=None):                      # P J M^-1 J^T v: right-hand P dropped
        return lambda v: p * (J @ (Minv @ (J.T @ v)))

    monkeypatch.setattr(PA, "delassus_matrix_free", one_sided)
    assert _fails(TCR.test_matrix_free_delassus_is_the_scaled_delassus_matrix)


def test_pd_target_with_the_wrong_sign_is_caught(monkeypatch):
    import tests.test_oracle_drives as TD
    orig = C.drive_row

    def flipped(d, d_dot, target, dt, kp, kd, armature, damping):     # Kp (d - target)
        return orig(d, d_dot, 2 * d - target, dt, kp, kd, armature, damping)

    monkeypatch.setattr(C, "drive_row", flipped)
    assert _fails(TD.test_implicit_pd_follows_the_hinge_recurrence, 50.0, 2.0, 0.0, 0.0)


def test_armature_missing_from_the_drive_compliance_is_caught(monkeypatch):
    import tests.test_oracle_drives as TD
    orig = C.drive_row

    def no_armature_in_c(d, d_dot, target, dt, kp, kd, armature, damping):
        R, v = orig(d, d_dot, target, dt, kp, kd, 0.0, damping) if (kp or kd or damping) else (None, None)
        if R is None:
            return None
        return R, v - armature * d_dot * R                              # C without I_a, v* with it

    monkeypatch.setattr(C, "drive_row", no_armature_in_c)
    assert _fails(TD.test_armature_and_damping_under_a_constant_torque, 0.05, 0.4)


def test_limit_rows_treated_as_bilateral_are_caught(monkeypatch):
    import tests.test_oracle_drives as TD
    orig = PA.project_cone

    def no_ray(x, n_bilateral, mu, unilateral=None):                    # lambda < 0 allowed
        return orig(x, n_bilateral, mu)

    monkeypatch.setattr(PA, "project_cone", no_ray)
    assert _fails(TD.test_active_limit_lets_the_joint_move_away)


def test_fk_coordinate_rows_with_the_wrong_sign_are_caught(monkeypatch):
    import oracle.kinematics as K
    import tests.test_oracle_kinematics as TK
    orig = K.residual_and_jacobian

    def flipped(ws, w, q, joints, targets, free):
        F, Jf = orig(ws, w, q, joints, targets, free)
        Jf = Jf.copy()
        if len(joints):
            Jf[-len(joints):] *= -1.0
        return F, Jf

    monkeypatch.setattr(K, "residual_and_jacobian", flipped)
    assert _fails(TK.test_fourbar_fk_matches_the_position_analysis)


def test_fk_update_in_the_body_frame_is_caught(monkeypatch):
    import oracle.kinematics as K
    import tests.test_oracle_kinematics as TK
    monkeypatch.setattr(K, "quat_mul", lambda a, b: rigid.quat_mul(b, a))   # q (x) exp(dw)
    assert _fails(TK.test_biped_fk_round_trip, 0)


def test_matrix_free_operator_without_r_is_caught(monkeypatch):
    import tests.test_oracle_drives as TD
    orig = PA.delassus_matrix_free
    monkeypatch.setattr(PA, "delassus_matrix_free", lambda J, Minv, p, R=None: orig(J, Minv, p))
    assert _fails(TD.test_drives_on_a_bilateral_world_match_the_direct_kkt_solve, 9)


def test_wrong_nesterov_weight_is_caught(monkeypatch):
    orig = PA.nesterov_coefficient

    def shifted(a):                             # a / a' instead of (a - 1) / a'
        a_next, _ = orig(a)
        return a_next, a / a_next

    monkeypatch.setattr(PA, "nesterov_coefficient", shifted)
    assert _fails(TP.test_nesterov_sequence_matches_hand_recurrence)


def test_restart_test_that_always_fires_is_caught(monkeypatch):
    """A restart test whose comparison never holds (every iteration restarts, so there is no
    acceleration at all) changes the sequence from the second iteration on."""
    src = PA.padmm

    def no_reset(*a, **k):
        k = dict(k)
        k["restart_factor"] = 1e-300            # every iteration restarts
        return src(*a, **k)

    monkeypatch.setattr(PA, "padmm", no_reset)
    assert _fails(TP.test_nesterov_sequence_matches_hand_recurrence)
