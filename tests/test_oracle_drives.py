"""Pins of the oracle's joint-space dynamics (Sec. 3; Eq. 2's R and v*, Eq. 4's D = J M^-1 J^T + R):
implicit PD drives, armature and viscous damping as regularised rows on the joint coordinate, and
unilateral joint limits.  The references are a hinge's scalar recurrences derived by hand (a rod
on a frictionless hinge without gravity is a one-degree-of-freedom system with inertia I_p about
the hinge), the static balance of a pendulum held by a limit, the direct KKT solve of Eq. 2 with R,
finite differences for the joint coordinate's row, and the NCP conditions."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import worldgen as wg
from oracle import audit as A, constraints as C, timestep as T

L, MASS, WIDTH, G = 0.5, 1.0, 0.02, 9.81
I_P = MASS * (L * L + WIDTH * WIDTH) / 12.0 + MASS * (L / 2) ** 2     # rod about its end, axis y
PARAMS = T.SolverParams(eps=1e-12, n_max=20000, rho=0.1)


def _hinge_angle(st):
    """Hinge coordinate of the pendulum read from its pose: theta0 - theta, theta the rod's angle
    from hanging (the hinge axis is +y, so a positive rotation swings the rod towards hanging)."""
    d = Rotation.from_quat(st.q[0, 3:]).as_matrix()[:, 0]
    return 0.5 - math.atan2(d[0], -d[2])


def _free_hinge(mode, kp=0.0, kd=0.0, armature=0.0, damping=0.0):
    ws = wg.with_joint_drives(wg.make_pendulum(theta0=0.5, actuated=True), mode, kp, kd, armature, damping)
    ws.gravity = np.zeros(3)
    return ws


# ----------------------------------------------------------------------------- joint coordinate
def test_joint_coordinate_is_the_hinge_rotation():
    ws = wg.make_pendulum(theta0=0.5)
    st = T.initial_state(ws)
    for alpha in (0.0, 0.3, -1.1, 2.5):
        q = st.q.copy()
        q[0, 3:] = (Rotation.from_rotvec([0.0, alpha, 0.0]) * Rotation.from_quat(q[0, 3:])).as_quat()
        q[0, :3] = Rotation.from_rotvec([0.0, alpha, 0.0]).apply(q[0, :3])      # about the pivot
        R = np.array([Rotation.from_quat(q[0, 3:]).as_matrix()])
        d, _, _ = C.joint_coordinate(C.REVOLUTE, -1, 0, ws.joint_frame_parent[0], ws.joint_frame_child[0],
                                     q[:, :3], R)
        assert abs(d - alpha) < 1e-12


@pytest.mark.parametrize("maker,jtype", [(wg.make_biped, C.REVOLUTE), (wg.make_excavator, C.PRISMATIC)])
def test_joint_coordinate_row_is_its_time_derivative(maker, jtype):
    """J_d u = d-dot by central differences along random twists (world-anchored hinges and body-body
    slides alike)."""
    ws = maker(num_worlds=1, seed=9)
    rng = np.random.default_rng(9)
    bs = ws.bodies(0)
    r0, q0 = ws.body_q0[bs, :3], ws.body_q0[bs, 3:]
    js = [j for j in range(*ws.joints(0).indices(len(ws.joint_type))) if ws.joint_type[j] == jtype]
    assert js
    for j in js[:6]:
        par, ch = int(ws.joint_parent[j]), int(ws.joint_child[j])
        u = rng.standard_normal((bs.stop - bs.start, 6))

        def d_at(h):
            r = r0 + h * u[:, :3]
            R = np.array([(Rotation.from_rotvec(h * u[i, 3:]) * Rotation.from_quat(q0[i])).as_matrix()
                          for i in range(len(q0))])
            return C.joint_coordinate(jtype, par, ch, ws.joint_frame_parent[j], ws.joint_frame_child[j], r, R)

        _, Ja, Jb = d_at(0.0)
        rate = Jb @ u[ch] + (Ja @ u[par] if par >= 0 else 0.0)
        h = 1e-6
        fd = (d_at(h)[0] - d_at(-h)[0]) / (2 * h)
        assert abs(rate - fd) < 1e-6 * max(1.0, abs(fd))


# ----------------------------------------------------------------------------- drives
@pytest.mark.parametrize("kp,kd,armature,damping", [(50.0, 2.0, 0.0, 0.0), (50.0, 2.0, 0.05, 0.3),
                                                     (1e7, 0.0, 0.0, 0.0)])
def test_implicit_pd_follows_the_hinge_recurrence(kp, kd, armature, damping):
    """Position target d_t, zero velocity target: the row's impulse makes
    (I_p + I_a) d-dot+ = (I_p + I_a) d-dot- + dt Kp (d_t - d - dt d-dot+) - dt (Kd + b) d-dot+ and
    d+ = d + dt d-dot+.  Also with Kp dt^2 = 120 I_p, far past the explicit PD's stability limit
    dt < 2 sqrt(I_p / Kp) = 0.18 ms (no blow-up: implicit)."""
    ws = _free_hinge(wg.DRIVE_PD, kp, kd, armature, damping)
    st = T.initial_state(ws)
    target = 0.02
    d = d_dot = peak = 0.0
    for k in range(300):
        st, infos = T.step(ws, st, np.array([[target]]), 1e-3, PARAMS)
        d_dot = ((I_P + armature) * d_dot + 1e-3 * kp * (target - d)) / (
            I_P + armature + 1e-6 * kp + 1e-3 * (kd + damping))
        d += 1e-3 * d_dot
        peak = max(peak, abs(d_dot))
        assert abs(_hinge_angle(st) - d) < 2e-6 * target
        # the rate about the hinge is omega_y; the scalar recurrence ignores the chord the rod's
        # centre travels in one step, a relative effect of order (dt d-dot)^2
        assert abs(st.u[0, 4] - d_dot) < 1e-4 * peak
    i = infos[0]
    assert i.reg is not None and i.reg[i.n_bilateral - 1] > 0          # the drive row is regularised
    assert max(A.ncp_residual(i.J, i.u_plus, i.v_star, i.lam, i.p, i.n_bilateral, i.mu, i.reg)) < 1e-9


@pytest.mark.parametrize("armature,damping", [(0.05, 0.0), (0.05, 0.4), (0.0, 0.4)])
def test_armature_and_damping_under_a_constant_torque(armature, damping):
    """Torque mode: the input torque acts as a force and the row adds reflected inertia and viscous
    damping, (I_p + I_a) d-dot+ = (I_p + I_a) d-dot- + dt tau - dt b d-dot+ (terminal rate tau/b)."""
    ws = _free_hinge(wg.DRIVE_TORQUE, 0.0, 0.0, armature, damping)
    st = T.initial_state(ws)
    tq = 0.01
    d = d_dot = 0.0
    for k in range(300):
        st, _ = T.step(ws, st, np.array([[tq]]), 1e-3, PARAMS)
        d_dot = ((I_P + armature) * d_dot + 1e-3 * tq) / (I_P + armature + 1e-3 * damping)
        d += 1e-3 * d_dot
        assert abs(st.u[0, 4] - d_dot) < 1e-7 * d_dot
        assert abs(_hinge_angle(st) - d) < 1e-6 * d


@pytest.mark.parametrize("cr_iters", [None, 9])
def test_drives_on_a_bilateral_world_match_the_direct_kkt_solve(cr_iters):
    """Excavator (hinges and slides in closed loops) with implicit PD on its actuated joints: PADMM
    reaches the solution of Eq. 2 with R solved directly, with the dense factorisation and with the
    matrix-free operator (which adds P R P to its chain of products)."""
    ws = wg.with_joint_drives(wg.make_excavator(num_worlds=2, seed=4), wg.DRIVE_PD, 400.0, 20.0, 0.02, 1.0)
    st = T.initial_state(ws)
    tau = 0.05 * wg.actuation(ws, 4, 0) / 5.0
    st, infos = T.step(ws, st, tau, 2e-3, T.SolverParams(eps=1e-12, n_max=50000, rho=0.1, cr_iters=cr_iters))
    for i in infos:
        assert i.converged and i.reg is not None
        M = np.linalg.inv(i.Minv)
        u_kkt, _ = A.kkt_direct(i.J, M, M @ i.u_free, i.v_star, R=np.diag(i.reg))
        assert np.abs(i.u_plus - u_kkt).max() / max(np.abs(u_kkt).max(), 9.81 * 2e-3) < 1e-8


# ----------------------------------------------------------------------------- limits
def test_limit_stops_the_swing_and_holds_the_pendulum_statically():
    """An upper limit at d = 0.2 (theta = 0.3 from hanging): the swing ends there without
    overshoot (the gap closes within a step and no further), the rod comes to rest (restitution
    0), and the limit impulse balances gravity's torque, dt m g (L/2) sin(0.3)."""
    ws = wg.with_joint_limits(wg.make_pendulum(theta0=0.5), -np.inf, 0.2)
    st = T.initial_state(ws)
    peak = -1.0
    for k in range(600):
        st, infos = T.step(ws, st, None, 1e-3, PARAMS)
        peak = max(peak, _hinge_angle(st))
    i = infos[0]
    assert peak < 0.2 + 1e-12
    assert abs(_hinge_angle(st) - 0.2) < 1e-12 and np.abs(st.u).max() < 1e-10
    assert len(i.unilateral) == 1
    assert abs(i.lam[i.unilateral[0]] - 1e-3 * MASS * G * (L / 2) * math.sin(0.3)) < 1e-12
    assert max(A.ncp_residual(i.J, i.u_plus, i.v_star, i.lam, i.p, i.n_bilateral, i.mu, i.reg,
                              i.unilateral)) < 1e-9


def test_active_limit_lets_the_joint_move_away():
    """A lower limit just below the start (inside the activation margin) while gravity swings the
    rod away from it: the row is present but slack (lambda = 0) and the step equals the free one."""
    free = wg.make_pendulum(theta0=0.5)
    limited = wg.with_joint_limits(wg.make_pendulum(theta0=0.5), -0.001, np.inf)
    st_f, _ = T.step(free, T.initial_state(free), None, 1e-3, PARAMS)
    st_l, infos = T.step(limited, T.initial_state(limited), None, 1e-3, PARAMS)
    i = infos[0]
    assert len(i.unilateral) == 1 and abs(i.lam[i.unilateral[0]]) < 1e-12
    np.testing.assert_allclose(st_l.u, st_f.u, rtol=1e-8, atol=1e-12)


def test_inactive_limits_add_no_rows():
    ws = wg.make_biped(num_worlds=1, seed=3)
    wl = wg.with_joint_limits(ws, -3.0, 3.0)
    tau = wg.actuation(ws, 3, 0)
    _, a = T.step(ws, T.initial_state(ws), tau, 2e-3, T.SolverParams(eps=1e-9, n_max=20000, rho=0.1))
    _, b = T.step(wl, T.initial_state(wl), tau, 2e-3, T.SolverParams(eps=1e-9, n_max=20000, rho=0.1))
    assert a[0].m == b[0].m and not b[0].unilateral
    np.testing.assert_allclose(a[0].u_plus, b[0].u_plus, rtol=0, atol=0)
