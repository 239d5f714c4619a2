"""Pins of the oracle's Moreau-Jean midpoint step (Sec. 3): poses move half a step with the old
velocity, everything is evaluated there, Eq. 2 gives u+, and the poses take the second half step
with u+.  Pinned by closed forms that tell it apart from semi-implicit Euler: an exact ballistic
parabola, second-order convergence of a pendulum to the solution of its exact ODE, and the
joint-error decay that the Baumgarte bias at the half-step pose implies."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import worldgen as wg
from oracle import rigid, timestep as T


def test_midpoint_free_body_follows_the_exact_parabola():
    """u_{k+1} = u_k + g dt and r_{k+1} = r_k + dt (u_k + u_{k+1}) / 2 give r(t) = r0 + v0 t + g t^2 / 2
    exactly (semi-implicit Euler is off by g dt t / 2)."""
    g = np.array([0.0, 0.0, -9.81])
    ws = wg.make_free_body(mass=2.0, inertia=(0.1, 0.2, 0.3), w0=(1.0, 2.0, 3.0), v0=(0.5, 0.0, 1.0), gravity=g)
    st0 = T.initial_state(ws)
    for dt in (2e-4, 1e-4):
        N = int(round(0.2 / dt))
        t = N * dt
        st = T.simulate(ws, st0, dt, N, T.SolverParams(integrator="midpoint"))
        expect = st0.q[0, :3] + np.array([0.5, 0.0, 1.0]) * t + 0.5 * g * t * t
        np.testing.assert_allclose(st.q[0, :3], expect, rtol=0, atol=1e-12)


def _pendulum_angle(st):
    d = rigid.quat_to_rot(st.q[0, 3:])[:, 0]
    return math.atan2(d[0], -d[2])


def _pendulum_ode(theta0, k, t_end, h=1e-5):
    """theta'' = -k sin(theta) from rest, classical RK4 with a step far below the simulator's."""
    th, om = theta0, 0.0
    for _ in range(int(round(t_end / h))):
        a1, b1 = om, -k * math.sin(th)
        a2, b2 = om + 0.5 * h * b1, -k * math.sin(th + 0.5 * h * a1)
        a3, b3 = om + 0.5 * h * b2, -k * math.sin(th + 0.5 * h * a2)
        a4, b4 = om + h * b3, -k * math.sin(th + h * a3)
        th += h / 6 * (a1 + 2 * a2 + 2 * a3 + a4)
        om += h / 6 * (b1 + 2 * b2 + 2 * b3 + b4)
    return th


def test_midpoint_pendulum_converges_at_second_order():
    """Compound pendulum (I_p = m (L^2 + w^2) / 12 + m (L/2)^2, k = m g (L/2) / I_p) released at
    1.2 rad: halving dt divides the midpoint scheme's angle error by ~4, semi-implicit Euler's by ~2."""
    L, m, wdt, g, th0, t_end = 0.5, 1.0, 0.02, 9.81, 1.2, 0.3
    ws = wg.make_pendulum(theta0=th0, length=L, mass=m, width=wdt)
    Ip = m * (L * L + wdt * wdt) / 12.0 + m * (L / 2) ** 2
    ref = _pendulum_ode(th0, m * g * (L / 2) / Ip, t_end)
    errs = {}
    for integ in ("euler", "midpoint"):
        errs[integ] = []
        for dt in (2e-3, 1e-3, 5e-4):
            params = T.SolverParams(eps=1e-12, n_max=5000, rho=0.1, integrator=integ)
            st = T.simulate(ws, T.initial_state(ws), dt, int(round(t_end / dt)), params)
            errs[integ].append(abs(_pendulum_angle(st) - ref))
    mid, eul = errs["midpoint"], errs["euler"]
    assert mid[0] / mid[1] > 3.5 and mid[1] / mid[2] > 3.5
    assert 1.8 < eul[0] / eul[1] < 2.2 and 1.8 < eul[1] / eul[2] < 2.2
    assert mid[2] < 3e-5


def test_midpoint_baumgarte_decay_closed_form():
    """A hinge at rest with a small anchor gap and axis tilt, no gravity.  With m_k the joint error
    at the half-step pose of step k and e_k the one at its end (to first order in the error):
    the rows enforce J u_k = -(beta/dt) m_k, so e_k = m_k + (dt/2) J u_k = (1 - beta/2) m_k, and the
    next half step moves with u_k again: m_{k+1} = e_k + (dt/2) J u_k = (1 - beta) m_k.  At rest
    m_1 = f_0, hence e_k = (1 - beta/2)(1 - beta)^(k-1) f_0."""
    ws = wg.make_pendulum(theta0=0.5)
    ws.gravity = np.zeros(3)
    st = T.initial_state(ws)
    st.q[0, :3] += np.array([1e-6, 2e-6, -1.5e-6])
    tilt = Rotation.from_rotvec([1e-6, 0.0, -0.7e-6])
    st.q[0, 3:] = (tilt * Rotation.from_quat(st.q[0, 3:])).as_quat()
    anchor = ws.joint_frame_child[0][:3]
    axis = Rotation.from_quat(ws.joint_frame_child[0][3:]).as_matrix()[:, 2]

    def joint_error(s):
        R = Rotation.from_quat(s.q[0, 3:]).as_matrix()
        a = R @ axis
        return np.concatenate([s.q[0, :3] + R @ anchor, [a[0], a[2]]])

    params = T.SolverParams(eps=1e-12, n_max=20000, rho=0.1, integrator="midpoint")
    b = params.beta
    e0 = joint_error(st)
    for k in range(1, 11):
        st, _ = T.step(ws, st, None, 1e-3, params)
        np.testing.assert_allclose(joint_error(st), (1 - b / 2) * (1 - b) ** (k - 1) * e0, rtol=0, atol=2e-12)


def test_midpoint_resting_box_carries_its_weight():
    """At rest the half step does not move the box, so the normal impulses sum to m g dt as in
    the semi-implicit step, and the box stays at rest."""
    m, dt = 1.3, 2e-3
    ws = wg.make_box(mass=m, mu=0.6)
    params = T.SolverParams(eps=1e-10, n_max=20000, rho=0.1, integrator="midpoint")
    st, infos = T.step(ws, T.initial_state(ws), None, dt, params)
    lam = infos[0].lam.reshape(-1, 3)
    assert abs(lam[:, 2].sum() - m * 9.81 * dt) < 1e-8
    assert np.abs(st.u[0]).max() < 1e-8
    np.testing.assert_allclose(st.q, T.initial_state(ws).q, atol=1e-12)


def test_unknown_integrator_is_rejected():
    ws = wg.make_free_body()
    with pytest.raises(ValueError):
        T.step(ws, T.initial_state(ws), None, 1e-3, T.SolverParams(integrator="rk4"))


def test_midpoint_sliding_box_follows_the_exact_parabola():
    """Coulomb sliding under the midpoint scheme: the speed falls by mu g dt per step as before,
    and the position, advanced with the mean of the old and new speeds, is exactly
    x0 + v0 t - mu g t^2 / 2 while the box slides (semi-implicit Euler is off by mu g dt t / 2)."""
    mu, v0, dt = 0.4, 0.5, 1e-3
    ws = wg.make_box(mass=1.0, mu=mu, v0=(v0, 0.0, 0.0))
    st = T.initial_state(ws)
    x0 = st.q[0, 0]
    params = T.SolverParams(eps=1e-10, n_max=20000, rho=0.1, integrator="midpoint")
    for k in range(1, 101):
        st, _ = T.step(ws, st, None, dt, params)
        t = k * dt
        assert abs(st.q[0, 0] - (x0 + v0 * t - 0.5 * mu * 9.81 * t * t)) < 1e-11
        assert abs(st.u[0, 0] - (v0 - mu * 9.81 * t)) < 2e-6
    assert abs(st.q[0, 2] - 0.025) < 1e-12 and np.abs(st.u[0, 1:]).max() < 1e-9
