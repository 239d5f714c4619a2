"""Whole-step pins of the oracle against closed forms and independent formulations:
the compound-pendulum period (elliptic integral), a reduced-coordinate four-bar integrated with
RK4, and the invariants of the closed loop (Sec. 3: loop closures are ordinary joints)."""
import math

import numpy as np
import pytest

import worldgen as wg
from oracle import rigid, timestep as T


def _agm(a, b):
    while abs(a - b) > 1e-15 * a:
        a, b = 0.5 * (a + b), math.sqrt(a * b)
    return a


def _ellipk(k):
    """Complete elliptic integral of the first kind by the arithmetic-geometric mean."""
    return math.pi / (2.0 * _agm(1.0, math.sqrt(1.0 - k * k)))


def _pendulum_angle(st):
    # rod axis (body x) points from the pivot to the tip; the angle is measured from hanging (-z)
    R = rigid.quat_to_rot(st.q[0, 3:])
    d = R[:, 0]
    return math.atan2(d[0], -d[2])


@pytest.mark.parametrize("theta0", [0.3, 1.2])
def test_compound_pendulum_period(theta0):
    """T = 4 sqrt(I_p / (m g d)) K(sin(theta0 / 2)), I_p = m L^2 / 3 (+ rod width term), d = L / 2."""
    L, m, wdt, g = 0.5, 1.0, 0.02, 9.81
    ws = wg.make_pendulum(theta0=theta0, length=L, mass=m, width=wdt)
    Ip = m * (L * L + wdt * wdt) / 12.0 + m * (L / 2) ** 2
    T_exact = 4.0 * math.sqrt(Ip / (m * g * L / 2)) * _ellipk(math.sin(theta0 / 2))
    dt = 5e-4
    params = T.SolverParams(eps=1e-11, n_max=5000, rho=0.1)
    st = T.initial_state(ws)
    prev = _pendulum_angle(st)
    crossings = []
    t = 0.0
    while len(crossings) < 3 and t < 3 * T_exact:
        st, _ = T.step(ws, st, None, dt, params)
        t += dt
        ang = _pendulum_angle(st)
        if prev > 0 >= ang:           # downward zero crossing, linear interpolation in time
            crossings.append(t - dt * ang / (ang - prev))
        prev = ang
    period = crossings[2] - crossings[1]
    assert abs(period - T_exact) / T_exact < 2e-3


def _fourbar_geometry(lg, l1, l2, l3, th):
    """Closed-form planar four-bar in the x-z plane: pivots O=(0,0), G=(lg,0); crank angle th;
    the coupler-rocker joint B on the upper branch.  Returns link (centre_x, centre_z, angle)."""
    ax, az = l1 * math.cos(th), l1 * math.sin(th)
    dx, dz = lg - ax, -az
    d = math.hypot(dx, dz)
    x = (l2 * l2 - l3 * l3 + d * d) / (2 * d)
    h = math.sqrt(l2 * l2 - x * x)
    ex, ez = dx / d, dz / d
    px, pz = -ez, ex
    b1 = (ax + x * ex + h * px, az + x * ez + h * pz)
    b2 = (ax + x * ex - h * px, az + x * ez - h * pz)
    bx, bz = b1 if b1[1] >= b2[1] else b2
    links = [((0, 0), (ax, az)), ((ax, az), (bx, bz)), ((lg, 0), (bx, bz))]
    out = []
    for (x0, z0), (x1, z1) in links:
        out.append((0.5 * (x0 + x1), 0.5 * (z0 + z1), math.atan2(z1 - z0, x1 - x0)))
    return out


def test_fourbar_matches_reduced_coordinate_rk4():
    """One-DoF Lagrangian of the same four-bar in its crank angle theta, integrated with RK4:
    m(theta) theta'' + m'(theta) theta'^2 / 2 + V'(theta) = 0, with m(theta) = sum_i
    (m_i |dc_i/dtheta|^2 + I_i (dphi_i/dtheta)^2) and V = sum_i m_i g z_i.  The maximal-coordinate
    oracle must follow it to O(dt) over 0.1 s."""
    ws = wg.make_fourbar(num_worlds=1, seed=11)
    jp = ws.joint_frame_parent
    lg = jp[3, 0]
    bs = ws.bodies(0)
    q0 = ws.body_q0[bs]
    # link lengths and inertias about the hinge axis (+y), from the description
    mass = ws.body_mass[bs]
    Iy = ws.body_inertia[bs][:, 2]      # rods: body x along the rod, body z along the hinge (+y world)
    crank_tip = 2 * q0[0, :3]                              # crank starts at the origin
    b = 2 * q0[2, :3] - np.array([lg, 0, 0])               # rocker starts at G
    l1 = np.linalg.norm(crank_tip)
    l2 = np.linalg.norm(b - crank_tip)
    l3 = np.linalg.norm(b - np.array([lg, 0, 0]))
    th0 = math.atan2(crank_tip[2], crank_tip[0])
    g = 9.81

    def geom(th):
        return np.array(_fourbar_geometry(lg, l1, l2, l3, th))

    def mass_pot(th, hstep=1e-6):
        dg = (geom(th + hstep) - geom(th - hstep)) / (2 * hstep)
        mth = float(np.sum(mass * (dg[:, 0] ** 2 + dg[:, 1] ** 2) + Iy * dg[:, 2] ** 2))
        return mth, float(np.sum(mass * g * geom(th)[:, 1]))

    def accel(th, om):
        h = 1e-5
        m0, _ = mass_pot(th)
        mp, vp = mass_pot(th + h)
        mm, vm = mass_pot(th - h)
        return -(0.5 * (mp - mm) / (2 * h) * om * om + (vp - vm) / (2 * h)) / m0

    # RK4 reference
    t_end, h = 0.1, 1e-4
    th, om = th0, 0.0
    for _ in range(int(round(t_end / h))):
        k1 = (om, accel(th, om))
        k2 = (om + 0.5 * h * k1[1], accel(th + 0.5 * h * k1[0], om + 0.5 * h * k1[1]))
        k3 = (om + 0.5 * h * k2[1], accel(th + 0.5 * h * k2[0], om + 0.5 * h * k2[1]))
        k4 = (om + h * k3[1], accel(th + h * k3[0], om + h * k3[1]))
        th += h / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
        om += h / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])

    errs = []
    for dt in (1e-3, 5e-4):
        params = T.SolverParams(eps=1e-11, n_max=5000, rho=0.1)
        st = T.simulate(ws, T.initial_state(ws), dt, int(round(t_end / dt)), params)
        tip = 2 * st.q[0, :3]
        errs.append(abs(math.atan2(tip[2], tip[0]) - th))
    assert abs(th - th0) > 0.05                        # the linkage really moved
    assert errs[1] < 0.7 * errs[0]                     # first-order convergence to the reference
    assert errs[1] < 2e-3


def test_fourbar_invariants_loop_closure_energy_rank():
    """Over 1000 steps of 1 ms: loop-closure error stays bounded (Baumgarte), the energy of the
    frictionless linkage drifts boundedly, and J has rank 17 of 20 rows (three redundant rows of
    a planar loop in 3-D)."""
    ws = wg.make_fourbar(num_worlds=1, seed=12)
    params = T.SolverParams(eps=1e-10, n_max=5000, rho=0.1)
    st = T.initial_state(ws)
    bs = ws.bodies(0)

    def energy(s):
        e = 0.0
        for i in range(3):
            R = rigid.quat_to_rot(s.q[i, 3:])
            wb = R.T @ s.u[i, 3:]
            e += 0.5 * ws.body_mass[i] * s.u[i, :3] @ s.u[i, :3] + 0.5 * wb @ (ws.body_inertia[i] * wb)
            e += ws.body_mass[i] * 9.81 * s.q[i, 2]
        return e

    e0 = energy(st)
    errs = []
    energies = []
    rank = None
    for k in range(1000):
        st, infos = T.step(ws, st, None, 1e-3, params)
        i = infos[0]
        errs.append(np.abs(i.v_star).max() * 1e-3 / params.beta)      # |f(q)| from the bias
        energies.append(energy(st))
        if rank is None:
            rank = np.linalg.matrix_rank(i.J, tol=1e-9)
    assert rank == 17
    assert max(errs) < 5e-4
    assert max(errs[500:]) < 3.0 * max(errs[:500]) + 1e-6          # bounded, not growing
    swing = max(abs(e - e0) for e in energies)
    scale = sum(ws.body_mass[i] * 9.81 * 0.1 for i in range(3))
    assert swing < 0.05 * scale


def test_baumgarte_shrinks_joint_error_by_one_minus_beta_per_step():
    """Sec. 3's stabilisation: the bilateral rows enforce J u+ = -(beta/dt) f(q), so a hinge whose
    anchor gap and axis tilt are small (and which nothing else moves: no gravity, at rest) has
    f_k = (1 - beta)^k f_0 to first order.  The error is read from the poses with scipy's
    rotations, not from the oracle's rows."""
    from scipy.spatial.transform import Rotation

    ws = wg.make_pendulum(theta0=0.5)
    ws.gravity = np.zeros(3)
    st = T.initial_state(ws)
    st.q[0, :3] += np.array([1e-6, 2e-6, -1.5e-6])
    tilt = Rotation.from_rotvec([1e-6, 0.0, -0.7e-6])
    st.q[0, 3:] = (tilt * Rotation.from_quat(st.q[0, 3:])).as_quat()
    anchor = ws.joint_frame_child[0][:3]
    axis = Rotation.from_quat(ws.joint_frame_child[0][3:]).as_matrix()[:, 2]

    def joint_error(s):
        # the hinge is at the world origin about +y: anchor gap and the axis' x and z components
        R = Rotation.from_quat(s.q[0, 3:]).as_matrix()
        a = R @ axis
        return np.concatenate([s.q[0, :3] + R @ anchor, [a[0], a[2]]])

    params = T.SolverParams(eps=1e-12, n_max=20000, rho=0.1)
    e0 = joint_error(st)
    for k in range(1, 11):
        st, _ = T.step(ws, st, None, 1e-3, params)
        np.testing.assert_allclose(joint_error(st), (1.0 - params.beta) ** k * e0, rtol=0, atol=2e-12)
