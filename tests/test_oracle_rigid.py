"""Pins of the oracle's rigid-body layer (Sec. 3, Eq. 1; semi-implicit Euler on SO(3))."""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import worldgen as wg
from oracle import rigid, timestep as T

HERE = os.path.dirname(__file__)


def _rand_quat(rng):
    q = rng.standard_normal(4)
    return q / np.linalg.norm(q)


def test_quaternion_matches_scipy():
    """quat_to_rot, quat_mul and quat_exp agree with scipy's independent rotation library."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        a, b = _rand_quat(rng), _rand_quat(rng)
        np.testing.assert_allclose(rigid.quat_to_rot(a), Rotation.from_quat(a).as_matrix(), atol=1e-12)
        ab = rigid.quat_mul(a, b)
        np.testing.assert_allclose(rigid.quat_to_rot(ab), rigid.quat_to_rot(a) @ rigid.quat_to_rot(b), atol=1e-12)
        th = rng.standard_normal(3)
        np.testing.assert_allclose(rigid.quat_to_rot(rigid.quat_exp(th)), Rotation.from_rotvec(th).as_matrix(),
                                   atol=1e-12)
    np.testing.assert_allclose(rigid.quat_exp(np.zeros(3)), [0, 0, 0, 1])


def test_mass_matrix_kinetic_energy():
    """Eq. 1: 1/2 u^T M u equals the kinetic energy computed in the body frame."""
    rng = np.random.default_rng(2)
    m, I = 1.7, np.array([0.1, 0.25, 0.4])
    R = Rotation.from_quat(_rand_quat(rng)).as_matrix()
    u = rng.standard_normal(6)
    M = rigid.mass_matrix_block(m, I, R)
    w_body = R.T @ u[3:]
    ke = 0.5 * m * u[:3] @ u[:3] + 0.5 * w_body @ (I * w_body)
    assert abs(0.5 * u @ M @ u - ke) < 1e-12


def test_torque_free_symmetric_top_precession():
    """Torque-free axisymmetric body (I1 = I2): in the body frame omega precesses about the symmetry
    axis at Omega = (I3 - I1) omega3 / I1 (Euler's equations).  A sign error in the gyroscopic
    term reverses the precession; the step error is O(dt)."""
    I1, I3, w_perp, w3 = 0.2, 0.5, 1.0, 3.0
    ws = wg.make_free_body(mass=1.0, inertia=(I1, I1, I3), w0=(w_perp, 0.0, w3))
    st = T.initial_state(ws)
    dt, t_end = 1e-4, 0.5
    params = T.SolverParams()
    st = T.simulate(ws, st, dt, int(round(t_end / dt)), params)
    R = rigid.quat_to_rot(st.q[0, 3:])
    wb = R.T @ st.u[0, 3:]
    Om = (I3 - I1) * w3 / I1
    expect = np.array([w_perp * math.cos(Om * t_end), w_perp * math.sin(Om * t_end), w3])
    np.testing.assert_allclose(wb, expect, atol=5e-3)
    assert abs(np.linalg.norm(st.q[0, 3:]) - 1.0) < 1e-12


def test_free_body_momentum_and_ballistics():
    """Asymmetric free body: angular momentum drift is O(dt) and the centre of mass follows the
    ballistic parabola of semi-implicit Euler exactly: r_N = r_0 + v_0 T + g dt^2 N(N+1)/2."""
    g = np.array([0.0, 0.0, -9.81])
    ws = wg.make_free_body(mass=2.0, inertia=(0.1, 0.2, 0.3), w0=(1.0, 2.0, 3.0), v0=(0.5, 0.0, 1.0), gravity=g)
    st0 = T.initial_state(ws)
    params = T.SolverParams()

    def ang_mom(st):
        R = rigid.quat_to_rot(st.q[0, 3:])
        return R @ (np.array([0.1, 0.2, 0.3]) * (R.T @ st.u[0, 3:]))

    drifts = []
    for dt in (2e-4, 1e-4):
        N = int(round(0.2 / dt))
        st = T.simulate(ws, st0, dt, N, params)
        drifts.append(np.linalg.norm(ang_mom(st) - ang_mom(st0)))
        expect = st0.q[0, :3] + np.array([0.5, 0.0, 1.0]) * N * dt + g * dt * dt * N * (N + 1) / 2
        np.testing.assert_allclose(st.q[0, :3], expect, atol=1e-12)
    assert drifts[1] < 0.7 * drifts[0]          # first-order convergence
    assert drifts[1] < 1e-2


def test_biped_matches_paper_table1_counts():
    """The synthetic biped has DR Legs' counts from the paper's Table 1."""
    ref = json.load(open(os.path.join(HERE, "golden", "paper_table1_drlegs.json")))
    ws = wg.make_biped(num_worlds=2)
    for w in range(2):
        js = ws.joints(w)
        assert ws.world_body_offset[w + 1] - ws.world_body_offset[w] == ref["bodies"]
        assert int(np.sum(ws.joint_actuator[js] >= 0)) == ref["actuated"]
        assert int(np.sum(ws.joint_actuator[js] < 0)) == ref["passive"]
        assert wg.count_loops(ws, w) == ref["loops"]


@pytest.mark.parametrize("maker,loops,rows", [(wg.make_fourbar, 1, 20), (wg.make_stewart, 5, 72),
                                              (wg.make_excavator, 3, 60)])
def test_topology_counts(maker, loops, rows):
    ws = maker(num_worlds=3)
    for w in range(3):
        assert wg.count_loops(ws, w) == loops
        assert ws.bilateral_rows(w) == rows
