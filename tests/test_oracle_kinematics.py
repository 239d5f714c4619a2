"""Pins of the oracle's Gauss-Newton forward kinematics for resets (Sec. 6.3): the four-bar's
closed-form position analysis (circle intersection), a biped round trip through random joint
targets, the quadratic convergence that distinguishes Gauss-Newton on a zero-residual problem,
and poses a time step can start from."""
import math

import numpy as np
import pytest

import worldgen as wg
from oracle import kinematics as K, rigid, timestep as T


def _anchor(ws, q, j):
    """World position of joint j's anchor on its child body."""
    ch = int(ws.joint_child[j])
    return q[ch, :3] + rigid.quat_to_rot(q[ch, 3:]) @ ws.joint_frame_child[j][:3]


def _upper_intersection(a, ra, b, rb):
    d = np.linalg.norm(b - a)
    x = (ra * ra - rb * rb + d * d) / (2 * d)
    h2 = ra * ra - x * x
    if h2 < 1e-4:
        return None
    e = (b - a) / d
    perp = np.array([-e[2], 0.0, e[0]])
    p1, p2 = a + x * e + math.sqrt(h2) * perp, a + x * e - math.sqrt(h2) * perp
    return p1 if p1[2] >= p2[2] else p2


def test_fourbar_fk_matches_the_position_analysis():
    """Crank turned by the hinge coordinate delta (a rotation about +y takes the crank angle theta,
    measured in the x-z plane, to theta - delta): the coupler joints land where the circles of
    radius l2 about the crank tip and l3 about the rocker's ground pivot meet (upper branch)."""
    ws = wg.make_fourbar(num_worlds=6, seed=1)
    checked = 0
    for w in range(ws.num_worlds):
        bs, js = ws.bodies(w), ws.joints(w)
        q0 = ws.body_q0[bs]
        o, a, b, g = (_anchor(ws, q0, js.start + k) for k in range(4))
        l1, l2, l3 = np.linalg.norm(a - o), np.linalg.norm(b - a), np.linalg.norm(b - g)
        th = math.atan2(a[2] - o[2], a[0] - o[0])
        for delta in (0.15, -0.25):
            a_exp = o + l1 * np.array([math.cos(th - delta), 0.0, math.sin(th - delta)])
            b_exp = _upper_intersection(a_exp, l2, g, l3)
            if b_exp is None:                           # the linkage cannot reach this crank angle
                continue
            res = K.forward_kinematics(ws, w, q0, [delta], joints=[0])
            assert res.converged and res.iterations <= 10
            np.testing.assert_allclose(_anchor(ws, res.q, js.start + 1), a_exp, atol=1e-11)
            np.testing.assert_allclose(_anchor(ws, res.q, js.start + 2), b_exp, atol=1e-11)
            checked += 1
    assert checked >= 8


def _independent_joints(ws, w):
    """World-local joints whose coordinates are independent: the actuated ones (each loop is a
    four-bar driven through its crank) and the passive joints on no loop."""
    js = ws.joints(w)
    edges = [(int(ws.joint_parent[j]), int(ws.joint_child[j])) for j in range(js.start, js.stop)]

    def on_a_loop(skip):
        parent = {}

        def find(x):
            while parent.get(x, x) != x:
                x = parent[x]
            return x
        for k, (p, c) in enumerate(edges):
            if k != skip:
                parent[find(p)] = find(c)
        return find(edges[skip][0]) == find(edges[skip][1])

    return [k for k in range(len(edges)) if ws.joint_actuator[js.start + k] >= 0 or not on_a_loop(k)]


@pytest.mark.parametrize("w", [0, 1])
def test_biped_fk_round_trip(w):
    """Random targets on the biped's 18 independent coordinates with the pelvis held: the result
    closes every loop and meets every target, converging quadratically; FK back to the standing
    coordinates returns the standing poses."""
    ws = wg.make_biped(num_worlds=2, seed=3)
    bs = ws.bodies(w)
    q0 = ws.body_q0[bs]
    sel = _independent_joints(ws, w)
    assert len(sel) == 18
    rng = np.random.default_rng(10 + w)
    target = rng.uniform(-0.15, 0.15, len(sel))
    res = K.forward_kinematics(ws, w, q0, target, joints=sel, fixed=(0,))
    assert res.converged and res.iterations <= 6
    np.testing.assert_array_equal(res.q[0], q0[0])
    F, _ = K.residual_and_jacobian(ws, w, res.q, sel, target, list(range(1, bs.stop - bs.start)))
    assert np.abs(F).max() < 1e-12
    h = res.history
    for r0, r1 in zip(h, h[1:]):
        if 1e-7 < r0 < 0.05:
            assert r1 <= 10.0 * r0 * r0, h                  # quadratic: Gauss-Newton, zero residual
    back = K.forward_kinematics(ws, w, res.q, np.zeros(len(sel)), joints=sel, fixed=(0,))
    np.testing.assert_allclose(back.q, q0, rtol=0, atol=1e-12)


def test_fk_at_the_targets_does_not_move():
    ws = wg.make_biped(num_worlds=1, seed=3)
    q0 = ws.body_q0[ws.bodies(0)]
    sel = _independent_joints(ws, 0)
    res = K.forward_kinematics(ws, 0, q0, np.zeros(len(sel)), joints=sel, fixed=(0,))
    assert res.iterations == 0
    np.testing.assert_array_equal(res.q, q0)


def test_fk_poses_start_a_step_without_joint_bias():
    """A reset pose from FK satisfies the joints, so the first step's joint bias (beta/dt) f(q) is
    at rounding level."""
    ws = wg.make_fourbar(num_worlds=1, seed=1)
    q0 = ws.body_q0[ws.bodies(0)]
    res = K.forward_kinematics(ws, 0, q0, [0.15], joints=[0])
    st = T.WorldState(q=res.q.copy(), u=np.zeros((3, 6)), cache=[None])
    _, infos = T.step(ws, st, None, 1e-3, T.SolverParams(eps=1e-10, n_max=5000, rho=0.1))
    assert np.abs(infos[0].v_star).max() * 1e-3 / 0.2 < 1e-12
