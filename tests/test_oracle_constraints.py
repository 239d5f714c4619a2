"""Pins of the oracle's constraint layer (Sec. 3): Jacobians against finite differences of f(q),
contact frames, terrain queries and actuation by virtual work."""
import math

import numpy as np
import pytest

import worldgen as wg
from worldgen.worlds import _World, _assemble, frame_z, frame_xy, frame_x
from oracle import constraints as C, rigid


def _two_body_world(jtype, rng, parent_is_world=False):
    wd = _World(wg.worlds.KIND_PIN)
    rot = lambda: rigid.quat_to_rot(rng.standard_normal(4) / np.linalg.norm(rng.standard_normal(4)))

    def rrot():
        q = rng.standard_normal(4)
        return rigid.quat_to_rot(q / np.linalg.norm(q))

    a = wd.body(1.0, (0.3, 0.2, 0.1), pos=rng.standard_normal(3) * 0.3, rot=rrot())
    b = wd.body(0.5, (0.2, 0.1, 0.1), pos=rng.standard_normal(3) * 0.3, rot=rrot())
    anchor = rng.standard_normal(3) * 0.2
    if jtype == C.UNIVERSAL:
        a1 = rng.standard_normal(3)
        a1 /= np.linalg.norm(a1)
        a2 = np.cross(a1, rng.standard_normal(3))
        frame = frame_xy(a1, a2)
    else:
        frame = frame_z(rng.standard_normal(3))
    wd.joint(jtype, -1 if parent_is_world else a, b, anchor, frame)
    return _assemble([wd])


def _state(ws):
    r = ws.body_q0[:, :3].copy()
    R = np.array([rigid.quat_to_rot(q) for q in ws.body_q0[:, 3:]])
    return r, R


def _advance(r, R, u, h):
    r2 = r + h * u[:, :3]
    R2 = np.array([rigid.quat_to_rot(rigid.quat_exp(h * u[i, 3:])) @ R[i] for i in range(len(r))])
    return r2, R2


def _f_and_J(ws, r, R):
    rows = C.joint_rows(int(ws.joint_type[0]), int(ws.joint_parent[0]), int(ws.joint_child[0]),
                        ws.joint_frame_parent[0], ws.joint_frame_child[0], r, R)
    nb = len(r)
    J = np.zeros((len(rows), 6 * nb))
    for i, (ba, Ja, bb, Jb, _) in enumerate(rows):
        if ba >= 0:
            J[i, 6 * ba:6 * ba + 6] += Ja
        J[i, 6 * bb:6 * bb + 6] += Jb
    return np.array([row[4] for row in rows]), J


@pytest.mark.parametrize("jtype", [C.REVOLUTE, C.PRISMATIC, C.UNIVERSAL, C.SPHERICAL, C.FIXED])
@pytest.mark.parametrize("world_parent", [False, True])
def test_joint_jacobian_is_derivative_of_error(jtype, world_parent):
    """J u = d f(q(t)) / dt at a configuration that satisfies the joint (central differences along
    random twists).  Catches a wrong sign, lever arm or axis in any row."""
    rng = np.random.default_rng(10 + jtype)
    ws = _two_body_world(jtype, rng, world_parent)
    r, R = _state(ws)
    f0, J = _f_and_J(ws, r, R)
    np.testing.assert_allclose(f0, 0.0, atol=1e-12)
    assert J.shape[0] == C.ROWS[jtype]
    for _ in range(5):
        u = rng.standard_normal((2, 6))
        h = 1e-6
        fp, _ = _f_and_J(ws, *_advance(r, R, u, h))
        fm, _ = _f_and_J(ws, *_advance(r, R, u, -h))
        np.testing.assert_allclose((fp - fm) / (2 * h), J @ u.reshape(-1), atol=1e-7)


@pytest.mark.parametrize("jtype", [C.REVOLUTE, C.PRISMATIC])
def test_joint_rows_have_joint_nullspace(jtype):
    """The free motion of the joint (rotation about the hinge / slide along the axis, applied to the
    child about / along the anchor) lies in the null space of J."""
    rng = np.random.default_rng(3)
    ws = _two_body_world(jtype, rng)
    r, R = _state(ws)
    _, J = _f_and_J(ws, r, R)
    axis = R[0] @ rigid.quat_to_rot(ws.joint_frame_parent[0, 3:])[:, 2]
    anchor = r[0] + R[0] @ ws.joint_frame_parent[0, :3]
    u = np.zeros((2, 6))
    if jtype == C.REVOLUTE:
        u[1, 3:] = axis
        u[1, :3] = np.cross(axis, r[1] - anchor)
    else:
        u[1, :3] = axis
    np.testing.assert_allclose(J @ u.reshape(-1), 0.0, atol=1e-12)


def test_actuation_is_virtual_work_of_joint_coordinate():
    """A revolute torque does work tau (w_B - w_A).a3; a prismatic force f does f d/dt(slide); both
    wrenches are internal (zero net force and zero net moment about the origin)."""
    rng = np.random.default_rng(4)
    for jtype in (C.REVOLUTE, C.PRISMATIC):
        ws = _two_body_world(jtype, rng)
        r, R = _state(ws)
        wr = C.actuation_wrench(jtype, 0, 1, ws.joint_frame_parent[0], ws.joint_frame_child[0], r, R, 2.5)
        W = np.zeros((2, 6))
        for b, w in wr.items():
            W[b] = w
        np.testing.assert_allclose(W[0, :3] + W[1, :3], 0.0, atol=1e-12)
        moment = sum(W[b, 3:] + np.cross(r[b], W[b, :3]) for b in range(2))
        np.testing.assert_allclose(moment, 0.0, atol=1e-12)
        a3 = R[0] @ rigid.quat_to_rot(ws.joint_frame_parent[0, 3:])[:, 2]
        u = rng.standard_normal((2, 6))
        if jtype == C.REVOLUTE:
            rate = a3 @ (u[1, 3:] - u[0, 3:])
        else:
            pB = r[1] + R[1] @ ws.joint_frame_child[0, :3]
            pA = r[0] + R[0] @ ws.joint_frame_parent[0, :3]
            h = 1e-6
            d = lambda rr, RR: (RR[0] @ rigid.quat_to_rot(ws.joint_frame_parent[0, 3:])[:, 2]) @ (
                (rr[1] + RR[1] @ ws.joint_frame_child[0, :3]) - (rr[0] + RR[0] @ ws.joint_frame_parent[0, :3]))
            rate = (d(*_advance(r, R, u, h)) - d(*_advance(r, R, u, -h))) / (2 * h)
        assert abs(np.sum(W * u) - 2.5 * rate) < 1e-6


def test_orthonormal_basis():
    rng = np.random.default_rng(5)
    normals = [np.array([0, 0, 1.0]), np.array([0, 0, -1.0]), np.array([1.0, 0, 0])]
    normals += [v / np.linalg.norm(v) for v in rng.standard_normal((30, 3))]
    for n in normals:
        t1, t2 = C.orthonormal_basis(n)
        F = np.stack([t1, t2, n], axis=1)
        np.testing.assert_allclose(F.T @ F, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(F) - 1.0) < 1e-12


def test_heightfield_query():
    """Flat heightfield -> phi = z - h0; a sloped heightfield z = a x + b y (exactly representable by
    the triangles) -> phi = signed distance to that plane; points outside the grid are clamped."""
    class HF:
        terrain_kind = wg.TERRAIN_HEIGHTFIELD
        hf_origin = np.array([-1.0, -1.0])
        hf_cell = 0.1
        hf_nx = 21
        hf_ny = 21

    hf = HF()
    xs = hf.hf_origin[0] + hf.hf_cell * np.arange(21)
    ys = hf.hf_origin[1] + hf.hf_cell * np.arange(21)
    hf.hf_heights = np.full((21, 21), 0.03).reshape(-1)
    phi, n = C.terrain_query(hf, np.array([0.123, -0.456, 0.2]))
    assert abs(phi - 0.17) < 1e-12 and np.allclose(n, [0, 0, 1])
    a, b = 0.2, -0.1
    hf.hf_heights = (a * xs[None, :] + b * ys[:, None]).reshape(-1)
    nrm = np.array([-a, -b, 1.0]) / math.sqrt(a * a + b * b + 1)
    rng = np.random.default_rng(6)
    for _ in range(20):
        p = np.array([rng.uniform(-0.95, 0.95), rng.uniform(-0.95, 0.95), rng.uniform(-0.5, 0.5)])
        phi, n = C.terrain_query(hf, p)
        np.testing.assert_allclose(n, nrm, atol=1e-12)
        assert abs(phi - (p[2] - a * p[0] - b * p[1]) * nrm[2]) < 1e-12
    phi_out, _ = C.terrain_query(hf, np.array([5.0, 0.0, 1.0]))
    phi_edge, _ = C.terrain_query(hf, np.array([1.0, 0.0, 1.0]))
    assert abs(phi_out - phi_edge) < 1e-12


def test_contact_rows_are_point_velocity():
    """Contact rows (t1, t2, n) times the twist = contact-point velocity in the contact frame."""
    rng = np.random.default_rng(7)
    q = rng.standard_normal(4)
    R = rigid.quat_to_rot(q / np.linalg.norm(q))
    rb = rng.standard_normal(3)
    p = rb + rng.standard_normal(3) * 0.1
    n = rng.standard_normal(3)
    n /= np.linalg.norm(n)
    rows = C.contact_rows(0, p, n, rb)
    u = rng.standard_normal(6)
    vp = u[:3] + np.cross(u[3:], p - rb)
    t1, t2 = C.orthonormal_basis(n)
    np.testing.assert_allclose([row[3] @ u for row in rows], [t1 @ vp, t2 @ vp, n @ vp], atol=1e-12)
