"""Joint and contact constraints: rows of the Jacobian J and the bias v* (Sec. 3), FP64.

Test infrastructure only (see ``oracle/__init__``).

A row is returned as ``(body_a, Ja, body_b, Jb, f)``: the two 1x6 blocks acting on the twists
(v, omega) of the two bodies (``body_a = -1`` for the world, whose block is dropped) and the
position-level error f(q) used by the Baumgarte bias.  J u is the rate of change of f to first
order, so the bias ``v* = (beta / dt) f`` makes ``J u+ = -v*`` shrink the error by (1 - beta).

Row layouts (frame axes a1, a2, a3 of the parent-side joint frame, b1, b2, b3 of the child side,
anchors p_A, p_B, lever arms c_A = p_A - r_A, c_B = p_B - r_B):

* positional rows, world axes e_k:      f = e_k.(p_B - p_A),    J_B = [e_k, c_B x e_k],
                                                                J_A = [-e_k, -(c_A x e_k)]
* revolute (hinge a3): 3 positional rows + rows k = 1, 2:  f = a_k.(a3 x b3),  J = [0, +-a_k]
* prismatic (slide a3): rows along a1, a2:  f = a_k.(p_B - p_A), J_B = [a_k, c_B x a_k],
  J_A = [-a_k, -((p_B - r_A) x a_k)]; then 3 rotation rows  f = a_k . 1/2 sum_i (a_i x b_i),
  J = [0, +-a_k]
* universal (free about a1 and b2): 3 positional rows + f = a1.b2,  J_A = [0, a1 x b2],
  J_B = [0, -(a1 x b2)]
* spherical: 3 positional rows;  fixed: 3 positional rows + the 3 prismatic rotation rows.

Contacts (Sec. 3, Signorini-Coulomb-Newton): rows (t1, t2, n) with the branchless orthonormal
basis of Duff et al. 2017 built from the terrain normal n; J_b = [d, c x d] for d in (t1, t2, n).

Joint-space dynamics (Sec. 3, Eq. 2's R and v*): the joint coordinate d(q) of a revolute or
prismatic joint and its row J_d (J_d u = d-dot), one regularised row per driven joint for
implicit PD, armature and viscous damping (``drive_row``), and unilateral joint-limit rows whose
bias follows the contact normal's (``unilateral_bias``).
"""
from __future__ import annotations

import math

import numpy as np

from .rigid import quat_to_rot

REVOLUTE, PRISMATIC, UNIVERSAL, SPHERICAL, FIXED = 0, 1, 2, 3, 4
ROWS = {REVOLUTE: 5, PRISMATIC: 5, UNIVERSAL: 4, SPHERICAL: 3, FIXED: 6}
_E = np.eye(3)


def _frames(parent, child, fp, fc, r, R):
    """World anchors, lever arms and frame axes of a joint at configuration (r, R)."""
    if parent < 0:
        rA, RA = np.zeros(3), np.eye(3)
    else:
        rA, RA = r[parent], R[parent]
    rB, RB = r[child], R[child]
    pA = rA + RA @ fp[:3]
    pB = rB + RB @ fc[:3]
    FA = RA @ quat_to_rot(fp[3:])
    FB = RB @ quat_to_rot(fc[3:])
    return rA, pA, pA - rA, FA, rB, pB, pB - rB, FB


def joint_rows(jtype, parent, child, fp, fc, r, R):
    rA, pA, cA, FA, rB, pB, cB, FB = _frames(parent, child, fp, fc, r, R)
    a = [FA[:, 0], FA[:, 1], FA[:, 2]]
    b = [FB[:, 0], FB[:, 1], FB[:, 2]]
    rows = []

    def lin(d, lever_a):
        Ja = np.concatenate([-d, -np.cross(lever_a, d)])
        Jb = np.concatenate([d, np.cross(cB, d)])
        return Ja, Jb

    def ang(d):
        return np.concatenate([np.zeros(3), -d]), np.concatenate([np.zeros(3), d])

    if jtype in (REVOLUTE, UNIVERSAL, SPHERICAL, FIXED):
        for k in range(3):
            Ja, Jb = lin(_E[k], cA)
            rows.append((Ja, Jb, float(_E[k] @ (pB - pA))))
    if jtype == REVOLUTE:
        err = np.cross(a[2], b[2])
        for k in range(2):
            Ja, Jb = ang(a[k])
            rows.append((Ja, Jb, float(a[k] @ err)))
    elif jtype == PRISMATIC:
        for k in range(2):
            Ja, Jb = lin(a[k], pB - rA)
            rows.append((Ja, Jb, float(a[k] @ (pB - pA))))
    if jtype in (PRISMATIC, FIXED):
        err = 0.5 * sum(np.cross(a[i], b[i]) for i in range(3))
        for k in range(3):
            Ja, Jb = ang(a[k])
            rows.append((Ja, Jb, float(a[k] @ err)))
    if jtype == UNIVERSAL:
        n = np.cross(a[0], b[1])
        rows.append((np.concatenate([np.zeros(3), n]), np.concatenate([np.zeros(3), -n]),
                     float(a[0] @ b[1])))
    assert len(rows) == ROWS[jtype]
    return [(parent, Ja, child, Jb, f) for Ja, Jb, f in rows]


def joint_coordinate(jtype, parent, child, fp, fc, r, R):
    """The joint coordinate d(q) and its row J_d (J_d u = d-dot): for a revolute the angle of the
    child frame about the hinge a3, measured from a1 towards a2, d = atan2(a2.b1, a1.b1); for a
    prismatic the slide d = a3.(p_B - p_A).  Drives and limits act on it (Sec. 3).
    Returns (d, Ja, Jb)."""
    rA, pA, cA, FA, rB, pB, cB, FB = _frames(parent, child, fp, fc, r, R)
    a1, a2, a3 = FA[:, 0], FA[:, 1], FA[:, 2]
    if jtype == REVOLUTE:
        b1 = FB[:, 0]
        d = math.atan2(float(a2 @ b1), float(a1 @ b1))
        Ja = np.concatenate([np.zeros(3), -a3])
        Jb = np.concatenate([np.zeros(3), a3])
    elif jtype == PRISMATIC:
        d = float(a3 @ (pB - pA))
        Ja = np.concatenate([-a3, -np.cross(pB - rA, a3)])
        Jb = np.concatenate([a3, np.cross(cB, a3)])
    else:
        raise ValueError("only revolute and prismatic joints have a joint coordinate")
    return d, Ja, Jb


def actuation_wrench(jtype, parent, child, fp, fc, r, R, value):
    """Generalised force of a joint actuator: J_d^T value for the joint coordinate d (rotation about
    the hinge a3 for a revolute, slide along a3 for a prismatic).  Returns {body: wrench[6]}."""
    if jtype not in (REVOLUTE, PRISMATIC):
        raise ValueError("only revolute and prismatic joints carry actuators")
    _, Ja, Jb = joint_coordinate(jtype, parent, child, fp, fc, r, R)
    out = {}
    if parent >= 0:
        out[parent] = value * Ja
    out[child] = out.get(child, 0.0) + value * Jb
    return out


# ----------------------------------------------------------------------------- contacts
def orthonormal_basis(n):
    """Duff et al. 2017, 'Building an Orthonormal Basis, Revisited': (t1, t2) with (t1, t2, n)
    right-handed."""
    sign = math.copysign(1.0, n[2])
    a = -1.0 / (sign + n[2])
    b = n[0] * n[1] * a
    t1 = np.array([1.0 + sign * n[0] * n[0] * a, sign * b, -sign * n[0]])
    t2 = np.array([b, sign + n[1] * n[1] * a, -n[1]])
    return t1, t2


def terrain_query(ws, p):
    """Signed distance phi of world point p to the terrain and the terrain normal there.

    Plane: z = 0, normal +z.  Heightfield: vertices (x0 + i h, y0 + j h, H[j, i]); every cell is
    split along the diagonal from vertex (i, j) to (i+1, j+1); the point's (x, y) is clamped into
    the grid; phi is the distance to the plane of the triangle under it, along its normal.
    """
    if ws.terrain_kind == 1:
        return float(p[2]), np.array([0.0, 0.0, 1.0])
    h = ws.hf_cell
    nx, ny = ws.hf_nx, ws.hf_ny
    H = ws.hf_heights.reshape(ny, nx)
    gx = min(max((p[0] - ws.hf_origin[0]) / h, 0.0), nx - 1.0)
    gy = min(max((p[1] - ws.hf_origin[1]) / h, 0.0), ny - 1.0)
    i = min(int(math.floor(gx)), nx - 2)
    j = min(int(math.floor(gy)), ny - 2)
    fx, fy = gx - i, gy - j

    def vert(ii, jj):
        return np.array([ws.hf_origin[0] + ii * h, ws.hf_origin[1] + jj * h, H[jj, ii]])

    v00, v11 = vert(i, j), vert(i + 1, j + 1)
    if fx >= fy:
        v1 = vert(i + 1, j)
        n = np.cross(v1 - v00, v11 - v00)
    else:
        v1 = vert(i, j + 1)
        n = np.cross(v11 - v00, v1 - v00)
    n = n / np.linalg.norm(n)
    q = np.array([ws.hf_origin[0] + gx * h, ws.hf_origin[1] + gy * h, p[2]])
    return float((q - v00) @ n), n


def contacts(ws, w, r, R):
    """Active contacts of world w: candidates with phi < margin, in candidate order.
    Returns a list of (candidate_index, body, point_world, normal, phi)."""
    out = []
    cs = ws.contacts(w)
    for k, (b, pt) in enumerate(zip(ws.contact_body[cs], ws.contact_point[cs])):
        p = r[b] + R[b] @ pt
        phi, n = terrain_query(ws, p)
        out.append((k, int(b), p, n, phi))
    return out


def contact_rows(body, p, n, rb):
    """Rows (t1, t2, n) of one contact on ``body``: J_b = [d, c x d], c = p - r_b."""
    t1, t2 = orthonormal_basis(n)
    c = p - rb
    return [(-1, None, body, np.concatenate([d, np.cross(c, d)]), 0.0) for d in (t1, t2, n)]


def contact_bias(phi, beta, dt):
    """Bias of the rows (t1, t2, n) of an active contact at signed distance ``phi`` (Sec. 3): none
    on the friction rows; on the normal row phi/dt while the point is still apart (phi > 0, the
    gap may close within the step but no further) and Baumgarte's beta phi/dt once it penetrates."""
    return [0.0, 0.0, (phi if phi > 0 else beta * phi) / dt]


def drive_row(d, d_dot, target, dt, kp, kd, armature, damping):
    """Joint-space dynamics on the joint coordinate as one regularised row (Sec. 3, Eq. 2's R and
    v*).  The row's impulse over the step is the armature's inertial reaction plus dt times the
    implicit PD and damping forces, all taken at the end-of-step rate d-dot+ = J_d u+ and the
    semi-implicit end pose d + dt d-dot+:
        lambda = I_a (d-dot- - d-dot+) + dt Kp (target - d - dt d-dot+) - dt (Kd + b) d-dot+,
    i.e. J_d u+ + lambda / C + v* = 0 with C = I_a + dt^2 Kp + dt (Kd + b) and
    v* = -(I_a d-dot- + dt Kp (target - d)) / C.  Returns (R, v*), or None when C = 0."""
    C = armature + dt * dt * kp + dt * (kd + damping)
    if C <= 0.0:
        return None
    return 1.0 / C, -(armature * d_dot + dt * kp * (target - d)) / C


def unilateral_bias(g, beta, dt):
    """Bias of a unilateral row g(q) >= 0 (a joint limit): like a contact's normal row, the gap
    may close within the step (g/dt while g > 0) and a violation is removed at Baumgarte's rate
    (beta g/dt once g <= 0)."""
    return (g if g > 0 else beta * g) / dt
