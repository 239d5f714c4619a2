"""Rigid-body kinematics and dynamics in maximal coordinates (Sec. 3, Eq. 1), FP64.

Test infrastructure only (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np


def quat_mul(a, b):
    """Hamilton product a (x) b of quaternions stored (x, y, z, w)."""
    ax, ay, az, aw = a
    bx, by, bz, bw = b
    return np.array([aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw,
                     aw * bw - ax * bx - ay * by - az * bz])


def quat_to_rot(q):
    """Rotation matrix R of the rotation the quaternion (x, y, z, w) stands for: v_world = R v_body.
    The quaternion is normalised first, so a stored state whose norm drifted by rounding maps to
    the rotation it represents."""
    x, y, z, w = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    return np.array([
        [w * w + x * x - y * y - z * z, 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), w * w - x * x + y * y - z * z, 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), w * w - x * x - y * y + z * z]])


def quat_exp(theta):
    """Unit quaternion of the rotation vector ``theta`` (angle |theta| about theta/|theta|)."""
    ang = float(np.linalg.norm(theta))
    if ang == 0.0:
        return np.array([0.0, 0.0, 0.0, 1.0])
    axis = theta / ang
    return np.concatenate([np.sin(0.5 * ang) * axis, [np.cos(0.5 * ang)]])


def skew(c):
    return np.array([[0.0, -c[2], c[1]], [c[2], 0.0, -c[0]], [-c[1], c[0], 0.0]])


def mass_matrix_block(mass, inertia_diag, R):
    """Eq. 1: M_i = diag(m_i I_3, R_i I_i^b R_i^T) (6x6), twist ordered (v, omega)."""
    M = np.zeros((6, 6))
    M[:3, :3] = mass * np.eye(3)
    M[3:, 3:] = R @ np.diag(inertia_diag) @ R.T
    return M


def newton_euler_h(mass, inertia_diag, R, omega, gravity, force=None, torque=None):
    """h = [m g + f_ext ; tau_ext - omega x (I_w omega)]: gravity, external and gyroscopic terms
    (Sec. 3, equations of motion M du/dt = h + J^T lambda), evaluated at the start of the step."""
    Iw = R @ np.diag(inertia_diag) @ R.T
    f = mass * np.asarray(gravity, dtype=np.float64)
    t = -np.cross(omega, Iw @ omega)
    if force is not None:
        f = f + force
    if torque is not None:
        t = t + torque
    return np.concatenate([f, t])


def integrate_pose(r, q, v_plus, w_plus, dt):
    """Semi-implicit Euler (Sec. 3): r+ = r + dt v+, q+ = exp(dt w+) (x) q, renormalised.
    The angular velocity is in the world frame, hence the left product."""
    r_new = r + dt * v_plus
    q_new = quat_mul(quat_exp(dt * w_plus), q)
    return r_new, q_new / np.linalg.norm(q_new)
