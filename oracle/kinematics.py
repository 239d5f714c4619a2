"""Forward kinematics for resets: consistent body poses from joint coordinates (Sec. 6.3, the
Gauss-Newton FK solver used to reset mechanisms with kinematic loops), FP64.

Test infrastructure only (see ``oracle/__init__``).

Given target values for the coordinates of a chosen set of joints (hinge angles, slides) and a
set of bodies held fixed (the floating base), find the poses of the other bodies such that every
joint constraint holds, f(q) = 0, and every chosen coordinate takes its target.  Gauss-Newton on
the residual F(q) = [f(q); d_sel(q) - d_target]: each iteration linearises F with the constraint
rows J (the same rows the dynamics use; J u is the rate of f) and the joint-coordinate rows, takes
the least-squares step of minimum norm, delta = -J_F^+ F (the loops make rows redundant and a
partial selection leaves directions free), and moves the poses along it, r += delta_v and
q = exp(delta_w) (x) q, as the integrator does.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import constraints as C
from .rigid import quat_exp, quat_mul, quat_to_rot


@dataclass
class FKResult:
    q: np.ndarray               # [nb, 7] poses of the world's bodies
    iterations: int
    residual: float             # max |F| at the returned poses
    history: list               # max |F| before each iteration, then at the end
    converged: bool


def _wrap(a):
    """Angle difference wrapped into (-pi, pi]."""
    return a - 2.0 * math.pi * math.floor((a + math.pi) / (2.0 * math.pi))


def residual_and_jacobian(ws, w, q, joints, targets, free):
    """F(q) and its rows with respect to the twists of the free bodies (columns 6 per free body)."""
    js = ws.joints(w)
    nb = q.shape[0]
    r = q[:, :3]
    R = np.array([quat_to_rot(q[i, 3:]) for i in range(nb)])
    col = {b: 6 * k for k, b in enumerate(free)}
    F, rows = [], []

    def add(par, Ja, ch, Jb, value):
        row = np.zeros(6 * len(free))
        if par >= 0 and par in col:
            row[col[par]:col[par] + 6] += Ja
        if ch in col:
            row[col[ch]:col[ch] + 6] += Jb
        rows.append(row)
        F.append(value)

    for j in range(js.start, js.stop):
        for par, Ja, ch, Jb, f in C.joint_rows(int(ws.joint_type[j]), int(ws.joint_parent[j]),
                                               int(ws.joint_child[j]), ws.joint_frame_parent[j],
                                               ws.joint_frame_child[j], r, R):
            add(par, Ja, ch, Jb, f)
    for j, target in zip(joints, targets):
        g = js.start + j
        par, ch = int(ws.joint_parent[g]), int(ws.joint_child[g])
        d, Ja, Jb = C.joint_coordinate(int(ws.joint_type[g]), par, ch, ws.joint_frame_parent[g],
                                       ws.joint_frame_child[g], r, R)
        diff = _wrap(d - target) if int(ws.joint_type[g]) == C.REVOLUTE else d - target
        add(par, Ja, ch, Jb, diff)
    return np.array(F), np.array(rows).reshape(len(F), 6 * len(free))


def forward_kinematics(ws, w, q_start, targets, joints=None, fixed=(), tol=1e-12, max_iters=50):
    """Gauss-Newton FK for world ``w`` from the poses ``q_start`` ([nb, 7], the world's bodies).
    ``joints`` are world-local joint indices (default: the actuated ones) with coordinate targets
    ``targets``; ``fixed`` lists world-local bodies that keep their poses (a floating base)."""
    js = ws.joints(w)
    if joints is None:
        joints = [k for k in range(js.stop - js.start) if ws.joint_actuator[js.start + k] >= 0]
    q = np.array(q_start, dtype=np.float64)
    free = [b for b in range(q.shape[0]) if b not in set(fixed)]
    history = []
    it = 0
    for it in range(max_iters + 1):
        F, Jf = residual_and_jacobian(ws, w, q, joints, targets, free)
        res = float(np.max(np.abs(F))) if F.size else 0.0
        history.append(res)
        if res < tol or it == max_iters:
            break
        delta, *_ = np.linalg.lstsq(Jf, -F, rcond=1e-12)
        for k, b in enumerate(free):
            dv, dw = delta[6 * k:6 * k + 3], delta[6 * k + 3:6 * k + 6]
            q[b, :3] += dv
            qr = quat_mul(quat_exp(dw), q[b, 3:])
            q[b, 3:] = qr / np.linalg.norm(qr)
    return FKResult(q=q, iterations=it, residual=history[-1], history=history, converged=history[-1] < tol)
