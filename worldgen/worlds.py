"""World descriptions: seeded builders for the synthetic systems and the pin cases.

Every builder returns a :class:`WorldSet`, a flat, sum-allocated description of one or more
independent worlds (heterogeneous sets are made with :func:`concat`).  Per-world draws come from
``numpy.random.default_rng([seed, kind, w])`` so a world does not depend on how many worlds are
built beside it.  Actuation inputs for step ``k`` come from the counter-based Philox generator
keyed by ``(seed, k)``.

The builders place every body and joint at an initial pose in which all joint constraints hold
exactly; they do no dynamics.
"""
from __future__ import annotations

import copy
import math
from dataclasses import dataclass, field

import numpy as np

JOINT_REVOLUTE, JOINT_PRISMATIC, JOINT_UNIVERSAL, JOINT_SPHERICAL, JOINT_FIXED = 0, 1, 2, 3, 4
JOINT_ROWS = {JOINT_REVOLUTE: 5, JOINT_PRISMATIC: 5, JOINT_UNIVERSAL: 4, JOINT_SPHERICAL: 3,
              JOINT_FIXED: 6}
TERRAIN_NONE, TERRAIN_PLANE, TERRAIN_HEIGHTFIELD = 0, 1, 2
DRIVE_TORQUE, DRIVE_PD = 0, 1

# world-type tags (used for the stream key and for per-type bookkeeping)
KIND_PIN, KIND_FOURBAR, KIND_BIPED, KIND_STEWART, KIND_EXCAVATOR = 0, 1, 2, 3, 4
KIND_BIPED_TEAM = 5


@dataclass
class WorldSet:
    num_worlds: int
    world_type: np.ndarray            # int32 [W]
    world_body_offset: np.ndarray     # int32 [W+1]
    world_joint_offset: np.ndarray    # int32 [W+1]
    world_contact_offset: np.ndarray  # int32 [W+1]
    world_num_actuators: np.ndarray   # int32 [W]
    world_mu: np.ndarray              # f64 [W]
    body_mass: np.ndarray             # f64 [B]
    body_inertia: np.ndarray          # f64 [B,3]   principal moments
    joint_type: np.ndarray            # int32 [J]
    joint_parent: np.ndarray          # int32 [J]   body index local to the world, -1 = world
    joint_child: np.ndarray           # int32 [J]   body index local to the world
    joint_actuator: np.ndarray        # int32 [J]   slot in the world's actuation vector or -1
    joint_frame_parent: np.ndarray    # f64 [J,7]   pos(3) + quat xyzw(4) in the parent frame
    joint_frame_child: np.ndarray     # f64 [J,7]   pos(3) + quat xyzw(4) in the child frame
    contact_body: np.ndarray          # int32 [C]   body index local to the world
    contact_point: np.ndarray         # f64 [C,3]   point in the body frame
    body_q0: np.ndarray               # f64 [B,7]   r(3) + q xyzw(4)
    body_u0: np.ndarray               # f64 [B,6]   v(3) + omega(3), world frame
    gravity: np.ndarray = field(default_factory=lambda: np.array([0.0, 0.0, -9.81]))
    terrain_kind: int = TERRAIN_NONE
    hf_origin: np.ndarray = field(default_factory=lambda: np.zeros(2))
    hf_cell: float = 0.0
    hf_nx: int = 0
    hf_ny: int = 0
    hf_heights: np.ndarray = field(default_factory=lambda: np.zeros(0))  # f64 [ny*nx] row-major (j, i)
    # Joint-space dynamics (optional; None = none anywhere).  joint_drive[j] = (mode, Kp, Kd,
    # armature, damping): mode DRIVE_TORQUE takes the actuation input as a joint torque/force,
    # DRIVE_PD as the position target of an implicit PD controller (zero velocity target).
    # joint_limit[j] = (lower, upper) on the joint coordinate, +-inf for no bound.
    joint_drive: np.ndarray | None = None   # f64 [J,5]
    joint_limit: np.ndarray | None = None   # f64 [J,2]

    @property
    def n_act_max(self) -> int:
        return int(self.world_num_actuators.max()) if self.num_worlds else 0

    def bodies(self, w):
        return slice(int(self.world_body_offset[w]), int(self.world_body_offset[w + 1]))

    def joints(self, w):
        return slice(int(self.world_joint_offset[w]), int(self.world_joint_offset[w + 1]))

    def contacts(self, w):
        return slice(int(self.world_contact_offset[w]), int(self.world_contact_offset[w + 1]))

    def bilateral_rows(self, w):
        return int(sum(JOINT_ROWS[int(t)] for t in self.joint_type[self.joints(w)]))


# ----------------------------------------------------------------------------- geometry helpers
def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def _quat_to_mat(q):
    x, y, z, w = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def _mat_to_quat(m):
    """Rotation matrix -> unit quaternion (x, y, z, w), branch on the largest diagonal term."""
    t = np.trace(m)
    if t > 0:
        s = math.sqrt(t + 1.0) * 2
        q = [(m[2, 1] - m[1, 2]) / s, (m[0, 2] - m[2, 0]) / s, (m[1, 0] - m[0, 1]) / s, 0.25 * s]
    elif m[0, 0] > m[1, 1] and m[0, 0] > m[2, 2]:
        s = math.sqrt(1.0 + m[0, 0] - m[1, 1] - m[2, 2]) * 2
        q = [0.25 * s, (m[0, 1] + m[1, 0]) / s, (m[0, 2] + m[2, 0]) / s, (m[2, 1] - m[1, 2]) / s]
    elif m[1, 1] > m[2, 2]:
        s = math.sqrt(1.0 + m[1, 1] - m[0, 0] - m[2, 2]) * 2
        q = [(m[0, 1] + m[1, 0]) / s, 0.25 * s, (m[1, 2] + m[2, 1]) / s, (m[0, 2] - m[2, 0]) / s]
    else:
        s = math.sqrt(1.0 + m[2, 2] - m[0, 0] - m[1, 1]) * 2
        q = [(m[0, 2] + m[2, 0]) / s, (m[1, 2] + m[2, 1]) / s, 0.25 * s, (m[1, 0] - m[0, 1]) / s]
    q = np.array(q)
    q /= np.linalg.norm(q)
    return q if q[3] >= 0 else -q


def frame_z(axis):
    """Right-handed frame (columns e1, e2, e3) whose e3 is ``axis``."""
    e3 = _unit(axis)
    helper = np.array([1.0, 0.0, 0.0]) if abs(e3[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = _unit(np.cross(helper, e3))
    e2 = np.cross(e3, e1)
    return np.stack([e1, e2, e3], axis=1)


def frame_x(axis, up=(0.0, 0.0, 1.0)):
    """Right-handed frame whose e1 is ``axis`` (used to orient rod-like bodies)."""
    e1 = _unit(axis)
    up = np.asarray(up, dtype=np.float64)
    if abs(np.dot(up, e1)) > 0.95:
        up = np.array([0.0, 1.0, 0.0])
    e2 = _unit(np.cross(up, e1))
    e3 = np.cross(e1, e2)
    return np.stack([e1, e2, e3], axis=1)


def frame_xy(a1, a2):
    """Frame with e1 = a1 and e2 = a2 (a1 must be perpendicular to a2)."""
    e1 = _unit(a1)
    e2 = _unit(a2)
    return np.stack([e1, e2, np.cross(e1, e2)], axis=1)


def box_inertia(mass, dims):
    a, b, c = dims
    return mass / 12.0 * np.array([b * b + c * c, a * a + c * c, a * a + b * b])


# ----------------------------------------------------------------------------- one-world builder
class _World:
    def __init__(self, kind, mu=0.0):
        self.kind = kind
        self.mu = mu
        self.bodies = []      # (mass, inertia[3], pos[3], quat[4], v[3], w[3])
        self.joints = []      # (type, parent, child, fp[7], fc[7], actuator)
        self.contacts = []    # (body, point[3])
        self.n_act = 0

    def body(self, mass, dims=None, pos=(0, 0, 0), rot=None, inertia=None, v=(0, 0, 0), w=(0, 0, 0)):
        rot = np.eye(3) if rot is None else np.asarray(rot, dtype=np.float64)
        inertia = box_inertia(mass, dims) if inertia is None else np.asarray(inertia, dtype=np.float64)
        self.bodies.append((float(mass), inertia, np.asarray(pos, dtype=np.float64), _mat_to_quat(rot),
                            np.asarray(v, dtype=np.float64), np.asarray(w, dtype=np.float64)))
        return len(self.bodies) - 1

    def _local(self, body, anchor, frame):
        if body < 0:
            return np.concatenate([anchor, _mat_to_quat(frame)])
        _, _, r, q, _, _ = self.bodies[body]
        rm = _quat_to_mat(q)
        return np.concatenate([rm.T @ (anchor - r), _mat_to_quat(rm.T @ frame)])

    def joint(self, jtype, parent, child, anchor, frame, actuated=False, anchor_child=None):
        anchor = np.asarray(anchor, dtype=np.float64)
        anchor_child = anchor if anchor_child is None else np.asarray(anchor_child, dtype=np.float64)
        act = -1
        if actuated:
            act = self.n_act
            self.n_act += 1
        self.joints.append((jtype, parent, child, self._local(parent, anchor, frame),
                            self._local(child, anchor_child, frame), act))
        return len(self.joints) - 1

    def contact_box_corners(self, body, dims):
        a, b, c = (0.5 * d for d in dims)
        for sx in (-1, 1):
            for sy in (-1, 1):
                for sz in (-1, 1):
                    self.contacts.append((body, np.array([sx * a, sy * b, sz * c])))

    def contact_grid_bottom(self, body, dims, n=4):
        a, b, c = (0.5 * d for d in dims)
        for i in range(n):
            for j in range(n):
                x = -a + 2 * a * i / (n - 1)
                y = -b + 2 * b * j / (n - 1)
                self.contacts.append((body, np.array([x, y, -c])))


def _assemble(worlds, gravity=(0.0, 0.0, -9.81), terrain=None):
    W = len(worlds)
    bo = np.zeros(W + 1, np.int32)
    jo = np.zeros(W + 1, np.int32)
    co = np.zeros(W + 1, np.int32)
    for i, wd in enumerate(worlds):
        bo[i + 1] = bo[i] + len(wd.bodies)
        jo[i + 1] = jo[i] + len(wd.joints)
        co[i + 1] = co[i] + len(wd.contacts)
    B, J, C = int(bo[-1]), int(jo[-1]), int(co[-1])
    ws = WorldSet(
        num_worlds=W,
        world_type=np.array([wd.kind for wd in worlds], np.int32),
        world_body_offset=bo, world_joint_offset=jo, world_contact_offset=co,
        world_num_actuators=np.array([wd.n_act for wd in worlds], np.int32),
        world_mu=np.array([wd.mu for wd in worlds], np.float64),
        body_mass=np.zeros(B), body_inertia=np.zeros((B, 3)),
        joint_type=np.zeros(J, np.int32), joint_parent=np.zeros(J, np.int32),
        joint_child=np.zeros(J, np.int32), joint_actuator=np.zeros(J, np.int32),
        joint_frame_parent=np.zeros((J, 7)), joint_frame_child=np.zeros((J, 7)),
        contact_body=np.zeros(C, np.int32), contact_point=np.zeros((C, 3)),
        body_q0=np.zeros((B, 7)), body_u0=np.zeros((B, 6)),
        gravity=np.asarray(gravity, np.float64))
    for i, wd in enumerate(worlds):
        for k, (m, inert, r, q, v, om) in enumerate(wd.bodies):
            g = bo[i] + k
            ws.body_mass[g] = m
            ws.body_inertia[g] = inert
            ws.body_q0[g, :3] = r
            ws.body_q0[g, 3:] = q
            ws.body_u0[g, :3] = v
            ws.body_u0[g, 3:] = om
        for k, (t, p, c, fp, fc, a) in enumerate(wd.joints):
            g = jo[i] + k
            ws.joint_type[g] = t
            ws.joint_parent[g] = p
            ws.joint_child[g] = c
            ws.joint_actuator[g] = a
            ws.joint_frame_parent[g] = fp
            ws.joint_frame_child[g] = fc
        for k, (b, pt) in enumerate(wd.contacts):
            g = co[i] + k
            ws.contact_body[g] = b
            ws.contact_point[g] = pt
    if terrain is not None:
        ws.terrain_kind = terrain["kind"]
        if terrain["kind"] == TERRAIN_HEIGHTFIELD:
            ws.hf_origin = np.asarray(terrain["origin"], np.float64)
            ws.hf_cell = float(terrain["cell"])
            ws.hf_nx = int(terrain["nx"])
            ws.hf_ny = int(terrain["ny"])
            ws.hf_heights = np.asarray(terrain["heights"], np.float64).reshape(-1)
    return ws


def with_joint_drives(ws, mode, kp=0.0, kd=0.0, armature=0.0, damping=0.0, joints=None):
    """A copy of ``ws`` whose joints (default: every actuated joint) carry the given drive."""
    out = copy.copy(ws)
    drive = np.zeros((len(ws.joint_type), 5)) if ws.joint_drive is None else ws.joint_drive.copy()
    sel = np.flatnonzero(ws.joint_actuator >= 0) if joints is None else np.asarray(joints)
    drive[sel] = (mode, kp, kd, armature, damping)
    out.joint_drive = drive
    return out


def with_joint_limits(ws, lower, upper, joints=None):
    """A copy of ``ws`` whose joints (default: every revolute and prismatic joint) have bounds."""
    out = copy.copy(ws)
    lim = np.tile([-np.inf, np.inf], (len(ws.joint_type), 1)) if ws.joint_limit is None else ws.joint_limit.copy()
    if joints is None:
        joints = np.flatnonzero(np.isin(ws.joint_type, (JOINT_REVOLUTE, JOINT_PRISMATIC)))
    lim[np.asarray(joints)] = (lower, upper)
    out.joint_limit = lim
    return out


def concat(sets, terrain="auto"):
    """Concatenate world sets (same gravity, else ValueError) into one heterogeneous set.

    ``terrain="auto"`` takes the terrain of the sets whose worlds have contact candidates (they
    must agree; worlds without candidates never touch it), else the first set's.  An explicit
    TERRAIN_NONE or TERRAIN_PLANE overrides it for every world."""
    if any(s.joint_drive is not None or s.joint_limit is not None for s in sets):
        raise NotImplementedError("concat of worlds with joint drives or limits")
    if any(not np.array_equal(s.gravity, sets[0].gravity) for s in sets[1:]):
        raise ValueError("concat of sets with different gravity")
    with_contacts = [s for s in sets if int(s.world_contact_offset[-1]) > 0]
    base = with_contacts[0] if with_contacts else sets[0]
    for s in with_contacts[1:]:
        if s.terrain_kind != base.terrain_kind or not np.array_equal(s.hf_heights, base.hf_heights):
            raise ValueError("concat of sets with contact candidates on different terrains")
    kind = base.terrain_kind
    if terrain != "auto":
        if terrain not in (TERRAIN_NONE, TERRAIN_PLANE):
            raise ValueError(f"terrain override must be TERRAIN_NONE or TERRAIN_PLANE, not {terrain!r}")
        kind = terrain
    out = {}
    W = sum(s.num_worlds for s in sets)

    def offs(name):
        parts, acc = [np.zeros(1, np.int32)], 0
        for s in sets:
            o = getattr(s, name)
            parts.append((o[1:] + acc).astype(np.int32))
            acc += int(o[-1])
        return np.concatenate(parts)

    for name in ("world_body_offset", "world_joint_offset", "world_contact_offset"):
        out[name] = offs(name)
    for name in ("world_type", "world_num_actuators", "world_mu", "body_mass", "body_inertia", "joint_type",
                 "joint_parent", "joint_child", "joint_actuator", "joint_frame_parent", "joint_frame_child",
                 "contact_body", "contact_point", "body_q0", "body_u0"):
        out[name] = np.concatenate([getattr(s, name) for s in sets])
    return WorldSet(num_worlds=W, gravity=base.gravity.copy(), terrain_kind=kind,
                    hf_origin=base.hf_origin, hf_cell=base.hf_cell, hf_nx=base.hf_nx, hf_ny=base.hf_ny,
                    hf_heights=base.hf_heights, **out)


def _rng(seed, kind, w):
    return np.random.default_rng([int(seed), int(kind), int(w)])


# ----------------------------------------------------------------------------- pin cases
def make_pendulum(theta0=0.5, length=0.5, mass=1.0, width=0.02, num_worlds=1, actuated=False):
    """Compound pendulum: a rod hinged at the world origin about +y, released at rest at ``theta0``
    from the hanging position (the hinge coordinate is 0 there and grows as the rod swings
    towards hanging).  ``actuated`` gives the hinge actuation slot 0."""
    worlds = []
    for _ in range(num_worlds):
        wd = _World(KIND_PIN)
        d = np.array([math.sin(theta0), 0.0, -math.cos(theta0)])
        rod = wd.body(mass, (length, width, width), pos=0.5 * length * d, rot=frame_x(d, up=(0, 1, 0)))
        wd.joint(JOINT_REVOLUTE, -1, rod, (0, 0, 0), frame_z((0, 1, 0)), actuated=actuated)
        worlds.append(wd)
    return _assemble(worlds)


def make_free_body(mass=2.0, inertia=(0.1, 0.2, 0.3), w0=(1.0, 2.0, 3.0), v0=(0, 0, 0), gravity=(0, 0, 0)):
    """One unconstrained rigid body (no joints, no contacts)."""
    wd = _World(KIND_PIN)
    wd.body(mass, inertia=inertia, pos=(0, 0, 1.0), v=v0, w=w0)
    return _assemble([wd], gravity=gravity)


def make_box(dims=(0.2, 0.1, 0.05), mass=1.0, mu=0.5, pos=None, rot=None, v0=(0, 0, 0), w0=(0, 0, 0),
             gravity=(0, 0, -9.81), num_worlds=1, terrain=None):
    """A box with its 8 corners as contact candidates; by default resting on the plane z = 0."""
    worlds = []
    for _ in range(num_worlds):
        wd = _World(KIND_PIN, mu=mu)
        p = (0.0, 0.0, 0.5 * dims[2]) if pos is None else pos
        b = wd.body(mass, dims, pos=p, rot=rot, v=v0, w=w0)
        wd.contact_box_corners(b, dims)
        worlds.append(wd)
    return _assemble(worlds, gravity=gravity, terrain=terrain or {"kind": TERRAIN_PLANE})


# ----------------------------------------------------------------------------- four-bar (x-z plane)
def _circle_intersection_up(a, ra, b, rb):
    """Intersection of circle(a, ra) and circle(b, rb) in the x-z plane with the larger z, plus the
    half-chord length (0 when the circles do not meet)."""
    d = np.linalg.norm(b - a)
    if d < 1e-9 or d > ra + rb or d < abs(ra - rb):
        return None, 0.0
    x = (ra * ra - rb * rb + d * d) / (2 * d)
    h = math.sqrt(max(ra * ra - x * x, 0.0))
    e = (b - a) / d
    perp = np.array([-e[2], 0.0, e[0]])
    p1, p2 = a + x * e + h * perp, a + x * e - h * perp
    return (p1 if p1[2] >= p2[2] else p2), h


def _rod(wd, mass, p0, p1, width=0.02):
    d = p1 - p0
    return wd.body(mass, (float(np.linalg.norm(d)), width, width), pos=0.5 * (p0 + p1),
                   rot=frame_x(d, up=(0, 1, 0)))


def make_fourbar(num_worlds=64, seed=0):
    """Planar four-bar: ground + crank, coupler, rocker, closed by four revolute joints about +y.

    Link lengths U[0.1, 0.3] m, masses U[0.1, 1] kg, crank angle U[0, 2 pi); the loop is closed on
    the branch with the higher coupler-rocker joint, redrawing until the circles meet with a
    half-chord of at least 1 cm.  Gravity only, no contacts, no actuators.
    """
    worlds = []
    hinge = frame_z((0, 1, 0))
    for w in range(num_worlds):
        rng = _rng(seed, KIND_FOURBAR, w)
        while True:
            lg, l1, l2, l3 = rng.uniform(0.1, 0.3, size=4)
            m1, m2, m3 = rng.uniform(0.1, 1.0, size=3)
            th = rng.uniform(0.0, 2 * math.pi)
            o = np.zeros(3)
            g = np.array([lg, 0.0, 0.0])
            a = o + l1 * np.array([math.cos(th), 0.0, math.sin(th)])
            b, h = _circle_intersection_up(a, l2, g, l3)
            if b is not None and h > 0.01:
                break
        wd = _World(KIND_FOURBAR)
        crank = _rod(wd, m1, o, a)
        coupler = _rod(wd, m2, a, b)
        rocker = _rod(wd, m3, g, b)
        wd.joint(JOINT_REVOLUTE, -1, crank, o, hinge)
        wd.joint(JOINT_REVOLUTE, crank, coupler, a, hinge)
        wd.joint(JOINT_REVOLUTE, coupler, rocker, b, hinge)
        wd.joint(JOINT_REVOLUTE, -1, rocker, g, hinge)
        worlds.append(wd)
    return _assemble(worlds)


# ----------------------------------------------------------------------------- biped
BIPED_FOOT_DIMS = (0.20, 0.10, 0.04)


def _biped_world(rng, kind=KIND_BIPED, foot_points="corners", z_lift=0.0):
    """Synthetic closed-loop biped: 31 bodies, 36 revolute joints (12 actuated), 6 loops.

    Per leg (15 bodies, 18 joints): hip yaw / roll / pitch in series (actuated); a knee
    parallelogram four-bar on the thigh whose rocker is the shank; an ankle four-bar on the shank
    whose rocker is the ankle link; a passive ankle-roll link; a foot four-bar on the ankle-roll
    link whose rocker is the foot box; a two-segment passive toe.  Every four-bar adds three bodies
    and four joints and is driven through its crank joint (actuated).
    """
    mu = rng.uniform(0.5, 1.0)
    wd = _World(kind, mu=mu)
    light = lambda: 10.0 * 10.0 ** (-rng.uniform(2.0, 3.0))   # 0.01 .. 0.1 kg
    mid = lambda: rng.uniform(0.2, 0.6)
    heavy = lambda: rng.uniform(0.8, 2.0)
    y_hinge, x_hinge, z_hinge = frame_z((0, 1, 0)), frame_z((1, 0, 0)), frame_z((0, 0, 1))
    zp = 0.97 + z_lift
    pelvis = wd.body(10.0, (0.20, 0.30, 0.10), pos=(0, 0, zp))
    ez = np.array([0.0, 0.0, 1.0])
    ex = np.array([1.0, 0.0, 0.0])
    for side in (1.0, -1.0):
        H = np.array([0.0, 0.1 * side, zp - 0.05])
        hip_yaw = wd.body(light(), (0.05, 0.05, 0.05), pos=H - 0.03 * ez)
        wd.joint(JOINT_REVOLUTE, pelvis, hip_yaw, H, z_hinge, actuated=True)
        hip_roll = wd.body(light(), (0.05, 0.05, 0.05), pos=H - 0.08 * ez)
        wd.joint(JOINT_REVOLUTE, hip_yaw, hip_roll, H - 0.055 * ez, x_hinge, actuated=True)
        thigh = wd.body(heavy(), (0.05, 0.05, 0.30), pos=H - 0.26 * ez)
        wd.joint(JOINT_REVOLUTE, hip_roll, thigh, H - 0.11 * ez, y_hinge, actuated=True)

        def fourbar(ground, o1, o2, crank_dir, crank_len, rocker_mass, rocker_dims, rocker_center,
                    hinge=y_hinge):
            a = o1 + crank_len * crank_dir
            b = o2 + crank_len * crank_dir
            crank = wd.body(light(), (crank_len, 0.02, 0.02), pos=0.5 * (o1 + a))
            coupler = wd.body(light(), (0.02, 0.02, float(np.linalg.norm(b - a))), pos=0.5 * (a + b))
            rocker = wd.body(rocker_mass, rocker_dims, pos=rocker_center)
            wd.joint(JOINT_REVOLUTE, ground, crank, o1, hinge, actuated=True)
            wd.joint(JOINT_REVOLUTE, crank, coupler, a, hinge)
            wd.joint(JOINT_REVOLUTE, coupler, rocker, b, hinge)
            wd.joint(JOINT_REVOLUTE, ground, rocker, o2, hinge)   # loop closure
            return rocker

        o2k = H - 0.40 * ez
        shank = fourbar(thigh, H - 0.15 * ez, o2k, ex, 0.06, heavy(), (0.05, 0.05, 0.30), o2k - 0.15 * ez)
        o2a = o2k - 0.30 * ez
        ankle = fourbar(shank, o2k - 0.06 * ez, o2a, -ex, 0.05, mid(), (0.04, 0.04, 0.10), o2a - 0.05 * ez)
        o_roll = o2a - 0.10 * ez
        ankle_roll = wd.body(mid(), (0.06, 0.08, 0.06), pos=o_roll - 0.03 * ez)
        wd.joint(JOINT_REVOLUTE, ankle, ankle_roll, o_roll, x_hinge)
        fc = o_roll + np.array([0.02, 0.0, -0.10])          # foot centre; foot top at o_roll - 0.08
        foot = fourbar(ankle_roll, o_roll - 0.01 * ez + np.array([0.0, 0.03 * side, 0.0]),
                       o_roll - 0.07 * ez + np.array([0.0, 0.03 * side, 0.0]), np.array([0.0, 0.0, 0.0]) + ex,
                       0.04, mid(), BIPED_FOOT_DIMS, fc)
        toe1 = wd.body(light(), (0.03, 0.10, 0.02), pos=fc + np.array([0.115, 0.0, -0.01]))
        wd.joint(JOINT_REVOLUTE, foot, toe1, fc + np.array([0.10, 0.0, -0.01]), y_hinge)
        toe2 = wd.body(light(), (0.03, 0.10, 0.02), pos=fc + np.array([0.145, 0.0, -0.01]))
        wd.joint(JOINT_REVOLUTE, toe1, toe2, fc + np.array([0.13, 0.0, -0.01]), y_hinge)
        if foot_points == "corners":
            wd.contact_box_corners(foot, BIPED_FOOT_DIMS)
        else:
            wd.contact_grid_bottom(foot, BIPED_FOOT_DIMS, n=4)
    return wd


def make_biped(num_worlds=4096, seed=0, terrain=None, foot_points="corners", z_lift=0.0):
    """Config of 4096 closed-loop bipeds standing on the plane (bottom foot corners at z = 0).

    Friction mu ~ U[0.5, 1] per world; pelvis 10 kg, thigh/shank 0.8-2 kg, ankle/foot 0.2-0.6 kg,
    small links 0.01-0.1 kg (mass ratio up to 1000).
    """
    worlds = [_biped_world(_rng(seed, KIND_BIPED, w), foot_points=foot_points, z_lift=z_lift)
              for w in range(num_worlds)]
    return _assemble(worlds, terrain=terrain or {"kind": TERRAIN_PLANE})


def _biped_team_world(seed, w, per_world, spacing=1.0):
    """``per_world`` bipeds side by side (x offsets of ``spacing`` m) in one world: one large system
    of independent mechanisms (31 k bodies, 180 k joint rows, 16 k foot-corner candidates).  Each
    biped is drawn from its own stream; the world keeps the first one's friction."""
    team = _World(KIND_BIPED_TEAM)
    for i in range(per_world):
        wd = _biped_world(_rng(seed, KIND_BIPED_TEAM, per_world * w + i))
        if i == 0:
            team.mu = wd.mu
        nb0, act0 = len(team.bodies), team.n_act
        for (m, inertia, pos, quat, v, om) in wd.bodies:
            team.bodies.append((m, inertia, pos + np.array([spacing * i, 0.0, 0.0]), quat, v, om))
        for (jt, par, ch, fp, fc, act) in wd.joints:
            # every biped joint joins two of its own bodies (the pelvis floats), so the body-local
            # frames move with the bodies
            assert par >= 0
            team.joints.append((jt, par + nb0, ch + nb0, fp, fc, act + act0 if act >= 0 else -1))
        for (b, pt) in wd.contacts:
            team.contacts.append((b + nb0, pt))
        team.n_act += wd.n_act
    return team


def make_biped_team(num_worlds=1024, seed=0, per_world=2):
    """Large worlds for the sparse formulation: ``per_world`` closed-loop bipeds standing side by side
    in every world (2: 62 bodies, 360 joint rows, up to 456 rows; 4: up to 912 rows), on the plane."""
    worlds = [_biped_team_world(seed, w, per_world) for w in range(num_worlds)]
    return _assemble(worlds, terrain={"kind": TERRAIN_PLANE})


def make_biped_heightfield(num_worlds=16384, seed=0, hmax=0.05):
    """Bipeds on a seeded 64 x 64 heightfield (heights U[0, hmax], 1/32 m cells): 4 x 4 sample
    points under each foot (32 candidates per world, up to 276 rows), pelvis raised by hmax so the
    feet start above the terrain."""
    hf = make_heightfield(seed=seed, hmax=hmax)
    return make_biped(num_worlds=num_worlds, seed=seed, terrain=hf, foot_points="grid", z_lift=hmax)


# ----------------------------------------------------------------------------- Stewart platform
def _stewart_world(rng):
    wd = _World(KIND_STEWART)
    rb, rp, leg = 0.3, 0.2, 0.5
    pmass = rng.uniform(2.0, 5.0)
    base_pts, plat_pts = [], []
    for k in range(3):
        for s in (-1, 1):
            ab = math.radians(120 * k + 15 * s)
            ap = math.radians(120 * k + 45 * s)
            base_pts.append(np.array([rb * math.cos(ab), rb * math.sin(ab), 0.0]))
            plat_pts.append(np.array([rp * math.cos(ap), rp * math.sin(ap), 0.0]))
    dh = np.linalg.norm(base_pts[0][:2] - plat_pts[0][:2])
    hgt = math.sqrt(leg * leg - dh * dh)
    zc = hgt
    platform = wd.body(pmass, (0.45, 0.45, 0.04), pos=(0, 0, zc))
    for b, p in zip(base_pts, plat_pts):
        p = p + np.array([0.0, 0.0, zc])
        ell = _unit(p - b)
        lower = wd.body(rng.uniform(0.5, 1.0), (0.30, 0.04, 0.04), pos=b + 0.15 * ell, rot=frame_x(ell))
        upper = wd.body(rng.uniform(0.1, 0.5), (0.30, 0.03, 0.03), pos=p - 0.15 * ell, rot=frame_x(ell))
        t = _unit(np.cross(np.array([0.0, 0.0, 1.0]), ell))
        wd.joint(JOINT_UNIVERSAL, -1, lower, b, frame_xy(t, np.cross(ell, t)))
        wd.joint(JOINT_PRISMATIC, lower, upper, 0.5 * (b + p), frame_z(ell), actuated=True,
                 anchor_child=0.5 * (b + p))
        wd.joint(JOINT_SPHERICAL, upper, platform, p, np.eye(3))
    return wd


def make_stewart(num_worlds=2048, seed=0):
    """6-UPS Stewart platform: base radius 0.3 m, platform radius 0.2 m, legs 0.5 m; 13 bodies,
    18 joints (U base, actuated P, S platform), 72 rows."""
    return _assemble([_stewart_world(_rng(seed, KIND_STEWART, w)) for w in range(num_worlds)])


# ----------------------------------------------------------------------------- excavator arm
def _excavator_world(rng):
    wd = _World(KIND_EXCAVATOR)
    hinge = frame_z((0, 1, 0))
    ob = np.array([0.0, 0.0, 0.5])
    e1 = ob + np.array([1.0, 0.0, 0.5])
    e2 = e1 + np.array([0.6, 0.0, -0.6])
    e3 = e2 + np.array([0.2, 0.0, -0.2])
    boom = _rod(wd, rng.uniform(5.0, 10.0), ob, e1, width=0.08)
    stick = _rod(wd, rng.uniform(3.0, 6.0), e1, e2, width=0.06)
    bucket = _rod(wd, rng.uniform(1.0, 3.0), e2, e3, width=0.05)
    wd.joint(JOINT_REVOLUTE, -1, boom, ob, hinge)
    wd.joint(JOINT_REVOLUTE, boom, stick, e1, hinge)
    wd.joint(JOINT_REVOLUTE, stick, bucket, e2, hinge)
    lift = np.array([0.0, 0.0, 0.08])
    cylinders = [(-1, np.array([0.3, 0.0, 0.2]), boom, ob + 0.5 * (e1 - ob) - lift),
                 (boom, ob + 0.6 * (e1 - ob) + lift, stick, e1 + 0.3 * (e2 - e1) + lift),
                 (stick, e1 + 0.5 * (e2 - e1) + lift, bucket, e2 + 0.5 * (e3 - e2) + lift)]
    for body_a, pa, body_b, pb in cylinders:
        ell = _unit(pb - pa)
        dist = float(np.linalg.norm(pb - pa))
        mid = 0.5 * (pa + pb)
        barrel = wd.body(rng.uniform(0.5, 1.0), (0.6 * dist, 0.04, 0.04), pos=pa + 0.3 * dist * ell,
                         rot=frame_x(ell, up=(0, 1, 0)))
        rod = wd.body(rng.uniform(0.2, 0.5), (0.6 * dist, 0.03, 0.03), pos=pb - 0.3 * dist * ell,
                      rot=frame_x(ell, up=(0, 1, 0)))
        wd.joint(JOINT_REVOLUTE, body_a, barrel, pa, hinge)
        wd.joint(JOINT_PRISMATIC, barrel, rod, mid, frame_z(ell), actuated=True)
        wd.joint(JOINT_REVOLUTE, rod, body_b, pb, hinge)
    return wd


def make_excavator(num_worlds=2048, seed=0):
    """Planar excavator-style arm on a fixed base: boom, stick, bucket and three hydraulic
    cylinders (barrel + rod, R-P-R each); 9 bodies, 12 joints, 60 rows, 3 loops."""
    return _assemble([_excavator_world(_rng(seed, KIND_EXCAVATOR, w)) for w in range(num_worlds)])


# ----------------------------------------------------------------------------- terrain
def make_heightfield(seed=0, n=64, cell=1.0 / 32.0, hmax=0.05, origin=(-1.0, -1.0)):
    """Heightfield terrain: ``n`` x ``n`` vertices ``cell`` apart, heights U[0, hmax]."""
    rng = np.random.default_rng([int(seed), 99])
    return {"kind": TERRAIN_HEIGHTFIELD, "origin": np.asarray(origin, np.float64), "cell": cell, "nx": n,
            "ny": n, "heights": rng.uniform(0.0, hmax, size=(n, n))}


# ----------------------------------------------------------------------------- inputs and checks
def actuation(ws: WorldSet, seed: int, step: int, sigma: float = 5.0) -> np.ndarray:
    """Gaussian actuation (N m or N) for step ``step``: float64 [W, n_act_max], zero in unused slots.
    Drawn from the counter-based Philox stream keyed by (seed, step)."""
    gen = np.random.Generator(np.random.Philox(key=[int(seed) & (2**64 - 1), int(step) & (2**64 - 1)]))
    na = max(ws.n_act_max, 1)
    tau = sigma * gen.standard_normal((ws.num_worlds, na))
    mask = np.arange(na)[None, :] < ws.world_num_actuators[:, None]
    return np.where(mask, tau, 0.0)


def count_loops(ws: WorldSet, w: int) -> int:
    """Independent loops of world ``w``'s joint graph: joints - nodes + components (world = node)."""
    nb = ws.world_body_offset[w + 1] - ws.world_body_offset[w]
    parent = list(range(nb + 1))     # node nb is the world

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    js = ws.joints(w)
    used_world = False
    for p, c in zip(ws.joint_parent[js], ws.joint_child[js]):
        p = nb if p < 0 else p
        used_world |= p == nb
        ra, rb = find(p), find(c)
        if ra != rb:
            parent[ra] = rb
    nodes = nb + (1 if used_world else 0)
    comps = len({find(i) for i in range(nodes)})
    nj = js.stop - js.start
    return nj - nodes + comps
