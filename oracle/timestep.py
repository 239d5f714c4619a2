"""One time step of a set of worlds (Sec. 3 and Sec. 4), FP64, world by world.

Test infrastructure only (see ``oracle/__init__``).

Per world, in the paper's order:
  1. body kinematics, M (Eq. 1), h, u_free = u^- + dt M^-1 h
  2. contacts with the terrain (candidates with phi below the margin) and joint rows: J, v*;
     when the world carries them, drive rows (R, v*) and the active joint limits
  3. D = J M^-1 J^T + R and v_f (Eq. 4), Jacobi scaling P (Sec. 4.1)
  4. warm start from the cached lambda* (Sec. 4.1), matched by row for joints and by
     (body, candidate point) for contacts
  5. Proximal-ADMM, Alg. 1, returning lambda = P y~ (dense factorisation, or the matrix-free
     operator with Conjugate Residual x-steps of Sec. 5.1)
  6. u+ = u_free + M^-1 J^T lambda (the solution of Eq. 2), then poses by the exponential map
     (semi-implicit Euler, or the Moreau-Jean midpoint scheme: see ``step``).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import constraints as C
from . import padmm as PA
from .rigid import integrate_pose, mass_matrix_block, newton_euler_h, quat_to_rot

DRIVE_PD = 1                    # joint_drive mode whose actuation input is a position target


@dataclass
class SolverParams:
    eta: float = 1e-6           # proximal regularisation (scaled units)
    rho: float = 1.0            # augmented-Lagrangian penalty (scaled units)
    beta: float = 0.2           # Baumgarte factor
    margin: float = 0.005       # contact activation distance (m)
    eps: float = 1e-6           # residual tolerance (Sec. 4.1)
    n_max: int = 200            # iteration cap
    nesterov: bool = True
    precond: bool = True
    warm: str = "cold"          # "cold" | "cached"
    cr_iters: int | None = None # None: dense D, factorised once (Sec. 5.1's dense formulation);
                                # k: matrix-free D with k Conjugate Residual iterations per x-step
    integrator: str = "euler"   # "euler": semi-implicit Euler | "midpoint": Moreau-Jean (Sec. 3)


@dataclass
class WorldState:
    q: np.ndarray               # [B,7] r + quat xyzw
    u: np.ndarray               # [B,6] v + omega (world)
    cache: list = field(default_factory=list)   # per world: (lambda_bilateral, {candidate: lambda3})


def initial_state(ws):
    return WorldState(q=ws.body_q0.copy(), u=ws.body_u0.copy(),
                      cache=[None] * ws.num_worlds)


@dataclass
class WorldInfo:
    m: int
    n_bilateral: int
    contact_ids: list
    iterations: int
    r_p: float
    r_d: float
    r_c: float
    converged: bool
    lam: np.ndarray             # physical impulses, rows in solver order
    J: np.ndarray
    v_star: np.ndarray
    u_free: np.ndarray
    Minv: np.ndarray
    D: np.ndarray
    v_f: np.ndarray
    p: np.ndarray
    mu: np.ndarray
    u_plus: np.ndarray
    reg: np.ndarray | None = None   # R of Eq. 4 per row (None: all zero)
    unilateral: list = field(default_factory=list)  # rows whose set is R+ (joint limits)


def build_world(ws, w, q, u, tau, dt, params):
    """Steps 1-3 for world w at configuration q (rows of the world only). Returns a dict."""
    bs = ws.bodies(w)
    nb = bs.stop - bs.start
    r = q[bs, :3]
    R = np.array([quat_to_rot(q[bs.start + i, 3:]) for i in range(nb)])
    mass = ws.body_mass[bs]
    inertia = ws.body_inertia[bs]
    n = 6 * nb

    # actuation: generalised joint forces J_d^T tau (joints whose drive is a PD controller take
    # their input as a position target instead, through a drive row below)
    wrench = np.zeros((nb, 6))
    js = ws.joints(w)
    drive = ws.joint_drive[js] if ws.joint_drive is not None else None
    pd_mode = [drive is not None and int(drive[k, 0]) == DRIVE_PD for k in range(js.stop - js.start)]
    for k, (jt, par, ch, fp, fc, act) in enumerate(zip(ws.joint_type[js], ws.joint_parent[js], ws.joint_child[js],
                                                       ws.joint_frame_parent[js], ws.joint_frame_child[js],
                                                       ws.joint_actuator[js])):
        if act >= 0 and tau is not None and not pd_mode[k]:
            for b, wr in C.actuation_wrench(int(jt), int(par), int(ch), fp, fc, r, R, float(tau[act])).items():
                wrench[b] += wr

    # Eq. 1 and h; u_free = u + dt M^-1 h
    Minv = np.zeros((n, n))
    u_free = np.zeros(n)
    for i in range(nb):
        Mi = mass_matrix_block(mass[i], inertia[i], R[i])
        Mi_inv = np.linalg.inv(Mi)
        Minv[6 * i:6 * i + 6, 6 * i:6 * i + 6] = Mi_inv
        h = newton_euler_h(mass[i], inertia[i], R[i], u[bs.start + i, 3:], ws.gravity,
                           force=wrench[i, :3], torque=wrench[i, 3:])
        u_free[6 * i:6 * i + 6] = u[bs.start + i] + dt * (Mi_inv @ h)

    # rows: joints (in joint order), then drive rows, then active joint limits (in joint order,
    # lower before upper), then active contacts (in candidate order)
    rows, bias = [], []
    for jt, par, ch, fp, fc in zip(ws.joint_type[js], ws.joint_parent[js], ws.joint_child[js],
                                   ws.joint_frame_parent[js], ws.joint_frame_child[js]):
        for row in C.joint_rows(int(jt), int(par), int(ch), fp, fc, r, R):
            rows.append(row)
            bias.append(params.beta / dt * row[4])
    n_fixed = len(rows)
    reg = [0.0] * n_fixed
    uvel = u[bs]

    def coord(k):
        j = js.start + k
        par, ch = int(ws.joint_parent[j]), int(ws.joint_child[j])
        d, Ja, Jb = C.joint_coordinate(int(ws.joint_type[j]), par, ch, ws.joint_frame_parent[j],
                                       ws.joint_frame_child[j], r, R)
        d_dot = float(Jb @ uvel[ch]) + (float(Ja @ uvel[par]) if par >= 0 else 0.0)
        return par, ch, d, d_dot, Ja, Jb

    if drive is not None:
        for k in range(js.stop - js.start):
            _, kp, kd, arm, damp = drive[k]
            if kp == 0.0 and kd == 0.0 and arm == 0.0 and damp == 0.0:
                continue
            par, ch, d, d_dot, Ja, Jb = coord(k)
            act = int(ws.joint_actuator[js.start + k])
            target = float(tau[act]) if (pd_mode[k] and tau is not None and act >= 0) else d
            if not pd_mode[k]:
                kp = kd = 0.0                       # torque mode: the input is applied as a force
            row = C.drive_row(d, d_dot, target, dt, kp, kd, arm, damp)
            if row is None:
                continue
            rows.append((par, Ja, ch, Jb, 0.0))
            reg.append(row[0])
            bias.append(row[1])
    n_fixed = len(rows)
    unilateral, limit_ids = [], []
    if ws.joint_limit is not None:
        for k in range(js.stop - js.start):
            lo, hi = ws.joint_limit[js.start + k]
            if not (np.isfinite(lo) or np.isfinite(hi)):
                continue
            par, ch, d, _, Ja, Jb = coord(k)
            for side, g, sgn in ((0, d - lo, 1.0), (1, hi - d, -1.0)):
                if np.isfinite(g) and g < params.margin:
                    unilateral.append(len(rows))
                    limit_ids.append((k, side))
                    rows.append((par, sgn * Ja, ch, sgn * Jb, 0.0))
                    reg.append(0.0)
                    bias.append(C.unilateral_bias(g, params.beta, dt))
    n_bilateral = len(rows)
    contact_ids = []
    if ws.terrain_kind != 0:
        for k, b, p, nrm, phi in C.contacts(ws, w, r, R):
            if phi < params.margin:
                contact_ids.append(k)
                for row in C.contact_rows(b, p, nrm, r[b]):
                    rows.append(row)
                bias.extend(C.contact_bias(phi, params.beta, dt))
    m = len(rows)
    J = np.zeros((m, n))
    for i, (ba, Ja, bb, Jb, _) in enumerate(rows):
        if ba >= 0:
            J[i, 6 * ba:6 * ba + 6] += Ja
        J[i, 6 * bb:6 * bb + 6] += Jb
    v_star = np.array(bias)
    mu = np.full(len(contact_ids), ws.world_mu[w])
    reg = np.array(reg + [0.0] * (m - n_bilateral))
    return dict(J=J, Minv=Minv, u_free=u_free, v_star=v_star, n_bilateral=n_bilateral,
                contact_ids=contact_ids, mu=mu, r=r, R=R, nb=nb, n_fixed=n_fixed,
                reg=reg if reg.any() else None, unilateral=unilateral, limit_ids=limit_ids)


def solve_world(ws, w, q, u, tau, dt, params, cache=None):
    """Steps 1-6 for world w.  Returns (u_plus [nb,6], WorldInfo, new cache entry)."""
    B = build_world(ws, w, q, u, tau, dt, params)
    J, Minv, u_free, v_star = B["J"], B["Minv"], B["u_free"], B["v_star"]
    nbil, cids, mu = B["n_bilateral"], B["contact_ids"], B["mu"]
    reg, uni, n_fixed = B["reg"], B["unilateral"], B["n_fixed"]
    m = J.shape[0]
    D = PA.delassus(J, Minv, reg)
    v_f = PA.free_velocity(J, u_free, v_star)
    if params.cr_iters is None:
        p = PA.jacobi_scaling(D, nbil, len(cids), params.precond)
        Ds = p[:, None] * D * p[None, :]
        apply_Ds = Ds.__matmul__
    else:                       # the solve sees only the operator and diag(D), never D itself
        p = PA.jacobi_scaling(PA.delassus_diagonal(J, Minv, reg), nbil, len(cids), params.precond)
        Ds = apply_Ds = PA.delassus_matrix_free(J, Minv, p, reg)
    vs = p * v_f
    mus = mu.copy()
    for k in range(len(cids)):
        i = nbil + 3 * k
        mus[k] = mu[k] * p[i + 2] / p[i]

    x0 = z0 = None
    if params.warm == "cached" and cache is not None and m:
        lam0 = np.zeros(m)
        lam0[:n_fixed] = cache[0]
        limits = cache[2] if len(cache) > 2 else {}
        for i, key in zip(uni, B["limit_ids"]):
            lam0[i] = limits.get(key, 0.0)
        for k, cid in enumerate(cids):
            if cid in cache[1]:
                lam0[nbil + 3 * k:nbil + 3 * k + 3] = cache[1][cid]
        x0 = lam0 / p
        v0 = apply_Ds(x0) + vs
        z0 = v0 + PA.desaxce(v0, nbil, mus)

    res = PA.padmm(Ds, vs, nbil, mus, params.eta, params.rho, params.eps, params.n_max, x0=x0, z0=z0,
                   nesterov=params.nesterov, cr_iters=params.cr_iters, unilateral=uni)
    lam = p * res.y
    u_plus = u_free + Minv @ (J.T @ lam)
    new_cache = (lam[:n_fixed].copy(), {cid: lam[nbil + 3 * k:nbil + 3 * k + 3].copy() for k, cid in enumerate(cids)})
    if uni:
        new_cache = new_cache + ({key: float(lam[i]) for i, key in zip(uni, B["limit_ids"])},)
    info = WorldInfo(m=m, n_bilateral=nbil, contact_ids=cids, iterations=res.iterations, r_p=res.r_p,
                     r_d=res.r_d, r_c=res.r_c, converged=res.converged, lam=lam, J=J, v_star=v_star,
                     u_free=u_free, Minv=Minv, D=D, v_f=v_f, p=p, mu=mu, u_plus=u_plus, reg=reg,
                     unilateral=list(uni))
    return u_plus.reshape(-1, 6), info, new_cache


def step(ws, state: WorldState, tau, dt, params: SolverParams, worlds=None):
    """Advance the given worlds (default: all) by dt.  ``tau`` is [W, n_act_max] or None.
    Returns (new WorldState, list of WorldInfo for the stepped worlds).

    Semi-implicit Euler (Sec. 3): everything is evaluated at q^-, then q+ = q^- (+) dt u+.
    Moreau-Jean midpoint (Sec. 3, after Jean 1999): the poses first move half a step with the
    old velocity, q_m = q^- (+) (dt/2) u^-; kinematics, M, h, the rows, the contacts and their
    biases are evaluated at q_m, Eq. 2 gives u+ over the whole step, and q+ = q_m (+) (dt/2) u+.
    (+) is r + dt v for positions and exp(dt w) (x) q for orientations."""
    midpoint = params.integrator == "midpoint"
    if not midpoint and params.integrator != "euler":
        raise ValueError(f"unknown integrator {params.integrator!r}")
    q_new = state.q.copy()
    u_new = state.u.copy()
    cache = list(state.cache)
    infos = []
    for w in (range(ws.num_worlds) if worlds is None else worlds):
        bs = ws.bodies(w)
        q_eval = state.q
        if midpoint:
            q_eval = state.q.copy()
            for g in range(bs.start, bs.stop):
                r_m, q_m = integrate_pose(state.q[g, :3], state.q[g, 3:], state.u[g, :3], state.u[g, 3:], 0.5 * dt)
                q_eval[g, :3] = r_m
                q_eval[g, 3:] = q_m
        u_plus, info, cache[w] = solve_world(ws, w, q_eval, state.u, None if tau is None else tau[w], dt,
                                             params, cache[w])
        h_pose = 0.5 * dt if midpoint else dt
        for i in range(bs.stop - bs.start):
            g = bs.start + i
            u_new[g] = u_plus[i]
            r1, q1 = integrate_pose(q_eval[g, :3], q_eval[g, 3:], u_plus[i, :3], u_plus[i, 3:], h_pose)
            q_new[g, :3] = r1
            q_new[g, 3:] = q1
        infos.append(info)
    return WorldState(q=q_new, u=u_new, cache=cache), infos


def simulate(ws, state, dt, steps, params, tau_fn=None, worlds=None, callback=None):
    """Run ``steps`` steps; ``tau_fn(k)`` gives the actuation of step k (or None)."""
    for k in range(steps):
        state, infos = step(ws, state, None if tau_fn is None else tau_fn(k), dt, params, worlds=worlds)
        if callback is not None:
            callback(k, state, infos)
    return state
