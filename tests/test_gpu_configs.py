"""The benchmark configurations that a one-step parity test does not cover, run on the GPU as
configured and compared with the FP64 oracle:
  - 64 planar four-bars (lengths U[0.1, 0.3] m, masses U[0.1, 1] kg, gravity only, dt = 1 ms) for
    1000 steps in FP64 and FP32: the loop-closure drift and the energy of the GPU trajectory against
    the oracle's own trajectory (Sec. 3 invariants);
  - the heterogeneous set (four-bar, 6-UPS Stewart platform, excavator arm, biped) with the bipeds
    standing on the plane, in the bucketed persistent plan, under the contact-world criterion."""
import numpy as np
import pytest

import worldgen as wg
from oracle import constraints as Cn, rigid, timestep as T
from tests.test_gpu_parity import K, _biped_parity, rnd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
assert K                                 # the fixture, re-exported for this module


def _energy_and_closure(ws, q, u):
    """Per world: kinetic + potential energy (J) and the largest joint-row error |f(q)| (m, rad)."""
    E, f = np.zeros(ws.num_worlds), np.zeros(ws.num_worlds)
    g = -float(ws.gravity[2])
    for w in range(ws.num_worlds):
        bs, js = ws.bodies(w), ws.joints(w)
        r = q[bs, :3]
        R = np.array([rigid.quat_to_rot(x) for x in q[bs, 3:]])
        for i, b in enumerate(range(bs.start, bs.stop)):
            wb = R[i].T @ u[b, 3:]
            E[w] += 0.5 * ws.body_mass[b] * u[b, :3] @ u[b, :3] + 0.5 * wb @ (ws.body_inertia[b] * wb)
            E[w] += ws.body_mass[b] * g * q[b, 2]
        for j in range(js.start, js.stop):
            for row in Cn.joint_rows(int(ws.joint_type[j]), int(ws.joint_parent[j]), int(ws.joint_child[j]),
                                     ws.joint_frame_parent[j], ws.joint_frame_child[j], r, R):
                f[w] = max(f[w], abs(row[4]))
    return E, f


SAMPLE = list(range(0, 64, 8))           # the worlds the oracle follows (it steps only those)
_ORACLE = {}


def _oracle_fourbar_trajectory(ws, dt, steps):
    """Energy and loop-closure error of the sampled worlds every 10 steps of the oracle's own
    trajectory (computed once per module, shared by both precisions)."""
    if "traj" not in _ORACLE:
        ost = T.initial_state(ws)
        params = T.SolverParams(rho=0.1, eps=1e-12, n_max=20000)
        out = []
        for k in range(steps):
            ost, _ = T.step(ws, ost, None, dt, params, worlds=SAMPLE)
            if k % 10 == 9:
                E, f = _energy_and_closure(ws, ost.q, ost.u)
                out.append((E[SAMPLE], f[SAMPLE], ost.q.copy()))
        _ORACLE["traj"] = out
    return _ORACLE["traj"]


@pytest.mark.parametrize("precision,tol,e_bar", [("fp64", 1e-12, 1e-7), ("fp32", 1e-8, 1e-3)])
def test_fourbars_1000_steps_drift_and_energy(K, precision, tol, e_bar):
    """64 four-bars, 1000 steps of 1 ms from the initial state on the GPU; the oracle follows every
    eighth world on its own trajectory.  Bars from the arithmetic: FP64 solves to 1e-12 (errors of
    ~1e-12 per step, at most ~1e-9 after 1000 steps; bar 1e-7 of the energy scale), FP32 stores the
    state in FP32 (6e-8 per step, ~1e-4 after 1000 steps in the worst case; bar 1e-3).  The
    loop-closure error is the Baumgarte-stabilised drift and must match the oracle's: at most twice
    the oracle's plus the storage rounding (1e-12 / 1e-6)."""
    ws = wg.make_fourbar(num_worlds=64, seed=0)
    dt, steps = 1e-3, 1000
    traj = _oracle_fourbar_trajectory(ws, dt, steps)
    model = K.Model(ws, precision, K.make_params(rho=0.1))
    st = K.State(model)
    E0, _ = _energy_and_closure(ws, ws.body_q0, ws.body_u0)
    scale = np.abs(E0[SAMPLE]).max()
    bodies = np.concatenate([np.arange(ws.bodies(w).start, ws.bodies(w).stop) for w in SAMPLE])
    worst_e, worst_f_gpu, worst_f_orc, worst_q = 0.0, 0.0, 0.0, 0.0
    for k in range(steps):
        st.step(dt, 20000, tol, None)
        if k % 10 == 9:
            torch.cuda.synchronize()
            qg, ug = st.body_q.double().cpu().numpy(), st.body_u.double().cpu().numpy()
            Eg, fg = _energy_and_closure(ws, qg, ug)
            Eo, fo, qo = traj[k // 10]
            worst_e = max(worst_e, float(np.abs(Eg[SAMPLE] - Eo).max()))
            worst_f_gpu, worst_f_orc = max(worst_f_gpu, float(fg[SAMPLE].max())), max(worst_f_orc, float(fo.max()))
            worst_q = max(worst_q, float(np.abs(qg[bodies] - qo[bodies]).max()))
    rep = st.residuals()
    print(f"{precision}: energy scale {scale:.3f} J, max |E_gpu - E_oracle| {worst_e:.2e} J, loop-closure drift "
          f"gpu {worst_f_gpu:.2e} oracle {worst_f_orc:.2e}, max |q_gpu - q_oracle| {worst_q:.2e}, "
          f"energy change of the oracle {float(np.abs(traj[-1][0] - E0[SAMPLE]).max()):.2e} J")
    assert np.all(rep["status"] & K.WORLD_NONFINITE == 0)
    assert worst_e <= e_bar * scale
    assert worst_f_gpu <= 2.0 * worst_f_orc + (1e-12 if precision == "fp64" else 1e-6)


def test_heterogeneous_set_with_standing_bipeds_in_the_persistent_plan(K):
    """Four-bars, Stewart platforms, excavator arms and bipeds standing on the plane (3 each), one
    actuated FP32 step to 1e-8 in the bucketed persistent plan (groups of 32-256 threads pulling
    worlds from a counter), world by world under the contact-world criterion."""
    sets = [wg.make_fourbar(3, seed=4), wg.make_stewart(3, seed=4), wg.make_excavator(3, seed=4),
            wg.make_biped(3, seed=4)]
    ws = wg.concat(sets)
    assert ws.terrain_kind != wg.TERRAIN_NONE
    q, u = rnd(ws.body_q0), rnd(ws.body_u0)
    lines = _biped_parity(K, ws, q, u, wg.actuation(ws, 4, 0), 2e-3, "fp32", launch_mode=K.LAUNCH_PERSISTENT)
    assert sum(1 for ln in lines if ln["world"] >= 9) == 3
