"""GPU parity of the Gauss-Newton forward kinematics for resets (Sec. 6.3, kamino_fk) against the
oracle's (oracle.kinematics) and the closed forms that pin it: the four-bar's position analysis
(circle intersection), the biped's round trip through random targets on its 18 independent
coordinates, a target the mechanism cannot reach, and FP32 storage."""
import math

import numpy as np
import pytest

import worldgen as wg
from oracle import kinematics as KN
from tests.test_gpu_parity import K
from tests.test_oracle_kinematics import _anchor, _independent_joints, _upper_intersection

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
assert K                                 # the fixture, re-exported for this module


def _fk(K, ws, precision, targets, select=None, fixed=None, q=None, iters=50, tol=1e-12):
    """FK on every world from `q` (default: the model's initial poses); returns (poses, report).  The
    model takes the sparse formulation's working set: FK has its own, and an FP64 biped's dense step
    does not fit in shared memory."""
    model = K.Model(ws, precision, K.make_params(cr_iters=9))
    st = K.State(model)
    if q is not None:
        st.body_q.copy_(torch.tensor(q.reshape(-1, 7), dtype=st.dtype))
    dev = lambda a, dt: None if a is None else torch.tensor(np.asarray(a), dtype=dt, device="cuda").contiguous()
    st.fk(dev(targets, torch.float64), dev(select, torch.int32), dev(fixed, torch.int32), iters, tol)
    torch.cuda.synchronize()
    return st.body_q.double().cpu().numpy(), st.residuals()


def test_fourbar_fk_matches_the_position_analysis(K):
    """Cranks turned by delta in 6 four-bars (FP64): the coupler joints land where the circles of
    radius l2 about the crank tip and l3 about the rocker's ground pivot meet (upper branch)."""
    ws = wg.make_fourbar(num_worlds=6, seed=1)
    J = len(ws.joint_type)
    for delta in (0.15, -0.25):
        targets = np.zeros(J)
        select = np.zeros(J, np.int32)
        for w in range(ws.num_worlds):
            targets[ws.joints(w).start] = delta
            select[ws.joints(w).start] = 1
        qg, rep = _fk(K, ws, "fp64", targets, select)
        checked = 0
        for w in range(ws.num_worlds):
            bs, js = ws.bodies(w), ws.joints(w)
            q0 = ws.body_q0[bs]
            o, a, b, g = (_anchor(ws, q0, js.start + k) for k in range(4))
            l1, l2, l3 = np.linalg.norm(a - o), np.linalg.norm(b - a), np.linalg.norm(b - g)
            th = math.atan2(a[2] - o[2], a[0] - o[0])
            a_exp = o + l1 * np.array([math.cos(th - delta), 0.0, math.sin(th - delta)])
            b_exp = _upper_intersection(a_exp, l2, g, l3)
            if b_exp is None:
                assert rep["status"][w] & K.WORLD_NOT_CONVERGED
                continue
            assert rep["status"][w] == 0 and rep["iterations"][w] <= 10, (w, rep["iterations"][w])
            np.testing.assert_allclose(_anchor(ws, qg[bs], js.start + 1), a_exp, atol=1e-11)
            np.testing.assert_allclose(_anchor(ws, qg[bs], js.start + 2), b_exp, atol=1e-11)
            checked += 1
        assert checked >= 4


def test_biped_fk_round_trip_matches_the_oracle(K):
    """4 bipeds, random targets U(-0.15, 0.15) rad on the 18 independent coordinates, pelvis held
    (FP64): every loop closes and every target is met (max |F| < 1e-12) in at most 8 iterations, the
    poses equal the oracle's FK, and FK back to the standing coordinates returns the standing poses."""
    ws = wg.make_biped(num_worlds=4, seed=3)
    J, B = len(ws.joint_type), int(ws.world_body_offset[-1])
    targets, select, fixed = np.zeros(J), np.zeros(J, np.int32), np.zeros(B, np.int32)
    rng = np.random.default_rng(10)
    per_world = []
    for w in range(ws.num_worlds):
        sel = _independent_joints(ws, w)
        t = rng.uniform(-0.15, 0.15, len(sel))
        js = ws.joints(w)
        targets[[js.start + k for k in sel]] = t
        select[[js.start + k for k in sel]] = 1
        fixed[ws.bodies(w).start] = 1
        per_world.append((sel, t))
    qg, rep = _fk(K, ws, "fp64", targets, select, fixed)
    print("FK iterations:", rep["iterations"].tolist(), "max |F|:", rep["r_primal"].tolist())
    assert np.all(rep["status"] == 0) and np.all(rep["iterations"] <= 8)
    assert np.all(rep["num_rows"] == 180 + 18)
    for w, (sel, t) in enumerate(per_world):
        bs = ws.bodies(w)
        ref = KN.forward_kinematics(ws, w, ws.body_q0[bs], t, joints=sel, fixed=(0,))
        assert ref.converged
        np.testing.assert_allclose(qg[bs], ref.q, rtol=0, atol=1e-10)
        F, _ = KN.residual_and_jacobian(ws, w, qg[bs], sel, t, list(range(1, bs.stop - bs.start)))
        assert np.abs(F).max() < 1e-11
    back, rep2 = _fk(K, ws, "fp64", np.zeros(J), select, fixed, q=qg)
    assert np.all(rep2["status"] == 0)
    np.testing.assert_allclose(back, ws.body_q0, rtol=0, atol=1e-11)


def test_fk_at_the_targets_takes_no_iteration(K):
    """The standing poses with every actuated coordinate at its standing value (0): no step."""
    ws = wg.make_biped(num_worlds=2, seed=3)
    J = len(ws.joint_type)
    qg, rep = _fk(K, ws, "fp64", np.zeros(J), tol=1e-9)
    assert np.all(rep["iterations"] == 0) and np.all(rep["status"] == 0)
    np.testing.assert_array_equal(qg, ws.body_q0)


def test_unreachable_target_reports_non_convergence(K):
    """A crank angle at which the four-bar's circles do not meet: the residual cannot vanish, the
    world reports KAMINO_WORLD_NOT_CONVERGED with max |F| > 0 and keeps finite poses (a diverging
    step is undone)."""
    ws = wg.make_fourbar(num_worlds=1, seed=1)
    J = len(ws.joint_type)
    found = None
    q0 = ws.body_q0[ws.bodies(0)]
    o, a, b, g = (_anchor(ws, q0, k) for k in range(4))
    l1, l2, l3 = np.linalg.norm(a - o), np.linalg.norm(b - a), np.linalg.norm(b - g)
    th = math.atan2(a[2] - o[2], a[0] - o[0])
    for delta in np.linspace(0.0, 2 * math.pi, 721)[1:]:
        a_exp = o + l1 * np.array([math.cos(th - delta), 0.0, math.sin(th - delta)])
        dd = np.linalg.norm(g - a_exp)
        if dd > l2 + l3 + 0.01 or dd < abs(l2 - l3) - 0.01:
            found = delta
            break
    if found is None:
        pytest.skip("this four-bar reaches every crank angle")
    targets = np.zeros(J)
    targets[0] = found
    select = np.zeros(J, np.int32)
    select[0] = 1
    qg, rep = _fk(K, ws, "fp64", targets, select, iters=30)
    assert rep["status"][0] & K.WORLD_NOT_CONVERGED
    assert rep["iterations"][0] <= 30 and rep["r_primal"][0] > 1e-6
    assert np.isfinite(qg).all()


def test_fk_in_fp32_storage(K):
    """FP32 state: the iteration runs on FP64 poses on chip and only the result is stored in FP32, so
    the same biped targets converge (1e-11) and the stored poses are the FP64 result rounded."""
    ws = wg.make_biped(num_worlds=2, seed=3)
    J, B = len(ws.joint_type), int(ws.world_body_offset[-1])
    targets, select, fixed = np.zeros(J), np.zeros(J, np.int32), np.zeros(B, np.int32)
    rng = np.random.default_rng(11)
    for w in range(ws.num_worlds):
        sel = _independent_joints(ws, w)
        js = ws.joints(w)
        targets[[js.start + k for k in sel]] = rng.uniform(-0.15, 0.15, len(sel))
        select[[js.start + k for k in sel]] = 1
        fixed[ws.bodies(w).start] = 1
    q64, _ = _fk(K, ws, "fp64", targets, select, fixed)
    q32, rep = _fk(K, ws, "fp32", targets, select, fixed, tol=1e-11)
    assert np.all(rep["status"] == 0), (rep["status"], rep["r_primal"])
    assert np.abs(q32 - q64).max() < 1e-6
