"""GPU parity of the time-stepping and joint-space options of Sec. 3 against the FP64 oracle:
the Moreau-Jean midpoint scheme, the joint-space dynamics rows (implicit PD, armature and viscous
damping as Eq. 2's R and v*, Eq. 4's D + R) and unilateral joint limits, in both formulations.
Bars as elsewhere: FP64 <= 1e-9, FP32 <= 1e-4 on worlds whose answer is unique; contact worlds
under the contact-world criterion."""
import math

import numpy as np
import pytest

import worldgen as wg
from tests.test_gpu_parity import (K, _biped_case, _biped_parity, _margin_clear, check_report, errors, gpu_step,
                                   oracle_step, rnd)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
assert K                                 # the fixture, re-exported for this module

MID = 1                                  # KAMINO_INTEGRATOR_MIDPOINT


def _run(K, ws, steps, dt, precision, tol, tau_fn=None, pkw=None, okw=None, require_converged=True):
    """`steps` GPU steps, each compared with the oracle started from the GPU state; returns the worst
    (err_u, err_q) and the last reports.  Bipeds in the air drift off their redundant loops within a
    few steps, after which the dual residual has a floor (reading of redundant rows) and neither side
    reaches a tight tolerance; their u+ is still unique, so `require_converged=False` checks u+ and
    the pose increment only."""
    q, u = rnd(ws.body_q0, precision), rnd(ws.body_u0, precision)
    model = K.Model(ws, precision, K.make_params(rho=0.1, **(pkw or {})))
    worst = (0.0, 0.0)
    for k in range(steps):
        tau = None if tau_fn is None else tau_fn(k)
        qg, ug, rep, _ = gpu_step(K, ws, q, u, tau, dt, 20000, tol, precision, model=model)
        ref, infos = oracle_step(ws, q, u, tau, dt, eps=1e-12, **(okw or {}))
        check_report(rep, infos)
        if require_converged:
            assert np.all(rep["status"] == 0), rep["status"]
        assert np.all(rep["status"] & K.WORLD_NONFINITE == 0)
        eu, eq = errors(q, qg, ug, ref.q, ref.u, dt, precision)
        worst = (max(worst[0], eu), max(worst[1], eq))
        q, u = qg, ug
    return worst, rep, infos


# ----------------------------------------------------------------------------- midpoint
@pytest.mark.parametrize("cr", [0, 9])
@pytest.mark.parametrize("precision,bar,tol", [("fp64", 1e-9, 1e-12), ("fp32", 1e-4, 1e-8)])
def test_midpoint_fourbars(K, precision, bar, tol, cr):
    """64 four-bars with the Moreau-Jean midpoint scheme, 10 steps of 1 ms (dense and sparse)."""
    ws = wg.make_fourbar(num_worlds=64, seed=0)
    okw = dict(integrator="midpoint", cr_iters=cr or None)
    (eu, eq), _, _ = _run(K, ws, 10, 1e-3, precision, tol, pkw=dict(integrator=MID, cr_iters=cr), okw=okw)
    print(f"midpoint four-bars ({precision}, cr {cr}): err_u {eu:.2e}, err_q {eq:.2e}")
    assert eu <= bar and eq <= bar


def test_midpoint_bipeds_in_the_air(K):
    """Bipeds in the air (180 bilateral rows, unique answer) under random torques, 4 midpoint steps:
    from the second step on the half-step pose differs from the start pose."""
    ws = wg.make_biped(num_worlds=4, seed=3, z_lift=0.2)
    (eu, eq), _, _ = _run(K, ws, 4, 2e-3, "fp32", 1e-8, tau_fn=lambda k: wg.actuation(ws, 3, k),
                          pkw=dict(integrator=MID), okw=dict(integrator="midpoint"), require_converged=False)
    print(f"midpoint bipeds in the air: err_u {eu:.2e}, err_q {eq:.2e}")
    assert eu <= 1e-4 and eq <= 1e-4


def test_midpoint_biped_standing(K):
    """8 standing bipeds, one actuated midpoint step from rest (the pose update is the half step's)."""
    ws, q, u = _biped_case(8, seed=2)
    assert _margin_clear(None, ws, q)
    _biped_parity(K, ws, q, u, wg.actuation(ws, 2, 0), 2e-3, "fp32", pkw=dict(integrator=MID),
                  okw=dict(integrator="midpoint"))


# ----------------------------------------------------------------------------- drive rows
@pytest.mark.parametrize("cr", [0, 9])
@pytest.mark.parametrize("precision,bar,tol", [("fp64", 1e-9, 1e-12), ("fp32", 1e-4, 1e-8)])
def test_implicit_pd_excavators(K, precision, bar, tol, cr):
    """Excavator arms (hinges and slides in closed loops, bilateral: unique answer) with implicit PD,
    armature and damping on the actuated joints; position targets as actuation, 5 steps."""
    ws = wg.with_joint_drives(wg.make_excavator(num_worlds=16, seed=4), wg.DRIVE_PD, 400.0, 20.0, 0.02, 1.0)
    (eu, eq), rep, infos = _run(K, ws, 5, 2e-3, precision, tol, tau_fn=lambda k: 0.01 * wg.actuation(ws, 4, k),
                                pkw=dict(cr_iters=cr), okw=dict(cr_iters=cr or None))
    assert all(i.reg is not None for i in infos)
    print(f"PD excavators ({precision}, cr {cr}): err_u {eu:.2e}, err_q {eq:.2e}")
    assert eu <= bar and eq <= bar


def test_armature_and_damping_in_torque_mode(K):
    """Torque-mode drive rows (armature and damping only; the actuation stays a torque) on the
    biped in the air: 180 joint rows + 12 regularised rows, unique answer."""
    ws = wg.with_joint_drives(wg.make_biped(num_worlds=4, seed=3, z_lift=0.2), wg.DRIVE_TORQUE,
                              armature=0.01, damping=0.5)
    (eu, eq), rep, infos = _run(K, ws, 3, 2e-3, "fp32", 1e-8, tau_fn=lambda k: wg.actuation(ws, 3, k))
    assert np.all(rep["num_rows"] == 192)
    print(f"armature/damping bipeds: err_u {eu:.2e}, err_q {eq:.2e}")
    assert eu <= 1e-4 and eq <= 1e-4


@pytest.mark.parametrize("cr", [0, 9])
def test_implicit_pd_bipeds_standing(K, cr):
    """The paper's position-actuated set-up (Kp = 15, Kd = 0.6 on the 12 actuated joints), 8 standing
    bipeds with targets N(0, 0.1^2) rad, one step under the contact-world criterion."""
    base, q, u = _biped_case(8, seed=5)
    ws = wg.with_joint_drives(base, wg.DRIVE_PD, 15.0, 0.6)
    assert _margin_clear(None, ws, q)
    tau = wg.actuation(ws, 5, 0, sigma=0.1)
    _biped_parity(K, ws, q, u, tau, 2e-3, "fp32", pkw=dict(cr_iters=cr), okw=dict(cr_iters=cr or None))


# ----------------------------------------------------------------------------- joint limits
@pytest.mark.parametrize("cr", [0, 9])
def test_limit_holds_the_pendulum_on_gpu(K, cr):
    """An upper limit at d = 0.2 stops the swing (FP64): the GPU follows the oracle step by step,
    the rod ends at rest against the limit, whose impulse balances gravity's torque
    dt m g (L/2) sin(0.3) (rod 0.5 m, 1 kg)."""
    ws = wg.with_joint_limits(wg.make_pendulum(theta0=0.5), -np.inf, 0.2)
    q, u = ws.body_q0.copy(), ws.body_u0.copy()
    model = K.Model(ws, "fp64", K.make_params(rho=0.1, cr_iters=cr))
    worst = 0.0
    for k in range(600):
        qg, ug, rep, cache = gpu_step(K, ws, q, u, None, 1e-3, 20000, 1e-12, "fp64", model=model)
        if k % 50 == 0:
            ref, _ = oracle_step(ws, q, u, None, 1e-3, eps=1e-12, cr_iters=cr or None)
            worst = max(worst, errors(q, qg, ug, ref.q, ref.u, 1e-3, "fp64")[0])
        q, u = qg, ug
    assert worst <= 1e-9, worst
    assert np.abs(u).max() < 1e-8
    # cache: 5 hinge rows, then one impulse per finite bound (the upper one)
    assert abs(cache[5] - 1e-3 * 1.0 * 9.81 * 0.25 * math.sin(0.3)) < 1e-9
    assert rep["num_rows"][0] == 6


@pytest.mark.parametrize("cr", [0, 9])
def test_joint_limits_on_bipeds_in_the_air(K, cr):
    """Tight limits (+-2 mrad, inside the activation margin: both bounds of each of the 12 actuated
    joints are rows) on bipeds in the air under random torques, one FP32 step to 1e-8: 24 limit
    rows in the launch, unique u+.  (From the next step on, the oracle itself no longer converges on
    this set within 50,000 iterations, and its 1e-8 and 1e-12 answers differ by ~1e-3.)"""
    base = wg.make_biped(num_worlds=4, seed=3, z_lift=0.2)
    ws = wg.with_joint_limits(base, -0.002, 0.002, joints=np.flatnonzero(base.joint_actuator >= 0))
    (eu, eq), rep, infos = _run(K, ws, 1, 2e-3, "fp32", 1e-8, tau_fn=lambda k: wg.actuation(ws, 3, k),
                                pkw=dict(cr_iters=cr), okw=dict(cr_iters=cr or None))
    assert all(len(i.unilateral) == 24 for i in infos)
    print(f"limited bipeds (cr {cr}): err_u {eu:.2e}, err_q {eq:.2e}, rows {rep['num_rows'].tolist()}")
    assert eu <= 1e-4 and eq <= 1e-4
