"""The GPU step's x-step, modelled in FP64 on the CPU: every PADMM iteration takes one refinement step
from the previous iterate, x^i = x^{i-1} - S (b^i + A x^{i-1}), with S a reduced-precision inverse
of A = D~ + (eta + rho) I (the kernel's swept inverse; its tensor-core products round to TF32, its
tiles for large worlds to BF16).  A fixed point satisfies A x = -b whatever S is, provided the
step contracts (||I - A S|| < 1), so the rounded inverse only preconditions the refinement and the
iteration reaches the exact x-step's solution.  Used directly as the solution, the same BF16
inverse moves u+ visibly.  This checks the design argument of the CUDA path on the CPU; the
oracle itself keeps the paper's factorised solve."""
import math

import numpy as np
import pytest

import worldgen as wg
from oracle import audit as A, padmm as PA, timestep as T


def _round_mantissa(X, bits):
    """Round to `bits` stored mantissa bits (FP32 23, TF32 10, BF16 7), nearest."""
    m, e = np.frexp(X)
    return np.ldexp(np.round(m * 2.0 ** (bits + 1)) / 2.0 ** (bits + 1), e)


def _padmm_x_step(Ds, vs, nbil, mu, eta, rho, eps, n_max, x_step):
    """Alg. 1 with Nesterov and restart as in the oracle, the x-step supplied by the caller."""
    m = len(vs)
    x = np.zeros(m)
    y, z = x.copy(), np.zeros(m)
    yh, zh = y.copy(), z.copy()
    a, c_prev = 1.0, math.inf
    for it in range(1, n_max + 1):
        b = vs + PA.desaxce(zh, nbil, mu) - eta * x - rho * yh - zh
        xn = x_step(b, x)
        yn = PA.project_cone(xn - zh / rho, nbil, mu)
        zn = zh - rho * (xn - yn)
        rp, rd, rc = PA.residuals(xn, x, yn, yh, zn, eta, rho, nbil, len(mu))
        c = float((zn - zh) @ (zn - zh) / rho + rho * (yn - yh) @ (yn - yh))
        if c < 0.999 * c_prev:
            an = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * a * a))
            beta = (a - 1.0) / an
            yhn, zhn = yn + beta * (yn - y), zn + beta * (zn - z)
            a, c_prev = an, c
        else:
            a, c_prev = 1.0, c_prev / 0.999
            yhn, zhn = y.copy(), z.copy()
        x, y, z, yh, zh = xn, yn, zn, yhn, zhn
        if rp < eps and rd < eps and rc < eps:
            return y, it, True
    return y, n_max, False


def _problem(maker, dt, seed=3):
    ws = maker(num_worlds=1, seed=seed)
    tau = wg.actuation(ws, seed, 0)
    B = T.build_world(ws, 0, ws.body_q0, ws.body_u0, None if tau.shape[1] == 0 else tau[0], dt, T.SolverParams())
    D = PA.delassus(B["J"], B["Minv"])
    nbil, nc = B["n_bilateral"], len(B["contact_ids"])
    p = PA.jacobi_scaling(D, nbil, nc)
    mus = np.array([B["mu"][k] * p[nbil + 3 * k + 2] / p[nbil + 3 * k] for k in range(nc)])
    return B, p[:, None] * D * p[None, :], p * PA.free_velocity(B["J"], B["u_free"], B["v_star"]), p, mus


@pytest.mark.parametrize("maker,dt", [(wg.make_fourbar, 1e-3), (wg.make_stewart, 2e-3), (wg.make_biped, 2e-3)])
def test_refinement_with_a_rounded_inverse_reaches_the_exact_solution(maker, dt):
    B, Ds, vs, p, mus = _problem(maker, dt)
    J, Minv, uf, nbil = B["J"], B["Minv"], B["u_free"], B["n_bilateral"]
    eta, rho = 1e-6, 0.1
    Amat = Ds + (eta + rho) * np.eye(len(vs))
    Ainv = np.linalg.inv(Amat)
    runs = {}
    for name, bits in (("exact", None), ("fp32", 23), ("tf32", 10), ("bf16", 7)):
        S = Ainv if bits is None else _round_mantissa(Ainv, bits)
        assert np.linalg.norm(np.eye(len(vs)) - Amat @ S, 2) < 0.5
        y, it, conv = _padmm_x_step(Ds, vs, nbil, mus, eta, rho, 1e-12, 50000, lambda b, x: x - S @ (b + Amat @ x))
        assert conv
        lam = p * y
        runs[name] = (uf + Minv @ (J.T @ lam), lam, it)
    u_ref, _, it_ref = runs["exact"]
    scale = max(np.abs(u_ref).max(), 9.81 * dt)
    for name, (u, lam, it) in runs.items():
        assert abs(it - it_ref) <= 0.05 * it_ref + 2, (name, it, it_ref)
        if B["contact_ids"]:       # frictional solutions need not be unique: audit the NCP conditions
            assert max(A.ncp_residual(J, u, B["v_star"], lam, p, nbil, B["mu"])) < 1e-10, name
        else:
            M = np.linalg.inv(Minv)
            u_kkt, _ = A.kkt_direct(J, M, M @ uf, B["v_star"])
            assert np.abs(u - u_kkt).max() / scale < 1e-8, name
            assert np.abs(u - u_ref).max() / scale < 1e-9, name


def test_the_rounded_inverse_alone_is_not_the_solution():
    """Without the refinement step (x = -S b with the BF16 inverse) the bilateral Stewart platform's
    u+ moves by far more than the solver tolerance: the refinement is what makes it exact."""
    B, Ds, vs, p, mus = _problem(wg.make_stewart, 2e-3)
    J, Minv, uf, nbil = B["J"], B["Minv"], B["u_free"], B["n_bilateral"]
    Amat = Ds + (1e-6 + 0.1) * np.eye(len(vs))
    S = _round_mantissa(np.linalg.inv(Amat), 7)
    y, _, _ = _padmm_x_step(Ds, vs, nbil, mus, 1e-6, 0.1, 1e-12, 5000, lambda b, x: -S @ b)
    M = np.linalg.inv(Minv)
    u_kkt, _ = A.kkt_direct(J, M, M @ uf, B["v_star"])
    u = uf + Minv @ (J.T @ (p * y))
    assert np.abs(u - u_kkt).max() / max(np.abs(u_kkt).max(), 9.81 * 2e-3) > 1e-4


def _lagged_x_step(S, Amat, every):
    """The x-step of the kernel with ``residual_every`` = every: the refinement residual b + A x is
    evaluated matrix-free in iterations 1, every + 1, 2 every + 1, ...; the others take
    c = b^i - b^{i-1}, which is that residual whenever the previous x-step solved A x = -b exactly."""
    state = {"it": 0, "b_prev": None}

    def step(b, x):
        state["it"] += 1
        if (state["it"] - 1) % every == 0:
            c = b + Amat @ x
        else:
            c = b - state["b_prev"]
        state["b_prev"] = b
        return x - S @ c
    return step


@pytest.mark.parametrize("every,bits", [(4, 10), (4, 7), (8, 10)])
@pytest.mark.parametrize("maker,dt", [(wg.make_fourbar, 1e-3), (wg.make_stewart, 2e-3), (wg.make_biped, 2e-3)])
def test_lagged_refinement_residual_keeps_the_fixed_point(maker, dt, every, bits):
    """Evaluating the refinement residual only every 4th iteration (c = b^i - b^{i-1} in between)
    with the TF32- or BF16-rounded inverse, or every 8th with the TF32 one: the error the rounded
    inverse leaves in the skipped iterations is corrected at the next evaluated one, so the
    iteration reaches the exact x-step's solution (direct KKT solve without contacts, the NCP
    conditions with them) in the same number of iterations.  (A BF16 inverse lagged 8 iterations
    costs the short four-bar and Stewart solves ~40 % more iterations, so the kernel lags BF16
    inverses 4 iterations at most.)"""
    B, Ds, vs, p, mus = _problem(maker, dt)
    J, Minv, uf, nbil = B["J"], B["Minv"], B["u_free"], B["n_bilateral"]
    eta, rho = 1e-6, 0.1
    Amat = Ds + (eta + rho) * np.eye(len(vs))
    Ainv = np.linalg.inv(Amat)
    y_ref, it_ref, conv = _padmm_x_step(Ds, vs, nbil, mus, eta, rho, 1e-12, 50000, lambda b, x: -Ainv @ b)
    assert conv
    u_ref = uf + Minv @ (J.T @ (p * y_ref))
    scale = max(np.abs(u_ref).max(), 9.81 * dt)
    S = _round_mantissa(Ainv, bits)
    y, it, conv = _padmm_x_step(Ds, vs, nbil, mus, eta, rho, 1e-12, 50000, _lagged_x_step(S, Amat, every))
    assert conv
    assert abs(it - it_ref) <= 0.05 * it_ref + 2, (it, it_ref)
    lam = p * y
    u = uf + Minv @ (J.T @ lam)
    if B["contact_ids"]:
        assert max(A.ncp_residual(J, u, B["v_star"], lam, p, nbil, B["mu"])) < 1e-10
    else:
        M = np.linalg.inv(Minv)
        u_kkt, _ = A.kkt_direct(J, M, M @ uf, B["v_star"])
        assert np.abs(u - u_kkt).max() / scale < 1e-8
        assert np.abs(u - u_ref).max() / scale < 1e-9


def test_lagged_residual_without_evaluation_drifts():
    """Planted mistake for the test above: never evaluating the residual (c = b^i - b^{i-1} in every
    iteration after the first) lets the BF16 inverse's error accumulate, and the bilateral Stewart
    platform's u+ leaves the direct KKT solution."""
    B, Ds, vs, p, mus = _problem(wg.make_stewart, 2e-3)
    J, Minv, uf, nbil = B["J"], B["Minv"], B["u_free"], B["n_bilateral"]
    Amat = Ds + (1e-6 + 0.1) * np.eye(len(vs))
    S = _round_mantissa(np.linalg.inv(Amat), 7)
    y, _, _ = _padmm_x_step(Ds, vs, nbil, mus, 1e-6, 0.1, 1e-12, 5000, _lagged_x_step(S, Amat, 10 ** 9))
    M = np.linalg.inv(Minv)
    u_kkt, _ = A.kkt_direct(J, M, M @ uf, B["v_star"])
    u = uf + Minv @ (J.T @ (p * y))
    assert np.abs(u - u_kkt).max() / max(np.abs(u_kkt).max(), 9.81 * 2e-3) > 1e-4
