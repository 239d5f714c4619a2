"""Pins of the oracle's sparse formulation (Sec. 5.1): the matrix-free Delassus operator and the
Conjugate Residual x-step of Alg. 1, warm-started at the previous iterate with a fixed budget.

CR is pinned by its defining property (each iterate minimises the 2-norm residual over the shifted
Krylov space, checked against a least-squares solve over an explicit Krylov basis) and by finite
termination; the whole step by the same references as the dense path: the direct KKT solve of
Eq. 2 on bilateral worlds, the box closed forms, and the NCP conditions on bipeds (whose frictional
contact problem can have several solutions, so the biped is audited rather than compared)."""
import numpy as np
import pytest

import worldgen as wg
from oracle import audit as A, padmm as PA, timestep as T


def _spd(m, cond, rng):
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    return Q @ np.diag(np.geomspace(1.0, cond, m)) @ Q.T


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_cr_iterate_minimises_residual_over_krylov_space(k):
    rng = np.random.default_rng(40 + k)
    m = 24
    Amat = _spd(m, 50.0, rng)
    c, x0 = rng.standard_normal(m), rng.standard_normal(m)
    x = PA.conjugate_residual(lambda v: Amat @ v, c, x0, k)
    r0 = c - Amat @ x0
    K = np.empty((m, k))
    v = r0.copy()
    for j in range(k):
        K[:, j] = v / np.linalg.norm(v)
        v = Amat @ K[:, j]
    a, *_ = np.linalg.lstsq(Amat @ K, r0, rcond=None)
    x_best = x0 + K @ a
    np.testing.assert_allclose(x, x_best, rtol=0, atol=1e-9 * np.abs(x_best).max())
    res = [np.linalg.norm(c - Amat @ PA.conjugate_residual(lambda v: Amat @ v, c, x0, j)) for j in range(k + 1)]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(res, res[1:]))      # residual never grows


def test_cr_reaches_the_solution_in_m_iterations():
    rng = np.random.default_rng(7)
    m = 16
    Amat = _spd(m, 20.0, rng)
    c = rng.standard_normal(m)
    x = PA.conjugate_residual(lambda v: Amat @ v, c, np.zeros(m), m)
    np.testing.assert_allclose(x, np.linalg.solve(Amat, c), rtol=0, atol=1e-10)
    # a warm start at the solution stays there (zero residual, no division by zero)
    xs = np.linalg.solve(Amat, c)
    np.testing.assert_allclose(PA.conjugate_residual(lambda v: Amat @ v, Amat @ xs, xs, 5), xs, atol=1e-14)


def test_matrix_free_delassus_is_the_scaled_delassus_matrix():
    ws = wg.make_biped(num_worlds=1, seed=2)
    B = T.build_world(ws, 0, ws.body_q0, ws.body_u0, wg.actuation(ws, 2, 0)[0], 2e-3, T.SolverParams())
    J, Minv = B["J"], B["Minv"]
    D = J @ Minv @ J.T
    np.testing.assert_allclose(PA.delassus_diagonal(J, Minv), np.diag(D), rtol=1e-13)
    p = PA.jacobi_scaling(np.diag(D), B["n_bilateral"], len(B["contact_ids"]))
    np.testing.assert_allclose(p, PA.jacobi_scaling(D, B["n_bilateral"], len(B["contact_ids"])), rtol=0)
    op = PA.delassus_matrix_free(J, Minv, p)
    rng = np.random.default_rng(3)
    for _ in range(3):
        v = rng.standard_normal(J.shape[0])
        np.testing.assert_allclose(op(v), p * (D @ (p * v)), rtol=0, atol=1e-12 * np.abs(p * (D @ (p * v))).max())


@pytest.mark.parametrize("cr_iters", [1, 9])
@pytest.mark.parametrize("maker,dt", [(wg.make_fourbar, 1e-3), (wg.make_excavator, 2e-3), (wg.make_stewart, 2e-3)])
def test_cr_padmm_matches_direct_kkt(maker, dt, cr_iters):
    """Bilateral worlds: u+ is unique, and the CR x-step reaches the KKT solution of Eq. 2 even on
    a budget of one CR iteration per ADMM step (the stopping test sees what the x-step left)."""
    ws = maker(num_worlds=2, seed=3)
    params = T.SolverParams(eps=1e-10, n_max=20000, rho=0.1, cr_iters=cr_iters)
    st = T.initial_state(ws)
    st, _ = T.step(ws, st, wg.actuation(ws, 3, 0), dt, params)
    st, infos = T.step(ws, st, wg.actuation(ws, 3, 1), dt, params)
    for i in infos:
        M = np.linalg.inv(i.Minv)
        u_kkt, _ = A.kkt_direct(i.J, M, M @ i.u_free, i.v_star)
        scale = max(np.abs(u_kkt).max(), 9.81 * dt)
        assert i.converged
        assert np.abs(i.u_plus - u_kkt).max() / scale < 2e-7


def test_cr_padmm_box_closed_forms():
    """The resting box carries m g dt; the box sliding along either tangent decelerates at mu g."""
    m, dt = 1.3, 2e-3
    params = T.SolverParams(eps=1e-10, n_max=20000, rho=0.1, cr_iters=9)
    _, infos = T.step(wg.make_box(mass=m, mu=0.6), T.initial_state(wg.make_box(mass=m, mu=0.6)), None, dt, params)
    lam = infos[0].lam.reshape(-1, 3)
    assert abs(lam[:, 2].sum() - m * 9.81 * dt) < 1e-8
    assert np.abs(infos[0].u_plus).max() < 1e-8
    mu, v0, dt = 0.4, 0.5, 1e-3
    for axis in (0, 1):
        vel = [0.0, 0.0, 0.0]
        vel[axis] = v0
        ws = wg.make_box(mass=1.0, mu=mu, v0=tuple(vel))
        st = T.initial_state(ws)
        vs = []
        for k in range(60):
            st, _ = T.step(ws, st, None, dt, params)
            vs.append(st.u[0, axis])
        np.testing.assert_allclose(vs, v0 - mu * 9.81 * dt * np.arange(1, 61), atol=2e-6)


def test_cr_padmm_biped_step_satisfies_ncp_conditions():
    """Actuated bipeds on the ground: the CR path's (lambda, u+) satisfy the NCP conditions (the
    natural-map residual) and the bilateral rows on the range of J, to the solver tolerance."""
    ws = wg.make_biped(num_worlds=2, seed=5)
    params = T.SolverParams(eps=1e-10, n_max=50000, rho=0.1, cr_iters=9)
    _, infos = T.step(ws, T.initial_state(ws), wg.actuation(ws, 5, 0), 2e-3, params)
    for i in infos:
        assert i.converged and len(i.contact_ids) > 0
        r_c, r_b = A.ncp_residual(i.J, i.u_plus, i.v_star, i.lam, i.p, i.n_bilateral, i.mu)
        assert r_c < 1e-8 and r_b < 1e-8
