"""Pins of the oracle's dual solver (Sec. 4: Eq. 3, Eq. 4, Alg. 1): cone projection against its
definition, Proximal-ADMM against a direct KKT solve and against brute-force enumeration of
contact modes, and the NCP conditions of the returned impulses."""
import itertools
import math

import numpy as np
import pytest

import worldgen as wg
from oracle import audit as A, padmm as PA, timestep as T


# ----------------------------------------------------------------------------- cone projection
def _proj_reference(x, mu):
    """Euclidean projection onto {||t|| <= mu n} by brute force: a dense sample of the cone's
    boundary plus the apex and x itself when feasible."""
    best, bestd = np.zeros(3), np.linalg.norm(x)
    if np.hypot(x[0], x[1]) <= mu * x[2]:
        return x.copy()
    for n in np.linspace(0.0, 3.0, 601):
        for a in np.linspace(0.0, 2 * math.pi, 361):
            y = np.array([mu * n * math.cos(a), mu * n * math.sin(a), n])
            d = np.linalg.norm(x - y)
            if d < bestd:
                best, bestd = y, d
    return best


@pytest.mark.parametrize("mu", [0.0, 0.3, 1.0])
def test_cone_projection_kkt_and_brute_force(mu):
    rng = np.random.default_rng(20)
    for _ in range(8):
        x = rng.standard_normal(3)
        y = PA.project_cone(x, 0, [mu])
        # feasibility, the polar-cone condition and orthogonality (KKT of min ||y - x||, y in K)
        assert math.hypot(y[0], y[1]) <= mu * y[2] + 1e-12
        w = x - y                           # must lie in the polar cone  {mu ||t|| <= -n}
        assert mu * math.hypot(w[0], w[1]) <= -w[2] + 1e-12 or np.linalg.norm(w) < 1e-12
        assert abs(y @ w) < 1e-12
        if mu > 0:
            ref = _proj_reference(x, mu)
            assert np.linalg.norm(x - y) <= np.linalg.norm(x - ref) + 1e-9
    # bilateral rows pass through unchanged
    x = rng.standard_normal(7)
    np.testing.assert_array_equal(PA.project_cone(x, 4, [0.5])[:4], x[:4])


def test_desaxce_operator():
    v = np.array([1.0, 2.0, 3.0, 4.0, 0.0, -1.0])
    s = PA.desaxce(v, 0, [0.5, 2.0])
    np.testing.assert_allclose(s, [0, 0, 0.5 * math.hypot(1, 2), 0, 0, 2.0 * 4.0])


# ----------------------------------------------------------------------------- bilateral worlds
@pytest.mark.parametrize("maker,dt", [(wg.make_fourbar, 1e-3), (wg.make_excavator, 2e-3), (wg.make_stewart, 2e-3)])
def test_padmm_matches_direct_kkt(maker, dt):
    """Alg. 1 reaches the unique u+ of the KKT system Eq. 2 (solved directly) on worlds without
    contacts, including over-constrained loops whose impulses are not unique."""
    ws = maker(num_worlds=2, seed=3)
    params = T.SolverParams(eps=1e-12, n_max=20000, rho=0.1)
    st = T.initial_state(ws)
    st, _ = T.step(ws, st, wg.actuation(ws, 3, 0), dt, params)      # move off the rest state
    st, infos = T.step(ws, st, wg.actuation(ws, 3, 1), dt, params)
    for i in infos:
        M = np.linalg.inv(i.Minv)
        u_kkt, _ = A.kkt_direct(i.J, M, M @ i.u_free, i.v_star)
        scale = max(np.abs(u_kkt).max(), 9.81 * dt)
        assert np.abs(i.u_plus - u_kkt).max() / scale < 1e-8
        assert i.converged


def test_nesterov_and_preconditioning_do_not_change_the_solution():
    ws = wg.make_fourbar(num_worlds=2, seed=4)
    st = T.initial_state(ws)
    outs = []
    for nest in (True, False):
        for pre in (True, False):
            params = T.SolverParams(eps=1e-12, n_max=50000, rho=0.1, nesterov=nest, precond=pre)
            _, infos = T.step(ws, st, None, 1e-3, params)
            outs.append(np.concatenate([i.u_plus for i in infos]))
    for o in outs[1:]:
        np.testing.assert_allclose(o, outs[0], atol=1e-9)


# ----------------------------------------------------------------------------- contact closed forms
def test_box_resting_on_plane_carries_its_weight():
    """A box at rest on the plane: the normal impulses sum to m g dt, no friction, u+ = 0.  The
    split among the corners is not unique, so only the sum is checked."""
    m, dt = 1.3, 2e-3
    ws = wg.make_box(mass=m, mu=0.6)
    params = T.SolverParams(eps=1e-10, n_max=20000, rho=0.1)
    st, infos = T.step(ws, T.initial_state(ws), None, dt, params)
    i = infos[0]
    assert len(i.contact_ids) == 4                 # the four bottom corners
    lam = i.lam.reshape(-1, 3)
    assert abs(lam[:, 2].sum() - m * 9.81 * dt) < 1e-8
    assert np.abs(lam[:, :2]).max() < 1e-8
    assert np.abs(i.u_plus).max() < 1e-8


@pytest.mark.parametrize("axis", [0, 1])
def test_sliding_box_decelerates_at_mu_g_and_stops(axis):
    """Coulomb sliding: v(t) = v0 - mu g t until rest at t = v0 / (mu g), then it stays at rest.
    Along either edge of the box (the plane's two tangent directions), where the corners' friction
    torques about the vertical cancel by symmetry, so the box does not spin."""
    mu, v0, dt = 0.4, 0.5, 1e-3
    vel = [0.0, 0.0, 0.0]
    vel[axis] = v0
    ws = wg.make_box(mass=1.0, mu=mu, v0=tuple(vel))
    params = T.SolverParams(eps=1e-10, n_max=20000, rho=0.1)
    st = T.initial_state(ws)
    vs = []
    for k in range(150):
        st, infos = T.step(ws, st, None, dt, params)
        vs.append(st.u[0, axis])
    t = dt * np.arange(1, 151)
    expect = np.maximum(v0 - mu * 9.81 * t, 0.0)
    np.testing.assert_allclose(vs, expect, atol=2e-6)
    assert np.abs(np.delete(st.u[0], axis)).max() < 1e-6


@pytest.mark.parametrize("angle,mu,sticks", [(0.3, 0.5, True), (0.5, 0.5, False), (0.2, 0.1, False)])
def test_box_on_incline_sticks_iff_tan_theta_le_mu(angle, mu, sticks):
    """Tilting gravity by theta is an incline of angle theta: the box sticks iff tan(theta) <= mu,
    otherwise it accelerates at g (sin theta - mu cos theta) along the slope."""
    g = 9.81
    grav = (g * math.sin(angle), 0.0, -g * math.cos(angle))
    ws = wg.make_box(mass=1.0, mu=mu, gravity=grav)
    params = T.SolverParams(eps=1e-10, n_max=20000, rho=0.1)
    st = T.initial_state(ws)
    dt, n = 1e-3, 50
    for _ in range(n):
        st, _ = T.step(ws, st, None, dt, params)
    a_expect = 0.0 if sticks else g * (math.sin(angle) - mu * math.cos(angle))
    assert (math.tan(angle) <= mu) == sticks
    assert abs(st.u[0, 0] - a_expect * n * dt) < 1e-6
    assert abs(st.u[0, 2]) < 1e-6


# ----------------------------------------------------------------------------- brute force
def _planar_modes(D2, vf2, mu):
    """All solutions of the planar (1-D friction) De Saxce NCP by enumeration of the contact modes
    separate / stick / slide+ / slide-.  Each mode fixes two linear equations per contact in
    (lambda, v = D lambda + v_f); a mode's solution is kept when its inequalities hold."""
    k = len(mu)
    sols = []
    for modes in itertools.product(range(4), repeat=k):
        A_ = np.zeros((2 * k, 2 * k))
        b_ = np.zeros(2 * k)
        for c, mode in enumerate(modes):
            it, inn = 2 * c, 2 * c + 1
            rows = []
            if mode == 0:            # separate: lambda = 0
                rows = [(np.eye(2 * k)[it], 0.0), (np.eye(2 * k)[inn], 0.0)]
            elif mode == 1:          # stick: v = 0
                rows = [(D2[it], -vf2[it]), (D2[inn], -vf2[inn])]
            else:                    # slide: v_n = 0, lambda_t = -+ mu lambda_n
                s = 1.0 if mode == 2 else -1.0
                e = np.zeros(2 * k)
                e[it] = 1.0
                e[inn] = s * mu[c]
                rows = [(D2[inn], -vf2[inn]), (e, 0.0)]
            for j, (a, bb) in enumerate(rows):
                A_[it + j] = a
                b_[it + j] = bb
        try:
            lam = np.linalg.solve(A_, b_)
        except np.linalg.LinAlgError:
            continue
        v = D2 @ lam + vf2
        ok = True
        for c, mode in enumerate(modes):
            lt, ln, vt, vn = lam[2 * c], lam[2 * c + 1], v[2 * c], v[2 * c + 1]
            tol = 1e-9
            if mode == 0:
                ok &= vn >= -tol
            elif mode == 1:
                ok &= abs(lt) <= mu[c] * ln + tol
            else:
                s = 1.0 if mode == 2 else -1.0
                ok &= ln >= -tol and s * vt >= -tol
        if ok:
            sols.append(lam)
    return sols


@pytest.mark.parametrize("k", [1, 2, 3])
def test_padmm_solution_is_one_of_the_enumerated_contact_modes(k):
    """Random planar contact problems with k <= 3 contacts (embedded in 3-D with a decoupled second
    tangent): the impulses found by Alg. 1 coincide with one of the brute-force mode solutions."""
    rng = np.random.default_rng(30 + k)
    for trial in range(6):
        G = rng.standard_normal((2 * k, 2 * k + 1))
        D2 = G @ G.T / (2 * k) + 0.05 * np.eye(2 * k)
        vf2 = rng.standard_normal(2 * k)
        mu = rng.uniform(0.2, 1.0, size=k)
        m = 3 * k
        D = np.eye(m)
        vf = np.zeros(m)
        idx = [3 * c for c in range(k)] + [3 * c + 2 for c in range(k)]
        idx2 = [2 * c for c in range(k)] + [2 * c + 1 for c in range(k)]
        for a, a2 in zip(idx, idx2):
            vf[a] = vf2[a2]
            for b, b2 in zip(idx, idx2):
                D[a, b] = D2[a2, b2]
        res = PA.padmm(D, vf, 0, mu, eta=1e-8, rho=0.5, eps=1e-12, n_max=50000)
        lam2 = np.array([res.y[3 * c + j] for c in range(k) for j in (0, 2)])
        sols = _planar_modes(D2, vf2, mu)
        assert sols, "enumeration found no solution"
        assert min(np.abs(s - lam2).max() for s in sols) < 1e-6
        assert np.abs(res.y[1::3]).max() < 1e-9


def test_biped_step_satisfies_ncp_conditions():
    """One biped step from the assembled pose (consistent bias, so Alg. 1 can reach a tight
    tolerance): lambda lies in the friction cones, v + Gamma(v) in the dual cones, they are
    complementary, sliding contacts have zero normal velocity (Sec. 4), and the natural-map
    residual is at the solver tolerance."""
    ws = wg.make_biped(num_worlds=3, seed=5)
    params = T.SolverParams(eps=1e-10, n_max=20000, rho=0.1)
    st, infos = T.step(ws, T.initial_state(ws), wg.actuation(ws, 5, 0), 2e-3, params)
    for i in infos:
        assert i.converged
        nb = i.n_bilateral
        lam = i.lam[nb:].reshape(-1, 3)
        v = (i.J @ i.u_plus + i.v_star)[nb:].reshape(-1, 3)
        for (lt1, lt2, ln), (vt1, vt2, vn), mu in zip(lam, v, i.mu):
            vt = math.hypot(vt1, vt2)
            assert math.hypot(lt1, lt2) <= mu * ln + 1e-7
            assert vn + mu * vt >= -1e-6
            assert abs(lt1 * vt1 + lt2 * vt2 + ln * (vn + mu * vt)) < 1e-6
            if vt > 1e-4 and ln > 1e-6:
                assert abs(vn) < 1e-5
        r_c, r_b = A.ncp_residual(i.J, i.u_plus, i.v_star, i.lam, i.p, nb, i.mu)
        assert r_c < 1e-6 and r_b < 1e-6


def test_penetrating_box_rises_at_beta_depth_over_dt():
    """Without gravity, a box sunk by d is pushed out by the Baumgarte bias of its four bottom
    corners: the first step gives it the separating velocity beta d / dt exactly, after which the
    contacts are slack (J u >= bias holds with lambda = 0) and it keeps that velocity, so its height
    after k steps is -d + k beta d, through the surface and beyond (restitution 0, no damping)."""
    d, dt = 1e-3, 2e-3
    ws = wg.make_box(mass=1.0, mu=0.5, pos=(0.0, 0.0, 0.025 - d), gravity=(0.0, 0.0, 0.0))
    params = T.SolverParams(eps=1e-12, n_max=20000, rho=0.1)
    st = T.initial_state(ws)
    for k in range(1, 8):
        st, infos = T.step(ws, st, None, dt, params)
        assert abs(st.q[0, 2] - 0.025 - (-d + k * params.beta * d)) < 1e-12
        np.testing.assert_allclose(st.u[0], [0, 0, params.beta * d / dt, 0, 0, 0], atol=1e-12)
        assert len(infos[0].contact_ids) == 4
    assert infos[0].lam.size == 12 and np.abs(infos[0].lam).max() < 1e-12


def test_approaching_box_lands_on_the_surface_and_stops():
    """A box falling at 2 m/s, h = 2 mm above the plane (inside the activation margin), with
    v dt > h: the normal rows allow closing the gap in this step and no more, so the step ends
    with the box on the surface at velocity -h/dt, and the next one brings it to rest."""
    h, v, dt = 2e-3, -2.0, 2e-3
    ws = wg.make_box(mass=1.0, mu=0.5, pos=(0.0, 0.0, 0.025 + h), v0=(0.0, 0.0, v), gravity=(0.0, 0.0, 0.0))
    params = T.SolverParams(eps=1e-12, n_max=20000, rho=0.1)
    st, _ = T.step(ws, T.initial_state(ws), None, dt, params)
    assert abs(st.q[0, 2] - 0.025) < 1e-12
    np.testing.assert_allclose(st.u[0], [0, 0, -h / dt, 0, 0, 0], atol=1e-12)
    st, _ = T.step(ws, st, None, dt, params)
    assert abs(st.q[0, 2] - 0.025) < 1e-12
    assert np.abs(st.u[0]).max() < 1e-10


# One bilateral row with D = d, v_f = v, eta = 0: z stays 0 (the projection is the identity, so
# x - y = z^/rho and z = z^ - rho z^/rho = 0) and y = x, so Alg. 1 reduces to the scalar recurrence
#   x_i = (-v + rho y^_{i-1}) / (d + rho),  c_i = rho (x_i - y^_{i-1})^2,
#   c_i < 0.999 c_{i-1}: a' = (1 + sqrt(1 + 4 a^2)) / 2,  y^_i = x_i + (a - 1) / a' (x_i - x_{i-1}),
#   otherwise a = 1, y^_i = x_{i-1}, c_i = c_{i-1} / 0.999.
# The values below were worked out from that recurrence with 40-digit decimal arithmetic.
_FAST = [(1, 0.5, 0.5), (2, 0.75, 0.8204383812813302), (3, 0.9102191906406651, 0.9797611740011472),
         (4, 0.9898805870005736, 1.0321858712953011)]
_SLOW_X = {10: 0.181497699038228, 20: 0.510415621930859, 36: 0.9818578599895553, 37: 1.0006365656364018,
           38: 1.017839886484623, 39: 1.0006302630063384, 40: 1.000624022778553}


def _scalar(d, v, n):
    D = np.array([[d]])
    return PA.padmm(D, np.array([v]), 1, [], eta=0.0, rho=1.0, eps=0.0, n_max=n)


def test_nesterov_sequence_matches_hand_recurrence():
    """Sec. 4.1's acceleration, pinned by the hand-worked scalar recurrence above: the momentum
    weights (a - 1)/a' of the first iterations (d = 1, v = -1) and, on a slow problem (d = 0.01,
    v = -0.01, solution 1), the first adaptive restart, which comes at iteration 38 when the
    extrapolated iterate overshoots and the combined residual grows."""
    for i, x, yh in _FAST:
        res = _scalar(1.0, -1.0, i)
        assert res.x[0] == pytest.approx(x, rel=1e-13) and res.restarts == 0
    for i, x in _SLOW_X.items():
        res = _scalar(0.01, -0.01, i)
        assert res.x[0] == pytest.approx(x, rel=1e-12), i
        assert res.restarts == (1 if i >= 38 else 0), i
