"""GPU parity of the sparse formulation (Sec. 5.1): the Delassus operator applied matrix-free and
every PADMM x-step as 9 warm-started Conjugate Residual iterations, against the FP64 oracle running
the same formulation (``cr_iters=9``).  Same metric and bars as the dense tests: where the answer
is unique (bilateral worlds, the box closed forms) the GPU must match it; with frictional contacts
every world passes the criterion fixed for the contact worlds (match within 1e-4, or an NCP
solution within NCP_FACTOR of the oracle's own FP32 floor)."""
import numpy as np
import pytest

import worldgen as wg
from tests.test_gpu_parity import (K, _biped_case, _biped_parity, _hetero, _margin_clear, check_report, errors,
                                   gpu_step, oracle_step, rnd)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CR = 9                                   # the paper's CR budget per x-step
assert K                                 # the fixture, re-exported for this module


@pytest.mark.parametrize("precision,bar,tol", [("fp64", 1e-9, 1e-12), ("fp32", 1e-4, 1e-8)])
def test_sparse_fourbar_parity_over_steps(K, precision, bar, tol):
    """64 four-bars (1 ms), 10 steps; every step starts the oracle (sparse formulation, 1e-12) from
    the GPU state."""
    ws = wg.make_fourbar(num_worlds=64, seed=0)
    dt = 1e-3
    q, u = rnd(ws.body_q0, precision), rnd(ws.body_u0, precision)
    model = K.Model(ws, precision, K.make_params(rho=0.1, cr_iters=CR))
    worst = (0.0, 0.0)
    for k in range(10):
        qg, ug, rep, _ = gpu_step(K, ws, q, u, None, dt, 20000, tol, precision, model=model)
        ref, infos = oracle_step(ws, q, u, None, dt, eps=1e-12, cr_iters=CR)
        eu, eq = errors(q, qg, ug, ref.q, ref.u, dt, precision)
        worst = (max(worst[0], eu), max(worst[1], eq))
        check_report(rep, infos)
        assert np.all(rep["status"] == 0), rep["status"]
        q, u = qg, ug
    print(f"sparse four-bar ({precision}): worst err_u {worst[0]:.2e}, err_q {worst[1]:.2e}")
    assert worst[0] <= bar and worst[1] <= bar, worst


def test_sparse_biped_in_the_air_matches_the_oracle(K):
    """180 bilateral rows with six redundant loops (unique u+): FP32 sparse step to tol 1e-8 (the
    FP64 end game) against the oracle."""
    ws, q, u = _biped_case(4, seed=3, z_lift=0.2)
    tau = wg.actuation(ws, 3, 0)
    qg, ug, rep, _ = gpu_step(K, ws, q, u, tau, 2e-3, 20000, 1e-8, cr_iters=CR)
    ref, infos = oracle_step(ws, q, u, tau, 2e-3, cr_iters=CR)
    check_report(rep, infos)
    assert np.all(rep["num_contacts"] == 0)
    eu, eq = errors(q, qg, ug, ref.q, ref.u, 2e-3)
    print(f"sparse biped in the air: err_u {eu:.2e}, err_q {eq:.2e}, iterations {rep['iterations'].tolist()}")
    assert eu <= 1e-4 and eq <= 1e-4


@pytest.mark.parametrize("seed", [2, 5])
def test_sparse_biped_parity_standing(K, seed):
    """8 standing bipeds (8 active contacts each), one actuated FP32 sparse step to tol 1e-8 against
    the oracle's sparse formulation to 1e-11, world by world under the contact-world criterion."""
    ws, q, u = _biped_case(8, seed=seed)
    assert _margin_clear(None, ws, q)
    _biped_parity(K, ws, q, u, wg.actuation(ws, seed, 0), 2e-3, "fp32", pkw=dict(cr_iters=CR),
                  okw=dict(cr_iters=CR))


def test_sparse_cached_warm_start(K):
    """Two steps with the cached warm start: the second starts Alg. 1 from the first step's impulses
    on both sides."""
    ws, q, u = _biped_case(4, seed=5)
    dt = 2e-3
    model = K.Model(ws, "fp32", K.make_params(rho=0.1, warm_mode=K.WARM_CACHED, cr_iters=CR))
    qg1, ug1, _, cache1 = gpu_step(K, ws, q, u, wg.actuation(ws, 5, 0), dt, 20000, 1e-8, model=model)
    ref1, _ = oracle_step(ws, q, u, wg.actuation(ws, 5, 0), dt, warm="cached", cr_iters=CR)
    lines = _biped_parity(K, ws, qg1, ug1, wg.actuation(ws, 5, 1), dt, "fp32", warm=K.WARM_CACHED,
                          cache_gpu=cache1, cache_oracle=ref1.cache, require_oracle_converged=False,
                          pkw=dict(cr_iters=CR), okw=dict(cr_iters=CR))
    assert len(lines) == 4


def test_sparse_box_at_rest_carries_its_weight(K):
    """Closed form: the normal impulses of a resting box sum to m g dt, its velocity stays zero."""
    m, dt = 1.3, 2e-3
    ws = wg.make_box(mass=m, mu=0.6, num_worlds=5)
    qg, ug, rep, cache = gpu_step(K, ws, ws.body_q0, ws.body_u0, None, dt, 5000, 1e-7, cr_iters=CR)
    lam = cache.reshape(5, 8, 3)
    np.testing.assert_allclose(lam[:, :, 2].sum(axis=1), m * 9.81 * dt, rtol=1e-4)
    assert np.abs(ug).max() < 1e-5
    assert np.all(rep["num_contacts"] == 4)


def test_sparse_matches_dense_and_oracle_on_heterogeneous_worlds(K):
    """Four world types (20 to 180 bilateral rows, no terrain) in one launch: the sparse and the dense
    formulations reach the same unique u+, and both match the oracle; the persistent plan gives the
    single launch's result."""
    ws = _hetero()
    tau = wg.actuation(ws, 7, 0)
    dt = 2e-3
    q0, u0 = rnd(ws.body_q0), rnd(ws.body_u0)
    _, u_dense, _, _ = gpu_step(K, ws, q0, u0, tau, dt, 20000, 1e-8)
    model = K.Model(ws, "fp32", K.make_params(rho=0.1, cr_iters=CR))
    q1, u1, rep1, _ = gpu_step(K, ws, q0, u0, tau, dt, 20000, 1e-8, model=model)
    model.set_launch_mode(K.LAUNCH_PERSISTENT)
    q2, u2, rep2, _ = gpu_step(K, ws, q0, u0, tau, dt, 20000, 1e-8, model=model)
    ref, infos = oracle_step(ws, q0, u0, tau, dt, eps=1e-11, cr_iters=CR)
    check_report(rep1, infos)
    check_report(rep2, infos)
    scale = max(np.abs(ref.u).max(), 9.81 * dt)
    assert np.abs(u1 - u_dense).max() / scale <= 1e-4
    np.testing.assert_allclose(u2, u1, atol=1e-5 * max(1.0, np.abs(u1).max()))
    for qq, uu in ((q1, u1), (q2, u2)):
        eu, eq = errors(q0, qq, uu, ref.q, ref.u, dt)
        assert eu <= 1e-4 and eq <= 1e-4, (eu, eq)


def test_sparse_heightfield_bipeds(K):
    """Bipeds on the heightfield after landing (up to 276 rows), one FP32 sparse step against the
    oracle's sparse formulation under the contact-world criterion."""
    from oracle import timestep as T
    ws = wg.make_biped_heightfield(num_worlds=4, seed=9)
    st = T.initial_state(ws)
    params = T.SolverParams(rho=0.1, eps=1e-8, n_max=20000)
    for k in range(15):
        st, infos = T.step(ws, st, wg.actuation(ws, 9, k), 2e-3, params)
    assert sum(len(i.contact_ids) for i in infos) > 0
    q, u = rnd(st.q), rnd(st.u)
    if not _margin_clear(None, ws, q):
        pytest.skip("a candidate sits on the activation threshold")
    _biped_parity(K, ws, q, u, wg.actuation(ws, 9, 15), 2e-3, "fp32", require_oracle_converged=False,
                  pkw=dict(cr_iters=CR), okw=dict(cr_iters=CR))


def test_sparse_full_size_bipeds(K):
    """4096 standing bipeds in the benchmark's sparse launch (tol 1e-5, N_max 1000): finite results,
    and on 16 evenly spaced worlds the rows match the oracle's and the device NCP residual agrees with
    the oracle's audit of the GPU's own (lambda, u+) on the contact blocks."""
    from oracle import timestep as T
    from tests.test_gpu_parity import _all_infos_like, _cache_offsets, _gpu_lambda, _ncp_parts
    ws = wg.make_biped(num_worlds=4096, seed=0)
    model = K.Model(ws, "fp32", K.make_params(rho=0.1, cr_iters=CR))
    st = K.State(model)
    q0 = st.body_q.double().cpu().numpy()
    u0 = st.body_u.double().cpu().numpy()
    tau = wg.actuation(ws, 0, 0)
    st.step(2e-3, 1000, 1e-5, torch.tensor(tau, dtype=torch.float32, device="cuda").contiguous())
    torch.cuda.synchronize()
    ug = st.body_u.double().cpu().numpy()
    rep = st.residuals()
    cache = st.cache.double().cpu().numpy()
    assert np.isfinite(ug).all()
    assert np.all(rep["status"] & K.WORLD_NONFINITE == 0)
    sample = [int(w) for w in np.linspace(0, 4095, 16).astype(int)]
    st0 = T.WorldState(q=q0.copy(), u=u0.copy(), cache=[None] * ws.num_worlds)
    _, infos = T.step(ws, st0, tau, 2e-3, T.SolverParams(rho=0.1, eps=1e-5, n_max=1000, cr_iters=CR), worlds=sample)
    off = _cache_offsets(ws, _all_infos_like(ws))
    for w, info in zip(sample, infos):
        assert rep["num_rows"][w] == info.m
        lam = _gpu_lambda(info, cache[off[w]:off[w + 1]])
        r, _ = _ncp_parts(info, ug[ws.bodies(w)].reshape(-1), lam)
        assert abs(float(rep["r_ncp"][w]) - r) <= 1e-6 + 0.1 * r, (w, float(rep["r_ncp"][w]), r)
    print(f"sparse 4096 bipeds: mean iterations {rep['iterations'].mean():.1f}, converged "
          f"{np.mean(rep['status'] == 0):.3f}, median r_ncp {np.median(rep['r_ncp']):.2e}")


def test_fp64_bipeds_in_the_air_match_to_1e9(K):
    """FP64 on the biped (the dense FP64 working set does not fit in shared memory; the sparse one
    does): 180 bilateral rows with six redundant loops, unique u+, one actuated step to 1e-12 against
    the oracle's sparse formulation to 1e-12, within the FP64 bar 1e-9."""
    ws = wg.make_biped(num_worlds=4, seed=3, z_lift=0.2)
    q, u = np.asarray(ws.body_q0, np.float64), np.asarray(ws.body_u0, np.float64)
    tau = wg.actuation(ws, 3, 0)
    qg, ug, rep, _ = gpu_step(K, ws, q, u, tau, 2e-3, 50000, 1e-12, "fp64", cr_iters=CR)
    ref, infos = oracle_step(ws, q, u, tau, 2e-3, eps=1e-12, cr_iters=CR)
    check_report(rep, infos)
    eu, eq = errors(q, qg, ug, ref.q, ref.u, 2e-3, "fp64")
    print(f"FP64 sparse bipeds in the air: err_u {eu:.2e}, err_q {eq:.2e}, iterations {rep['iterations'].tolist()}, "
          f"oracle converged {[i.converged for i in infos]}")
    assert eu <= 1e-9 and eq <= 1e-9


def test_fp64_standing_bipeds(K):
    """FP64 standing bipeds (8 active contacts each), one actuated step to 1e-12: every world matches
    the oracle within the FP64 bar 1e-9 or, where the frictional solution is not unique (reading 19),
    is an NCP solution within 10x the oracle's own residual."""
    from tests.test_gpu_parity import _all_infos_like, _cache_offsets, _gpu_lambda, _ncp
    ws = wg.make_biped(num_worlds=4, seed=2)
    q, u = np.asarray(ws.body_q0, np.float64), np.asarray(ws.body_u0, np.float64)
    tau = wg.actuation(ws, 2, 0)
    qg, ug, rep, cache = gpu_step(K, ws, q, u, tau, 2e-3, 50000, 1e-12, "fp64", cr_iters=CR)
    ref, infos = oracle_step(ws, q, u, tau, 2e-3, eps=1e-12, cr_iters=CR)
    check_report(rep, infos)
    off = _cache_offsets(ws, _all_infos_like(ws))
    for w, info in enumerate(infos):
        bs = ws.bodies(w)
        eu, eq = errors(q[bs], qg[bs], ug[bs], ref.q[bs], ref.u[bs], 2e-3, "fp64")
        r_gpu = _ncp(info, ug[bs].reshape(-1), _gpu_lambda(info, cache[off[w]:off[w + 1]]))
        r_orc = _ncp(info, info.u_plus, info.lam)
        print(f"world {w}: err_u {eu:.2e}, err_q {eq:.2e}, iterations {int(rep['iterations'][w])}, "
              f"ncp gpu {r_gpu:.2e} oracle {r_orc:.2e}")
        assert (eu <= 1e-9 and eq <= 1e-9) or r_gpu <= 10.0 * max(r_orc, 1e-13), (w, eu, r_gpu, r_orc)


@pytest.mark.parametrize("per_world", [2, 4])
def test_sparse_beyond_the_dense_limit(K, per_world):
    """Worlds of 2 and 4 standing bipeds (408 and 816 rows: beyond the 288 padded rows the dense
    formulation's matrix can hold, which refuses them): one actuated FP32 sparse step to 1e-8 against
    the oracle's sparse formulation under the contact-world criterion (2 and 4 units per thread)."""
    ws = wg.make_biped_team(num_worlds=2, seed=3, per_world=per_world)
    with pytest.raises(K.KaminoError) as err:
        K.Model(ws, "fp32", K.make_params(rho=0.1))
    assert err.value.status == 7
    q, u = rnd(ws.body_q0), rnd(ws.body_u0)
    assert _margin_clear(None, ws, q)
    lines = _biped_parity(K, ws, q, u, wg.actuation(ws, 3, 0), 2e-3, "fp32", pkw=dict(cr_iters=CR),
                          okw=dict(cr_iters=CR))
    assert len(lines) == 2
