"""The seeded synthetic inputs hold to their recipe: a world's draws do not depend on how many worlds
are built beside it, the actuation stream is reproducible per (seed, step) with the stated
Gaussian scale, the biped's masses, friction and standing contact geometry are as described, the
heightfield grid is the stated one, and worlds stepped together equal worlds stepped apart (the
batch only concatenates independent problems)."""
import numpy as np
import pytest

import worldgen as wg
from oracle import rigid, timestep as T

PER_WORLD = ("body_mass", "body_inertia", "joint_type", "joint_parent", "joint_child", "joint_actuator",
             "joint_frame_parent", "joint_frame_child", "contact_body", "contact_point", "body_q0", "body_u0")


def _world_slice(ws, w, name):
    a = getattr(ws, name)
    if name.startswith("body"):
        return a[ws.bodies(w)]
    if name.startswith("joint"):
        return a[ws.joints(w)]
    return a[ws.contacts(w)]


def test_a_world_does_not_depend_on_the_batch_size():
    small, large = wg.make_biped(num_worlds=2, seed=4), wg.make_biped(num_worlds=7, seed=4)
    for w in range(2):
        for name in PER_WORLD:
            np.testing.assert_array_equal(_world_slice(small, w, name), _world_slice(large, w, name))
        assert small.world_mu[w] == large.world_mu[w]


def test_actuation_stream_is_reproducible_and_gaussian():
    ws = wg.make_biped(num_worlds=512, seed=1)
    a, b = wg.actuation(ws, 1, 3), wg.actuation(ws, 1, 3)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, wg.actuation(ws, 1, 4)) and not np.array_equal(a, wg.actuation(ws, 2, 3))
    x = a[:, :12].reshape(-1)
    assert abs(x.mean()) < 0.5 and abs(x.std() - 5.0) < 0.25          # N(0, 5^2) N m, 6144 draws


def test_biped_recipe():
    ws = wg.make_biped(num_worlds=32, seed=0)
    for w in range(ws.num_worlds):
        m = ws.body_mass[ws.bodies(w)]
        assert m[0] == 10.0                                              # pelvis
        assert 100.0 <= m.max() / m.min() <= 1000.0                      # mass ratio up to 1000
        assert 0.5 <= ws.world_mu[w] <= 1.0
        # standing: the bottom corners of both feet touch the plane, the top ones are above it
        q = ws.body_q0[ws.bodies(w)]
        cs = ws.contacts(w)
        z = np.array([q[b, 2] + (rigid.quat_to_rot(q[b, 3:]) @ p)[2]
                      for b, p in zip(ws.contact_body[cs], ws.contact_point[cs])])
        assert len(z) == 16 and np.sum(np.abs(z) < 1e-12) == 8 and np.all(z > -1e-12)
        assert ws.bilateral_rows(w) + 3 * 16 == 228                      # m <= 228 with every candidate


def test_heightfield_recipe():
    ws = wg.make_biped_heightfield(num_worlds=4, seed=0)
    assert ws.terrain_kind == wg.TERRAIN_HEIGHTFIELD
    assert (ws.hf_nx, ws.hf_ny) == (64, 64) and ws.hf_cell == 1.0 / 32.0
    assert ws.hf_heights.min() >= 0.0 and ws.hf_heights.max() <= 0.05
    assert all(ws.contacts(w).stop - ws.contacts(w).start == 32 for w in range(4))
    assert ws.bilateral_rows(0) + 3 * 32 == 276
    flat = wg.make_biped(num_worlds=4, seed=0)
    assert abs(ws.body_q0[0, 2] - flat.body_q0[0, 2] - 0.05) < 1e-12            # pelvis raised 5 cm


def test_worlds_stepped_together_equal_worlds_stepped_apart():
    parts = [wg.make_fourbar(2, seed=5), wg.make_biped(2, seed=5)]
    both = wg.concat(parts)
    params = T.SolverParams(eps=1e-10, n_max=20000, rho=0.1)
    tau = np.zeros((both.num_worlds, both.n_act_max))
    tau[2:, :12] = wg.actuation(parts[1], 5, 0)
    st_both, _ = T.step(both, T.initial_state(both), tau, 2e-3, params)
    st_four, _ = T.step(parts[0], T.initial_state(parts[0]), None, 2e-3, params)
    st_bip, _ = T.step(parts[1], T.initial_state(parts[1]), wg.actuation(parts[1], 5, 0), 2e-3, params)
    nb4 = int(parts[0].world_body_offset[-1])
    np.testing.assert_array_equal(st_both.q[:nb4], st_four.q)
    np.testing.assert_array_equal(st_both.q[nb4:], st_bip.q)
    np.testing.assert_array_equal(st_both.u[nb4:], st_bip.u)


def test_concat_takes_the_terrain_of_the_worlds_with_contacts():
    four, biped = wg.make_fourbar(2, seed=1), wg.make_biped(2, seed=1)
    assert four.terrain_kind == wg.TERRAIN_NONE and biped.terrain_kind == wg.TERRAIN_PLANE
    assert wg.concat([four, biped]).terrain_kind == wg.TERRAIN_PLANE           # four-bars have no candidates
    assert wg.concat([four, biped], terrain=wg.TERRAIN_NONE).terrain_kind == wg.TERRAIN_NONE
    assert wg.concat([four, wg.make_stewart(2, seed=1)]).terrain_kind == wg.TERRAIN_NONE
    with pytest.raises(ValueError):
        wg.concat([biped, wg.make_biped_heightfield(2, seed=1)])               # two different grounds
    with pytest.raises(ValueError):
        wg.concat([four, wg.make_free_body()])                                 # zero gravity
