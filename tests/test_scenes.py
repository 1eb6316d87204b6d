"""Input generators (no arithmetic of the method): seeded determinism,
sizes, orientation and a penetration-free start of the generated scenes."""
import numpy as np

from paper_2512_12151_b300 import scenes


def _signed_volumes(s):
    d = s.rest[s.tets[:, 1:]] - s.rest[s.tets[:, :1]]
    return np.linalg.det(d) / 6.0


def test_batch_scene_seeded_and_sized():
    a, b = scenes.batch_scene(17), scenes.batch_scene(17)
    assert np.array_equal(a.x0, b.x0) and np.array_equal(a.tets, b.tets)
    nts = [scenes.batch_scene(i).nt for i in range(64)]
    assert 700 <= min(nts) and max(nts) <= 2.2e4
    s = scenes.batch_scene(3)
    assert (_signed_volumes(s) > 0).all()
    free = s.x0[s.dirichlet == 0]
    assert free[:, 2].min() > 0.005  # above the ground quad at z = 0


def test_spiky_balls_coarse():
    s = scenes.spiky_balls(cell=0.012)  # coarse cells keep the test fast
    assert (_signed_volumes(s) > 0).all()
    assert s.dirichlet.sum() == 12  # 8 box vertices + 4 plate vertices
    free = s.x0[s.dirichlet == 0]
    z = free[:, 2]
    assert z.min() > 0.0 and z.max() < scenes.plate_schedule_z(s, -1)
    # the plate descends at 0.5 m/s, stops at 30 % of its height, then rises
    z0 = s.meta["plate_z0"]
    h = s.params.dt
    assert np.isclose(scenes.plate_schedule_z(s, 0), z0 - 0.5 * h)
    steps = [scenes.plate_schedule_z(s, i) for i in range(200)]
    assert np.isclose(min(steps), 0.3 * z0, atol=0.5 * h)
    assert steps[-1] > min(steps)


def test_spiky_ball_solid_is_one_piece():
    rng = np.random.default_rng(0)
    v, t = scenes.spiky_ball(rng, (0.0, 0.0, 0.0), cell=0.01)
    # every vertex is used and the tets form one face-connected solid
    assert len(np.unique(t)) == len(v)
    r = np.linalg.norm(v, axis=1)
    assert r.max() <= 0.1 + 0.05 + 0.02 and r.min() < 0.02
