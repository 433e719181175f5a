"""The seeded input generators that stand in for the paper's meshes (CPU):
batch sizes follow the log-uniform recipe, a batch concatenates independent
cube grids with consistent offsets and mesh ids, and the generators repeat
exactly for a seed."""
import numpy as np

import meshgen


def test_batched_sizes_follow_the_recipe():
    n = meshgen.batched_sizes(4096, 4, 24, seed=4)
    assert n.min() >= 4 and n.max() <= 24
    # log-uniform: ln n is uniform on [ln 4, ln 24] before rounding, so the
    # median side is near sqrt(4 * 24) ~ 9.8 and each end is reached
    assert 9 <= np.median(n) <= 11
    assert (n == 4).any() and (n == 24).any()
    assert np.array_equal(n, meshgen.batched_sizes(4096, 4, 24, seed=4))


def test_batch_is_independent_meshes_with_consistent_offsets():
    sides = [2, 5, 3]
    b = meshgen.cube_grid_batch(sides, jitter=0.01, seed=21)
    assert np.array_equal(b.vert_off, np.cumsum([0] + [(s + 1) ** 3 for s in sides]))
    assert np.array_equal(b.tet_off, np.cumsum([0] + [5 * s ** 3 for s in sides]))
    assert np.all(np.diff(b.batch) >= 0)
    for m, s in enumerate(sides):
        a, e = b.vert_off[m], b.vert_off[m + 1]
        assert (b.batch[a:e] == m).all()
        X, tets, pinned = b.mesh(m)
        g = meshgen.cube_grid(s, jitter=0.01, seed=21 + m)
        assert np.array_equal(X, g.X) and np.array_equal(tets, g.tets) and np.array_equal(pinned, g.pinned)
        # no tet reaches outside its own mesh
        ta, te = b.tet_off[m], b.tet_off[m + 1]
        assert (b.tets[ta:te] >= a).all() and (b.tets[ta:te] < e).all()


def test_generators_repeat_for_a_seed():
    a = meshgen.cube_grid(4, jitter=0.01, seed=9, permute=True)
    c = meshgen.cube_grid(4, jitter=0.01, seed=9, permute=True)
    assert np.array_equal(a.X, c.X) and np.array_equal(a.tets, c.tets)
    u1 = meshgen.random_displacement(a.X, 4, amp=0.05, seed=3, smooth=0.01)
    u2 = meshgen.random_displacement(a.X, 4, amp=0.05, seed=3, smooth=0.01)
    assert np.array_equal(u1, u2)
    mu1, lam1 = meshgen.material_loguniform_E(a.n_tets, 1e4, 1e6, 0.4, 2)
    mu2, lam2 = meshgen.material_loguniform_E(a.n_tets, 1e4, 1e6, 0.4, 2)
    assert np.array_equal(mu1, mu2) and np.array_equal(lam1, lam2)
    # E = mu (3 lam + 2 mu) / (lam + mu) stays inside [1e4, 1e6]
    E = mu1 * (3 * lam1 + 2 * mu1) / (lam1 + mu1)
    assert E.min() >= 1e4 * (1 - 1e-12) and E.max() <= 1e6 * (1 + 1e-12)


def test_hub_fan_counts_valence_and_orientation():
    for segments, apexes in ((1, 700), (16, 24)):
        m = meshgen.hub_fan(segments, apexes, seed=3)
        assert m.n_tets == segments * apexes and m.n_verts == segments + 2 + apexes
        cnt = np.bincount(m.tets.ravel(), minlength=m.n_verts)
        assert cnt[0] == segments * apexes                 # the hub is in every tet
        assert cnt[segments + 2:].tolist() == [segments] * apexes
        e = m.X[m.tets[:, 1:]] - m.X[m.tets[:, :1]]
        assert np.all(np.linalg.det(e.transpose(0, 2, 1)) > 0)
        assert len({tuple(t) for t in np.sort(m.tets, axis=1).tolist()}) == m.n_tets
    a = meshgen.hub_fan(16, 24, seed=3)
    b = meshgen.hub_fan(16, 24, seed=3)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.tets, b.tets)
