"""The seeded generator: determinism and the stated distributions."""
import numpy as np

from paper_1609_06779_gb300 import synth


def test_generator_is_deterministic_and_well_formed():
    a = synth.random_chains([7, 3, 32], seed=0)
    b = synth.random_chains([7, 3, 32], seed=0)
    for f in ("axes", "frames", "inertias", "offsets"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    assert a.n_chains == 3 and a.n_links_total == 42
    np.testing.assert_allclose(np.linalg.norm(a.axes, axis=1), 1.0, rtol=1e-14)
    J = a.inertias.reshape(-1, 6, 6)
    np.testing.assert_allclose(J, np.swapaxes(J, 1, 2), atol=1e-15)
    assert np.linalg.eigvalsh(J).min() > 0
    m = J[:, 5, 5]
    assert m.min() >= 0.5 and m.max() <= 5.0
    lens = np.linalg.norm(a.frames[:, 9:], axis=1)
    assert lens.min() >= 0.1 and lens.max() <= 0.5
    np.testing.assert_array_equal(a.frames[:, :9], np.tile(np.eye(3).reshape(9), (42, 1)))
    r = synth.random_chains([5], seed=1, random_home_rotation=True)
    R = r.frames[:, :9].reshape(-1, 3, 3)
    np.testing.assert_allclose(R @ np.swapaxes(R, 1, 2), np.broadcast_to(np.eye(3), R.shape),
                               atol=1e-14)


def test_states_and_lengths():
    s = synth.random_states(10000, seed=0)
    assert np.abs(s.q).max() <= np.pi
    assert 0.9 < s.qdot.std() < 1.1 and 9 < s.tau.std() < 11
    n = synth.log_uniform_lengths(5000, 6, 512, seed=0)
    assert n.min() >= 6 and n.max() <= 512
    assert 90 < n.mean() < 140


def test_random_trees_and_loops():
    """Trees: parents precede their children (or are the base), the link draws
    are random_chains' own, the same seed gives the same tree. Loops: links
    within their tree, a != b, at least six joints between the two paths to the
    base, five of them in no other loop of the tree; rotations orthonormal."""
    m = synth.random_trees([1, 7, 20, 32], seed=5)
    c = synth.random_chains([1, 7, 20, 32], seed=5)
    np.testing.assert_array_equal(m.axes, c.axes)
    np.testing.assert_array_equal(m.inertias, c.inertias)
    for t in range(m.n_chains):
        a, z = m.offsets[t], m.offsets[t + 1]
        par = m.parents[a:z]
        assert par[0] == -1
        assert all(-1 <= par[i] < i for i in range(z - a))
    np.testing.assert_array_equal(m.parents, synth.random_trees([1, 7, 20, 32], seed=5).parents)
    big = synth.random_trees([32] * 20, seed=6)
    loops = synth.random_loops(big, per_tree=2, seed=7)
    assert len(loops["a"]) == 40
    for k in range(40):
        t, a, b = loops["tree"][k], int(loops["a"][k]), int(loops["b"][k])
        par = big.parents[big.offsets[t]:big.offsets[t + 1]]

        def path(i):
            out = set()
            while i >= 0:
                out.add(i)
                i = int(par[i])
            return out
        assert a != b and 0 <= b < 32 and -1 <= a < 32
        assert len(path(a) ^ path(b)) >= 6
        for fr in (loops["frame_a"][k], loops["frame_b"][k]):
            R = fr[:9].reshape(3, 3)
            np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-12)
    for t in range(20):
        ks = np.nonzero(loops["tree"] == t)[0]
        par = big.parents[big.offsets[t]:big.offsets[t + 1]]

        def path(i):
            out = set()
            while i >= 0:
                out.add(i)
                i = int(par[i])
            return out
        j0 = path(int(loops["a"][ks[0]])) ^ path(int(loops["b"][ks[0]]))
        j1 = path(int(loops["a"][ks[1]])) ^ path(int(loops["b"][ks[1]]))
        assert len(j1 - j0) >= 5
