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
