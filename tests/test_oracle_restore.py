"""Pins of the water-removal oracle (per-pixel inverse of Eq. 5)."""
import numpy as np

from oracle import restore as RS


def _compose(J, z, med):
    """Eq. 5 per pixel, written out independently of the oracle."""
    out = np.empty_like(J)
    for c in range(3):
        a = np.exp(-med[c] * z)
        b = np.exp(-med[3 + c] * z)
        out[c] = J[c] * a + med[6 + c] * (1 - b)
    return out


def test_round_trip_recovers_the_direct_colour():
    rng = np.random.default_rng(0)
    J = rng.uniform(0, 1, (3, 20, 30))
    z = rng.uniform(0.5, 15, (20, 30))
    med = np.concatenate([rng.uniform(0.05, 0.6, 6), rng.uniform(0.05, 0.4, 3)])
    np.testing.assert_allclose(RS.restore(_compose(J, z, med), z, med), J, rtol=1e-9, atol=1e-12)


def test_no_water_is_the_identity_and_pure_backscatter_is_black():
    rng = np.random.default_rng(1)
    I = rng.uniform(0, 1, (3, 8, 9))
    z = rng.uniform(1, 9, (8, 9))
    assert np.array_equal(RS.restore(I, z, np.zeros(9)), I)
    med = np.array([0.3, 0.2, 0.1, 0.4, 0.3, 0.2, 0.25, 0.2, 0.15])
    pure = _compose(np.zeros((3, 8, 9)), z, med)
    np.testing.assert_allclose(RS.restore(pure, z, med), 0.0, atol=1e-15)


def test_darker_than_backscatter_clips_to_zero():
    med = np.array([0.3, 0.2, 0.1, 0.4, 0.3, 0.2, 0.25, 0.2, 0.15])
    z = np.full((2, 2), 5.0)
    I = _compose(np.zeros((3, 2, 2)), z, med) - 0.01
    assert np.all(RS.restore(I, z, med) == 0.0)
