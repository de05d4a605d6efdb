"""Input generators: the device-side variants reproduce the host definitions."""
import numpy as np
import pytest

from paper_1803_01262_gb300 import inputs as I

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("shape", [(12, 10, 14), (1, 9, 16), (7, 7, 7)])
def test_random_velocity_torch_matches_numpy(shape):
    h = 1.0 / max(shape)
    ref = I.random_velocity(shape, h, 32, 4, 5)
    got = I.random_velocity_torch(shape, h, 32, 4, 5, device="cpu")
    for a, b in zip(ref, got):
        assert np.abs(a - b.numpy()).max() <= 1e-14


def test_random_velocity_torch_is_divergence_free():
    shape = (16, 12, 20)
    h = 1.0 / 20
    u, v, w = (x.numpy() for x in I.random_velocity_torch(shape, h, 32, 4, 3, device="cpu"))
    div = (u - np.roll(u, 1, 2)) + (v - np.roll(v, 1, 1)) + (w - np.roll(w, 1, 0))
    assert np.abs(div).max() <= 1e-12
    assert max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max()) == pytest.approx(1.0, abs=1e-15)


def test_spheres_phi_torch_matches_numpy():
    shape = (12, 10, 14)
    h = 1.0 / 14
    sph = [((0.3, 0.4, 0.5), 0.2), ((0.7, 0.6, 0.2), 0.15)]
    s = np.maximum(*(I.sphere_distance(shape, h, c, r) for c, r in sph))
    ref = I.tanh_profile(s, 1.5 * h)
    got = I.spheres_phi_torch(shape, h, sph, 1.5 * h, device="cpu", zchunk=5)
    assert np.abs(ref - got.numpy()).max() <= 1e-15
