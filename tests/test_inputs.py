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


def test_random_boxes_recipe():
    """The batched workload's boxes: edges in [nmin, nmax], the shortest edge of length 1,
    phi a tanh profile in [0, 1] with interface inside the box, a discretely divergence-free
    velocity with U = 1, eps/dx in {1, 1.5}, and gamma exactly on the crossover line
    (Eq. 17: eps/dx = (gamma/U + 1) / (2 gamma/U))."""
    from paper_1803_01262_gb300 import build as B
    from paper_1803_01262_gb300 import cdi
    B.build()   # cdi.check_condition is a host entry point of the library
    boxes = I.random_boxes(6, 8, 20, seed=5, nmodes=8, kmax=3)
    assert len(boxes) == 6
    for b in boxes:
        f = b["fields"]
        nz, ny, nx = f.phi.shape
        assert all(8 <= n <= 20 for n in (nx, ny, nz))
        assert f.h == 1.0 / min(nx, ny, nz)
        assert f.phi.min() >= 0.0 and f.phi.max() <= 1.0 and (f.phi > 0.5).any() and (f.phi < 0.5).any()
        div = (f.u - np.roll(f.u, 1, 2)) + (f.v - np.roll(f.v, 1, 1)) + (f.w - np.roll(f.w, 1, 0))
        assert np.abs(div).max() < 1e-12 and abs(f.U - 1.0) < 1e-15
        eoh = b["eps"] / f.h
        assert b["eps_over_h"] in (1.0, 1.5) and abs(eoh - b["eps_over_h"]) < 1e-15
        g = b["gamma"] / f.U
        assert abs(eoh - (g + 1) / (2 * g)) < 1e-14
        assert cdi.check_condition(eoh, g, 0.1, 3)
