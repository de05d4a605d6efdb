"""Driver of the checked-build test (run in its own process with CDI_LIBRARY=checked, since
two builds of the library must not share a process).

Steps odd shapes through every forward tile that takes them, the adjoint tiles and a small
batch with the bounds-checked library, each against the FP64 oracle; every statistics
read-back would raise CDI_ERR_BOUNDS had a kernel derived an index out of range.  Then makes
the check record one planted index and expects the error.  Prints "checked ok".
"""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1803_01262_gb300 import build as B  # noqa: E402


def main():
    assert os.environ.get("CDI_LIBRARY") == "checked"
    B.build(checked=True)
    from paper_1803_01262_gb300 import cdi
    from paper_1803_01262_gb300 import inputs as I
    assert cdi.is_checked_build()
    tol = {torch.float64: 1e-12, torch.float32: 1e-6}
    npt = {torch.float64: np.float64, torch.float32: np.float32}
    shapes = [(1, 5, 3), (3, 1, 8), (7, 19, 45), (33, 20, 70), (1, 130, 67), (19, 17, 40), (5, 32, 128)]
    for dtype in (torch.float64, torch.float32):
        for shape in shapes:
            nz, ny, nx = shape
            h = 1.0 / max(shape)
            phi = I.random_phi(shape, 3 + nx, smooth=True)
            u, v, w = I.random_velocity(shape, h, 8, 3, 5 + ny)
            r = [np.asarray(x, npt[dtype]).astype(np.float64) for x in (phi, u, v, w)]
            eps, gamma = 1.2 * h, 1.1
            dt = 0.1 * h * h / (gamma * eps)
            g = cdi.Grid(nx, ny, nz, h, dtype)
            vel = [torch.from_numpy(x).to("cuda", dtype) for x in (u, v, w)]
            g.set_velocity(*vel)
            a = torch.from_numpy(phi).to("cuda", dtype)
            ref = oracle.step(*r, h, dt, eps, gamma, 0.9, tiny=oracle.floor_of(npt[dtype]))
            for tile in range(cdi.FWD_TILES):
                try:
                    g.set_launch(cdi.CDI_KERNEL_FORWARD, tile, 0, 0)
                except cdi.CDIError:
                    continue  # tile does not take this shape
                b = torch.empty_like(a)
                g.step(a, b, dt, eps, gamma, 0.9)
                g.stats()  # raises CDI_ERR_BOUNDS if any index was out of range
                err = float(np.abs(b.double().cpu().numpy() - ref).max())
                assert err <= tol[dtype], (dtype, shape, tile, err)
            lam = np.random.default_rng(nx).standard_normal(shape)
            ra = oracle.adjoint(*r, np.asarray(lam, npt[dtype]).astype(np.float64), h, dt, eps, gamma,
                                tiny=oracle.adjoint_floor_of(npt[dtype]))
            for tile in range(cdi.ADJ_TILES):
                try:
                    g.set_launch(cdi.CDI_KERNEL_ADJOINT, tile, 0, 0)
                except cdi.CDIError:
                    continue
                out = torch.empty_like(a)
                g.step_adjoint(a, torch.from_numpy(lam).to("cuda", dtype), out, dt, eps, gamma)
                g.mass_and_bounds(out)  # reads (and clears) the status words
                aerr = float(np.abs(out.double().cpu().numpy() - ra).max()) / max(1.0, float(np.abs(ra).max()))
                assert aerr <= (1e-12 if dtype == torch.float64 else 2e-6), (dtype, shape, tile, aerr)
            g.close()
    # a small batch of uneven boxes, every batch tile from the same state
    boxes, refs, init = [], [], []
    for i, shape in enumerate([(9, 17, 33), (4, 40, 21), (1, 23, 50)]):
        h = 1.0 / max(shape)
        phi = I.random_phi(shape, 40 + i, smooth=True)
        u, v, w = I.random_velocity(shape, h, 8, 3, 50 + i)
        eps, gamma = 1.3 * h, 1.0
        dt = 0.1 * h * h / (gamma * eps)
        d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to("cuda", torch.float64)
        boxes.append(dict(dx=h, dt=dt, eps=eps, gamma=gamma, u=d(u), v=d(v), w=d(w), phi_a=d(phi),
                          phi_b=torch.empty(shape, dtype=torch.float64, device="cuda")))
        init.append(d(phi))
        refs.append(oracle.step(phi, u, v, w, h, dt, eps, gamma, 1.0, tiny=oracle.floor_of(np.float64)))
    for tile in range(4):
        for b, p0 in zip(boxes, init):
            b["phi_a"].copy_(p0)
        bt = cdi.Batch(boxes)
        bt.set_launch(tile, 8)
        bt.step()
        bt.stats()  # raises CDI_ERR_BOUNDS if any index was out of range
        for i in range(len(boxes)):
            got = bt.current(i).cpu().numpy()
            assert np.abs(got - refs[i]).max() <= 1e-12, (tile, i)
        bt.close()
    # the check itself: one planted index must be recorded
    g = cdi.Grid(8, 8, 8, 1.0 / 8, torch.float32)
    try:
        g.probe_bounds_check()
    except cdi.CDIError as e:
        assert e.code == cdi.CDI_ERR_BOUNDS, e
    else:
        raise AssertionError("the checked build did not record a planted index")
    print("checked ok")


if __name__ == "__main__":
    main()
