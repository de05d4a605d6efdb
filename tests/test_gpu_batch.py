"""Batched boxes (one launch per step for every box) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1803_01262_gb300 import cdi
from paper_1803_01262_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def make_boxes(dtype, nbox=7, nmin=5, nmax=40, seed=3):
    raw = I.random_boxes(nbox, nmin, nmax, seed=seed, nmodes=8, kmax=3)
    boxes = []
    for r in raw:
        f = r["fields"]
        Df = sum(1 for s in f.phi.shape if s > 1)
        dt = 0.8 * f.h * f.h / (2 * Df * r["gamma"] * r["eps"])
        boxes.append(dict(dx=f.h, dt=dt, eps=r["eps"], gamma=r["gamma"],
                          u=dev(f.u, dtype), v=dev(f.v, dtype), w=dev(f.w, dtype),
                          phi_a=dev(f.phi, dtype), phi_b=torch.empty(f.phi.shape, dtype=dtype, device="cuda"),
                          fields=f))
    return boxes


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batch_matches_oracle(dtype):
    boxes = make_boxes(dtype)
    b = cdi.Batch(boxes)
    info = b.info()
    assert info["units"] > 0 and info["cells"] == sum(x["fields"].phi.size for x in boxes)
    nsteps = 3
    for i in range(nsteps):
        b.step(1.0)
    st = b.stats()
    t = np.float64 if dtype == torch.float64 else np.float32
    tol = 1e-12 if dtype == torch.float64 else 3e-6
    for i, x in enumerate(boxes):
        f = x["fields"]
        rin = [np.asarray(a, t).astype(np.float64) for a in (f.phi, f.u, f.v, f.w)]
        ref = oracle.run(*rin, f.h, x["dt"], x["eps"], x["gamma"], nsteps)
        ours = b.current(i).double().cpu().numpy()
        assert np.abs(ours - ref).max() <= tol, i
        assert st[i]["steps_run"] == nsteps and st[i]["n_tol_run"] == 0
        assert abs(st[i]["sum"] - ours.sum()) <= 1e-7 * abs(ours.sum())
        assert st[i]["min"] == ours.min() and st[i]["max"] == ours.max()


def test_batch_graph_run_equals_steps():
    boxes = make_boxes(torch.float32, nbox=5, seed=11)
    twins = [dict(x, phi_a=x["phi_a"].clone(), phi_b=torch.empty_like(x["phi_b"])) for x in boxes]
    b1, b2 = cdi.Batch(boxes), cdi.Batch(twins)
    for _ in range(5):
        b1.step(1.0)
    b2.run(2)
    b2.run(3)   # odd: captures the (3, parity 0) graph
    torch.cuda.synchronize()
    assert b1.info()["parity"] == b2.info()["parity"] == 1
    for i in range(len(boxes)):
        assert torch.equal(b1.current(i), b2.current(i))
    s1, s2 = b1.stats(), b2.stats()
    for a, c in zip(s1, s2):
        assert a["sum"] == c["sum"] and a["steps_run"] == c["steps_run"] == 5


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("tile", [0, 1, 2, 3, 5, 6])
@pytest.mark.parametrize("zdepth", [0, 5, 32])
def test_batch_every_launch_configuration(dtype, tile, zdepth):
    """Each work-unit tile and z depth gives the oracle's steps (ragged tiles and chunks)."""
    boxes = make_boxes(dtype, nbox=5, nmin=5, nmax=28, seed=20 + tile)
    b = cdi.Batch(boxes)
    b.set_launch(tile, zdepth)
    cfg = b.get_launch()
    assert cfg["tile"] == tile and cfg["zdepth"] == zdepth and cfg["units"] > 0
    for _ in range(2):
        b.step(1.0)
    st = b.stats()
    t = np.float64 if dtype == torch.float64 else np.float32
    tol = 1e-12 if dtype == torch.float64 else 3e-6
    for i, x in enumerate(boxes):
        f = x["fields"]
        rin = [np.asarray(a, t).astype(np.float64) for a in (f.phi, f.u, f.v, f.w)]
        ref = oracle.run(*rin, f.h, x["dt"], x["eps"], x["gamma"], 2)
        ours = b.current(i).double().cpu().numpy()
        assert np.abs(ours - ref).max() <= tol, i
        assert st[i]["steps_run"] == 2
        assert st[i]["min"] == ours.min() and st[i]["max"] == ours.max()


def test_batch_autotune_keeps_state_and_records():
    boxes = make_boxes(torch.float32, nbox=6, nmin=8, nmax=40, seed=31)
    b = cdi.Batch(boxes)
    b.step(1.0)
    state = [b.current(i).clone() for i in range(len(boxes))]
    before = b.stats()
    ms = b.autotune(reps=1)
    assert ms > 0
    cfg = b.get_launch()
    assert cfg["tile"] in (0, 1, 2, 3, 5) and cfg["units"] > 0
    assert b.info()["parity"] == 1
    for i in range(len(boxes)):
        assert torch.equal(b.current(i), state[i])
    after = b.stats()
    for x, y in zip(before, after):
        assert x == y
    b.step(1.0)
    for i, x in enumerate(boxes):
        f = x["fields"]
        rin = [np.asarray(a, np.float32).astype(np.float64) for a in (f.phi, f.u, f.v, f.w)]
        ref = oracle.run(*rin, f.h, x["dt"], x["eps"], x["gamma"], 2)
        assert np.abs(b.current(i).double().cpu().numpy() - ref).max() <= 3e-6, i
    assert b.stats()[0]["steps_run"] == 2


def flat_boxes(dtype, sizes, seed):
    """2D boxes (nz == 1): a smoothed random field and a random divergence-free velocity."""
    boxes = []
    for i, (ny, nx) in enumerate(sizes):
        shape = (1, ny, nx)
        h = 1.0 / max(shape)
        phi = I.random_phi(shape, seed + i, smooth=True)
        u, v, w = I.random_velocity(shape, h, 8, 3, seed + 50 + i)
        eps, gamma = 1.1 * h, 1.0
        dt = 0.8 * h * h / (2 * 2 * gamma * eps)
        f = I.Fields(phi, u, v, w, h, I.face_umax(u, v, w))
        boxes.append(dict(dx=h, dt=dt, eps=eps, gamma=gamma, u=dev(u, dtype), v=dev(v, dtype),
                          w=dev(w, dtype), phi_a=dev(phi, dtype),
                          phi_b=torch.empty(shape, dtype=dtype, device="cuda"), fields=f))
    return boxes


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("mixed", [False, True])
def test_batch_of_2d_boxes_matches_oracle(dtype, mixed):
    """A batch of only 2D boxes runs the single-plane kernel; mixed with 3D boxes, the 3D
    one.  Both give the oracle's steps, every launch configuration."""
    boxes = flat_boxes(dtype, [(7, 9), (33, 40), (16, 64), (1, 37), (50, 50)], 11)
    if mixed:
        boxes += make_boxes(dtype, nbox=3, seed=9)
    t = np.float64 if dtype == torch.float64 else np.float32
    tol = 1e-12 if dtype == torch.float64 else 3e-6
    for tile in range(4):
        for x in boxes:
            x["phi_a"].copy_(dev(x["fields"].phi, dtype))
        b = cdi.Batch(boxes)
        b.set_launch(tile, 0)
        for i in range(3):
            b.step(0.9)
        st = b.stats()
        for i, x in enumerate(boxes):
            f = x["fields"]
            rin = [np.asarray(a, t).astype(np.float64) for a in (f.phi, f.u, f.v, f.w)]
            ref = rin[0]
            for _ in range(3):
                ref = oracle.step(ref, *rin[1:], f.h, x["dt"], x["eps"], x["gamma"], 0.9)
            ours = b.current(i).double().cpu().numpy()
            assert np.abs(ours - ref).max() <= tol, (tile, i)
            assert st[i]["min"] == ours.min() and st[i]["max"] == ours.max()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_whole_plane_tile(dtype):
    """Batch tile 4 (one unit per whole 2D box, the plane held in shared memory) gives the
    oracle's steps and, bit for bit, the single-plane tiles' fields, extrema and counts
    (the sums group the cells differently), stepped one launch at a time and as a graph
    run; extents 1 and 2 included."""
    sizes = [(7, 9), (33, 40), (16, 64), (1, 37), (37, 1), (2, 5), (1, 1), (50, 50), (3, 2)]
    boxes = flat_boxes(dtype, sizes, 23)
    twins = [dict(x, phi_a=x["phi_a"].clone(), phi_b=torch.empty_like(x["phi_b"])) for x in boxes]
    bp, bt = cdi.Batch(boxes), cdi.Batch(twins)
    bp.set_launch(4, 0)
    bt.set_launch(0, 0)
    lp = bp.get_launch()
    assert lp["tile"] == 4 and lp["units"] == len(sizes)
    for _ in range(3):
        bp.step(0.9)
        bt.step(0.9)
    sp, stt = bp.stats(), bt.stats()
    t = np.float64 if dtype == torch.float64 else np.float32
    tol = 1e-12 if dtype == torch.float64 else 3e-6
    for i, x in enumerate(boxes):
        ours = bp.current(i)
        assert torch.equal(ours, bt.current(i)), i
        same_stats(sp[i], stt[i], dtype)
        f = x["fields"]
        rin = [np.asarray(a, t).astype(np.float64) for a in (f.phi, f.u, f.v, f.w)]
        ref = rin[0]
        for _ in range(3):
            ref = oracle.step(ref, *rin[1:], f.h, x["dt"], x["eps"], x["gamma"], 0.9)
        assert np.abs(ours.double().cpu().numpy() - ref).max() <= tol, i
    bp.run(4)
    bt.run(4)
    for i, (a, b) in enumerate(zip(bp.stats(), bt.stats())):
        assert torch.equal(bp.current(i), bt.current(i)), i
        same_stats(a, b, dtype)


def same_stats(a, b, dtype):
    """Equal statistics records: extrema and counts exactly, sums to rounding."""
    rel = 1e-13 if dtype == torch.float64 else 1e-6
    for k in a:
        if k in ("mass", "sum"):
            assert abs(a[k] - b[k]) <= rel * max(abs(b[k]), 1e-300), k
        else:
            assert a[k] == b[k], k


def test_whole_plane_tile_refusals():
    """Tile 4 is refused for 3D boxes and for planes larger than shared memory (the launch
    stays as it was), and the autotuner then does not try it."""
    b3 = cdi.Batch(make_boxes(torch.float32, nbox=2, seed=5))
    with pytest.raises(cdi.CDIError):
        b3.set_launch(4, 0)
    assert b3.get_launch()["tile"] == 0
    big = cdi.Batch(flat_boxes(torch.float64, [(200, 200), (10, 10)], 3))  # 3 x 40000 x 8 B
    with pytest.raises(cdi.CDIError):
        big.set_launch(4, 0)
    big.autotune(reps=1)
    assert big.get_launch()["tile"] != 4


def test_whole_plane_batches_of_different_sizes():
    """Two batches whose planes need different shared memory (about 190 KB and 3 KB),
    stepped alternately with tile 4: both follow the oracle."""
    A = flat_boxes(torch.float64, [(90, 90), (20, 30)], 7)
    B = flat_boxes(torch.float64, [(10, 12)], 8)
    ba, bb = cdi.Batch(A), cdi.Batch(B)
    ba.set_launch(4, 0)
    bb.set_launch(4, 0)
    for _ in range(2):
        ba.step(1.0)
        bb.step(1.0)
    for bt, boxes in ((ba, A), (bb, B)):
        for i, x in enumerate(boxes):
            f = x["fields"]
            ref = oracle.run(f.phi, f.u, f.v, f.w, f.h, x["dt"], x["eps"], x["gamma"], 2)
            assert np.abs(bt.current(i).cpu().numpy() - ref).max() <= 1e-12, i


def odd_boxes(dtype, shapes, seed):
    """3D (and 2D) boxes of the given (nz, ny, nx) shapes with random smooth fields."""
    boxes = []
    for i, shape in enumerate(shapes):
        h = 1.0 / max(shape)
        phi = I.random_phi(shape, seed + i, smooth=True)
        u, v, w = I.random_velocity(shape, h, 8, 3, seed + 70 + i)
        eps, gamma = 1.2 * h, 1.0
        Df = sum(1 for q in shape if q > 1)
        dt = 0.8 * h * h / (2 * max(Df, 1) * gamma * eps)
        f = I.Fields(phi, u, v, w, h, I.face_umax(u, v, w))
        boxes.append(dict(dx=h, dt=dt, eps=eps, gamma=gamma, u=dev(u, dtype), v=dev(v, dtype),
                          w=dev(w, dtype), phi_a=dev(phi, dtype),
                          phi_b=torch.empty(shape, dtype=dtype, device="cuda"), fields=f))
    return boxes


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("zdepth", [0, 3, 16])
def test_band_tile_bit_for_bit(dtype, zdepth):
    """Batch tile 5 (bands of whole rows, 16-byte staging at any row alignment) gives the
    one-cell-per-thread tiles' fields bit for bit and the oracle's steps: rows of one cell,
    one row, rows wider than a band of several rows (one row per band), bands that wrap in y
    several times, a 2D box among 3D ones, stepped one launch at a time and as a graph run."""
    shapes = [(5, 7, 9), (9, 17, 33), (4, 1, 45), (6, 3, 1), (3, 2, 2), (7, 40, 150), (2, 5, 400),
              (1, 23, 50), (11, 19, 70), (8, 64, 16), (3, 1, 1)]
    boxes = odd_boxes(dtype, shapes, 31)
    twins = [dict(x, phi_a=x["phi_a"].clone(), phi_b=torch.empty_like(x["phi_b"])) for x in boxes]
    bb, bt = cdi.Batch(boxes), cdi.Batch(twins)
    bb.set_launch(5, zdepth)
    bt.set_launch(0, zdepth)
    assert bb.get_launch()["tile"] == 5
    for i in range(3):
        bb.step(0.9)
        bt.step(0.9)
    sb, st = bb.stats(), bt.stats()
    t = np.float64 if dtype == torch.float64 else np.float32
    tol = 1e-12 if dtype == torch.float64 else 3e-6
    for i, x in enumerate(boxes):
        ours = bb.current(i)
        assert torch.equal(ours, bt.current(i)), (i, shapes[i])
        same_stats(sb[i], st[i], dtype)
        f = x["fields"]
        rin = [np.asarray(a, t).astype(np.float64) for a in (f.phi, f.u, f.v, f.w)]
        ref = rin[0]
        for _ in range(3):
            ref = oracle.step(ref, *rin[1:], f.h, x["dt"], x["eps"], x["gamma"], 0.9)
        assert np.abs(ours.double().cpu().numpy() - ref).max() <= tol, (i, shapes[i])
    bb.run(4)
    bt.run(4)
    for i, (a, b) in enumerate(zip(bb.stats(), bt.stats())):
        assert torch.equal(bb.current(i), bt.current(i)), i
        same_stats(a, b, dtype)


def test_band_tile_refusals():
    """Tile 5 is refused for a batch of 2D boxes only and for rows wider than a band (the
    launch stays as it was)."""
    flat = cdi.Batch(flat_boxes(torch.float32, [(7, 9), (16, 64)], 3))
    with pytest.raises(cdi.CDIError):
        flat.set_launch(5, 0)
    assert flat.get_launch()["tile"] == 0
    wide = cdi.Batch(odd_boxes(torch.float32, [(3, 4, 1100)], 5))
    with pytest.raises(cdi.CDIError):
        wide.set_launch(5, 0)
    wide.autotune(reps=1)
    assert wide.get_launch()["tile"] != 5


def _twin_boxes(shapes, dtype, seed):
    boxes = []
    for i, s in enumerate(shapes):
        nz, ny, nx = s
        h = 1.0 / max(s)
        phi = dev(I.random_phi(s, seed + i, smooth=True), dtype)
        vel = [dev(x, dtype) for x in I.random_velocity(s, h, 8, 3, seed + 50 + i)]
        eps, gamma = 1.1 * h, 1.0
        boxes.append(dict(dx=h, dt=0.1 * h * h / (gamma * eps), eps=eps, gamma=gamma, u=vel[0], v=vel[1],
                          w=vel[2], phi_a=phi, phi_b=torch.empty_like(phi)))
    twins = [dict(x, phi_a=x["phi_a"].clone(), phi_b=torch.empty_like(x["phi_b"])) for x in boxes]
    return boxes, twins


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_padded_band_tile_bit_for_bit(dtype):
    """Tile 6 steps the batch's padded copies of the boxes (rows padded to 16 bytes, with
    periodic ghost cells) and writes the caller's arrays on the last step of each call.  On
    boxes of every row alignment, degenerate extents included, run() and step() give tile 0's
    fields bit for bit, and a state the caller writes between calls is the one stepped."""
    shapes = [(6, 9, 1), (5, 7, 2), (8, 11, 3), (9, 21, 68), (12, 33, 35), (1, 40, 61), (20, 1, 17),
              (7, 3, 4), (16, 48, 128), (3, 2, 5)]
    boxes, twins = _twin_boxes(shapes, dtype, 70)
    b0, b6 = cdi.Batch(boxes), cdi.Batch(twins)
    b0.set_launch(0, 0)
    b6.set_launch(6, 4)
    assert b6.get_launch()["tile"] == 6
    for b in (b0, b6):
        b.run(3)
    for i in range(len(shapes)):
        assert torch.equal(b0.current(i), b6.current(i)), ("run", i)
    for b in (b0, b6):
        b.step(1.0)
        b.step(0.5)
    for i in range(len(shapes)):
        assert torch.equal(b0.current(i), b6.current(i)), ("step", i)
    for b in (b0, b6):      # the caller changes the state between calls
        for i in range(len(shapes)):
            b.current(i).mul_(0.75)
        b.run(2)
    s0, s6 = b0.stats(), b6.stats()
    for i in range(len(shapes)):
        assert torch.equal(b0.current(i), b6.current(i)), ("written", i)
        assert s0[i]["min"] == s6[i]["min"] and s0[i]["max"] == s6[i]["max"]
        assert s0[i]["steps_run"] == s6[i]["steps_run"] == 7
        assert s6[i]["sum"] == pytest.approx(s0[i]["sum"], rel=1e-12 if dtype == torch.float64 else 1e-6)


STAT_KEYS = ("mass", "sum", "min", "max", "n_strict", "n_tol", "min_run", "max_run", "n_strict_run",
             "n_tol_run", "steps_run")


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("tile,zdepth", [(0, 0), (2, 8), (3, 0), (5, 0), (5, 16), (6, 0), (6, 8)])
def test_overlapping_run_equals_single_steps(dtype, tile, zdepth):
    """The launches of a run overlap: a unit of step i + 1 waits only for its own box to
    finish step i.  Forty uneven boxes (more units than blocks, so blocks of two steps share
    the SMs): fields and every statistic equal those of the same steps launched one at a
    time, bit for bit, over runs of several lengths, a run after single steps, and a run
    longer than any before (new counters)."""
    boxes = make_boxes(dtype, nbox=40, nmin=4, nmax=48, seed=60 + tile)
    twins = [dict(x, phi_a=x["phi_a"].clone(), phi_b=torch.empty_like(x["phi_b"])) for x in boxes]
    b1, b2 = cdi.Batch(boxes), cdi.Batch(twins)
    try:
        b1.set_launch(tile, zdepth)
    except cdi.CDIError:
        pytest.skip("the tile does not apply to these boxes")
    b2.set_launch(tile, zdepth)
    for n, single_first in ((7, False), (2, False), (3, True), (12, False), (1, False)):
        if single_first:
            b1.step(1.0)
            b2.step(1.0)
        for _ in range(n):
            b1.step(1.0)
        b2.run(n)
        torch.cuda.synchronize()
        for i in range(len(boxes)):
            assert torch.equal(b1.current(i), b2.current(i)), (n, i)
        s1, s2 = b1.stats(), b2.stats()
        for i, (a, c) in enumerate(zip(s1, s2)):
            for k in STAT_KEYS:
                assert a[k] == c[k], (n, i, k, a[k], c[k])


def test_run_wait_times_out_and_the_batch_stays_usable():
    """The run's per-box wait is bounded: a probe launch whose units wait for a step their
    boxes never reach reports CDI_ERR_TIMEOUT within the limit, steps nothing, and the next
    steps and runs are those of an untouched twin."""
    import time
    boxes = make_boxes(torch.float32, nbox=12, nmin=6, nmax=32, seed=71)
    twins = [dict(x, phi_a=x["phi_a"].clone(), phi_b=torch.empty_like(x["phi_b"])) for x in boxes]
    b1, b2 = cdi.Batch(boxes), cdi.Batch(twins)
    b1.run(3)
    b2.run(3)
    t0 = time.perf_counter()
    with pytest.raises(cdi.CDIError) as e:
        b1.probe_box_wait(0.05)
    assert e.value.code == cdi.CDI_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert b1.info()["parity"] == b2.info()["parity"]
    b1.step(1.0)
    b2.step(1.0)
    b1.run(4)
    b2.run(4)
    torch.cuda.synchronize()
    for i in range(len(boxes)):
        assert torch.equal(b1.current(i), b2.current(i)), i
    s1, s2 = b1.stats(), b2.stats()     # raises if the status word were still set
    for a, c in zip(s1, s2):
        for k in STAT_KEYS:
            assert a[k] == c[k], k
    with pytest.raises(cdi.CDIError):
        b1.probe_box_wait(5.0)          # limit out of range
