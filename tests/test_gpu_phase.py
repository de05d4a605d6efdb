"""Phase-diagram sweep of the (eps/dx, gamma/|u|) plane as one batched workload
(Section 2.2: the crossover line of Eq. 17, Table 2's uniform-velocity drop)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1803_01262_gb300 import inputs as I
from paper_1803_01262_gb300 import phase as P

pytestmark = pytest.mark.gpu

# Table 2: points 1-5 stay bounded, 6-7 do not
TABLE2 = [(1.5, 0.5, True), (1.0, 1.0, True), (5 / 6, 1.5, True), (1.5, 1.5, True),
          (0.9, 0.9, True), (0.8, 0.8, False), (0.7, 0.7, False)]


def test_table2_points_in_one_batch_match_the_oracle():
    """The seven Table 2 points as one batch: the classification of the paper, and for each
    box the oracle replaying it with the same step and step count gives the same classification,
    and for a bounded box the same run extremes (min and max of phi over every step) to 1e-9.
    (The extremes sit in the far field, where the unit normal follows rounding-level
    gradients, so 1e-16 differences per step grow to ~1e-11 over the run.)"""
    pts = [(e, g) for e, g, _ in TABLE2]
    rows, info = P.phase_diagram(pts)
    assert [r["bounded"] for r in rows] == [b for _, _, b in TABLE2]
    assert [r["sufficient"] for r in rows] == [True] * 5 + [False] * 2
    tol = np.finfo(np.float64).eps
    for r, (e, g, _) in zip(rows, TABLE2):
        f, _ = I.drop_2d_uniform(e)
        p, mn, mx, bad = f.phi, np.inf, -np.inf, 0
        for _ in range(info["nsteps"]):
            p = oracle.step(p, f.u, f.v, f.w, f.h, r["dt"], e * f.h, g)
            mn, mx = min(mn, p.min()), max(mx, p.max())
            bad += int(((p < -tol) | (p > 1 + tol)).sum())
        assert (bad == 0) == r["bounded"], (e, g, bad, r["n_tol_run"])
        if bad:
            # once phi leaves [0, 1], phi (1 - phi) < 0 makes the sharpening anti-diffusive there
            # and two runs drift apart: counts and extremes agree to 1%
            assert abs(r["n_tol_run"] - bad) <= 0.01 * bad, (e, g, bad, r["n_tol_run"])
            assert abs(r["min_run"] - mn) <= 0.01 * abs(mn) and abs(r["max_run"] - mx) <= 0.01 * abs(mx)
        else:
            assert abs(r["min_run"] - mn) <= 1e-9 and abs(r["max_run"] - mx) <= 1e-9, (e, g, r, mn, mx)


def test_sweep_bounded_wherever_the_condition_holds():
    """A 12 x 12 grid of (eps/dx, gamma/|u|) in one batch: every point that satisfies the
    sufficient condition (Eq. 17 with A <= 1/(2 D_f)) stays in [0, 1] to machine precision;
    the grid has unbounded points below the line, and bounded ones below it too (the bounded
    region extends past the sufficient condition, as Table 2's point 5 region shows)."""
    e = np.linspace(0.55, 2.0, 12)
    g = np.linspace(0.3, 3.0, 12)
    pts = [(float(a), float(b)) for a in e for b in g]
    rows, info = P.phase_diagram(pts)
    assert info["cells"] == 144 * 50 * 50
    suff = [r for r in rows if r["sufficient"]]
    assert len(suff) > 20 and all(r["bounded"] for r in suff)
    assert any(not r["bounded"] for r in rows)
    assert any(r["bounded"] and not r["sufficient"] for r in rows)
    # conservation holds everywhere, bounded or not
    bt = info["batch"]
    for i, r in enumerate(rows):
        f, _ = I.drop_2d_uniform(r["eps_over_dx"])
        cur = bt.current(i).double().sum().item()
        assert abs(cur - f.phi.sum()) <= 1e-11 * f.phi.sum()


def test_fp32_sweep_matches_fp64_classification_above_the_line():
    """The FP32 batch (tolerance FLT_EPSILON) agrees that the sufficient region is bounded."""
    pts = [(float(a), float(b)) for a in np.linspace(0.6, 2.0, 6) for b in np.linspace(0.5, 3.0, 6)]
    rows, _ = P.phase_diagram(pts, dtype=torch.float32)
    assert all(r["bounded"] for r in rows if r["sufficient"])


def test_face_product_sweep_matches_the_oracle():
    """The face-product sharpening in the batched sweep: a few points on and around the
    crossover line replayed by the oracle's face-product step give the same classification
    over 300 steps, and the same fields to 1e-10 over the first 30; the whole-plane tile and
    tile 0 give the same fields bit for bit.  (Each step agrees with the oracle to 1e-12,
    tests/test_gpu_face.py; over hundreds of steps the bulk, where the unit normal follows
    rounding-level gradients and the face form's sharpening does not vanish with them,
    amplifies rounding differences of the two evaluation orders to ~1e-6.)"""
    pts = [(1.5, 0.5), (1.0, 1.0), (0.9, 0.9), (0.7, 0.7), (2.0, 3.0)]
    rows, info = P.phase_diagram(pts, nsteps=300, autotune=False, sharpen="face")
    assert info["batch"].get_sharpening() == "face"
    tol = np.finfo(np.float64).eps
    for i, (r, (e, g)) in enumerate(zip(rows, pts)):
        f, _ = I.drop_2d_uniform(e)
        p, bad = f.phi, 0
        for _ in range(300):
            p = oracle.step(p, f.u, f.v, f.w, f.h, r["dt"], e * f.h, g, sharpen="face")
            bad += int(((p < -tol) | (p > 1 + tol)).sum())
        assert (bad == 0) == r["bounded"], (e, g, bad, r["n_tol_run"])
    # the first 30 steps field by field; tile 0 and the whole-plane tile bit for bit
    from paper_1803_01262_gb300 import cdi
    boxes = P.phase_boxes(pts)
    twins = [dict(x, phi_a=x["phi_a"].clone(), phi_b=torch.empty_like(x["phi_b"])) for x in boxes]
    b0, b4 = cdi.Batch(boxes), cdi.Batch(twins)
    for b, tile in ((b0, 0), (b4, 4)):
        b.set_sharpening("face")
        b.set_launch(tile, 0)
        b.run(30)
    for i, (e, g) in enumerate(pts):
        assert torch.equal(b0.current(i), b4.current(i)), i
        f, _ = I.drop_2d_uniform(e)
        x = boxes[i]
        ref = oracle.run(f.phi, f.u, f.v, f.w, f.h, x["dt"], x["eps"], x["gamma"], 30, sharpen="face")
        assert np.abs(b0.current(i).cpu().numpy() - ref).max() <= 1e-10, (e, g)
    with pytest.raises(cdi.CDIError):
        b0.set_launch(1, 0)   # the face form runs on tiles 0 and 4 only
