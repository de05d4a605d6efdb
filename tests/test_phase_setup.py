"""Host side of the phase-diagram sweep (no GPU): each point's box is Table 2's drop
(Section 3.2.1) with its own eps and gamma, and its Euler step is the smaller of the
diffusive and the mixed advective-diffusive limits."""
import math

import numpy as np
import pytest
import torch

from paper_1803_01262_gb300 import phase as P


def test_period_and_step_rule():
    # one period: the drop, advected by (sqrt2/2, sqrt2/2) in a 2 x 2 box, returns at t = 2 sqrt2
    assert P.PERIOD == 2.0 * math.sqrt(2.0)
    h = 2.0 / 50
    for eoh, gu in ((1.5, 0.5), (1.0, 1.0), (0.7, 0.7), (2.0, 3.0), (0.55, 0.3)):
        eps, gamma = eoh * h, gu
        dif = h * h / (4.0 * gamma * eps)          # A = dt gamma eps / h^2 = 1/(2 D_f), D_f = 2
        adv = h / (math.sqrt(2.0) + 2.0 * gamma)   # dx / (max u + max v + 2 gamma)
        assert P.euler_dt(eoh, gu) == pytest.approx(min(dif, adv), rel=1e-15)
        A = P.euler_dt(eoh, gu) * gamma * eps / h ** 2
        assert A <= 0.25 * (1 + 1e-15)


def test_boxes_are_table2_drops():
    pts = [(1.0, 1.0), (0.8, 0.8), (1.5, 0.5)]
    boxes = P.phase_boxes(pts, n=50, dtype=torch.float64, device="cpu")
    assert len(boxes) == len(pts)
    for (eoh, gu), b in zip(pts, boxes):
        h = b["dx"]
        assert h == 2.0 / 50 and b["eps"] == eoh * h and b["gamma"] == gu
        assert b["dt"] == P.euler_dt(eoh, gu, 50)
        phi = b["phi_a"].numpy()
        assert phi.shape == (1, 50, 50) and b["phi_b"].shape == phi.shape
        # diameter-1 drop at the box centre: the 0.5 level encloses an area of about pi/4
        assert abs((phi > 0.5).sum() * h * h - math.pi / 4) < 0.05
        assert np.allclose(b["u"].numpy(), math.sqrt(2.0) / 2) and np.allclose(b["v"].numpy(), math.sqrt(2.0) / 2)
        assert not b["w"].numpy().any()
