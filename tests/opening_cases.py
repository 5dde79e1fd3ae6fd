"""Hand-built group/cell pairs that pin the opening rule of the tree walk
(Sec. 2.4, Barnes-Hut with opening angle theta, plus the r_out box test that
keeps every accepted cell beyond the changeover of Eq. 6) one decision at a
time.  Inputs and expected decisions only: no tree arithmetic lives here.

Layout (every coordinate dyadic, so every FP64 step below is exact):
- a massless ballast of 600 coincident particles at (4, 4, 4) fixes the
  bounding cube at [0, 4]^3 and makes the root hold more than 16 G particles,
  so that walk groups are cut from the root's children (G = 32);
- the group: g1 = (0, 0, 0) and g2 = (1, gy, 0), unit masses, in octant 0 of
  the root (a leaf at leaf capacity 2): box [0, 1] x [0, gy] x [0, 0];
- the cell: c1 = (X, 0, 0) of mass 3 and c2 = (X + sx, sy, 0) of mass 1, in
  octant 4 (2 <= x < 4): a leaf.  Its centre of mass is (X + sx/4, sy/4, 0),
  its box centre (X + sx/2, sy/2, 0), so delta_c = |(sx, sy)|/4; its size l_c
  is max(sx, sy).  With gy >= sy/4 the distance from the group box to the
  centre of mass runs along x alone: X + sx/4 - 1.  The box-to-box distance is
  X - 1.

For the group the walk opens the root and the group's own leaf, and accepts
the ballast's octant (a massless point: opening radius 0, far beyond r_out),
so the expected counts are
    n_cell = 1 + (cell accepted),  n_part = 2 + 2 * (cell opened).

Each case states the hand-computed decision and which plausible mistake in
the rule it would expose (by flipping the decision).
"""
from __future__ import annotations

import numpy as np

BALLAST = 600
GROUP_SIZE = 32
LEAF_CAP = 2

# (id, theta, r_out, X, sx, sy, gy, opened, why)
CASES = [
    # theta = 0.5, cell along x of size 1: r_open = 1/0.5 + 1/4 = 2.25, d = X - 0.75
    ("mac_inside", 0.5, 0.01, 3.0 - 2.0 ** -20, 1.0, 0.0, 0.0, True,
     "d = 2.25 - 2^-20 < 2.25: opened"),
    ("mac_equal", 0.5, 0.01, 3.0, 1.0, 0.0, 0.0, False,
     "d = 2.25 = r_open: accepted by the strict '<'; '<=' would open it, and so would "
     "measuring to the cell box (d = 2)"),
    ("mac_outside", 0.5, 0.01, 3.0 + 2.0 ** -20, 1.0, 0.0, 0.0, False,
     "d = 2.25 + 2^-20: accepted"),
    ("mac_delta", 0.5, 0.01, 2.875, 1.0, 0.0, 0.0, True,
     "d = 2.125 < 2.25 opened; without delta_c (r_open = 2) it would be accepted"),
    ("mac_group_box", 0.5, 0.01, 2.875, 1.0, 0.0, 1.0, True,
     "d = 2.125 from the group box; from the group centre (0.5, 0.5, 0) it is "
     "sqrt(2.625^2 + 0.25) > 2.25, and from g1 it is 3.125: both would accept"),
    # cell of extent (0.75, 1): l_c = 1, delta_c = |(0.75, 1)|/4 = 0.3125, r_open = 2.3125,
    # centre of mass (X + 0.1875, 0.25, 0); the group spans y in [0, 1], so d = X - 0.8125
    ("mac_longest_side", 0.5, 0.01, 3.0, 0.75, 1.0, 1.0, True,
     "d = 2.1875 < 2.3125 opened; l_c taken along x (0.75, r_open = 1.8125) would accept"),
    ("mac_longest_side_equal", 0.5, 0.01, 3.125, 0.75, 1.0, 1.0, False,
     "d = 2.3125 = r_open: accepted"),
    ("mac_not_diagonal", 0.5, 0.01, 3.1875, 0.75, 1.0, 1.0, False,
     "d = 2.375 > 2.3125 accepted; l_c as the box diagonal (1.25, r_open = 2.8125) "
     "would open it"),
    # theta = 0.25, cell along x of size 0.5: r_open = 0.5/0.25 + 0.125 = 2.125, d = X - 0.875
    ("mac_theta_quarter_inside", 0.25, 0.01, 3.0 - 2.0 ** -20, 0.5, 0.0, 0.0, True,
     "d = 2.125 - 2^-20 opened; l_c * theta (r_open = 0.25) would accept"),
    ("mac_theta_quarter_equal", 0.25, 0.01, 3.0, 0.5, 0.0, 0.0, False,
     "d = 2.125 = r_open: accepted"),
    # r_out box test on a cell the angle test accepts (X = 3, d = 2.25 = r_open); the
    # boxes are X - 1 = 2 apart along x
    ("rout_inside", 0.5, 2.0 + 2.0 ** -20, 3.0, 1.0, 0.0, 0.0, True,
     "box distance 2 < r_out: opened"),
    ("rout_equal", 0.5, 2.0, 3.0, 1.0, 0.0, 0.0, False,
     "box distance 2 = r_out: accepted by the strict '<'"),
    ("rout_outside", 0.5, 2.0 - 2.0 ** -20, 3.0, 1.0, 0.0, 0.0, False,
     "box distance 2 > r_out: accepted"),
    ("rout_box_not_com", 0.5, 2.125, 3.0, 1.0, 0.0, 0.0, True,
     "box distance 2 < 2.125 opened; the distance to the centre of mass (2.25) or "
     "from g1 (3) would accept"),
]


def particles(X, sx, sy, gy):
    """Positions and masses of one case, in input order: group, cell, ballast."""
    x = [0.0, 1.0, X, X + sx] + [4.0] * BALLAST
    y = [0.0, gy, 0.0, sy] + [4.0] * BALLAST
    z = [0.0, 0.0, 0.0, 0.0] + [4.0] * BALLAST
    m = [1.0, 1.0, 3.0, 1.0] + [0.0] * BALLAST
    return tuple(np.array(a, dtype=np.float64) for a in (x, y, z, m))


def expected_counts(opened):
    """(n_cell, n_part) of the group holding particle 0."""
    return (1, 4) if opened else (2, 2)
