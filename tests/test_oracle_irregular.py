"""Pins of the oracle's irregular force and jerk (Eqs. 1, 2, 6, 7)."""
import numpy as np
import pytest

import oracle
import synth

R_IN, R_OUT = 0.005, 0.05


def test_dWdx_is_the_derivative_of_W():
    for x in np.linspace(0.0, 0.999, 37):
        r = R_IN + x * (R_OUT - R_IN)
        assert oracle.changeover_dWdx(r, R_IN, R_OUT) == pytest.approx(140 * x ** 3 * (1 - x) ** 3, abs=1e-12)
        h = 1e-6
        if 1e-5 < x < 0.999:
            dr = h * (R_OUT - R_IN)
            fd = (oracle.changeover_W(r + dr, R_IN, R_OUT) - oracle.changeover_W(r - dr, R_IN, R_OUT)) / (2 * h)
            # W near x = 1 is a sum of terms up to 84 with value ~1: ~1e-14 absolute rounding,
            # which the difference quotient amplifies to ~1e-8
            assert oracle.changeover_dWdx(r, R_IN, R_OUT) == pytest.approx(fd, rel=1e-6, abs=1e-7)
    assert oracle.changeover_dWdx(0.5 * R_IN, R_IN, R_OUT) == 0.0
    assert oracle.changeover_dWdx(1.5 * R_OUT, R_IN, R_OUT) == 0.0


def _rows(c, r_list):
    offs, idx = oracle.neighbours_brute(c.x, c.y, c.z, r_list)
    return offs, idx


def test_two_body_force_and_jerk_closed_form():
    r = 0.02
    x = np.array([0.0, r]); y = np.zeros(2); z = np.zeros(2)
    m = np.array([0.3, 0.7])
    vx = np.array([0.0, 0.4]); vy = np.array([0.0, 0.1]); vz = np.zeros(2)
    offs = np.array([0, 1, 2]); idx = np.array([1, 0], np.int32)
    f, j = oracle.irregular(x, y, z, m, vx, vy, vz, R_IN, R_OUT, offs, idx)
    xx = (r - R_IN) / (R_OUT - R_IN)
    K = 1 - (-20 * xx ** 7 + 70 * xx ** 6 - 84 * xx ** 5 + 35 * xx ** 4)
    assert f[0] == pytest.approx([K * 0.7 / r ** 2, 0, 0], rel=1e-13)
    assert f[1] == pytest.approx([-K * 0.3 / r ** 2, 0, 0], rel=1e-13)
    # jerk of particle 0 by hand: d = (r,0,0), u = (0.4,0.1,0)
    du = r * 0.4
    Kdot = -140 * xx ** 3 * (1 - xx) ** 3 * du / (r * (R_OUT - R_IN))
    jx = 0.7 * (K * 0.4 / r ** 3 - 3 * K * du * r / r ** 5 + Kdot * r / r ** 3)
    jy = 0.7 * K * 0.1 / r ** 3
    assert j[0] == pytest.approx([jx, jy, 0], rel=1e-12)


def test_jerk_equals_finite_difference_of_force():
    # straight-line motion x(t) = x + v t: dF/dt by central differences must match
    # the analytic jerk (this fixes the sign of K' and every term of Eq. 2)
    c = synth.plummer(64, 21)
    s = 0.12  # squeeze so that many pairs sit inside [r_in, r_out)
    x, y, z = c.x * s, c.y * s, c.z * s
    vx, vy, vz = c.vx, c.vy, c.vz
    offs, idx = oracle.neighbours_brute(x, y, z, 2.0 * R_OUT)
    f0, j0, sf, sj = oracle.irregular(x, y, z, c.m, vx, vy, vz, R_IN, R_OUT, offs, idx, scales=True)
    h = 1e-7
    fp, _ = oracle.irregular(x + h * vx, y + h * vy, z + h * vz, c.m, vx, vy, vz, R_IN, R_OUT, offs, idx)
    fm, _ = oracle.irregular(x - h * vx, y - h * vy, z - h * vz, c.m, vx, vy, vz, R_IN, R_OUT, offs, idx)
    fd = (fp - fm) / (2 * h)
    err = np.abs(fd - j0).max(axis=1)
    assert (sj > 0).sum() > 20
    assert np.all(err <= 1e-5 * sj + 1e-9), err.max()
    # a jerk with the printed sign of K' would fail by far
    k_part = np.zeros_like(j0)
    for i in range(c.n):
        for e in range(offs[i], offs[i + 1]):
            jj = idx[e]
            d = np.array([x[jj] - x[i], y[jj] - y[i], z[jj] - z[i]])
            u = np.array([vx[jj] - vx[i], vy[jj] - vy[i], vz[jj] - vz[i]])
            rr = np.linalg.norm(d)
            kd = -oracle.changeover_dWdx(rr, R_IN, R_OUT) * d.dot(u) / (rr * (R_OUT - R_IN))
            k_part[i] += c.m[jj] * kd * d / rr ** 3
    flipped = j0 - 2 * k_part
    assert np.abs(fd - flipped).max() > 1e3 * np.abs(fd - j0).max()


def test_irregular_force_is_the_near_part_of_the_direct_sum():
    c = synth.plummer(400, 22)
    s = 0.3
    x, y, z = c.x * s, c.y * s, c.z * s
    offs, idx = _rows(synth.Cluster(x, y, z, c.m, c.vx, c.vy, c.vz), R_OUT)
    f, _, sf, _ = oracle.irregular(x, y, z, c.m, c.vx, c.vy, c.vz, R_IN, R_OUT, offs, idx, scales=True)
    near = oracle.direct_split(x, y, z, c.m, R_IN, R_OUT)["near"]
    assert np.all(np.abs(f - near).max(axis=1) <= 1e-13 * sf + 1e-300)
    assert (np.abs(f).max(axis=1) > 0).sum() > 100


def test_momentum_of_irregular_force_and_jerk():
    c = synth.plummer(500, 23)
    s = 0.25
    x, y, z = c.x * s, c.y * s, c.z * s
    offs, idx = oracle.neighbours_brute(x, y, z, R_OUT)  # symmetric rows
    f, j, sf, sj = oracle.irregular(x, y, z, c.m, c.vx, c.vy, c.vz, R_IN, R_OUT, offs, idx, scales=True)
    p = (c.m[:, None] * f).sum(axis=0)
    pdot = (c.m[:, None] * j).sum(axis=0)
    assert np.abs(p).max() <= 1e-13 * (c.m * sf).sum()
    assert np.abs(pdot).max() <= 1e-13 * (c.m * sj).sum()


def test_pairs_beyond_r_out_and_coincident_pairs_add_nothing():
    c = synth.plummer(300, 24)
    s = 0.3
    x, y, z = c.x * s, c.y * s, c.z * s
    x[1], y[1], z[1] = x[0], y[0], z[0]  # a coincident pair (singular, skipped)
    o1, i1 = oracle.neighbours_brute(x, y, z, R_OUT)
    o3, i3 = oracle.neighbours_brute(x, y, z, 3 * R_OUT)
    args = (x, y, z, c.m, c.vx, c.vy, c.vz, R_IN, R_OUT)
    f1, j1 = oracle.irregular(*args, o1, i1)
    f3, j3 = oracle.irregular(*args, o3, i3)
    assert np.array_equal(f1, f3) and np.array_equal(j1, j3)
    assert np.all(np.isfinite(f1)) and np.all(np.isfinite(j1))
    assert (np.diff(o3) > np.diff(o1)).any()
