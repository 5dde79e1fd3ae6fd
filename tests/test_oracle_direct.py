"""Pins of the oracle's changeover function, direct split sum, kick and neighbours.

Each test checks the oracle against something other than itself: closed forms,
a library routine (the Beta(4,4) distribution), conservation laws, the
two-body problem, and brute force.
"""
import math

import numpy as np
import pytest
from scipy.special import betainc

import oracle
import synth

R_IN, R_OUT = 0.005, 0.05


# --- Eq. 6: W = 1 - K ------------------------------------------------------

def test_W_end_values():
    # Sec. 2.1: below r_in the pair is wholly near, above r_cut wholly far
    assert oracle.changeover_W(0.0, R_IN, R_OUT) == 0.0
    assert oracle.changeover_W(R_IN * 0.999, R_IN, R_OUT) == 0.0
    assert oracle.changeover_W(R_IN, R_IN, R_OUT) == 0.0
    assert oracle.changeover_W(R_OUT, R_IN, R_OUT) == 1.0
    assert oracle.changeover_W(10 * R_OUT, R_IN, R_OUT) == 1.0
    assert oracle.changeover_K(0.001, R_IN, R_OUT) == 1.0
    assert oracle.changeover_K(1.0, R_IN, R_OUT) == 0.0


def test_W_is_beta44_cdf():
    # -20x^7+70x^6-84x^5+35x^4 is the regularised incomplete beta I_x(4,4)
    for x in np.linspace(0.0, 1.0, 257):
        r = R_IN + x * (R_OUT - R_IN)
        assert abs(oracle.changeover_W(r, R_IN, R_OUT) - betainc(4, 4, x)) < 1e-13  # cancellation near x = 1


def test_W_symmetry_and_derivative():
    # W(x) + W(1-x) = 1 and dW/dx = 140 x^3 (1-x)^3 (the bracket of Eq. 7)
    d = R_OUT - R_IN
    for x in np.linspace(0.01, 0.99, 97):
        w = oracle.changeover_W(R_IN + x * d, R_IN, R_OUT)
        w1 = oracle.changeover_W(R_IN + (1 - x) * d, R_IN, R_OUT)
        assert abs(w + w1 - 1.0) < 1e-13
        h = 1e-6
        num = (oracle.changeover_W(R_IN + (x + h) * d, R_IN, R_OUT)
               - oracle.changeover_W(R_IN + (x - h) * d, R_IN, R_OUT)) / (2 * h)
        assert abs(num - 140 * x ** 3 * (1 - x) ** 3) < 1e-7
    assert abs(oracle.changeover_W(R_IN + 0.5 * d, R_IN, R_OUT) - 0.5) < 1e-15
    ws = [oracle.changeover_W(r, R_IN, R_OUT) for r in np.linspace(0, 0.06, 600)]
    assert all(b >= a for a, b in zip(ws, ws[1:]))


# --- Eqs. 1, 3: direct split sum ---------------------------------------------

def test_two_body_closed_form():
    # two particles: a_far on particle 0 = W(r) m_1 / r^2 towards particle 1
    for r in [0.001, 0.0075, 0.02, 0.0275, 0.049, 0.05, 0.3]:
        x = np.array([0.1, 0.1 + r])
        y = np.array([-0.2, -0.2])
        z = np.array([0.3, 0.3])
        m = np.array([0.25, 0.75])
        d = oracle.direct_split(x, y, z, m, R_IN, R_OUT)
        w = betainc(4, 4, min(1.0, max(0.0, (r - R_IN) / (R_OUT - R_IN))))
        assert d["far"][0, 0] == pytest.approx(w * 0.75 / r ** 2, rel=1e-12, abs=1e-300)
        assert d["far"][1, 0] == pytest.approx(-w * 0.25 / r ** 2, rel=1e-12, abs=1e-300)
        assert d["full"][0, 0] == pytest.approx(0.75 / r ** 2, rel=1e-12)
        assert d["far"][0, 1] == 0.0 and d["far"][0, 2] == 0.0
        assert d["pot"][0] == pytest.approx(-0.75 / r, rel=1e-14)


def test_split_identity_and_momentum(plummer_4096):
    c = plummer_4096
    d = oracle.direct_split(c.x, c.y, c.z, c.m, R_IN, R_OUT)
    full = d["full"]
    scale = np.abs(full).max()
    # near + far = full Newtonian (Eq. 3), per particle, to round-off
    assert np.abs(d["near"] + d["far"] - full).max() < 1e-12 * scale
    # Newton's third law: sum m a = 0 for full and for far (W symmetric in i, j)
    for key in ("full", "far", "near"):
        p = (c.m[:, None] * d[key]).sum(axis=0)
        assert np.abs(p).max() < 1e-11 * (c.m[:, None] * np.abs(d[key])).sum()
    # the near part only sees pairs closer than r_out: far == full for isolated particles
    offs, idx = oracle.neighbours_brute(c.x, c.y, c.z, R_OUT)
    iso = np.diff(offs) == 0
    assert iso.sum() > 1000
    assert np.abs(d["far"][iso] - full[iso]).max() < 1e-12 * scale


def test_far_equals_full_when_cutoff_vanishes(plummer_4096):
    c = plummer_4096
    t = np.arange(0, 4096, 37)
    d = oracle.direct_split(c.x, c.y, c.z, c.m, 1e-12, 2e-12, targets=t)
    assert np.abs(d["far"] - d["full"]).max() == 0.0
    assert np.abs(d["near"]).max() == 0.0


def test_plummer_potential_energy(plummer_4096):
    # Plummer in Henon units: U = -3 pi G M^2 / (32 a) = -1/2 with a = 3 pi/16
    c = plummer_4096
    d = oracle.direct_split(c.x, c.y, c.z, c.m, R_IN, R_OUT)
    u = 0.5 * (c.m * d["pot"]).sum()
    a = 3 * math.pi / 16
    assert u == pytest.approx(-3 * math.pi / (32 * a), rel=4.0 / math.sqrt(c.n))
    t = 0.5 * (c.m * (c.vx ** 2 + c.vy ** 2 + c.vz ** 2)).sum()
    assert 2 * t / abs(u) == pytest.approx(1.0, rel=5.0 / math.sqrt(c.n))


def test_attraction_sign():
    # a test particle on the +x axis of a point mass is pulled towards -x
    d = oracle.direct_split([0.0, 1.0], [0.0, 0.0], [0.0, 0.0], [1.0, 1e-9], R_IN, R_OUT)
    assert d["far"][1, 0] < 0 and d["far"][1, 0] == pytest.approx(-1.0, rel=1e-14)


# --- Eq. 12: kick --------------------------------------------------------------

def test_kick_closed_form():
    rng = np.random.default_rng(3)
    v = rng.normal(size=(3, 100))
    a = rng.normal(size=(3, 100))
    dt = 1.0 / 256
    vx, vy, vz = oracle.kick(dt, *a, *v)
    for got, v0, a0 in zip((vx, vy, vz), v, a):
        assert np.array_equal(got, v0 + (0.5 * dt) * a0)


# --- Sec. 2.3: neighbour lists ------------------------------------------------

def test_neighbours_brute_tiny_by_hand():
    # points on a line, spacing 1: with r_list = 1.5 each sees its direct neighbours
    x = np.array([3.0, 0.0, 1.0, 2.0, 10.0])
    zeros = np.zeros(5)
    offs, idx = oracle.neighbours_brute(x, zeros, zeros, 1.5)
    rows = [list(idx[offs[i]:offs[i + 1]]) for i in range(5)]
    assert rows == [[3], [2], [1, 3], [0, 2], []]
    # the test is strict: a pair exactly at r_list is not a neighbour
    offs, idx = oracle.neighbours_brute(x, zeros, zeros, 1.0)
    assert offs[-1] == 0


def test_paper_radius_gives_under_one_neighbour():
    # Sec. 2.3 and the neighbour-number figure: with r_cut = 4 tau (Eq. 21) the
    # mean neighbour number stays below one, ~0.45 for a Plummer sphere
    for n in (2048, 4096, 8192):
        c = synth.plummer(n, synth.BASE_SEED + n)
        rc = synth.paper_run_params(n)["r_cut"]
        offs, _ = oracle.neighbours_brute(c.x, c.y, c.z, rc)
        mean = offs[-1] / n
        assert mean < 1.0
        assert mean == pytest.approx(0.9006 * n * rc ** 3, rel=0.25)
