"""Regression fixture of the oracle and sanity pins of the input generators."""
import hashlib
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "plummer4096_oracle.json")


def test_oracle_matches_committed_fixture():
    g = json.load(open(GOLD))
    c = synth.plummer(4096, synth.BASE_SEED)
    t = oracle.Tree(c.x, c.y, c.z, c.m, theta=0.5, r_out=0.05, leaf_cap=16, group_size=64)
    d = t.export()
    assert hashlib.sha256(d["keys"].tobytes()).hexdigest() == g["keys_sha256"]
    assert hashlib.sha256(d["perm"].tobytes()).hexdigest() == g["perm_sha256"]
    assert (t.n_nodes, t.n_groups, int(d["level"].max())) == (g["n_nodes"], g["n_groups"], g["depth"])
    f = t.far(0.005)
    assert int(f["n_cell"].sum()) == g["n_cell_total"]
    assert int(f["n_part"].sum()) == g["n_part_total"]
    assert np.allclose(f["a"][:8], g["a_far_first8"], rtol=1e-14, atol=0)
    assert np.allclose(f["pot"][:8], g["pot_first8"], rtol=1e-14, atol=0)
    _, offs, idx = t.neighbours(0.05)
    assert int(offs[-1]) == g["nbr_total"]
    assert hashlib.sha256(idx.tobytes()).hexdigest() == g["nbr_sha256"]


def test_generators_are_seeded():
    a = synth.plummer(1000, 5)
    b = synth.plummer(1000, 5)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.vz, b.vz)
    assert not np.array_equal(a.x, synth.plummer(1000, 6).x)


def test_kroupa_segment_fractions():
    # number fraction below the break vs the analytic integral of the two-part IMF
    rng = np.random.default_rng(1)
    m = synth.kroupa_masses(200000, rng)
    mm = m * (1 / m.min()) * 0.08  # undo the normalisation, approximately
    w1 = (0.5 ** -0.3 - 0.08 ** -0.3) / -0.3
    w2 = 0.5 ** 1.0 * (100 ** -1.3 - 0.5 ** -1.3) / -1.3
    frac = w1 / (w1 + w2)
    assert (mm < 0.5).mean() == pytest.approx(frac, abs=0.01)
    assert m.sum() == pytest.approx(1.0, rel=1e-12)


def test_king_w0_7_concentration_and_virial():
    # King W0 = 7: concentration log10(r_t / r_c) ~ 1.53 (textbook value)
    rg, w, mr, rt = synth._king_profile(7.0)
    assert math.log10(rt) == pytest.approx(1.53, abs=0.02)
    c = synth.king(40000, 3, 7.0)
    t = 0.5 * (c.m * (c.vx ** 2 + c.vy ** 2 + c.vz ** 2)).sum()
    assert t == pytest.approx(0.25, rel=0.05)  # virial equilibrium at E = -1/4


def test_paper_run_parameters():
    # Eqs. 20-25 at N = 2^14: tau = 1/128, r_cut = 1/32, dt_reg = 1/128
    p = synth.paper_run_params(2 ** 14)
    assert p["tau"] == pytest.approx(1 / 128)
    assert p["r_cut"] == pytest.approx(1 / 32)
    assert p["dt_reg"] == 1 / 128 and p["dt_max"] == 1 / 512
    assert p["r_buff"] == pytest.approx(3 / 128 / math.sqrt(2))
    assert synth.paper_run_params(10 ** 6)["dt_reg"] == 1 / 512
