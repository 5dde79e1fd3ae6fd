"""Seeded synthetic star clusters for the distant-force path of the P3T scheme.

This module only draws inputs: particle positions, velocities and masses of
Plummer spheres, King models and Kroupa mass spectra, plus the run parameters
of the paper (Sec. 3.1, Eqs. 20-25).  It holds none of the force, tree or
neighbour arithmetic, so both the CPU oracle tests and the CUDA path take their
inputs from here without sharing any method code.

Units are Henon N-body units (Sec. 3.1): G = M = 1, E = -1/4.

Workload recipes (the paper's runs are Plummer spheres, Sec. 3.1; King models
and Kroupa masses are the extended workloads of the ensemble benchmarks):

* ``plummer``: Aarseth-Henon-Wielen sampling of the Plummer model, radii
  truncated at 10 scale radii, centred on the centre of mass and of velocity,
  scale radius a = 3*pi/16 so that E = -1/4 for equal masses.
* ``kroupa_masses``: two-segment broken power law (slope 1.3 on 0.08-0.5,
  2.3 on 0.5-100 solar masses), normalised to total mass 1.
* ``king``: King (1966) lowered isothermal model of central depth W0, sampled
  from the solved Poisson equation and its distribution function, rescaled to
  Henon units through the model's own potential energy.
* ``segregate``: the heaviest 10 % of the stars by number have their
  positions scaled by 0.7 about the centre, then the cluster is re-centred.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BASE_SEED = 20211022


@dataclass
class Cluster:
    """Particle arrays (FP64, length n) of one synthetic cluster."""

    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    m: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def pos(self) -> np.ndarray:
        return np.stack([self.x, self.y, self.z], axis=1)

    def vel(self) -> np.ndarray:
        return np.stack([self.vx, self.vy, self.vz], axis=1)


def _isotropic(rng: np.random.Generator, r: np.ndarray):
    """Uniform random directions scaled by r (three arrays)."""
    u = 1.0 - 2.0 * rng.random(r.shape[0])
    phi = 2.0 * math.pi * rng.random(r.shape[0])
    s = np.sqrt(np.maximum(0.0, 1.0 - u * u))
    return r * s * np.cos(phi), r * s * np.sin(phi), r * u


def _centre(c: Cluster) -> Cluster:
    mt = c.m.sum()
    for a in ("x", "y", "z"):
        v = getattr(c, a)
        setattr(c, a, v - (c.m * v).sum() / mt)
    for a in ("vx", "vy", "vz"):
        v = getattr(c, a)
        setattr(c, a, v - (c.m * v).sum() / mt)
    return c


def kroupa_masses(n: int, rng: np.random.Generator, m_lo: float = 0.08,
                  m_br: float = 0.5, m_hi: float = 100.0,
                  a1: float = 1.3, a2: float = 2.3) -> np.ndarray:
    """Two-segment power-law IMF dN/dm ~ m^-a, continuous at m_br; total mass 1."""
    def seg_int(lo, hi, a):  # integral of m^-a
        return (hi ** (1 - a) - lo ** (1 - a)) / (1 - a)

    c2 = m_br ** (a2 - a1)  # continuity factor of the second segment
    w1 = seg_int(m_lo, m_br, a1)
    w2 = c2 * seg_int(m_br, m_hi, a2)
    u = rng.random(n)
    pick2 = rng.random(n) < w2 / (w1 + w2)

    def inv(lo, hi, a, uu):
        p = 1 - a
        return (lo ** p + uu * (hi ** p - lo ** p)) ** (1.0 / p)

    m = np.where(pick2, inv(m_br, m_hi, a2, u), inv(m_lo, m_br, a1, u))
    return m / m.sum()


def plummer(n: int, seed: int, masses: str = "equal") -> Cluster:
    """Plummer sphere in Henon units (Aarseth, Henon & Wielen 1974 sampling)."""
    rng = np.random.default_rng(seed)
    # radii from the inverted cumulative mass, truncated at 10 scale radii
    r = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        x1 = rng.random(todo.size)
        x1 = np.maximum(x1, 1e-300)
        rr = 1.0 / np.sqrt(x1 ** (-2.0 / 3.0) - 1.0)
        ok = rr <= 10.0
        r[todo[ok]] = rr[ok]
        todo = todo[~ok]
    x, y, z = _isotropic(rng, r)
    # speeds: q = v/v_esc from g(q) = q^2 (1-q^2)^(7/2) by rejection
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        x4 = rng.random(todo.size)
        x5 = rng.random(todo.size)
        ok = 0.1 * x5 < x4 * x4 * (1.0 - x4 * x4) ** 3.5
        q[todo[ok]] = x4[ok]
        todo = todo[~ok]
    vesc = np.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
    vx, vy, vz = _isotropic(rng, q * vesc)
    if masses == "equal":
        m = np.full(n, 1.0 / n)
    elif masses == "kroupa":
        m = kroupa_masses(n, rng)
    else:
        raise ValueError(masses)
    a = 3.0 * math.pi / 16.0  # Henon units: E = -1/4 for equal masses
    sv = 1.0 / math.sqrt(a)
    c = Cluster(x * a, y * a, z * a, m, vx * sv, vy * sv, vz * sv)
    return _centre(c)


def _king_rho(w):
    """Density of the lowered isothermal model, up to the constant rho_1."""
    w = np.maximum(w, 0.0)
    from scipy.special import erf
    sw = np.sqrt(w)
    return np.exp(w) * erf(sw) - np.sqrt(4.0 * w / math.pi) * (1.0 + 2.0 * w / 3.0)


def _king_profile(w0: float):
    """Solve W'' + 2 W'/r = -9 rho(W)/rho(W0) from r=0 to the tidal radius."""
    from scipy.integrate import solve_ivp
    rho0 = float(_king_rho(np.array(w0)))

    def rhs(r, s):
        w, dw = s
        return [dw, -9.0 * float(_king_rho(np.array(w))) / rho0 - 2.0 * dw / r]

    def hit(r, s):
        return s[0]
    hit.terminal = True
    hit.direction = -1
    r0 = 1e-6
    s0 = [w0 - 1.5 * r0 * r0, -3.0 * r0]  # series W = W0 - (3/2) r^2 near 0
    sol = solve_ivp(rhs, (r0, 1e4), s0, events=hit, rtol=1e-11, atol=1e-13,
                    dense_output=True, max_step=0.05)
    rt = float(sol.t_events[0][0])
    rg = np.concatenate([[0.0], np.geomspace(r0, rt, 20000)])
    ws = sol.sol(np.maximum(rg, r0))
    w = np.where(rg > 0, ws[0], w0)
    dw = np.where(rg > 0, ws[1], 0.0)
    w[-1] = 0.0
    # G = sigma = r_core = 1 units: M(r) = -r^2 W'(r), rho = (9/4pi) rho~/rho~0
    mr = -rg * rg * dw
    mr[0] = 0.0
    mr = np.maximum.accumulate(mr)
    return rg, np.maximum(w, 0.0), mr, rt


def king(n: int, seed: int, w0: float, masses: str = "equal") -> Cluster:
    """King model of central depth w0 in Henon units."""
    rng = np.random.default_rng(seed)
    rg, wg, mr, rt = _king_profile(w0)
    mt = mr[-1]
    # potential energy U = -int G M(r) dM / r (model units)
    dm = np.diff(mr)
    rmid = 0.5 * (rg[1:] + rg[:-1])
    mmid = 0.5 * (mr[1:] + mr[:-1])
    u_model = -np.sum(mmid * dm / np.maximum(rmid, 1e-30))
    # positions from the cumulative mass
    r = np.interp(rng.random(n) * mt, mr, rg)
    x, y, z = _isotropic(rng, r)
    w = np.interp(r, rg, wg)
    # speeds from f ~ exp(W - v^2/2) - 1, v < sqrt(2W), by rejection
    v = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        wt = w[todo]
        ve = np.sqrt(2.0 * wt)
        vv = ve * rng.random(todo.size)
        bound = ve * ve * np.expm1(wt)
        p = vv * vv * np.expm1(wt - 0.5 * vv * vv)
        ok = rng.random(todo.size) * bound <= p
        ok &= bound > 0
        v[todo[ok]] = vv[ok]
        bad = bound <= 0  # at the tidal radius: zero speed
        v[todo[bad]] = 0.0
        todo = todo[~(ok | bad)]
    vx, vy, vz = _isotropic(rng, v)
    # normalise total mass to 1 (G = 1): v^2 ~ M / r
    vs = 1.0 / math.sqrt(mt)
    u1 = u_model / (mt * mt)
    lam = u1 / -0.5  # length scale giving U = -1/2, E = -1/4
    sv = vs / math.sqrt(lam)
    if masses == "equal":
        m = np.full(n, 1.0 / n)
    elif masses == "kroupa":
        m = kroupa_masses(n, rng)
    else:
        raise ValueError(masses)
    c = Cluster(x * lam, y * lam, z * lam, m, vx * sv, vy * sv, vz * sv)
    return _centre(c)


def segregate(c: Cluster, frac: float = 0.1, scale: float = 0.7) -> Cluster:
    """Scale the positions of the heaviest `frac` of stars (ties by index) by `scale`."""
    k = int(round(frac * c.n))
    order = np.lexsort((np.arange(c.n), -c.m))  # by mass descending, then index
    heavy = order[:k]
    for a in ("x", "y", "z"):
        v = getattr(c, a).copy()
        v[heavy] *= scale
        setattr(c, a, v)
    return _centre(c)


def paper_run_params(n: int) -> dict:
    """Run parameters of Sec. 3.1 (Eqs. 20-25): tau, r_cut, r_buff, dt_reg, dt_max."""
    sigma = 1.0 / math.sqrt(2.0)
    tau = (1.0 / 128.0) * (n / 2.0 ** 14) ** (-1.0 / 3.0)
    dt_reg = 1.0
    while dt_reg > tau:
        dt_reg *= 0.5
    return {"tau": tau, "r_cut": 4.0 * tau, "r_buff": 3.0 * tau * sigma,
            "dt_reg": dt_reg, "dt_max": dt_reg / 4.0, "sigma": sigma}


def plummer_r_for_mean_neighbours(n: int, k: float) -> float:
    """Radius giving k mean neighbours in a Henon-unit Plummer sphere.

    <n_nb> = N (4 pi/3) r^3 int rho^2 dV / M^2 = 0.9006 N r^3 for small r.
    """
    a = 3.0 * math.pi / 16.0
    i_rho2 = 9.0 * 4.0 * (15.0 * math.pi / 768.0) / (16.0 * math.pi * a ** 3)
    coef = 4.0 * math.pi / 3.0 * i_rho2
    return (k / (coef * n)) ** (1.0 / 3.0)


def make(kind: str, n: int, seed: int, masses: str = "equal", w0: float = 7.0,
         segregated: bool = False) -> Cluster:
    """One cluster by recipe name: 'plummer' or 'king'."""
    if kind == "plummer":
        c = plummer(n, seed, masses)
    elif kind == "king":
        c = king(n, seed, w0, masses)
    else:
        raise ValueError(kind)
    if segregated:
        c = segregate(c)
    return c


def log_uniform_sizes(count: int, n_lo: float, n_hi: float, seed: int) -> np.ndarray:
    """`count` cluster sizes drawn log-uniformly in [n_lo, n_hi] (rounded)."""
    rng = np.random.default_rng(seed)
    s = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), count))
    return np.clip(np.rint(s), n_lo, n_hi).astype(np.int64)


def ensemble(count: int, n_lo: float, n_hi: float, seed: int, masses: str = "equal",
             w0: float = 5.0) -> list:
    """Independent clusters of log-uniform size, alternately Plummer and King(w0),
    each in its own Henon units (total mass 1) and seeded by seed + 1 + index."""
    sizes = log_uniform_sizes(count, n_lo, n_hi, seed)
    return [make("plummer" if k % 2 == 0 else "king", int(n), seed + 1 + k, masses=masses, w0=w0)
            for k, n in enumerate(sizes)]


def concat(clusters: list):
    """One particle set of several clusters, and its segment offsets (int64, count + 1)."""
    cat = lambda a: np.concatenate([getattr(c, a) for c in clusters])  # noqa: E731
    seg = np.zeros(len(clusters) + 1, np.int64)
    np.cumsum([c.n for c in clusters], out=seg[1:])
    return Cluster(*(cat(a) for a in ("x", "y", "z", "m", "vx", "vy", "vz"))), seg
