"""Pins of the oracle's bead-spring chains (harmonic bonds (k/2)(b - sigma)^2
with Boltzmann energies drawn at every event, Sec. II): the own logarithm
behind the energies against libm, and the bond-length distribution of a
free dimer, p(b) ~ b^2 exp(-k (b - sigma)^2 / 2) for b >= sigma (hard
spheres), in the serial and the domain form (the latter through
reflections at immotile partners).  The paper quotes <b> ~ 1.1 sigma for
k sigma^2 / kT = 30 in its melts; for a free dimer the exact mean is
1.1676 sigma.  No GPU."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle


def test_own_log_within_two_ulp():
    rng = np.random.default_rng(1)
    us = np.concatenate([rng.uniform(0, 1, 20000), 1 - rng.uniform(0, 1e-6, 2000),
                         np.exp(-rng.uniform(0, 700, 2000)), [1.0, 0.5, 2.0 ** -53]])
    us = us[us > 0]
    for u in us:
        a, b = oracle.own_log(u), math.log(u)
        assert abs(a - b) <= 2 * np.spacing(abs(b)) or a == b, (u, a, b)


def exact_bond_moments(k, sigma=1.0):
    w = lambda b: b * b * math.exp(-0.5 * k * (b - sigma) ** 2)
    z = integrate.quad(w, sigma, sigma + 12 / math.sqrt(k))[0]
    m1 = integrate.quad(lambda b: b * w(b), sigma, sigma + 12 / math.sqrt(k))[0] / z
    cdf = lambda x: integrate.quad(w, sigma, x)[0] / z
    return m1, cdf


def sample_dimer(mode, k, n_samples, ell=1.0, seed=3):
    L = 12.0
    r = np.array([[6.0, 6.0, 6.0], [7.1, 6.0, 6.0]])
    kw = dict(sigma=1.0, b_max=1.2, dir_mode=oracle.DIR_ISO, seed=seed, k_spring=k)
    if mode == "domain":
        s = oracle.System(r, (L, L, L), 2, mode=oracle.MODE_DOMAIN, D=(3, 3, 3), **kw)
    else:
        s = oracle.System(r, (L, L, L), 2, mode=oracle.MODE_SERIAL, **kw)
    b = np.empty(n_samples)
    for t in range(n_samples):
        if mode == "domain":
            res = s.run_domain(1, ell, sweep0=t)
        else:
            res = s.run_serial(4, ell, ec0=4 * t)
        assert res["rc"] == 0
        d = s.r[0] - s.r[1]
        d -= L * np.round(d / L)
        b[t] = math.sqrt(d @ d)
    return b


@pytest.mark.parametrize("mode", ["serial", "domain"])
def test_spring_dimer_bond_distribution(mode):
    k = 30.0
    b = sample_dimer(mode, k, 6000)[500:]
    m1, cdf = exact_bond_moments(k)
    assert m1 == pytest.approx(1.1676, abs=2e-4)
    assert b.min() >= 1.0 - 1e-12
    # batch means for the error of correlated samples
    bm = b[: len(b) // 50 * 50].reshape(50, -1).mean(axis=1)
    se = bm.std(ddof=1) / math.sqrt(len(bm))
    assert abs(b.mean() - m1) < 4 * se + 1e-3
    for x in (1.05, 1.15, 1.3):
        assert (b < x).mean() == pytest.approx(cdf(x), abs=0.04)


def test_springs_reject_swaps():
    r = np.array([[6.0, 6.0, 6.0], [7.1, 6.0, 6.0]])
    s = oracle.System(r, (12.0, 12.0, 12.0), 2, dir_mode=oracle.DIR_ISO, k_spring=30.0, p_swap=0.5)
    assert s.run_serial(1, 1.0)["rc"] == -1


def test_spring_event_against_its_definition():
    """The event distance x of a spring event solves
    integral_0^x max(0, dU/ds) ds = dE with U(s) = (k/2)(|d + s v| - sigma)^2:
    the energy the pivot's move adds (a falling stretch of the path is
    always admissible, Sec. II), found here by quadrature and root finding."""
    from scipy.optimize import brentq

    rng = np.random.default_rng(9)
    k, sigma = 30.0, 1.0
    for _ in range(300):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        d = u * rng.uniform(1.0, 1.6)
        dE = rng.exponential()
        bmin2 = d @ d - (d @ v) ** 2
        if d @ v < 0 and bmin2 < sigma * sigma:
            continue  # the beads touch first; the spring event is moot
        U = lambda s: 0.5 * k * (np.linalg.norm(d + s * v) - sigma) ** 2
        dU = lambda s: k * (np.linalg.norm(d + s * v) - sigma) * ((d + s * v) @ v) / np.linalg.norm(d + s * v)
        x0 = max(0.0, -(d @ v))  # closest approach: U falls before, rises after
        def rise(x):
            if x <= x0:
                return 0.0 - dE
            return (U(x) - U(x0)) - dE if d @ v < 0 else (U(x) - U(0.0)) - dE
        # the positive-part integral by quadrature agrees with the rise
        xt = x0 + 0.3
        assert integrate.quad(lambda s: max(0.0, dU(s)), 0.0, xt, points=[x0])[0] == pytest.approx(
            rise(xt) + dE, rel=1e-7, abs=1e-10)
        ref = brentq(rise, x0, x0 + 20.0, xtol=1e-14)
        assert oracle.spring_x(d, v, sigma, k, dE) == pytest.approx(ref, rel=1e-9, abs=1e-12)


def test_spring_motility_rule_on_domain_tags():
    """With springs, no bond joins motile beads of two different tiles
    (reading R23), and exactly the beads with such a bond lose their tile."""
    L, N = 16.0, 12
    r, img = oracle.phantom_chains((L, L, L), 60, N, bond=1.6, c=1.0, seed=5)  # long bonds cross joints
    kw = dict(sigma=1.0, b_max=1.2, mode=oracle.MODE_DOMAIN, D=(4, 4, 4), seed=11, img=img)
    springs = oracle.System(r, (L, L, L), N, k_spring=30.0, **kw)
    tethers = oracle.System(r, (L, L, L), N, **kw)
    crossing_seen = 0
    for sweep in range(20):
        ts, _ = springs.domain_tags(sweep)
        tt, _ = tethers.domain_tags(sweep)
        a, b = np.arange(len(r) - 1), np.arange(1, len(r))
        bond = (a // N) == (b // N)
        a, b = a[bond], b[bond]
        assert not np.any((ts[a] >= 0) & (ts[b] >= 0) & (ts[a] != ts[b]))
        cross = (tt[a] >= 0) & (tt[b] >= 0) & (tt[a] != tt[b])
        crossing_seen += int(cross.sum())
        dropped = np.zeros(len(r), dtype=bool)
        dropped[a[cross]] = True
        dropped[b[cross]] = True
        assert ((tt >= 0) & (ts < 0) == dropped).all()
        assert (ts[ts >= 0] == tt[ts >= 0]).all()
    assert crossing_seen > 0
