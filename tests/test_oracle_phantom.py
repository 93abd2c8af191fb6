"""Pins of the oracle's phantom-chain generator (non-reversal random walks
without excluded volume, the first stage of the paper's initial
configurations, Sec. II.B) against exact properties of the walk: bond
length, the cap bound, <cos theta> = (c - 1)/(c + 1) = cos^2(theta_max/2),
tangent correlations C^k (each tangent is uniform on a cap around the one
before, so <t_{j+k} . t_j> = C^k), the freely-rotating-chain <R^2>, a
uniform first bead and an isotropic first bond.  No GPU."""
import math

import numpy as np
import pytest

import oracle


def unwrap(r, img, L, nch, N):
    return (r + img * np.asarray(L)).reshape(nch, N, 3)


def frc_r2(n, C):
    """<R^2> / b^2 of a chain of n bonds with <t_i . t_{i+k}> = C^k."""
    return n * (1 + C) / (1 - C) - 2 * C * (1 - C ** n) / (1 - C) ** 2 if C != 1 else n * n


@pytest.mark.parametrize("c", [1.0, 1.9, 5.0])
def test_phantom_bonds_cap_and_mean_cosine(c):
    L = (30.0, 35.0, 40.0)
    nch, N, bond = 1500, 40, 1.05
    r, img = oracle.phantom_chains(L, nch, N, bond=bond, c=c, seed=11)
    assert (r >= 0).all() and (r < np.asarray(L)).all()
    u = unwrap(r, img, L, nch, N)
    b = np.diff(u, axis=1)
    assert np.allclose(np.linalg.norm(b, axis=2), bond, rtol=1e-12)
    t = b / bond
    cos = np.sum(t[:, 1:] * t[:, :-1], axis=2)
    ct = (c - 3) / (c + 1)
    assert cos.min() >= ct - 1e-12
    C = (c - 1) / (c + 1)
    se = cos.std() / math.sqrt(cos.size)
    assert abs(cos.mean() - C) < 4 * se + 1e-12
    # the paper's form of the same mean: cos^2(theta_max / 2)
    assert C == pytest.approx(math.cos(math.acos(ct) / 2) ** 2, rel=1e-12)


def test_phantom_tangent_correlations_and_r2():
    L = (50.0, 50.0, 50.0)
    nch, N, c = 4000, 60, 1.9
    r, img = oracle.phantom_chains(L, nch, N, bond=1.0, c=c, seed=12)
    u = unwrap(r, img, L, nch, N)
    t = np.diff(u, axis=1)
    C = (c - 1) / (c + 1)
    for k in (1, 2, 3, 5):
        ck = np.sum(t[:, k:] * t[:, :-k], axis=2)
        se = ck.std() / math.sqrt(ck.size / 4)  # correlated along a chain
        assert abs(ck.mean() - C ** k) < 4 * se
    R2 = np.sum((u[:, -1] - u[:, 0]) ** 2, axis=1)
    ref = frc_r2(N - 1, C)
    assert abs(R2.mean() - ref) < 4 * R2.std() / math.sqrt(nch)
    # long-chain limit: <R^2> / n -> c (the paper's 1.9)
    assert frc_r2(10 ** 6, C) / 10 ** 6 == pytest.approx(c, rel=1e-5)


def test_phantom_first_bead_and_bond():
    L = (20.0, 20.0, 20.0)
    nch, N = 20000, 2
    r, img = oracle.phantom_chains(L, nch, N, bond=1.0, c=1.9, seed=13)
    first = r.reshape(nch, N, 3)[:, 0]
    octant = (first[:, 0] > 10) * 1 + (first[:, 1] > 10) * 2 + (first[:, 2] > 10) * 4
    counts = np.bincount(octant, minlength=8)
    chi2 = np.sum((counts - nch / 8) ** 2 / (nch / 8))
    assert chi2 < 24.3  # 7 degrees of freedom, p = 0.001
    t = np.diff(unwrap(r, img, L, nch, N), axis=1)[:, 0]
    assert np.abs(t.mean(axis=0)).max() < 4 / math.sqrt(3 * nch)
    assert np.allclose((t * t).mean(axis=0), 1 / 3, atol=4 * math.sqrt(4 / 45 / nch))


def test_phantom_deterministic_per_seed():
    a = oracle.phantom_chains((10.0, 10.0, 10.0), 5, 7, seed=3)
    b = oracle.phantom_chains((10.0, 10.0, 10.0), 5, 7, seed=3)
    c = oracle.phantom_chains((10.0, 10.0, 10.0), 5, 7, seed=4)
    assert (a[0] == b[0]).all() and (a[1] == b[1]).all()
    assert not (a[0] == c[0]).all()
