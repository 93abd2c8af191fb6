"""Pins of the oracle's slow push-off (Sec. II.B): overlapping beads are
pushed apart by ECs that start at them and ignore their pivot's overlaps,
the diameter growing in stages.  Checked: the final state has no overlap
and every tether holds; a hand-built overlapping pair is resolved; chain
statistics R^2(n) change little (the paper's point for the slow push-off);
a stage that cannot finish reports ESTUCK.  No GPU."""
import numpy as np
import pytest

import oracle


def phantom_system(eta, N, L, seed, c=1.9, D=(3, 3, 3), k_spring=0.0):
    nch = int(round(eta * L ** 3 * 6 / np.pi / N))
    r, img = oracle.phantom_chains((L, L, L), nch, N, bond=1.0, c=c, seed=seed)
    s = oracle.System(r, (L, L, L), N, sigma=1.0, b_max=1.2, mode=oracle.MODE_DOMAIN,
                      dir_mode=oracle.DIR_ISO, D=D, seed=seed + 100, img=img, k_spring=k_spring)
    return s, r.copy(), img.copy()


def test_pushoff_resolves_a_melt():
    s, r0, img0 = phantom_system(0.35, 20, 14.0, 31)
    assert s.overlap_flags(1.0)[1] > 100
    r2n0 = oracle.System(r0, s.L, 20, img=img0).chain_struct()["r2n"]
    rc, sweeps, st = s.pushoff(0.5, 5, 2.0, 2000)
    assert rc == 0 and sweeps > 0 and st["ecs"] > 0
    assert s.overlap_flags(1.0)[1] == 0
    dmin, n_ov = s.min_pair()
    assert n_ov == 0 and dmin * dmin >= 1.0 - 1e-10
    _, bonds = s.chain_obs()
    assert bonds.max() <= 1.2 * (1 + 1e-10) and bonds.min() >= np.sqrt(1.0 - 1e-10)
    # the slow push-off keeps the chain statistics close to the phantom's
    r2n1 = s.chain_struct()["r2n"]
    for n in (5, 10, 19):
        assert r2n1[n] == pytest.approx(r2n0[n], rel=0.3)
    # unwrapped bonds are the wrapped ones: images follow the moves
    u = s.unwrapped().reshape(-1, 20, 3)
    assert np.allclose(np.linalg.norm(np.diff(u, axis=1), axis=2).ravel(), bonds, rtol=1e-9)


def test_pushoff_hand_built_pair():
    """Two single beads at distance 0.5 sigma in a large box: both start
    ECs (the pivot passes through its overlap partner) until they are at
    least sigma apart."""
    L = 12.0
    r = np.array([[6.0, 6.0, 6.0], [6.3, 6.4, 6.0]])
    s = oracle.System(r, (L, L, L), 1, sigma=1.0, b_max=1.2, mode=oracle.MODE_DOMAIN,
                      dir_mode=oracle.DIR_ISO, D=(3, 3, 3), seed=7)
    assert s.overlap_flags(1.0)[1] == 2
    rc, sweeps, st = s.pushoff(1.0, 1, 2.0, 200)
    assert rc == 0 and st["ecs"] >= 1
    d = s.r[0] - s.r[1]
    d -= L * np.round(d / L)
    assert d @ d >= 1.0 - 1e-10


def test_pushoff_deterministic_and_stuck():
    a, _, _ = phantom_system(0.3, 10, 10.0, 41)
    b, _, _ = phantom_system(0.3, 10, 10.0, 41)
    ra = a.pushoff(0.5, 3, 2.0, 3000)
    rb = b.pushoff(0.5, 3, 2.0, 3000)
    assert ra[0] == 0 and ra[:2] == rb[:2] and (a.r == b.r).all() and (a.img == b.img).all()
    c, _, _ = phantom_system(0.45, 10, 10.0, 42)
    rc, sweeps, _ = c.pushoff(0.9, 1, 2.0, 1)
    assert rc == -6 and sweeps == 1


@pytest.mark.parametrize("L,d", [(12.0, 1.0), (6.0, 1.0), (12.0, 0.6), (2.5, 1.0)])
def test_overlap_flags_brute_force(L, d):
    """The push-off's overlap flags (cell grid, or all pairs in small boxes)
    against a direct numpy evaluation over all minimum-image pairs."""
    rng = np.random.default_rng(int(L * 10 + d * 100))
    n = int(0.6 * L ** 3)
    r = rng.uniform(0, L, (n, 3))
    s = oracle.System(r, (L, L, L), 1, sigma=1.0, b_max=1.2)
    flag, m = s.overlap_flags(d)
    x = r[:, None, :] - r[None, :, :]
    x -= L * np.round(x / L)
    dd = (x[..., 0] * x[..., 0] + x[..., 1] * x[..., 1]) + x[..., 2] * x[..., 2]
    np.fill_diagonal(dd, np.inf)
    ref = (dd < d * d * (1.0 - 1e-10)).any(axis=1)
    assert (flag.astype(bool) == ref).all() and m == ref.sum()


def test_pushoff_with_springs_resolves_a_melt():
    """With bead springs (k = 30) acting during the push-off (rest length the
    current diameter): no overlap at sigma when it ends, bonded beads no
    closer than sigma either, bonds stretched beyond the tether length only
    a little (the springs are stiff: the free-bond law gives <b> = 1.168
    sigma at k = 30), images following the moves, and chain statistics near
    the phantom's."""
    s, r0, img0 = phantom_system(0.40, 16, 14.0, 53, k_spring=30.0)
    assert s.overlap_flags(1.0)[1] > 100
    r2n0 = oracle.System(r0, s.L, 16, img=img0).chain_struct()["r2n"]
    rc, sweeps, st = s.pushoff(0.5, 4, 2.0, 6000)
    assert rc == 0 and sweeps > 0
    dmin, n_ov = s.min_pair()
    assert n_ov == 0 and dmin * dmin >= 1.0 - 1e-10
    _, bonds = s.chain_obs()
    assert bonds.min() >= np.sqrt(1.0 - 1e-10)
    assert 1.0 < bonds.mean() < 1.3 and bonds.max() < 2.0
    r2n1 = s.chain_struct()["r2n"]
    for n in (5, 10, 15):
        assert r2n1[n] == pytest.approx(r2n0[n], rel=0.3)
    u = s.unwrapped().reshape(-1, 16, 3)
    assert np.allclose(np.linalg.norm(np.diff(u, axis=1), axis=2).ravel(), bonds, rtol=1e-9)
