"""Pins of the oracle's chain-structure observables (gyration tensor and
shape descriptors, Appendix A; R^2(n), Sec. II.B; W(R), Appendix A; the g2
summand, Sec. IV) against closed forms, brute force and the ideal-chain
values the paper prints.  No GPU."""
import math

import numpy as np
import pytest

import oracle


def rand_unit(rng, shape):
    v = rng.normal(size=shape + (3,))
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def system(u, N, L=2000.0):
    """Chains given by positions along them (any frame), placed in a large
    box so that no bond wraps."""
    r = np.asarray(u, dtype=np.float64).reshape(-1, 3) + 0.5 * L
    return oracle.System(r, (L, L, L), N, sigma=1.0, b_max=10.0)


def test_rod_closed_forms():
    """A straight rod of N beads at spacing a along a random direction e:
    S = a^2 (N^2 - 1)/12 e e^T, so lam = (0, 0, a^2 (N^2 - 1)/12),
    kappa2 = 1, b = lam3, c = 0; R^2(n) = n^2 a^2; |R_e| = (N - 1) a."""
    rng = np.random.default_rng(1)
    N, nch, a = 9, 40, 1.07
    e = rand_unit(rng, (nch,))
    u = (np.arange(N)[None, :, None] * a) * e[:, None, :] + rng.uniform(-5, 5, (nch, 1, 3))
    s = system(u, N)
    out = s.chain_struct(dR=0.25, nbins=64)
    sd = oracle.shape_descriptors(out["gyr"])
    lam3 = a * a * (N * N - 1) / 12.0
    assert np.allclose(sd["lam"][:, 2], lam3, rtol=1e-12)
    assert np.allclose(sd["lam"][:, :2], 0.0, atol=1e-12 * lam3)
    assert np.allclose(sd["T"], lam3, rtol=1e-12)
    assert np.allclose(sd["kappa2"], 1.0, atol=1e-9)
    assert np.allclose(sd["b"], lam3, rtol=1e-12) and np.allclose(sd["c"], 0.0, atol=1e-12 * lam3)
    S = out["gyr"]
    assert np.allclose(S[:, 0], lam3 * e[:, 0] ** 2, atol=1e-12 * lam3)
    assert np.allclose(S[:, 1], lam3 * e[:, 0] * e[:, 1], atol=1e-12 * lam3)
    assert np.allclose(S[:, 4], lam3 * e[:, 1] * e[:, 2], atol=1e-12 * lam3)
    n = np.arange(N)
    assert np.allclose(out["r2n"], (n * a) ** 2, rtol=1e-12)
    b = math.floor((N - 1) * a / 0.25)
    assert out["hist"][b] == nch and out["hist"].sum() == nch
    # the middle bead sits at the centre of a rod with odd N
    assert np.allclose(out["mid"], 0.0, atol=1e-12)


def test_square_closed_form():
    """Four beads on the corners of a square of side 2 (a chain around it),
    any orientation: S has eigenvalues (0, 1, 1), T = 2, P = 1, b = 1/2,
    c = 1, kappa2 = 1/4, 4 b^2 + 3 c^2 = 4 (T^2 - 3 P) = 4."""
    rng = np.random.default_rng(2)
    sq = np.array([[1, 1, 0], [1, -1, 0], [-1, -1, 0], [-1, 1, 0]], dtype=np.float64)
    us = []
    for _ in range(25):
        q, _r = np.linalg.qr(rng.normal(size=(3, 3)))
        us.append(sq @ q.T + rng.uniform(-3, 3, 3))
    out = system(np.array(us), 4).chain_struct(r2n=False)
    sd = oracle.shape_descriptors(out["gyr"])
    assert np.allclose(sd["lam"], [0.0, 1.0, 1.0], atol=1e-12)
    assert np.allclose(sd["T"], 2.0) and np.allclose(sd["P"], 1.0)
    assert np.allclose(sd["b"], 0.5) and np.allclose(sd["c"], 1.0)
    assert np.allclose(sd["kappa2"], 0.25) and np.allclose(sd["bc"], 4.0)
    assert np.allclose(4 * sd["b"] ** 2 + 3 * sd["c"] ** 2, sd["bc"])


def test_brute_force_small_periodic():
    """Chains that cross the periodic box: S, the middle bead, R^2(n) and
    the histogram against a direct numpy evaluation of the definitions
    (unwrap by minimum-image bonds, all pairs)."""
    rng = np.random.default_rng(3)
    N, nch, L = 12, 30, 6.0
    steps = rand_unit(rng, (nch, N - 1)) * rng.uniform(0.9, 1.2, (nch, N - 1, 1))
    u = np.concatenate([np.zeros((nch, 1, 3)), np.cumsum(steps, axis=1)], axis=1)
    u += rng.uniform(0, L, (nch, 1, 3))
    r = np.mod(u, L).reshape(-1, 3)
    s = oracle.System(r, (L, L, L), N, sigma=0.5, b_max=1.3)
    out = s.chain_struct(dR=0.5, nbins=12)
    w = r.reshape(nch, N, 3)
    d = np.diff(w, axis=1)
    d -= L * np.round(d / L)
    uu = np.concatenate([np.zeros((nch, 1, 3)), np.cumsum(d, axis=1)], axis=1)
    U = uu.mean(axis=1, keepdims=True)
    x = uu - U
    S = np.einsum("cja,cjb->cab", x, x) / N
    idx = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    for k, (a, b) in enumerate(idx):
        assert np.allclose(out["gyr"][:, k], S[:, a, b], rtol=1e-12, atol=1e-13)
    assert np.allclose(out["mid"], x[:, N // 2], atol=1e-12)
    for n in range(1, N):
        ref = np.mean(np.sum((uu[:, n:] - uu[:, :-n]) ** 2, axis=2))
        assert out["r2n"][n] == pytest.approx(ref, rel=1e-12)
    R = np.linalg.norm(uu[:, -1], axis=1)
    assert (out["hist"] == np.bincount(np.minimum((R // 0.5).astype(int), 11), minlength=12)).all()


def test_g2_summand_closed_forms():
    """Rigid translation of a chain leaves u_{N/2} - U unchanged (g2
    summand 0); moving bead N/2 alone by d gives |d|^2 (1 - 1/N)^2."""
    rng = np.random.default_rng(4)
    N, nch = 10, 20
    steps = rand_unit(rng, (nch, N - 1))
    u = np.concatenate([np.zeros((nch, 1, 3)), np.cumsum(steps, axis=1)], axis=1)
    m0 = system(u, N).chain_struct(r2n=False)["mid"]
    shifted = u + rng.uniform(-20, 20, (nch, 1, 3))
    m1 = system(shifted, N).chain_struct(r2n=False)["mid"]
    assert np.allclose(oracle.g2_terms(m0, m1), 0.0, atol=1e-20)
    dv = rng.uniform(-0.3, 0.3, (nch, 3))
    moved = u.copy()
    moved[:, N // 2] += dv
    m2 = system(moved, N).chain_struct(r2n=False)["mid"]
    expect = np.sum(dv * dv, axis=1) * (1.0 - 1.0 / N) ** 2
    assert np.allclose(oracle.g2_terms(m0, m2), expect, rtol=1e-10)


@pytest.fixture(scope="module")
def random_walks():
    """Freely jointed chains (unit bonds, isotropic, no excluded volume)."""
    rng = np.random.default_rng(5)
    N, nch = 600, 4000
    steps = rand_unit(rng, (nch, N - 1))
    u = np.concatenate([np.zeros((nch, 1, 3)), np.cumsum(steps, axis=1)], axis=1)
    s = system(u, N)
    return N, nch, s.chain_struct(dR=1.0, nbins=200, r2n=False)


def test_random_walk_shape_matches_paper_limits(random_walks):
    """Long ideal chains against the shape values printed with the paper's
    shape table (Appendix A): the ratios of the inertia-tensor eigenvalue
    combinations to its trace, quoted as 0.754, 0.175 and 0.0646 (an
    approximate theory; the paper's own runs give 0.757-0.767, 0.170-0.178
    and 0.062-0.065), <4 b^2 + 3 c^2> / <Tr I>^2 quoted as 2/3 (runs
    0.62-0.67) and <kappa2> quoted as 0.42 (runs 0.39-0.40).  The bounds
    take in the quoted values, the paper's spread and the sampling error of
    4000 chains; a wrong eigenvalue order or a dropped term lands far
    outside them."""
    N, nch, out = random_walks
    sd = oracle.shape_descriptors(out["gyr"])
    T = sd["T"].mean()
    lam = sd["lam"].mean(axis=0)
    # I1 + I2 - I3 = 2 N lam3, I1 - I2 + I3 = 2 N lam2, -I1 + I2 + I3 = 2 N lam1, Tr I = 2 N T
    assert 0.750 <= lam[2] / T <= 0.775
    assert 0.165 <= lam[1] / T <= 0.185
    assert 0.058 <= lam[0] / T <= 0.070
    # <4 b_I^2 + 3 c_I^2> / <Tr I>^2 with b_I = N b, c_I = N c, Tr I = 2 N T
    assert 0.62 <= sd["bc"].mean() / (4.0 * T * T) <= 0.69
    assert 0.37 <= sd["kappa2"].mean() <= 0.43
    # R_g^2 of a long random walk: <R^2>/6 with <R^2> = N - 1 unit bonds
    assert T == pytest.approx((N - 1) / 6.0, rel=0.03)


def test_random_walk_end_to_end_distribution(random_walks):
    """W(R) of long ideal chains: the Gaussian of the paper's Appendix A
    with <R^2> = (N - 1) b^2; compare the cumulative distribution."""
    N, nch, out = random_walks
    h = out["hist"]
    R2 = N - 1.0
    cdf = np.cumsum(h) / nch
    for Rb in (10, 20, 30, 40):
        x = Rb * math.sqrt(1.5 / R2)
        F = math.erf(x) - 2.0 / math.sqrt(math.pi) * x * math.exp(-x * x)
        assert cdf[Rb - 1] == pytest.approx(F, abs=0.03)


def test_random_walk_internal_distances():
    """Ideal chains: R^2(n) = n b^2 for every n (the linear law the paper's
    internal-distance plots compare with); unit bonds give R^2(1) = 1."""
    rng = np.random.default_rng(6)
    N, nch = 150, 800
    steps = rand_unit(rng, (nch, N - 1))
    u = np.concatenate([np.zeros((nch, 1, 3)), np.cumsum(steps, axis=1)], axis=1)
    out = system(u, N).chain_struct()
    r2n = out["r2n"]
    assert r2n[0] == 0.0 and r2n[1] == pytest.approx(1.0, rel=1e-12)
    for n in (5, 20, 60, 120):
        assert r2n[n] / n == pytest.approx(1.0, abs=4.0 * math.sqrt(2.0 / (3.0 * nch * (N - n) / n)) + 0.01)
