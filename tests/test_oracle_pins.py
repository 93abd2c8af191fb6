"""Pins of the oracle against what the paper and mathematics fix.

Each test names what it pins.  None re-types the oracle's formulas: they use
closed forms (Tonks gas, the tethered dimer's bond-length law, the simplex gap
law of rods on a ring), library routines (numpy's Philox), textbook equations
of state (Carnahan-Starling), invariants of the method (no overlap, bonds
within b_max, total displacement ell per EC) and hand-worked tiny geometries.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import DIR_CART3, DIR_ISO, DIR_PLUSX, MODE_DOMAIN, MODE_SERIAL


# ---------------------------------------------------------------- Philox
def test_philox_matches_numpy_philox4x64():
    """Pinned to numpy's independent Philox4x64-10 (a library routine).
    numpy advances its 256-bit counter before producing a block."""
    rng = np.random.default_rng(7)
    for _ in range(64):
        ctr = rng.integers(0, 2**63, size=4, dtype=np.uint64)
        key = rng.integers(0, 2**63, size=2, dtype=np.uint64)
        v = sum(int(ctr[i]) << (64 * i) for i in range(4)) - 1
        v %= 2**256
        prev = np.array([(v >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)
        ref = np.random.Philox(key=key, counter=prev).random_raw(4)
        assert (oracle.philox4x64_10(ctr, key) == ref).all()


def test_start_draws_uniform_and_isotropic():
    """Start bead uniform over the beads, isotropic v uniform on the sphere
    (first and second moments), |v| = 1 to rounding; Cartesian mode gives
    the three positive axes with equal weight."""
    s = oracle.System(np.zeros((7, 3)), 10.0, 1, dir_mode=DIR_ISO, seed=11)
    n = 60000
    idx, v = s.start_draws(n)
    cnt = np.bincount(idx, minlength=7)
    chi2 = ((cnt - n / 7) ** 2 / (n / 7)).sum()
    assert chi2 < 22.5  # 6 dof, p ~ 0.001
    assert np.abs(np.linalg.norm(v, axis=1) - 1).max() < 1e-15
    assert np.abs(v.mean(0)).max() < 4 * math.sqrt(1 / 3 / n)
    cov = v.T @ v / n
    assert np.abs(cov - np.eye(3) / 3).max() < 0.01
    s2 = oracle.System(np.zeros((7, 3)), 10.0, 1, dir_mode=DIR_CART3, seed=11)
    _, v2 = s2.start_draws(30000)
    assert set(map(tuple, v2)) == {(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)}
    frac = (v2 == 1.0).mean(0)
    assert np.abs(frac - 1 / 3).max() < 0.015


# ---------------------------------------------------------------- lattice
def test_lattice_is_a_snake_through_every_site():
    """Initial melt: every site of the n0 x n1 x n2 grid occupied once and
    consecutive beads one lattice step apart (a Hamiltonian path), so every
    bond of every chain has length a <= b_max."""
    dims, a = (5, 4, 3), 1.05
    r = oracle.lattice(dims, a)
    idx = np.rint(r / a - 0.5).astype(int)
    assert len({tuple(t) for t in idx}) == 60
    assert idx.min() == 0 and (idx.max(0) == np.array(dims) - 1).all()
    steps = np.abs(np.diff(idx, axis=0)).sum(1)
    assert (steps == 1).all()
    bond = np.linalg.norm(np.diff(r, axis=0), axis=1)
    assert np.allclose(bond, a, rtol=0, atol=1e-12)


# ---------------------------------------------------------------- worked example
def test_hand_worked_dimer_events():
    """Two bonded beads on the x axis, v = +x, b_max = 1.2, ell = 0.5.
    Worked by hand from the collision rule (Eq. 1) and the tether limit:
    the EC alternates hard-sphere contacts (gap closes) and tether events
    (bond reaches b_max), each carrying the chain to the other bead."""
    r = np.array([[1.0, 5.0, 5.0], [2.05, 5.0, 5.0]])
    s = oracle.System(r, (10.0, 10.0, 10.0), 2, b_max=1.2, s_cap=2.0, dir_mode=DIR_PLUSX,
                      use_cells=0, seed=3)
    start, _ = s.start_draws(1)
    res = s.run_serial(1, 0.5, log_cap=64)
    log = res["log"]
    # expected by hand
    xs, kinds, piv = [], [], []
    p = [1.0, 2.05]
    i, rem = int(start[0]), 0.5
    while True:
        j = 1 - i
        if p[j] > p[i]:   # partner ahead: contact after the gap closes
            x, kind = p[j] - p[i] - 1.0, 3
        else:             # partner behind: tether taut at b_max
            x, kind = 1.2 - (p[i] - p[j]), 5
        if x >= rem:
            xs.append(rem); kinds.append(0); piv.append(i)
            break
        p[i] += x
        rem -= x
        xs.append(x); kinds.append(kind); piv.append(i)
        i = j
    assert list(log["kind"]) == kinds
    assert list(log["pivot"]) == piv
    assert np.allclose(log["x"], xs, rtol=0, atol=1e-12)
    assert abs(log["x"].sum() - 0.5) < 1e-14


# ---------------------------------------------------------------- 1D exact laws
def _rods(n, Lx, seed, n_ec):
    """n unit rods on a ring (3-D code, all beads on one line, v = +x).  The
    EC length is drawn per EC from U(0.5, 2.5) by the test: a fixed length
    close to the free length mixes slowly on so small a ring."""
    r = np.zeros((n, 3))
    r[:, 0] = (np.arange(n) + 0.5) * (Lx / n)
    r[:, 1:] = 2.5
    s = oracle.System(r, (Lx, 10.0, 10.0), 1, s_cap=0.45 * Lx - 1.0, dir_mode=DIR_PLUSX,
                      use_cells=0, seed=seed)
    ells = np.random.default_rng(seed).uniform(0.5, 2.5, n_ec)
    gaps, lifts = [], []
    for j in range(n_ec):
        res = s.run_serial(1, ells[j], ec0=j)
        assert res["rc"] == 0
        # rods keep their cyclic order: the gap ahead of rod 0 is rod 1's
        gaps.append((s.r[1, 0] - s.r[0, 0]) % Lx - 1.0)
        lifts.append(res["stats"]["lift_sum"])
    return np.array(gaps), np.array(lifts), ells


def test_rods_on_ring_gap_law_and_pressure():
    """Three unit rods on a ring of length 6 (v = +x only, global balance):
    gaps are uniform on the simplex sum g = 3, so one gap has density
    2(3-g)/9.  The lift-distance estimator must give the exact canonical
    pressure of n rods on a ring, betaP = 1/L + (n-1)/(L - n sigma) (the
    configuration integral is L (L - n sigma)^(n-1)/(n-1)!), i.e.
    betaP/rho = 5/3 here; for n -> infinity this is Tonks' 1/(1 - rho sigma)."""
    Lx, n = 6.0, 3
    gaps, lifts, ells = _rods(n, Lx, 5, 30000)
    S = Lx - n
    edges = np.linspace(0, S, 7)
    cnt, _ = np.histogram(gaps[200:], edges)
    cdf = lambda g: 1 - (1 - g / S) ** 2
    exp = np.diff(cdf(edges)) * cnt.sum()
    chi2 = ((cnt - exp) ** 2 / exp).sum()
    assert chi2 < 30, (cnt, exp)  # 5 dof; samples mildly correlated
    zb = [1.0 + lb.sum() / eb.sum()
          for lb, eb in zip(np.array_split(lifts, 40), np.array_split(ells, 40))]
    se = np.std(zb, ddof=1) / math.sqrt(len(zb))
    z = 1.0 + lifts.sum() / ells.sum()
    rho = n / Lx
    exact = (1.0 / Lx + (n - 1) / (Lx - n)) / rho
    assert abs(z - exact) < 3 * se + 1e-3, (z, se, exact)


def test_two_rods_gap_uniform():
    """Two rods on a ring: the gap is uniform on [0, L - 2 sigma]."""
    gaps, _, _ = _rods(2, 5.0, 9, 20000)
    cnt, _ = np.histogram(gaps[100:], np.linspace(0, 3.0, 7))
    exp = cnt.sum() / 6
    assert ((cnt - exp) ** 2 / exp).sum() < 30


# ---------------------------------------------------------------- dimer
def _dimer_bonds(mode, seed, n_rounds):
    r = np.array([[3.0, 3.0, 3.0], [4.1, 3.0, 3.0]])
    kw = dict(b_max=1.2, dir_mode=DIR_ISO, use_cells=0, seed=seed)
    if mode == MODE_SERIAL:
        s = oracle.System(r, 9.0, 2, s_cap=2.0, **kw)
    else:
        s = oracle.System(r, 9.0, 2, s_cap=2.0, mode=MODE_DOMAIN, D=(3, 3, 3), w=1.2, **kw)
    out = []
    for j in range(n_rounds):
        if mode == MODE_SERIAL:
            s.run_serial(1, 0.7, ec0=j)
        else:
            s.run_domain(1, 0.7, sweep0=j)
        d = s.r[1] - s.r[0]
        d -= 9.0 * np.round(d / 9.0)
        out.append(np.linalg.norm(d))
    return np.array(out), s


@pytest.mark.parametrize("mode", [MODE_SERIAL, MODE_DOMAIN])
def test_dimer_bond_length_law(mode):
    """An isolated tethered dimer (N=2): the bond length b is distributed as
    3 b^2 / (b_max^3 - sigma^3) on [sigma, b_max].  In the domain mode the
    partner is often immotile (in a joint), so this pins the reflection at
    the plane normal to the bond (Fig. 2c) and at the tile walls."""
    b, s = _dimer_bonds(mode, 21 + mode, 8000)
    b = b[100:]
    assert b.min() >= 1.0 - 1e-12 and b.max() <= 1.2 + 1e-12
    edges = np.linspace(1.0, 1.2, 9)
    cnt, _ = np.histogram(b, edges)
    cdf = lambda x: (x ** 3 - 1.0) / (1.2 ** 3 - 1.0)
    exp = np.diff(cdf(edges)) * cnt.sum()
    chi2 = ((cnt - exp) ** 2 / exp).sum()
    assert chi2 < 40, (cnt, exp)


def test_domain_single_bead_uniform_in_box():
    """One free bead in the domain mode: the random tile shift plus wall
    reflections (a billiard in the tile, which keeps the uniform measure)
    must leave its stationary density uniform over the box."""
    s = oracle.System(np.array([[1.0, 1.0, 1.0]]), 9.0, 1, b_max=1.0, s_cap=2.0,
                      mode=MODE_DOMAIN, D=(3, 3, 3), w=1.0, dir_mode=DIR_ISO, use_cells=0,
                      seed=77)
    xs = []
    for j in range(30000):
        res = s.run_domain(1, 7.3, sweep0=j)
        assert res["rc"] == 0
        xs.append(s.r[0].copy())
    xs = np.array(xs[100::10])
    for a in range(3):
        cnt, _ = np.histogram(xs[:, a], np.linspace(0, 9.0, 10))
        exp = cnt.sum() / 9
        assert ((cnt - exp) ** 2 / exp).sum() < 40, cnt


# ---------------------------------------------------------------- 3D hard spheres
def _hs_fluid(phi, seed, n_eq, n_run, ell=2.0, blocks=50, delta=0.02):
    """Serial ECs on 252 unbonded spheres: per block the lift-distance
    pressure and the contact-value pressure of the block's last state."""
    dims = (6, 6, 7)
    a = (math.pi / (6 * phi)) ** (1 / 3)
    r = oracle.lattice(dims, a)
    s = oracle.System(r, tuple(d * a for d in dims), 1, s_cap=0.4, dir_mode=DIR_ISO,
                      seed=seed)
    s.run_serial(n_eq, ell)
    z, zc = [], []
    chunk = n_run // blocks
    for b in range(blocks):
        res = s.run_serial(chunk, ell, ec0=n_eq + b * chunk)
        z.append(1.0 + res["stats"]["lift_sum"] / (chunk * ell))
        zc.append(s.contact_pressure(delta))
    return np.array(z), np.array(zc), s


def test_hard_sphere_fluid_pressure_carnahan_starling():
    """Unbonded hard spheres (N=1) at phi = 0.30: the lift-distance estimator
    and the contact-value estimator must both reproduce Carnahan-Starling
    (1+e+e^2-e^3)/(1-e)^3 within 3 standard errors plus a 1% budget for CS
    itself and the 252-sphere finite size (the contact value also carries
    the bias of its linear extrapolation over 0.04 sigma)."""
    phi = 0.30
    z, zc, s = _hs_fluid(phi, 0xC5, 3000, 60000, blocks=150)
    zcs = (1 + phi + phi ** 2 - phi ** 3) / (1 - phi) ** 3
    se = z.std(ddof=1) / math.sqrt(len(z))
    assert abs(z.mean() - zcs) < 3 * se + 0.01 * zcs, (z.mean(), se, zcs)
    sec = zc.std(ddof=1) / math.sqrt(len(zc))
    assert abs(zc.mean() - zcs) < 3 * sec + 0.015 * zcs, (zc.mean(), sec, zcs)
    dmin, nov = s.min_pair()
    assert nov == 0 and dmin >= 1.0 - 1e-12


def test_contact_counts_hand_built():
    """Contact shells on a hand-built state (delta = 0.02): a dimer at 1.005
    (pair shell 1), a non-bonded pair at 1.03 across the periodic boundary
    (pair shell 2), dimers stretched to 1.19 and 1.17 (bond shells 1 and 2)
    and one at 1.1 (neither); everything else far apart."""
    L = 20.0
    r = np.array([
        [2.0, 2.0, 2.0], [3.005, 2.0, 2.0],      # dimer, pair shell 1
        [10.0, 10.0, 5.0], [10.0, 11.19, 5.0],   # bond shell 1
        [5.0, 15.0, 15.0], [5.0, 15.0, 16.17],   # bond shell 2
        [19.5, 8.0, 8.0], [19.5, 9.1, 8.0],      # plain dimer
        [0.53, 8.0, 8.0], [0.53, 12.0, 12.0],    # bead 8: 1.03 from bead 6 across x = L
    ])
    s = oracle.System(r, (L, L, L), 2, sigma=1.0, b_max=1.2)
    pairs, bonds = s.contacts(0.02)
    assert list(pairs) == [1, 1], pairs
    assert list(bonds) == [1, 1], bonds
# ---------------------------------------------------------------- invariants
def test_invariants_after_c1_sized_run():
    """C1 geometry (8x8x10 lattice, N=10): after serial ECs no pair overlaps,
    every bond within [sigma, b_max], and each EC displaced exactly ell."""
    from paper_1502_06447_gb300.configs import C1
    r = oracle.lattice(C1.dims, C1.spacing, C1.jitter, C1.seed)
    s = oracle.System(r, C1.L, C1.N, seed=C1.seed)
    n_ec = 3000
    res = s.run_serial(n_ec, C1.ell, digests=True)
    assert res["rc"] == 0
    st = res["stats"]
    assert st["ecs"] == n_ec and st["end"] == n_ec
    assert abs(st["disp_sum"] - n_ec * C1.ell) < 1e-12 * n_ec * C1.ell * 10
    dmin, nov = s.min_pair()
    assert nov == 0 and dmin >= 1.0 - 1e-12
    _, bonds = s.chain_obs()
    assert bonds.max() <= 1.2 * (1 + 1e-12) and bonds.min() >= 1.0 - 1e-12
    assert (s.r >= 0).all() and (s.r < np.array(C1.L)).all()


def test_cell_list_search_equals_all_pairs_search():
    """The oracle's cell-list search must reproduce the all-pairs search
    event for event (same per-EC digests and bit-identical positions), in
    serial and domain mode."""
    from paper_1502_06447_gb300.configs import C1
    r = oracle.lattice(C1.dims, C1.spacing, C1.jitter, 4)
    a = oracle.System(r, C1.L, C1.N, seed=4, use_cells=1)
    b = oracle.System(r, C1.L, C1.N, seed=4, use_cells=0)
    ra = a.run_serial(300, C1.ell, digests=True)
    rb = b.run_serial(300, C1.ell, digests=True)
    assert (ra["digest"] == rb["digest"]).all()
    assert (a.r == b.r).all() and (a.img == b.img).all()
    r = oracle.lattice((12, 12, 12), 1.05, 0.01, 5)
    L = 12 * 1.05
    kw = dict(mode=MODE_DOMAIN, D=(3, 3, 3), dir_mode=DIR_ISO, seed=5)
    a = oracle.System(r, L, 8, use_cells=1, **kw)
    b = oracle.System(r, L, 8, use_cells=0, **kw)
    ra = a.run_domain(3, 3.0, digests=True)
    rb = b.run_domain(3, 3.0, digests=True)
    assert (ra["digest"] == rb["digest"]).all()
    assert (a.r == b.r).all()


def test_swap_without_bonds_is_bookkeeping_only():
    """Sec. II.C: without bonds, EC with and without swaps are identical up
    to bookkeeping.  From the same state, one EC with p_swap = 1 must leave
    the same set of occupied positions as one EC without swaps, bit for bit,
    with every no-swap lift replaced by an accepted swap.  (Over several ECs
    the paths part: the next start bead is drawn by label, and swaps permute
    labels.)"""
    r = oracle.lattice((6, 6, 6), 1.2, 0.01, 12)
    kw = dict(s_cap=0.3, dir_mode=DIR_ISO, seed=12)
    a = oracle.System(r, 7.2, 1, p_swap=0.0, **kw)
    b = oracle.System(r, 7.2, 1, p_swap=1.0, **kw)
    n_swap = 0
    for j in range(300):
        b.r[:] = a.r
        ra = a.run_serial(1, 6.0, ec0=j)
        rb = b.run_serial(1, 6.0, ec0=j)
        assert ra["stats"]["hs_lift"] == rb["stats"]["swap"]
        assert rb["stats"]["hs_lift"] == 0
        assert ra["stats"]["events"] == rb["stats"]["events"]
        n_swap += rb["stats"]["swap"]
        ka = np.lexsort(a.r.T[::-1])
        kb = np.lexsort(b.r.T[::-1])
        assert (a.r[ka] == b.r[kb]).all()
    assert n_swap > 1000


def test_swap_keeps_tethers():
    """Swaps in a melt (Sec. II.C, accepted only if every bond stays within
    b_max): after swaps all bonds still within [sigma, b_max]."""
    r = oracle.lattice((8, 8, 8), 1.05, 0.01, 13)
    s = oracle.System(r, 8 * 1.05, 8, p_swap=1.0, dir_mode=DIR_ISO, seed=13)
    res = s.run_serial(6000, 3.0)
    st = res["stats"]
    assert st["swap"] > 0 and st["swap_tried"] > st["swap"]
    _, bonds = s.chain_obs()
    assert bonds.max() <= 1.2 * (1 + 1e-12) and bonds.min() >= 1.0 - 1e-12
    assert s.min_pair()[1] == 0


# ---------------------------------------------------------------- domain partition
def test_domain_tags_partition_geometry():
    """Tile-joint partition (Sec. II.A): motile beads of different tiles are
    more than w apart, joint beads are exactly the points within w of the
    upper faces, and the motile fraction is ((T-w)/T)^3."""
    rng = np.random.default_rng(3)
    L, D, w = 12.0, 4, 1.2
    r = rng.uniform(0, L, size=(20000, 3))
    s = oracle.System(r, L, 1, mode=MODE_DOMAIN, D=(D, D, D), w=w, seed=8)
    tags, shift = s.domain_tags(5)
    assert ((shift >= 0) & (shift < L / D)).all()
    T = L / D
    u = (r - shift) % L
    loc = u - np.floor(u / T) * T
    inside = (loc < T - w - 1e-9).all(1)
    outside = (loc >= T - w + 1e-9).any(1)
    assert (tags[inside] >= 0).all() and (tags[outside] == -1).all()
    frac = (tags >= 0).mean()
    assert abs(frac - ((T - w) / T) ** 3) < 0.01
    # beads of different tiles are separated by more than w
    sub = rng.choice(np.nonzero(tags >= 0)[0], 3000, replace=False)
    d = r[sub, None, :] - r[None, sub, :]
    d -= L * np.round(d / L)
    dist = np.linalg.norm(d, axis=2)
    diff = tags[sub][:, None] != tags[sub][None, :]
    assert dist[diff].min() > w


# ---------------------------------------------------------------- observables
def test_chain_end_to_end_closed_forms():
    """R_e^2 and bond lengths of chains built from known bond vectors and
    wrapped into the box: R_e = sum of the bond vectors (the construction),
    independent of how the oracle undoes the wrapping."""
    L = np.array([10.0, 9.0, 11.0])
    rng = np.random.default_rng(7)
    N, nch = 7, 3
    r = np.zeros((N * nch, 3))
    expect_re2, expect_b = [], []
    for c in range(nch):
        if c == 0:  # straight along x through the x = L boundary
            b = np.tile([1.1, 0.0, 0.0], (N - 1, 1))
            start = np.array([7.0, 4.5, 5.5])
        else:  # random directions, lengths in [1, 1.2]
            u = rng.normal(size=(N - 1, 3))
            b = u / np.linalg.norm(u, axis=1)[:, None] * rng.uniform(1.0, 1.2, size=(N - 1, 1))
            start = rng.uniform(0, 1, 3) * L
        pos = start + np.vstack([np.zeros(3), np.cumsum(b, axis=0)])
        r[c * N:(c + 1) * N] = np.mod(pos, L)
        expect_re2.append(float(np.sum(b.sum(axis=0) ** 2)))
        expect_b.extend(np.linalg.norm(b, axis=1))
    s = oracle.System(r, L, N)
    re2, bonds = s.chain_obs()
    assert abs(re2[0] - (6 * 1.1) ** 2) < 1e-12
    assert np.allclose(re2, expect_re2, rtol=1e-12, atol=1e-12)
    assert np.allclose(bonds, expect_b, rtol=1e-12, atol=1e-12)


def test_unwrapped_displacement_is_ell_along_each_ec_direction():
    """Serial ECs with v in {+x,+y,+z}: every free flight moves one bead along
    v, so the summed unwrapped displacement of all beads is ell times the sum
    of the ECs' directions (pins the image counters behind g1)."""
    from paper_1502_06447_gb300.configs import C1
    r = oracle.lattice(C1.dims, C1.spacing, C1.jitter, C1.seed)
    s = oracle.System(r, C1.L, C1.N, dir_mode=DIR_CART3, seed=C1.seed)
    u0 = s.unwrapped().copy()
    n_ec = 2000
    assert s.run_serial(n_ec, C1.ell)["rc"] == 0
    _, v = s.start_draws(n_ec)
    moved = (s.unwrapped() - u0).sum(axis=0)
    expect = C1.ell * v.sum(axis=0)
    assert np.allclose(moved, expect, rtol=0, atol=1e-8 * n_ec)
    # a wrong image sign would be off by whole box lengths
    assert np.abs(moved - expect).max() < 1e-3


def test_tile_subsets_split_a_sweep_exactly():
    """The all-core timing of the oracle splits a sweep's tiles over
    processes (tile t runs in part t % 3): the parts together do exactly the
    serial sweep's ECs (same per-EC digests, same event count), because
    tiles never interact within a sweep (Sec. II.A)."""
    from paper_1502_06447_gb300.configs import small_domain
    m = small_domain(N=8, dims=(16, 16, 16), D=(4, 4, 4), sweeps=1, ell=4.0)
    r = oracle.lattice(m.dims, m.spacing, m.jitter, m.seed)
    kw = dict(mode=MODE_DOMAIN, dir_mode=DIR_ISO, D=m.D, seed=m.seed)
    full = oracle.System(r, m.L, m.N, **kw).run_domain(1, m.ell, digests=True)
    dig = np.zeros_like(full["digest"])
    events = 0
    for rem in range(3):
        part = oracle.System(r, m.L, m.N, tile_mod=3, tile_rem=rem, **kw).run_domain(
            1, m.ell, digests=True)
        assert part["rc"] == 0
        mine = np.arange(len(dig)) % 3 == rem  # one EC per tile: ordinal = tile
        assert (part["digest"][~mine] == 0).all()
        dig[mine] = part["digest"][mine]
        events += part["stats"]["events"]
    assert (dig == full["digest"]).all() and events == full["stats"]["events"]
