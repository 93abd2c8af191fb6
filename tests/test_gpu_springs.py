"""Bead-spring chains on the GPU against the oracle (Sec. II: ECs for pair
potentials with a harmonic bond (k/2)(b - sigma)^2, a Boltzmann energy per
bond and event; Sec. II.A: reflection at an immotile spring partner, and
the motility rule that keeps tiles apart when bonds have no longest length).

Event digests, lift sums, event counts, final positions and images must
equal the oracle's bit for bit, in the serial and the domain form, plain
FP64 and FP32-screened, for every lane count.  k = 30 kT/sigma^2 is the
paper's stiffness; k = 2 stretches bonds far beyond the tether halo, so the
staging has to fetch bonded beads from anywhere in the box."""
import math

import numpy as np
import pytest

import oracle
from paper_1502_06447_gb300 import ecmc
from paper_1502_06447_gb300.configs import C1, Melt, small_domain

from helpers import gpu_context, oracle_system

pytestmark = pytest.mark.gpu

PRECS = {"fp64": ecmc.PREC_FP64, "fp32f": ecmc.PREC_FP32F}


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1502_06447_gb300 import build
    build.build()


def assert_same_state(gpu, orc):
    r, img = gpu.get_positions()
    bad = np.nonzero((r != orc.r).any(1))[0]
    assert bad.size == 0, f"{bad.size} beads differ, first {bad[:5]}"
    assert (img == orc.img).all()


def assert_same_counts(gpu, res):
    obs = gpu.observables()
    for k in oracle.OUT_NAMES:
        assert obs[k] == res["stats"][k], k
    assert obs["events_total"] == res["stats"]["events"]
    assert obs["overlaps"] == 0
    return obs


@pytest.mark.parametrize("prec", ["fp64", "fp32f"])
def test_spring_serial_parity(prec):
    """The C1 melt (64 chains x N = 10) as bead springs, 3000 serial ECs."""
    o = oracle_system(C1, k_spring=30.0)
    res = o.run_serial(3000, C1.ell, digests=True)
    assert res["rc"] == 0
    ctx = gpu_context(C1, precision=PRECS[prec], k_spring=30.0)
    ctx.run(C1.ell, chains_per_sweep=3000, seed=C1.seed)
    dig, lift, ev = ctx.records(3000)
    first = np.nonzero(dig != res["digest"])[0]
    assert first.size == 0, f"first differing EC {first[:3]}"
    assert (ev == res["ec_events"]).all() and (lift == res["ec_lift"]).all()
    assert_same_state(ctx, o)
    obs = assert_same_counts(ctx, res)
    assert obs["te_lift"] > 0


def test_spring_event_log_matches_oracle():
    o = oracle_system(C1, k_spring=30.0)
    res = o.run_serial(100, C1.ell, log_cap=100000)
    ctx = gpu_context(C1, k_spring=30.0)
    ctx.log_reserve(100000)
    ctx.run(C1.ell, chains_per_sweep=100, seed=C1.seed)
    log = ctx.event_log(100000)
    ref = res["log"]
    assert len(log) == len(ref)
    for f in ("unit", "pivot", "kind", "partner", "x"):
        assert (log[f] == ref[f]).all(), f


def stretched_dimers(seed, L=16.8, grid=6, bond=1.6):
    """Seeded input: dimers with bonds of 1.6 sigma in random directions,
    centred on a grid of spacing L / grid = 2.8 (beads of different dimers
    stay >= 1.2 apart), so that many bonds reach across a joint of 1.2."""
    rng = np.random.default_rng(seed)
    a = L / grid
    c = (np.stack(np.meshgrid(*(np.arange(grid),) * 3, indexing="ij"), -1).reshape(-1, 3) + 0.5) * a
    u = rng.normal(size=c.shape)
    u /= np.linalg.norm(u, axis=1)[:, None]
    r = np.empty((2 * len(c), 3))
    r[0::2] = c - 0.5 * bond * u
    r[1::2] = c + 0.5 * bond * u
    return np.mod(r, L), L


@pytest.mark.parametrize("seed", [1, 2])
def test_spring_domain_tags_match_oracle(seed):
    """Tile tags with the spring motility rule: a bead whose bonded bead is
    motile in another tile is immotile for the sweep (stretched dimers, so
    that the rule acts)."""
    r, L = stretched_dimers(seed)
    D = (3, 3, 3)
    ctx = ecmc.Context.create_phantom((L, L, L), len(r) // 2, 2, bond=1.0, seed=seed, b_max=1.2)
    ctx.configure(mode=ecmc.MODE_DOMAIN, dir_mode=ecmc.DIR_ISO, tiles=D, k_spring=30.0)
    ctx.set_positions(r)
    kw = dict(sigma=1.0, b_max=1.2, mode=oracle.MODE_DOMAIN, dir_mode=oracle.DIR_ISO, D=D,
              seed=seed)
    o = oracle.System(r, (L, L, L), 2, k_spring=30.0, **kw)
    plain = oracle.System(r, (L, L, L), 2, **kw)
    dropped = 0
    for sweep in (0, 3, 7):
        tags, shift = ctx.domain_tags(seed, sweep)
        ref, rshift = o.domain_tags(sweep)
        assert (shift == rshift).all()
        assert (tags == ref).all()
        dropped += int(((plain.domain_tags(sweep)[0] >= 0) & (ref < 0)).sum())
    assert dropped > 0  # the rule did act


RAGGED = Melt("ragged_15x17x16_N8", (15, 17, 16), 1.05, 8, ell=4.0, seed=0xEC00B2,
              mode="domain", dir_mode="iso", sweeps=3, D=(3, 4, 3))


@pytest.mark.parametrize("lanes", [32, 16, 8, 4])
@pytest.mark.parametrize("prec", ["fp64", "fp32f"])
@pytest.mark.parametrize("m", [small_domain(seed=0xEC00B1), RAGGED], ids=lambda m: m.name)
def test_spring_domain_parity(m, prec, lanes):
    k = 30.0
    o = oracle_system(m, k_spring=k)
    res = o.run_domain(m.sweeps, m.ell, digests=True)
    assert res["rc"] == 0
    ctx = gpu_context(m, precision=PRECS[prec], lanes=lanes, k_spring=k)
    ctx.run(m.ell, seed=m.seed, n_sweeps=m.sweeps)
    nt = m.D[0] * m.D[1] * m.D[2]
    dig, lift, ev = ctx.records(m.sweeps * nt)
    assert (dig == res["digest"]).all(), np.nonzero(dig != res["digest"])[0][:5]
    assert (lift == res["ec_lift"]).all() and (ev == res["ec_events"]).all()
    assert_same_state(ctx, o)
    obs = assert_same_counts(ctx, res)
    assert obs["te_reflect"] > 0  # spring events with immotile partners


@pytest.mark.parametrize("prec", ["fp64", "fp32f"])
def test_soft_springs_stage_partners_beyond_the_halo(prec):
    """k = 0.5 kT/sigma^2 at packing fraction 0.32: bonds stretch to 2-3
    sigma, far past the tether halo (b_max = 1.2 sigma), so bonded beads
    must be staged from anywhere; 40 sweeps with two ECs per tile still
    match the oracle bit for bit."""
    m = small_domain(N=6, dims=(12, 12, 12), spacing=1.18, seed=0xEC00B3, ell=3.0, sweeps=40)
    k = 0.5
    o = oracle_system(m, k_spring=k, ecs_per_tile=2)
    res = o.run_domain(m.sweeps, m.ell, digests=True)
    assert res["rc"] == 0
    _, bonds = o.chain_obs()
    assert bonds.max() > 1.6 * m.b_max
    ctx = gpu_context(m, precision=PRECS[prec], lanes=8, k_spring=k, ecs_per_tile=2)
    ctx.run(m.ell, seed=m.seed, n_sweeps=m.sweeps)
    nt = m.D[0] * m.D[1] * m.D[2]
    dig, _, _ = ctx.records(m.sweeps * nt * 2)
    assert (dig == res["digest"]).all(), np.nonzero(dig != res["digest"])[0][:5]
    assert_same_state(ctx, o)
    obs = assert_same_counts(ctx, res)
    assert obs["bond_max"] > 1.6 * m.b_max
    assert obs["bond_mean"] == pytest.approx(float(bonds.mean()), rel=1e-12)


def test_springs_refuse_swaps_and_batch():
    m = small_domain()
    ctx = gpu_context(m)
    with pytest.raises(ecmc.EcmcError):
        ctx.configure(mode=ecmc.MODE_DOMAIN, dir_mode=ecmc.DIR_ISO, tiles=m.D, k_spring=30.0,
                      p_swap=0.5)
    with pytest.raises(ecmc.EcmcError):
        ctx.configure(mode=ecmc.MODE_DOMAIN, dir_mode=ecmc.DIR_ISO, tiles=m.D, k_spring=-1.0)
    ctx.configure(mode=ecmc.MODE_DOMAIN, dir_mode=ecmc.DIR_ISO, tiles=m.D, k_spring=30.0)
    b = ecmc.Batch([dict(dims=(12, 12, 12), spacing=1.05, N=8)], jitter=0.01, seed=1)
    with pytest.raises(ecmc.EcmcError):
        b.configure(dir_mode=ecmc.DIR_ISO, k_spring=30.0)
    b.close()


def test_springs_system_one_size_matches_oracle():
    """48,000 beads (400 chains x N = 120 at packing fraction 0.39, the size
    and density of the paper's System I) as a lattice melt, in the
    benchmark's springs setting (FP32 screen, 8 lanes, 4 ECs per tile,
    k = 30 kT/sigma^2, 4.4-sigma tiles): two sweeps against the oracle,
    event for event, with positions, images and counts."""
    a = (math.pi / (6.0 * 0.39)) ** (1.0 / 3.0)
    m = Melt("system_one_lattice", (40, 40, 30), a, 120, ell=10.0, seed=0xEC00D1, mode="domain",
             dir_mode="iso", sweeps=2, D=(10, 10, 7))
    o = oracle_system(m, k_spring=30.0, ecs_per_tile=4)
    res = o.run_domain(m.sweeps, m.ell, digests=True)
    assert res["rc"] == 0
    ctx = gpu_context(m, precision=ecmc.PREC_FP32F, lanes=8, k_spring=30.0, ecs_per_tile=4)
    ctx.run(m.ell, seed=m.seed, n_sweeps=m.sweeps)
    dig, _, _ = ctx.records(m.sweeps * 700 * 4)
    assert (dig == res["digest"]).all(), np.nonzero(dig != res["digest"])[0][:5]
    assert_same_state(ctx, o)
    assert_same_counts(ctx, res)
