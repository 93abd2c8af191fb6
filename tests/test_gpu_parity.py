"""Parity of the CUDA library with the oracle (element by element, same seeds).

Integer and event data must match exactly; positions are compared bit for bit
(both sides evaluate every FP64 expression as written, IEEE, no FMA), and the
FP32-screened form must reproduce the plain FP64 event sequence exactly.
"""
import numpy as np
import pytest

import oracle
from paper_1502_06447_gb300 import ecmc
from paper_1502_06447_gb300.configs import C1, C2, Melt, small_domain

from helpers import gpu_context, oracle_system

pytestmark = pytest.mark.gpu

PRECS = {"fp64": ecmc.PREC_FP64, "fp32f": ecmc.PREC_FP32F}


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1502_06447_gb300 import build
    build.build()


def counters(st):
    return {k: st[k] for k in oracle.OUT_NAMES}


def assert_same_state(gpu, orc):
    r, img = gpu.get_positions()
    bad = np.nonzero((r != orc.r).any(1))[0]
    assert bad.size == 0, f"{bad.size} beads differ, first {bad[:5]}: {r[bad[:3]]} vs {orc.r[bad[:3]]}"
    assert (img == orc.img).all()


# ------------------------------------------------------------------ lattice
@pytest.mark.parametrize("m", [C1, C2], ids=lambda m: m.name)
def test_lattice_matches_oracle(m):
    ctx = ecmc.Context.create_lattice(m.dims, m.spacing, m.N, jitter=m.jitter, seed=m.seed)
    r, img = ctx.get_positions()
    ref = oracle.lattice(m.dims, m.spacing, m.jitter, m.seed)
    assert (r == ref).all() and (img == 0).all()


# ------------------------------------------------------------------ serial C1
@pytest.fixture(scope="module")
def c1_oracle():
    o = oracle_system(C1)
    res = o.run_serial(C1.n_ec, C1.ell, digests=True)
    assert res["rc"] == 0
    return o, res


@pytest.mark.parametrize("prec", ["fp64", "fp32f"])
def test_serial_c1_full_run(c1_oracle, prec):
    """C1: 64 chains x N=10, 1e5 serial ECs, ell = 5, v in {+x,+y,+z}:
    identical per-EC digests, lift sums and event counts, identical final
    positions and images."""
    o, res = c1_oracle
    ctx = gpu_context(C1, precision=PRECS[prec])
    ctx.run(C1.ell, chains_per_sweep=C1.n_ec, seed=C1.seed)
    dig, lift, ev = ctx.records(C1.n_ec)
    first = np.nonzero(dig != res["digest"])[0]
    assert first.size == 0, f"first differing EC {first[:3]}"
    assert (ev == res["ec_events"]).all()
    assert (lift == res["ec_lift"]).all()
    assert_same_state(ctx, o)
    obs = ctx.observables()
    for k, v in counters(res["stats"]).items():
        assert obs[k] == v, k
    assert obs["events_total"] == res["stats"]["events"]
    assert obs["overlaps"] == 0 and obs["tether_violations"] == 0


def test_serial_event_log_matches_oracle():
    """Event by event (pivot, outcome, partner, x) over the first 200 ECs."""
    o = oracle_system(C1)
    res = o.run_serial(200, C1.ell, log_cap=100000)
    ctx = gpu_context(C1)
    ctx.log_reserve(100000)
    ctx.run(C1.ell, chains_per_sweep=200, seed=C1.seed)
    log = ctx.event_log(100000)
    ref = res["log"]
    assert len(log) == len(ref)
    for f in ("unit", "pivot", "kind", "partner"):
        assert (log[f] == ref[f]).all(), f
    assert (log["x"] == ref["x"]).all()


# ------------------------------------------------------------------ domain
@pytest.mark.parametrize("m", [small_domain(), C2], ids=lambda m: m.name)
def test_domain_tags_match_oracle(m):
    ctx = gpu_context(m)
    o = oracle_system(m)
    for sweep in (0, 7):
        tags, shift = ctx.domain_tags(m.seed, sweep)
        ref, rshift = o.domain_tags(sweep)
        assert (shift == rshift).all()
        assert (tags == ref).all()


RAGGED = Melt("ragged_15x17x16_N8", (15, 17, 16), 1.05, 8, ell=4.0, seed=0xEC00A2,
              mode="domain", dir_mode="iso", sweeps=3, D=(3, 4, 3))


@pytest.mark.parametrize("schedule", [0, 1])
@pytest.mark.parametrize("lanes", [32, 16, 8, 4])
@pytest.mark.parametrize("prec", ["fp64", "fp32f"])
@pytest.mark.parametrize("m", [small_domain(), RAGGED], ids=lambda m: m.name)
def test_domain_parity_small(m, prec, lanes, schedule):
    """schedule 0 runs the screened form with 4-16 lanes in the block-lockstep
    kernel, schedule 1 in the warp-lockstep kernel; other settings ignore it."""
    if schedule == 1 and not (prec == "fp32f" and lanes in (4, 8, 16)):
        pytest.skip("schedule only selects among screened 4/8/16-lane kernels")
    o = oracle_system(m)
    res = o.run_domain(m.sweeps, m.ell, digests=True)
    assert res["rc"] == 0
    ctx = gpu_context(m, precision=PRECS[prec], lanes=lanes, schedule=schedule)
    ctx.run(m.ell, seed=m.seed, n_sweeps=m.sweeps)
    nt = m.D[0] * m.D[1] * m.D[2]
    dig, lift, ev = ctx.records(m.sweeps * nt)
    assert (dig == res["digest"]).all(), np.nonzero(dig != res["digest"])[0][:5]
    assert (lift == res["ec_lift"]).all()
    assert (ev == res["ec_events"]).all()
    assert_same_state(ctx, o)
    obs = ctx.observables()
    for k, v in counters(res["stats"]).items():
        assert obs[k] == v, k


@pytest.mark.parametrize("lanes,schedule", [(32, 0), (8, 0), (8, 1), (16, 0)])
def test_domain_two_ecs_per_tile(lanes, schedule):
    m = small_domain(seed=0xEC00A3)
    o = oracle_system(m, ecs_per_tile=2)
    res = o.run_domain(2, m.ell, digests=True)
    ctx = gpu_context(m, ecs_per_tile=2, lanes=lanes, precision=ecmc.PREC_FP32F,
                      schedule=schedule)
    ctx.run(m.ell, seed=m.seed, n_sweeps=2)
    dig, _, _ = ctx.records(2 * 27 * 2)
    assert (dig == res["digest"]).all()
    assert_same_state(ctx, o)


# 252 tiles of side 4.2: 32 of them fit one block's shared memory, and no
# block size divides 252
BLOCKS = Melt("blocks_24x24x28_N8", (24, 24, 28), 1.05, 8, ell=4.0, seed=0xEC00A6, mode="domain",
              dir_mode="iso", sweeps=2, D=(6, 6, 7))


@pytest.mark.parametrize("lanes,block_tiles", [(8, 4), (8, 8), (8, 16), (4, 8), (4, 32), (16, 2),
                                               (16, 8)])
def test_block_lockstep_block_sizes(lanes, block_tiles):
    """Every block size of the block-lockstep kernel (tiles per block from
    32 / lanes up to 128 threads, full and ragged last blocks) gives the
    oracle's events."""
    m = BLOCKS
    o = oracle_system(m)
    res = o.run_domain(m.sweeps, m.ell, digests=True)
    ctx = gpu_context(m, precision=ecmc.PREC_FP32F, lanes=lanes, block_tiles=block_tiles)
    ctx.run(m.ell, seed=m.seed, n_sweeps=m.sweeps)
    nt = m.D[0] * m.D[1] * m.D[2]
    dig, _, _ = ctx.records(m.sweeps * nt)
    assert (dig == res["digest"]).all()
    assert_same_state(ctx, o)


@pytest.mark.parametrize("lanes,request_cap", [(8, 1), (4, 1), (16, 1), (8, 2), (4, 3)])
def test_block_lockstep_exhaustive_evaluation(lanes, request_cap):
    """Request lists of 1-3 entries per tile (screening lists of 24-72 slots):
    with one, most tile steps take the exhaustive FP64 evaluation by the
    tile's own lanes; the events are still the oracle's."""
    m = BLOCKS
    o = oracle_system(m)
    res = o.run_domain(m.sweeps, m.ell, digests=True)
    ctx = gpu_context(m, precision=ecmc.PREC_FP32F, lanes=lanes, request_cap=request_cap)
    ctx.run(m.ell, seed=m.seed, n_sweeps=m.sweeps)
    nt = m.D[0] * m.D[1] * m.D[2]
    dig, _, _ = ctx.records(m.sweeps * nt)
    assert (dig == res["digest"]).all()
    assert_same_state(ctx, o)
    if request_cap == 1:  # 24 slots hold fewer than the 27 cells around most pivots
        ob = ctx.observables()
        assert ob["exhaustive"] > ob["events_total"] // 4


def test_exhaustive_evaluation_is_rare_by_default():
    """With the default request list the exhaustive evaluation is a rare
    path of the block-lockstep kernel, and the other kernels never take it."""
    m = BLOCKS
    ctx = gpu_context(m, precision=ecmc.PREC_FP32F, lanes=8)
    ctx.run(m.ell, seed=m.seed, n_sweeps=m.sweeps)
    ob = ctx.observables()
    assert ob["exhaustive"] < 1e-3 * ob["events_total"]
    ctx64 = gpu_context(m, precision=ecmc.PREC_FP64, lanes=8)
    ctx64.run(m.ell, seed=m.seed, n_sweeps=1)
    assert ctx64.observables()["exhaustive"] == 0


@pytest.fixture(scope="module")
def c2_oracle():
    o = oracle_system(C2)
    res = o.run_domain(3, C2.ell, digests=True)
    return o, res


@pytest.mark.parametrize("lanes", [32, 16, 8, 4])
@pytest.mark.parametrize("prec", ["fp64", "fp32f"])
def test_domain_parity_c2_full_size(c2_oracle, prec, lanes):
    """C2 at full size (4096 x 64 beads, 16^3 tiles): three sweeps identical."""
    o, res = c2_oracle
    ctx = gpu_context(C2, precision=PRECS[prec], lanes=lanes)
    ctx.run(C2.ell, seed=C2.seed, n_sweeps=3)
    dig, lift, ev = ctx.records(3 * 4096)
    assert (dig == res["digest"]).all(), np.nonzero(dig != res["digest"])[0][:5]
    assert (ev == res["ec_events"]).all()
    assert_same_state(ctx, o)


def test_run_split_equals_one_run():
    """Counter-based random numbers: 2 + 1 sweeps equal 3 sweeps."""
    m = small_domain()
    a = gpu_context(m, record=0)
    a.run(m.ell, seed=m.seed, n_sweeps=3)
    b = gpu_context(m, record=0)
    b.run(m.ell, seed=m.seed, n_sweeps=2)
    b.run(m.ell, seed=m.seed, n_sweeps=1)
    ra, ia = a.get_positions()
    rb, ib = b.get_positions()
    assert (ra == rb).all() and (ia == ib).all()


# ------------------------------------------------------------------ swap
@pytest.mark.parametrize("lanes,schedule", [(32, 0), (8, 0), (8, 1), (4, 0)])
@pytest.mark.parametrize("p_swap,N", [(0.5, 8), (1.0, 8), (1.0, 2), (0.5, 1)])
def test_swap_parity_domain(p_swap, N, lanes, schedule):
    """Swaps in the domain mode.  In the 8-bead chains every proposal is
    rejected (exchanging two touching beads over-stretches a tether), so
    dimers (about one in six accepted) and free spheres (all accepted) carry
    the accept branch."""
    m = small_domain(N=N, p_swap=p_swap, seed=0xEC00A4, ell=6.0)
    o = oracle_system(m)
    res = o.run_domain(3, m.ell, digests=True)
    ctx = gpu_context(m, lanes=lanes, precision=ecmc.PREC_FP32F, schedule=schedule)
    ctx.run(m.ell, seed=m.seed, n_sweeps=3)
    dig, _, _ = ctx.records(3 * 27)
    assert (dig == res["digest"]).all()
    assert_same_state(ctx, o)
    obs = ctx.observables()
    assert obs["swap_tried"] == res["stats"]["swap_tried"]
    assert obs["swap"] == res["stats"]["swap"]


def test_swap_parity_serial():
    m = Melt("serial_swap", (8, 8, 8), 1.05, 8, ell=3.0, seed=0xEC00A5, mode="serial",
             dir_mode="iso", p_swap=1.0)
    o = oracle_system(m)
    res = o.run_serial(3000, m.ell, digests=True)
    ctx = gpu_context(m, precision=ecmc.PREC_FP32F)
    ctx.run(m.ell, chains_per_sweep=3000, seed=m.seed)
    dig, _, _ = ctx.records(3000)
    assert (dig == res["digest"]).all()
    assert_same_state(ctx, o)


def test_swap_calibration_reaches_the_target_rate():
    """ecmc_swap sets p_swap from the contacts of the last ecmc_run, so the
    attempts per bead and sweep that follow match the target on a melted
    state, whatever the earlier (lattice-start) sweeps counted."""
    m = small_domain(seed=0xEC00A6, ell=6.0)
    ctx = gpu_context(m, lanes=8, precision=ecmc.PREC_FP32F, ecs_per_tile=4)
    with pytest.raises(ecmc.EcmcError):
        ctx.swap(0.1)  # no run yet
    ctx.run(m.ell, seed=m.seed, n_sweeps=20)  # melts the lattice start
    ctx.run(m.ell, seed=m.seed, n_sweeps=4)  # the calibration run
    ctx.swap(0.1)
    t0 = ctx.observables()["swap_tried"]
    ctx.run(m.ell, seed=m.seed, n_sweeps=12)
    n = ctx.observables()["n_beads"]
    rate = (ctx.observables()["swap_tried"] - t0) / (n * 12)
    assert rate == pytest.approx(0.1, rel=0.15)


# ------------------------------------------------------------------ observables
def test_observables_match_oracle():
    m = small_domain()
    o = oracle_system(m)
    ref0 = o.unwrapped()[np.arange(o.r.shape[0] // m.N) * m.N + m.N // 2].copy()
    o.run_domain(4, m.ell)
    ctx = gpu_context(m)
    ctx.g1_reset()
    ctx.run(m.ell, seed=m.seed, n_sweeps=4)
    obs = ctx.observables()
    re2, bonds = o.chain_obs()
    assert abs(obs["re2_mean"] - re2.mean()) <= 1e-12 * re2.mean()
    assert obs["bond_max"] == bonds.max() and obs["bond_min"] == bonds.min()
    dmin, nov = o.min_pair()
    assert obs["overlaps"] == nov == 0
    mid = o.unwrapped()[np.arange(o.r.shape[0] // m.N) * m.N + m.N // 2]
    g1 = ((mid - ref0) ** 2).sum(1).mean()
    assert abs(obs["g1"] - g1) <= 1e-12 * max(g1, 1.0)
    assert abs(obs["disp_sum"] - obs["ecs"] * m.ell) < 1e-9 * obs["ecs"] * m.ell
    pairs, bonds = o.contacts(obs["contact_delta"])
    assert obs["contact_delta"] == 0.02
    assert tuple(obs["contact_pairs"]) == tuple(pairs) and tuple(obs["taut_bonds"]) == tuple(bonds)
    assert bonds.sum() > 0 and pairs.sum() > 0
    assert abs(obs["pressure_contact"] - o.contact_pressure(0.02)) <= 1e-12 * abs(obs["pressure_contact"])


@pytest.mark.parametrize("lanes", [8, 32])
def test_contact_pressure_domain_mode_hard_spheres(lanes):
    """Unbonded hard spheres at phi = 0.30 run in the domain mode: the
    contact-value pressure of the sampled states matches Carnahan-Starling
    (within 3 standard errors plus 1.5 % for CS, 1000-sphere finite size and
    the shell extrapolation), while the lift-distance estimator, which misses
    the momentum carried by reflections at joint beads and tile walls, comes
    out far below it."""
    import math
    phi = 0.30
    a = (math.pi / (6 * phi)) ** (1 / 3)
    ctx = ecmc.Context.create_lattice((10, 10, 10), a, 1, jitter=0.05, seed=12)
    ctx.configure(mode=ecmc.MODE_DOMAIN, dir_mode=ecmc.DIR_ISO, precision=ecmc.PREC_FP32F,
                  tiles=(3, 3, 3), lanes=lanes, ecs_per_tile=4)
    ctx.run(3.0, seed=12, n_sweeps=300)
    o0 = ctx.observables()
    zc = []
    for _ in range(120):
        ctx.run(3.0, seed=12, n_sweeps=15)
        zc.append(ctx.observables()["pressure_contact"])
    o1 = ctx.observables()
    zc = np.array(zc)
    zcs = (1 + phi + phi ** 2 - phi ** 3) / (1 - phi) ** 3
    se = zc.std(ddof=1) / math.sqrt(len(zc))
    assert abs(zc.mean() - zcs) < 3 * se + 0.015 * zcs, (zc.mean(), se, zcs)
    z_lift = 1 + (o1["lift_sum"] - o0["lift_sum"]) / (o1["disp_sum"] - o0["disp_sum"])
    assert z_lift < 0.8 * zcs
    assert o1["overlaps"] == 0


# ------------------------------------------------------------------ checkpoint
def test_checkpoint_resume_is_bit_identical(tmp_path):
    m = small_domain()
    a = gpu_context(m, record=0)
    a.run(m.ell, seed=m.seed, n_sweeps=2)
    a.checkpoint(tmp_path / "ck.bin")
    a.run(m.ell, seed=m.seed, n_sweeps=2)
    b = gpu_context(m, record=0)
    b.restore(tmp_path / "ck.bin")
    b.run(m.ell, seed=m.seed, n_sweeps=2)
    ra, ia = a.get_positions()
    rb, ib = b.get_positions()
    assert (ra == rb).all() and (ia == ib).all()
    raw = bytearray((tmp_path / "ck.bin").read_bytes())
    raw[200] ^= 0xFF
    (tmp_path / "bad.bin").write_bytes(bytes(raw))
    with pytest.raises(ecmc.EcmcError) as e:
        b.restore(tmp_path / "bad.bin")
    assert e.value.code == -7


# ------------------------------------------------------------------ errors
def test_invalid_arguments_and_states():
    with pytest.raises(ecmc.EcmcError) as e:
        ecmc.Context.create_lattice((8, 8, 10), 0.9, 10)  # spacing < sigma
    assert e.value.code == -1
    ctx = ecmc.Context.create_lattice((8, 8, 8), 1.05, 8)
    r, _ = ctx.get_positions()
    bad = r.copy()
    bad[1] = bad[0] + np.array([0.5, 0, 0])
    with pytest.raises(ecmc.EcmcError) as e:
        ctx.set_positions(bad)
    assert e.value.code == -4
    bad = r.copy()
    bad[1] = bad[0] + np.array([0.0, 0, 1.5]) + 0.0
    bad[2] = bad[0] + np.array([3.0, 3.0, 3.0])
    with pytest.raises(ecmc.EcmcError) as e:
        ctx.set_positions(bad)
    assert e.value.code in (-4, -5)
    bad = r.copy()
    bad[3, 1] = np.nan
    with pytest.raises(ecmc.EcmcError) as e:
        ctx.set_positions(bad)
    assert e.value.code == -1
    # positions given outside the box come back wrapped, whole boxes in the
    # image counters (which start from the given ones)
    L = ctx.L
    shift = np.array([1, -2, 3])
    img0 = np.tile(np.array([5, 0, -1], dtype=np.int32), (len(r), 1))
    ctx.set_positions(r + shift * L, img0)
    r2, img2 = ctx.get_positions()
    assert np.abs(r2 - r).max() < 1e-9 * L.max()
    assert (img2 == img0 + shift).all()
    out = (np.empty_like(r2), np.empty_like(img2))
    got = ctx.get_positions(out=out)
    assert got[0] is out[0] and (out[0] == r2).all() and (out[1] == img2).all()
    with pytest.raises(ecmc.EcmcError) as e:
        ctx.configure(mode=ecmc.MODE_DOMAIN, tiles=(2, 3, 3))
    assert e.value.code == -1
    with pytest.raises(ecmc.EcmcError):
        ctx.run(1.0, chains_per_sweep=1)  # not configured after the failure
    for lanes, bt in ((8, 32), (16, 16), (8, 6)):  # > 128 threads, or not whole warps
        with pytest.raises(ecmc.EcmcError) as e:
            ctx.configure(mode=ecmc.MODE_DOMAIN, tiles=(3, 3, 3), precision=ecmc.PREC_FP32F,
                          lanes=lanes, block_tiles=bt)
        assert e.value.code == -1
    for rc in (-1, 7):
        with pytest.raises(ecmc.EcmcError) as e:
            ctx.configure(mode=ecmc.MODE_DOMAIN, tiles=(3, 3, 3), precision=ecmc.PREC_FP32F,
                          lanes=8, request_cap=rc)
        assert e.value.code == -1


def test_event_cap_and_stage_capacity_report_errors():
    m = small_domain()
    ctx = gpu_context(m, event_cap=3)
    with pytest.raises(ecmc.EcmcError) as e:
        ctx.run(m.ell, seed=m.seed, n_sweeps=1)
    assert e.value.code == -6
    ctx = gpu_context(m, stage_cap=32)
    with pytest.raises(ecmc.EcmcError) as e:
        ctx.run(m.ell, seed=m.seed, n_sweeps=1)
    assert e.value.code == -8
