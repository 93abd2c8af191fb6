"""Batched replicas: every replica must evolve exactly as a single melt with
the Philox key (seed, r) does in the oracle, event for event, with and
without the captured CUDA graph."""
import numpy as np
import pytest

import oracle
from paper_1502_06447_gb300 import ecmc
from paper_1502_06447_gb300.configs import replica_specs

pytestmark = pytest.mark.gpu

SEED = 0xEC0B01
JITTER = 0.01


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1502_06447_gb300 import build
    build.build()


def ragged_specs():
    # uneven N, bead counts, spacings (phi from 0.36 to 0.45)
    return [dict(dims=(12, 12, 12), spacing=1.05, N=8), dict(dims=(10, 12, 14), spacing=1.12, N=10),
            dict(dims=(16, 12, 10), spacing=1.18, N=20), dict(dims=(12, 14, 12), spacing=1.08, N=1),
            dict(dims=(14, 14, 14), spacing=1.15, N=7)]


def oracle_replica(sp, r, tiles, ell, sweeps, p_swap=0.0, jitter=JITTER):
    L = tuple(d * sp["spacing"] for d in sp["dims"])
    o = oracle.System(oracle.lattice(sp["dims"], sp["spacing"], jitter, SEED, replica=r), L,
                      sp["N"], mode=oracle.MODE_DOMAIN, dir_mode=oracle.DIR_ISO, D=tiles,
                      seed=SEED, replica=r, p_swap=p_swap)
    res = o.run_domain(sweeps, ell, digests=True)
    assert res["rc"] == 0
    return o, res


def check_batch(specs, lanes, prec, graph, sweeps=3, ell=3.0, p_swap=0.0, jitter=JITTER,
                schedule=0, **kw):
    b = ecmc.Batch(specs, jitter=jitter, seed=SEED)
    b.configure(dir_mode=ecmc.DIR_ISO, precision=prec, lanes=lanes, record=1, p_swap=p_swap,
                schedule=schedule, **kw)
    b.run(ell, seed=SEED, n_sweeps=sweeps, graph=graph)
    units = sum(int(np.prod(b.info(r)[0])) for r in range(len(specs)))
    dig, _, _ = b.records(sweeps * units)
    for r, sp in enumerate(specs):
        tiles, off, nb = b.info(r)
        nt = int(np.prod(tiles))
        o, res = oracle_replica(sp, r, tiles, ell, sweeps, p_swap, jitter)
        mine = np.concatenate([dig[s * units + off: s * units + off + nt] for s in range(sweeps)])
        assert (mine == res["digest"]).all(), (r, np.nonzero(mine != res["digest"])[0][:5])
        x, img = b.get_positions(r)
        assert (x == o.r).all() and (img == o.img).all(), r
    return b


@pytest.mark.parametrize("graph", [True, False])
@pytest.mark.parametrize("lanes,prec,schedule", [(8, ecmc.PREC_FP32F, 0), (16, ecmc.PREC_FP32F, 0),
                                                 (4, ecmc.PREC_FP32F, 0), (8, ecmc.PREC_FP32F, 1),
                                                 (32, ecmc.PREC_FP64, 0)])
def test_batch_replicas_match_oracle(lanes, prec, schedule, graph):
    check_batch(ragged_specs(), lanes, prec, graph, schedule=schedule)


@pytest.mark.parametrize("schedule", [0, 1])
def test_batch_swap_matches_oracle(schedule):
    # the N = 1 replica accepts every swap, the chains almost none
    check_batch(ragged_specs()[:4], 8, ecmc.PREC_FP32F, True, p_swap=0.5, ell=5.0,
                schedule=schedule)


@pytest.mark.parametrize("lanes", [8, 4])
def test_batch_exhaustive_evaluation_matches_oracle(lanes):
    # one request per tile: most steps take the exhaustive FP64 evaluation
    check_batch(ragged_specs(), lanes, ecmc.PREC_FP32F, True, sweeps=2, request_cap=1)


def test_batch_c4_replicas_sample():
    """The first replicas of the 256-replica workload (N in {10..160},
    2k-64k beads, phi in [0.35, 0.50]) against the oracle, two sweeps."""
    ms = replica_specs()[:6]
    specs = [dict(dims=m.dims, spacing=m.spacing, N=m.N) for m in ms]
    check_batch(specs, 8, ecmc.PREC_FP32F, True, sweeps=2, ell=5.0, jitter=ms[0].jitter)


def test_batch_graph_equals_plain_launches():
    specs = ragged_specs()
    a = ecmc.Batch(specs, jitter=JITTER, seed=SEED)
    a.configure(dir_mode=ecmc.DIR_ISO, precision=ecmc.PREC_FP32F, lanes=8)
    a.run(3.0, seed=SEED, n_sweeps=4, graph=True)
    c = ecmc.Batch(specs, jitter=JITTER, seed=SEED)
    c.configure(dir_mode=ecmc.DIR_ISO, precision=ecmc.PREC_FP32F, lanes=8)
    c.run(3.0, seed=SEED, n_sweeps=1, graph=False)
    c.run(3.0, seed=SEED, n_sweeps=3, graph=True)
    for r in range(len(specs)):
        assert (a.get_positions(r)[0] == c.get_positions(r)[0]).all()
    assert a.stats()["events_total"] == c.stats()["events_total"]


def test_batch_full_256_replicas_sampled():
    """The whole 256-replica workload (4.7 M beads) in the batch, in the
    launch setting the benchmark's tuner picks for it (8 lanes, 3.4-sigma
    tiles, 8 ECs per tile, 8 tiles per block, first-pass factor 1.16), one
    graph-replayed sweep after one plain sweep; every 32nd replica and the
    largest one against the oracle, event for event, with their positions
    and images."""
    ms = replica_specs()
    specs = [dict(dims=m.dims, spacing=m.spacing, N=m.N) for m in ms]
    ell, jitter = ms[0].ell, ms[0].jitter
    b = ecmc.Batch(specs, jitter=jitter, seed=SEED)
    b.configure(dir_mode=ecmc.DIR_ISO, precision=ecmc.PREC_FP32F, lanes=8, tile_side=3.4,
                ecs_per_tile=8, block_tiles=8, tight_factor=1.16, record=1)
    sweeps = 2
    b.run(ell, seed=SEED, n_sweeps=1, graph=False)
    b.run(ell, seed=SEED, n_sweeps=1, graph=True)
    units = sum(int(np.prod(b.info(r)[0])) for r in range(len(specs)))
    dig, _, _ = b.records(units * 8)
    assert len(dig) == units * 8  # the records of the last run (one sweep)
    sample = sorted(set(range(0, len(ms), 32)) | {int(np.argmax([m.n for m in ms]))})
    for r in sample:
        sp = specs[r]
        tiles, off, nb = b.info(r)
        nt = int(np.prod(tiles))
        L = tuple(d * sp["spacing"] for d in sp["dims"])
        o = oracle.System(oracle.lattice(sp["dims"], sp["spacing"], jitter, SEED, replica=r), L,
                          sp["N"], mode=oracle.MODE_DOMAIN, dir_mode=oracle.DIR_ISO, D=tiles,
                          seed=SEED, replica=r, ecs_per_tile=8)
        o.run_domain(1, ell)
        res = o.run_domain(1, ell, sweep0=1, digests=True)
        assert res["rc"] == 0
        mine = dig[off * 8: (off + nt) * 8]
        assert (mine == res["digest"]).all(), (r, np.nonzero(mine != res["digest"])[0][:5])
        x, img = b.get_positions(r)
        assert (x == o.r).all() and (img == o.img).all(), r
    b.close()
