"""Autotuner: it must leave the state exactly as it found it, pick an
admissible setting, and a run under the chosen setting must still match the
oracle event for event (with the chosen tiles and ECs per tile)."""
import numpy as np
import pytest

import oracle
from paper_1502_06447_gb300 import ecmc
from paper_1502_06447_gb300.configs import Melt

from helpers import gpu_context, oracle_system

pytestmark = pytest.mark.gpu

SEED = 0xEC0A70


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1502_06447_gb300 import build
    build.build()


def melt():
    # 24^3 sites: tile sides 3.4 .. 7 sigma all give >= 3 tiles per axis
    return Melt("tune_24", (24, 24, 24), 1.05, 12, ell=4.0, seed=SEED, mode="domain",
                dir_mode="iso", sweeps=2, D=(6, 6, 6))


def test_autotune_restores_state_and_keeps_parity():
    m = melt()
    ctx = gpu_context(m, precision=ecmc.PREC_FP32F, lanes=8)
    ctx.run(m.ell, seed=m.seed, n_sweeps=1)
    r0, i0 = ctx.get_positions()
    ob0 = ctx.observables()
    t = ctx.autotune(m.ell, seed=m.seed, trial_sweeps=1)
    assert t["n_trials"] >= 8 and t["ecs_per_s"] > 0
    assert t["lanes"] in (4, 8, 16, 32) and t["ecs_per_tile"] in (1, 2, 4)
    assert all(d >= 3 for d in t["tiles"])
    r1, i1 = ctx.get_positions()
    assert (r1 == r0).all() and (i1 == i0).all()
    ob1 = ctx.observables()
    for k in ("events_total", "ecs", "sweeps", "lift_sum", "disp_sum", "device_seconds"):
        assert ob1[k] == ob0[k], k
    # the oracle: sweep 0 with the original tiles, sweep 1 with the chosen ones
    o = oracle_system(m)
    assert o.run_domain(1, m.ell)["rc"] == 0
    assert (o.r == r0).all()
    o2 = oracle_system(m, D=t["tiles"], ecs_per_tile=t["ecs_per_tile"])
    o2.r[:], o2.img[:] = o.r, o.img
    res = o2.run_domain(1, m.ell, sweep0=1, digests=True)
    assert res["rc"] == 0
    ctx.configure(mode=ecmc.MODE_DOMAIN, dir_mode=ecmc.DIR_ISO, precision=ecmc.PREC_FP32F,
                  tiles=t["tiles"], lanes=t["lanes"], ecs_per_tile=t["ecs_per_tile"],
                  cell_side=t["cell_side"], record=1)
    ctx.run(m.ell, seed=m.seed, n_sweeps=1)
    dig, _, _ = ctx.records(len(res["digest"]))
    assert (dig == res["digest"]).all()
    r2, i2 = ctx.get_positions()
    assert (r2 == o2.r).all() and (i2 == o2.img).all()


def test_batch_autotune_restores_state_and_keeps_parity():
    specs = [dict(dims=(12, 12, 12), spacing=1.05, N=8), dict(dims=(10, 12, 14), spacing=1.12, N=10),
             dict(dims=(16, 12, 10), spacing=1.18, N=20)]
    b = ecmc.Batch(specs, jitter=0.01, seed=SEED)
    b.configure(dir_mode=ecmc.DIR_ISO, precision=ecmc.PREC_FP32F, lanes=8)
    before = [b.get_positions(r) for r in range(len(specs))]
    st0 = b.stats()
    t = b.autotune(3.0, seed=SEED, trial_sweeps=1)
    assert t["n_trials"] >= 4
    for r in range(len(specs)):
        x, img = b.get_positions(r)
        assert (x == before[r][0]).all() and (img == before[r][1]).all()
    assert b.stats() == st0
    # run two sweeps under the winner with records and check every replica
    b.configure(dir_mode=ecmc.DIR_ISO, precision=ecmc.PREC_FP32F, lanes=t["lanes"],
                tile_side=t["tile_side"], cell_side=t["cell_side"],
                ecs_per_tile=t["ecs_per_tile"], record=1)
    b.run(3.0, seed=SEED, n_sweeps=2, graph=True)
    k = t["ecs_per_tile"]
    units = sum(int(np.prod(b.info(r)[0])) for r in range(len(specs)))
    dig, _, _ = b.records(2 * units * k)
    for r, sp in enumerate(specs):
        tiles, off, _ = b.info(r)
        nt = int(np.prod(tiles))
        L = tuple(d * sp["spacing"] for d in sp["dims"])
        o = oracle.System(oracle.lattice(sp["dims"], sp["spacing"], 0.01, SEED, replica=r), L,
                          sp["N"], mode=oracle.MODE_DOMAIN, dir_mode=oracle.DIR_ISO, D=tiles,
                          seed=SEED, replica=r, ecs_per_tile=k)
        res = o.run_domain(2, 3.0, digests=True)
        assert res["rc"] == 0
        mine = np.concatenate([dig[(s * units + off) * k:(s * units + off + nt) * k]
                               for s in range(2)])
        assert (mine == res["digest"]).all(), r
        x, img = b.get_positions(r)
        assert (x == o.r).all() and (img == o.img).all(), r
