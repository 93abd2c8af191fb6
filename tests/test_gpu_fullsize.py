"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times.

- The 10^6-bead melt (1000 chains of 1000 on 100^3, ell = 20, swaps
  proposed at contacts) in the benchmark's pinned launch setting
  (configs.C5_LAUNCH: 25^3 tiles, 8 lanes, 8 ECs per tile, cell side 1.05,
  8 tiles per block, first-pass capacity factor 1.0): one sweep on the GPU
  and in the oracle, every per-EC digest, lift sum and event count and every
  position and image counter identical.
- The 512k melt at phi = 0.50 (2000 chains of 256 on 80^3): the FP32-screened
  form reproduces the plain FP64 kernel's event sequence over 20 sweeps
  (identical digests, max |dr| = 0), and its first sweep matches the oracle.
"""
import numpy as np
import pytest

from paper_1502_06447_gb300 import ecmc
from paper_1502_06447_gb300.configs import C3, C5, C5_LAUNCH

from helpers import gpu_context, oracle_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1502_06447_gb300 import build
    build.build()


def _compare_sweep(m, tiles, lanes, ecs, p_swap, **launch):
    nt = tiles[0] * tiles[1] * tiles[2]
    o = oracle_system(m, D=tiles, ecs_per_tile=ecs, p_swap=p_swap)
    res = o.run_domain(1, m.ell, digests=True)
    assert res["rc"] == 0
    ctx = gpu_context(m, precision=ecmc.PREC_FP32F, lanes=lanes, tiles=tiles, ecs_per_tile=ecs,
                      p_swap=p_swap, **launch)
    ctx.run(m.ell, seed=m.seed, n_sweeps=1)
    dig, lift, ev = ctx.records(nt * ecs)
    assert (dig == res["digest"]).all(), np.nonzero(dig != res["digest"])[0][:5]
    assert (lift == res["ec_lift"]).all() and (ev == res["ec_events"]).all()
    r, img = ctx.get_positions()
    assert (r == o.r).all() and (img == o.img).all()
    return ctx, res


def test_million_bead_melt_one_sweep_matches_oracle():
    L = C5_LAUNCH
    ctx, res = _compare_sweep(C5, L["tiles"], L["lanes"], L["ecs_per_tile"], 0.05,
                              cell_side=L["cell_side"], block_tiles=L["block_tiles"],
                              tight_factor=L["tight_factor"])
    assert res["stats"]["swap_tried"] > 0
    obs = ctx.observables()
    assert obs["swap_tried"] == res["stats"]["swap_tried"] and obs["overlaps"] == 0


def test_phi_050_melt_fp32_screen_equals_fp64_over_20_sweeps():
    tiles = (20, 20, 20)
    nt = 20 ** 3
    runs = {}
    for prec in (ecmc.PREC_FP64, ecmc.PREC_FP32F):
        ctx = gpu_context(C3, precision=prec, lanes=16 if prec == ecmc.PREC_FP64 else 8,
                          tiles=tiles)
        digs = []
        for s in range(C3.sweeps):
            ctx.run(C3.ell, seed=C3.seed, n_sweeps=1)
            digs.append(ctx.records(nt)[0].copy())
        runs[prec] = (np.concatenate(digs), ctx.get_positions())
    d64, (r64, i64) = runs[ecmc.PREC_FP64]
    d32, (r32, i32) = runs[ecmc.PREC_FP32F]
    assert (d64 == d32).all()
    assert np.abs(r64 - r32).max() == 0.0 and (i64 == i32).all()
    _compare_sweep(C3, tiles, 8, 1, 0.0)
