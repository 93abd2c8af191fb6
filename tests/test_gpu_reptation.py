"""The paper's reptation workload on the GPU against the oracle (Sec. IV.B,
Fig. 6): M = 20 chains of N = 500 hard-sphere beads with tethers of
1.4 sigma at packing fraction 0.298, built as the paper builds its melts
(phantom chains, slow push-off, Sec. II.B), then domain sweeps of the
FP32-screened kernel with the middle bead's g1 (Sec. IV, Eq. 3) tracked on
the device over log-spaced lags.

The oracle pushes the same phantom chains off and runs the same sweeps one
at a time, keeping the unwrapped middle beads after every sweep; its g1
table is the plain average of Eq. 3 over the same origins.  Push-off sweep
count and positions, per-EC digests of the EC sweeps, final positions and
the g1 table (sums over chains and origins, hence g1 itself) must be equal
bit for bit."""
import math

import numpy as np
import pytest

import oracle
from paper_1502_06447_gb300 import ecmc

pytestmark = pytest.mark.gpu

M, N, ETA, B_MAX = 20, 500, 0.298, 1.4
L = (M * N * math.pi / (6.0 * ETA)) ** (1.0 / 3.0)
TILES = (6, 6, 6)
PO_SEED, RUN_SEED, ELL, ECS = 72, 73, 10.0, 2
P, K, SWEEPS, CHUNK = 4, 4, 120, 20


def test_reptation_melt_and_g1_table_match_oracle():
    from paper_1502_06447_gb300 import build
    build.build()
    box = (L, L, L)
    r, img = oracle.phantom_chains(box, M, N, bond=1.0, c=1.9, seed=71)
    po = oracle.System(r, box, N, sigma=1.0, b_max=B_MAX, mode=oracle.MODE_DOMAIN,
                       dir_mode=oracle.DIR_ISO, D=TILES, seed=PO_SEED, img=img)
    rc, po_sweeps, _ = po.pushoff(0.5, 5, 2.0, 20000)
    assert rc == 0

    ctx = ecmc.Context.create_phantom(box, M, N, bond=1.0, c=1.9, seed=71, b_max=B_MAX)
    ctx.configure(mode=ecmc.MODE_DOMAIN, dir_mode=ecmc.DIR_ISO, precision=ecmc.PREC_FP64,
                  tiles=TILES, lanes=8)
    assert ctx.pushoff(f0=0.5, stages=5, ell=2.0, seed=PO_SEED, max_sweeps=20000) == po_sweeps
    rg, ig = ctx.get_positions()
    assert (rg == po.r).all() and (ig == po.img).all()

    ctx.configure(mode=ecmc.MODE_DOMAIN, dir_mode=ecmc.DIR_ISO, precision=ecmc.PREC_FP32F,
                  tiles=TILES, lanes=8, ecs_per_tile=ECS, record=1)
    ctx.g1_track(P, K)
    o = oracle.System(po.r, box, N, sigma=1.0, b_max=B_MAX, mode=oracle.MODE_DOMAIN,
                      dir_mode=oracle.DIR_ISO, D=TILES, seed=RUN_SEED, img=po.img,
                      ecs_per_tile=ECS)
    mid = lambda s: s.unwrapped().reshape(M, N, 3)[:, N // 2].copy()
    traj = [mid(o)]
    nt = TILES[0] * TILES[1] * TILES[2]
    for c0 in range(0, SWEEPS, CHUNK):
        ctx.run(ELL, seed=RUN_SEED, n_sweeps=CHUNK)
        dig, _, _ = ctx.records(CHUNK * nt * ECS)
        ref = []
        for s in range(CHUNK):
            res = o.run_domain(1, ELL, sweep0=po_sweeps + c0 + s, digests=True)
            assert res["rc"] == 0
            ref.append(res["digest"])
            traj.append(mid(o))
        ref = np.concatenate(ref)
        assert (dig == ref).all(), f"digests differ in sweeps {c0}..{c0 + CHUNK}"
    rg, ig = ctx.get_positions()
    assert (rg == o.r).all() and (ig == o.img).all()
    lags, g1, cnt = ctx.g1_table()
    rl, rg1, rcnt, _ = oracle.g1_table(np.array(traj), P, K)
    assert (lags == rl).all() and (cnt == rcnt).all()
    assert (g1 == rg1).all()
    assert (g1[cnt > 0] > 0).all()
    obs = ctx.observables()
    assert obs["overlaps"] == 0 and obs["tether_violations"] == 0
