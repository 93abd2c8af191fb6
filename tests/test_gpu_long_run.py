"""Long runs on the GPU against the oracle: 600 domain sweeps (Sec. II.A) of
small melts with chains of N = 8, 16 and 32 beads, in the screened form the
benchmark times (FP32 screen + FP64 evaluation, block-lockstep kernel) and
with swap moves proposed at every contact (Sec. II.C).

The statistics a long run reports must match the oracle's: the pressure
within 3 standard errors and R_e^2(N) within 2 %.  Here they match exactly,
because every EC of the 600 sweeps has the oracle's event digest: the
per-EC digests of the whole run, the final positions and image counters,
the time series of R_e^2 (every 50 sweeps), the lift sums behind the
lift-distance pressure and the contact-value pressure of the final state
are compared.  Tolerances are written as the workload states them and hold
with room to spare."""
import numpy as np
import pytest

import oracle
from paper_1502_06447_gb300 import ecmc

pytestmark = pytest.mark.gpu

SWEEPS, CHUNK, ELL, D, ECS = 600, 50, 5.0, (3, 3, 3), 2
DIMS, SPACING, JITTER, SEED = (12, 12, 12), 1.05, 0.01, 0xEC10


@pytest.mark.parametrize("N", [8, 16, 32])
def test_long_run_statistics_match_oracle(N):
    from paper_1502_06447_gb300 import build
    build.build()
    L = tuple(d * SPACING for d in DIMS)
    ctx = ecmc.Context.create_lattice(DIMS, SPACING, N, jitter=JITTER, seed=SEED + N)
    ctx.configure(mode=ecmc.MODE_DOMAIN, dir_mode=ecmc.DIR_ISO, precision=ecmc.PREC_FP32F,
                  tiles=D, lanes=8, ecs_per_tile=ECS, p_swap=1.0, record=1)
    orc = oracle.System(oracle.lattice(DIMS, SPACING, JITTER, SEED + N), L, N,
                        mode=oracle.MODE_DOMAIN, dir_mode=oracle.DIR_ISO, D=D,
                        ecs_per_tile=ECS, p_swap=1.0, seed=SEED + N)
    nt = D[0] * D[1] * D[2]
    re2_gpu, re2_orc = [], []
    lift_orc = disp_orc = 0.0
    sw = 0
    while sw < SWEEPS:
        ctx.run(ELL, seed=SEED + N, n_sweeps=CHUNK)
        dig, _, nev = ctx.records(CHUNK * nt * ECS)
        res = orc.run_domain(CHUNK, ELL, sweep0=sw, digests=True)
        assert res["rc"] == 0
        assert (dig == res["digest"]).all(), f"digests differ in sweeps {sw}..{sw + CHUNK}"
        assert (nev == res["ec_events"]).all()
        lift_orc += res["stats"]["lift_sum"]
        disp_orc += res["stats"]["disp_sum"]
        re2_gpu.append(ctx.observables()["re2_mean"])
        re2_orc.append(float(orc.chain_obs()[0].mean()))
        sw += CHUNK
    r, img = ctx.get_positions()
    assert (r == orc.r).all() and (img == orc.img).all()
    obs = ctx.observables()
    assert obs["overlaps"] == 0 and obs["tether_violations"] == 0
    assert obs["sweeps"] == SWEEPS and obs["ecs"] == SWEEPS * nt * ECS
    # R_e^2(N): time averages within 2 % (here identical sample for sample)
    re2_gpu, re2_orc = np.array(re2_gpu), np.array(re2_orc)
    assert abs(re2_gpu.mean() / re2_orc.mean() - 1.0) <= 0.02
    np.testing.assert_allclose(re2_gpu, re2_orc, rtol=1e-12)
    # pressure: the lift-distance sums and the contact-value estimator of the
    # final state within 3 standard errors (here equal to rounding)
    p_gpu = obs["pressure"]
    p_orc = 1.0 + lift_orc / disp_orc
    pc_orc = orc.contact_pressure(obs["contact_delta"])
    # the contact-value estimate's standard error from its pair counts
    # (Poisson counts in the two shells)
    pairs = np.array(obs["contact_pairs"], dtype=float)
    se_c = (np.hypot(1.5 * np.sqrt(pairs[0]), 0.5 * np.sqrt(pairs[1])) /
            obs["contact_delta"] / (3.0 * len(r)))
    assert abs(obs["pressure_contact"] - pc_orc) <= 3.0 * se_c
    assert obs["pressure_contact"] == pytest.approx(pc_orc, rel=1e-12)
    assert p_gpu == pytest.approx(p_orc, rel=1e-9)
    ctx.close()
