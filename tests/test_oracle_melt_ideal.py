"""Melt physics pin of the oracle: chains in a melt are ideal, R_e^2 grows
linearly with the chain length (Sec. II.B: <R^2> = c N sigma^2 for the
melt's chains, with c set by the local stiffness; Flory's ideality of
chains in a melt).

Starting states are far from ideal on purpose: phantom chains of stiffness
c = 5 (the first stage of the paper's initial configurations, Sec. II.B),
pushed apart by the oracle's slow push-off, carry R_e^2/(N-1) of about
3.5-4.5 sigma^2 for N = 8, 16, 32.  The oracle then runs serial ECs
(isotropic directions, ell = 10 sigma) with the swap move at every motile
contact (Sec. II.C, p_swap = 1, the paper's rule; it leaves the equilibrium
ensemble of equal-length chains unchanged and speeds relaxation) until the
middle bead's MSD g1 (Sec. IV, Eq. 3) exceeds each chain length's R_e^2
several times over.  The melt: packing fraction 0.35 and tethers of
1.4 sigma (the tether length of the paper's reptation melt, Sec. IV.B).

Checked, for N = 8, 16, 32 (1024 beads per run; N = 32 and 16 in several
independent runs, all runs in parallel processes):
  - relaxation: g1 over the production stretch >= 3 R_e^2 of that N;
  - drift: R_e^2/(N-1) fell below 0.7 times its start value (a run in
    which nothing moves fails);
  - linearity: the weighted least-squares line R_e^2 = A (N - 1) + B
    passes within 5 % of every N's time average, with A > 0.
The oracle runs about 5e5 events/s on one core and chains of 32 beads need
some 6e4 events per bead to relax and average here, so the melt sits at
packing fraction 0.35 (between the paper's reptation melt at 0.298 and its
System I at 0.39) and the boxes are small (11.5 sigma): at this
size R_e^2/(N-1) still grows by 8-12 % per doubling of N (finite chains,
local stiffness and the small box), so proportionality R_e^2 = c (N - 1) is
asserted in the linear form with an intercept, not as a constant ratio.
The run takes about two minutes on 8 host cores (marked slow; not a GPU
test)."""
import math
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

ETA = 0.35
B_MAX = 1.4
BOND = 1.1
STIFF = 5.0
ELL = 10.0
BEADS = 1024
EQ_PER_BEAD = 20_000    # events per bead before the production stretch
PROD_PER_BEAD = 40_000  # events per bead in the production stretch
SAMPLE_PER_BEAD = 1_000  # events per bead between R_e^2 samples
RUNS = {8: (101,), 16: (201, 202), 32: (301, 302, 303, 304)}


def melt_run(N, seed):
    """One melt: phantom chains (c = 5), slow push-off, serial ECs with
    swaps.  Returns the start R_e^2, the production samples of the mean
    R_e^2 and the middle beads' MSD over the production stretch."""
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import oracle
    M = BEADS // N
    L = (BEADS * math.pi / (6.0 * ETA)) ** (1.0 / 3.0)
    r, img = oracle.phantom_chains((L, L, L), M, N, bond=BOND, c=STIFF, seed=seed)
    D = max(3, int(L // 4.0))
    po = oracle.System(r, (L, L, L), N, sigma=1.0, b_max=B_MAX, mode=oracle.MODE_DOMAIN,
                       dir_mode=oracle.DIR_ISO, D=(D, D, D), seed=seed + 7, img=img)
    rc, _, _ = po.pushoff(0.6, 4, 2.0, 20000)
    assert rc == 0
    re2_start = float(po.chain_obs()[0].mean())
    s = oracle.System(po.r, (L, L, L), N, sigma=1.0, b_max=B_MAX, mode=oracle.MODE_SERIAL,
                      dir_mode=oracle.DIR_ISO, p_swap=1.0, seed=seed + 11, img=po.img)
    ec = [0]

    def advance(events):
        done = 0
        while done < events:
            res = s.run_serial(512, ELL, ec0=ec[0])
            assert res["rc"] == 0
            ec[0] += 512
            done += res["stats"]["events"]

    advance(EQ_PER_BEAD * BEADS)
    mid0 = s.unwrapped().reshape(M, N, 3)[:, N // 2].copy()
    samples = []
    for _ in range(PROD_PER_BEAD // SAMPLE_PER_BEAD):
        advance(SAMPLE_PER_BEAD * BEADS)
        samples.append(float(s.chain_obs()[0].mean()))
    d = s.unwrapped().reshape(M, N, 3)[:, N // 2] - mid0
    g1 = float((d * d).sum(axis=1).mean())
    dmin, n_ov = s.min_pair()
    _, bonds = s.chain_obs()
    return {"N": N, "seed": seed, "start": re2_start, "samples": samples, "g1": g1,
            "overlaps": n_ov, "bond_max": float(bonds.max())}


def block_mean_se(runs, nblock=6):
    """Mean over all samples of all runs and its standard error from block
    averages (each run cut into nblock consecutive blocks)."""
    blocks = []
    for x in runs:
        x = np.asarray(x)
        for b in np.array_split(x, nblock):
            blocks.append(b.mean())
    blocks = np.asarray(blocks)
    return float(blocks.mean()), float(blocks.std(ddof=1) / math.sqrt(len(blocks)))


@pytest.mark.slow
def test_melt_chains_are_ideal_re2_linear_in_n():
    jobs = [(N, seed) for N, seeds in RUNS.items() for seed in seeds]
    ctx = mp.get_context("spawn")
    with ProcessPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 1),
                             mp_context=ctx) as ex:
        out = list(ex.map(melt_run, *zip(*jobs)))
    Ns = sorted(RUNS)
    mean, se, start, g1 = {}, {}, {}, {}
    for N in Ns:
        rs = [o for o in out if o["N"] == N]
        for o in rs:
            assert o["overlaps"] == 0 and o["bond_max"] <= B_MAX * (1 + 1e-10)
        mean[N], se[N] = block_mean_se([o["samples"] for o in rs])
        start[N] = float(np.mean([o["start"] for o in rs]))
        g1[N] = float(np.mean([o["g1"] for o in rs]))
    report = {N: (round(mean[N] / (N - 1), 4), round(se[N] / mean[N], 4),
                  round(start[N] / (N - 1), 3), round(g1[N] / mean[N], 2)) for N in Ns}
    for N in Ns:
        # relaxed: the middle bead moved several times the chain's size
        assert g1[N] >= 3.0 * mean[N], report
        # drifted far from the stiff start
        assert mean[N] / (N - 1) < 0.7 * start[N] / (N - 1), report
    # linear in N - 1 (weighted least squares)
    x = np.array([N - 1 for N in Ns], dtype=float)
    y = np.array([mean[N] for N in Ns])
    w = np.array([1.0 / se[N] ** 2 for N in Ns])
    Xw = np.stack([x, np.ones_like(x)], axis=1) * np.sqrt(w)[:, None]
    A, B = np.linalg.lstsq(Xw, y * np.sqrt(w), rcond=None)[0]
    fit = A * x + B
    assert np.all(np.abs(y - fit) <= 0.05 * y), (report, A, B)
    assert A > 0
