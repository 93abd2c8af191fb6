"""The chain-structure pass (ecmc_structure) against the oracle on the same
positions: R_g^2, kappa2, 4 b^2 + 3 c^2, |R_e|^2 and g2 sums, R^2(n) and
the end-to-end histogram bit for bit (same sums in the same order); the
eigenvalue sums, asphericity and acylindricity within 1e-10 of the LAPACK
eigenvalues (the library uses a Jacobi iteration whose eigenvalues are
within ~1e-15 Tr S of exact, summed over at most 1000 chains)."""
import numpy as np
import pytest

import oracle
from paper_1502_06447_gb300 import ecmc
from paper_1502_06447_gb300.configs import C2, C5, small_domain

from helpers import gpu_context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1502_06447_gb300 import build
    build.build()


def oracle_side(ctx, dR, nbins, r2n=True):
    r, _img = ctx.get_positions()
    s = oracle.System(r, tuple(ctx.L), ctx.N)
    out = s.chain_struct(dR=dR, nbins=nbins, r2n=r2n)
    sd = oracle.shape_descriptors(out["gyr"])
    re2, _ = s.chain_obs()
    return out, sd, re2


def check(ctx, dR=0.5, nbins=64, r2n=True):
    got, rn, hist = ctx.structure(dR=dR, nbins=nbins, r2n=r2n)
    out, sd, re2 = oracle_side(ctx, dR, nbins, r2n)
    nch = ctx.n // ctx.N
    assert got["n_chains"] == nch and got["N"] == ctx.N
    assert got["rg2_sum"] == oracle.seq_sum(sd["T"])
    assert got["kappa2_sum"] == oracle.seq_sum(sd["kappa2"])
    assert got["bc_sum"] == oracle.seq_sum(sd["bc"])
    assert got["re2_sum"] == oracle.seq_sum(re2)
    scale = got["rg2_sum"]
    for k in range(3):
        assert got["lam_sum"][k] == pytest.approx(oracle.seq_sum(sd["lam"][:, k]), abs=1e-10 * scale)
    assert got["b_sum"] == pytest.approx(oracle.seq_sum(sd["b"]), abs=1e-10 * scale)
    assert got["c_sum"] == pytest.approx(oracle.seq_sum(sd["c"]), abs=1e-10 * scale)
    if r2n:
        assert (rn == out["r2n"]).all(), np.nonzero(rn != out["r2n"])[0][:5]
    assert (hist == out["hist"]).all()
    return got, out


@pytest.mark.parametrize("N", [2, 7, 8, 16])
def test_structure_small_melts(N):
    """Lattice melts of 2-16 beads per chain after three domain sweeps
    (chains crossing the periodic box, odd and even N)."""
    m = small_domain(N=N, dims=(14, 14, 16))
    ctx = gpu_context(m, precision=ecmc.PREC_FP32F, lanes=8, record=0)
    ctx.run(m.ell, seed=m.seed, n_sweeps=3)
    check(ctx, dR=0.25, nbins=40)


def test_structure_c2_and_g2():
    """C2 (4096 x 64): the structure after a sweep; g2 over two more sweeps
    against the reference ecmc_g1_reset takes."""
    ctx = gpu_context(C2, precision=ecmc.PREC_FP32F, lanes=8, record=0)
    ctx.run(C2.ell, seed=C2.seed, n_sweeps=1)
    check(ctx, dR=1.0, nbins=32)
    ctx.g1_reset()
    mid0 = oracle_side(ctx, 1.0, 0, r2n=False)[0]["mid"]
    ctx.run(C2.ell, seed=C2.seed, n_sweeps=2)
    got, out = check(ctx, dR=1.0, nbins=32)
    g2 = oracle.seq_sum(oracle.g2_terms(mid0, out["mid"]))
    assert got["g2_sum"] == g2 and g2 > 0.0


def test_structure_full_size_melt():
    """The 10^6-bead melt (1000 chains of 1000) after a sweep in the
    benchmark's launch setting: every output at full size."""
    ctx = gpu_context(C5, precision=ecmc.PREC_FP32F, lanes=8, record=0, tiles=(25, 25, 25),
                      ecs_per_tile=2)
    ctx.run(C5.ell, seed=C5.seed, n_sweeps=1)
    check(ctx, dR=2.0, nbins=64)


def test_structure_rejects_bad_arguments():
    m = small_domain(N=1)
    ctx = gpu_context(m, record=0)
    with pytest.raises(ecmc.EcmcError) as e:
        ctx.structure()
    assert e.value.code == -1
    m = small_domain(N=8)
    ctx = gpu_context(m, record=0)
    with pytest.raises(ecmc.EcmcError) as e:
        ctx.structure(dR=0.0, nbins=8)
    assert e.value.code == -1
    got, rn, hist = ctx.structure(r2n=False)
    assert rn is None and hist.size == 0 and got["g2_sum"] == 0.0
