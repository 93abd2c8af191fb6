"""Slow push-off on the GPU (ecmc_create_phantom + ecmc_pushoff) against the
oracle's push-off from the same phantom chains: the number of sweeps and
the final positions and image counters bit for bit; the context refuses
ecmc_run before the push-off and runs after it."""
import numpy as np
import pytest

import oracle
from paper_1502_06447_gb300 import ecmc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1502_06447_gb300 import build
    build.build()


def pair(eta, N, L, seed, po_seed, D, lanes, c=1.9, k_spring=0.0):
    nch = int(round(eta * L ** 3 * 6 / np.pi / N))
    ctx = ecmc.Context.create_phantom((L, L, L), nch, N, bond=1.0, c=c, seed=seed, sigma=1.0, b_max=1.2)
    ctx.configure(mode=ecmc.MODE_DOMAIN, dir_mode=ecmc.DIR_ISO, precision=ecmc.PREC_FP64, tiles=D,
                  lanes=lanes, k_spring=k_spring)
    r, img = oracle.phantom_chains((L, L, L), nch, N, bond=1.0, c=c, seed=seed)
    o = oracle.System(r, (L, L, L), N, sigma=1.0, b_max=1.2, mode=oracle.MODE_DOMAIN,
                      dir_mode=oracle.DIR_ISO, D=D, seed=po_seed, img=img, k_spring=k_spring)
    return ctx, o


@pytest.mark.parametrize("eta,N,L,D,lanes,stages", [
    (0.35, 20, 14.0, (3, 3, 3), 8, 5),
    (0.30, 10, 10.0, (3, 3, 3), 32, 3),
    (0.40, 16, 16.0, (4, 3, 4), 16, 6),
    (0.30, 1, 9.0, (3, 3, 3), 8, 2),
])
def test_pushoff_matches_oracle(eta, N, L, D, lanes, stages):
    ctx, o = pair(eta, N, L, seed=51, po_seed=0xEC0F0F, D=D, lanes=lanes)
    with pytest.raises(ecmc.EcmcError) as e:
        ctx.run(2.0, seed=1, n_sweeps=1)
    assert e.value.code == -4
    n = ctx.pushoff(f0=0.5, stages=stages, ell=2.0, seed=0xEC0F0F, max_sweeps=6000)
    rc, sweeps, st = o.pushoff(0.5, stages, 2.0, 6000)
    assert rc == 0 and n == sweeps > 0
    r, img = ctx.get_positions()
    bad = np.nonzero((r != o.r).any(axis=1))[0]
    assert bad.size == 0, (bad[:5], r[bad[:2]], o.r[bad[:2]])
    assert (img == o.img).all()
    obs = ctx.observables()
    assert obs["overlaps"] == 0 and obs["tether_violations"] == 0
    ctx.run(2.0, seed=1, n_sweeps=1)  # a normal sweep now runs


def test_pushoff_rejects_bad_settings():
    ctx = ecmc.Context.create_phantom((10.0, 10.0, 10.0), 20, 10, seed=1)
    ctx.configure(mode=ecmc.MODE_DOMAIN, precision=ecmc.PREC_FP32F, tiles=(3, 3, 3), lanes=8)
    with pytest.raises(ecmc.EcmcError) as e:
        ctx.pushoff()
    assert e.value.code == -1
    ctx.configure(mode=ecmc.MODE_DOMAIN, precision=ecmc.PREC_FP64, tiles=(3, 3, 3), lanes=8)
    for kw in (dict(f0=0.0), dict(stages=0), dict(max_sweeps=0)):
        with pytest.raises(ecmc.EcmcError) as e:
            ctx.pushoff(**kw)
        assert e.value.code == -1
    with pytest.raises(ecmc.EcmcError) as e:  # not resolved within one sweep
        ctx.pushoff(f0=1.0, stages=1, max_sweeps=1)
    assert e.value.code == -6


@pytest.mark.parametrize("lanes", [32, 8])
def test_pushoff_with_springs_matches_oracle(lanes):
    """Bead springs (k = 30 kT/sigma^2, rest length the current diameter)
    acting during the push-off: same sweeps, positions and images as the
    oracle; the springs then run as an ordinary spring melt."""
    ctx, o = pair(0.40, 16, 14.0, seed=53, po_seed=0xEC0F1F, D=(3, 3, 3), lanes=lanes, k_spring=30.0)
    n = ctx.pushoff(f0=0.5, stages=4, ell=2.0, seed=0xEC0F1F, max_sweeps=6000)
    rc, sweeps, _ = o.pushoff(0.5, 4, 2.0, 6000)
    assert rc == 0 and n == sweeps > 0
    r, img = ctx.get_positions()
    bad = np.nonzero((r != o.r).any(axis=1))[0]
    assert bad.size == 0, (bad[:5], r[bad[:2]], o.r[bad[:2]])
    assert (img == o.img).all()
    assert ctx.observables()["overlaps"] == 0
    ctx.run(5.0, seed=1, n_sweeps=1)
