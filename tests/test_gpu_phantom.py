"""Phantom chains on the GPU (ecmc_phantom_chains) against the oracle's
generator: positions and image counters bit for bit (same Philox stream,
same FP64 operations, no transcendental functions)."""
import numpy as np
import pytest

import oracle
from paper_1502_06447_gb300 import ecmc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1502_06447_gb300 import build
    build.build()


@pytest.mark.parametrize("L,nch,N,bond,c,seed", [
    ((40.0, 40.0, 40.0), 500, 121, 1.0, 1.9, 7),       # the paper's push-off example size
    ((12.0, 15.0, 9.5), 37, 64, 1.05, 1.0, 1),         # free walk, uneven box, crossing it often
    ((20.0, 20.0, 20.0), 300, 33, 0.97, 6.0, 2 ** 63 + 5),  # stiff chains, large seed
    ((105.0, 105.0, 105.0), 1000, 1000, 1.0, 1.9, 3),  # 10^6 beads
    ((5.0, 5.0, 5.0), 1000, 1, 1.0, 1.9, 4),            # single beads
])
def test_phantom_matches_oracle(L, nch, N, bond, c, seed):
    r, img = ecmc.phantom_chains(L, nch, N, bond=bond, c=c, seed=seed)
    ro, io = oracle.phantom_chains(L, nch, N, bond=bond, c=c, seed=seed)
    bad = np.nonzero((r != ro).any(axis=1))[0]
    assert bad.size == 0, (bad[:5], r[bad[:2]], ro[bad[:2]])
    assert (img == io).all()


def test_phantom_rejects_bad_arguments():
    for kw in (dict(c=0.5), dict(bond=0.0), dict(N=0), dict(n_chains=0)):
        args = dict(L=(10.0, 10.0, 10.0), n_chains=4, N=5, bond=1.0, c=1.9)
        args.update(kw)
        with pytest.raises(ecmc.EcmcError) as e:
            ecmc.phantom_chains(**args)
        assert e.value.code == -1
