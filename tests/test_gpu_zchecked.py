"""The bounds-checked build (ECMC_CHECKED=1: every index the EC kernels and
the staging compute is checked, the first one out of range is recorded in
the device status word and the access skipped) runs the domain forms on
ordinary inputs without a single out-of-range index and with the same
events as the oracle: the block-lockstep kernel in the benchmark's block
shape, the warp-lockstep kernel with bead springs, and a push-off of
clustered phantom chains (staging capacities and overflow lists sized for
them).  Run in a child process, because the binding picks its library when
it is first loaded."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys
sys.path.insert(0, os.path.join(ROOT, "tests"))
sys.path.insert(0, ROOT)
import numpy as np
import oracle
from paper_1502_06447_gb300 import build, ecmc
from paper_1502_06447_gb300.configs import small_domain
from helpers import gpu_context, oracle_system
build.build()
assert os.path.basename(ecmc.LIB_PATH) == "libecmc_checked.so", ecmc.LIB_PATH

def same(ctx, o, res, n):
    dig, _, _ = ctx.records(n)
    assert (dig == res["digest"]).all(), np.nonzero(dig != res["digest"])[0][:5]
    r, img = ctx.get_positions()
    assert (r == o.r).all() and (img == o.img).all()

# block-lockstep kernel, 8 lanes, 8 tiles per block, swaps
m = small_domain(seed=0xEC00C1, p_swap=0.3, sweeps=3)
o = oracle_system(m, ecs_per_tile=2)
res = o.run_domain(m.sweeps, m.ell, digests=True)
ctx = gpu_context(m, precision=ecmc.PREC_FP32F, lanes=8, block_tiles=8, ecs_per_tile=2)
ctx.run(m.ell, seed=m.seed, n_sweeps=m.sweeps)
same(ctx, o, res, m.sweeps * 27 * 2)

# warp-lockstep kernel with bead springs (far partners staged by id)
m = small_domain(seed=0xEC00C2, sweeps=3)
o = oracle_system(m, k_spring=30.0)
res = o.run_domain(m.sweeps, m.ell, digests=True)
ctx = gpu_context(m, precision=ecmc.PREC_FP32F, lanes=16, k_spring=30.0)
ctx.run(m.ell, seed=m.seed, n_sweeps=m.sweeps)
same(ctx, o, res, m.sweeps * 27)

# push-off of phantom chains (tiles staged past 256 beads: overflow lists of S/4)
L = 16.0
ctx = ecmc.Context.create_phantom((L, L, L), 100, 16, bond=1.0, c=1.9, seed=7)
ctx.configure(mode=ecmc.MODE_DOMAIN, dir_mode=ecmc.DIR_ISO, precision=ecmc.PREC_FP64,
              tiles=(3, 3, 3), lanes=32)
r, img = oracle.phantom_chains((L, L, L), 100, 16, bond=1.0, c=1.9, seed=7)
po = oracle.System(r, (L, L, L), 16, sigma=1.0, b_max=1.2, mode=oracle.MODE_DOMAIN,
                   dir_mode=oracle.DIR_ISO, D=(3, 3, 3), seed=9, img=img)
rc, sweeps, _ = po.pushoff(0.5, 4, 2.0, 6000)
assert rc == 0
assert ctx.pushoff(f0=0.5, stages=4, ell=2.0, seed=9, max_sweeps=6000) == sweeps
rg, ig = ctx.get_positions()
assert (rg == po.r).all() and (ig == po.img).all()
print("checked ok")
"""


def test_checked_build_runs_in_bounds_and_matches_oracle():
    env = dict(os.environ, ECMC_CHECKED="1")
    code = "ROOT = " + repr(ROOT) + "\n" + CHILD
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=1500)
    assert p.returncode == 0, (p.stdout[-3000:], p.stderr[-3000:])
    assert "checked ok" in p.stdout
