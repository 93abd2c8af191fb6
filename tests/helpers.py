"""Test helpers: build matching oracle and CUDA systems from one workload spec."""
import numpy as np

import oracle
from paper_1502_06447_gb300 import ecmc
from paper_1502_06447_gb300.configs import Melt

DIRS = {"cart3": (oracle.DIR_CART3, ecmc.DIR_CART3), "iso": (oracle.DIR_ISO, ecmc.DIR_ISO)}


def oracle_system(m: Melt, **kw) -> oracle.System:
    r = oracle.lattice(m.dims, m.spacing, m.jitter, m.seed)
    mode = oracle.MODE_DOMAIN if m.mode == "domain" else oracle.MODE_SERIAL
    args = dict(sigma=m.sigma, b_max=m.b_max, s_cap=0.25 * m.sigma, mode=mode,
                dir_mode=DIRS[m.dir_mode][0], D=m.D, w=m.b_max, p_swap=m.p_swap, seed=m.seed)
    args.update(kw)
    return oracle.System(r, m.L, m.N, **args)


def gpu_context(m: Melt, precision=ecmc.PREC_FP64, lanes=32, record=1, **kw) -> ecmc.Context:
    ctx = ecmc.Context.create_lattice(m.dims, m.spacing, m.N, sigma=m.sigma, b_max=m.b_max,
                                      jitter=m.jitter, seed=m.seed)
    mode = ecmc.MODE_DOMAIN if m.mode == "domain" else ecmc.MODE_SERIAL
    args = dict(mode=mode, dir_mode=DIRS[m.dir_mode][1], precision=precision, tiles=m.D,
                p_swap=m.p_swap, lanes=lanes, record=record)
    args.update(kw)
    ctx.configure(**args)
    return ctx


def sample_positions(r, k=2000, seed=0):
    idx = np.random.default_rng(seed).choice(len(r), size=min(k, len(r)), replace=False)
    return np.sort(idx)
