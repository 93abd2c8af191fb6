"""ecmc_cells_static: the domain assignment and cell list of one sweep for
callers that cannot allocate device memory (a host callback, a framework that
owns every device allocation, a real-time loop that must stay off the
driver's allocator).  The entry point writes into caller-owned device buffers
and keeps its temporaries in a fixed file-scope device array.

Checked against the library's own per-sweep domain assignment
(ecmc_domain_tags) on two calls in a row, so stale contents of the shared
scratch array from the first call cannot leak into the second.  This file is
named to be collected last.
"""
import math

import numpy as np
import pytest

from paper_1502_06447_gb300 import ecmc
from paper_1502_06447_gb300.configs import C2

from helpers import gpu_context

pytestmark = pytest.mark.gpu


def test_cells_static_matches_domain_assignment():
    torch = pytest.importorskip("torch")
    from paper_1502_06447_gb300 import build
    build.build()
    m = C2
    ctx = gpu_context(m, record=0)
    ctx.run(m.ell, seed=m.seed, n_sweeps=1)  # positions off the lattice
    r, _ = ctx.get_positions()
    n = len(r)
    cell_side = 1.0
    nc = [int(math.floor(L / cell_side)) for L in ctx.L]
    ncell = nc[0] * nc[1] * nc[2]
    dev = torch.device("cuda")
    d_r = torch.from_numpy(r).to(dev)
    tags = torch.empty(n, dtype=torch.int32, device=dev)
    start = torch.empty(ncell + 1, dtype=torch.int32, device=dev)
    ids = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    cs = np.array(ctx.L) / np.array(nc)
    host_cell = np.minimum((r / cs).astype(np.int64), np.array(nc) - 1)
    host_cell = (host_cell[:, 2] * nc[1] + host_cell[:, 1]) * nc[0] + host_cell[:, 0]
    for sweep in (3, 4):
        shift = ecmc.cells_static(d_r.data_ptr(), n, ctx.L, m.D, m.b_max, cell_side, m.seed,
                                  sweep, tags.data_ptr(), start.data_ptr(), ids.data_ptr(),
                                  stream=stream.cuda_stream)
        stream.synchronize()
        ref_tags, ref_shift = ctx.domain_tags(m.seed, sweep)
        assert (shift == ref_shift).all()
        assert (tags.cpu().numpy() == ref_tags).all()
        st = start.cpu().numpy()
        got = ids.cpu().numpy()
        assert st[0] == 0 and st[-1] == n and (np.diff(st) >= 0).all()
        assert (np.sort(got) == np.arange(n)).all()
        cell_of_slot = np.repeat(np.arange(ncell), np.diff(st))
        assert (cell_of_slot == host_cell[got]).all()


def test_cells_static_rejects_sizes_beyond_its_limit():
    from paper_1502_06447_gb300 import build
    build.build()
    dummy = 1 << 20
    with pytest.raises(ecmc.EcmcError) as e:
        ecmc.cells_static(dummy, (1 << 20) + 1, (200.0, 200.0, 200.0), (20, 20, 20), 1.2, 1.0,
                          0, 0, dummy, dummy, dummy)
    assert e.value.code == -1
    with pytest.raises(ecmc.EcmcError) as e:  # 200^3 cells of side 1 > 2^20
        ecmc.cells_static(dummy, 1000, (200.0, 200.0, 200.0), (20, 20, 20), 1.2, 1.0,
                          0, 0, dummy, dummy, dummy)
    assert e.value.code == -1
