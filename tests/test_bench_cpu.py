"""bench.py's structure and initial-configuration legs, run on the CPU
with stand-ins for the library and CUDA events: every name they use is
bound and the JSON fields come out as documented."""
import importlib.util
import os
import sys
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture()
def bench(monkeypatch):
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def test_structure_leg(bench, monkeypatch):
    import torch

    class Ev:
        def __init__(self, enable_timing=True):
            pass

        def record(self, s):
            pass

        def elapsed_time(self, other):
            return 10.0

    monkeypatch.setattr(torch.cuda, "Event", Ev)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    calls = []

    class Ctx:
        def structure(self, dR, nbins, r2n):
            calls.append(r2n)
            return ({"n_chains": 10, "N": 100, "rg2_sum": 160.0, "lam_sum": (10.0, 30.0, 120.0),
                     "kappa2_sum": 4.0, "bc_sum": 6758.4, "g2_sum": 1.0, "re2_sum": 990.0},
                    np.arange(100, dtype=float) if r2n else None, np.zeros(64))

    out = bench.structure_run(Ctx(), None)
    assert True in calls and False in calls
    assert out["lam_fractions"] == pytest.approx([0.0625, 0.1875, 0.75])
    assert out["rg2_mean"] == 16.0 and out["chains"] == 10
    assert set(out["r2n_over_n"]) == {"1", "10", "99"}


def test_init_leg(bench, monkeypatch):
    fake = types.ModuleType("paper_1502_06447_gb300.ecmc")

    class Ctx:
        @classmethod
        def create_phantom(cls, box, n_chains, N, **kw):
            assert len(box) == 3 and n_chains * N > 0
            return cls()

        def configure(self, **kw):
            assert kw["precision"] == fake.PREC_FP64

        def pushoff(self, **kw):
            return 839

        def structure(self, r2n):
            return {}, np.arange(20, dtype=float), None

        def observables(self):
            return {"overlaps": 0, "tether_violations": 0}

    fake.Context = Ctx
    fake.MODE_DOMAIN, fake.DIR_ISO, fake.PREC_FP64 = 1, 1, 0
    import paper_1502_06447_gb300
    monkeypatch.setitem(sys.modules, "paper_1502_06447_gb300.ecmc", fake)
    monkeypatch.setattr(paper_1502_06447_gb300, "ecmc", fake, raising=False)
    out = bench.init_run()
    assert out["pushoff_sweeps"] == 839 and out["overlaps"] == 0
    assert out["beads"] == bench.INIT["n_chains"] * bench.INIT["N"]
    assert 0.3 < out["eta"] < 0.4
