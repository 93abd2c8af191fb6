"""The autotuner's search (tune_search, host code) with synthetic objectives,
compiled with g++ (no GPU): coordinate descent over lanes, tile side, cell
side, ECs per tile, warps per block and the first-pass capacity factor
finds the optimum of separable and coupled scores,
times no point twice, skips inadmissible points and stops an abort."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")

SRC = r"""
#include <cmath>
#include <cstdio>
#include <vector>
#include "ecmc_internal.h"
using namespace ecmc;

struct Log { std::vector<TunePoint> pts; };

static bool same(const TunePoint &a, const TunePoint &b) {
  return a.lanes == b.lanes && a.tile_side == b.tile_side && a.cell_side == b.cell_side && a.ecs == b.ecs &&
         a.warps == b.warps && a.tight == b.tight;
}

template <class F>
static void run(const char *name, TunePoint start, F score, int bad_lanes = -1, int abort_after = -1) {
  Log log;
  auto trial = [&](const TunePoint &p, TuneScore *s) -> ecmc_status {
    if ((int)log.pts.size() == abort_after) return ECMC_ECUDA;
    for (const TunePoint &q : log.pts)
      if (same(p, q)) { std::printf("%s DUPLICATE\n", name); }
    log.pts.push_back(p);
    if (p.lanes == bad_lanes) return ECMC_EINVAL;
    s->ecs_per_s = score(p);
    s->events_per_s = 10.0 * s->ecs_per_s;
    return ECMC_OK;
  };
  TunePoint best{};
  TuneScore bs{};
  int n = 0;
  const ecmc_status st = tune_search(start, trial, &best, &bs, &n);
  std::printf("%s st=%d lanes=%d tile=%g cell=%g ecs=%d warps=%d tight=%g score=%g trials=%d calls=%d\n", name,
              (int)st, best.lanes, best.tile_side, best.cell_side, best.ecs, best.warps, best.tight, bs.ecs_per_s, n,
              (int)log.pts.size());
}

int main() {
  const TunePoint start{32, 4.2, 1.05, 1, 1, 1.08};
  // separable: optimum lanes 8, tile 5, cell 1.4, ecs 2, warps 2, tight 1.16
  auto sep = [](const TunePoint &p) {
    return -std::fabs(p.lanes - 8.0) - std::fabs(p.tile_side - 5.0) - 3.0 * std::fabs(p.cell_side - 1.4) -
           std::fabs(p.ecs - 2.0) - std::fabs(p.warps - 2.0) - 10.0 * std::fabs(p.tight - 1.16);
  };
  run("separable", start, sep);
  // coupled: the best lane count depends on ECs per tile, the last axis,
  // so only the second round can move lanes to 8 (optimum lanes 8, ecs 4)
  auto coupled = [](const TunePoint &p) {
    return (p.ecs == 4 ? 2.0 : 0.0) + (p.lanes == (p.ecs == 4 ? 8 : 32) ? 1.0 : 0.0);
  };
  run("coupled", start, coupled);
  // the same score with one round would stop at lanes 32: checked through
  // the first-round result (a second round only starts after a change)
  run("skip8", start, sep, 8);
  run("abort", start, sep, -1, 5);
  run("offgrid", TunePoint{8, 4.4, 1.05, 1, 1, 1.08},
      [](const TunePoint &p) { return p.tile_side == 4.4 ? 100.0 : 0.0; });
  return 0;
}
"""


def parse(out):
    res = {}
    for line in out.splitlines():
        name, *kv = line.split()
        res.setdefault(name, {})
        for item in kv:
            k, v = item.split("=") if "=" in item else (item, "1")
            res[name][k] = v
    return res


def test_tune_search_host(tmp_path):
    if not os.path.isdir(CUDA_INC):
        pytest.skip("CUDA headers not found")
    src = tmp_path / "t.cpp"
    src.write_text(SRC)
    exe = tmp_path / "t"
    r = subprocess.run(["g++", "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_1502_06447_gb300", "csrc"),
                        "-I", os.path.join(ROOT, "include"), "-I", CUDA_INC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr[-3000:])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    assert "DUPLICATE" not in out, out
    res = parse(out)
    s = res["separable"]
    assert (s["st"], s["lanes"], s["tile"], s["cell"], s["ecs"], s["warps"], s["tight"]) == (
        "0", "8", "5", "1.4", "2", "2", "1.16")
    assert int(s["trials"]) <= 1 + 2 * (4 + 7 + 2 + 4 + 3 + 3)
    c = res["coupled"]
    assert (c["lanes"], c["ecs"], c["score"]) == ("8", "4", "3")
    k = res["skip8"]
    assert k["st"] == "0" and k["lanes"] != "8"
    assert res["abort"]["st"] == str(-3) and res["abort"]["calls"] == "5"
    o = res["offgrid"]
    assert o["tile"] == "4.4" and o["trials"] != "0"


CAPS_SRC = r"""
#include <cmath>
#include <cstdio>
#include "ecmc_internal.h"
using namespace ecmc;
int main() {
  // round_up_f32: the smallest float >= x
  const double xs[] = {0.25, 0.1, 1.0 / 3.0, 1e-30, 12345.678901234, 0.2500000001};
  for (double x : xs) {
    const float f = round_up_f32(x);
    const float below = nextafterf(f, 0.0f);
    std::printf("ru %.17g %d %d\n", x, (double)f >= x, (double)below < x);
  }
  // staging capacities: the full bound covers a lattice and a 30 % density
  // excess; the tight caps never exceed it; multiples of 32 and 8
  const double rhos[] = {0.6, 0.8638, 0.95};
  const double sides[] = {3.0, 4.2, 5.4, 7.0};
  for (double rho : rhos)
    for (double e : sides) {
      const double E[3] = {e, e, e}, W[3] = {e - 2.4, e - 2.4, e - 2.4};
      const int32_t S = stage_bound(E, rho), M = stage_bound(W, rho);
      int32_t st = 0, mt = 0;
      tight_caps(E, W, rho, S, M, &st, &mt);
      const double lat = std::pow(std::floor((e + 0.02) * std::cbrt(rho)) + 1.0, 3) + 8.0;
      std::printf("cap %g %g %d %d %d %d %d\n", rho, e, S, M, st, mt,
                  S >= 1.3 * rho * e * e * e + 32 && S >= lat && S % 32 == 0 && st <= S && mt <= M &&
                      mt <= st && st % 8 == 0 && st >= rho * e * e * e);
    }
  return 0;
}
"""


def test_capacity_and_rounding_host(tmp_path):
    if not os.path.isdir(CUDA_INC):
        pytest.skip("CUDA headers not found")
    src = tmp_path / "c.cpp"
    src.write_text(CAPS_SRC)
    exe = tmp_path / "c"
    r = subprocess.run(["g++", "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_1502_06447_gb300", "csrc"),
                        "-I", os.path.join(ROOT, "include"), "-I", CUDA_INC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr[-3000:])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    for line in out.splitlines():
        f = line.split()
        if f[0] == "ru":
            assert f[2:] == ["1", "1"], line
        else:
            assert f[-1] == "1", line
