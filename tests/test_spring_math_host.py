"""The library's spring pieces (ec_log, spring_dE, spring_x in
ecmc_dev.cuh, host and device code) compiled for the host with g++ against
the oracle's own implementations (orc_log, orc_spring_x, Philox and its
draws): bit for bit.  The two sides share no code.  No GPU."""
import os
import subprocess
import struct

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r"""
#include <cstdio>
#include <cstring>
#include "ecmc_dev.cuh"
using namespace ecmc;
static unsigned long long bits(double x) { unsigned long long b; std::memcpy(&b, &x, 8); return b; }
int main() {
  char op[8];
  while (std::scanf("%7s", op) == 1) {
    if (!std::strcmp(op, "log")) {
      double u; std::scanf("%la", &u);
      std::printf("%016llx\n", bits(ec_log(u)));
    } else if (!std::strcmp(op, "sx")) {
      double a[9]; for (double &x : a) std::scanf("%la", &x);
      double dv;
      std::printf("%016llx\n", bits(spring_x(a[0], a[1], a[2], a[3], a[4], a[5], a[6], a[7], a[8], dv)));
    } else if (!std::strcmp(op, "de")) {
      unsigned long long c[4], k[2];
      for (auto &x : c) std::scanf("%llu", &x);
      for (auto &x : k) std::scanf("%llu", &x);
      const u64x4 w = philox(c[0], c[1], c[2], c[3], k[0], k[1]);
      std::printf("%016llx %016llx\n", bits(spring_dE(w.v[0])), bits(spring_dE(w.v[1])));
    }
  }
  return 0;
}
"""


def hexbits(x):
    return struct.pack(">d", x).hex()


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    d = tmp_path_factory.mktemp("springmath")
    src = d / "t.cpp"
    src.write_text(SRC)
    out = d / "t"
    r = subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-I",
                        os.path.join(ROOT, "paper_1502_06447_gb300", "csrc"), str(src), "-o", str(out)],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr[-3000:])
    return str(out)


def run(exe, lines):
    p = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return p.stdout.split("\n")


def test_log_bits(exe):
    rng = np.random.default_rng(2)
    us = list(rng.uniform(0, 1, 3000)) + list(np.exp(-rng.uniform(0, 700, 500))) + [1.0, 2.0 ** -53]
    us = [u for u in us if u > 0]
    out = run(exe, [f"log {float(u).hex()}" for u in us])
    for u, o in zip(us, out):
        assert o == hexbits(oracle.own_log(u)), u


def test_spring_event_bits(exe):
    rng = np.random.default_rng(3)
    lines, cases = [], []
    for _ in range(2000):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        d = rng.normal(size=3)
        d *= rng.uniform(1.0, 2.0) / np.linalg.norm(d)
        sigma, k, dE = 1.0, float(rng.choice([10.0, 30.0, 100.0])), float(rng.exponential())
        cases.append((d, v, sigma, k, dE))
        lines.append("sx " + " ".join(float(x).hex() for x in (*d, *v, sigma, k, dE)))
    out = run(exe, lines)
    for (d, v, sigma, k, dE), o in zip(cases, out):
        assert o == hexbits(oracle.spring_x(d, v, sigma, k, dE)), (d, v, k, dE)


def test_spring_energy_draw_bits(exe):
    """The Boltzmann energies of the two bonds at one event, from the
    counter (6 | ec << 8, sweep, unit, event) and key (seed, replica)."""
    rng = np.random.default_rng(4)
    lines, ctrs = [], []
    for _ in range(500):
        c = [6 | (int(rng.integers(0, 4)) << 8), int(rng.integers(0, 2 ** 40)), int(rng.integers(0, 2 ** 20)),
             int(rng.integers(0, 10 ** 6))]
        key = [int(rng.integers(0, 2 ** 63)), int(rng.integers(0, 300))]
        ctrs.append((c, key))
        lines.append("de " + " ".join(str(x) for x in c + key))
    out = run(exe, lines)
    for (c, key), o in zip(ctrs, out):
        w = oracle.philox4x64_10(c, key)
        ref = [hexbits(-oracle.own_log(1.0 - float(int(x) >> 11) * 2.0 ** -53)) for x in w[:2]]
        assert o.split() == ref, (c, key)
