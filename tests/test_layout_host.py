"""Shared-memory layout of a tile's staging area (host code, compiled with
nvcc, no GPU): for every staging capacity the kernels can be given (a
multiple of 8 slots), each tile's share is a multiple of 16 bytes, so that
the next tile's arrays (FP64 positions, 16-byte cell records read as one
vector) stay aligned, and the overflow list holds at least a quarter of
the staged beads."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r"""
#include <cstdio>
#include "ec_device.cuh"
using namespace ecmc;
int main() {
  long bad = 0, n = 0;
  const int ncs[] = {1, 27, 64, 125, 343, 1000};
  for (int S = 8; S <= 65536; S += 8) {
    const int ov = ovf_cap_for(S);
    if (ov % 8 != 0 || ov < S / 4 || ov < OVF_CAP) { ++bad; std::printf("ovf S=%d ov=%d\n", S, ov); }
    for (int M64 : {0, S, (S / 16) * 8 + 8}) {
      for (int MNB : {8, S, (S / 24) * 8 + 8}) {
        for (int NC : ncs) {
          ++n;
          if (group_bytes(S, M64, MNB, NC) % 16 != 0) {
            if (bad < 10) std::printf("S=%d M64=%d MNB=%d NC=%d bytes=%zu\n", S, M64, MNB, NC,
                                      group_bytes(S, M64, MNB, NC));
            ++bad;
          }
        }
      }
    }
  }
  std::printf("checked %ld bad %ld\n", n, bad);
  return bad != 0;
}
"""


def test_group_bytes_keep_16_byte_alignment(tmp_path):
    nvcc = shutil.which(os.environ.get("NVCC", "nvcc"))
    if nvcc is None:
        pytest.skip("nvcc not found")
    src = tmp_path / "t.cu"
    src.write_text(SRC)
    exe = tmp_path / "t"
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", os.path.join(ROOT, "paper_1502_06447_gb300", "csrc"),
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr[-3000:])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout[-2000:]
    assert "bad 0" in out.stdout
