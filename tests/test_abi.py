"""The C ABI: the library builds, loads, and exports every declared symbol.
No compute calls (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1502_06447_gb300 import build, ecmc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ecmc_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib_path():
    try:
        return build.build()
    except (OSError, RuntimeError) as e:  # nvcc missing
        pytest.skip(f"cannot build: {e}")


def test_every_declared_symbol_is_exported(lib_path):
    lib = ctypes.CDLL(lib_path)
    decl = declared_symbols()
    assert len(decl) >= 15
    missing = [n for n in sorted(decl) if not hasattr(lib, n)]
    assert not missing, missing
    assert decl == set(ecmc.EXPORTS)


def test_binding_refuses_without_library(tmp_path):
    with pytest.raises(RuntimeError):
        ecmc._lib = None
        ecmc.load(str(tmp_path / "missing.so"))
    ecmc._lib = None


def _c_layout(tmp_path, structs):
    """sizeof and offsetof of every named field, as gcc lays out include/ecmc.h."""
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ecmc.h"', "int main(void) {"]
    for cname, fields in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    import subprocess
    r = subprocess.run(["gcc", "-std=c11", "-Wall", "-I", os.path.join(ROOT, "include"), str(src),
                        "-o", str(exe)], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(f"include/ecmc.h does not compile as C:\n{r.stderr}")
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return {k: int(v) for k, v in (ln.split() for ln in out.splitlines())}


def test_binding_struct_layouts_match_header(tmp_path):
    """Every struct the binding passes by pointer has the header's size and
    field offsets (a mismatch would corrupt options or results silently)."""
    pairs = {"ecmc_opts": ecmc.Opts, "ecmc_obs": ecmc.Obs, "ecmc_tuning": ecmc.Tuning,
             "ecmc_replica_spec": ecmc.ReplicaSpec, "ecmc_struct": ecmc.Struct}
    structs = {c: [f for f, _ in py._fields_] for c, py in pairs.items()}
    structs["ecmc_event"] = list(ecmc.EVENT_DTYPE.names)
    got = _c_layout(tmp_path, structs)
    for cname, py in pairs.items():
        assert got[cname] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[f"{cname}.{f}"] == getattr(py, f).offset, (cname, f)
    assert got["ecmc_event"] == ecmc.EVENT_DTYPE.itemsize
    for f in ecmc.EVENT_DTYPE.names:
        assert got[f"ecmc_event.{f}"] == ecmc.EVENT_DTYPE.fields[f][1], f


@pytest.mark.parametrize("box,cell_side,tiles", [
    ((2.0 ** 22, 2.0 ** 21, 2.0 ** 21), 1.0, (20, 20, 20)),   # product of the axes wraps in int64
    ((1e300, 10.0, 10.0), 1.0, (3, 3, 3)),                      # one axis beyond int range
    ((200.0, 200.0, 200.0), 1.0, (20, 20, 20)),                 # 8e6 cells > 2^20
    ((float("inf"), 10.0, 10.0), 1.0, (3, 3, 3)),               # non-finite box
    ((1e5, 1e5, 1e5), 1e4, (2 ** 11, 2 ** 11, 2 ** 11)),        # 2^33 tiles
])
def test_cells_static_rejects_bad_sizes_before_any_launch(lib_path, box, cell_side, tiles):
    """ecmc_cells_static checks every size in double before an integer cast
    or product and refuses what its fixed scratch array or int32 tile
    numbering cannot hold; these calls return ECMC_EINVAL without touching a
    device (the pointers are never dereferenced), so they run on the CPU."""
    dummy = 1 << 20
    with pytest.raises(ecmc.EcmcError) as e:
        ecmc.cells_static(dummy, 1000, box, tiles, 1.2, cell_side, 0, 0, dummy, dummy, dummy)
    assert e.value.code == -1


def test_out_of_memory_is_reported_as_enomem(lib_path, monkeypatch):
    """Host-side fault injection: with ECMC_ALLOC_LIMIT set, a device
    allocation above the limit fails as cudaMalloc does on a full device;
    creating a context then returns ECMC_ENOMEM (no device is touched
    before the refused allocation, so this runs on the CPU)."""
    monkeypatch.setenv("ECMC_ALLOC_LIMIT", "1000")
    with pytest.raises(ecmc.EcmcError) as e:
        ecmc.Context.create_lattice((8, 8, 10), 1.05, 10, jitter=0.01, seed=1)
    assert e.value.code == -2 and "ENOMEM" in str(e.value)
