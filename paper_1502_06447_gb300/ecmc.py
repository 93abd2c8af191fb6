"""Thin Python binding of the C ABI in include/ecmc.h (argument marshalling only).

Every step of the EC path runs in the CUDA library libecmc.so; this module
only converts arguments.  There is no CPU fallback: if the library is missing
or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# ECMC_CHECKED=1: the bounds-checked build (see build.py)
LIB_PATH = os.path.join(_HERE, "libecmc_checked.so" if os.environ.get("ECMC_CHECKED") == "1"
                        else "libecmc.so")

MODE_SERIAL, MODE_DOMAIN = 0, 1
DIR_CART3, DIR_ISO = 0, 1
PREC_FP64, PREC_FP32F = 0, 1
EV_NAMES = ("end", "pass", "wall", "hs_lift", "hs_reflect", "te_lift", "te_reflect", "swap")
STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EOVERLAP", -5: "ETETHER",
          -6: "ESTUCK", -7: "ECKPT", -8: "ECAPACITY", -9: "EBOUNDS"}

# every symbol include/ecmc.h declares
EXPORTS = (
    "ecmc_create_lattice", "ecmc_create", "ecmc_destroy", "ecmc_last_error", "ecmc_set_stream",
    "ecmc_set_positions", "ecmc_get_positions", "ecmc_get_info", "ecmc_configure", "ecmc_run",
    "ecmc_swap", "ecmc_observables", "ecmc_g1_reset", "ecmc_records", "ecmc_log_reserve",
    "ecmc_event_log", "ecmc_domain_tags", "ecmc_checkpoint", "ecmc_restore",
    "ecmc_cells_static", "ecmc_batch_create", "ecmc_batch_destroy", "ecmc_batch_configure",
    "ecmc_batch_run", "ecmc_batch_get_positions", "ecmc_batch_info", "ecmc_batch_stats",
    "ecmc_batch_records", "ecmc_autotune", "ecmc_batch_autotune", "ecmc_structure",
    "ecmc_phantom_chains", "ecmc_create_phantom", "ecmc_pushoff", "ecmc_g1_track",
    "ecmc_g1_table",
)


class EcmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Opts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("dir_mode", C.c_int32), ("precision", C.c_int32),
                ("tiles", C.c_int32 * 3), ("joint", C.c_double), ("s_cap", C.c_double),
                ("event_cap", C.c_int64), ("p_swap", C.c_double), ("ecs_per_tile", C.c_int32),
                ("lanes", C.c_int32), ("record", C.c_int32), ("stage_cap", C.c_int32),
                ("cell_side", C.c_double), ("tile_side", C.c_double), ("schedule", C.c_int32),
                ("block_tiles", C.c_int32), ("request_cap", C.c_int32), ("k_spring", C.c_double),
                ("tight_factor", C.c_double)]


class Obs(C.Structure):
    _fields_ = [("n_beads", C.c_int64), ("n_chains", C.c_int64), ("N", C.c_int64),
                ("sweeps", C.c_int64), ("ecs", C.c_int64), ("events", C.c_int64 * 8),
                ("events_total", C.c_int64), ("swap_tried", C.c_int64),
                ("lift_sum", C.c_double), ("refl_sum", C.c_double), ("disp_sum", C.c_double),
                ("ell_sum", C.c_double), ("pressure", C.c_double), ("re2_mean", C.c_double),
                ("bond_max", C.c_double), ("bond_min", C.c_double), ("overlaps", C.c_int64),
                ("tether_violations", C.c_int64), ("g1", C.c_double),
                ("device_seconds", C.c_double), ("ec_kernel_seconds", C.c_double),
                ("confirmed", C.c_int64), ("contact_pairs", C.c_int64 * 2),
                ("taut_bonds", C.c_int64 * 2), ("contact_delta", C.c_double),
                ("pressure_contact", C.c_double), ("exhaustive", C.c_int64),
                ("bond_mean", C.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_
             if k not in ("events", "contact_pairs", "taut_bonds")}
        d["contact_pairs"] = tuple(self.contact_pairs)
        d["taut_bonds"] = tuple(self.taut_bonds)
        for i, name in enumerate(EV_NAMES):
            d[name] = self.events[i]
        return d


class Struct(C.Structure):
    _fields_ = [("n_chains", C.c_int64), ("N", C.c_int64), ("rg2_sum", C.c_double),
                ("lam_sum", C.c_double * 3), ("b_sum", C.c_double), ("c_sum", C.c_double),
                ("kappa2_sum", C.c_double), ("bc_sum", C.c_double), ("g2_sum", C.c_double),
                ("re2_sum", C.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "lam_sum"}
        d["lam_sum"] = tuple(self.lam_sum)
        return d


EVENT_DTYPE = np.dtype([("unit", "<i8"), ("seq", "<i4"), ("pivot", "<i4"), ("kind", "<i4"),
                        ("pad", "<i4"), ("partner", "<i8"), ("x", "<f8")])

_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load libecmc.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
        lib = C.CDLL(path)
        P = C.POINTER
        vp = C.c_void_p
        sig = {
            "ecmc_create_lattice": [P(C.c_int32), C.c_double, C.c_double, C.c_uint64, C.c_int32,
                                    C.c_double, C.c_double, P(vp)],
            "ecmc_create": [P(C.c_double), C.c_double, C.c_int32, C.c_int32, C.c_double,
                            C.c_double, P(vp)],
            "ecmc_set_stream": [vp, vp],
            "ecmc_set_positions": [vp, P(C.c_double), P(C.c_int32)],
            "ecmc_get_positions": [vp, P(C.c_double), P(C.c_int32)],
            "ecmc_get_info": [vp, P(C.c_double), P(C.c_int64), P(C.c_int32)],
            "ecmc_configure": [vp, P(Opts)],
            "ecmc_run": [vp, C.c_double, C.c_int64, C.c_uint64, C.c_int64],
            "ecmc_swap": [vp, C.c_double],
            "ecmc_observables": [vp, P(Obs)],
            "ecmc_g1_reset": [vp],
            "ecmc_records": [vp, P(C.c_uint64), P(C.c_double), P(C.c_int64), P(C.c_int64)],
            "ecmc_log_reserve": [vp, C.c_int64],
            "ecmc_event_log": [vp, vp, C.c_int64, P(C.c_int64)],
            "ecmc_domain_tags": [vp, C.c_uint64, C.c_int64, P(C.c_int32), P(C.c_double)],
            "ecmc_checkpoint": [vp, C.c_char_p],
            "ecmc_restore": [vp, C.c_char_p],
            "ecmc_cells_static": [vp, C.c_int64, P(C.c_double), P(C.c_int32), C.c_double,
                                  C.c_double, C.c_uint64, C.c_int64, vp, vp, vp,
                                  P(C.c_double), vp],
            "ecmc_batch_create": [P(ReplicaSpec), C.c_int32, C.c_double, C.c_uint64, P(vp)],
            "ecmc_batch_configure": [vp, P(Opts)],
            "ecmc_batch_run": [vp, C.c_double, C.c_uint64, C.c_int64, C.c_int32],
            "ecmc_batch_get_positions": [vp, C.c_int32, P(C.c_double), P(C.c_int32)],
            "ecmc_batch_info": [vp, C.c_int32, P(C.c_int32), P(C.c_int64), P(C.c_int64)],
            "ecmc_batch_stats": [vp, P(C.c_int64), P(C.c_int64), P(C.c_double)],
            "ecmc_batch_records": [vp, P(C.c_uint64), P(C.c_double), P(C.c_int64),
                                   P(C.c_int64)],
            "ecmc_autotune": [vp, C.c_double, C.c_uint64, C.c_int32, P(Tuning)],
            "ecmc_batch_autotune": [vp, C.c_double, C.c_uint64, C.c_int32, P(Tuning)],
            "ecmc_structure": [vp, P(Struct), vp, C.c_double, C.c_int64, vp],
            "ecmc_phantom_chains": [P(C.c_double), C.c_int64, C.c_int32, C.c_double, C.c_double,
                                    C.c_uint64, P(C.c_double), P(C.c_int32)],
            "ecmc_create_phantom": [P(C.c_double), C.c_int64, C.c_int32, C.c_double, C.c_double,
                                    C.c_uint64, C.c_double, C.c_double, P(vp)],
            "ecmc_pushoff": [vp, C.c_double, C.c_int32, C.c_double, C.c_uint64, C.c_int64,
                             P(C.c_int64)],
            "ecmc_g1_track": [vp, C.c_int32, C.c_int32],
            "ecmc_g1_table": [vp, P(C.c_int64), P(C.c_double), P(C.c_int64), C.c_int32,
                              P(C.c_int32)],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = C.c_int
        lib.ecmc_destroy.argtypes = [vp]
        lib.ecmc_destroy.restype = None
        lib.ecmc_batch_destroy.argtypes = [vp]
        lib.ecmc_batch_destroy.restype = None
        lib.ecmc_last_error.argtypes = []
        lib.ecmc_last_error.restype = C.c_char_p
        _lib = lib
        return lib


def _check(rc):
    if rc != 0:
        raise EcmcError(rc, load().ecmc_last_error().decode())
    return rc


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def opts(mode=MODE_SERIAL, dir_mode=DIR_CART3, precision=PREC_FP64, tiles=(3, 3, 3), joint=0.0,
         s_cap=0.0, event_cap=0, p_swap=0.0, ecs_per_tile=0, lanes=0, record=0, stage_cap=0,
         cell_side=0.0, tile_side=0.0, schedule=0, block_tiles=0, request_cap=0,
         k_spring=0.0, tight_factor=0.0) -> Opts:
    o = Opts()
    o.mode, o.dir_mode, o.precision = int(mode), int(dir_mode), int(precision)
    for a in range(3):
        o.tiles[a] = int(tiles[a])
    o.joint, o.s_cap, o.event_cap = float(joint), float(s_cap), int(event_cap)
    o.p_swap, o.ecs_per_tile, o.lanes = float(p_swap), int(ecs_per_tile), int(lanes)
    o.record, o.stage_cap, o.cell_side = int(record), int(stage_cap), float(cell_side)
    o.tile_side = float(tile_side)
    o.schedule, o.block_tiles = int(schedule), int(block_tiles)
    o.request_cap = int(request_cap)
    o.k_spring = float(k_spring)
    o.tight_factor = float(tight_factor)
    return o


class Tuning(C.Structure):
    _fields_ = [("lanes", C.c_int32), ("tile_side", C.c_double), ("cell_side", C.c_double),
                ("ecs_per_tile", C.c_int32), ("tiles", C.c_int32 * 3), ("ecs_per_s", C.c_double),
                ("events_per_s", C.c_double), ("n_trials", C.c_int32), ("block_tiles", C.c_int32),
                ("tight_factor", C.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "tiles"}
        d["tiles"] = tuple(self.tiles)
        return d


class ReplicaSpec(C.Structure):
    _fields_ = [("dims", C.c_int32 * 3), ("spacing", C.c_double), ("N", C.c_int32),
                ("sigma", C.c_double), ("b_max", C.c_double)]


def phantom_chains(L, n_chains, N, bond=1.0, c=1.9, seed=0):
    """Phantom chains (ecmc_phantom_chains): wrapped positions (n x 3) and
    image counters of n_chains non-reversal random walks of N beads."""
    n = int(n_chains) * int(N)
    r = np.zeros((n, 3), dtype=np.float64)
    img = np.zeros((n, 3), dtype=np.int32)
    Lc = np.ascontiguousarray(L, dtype=np.float64)
    _check(load().ecmc_phantom_chains(_p(Lc, C.c_double), int(n_chains), int(N), float(bond),
                                      float(c), int(seed) & (2**64 - 1), _p(r, C.c_double),
                                      _p(img, C.c_int32)))
    return r, img


class Context:
    """One melt on the GPU (wraps an ecmc_ctx)."""

    def __init__(self, handle):
        self._h = handle
        box = np.zeros(3)
        n = C.c_int64()
        N = C.c_int32()
        _check(load().ecmc_get_info(self._h, _p(box, C.c_double), C.byref(n), C.byref(N)))
        self.L, self.n, self.N = box, n.value, N.value

    # ---- creation
    @classmethod
    def create_lattice(cls, dims, spacing, N, sigma=1.0, b_max=1.2, jitter=0.0, seed=0):
        h = C.c_void_p()
        d = np.asarray(dims, dtype=np.int32)
        _check(load().ecmc_create_lattice(_p(d, C.c_int32), float(spacing), float(jitter),
                                          int(seed) & (2**64 - 1), int(N), float(sigma),
                                          float(b_max), C.byref(h)))
        return cls(h)

    @classmethod
    def create_phantom(cls, box, n_chains, N, bond=1.0, c=1.9, seed=0, sigma=1.0, b_max=1.2):
        """Context of phantom chains (they may overlap until pushoff())."""
        h = C.c_void_p()
        b = np.ascontiguousarray(box, dtype=np.float64)
        _check(load().ecmc_create_phantom(_p(b, C.c_double), int(n_chains), int(N), float(bond),
                                          float(c), int(seed) & (2**64 - 1), float(sigma),
                                          float(b_max), C.byref(h)))
        return cls(h)

    def pushoff(self, f0=0.5, stages=5, ell=2.0, seed=0, max_sweeps=1000):
        """Slow push-off (ecmc_pushoff); returns the number of sweeps run."""
        n = C.c_int64(0)
        _check(load().ecmc_pushoff(self._h, float(f0), int(stages), float(ell),
                                   int(seed) & (2**64 - 1), int(max_sweeps), C.byref(n)))
        return n.value

    @classmethod
    def create(cls, phi, n_chains, N, sigma=1.0, b_max=1.2, box=None):
        h = C.c_void_p()
        b = np.zeros(3) if box is None else np.asarray(box, dtype=np.float64)
        _check(load().ecmc_create(_p(b, C.c_double), float(phi), int(n_chains), int(N),
                                  float(sigma), float(b_max), C.byref(h)))
        return cls(h)

    def autotune(self, ell, seed=0, trial_sweeps=2):
        """Pick lanes, tile side, cell side and ECs per tile by timed trials;
        the state is unchanged on return and the context runs the winner."""
        t = Tuning()
        _check(load().ecmc_autotune(self._h, float(ell), int(seed) & (2**64 - 1),
                                    int(trial_sweeps), C.byref(t)))
        return t.as_dict()

    def close(self):
        if self._h:
            load().ecmc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- state
    def set_stream(self, stream_ptr):
        _check(load().ecmc_set_stream(self._h, C.c_void_p(stream_ptr)))

    def set_positions(self, r, img=None):
        r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1, 3)
        im = None if img is None else np.ascontiguousarray(img, dtype=np.int32).reshape(-1, 3)
        _check(load().ecmc_set_positions(self._h, _p(r, C.c_double),
                                          None if im is None else _p(im, C.c_int32)))

    def get_positions(self, out=None):
        """Positions (n, 3) float64 and image counters (n, 3) int32.  `out`
        = (r, img) writes into caller-owned C-contiguous arrays instead (for
        instance pinned host memory, which the copy reaches fastest)."""
        if out is None:
            r = np.zeros((self.n, 3))
            img = np.zeros((self.n, 3), dtype=np.int32)
        else:
            r, img = out
            if not (r.dtype == np.float64 and img.dtype == np.int32 and r.shape == (self.n, 3)
                    and img.shape == (self.n, 3) and r.flags.c_contiguous
                    and img.flags.c_contiguous):
                raise ValueError("out must be C-contiguous float64 / int32 arrays of shape (n, 3)")
        _check(load().ecmc_get_positions(self._h, _p(r, C.c_double), _p(img, C.c_int32)))
        return r, img

    # ---- running
    def configure(self, **kw):
        o = opts(**kw)
        _check(load().ecmc_configure(self._h, C.byref(o)))

    def run(self, ell, chains_per_sweep=0, seed=0, n_sweeps=0):
        _check(load().ecmc_run(self._h, float(ell), int(chains_per_sweep),
                               int(seed) & (2**64 - 1), int(n_sweeps)))

    def swap(self, attempts_per_bead_per_sweep):
        _check(load().ecmc_swap(self._h, float(attempts_per_bead_per_sweep)))

    def observables(self) -> dict:
        o = Obs()
        _check(load().ecmc_observables(self._h, C.byref(o)))
        return o.as_dict()

    def structure(self, dR=0.5, nbins=0, r2n=True):
        """Chain structure of the current state (ecmc_structure): the sums
        over chains as a dict, R^2(n) (N values, or None) and the end-to-end
        histogram (nbins counts of width dR)."""
        o = Struct()
        nb = int(nbins)
        hist = np.zeros(max(nb, 1), dtype=np.int64)
        rn = np.zeros(self.N, dtype=np.float64) if r2n else None
        _check(load().ecmc_structure(self._h, C.byref(o),
                                     rn.ctypes.data_as(C.c_void_p) if rn is not None else None,
                                     float(dR), nb, hist.ctypes.data_as(C.c_void_p) if nb else None))
        return o.as_dict(), rn, hist[:nb]

    def g1_reset(self):
        _check(load().ecmc_g1_reset(self._h))

    def g1_track(self, P=0, K=0):
        """Start a g1 table over the lags j P^k sweeps (ecmc_g1_track);
        P = 0 stops tracking."""
        _check(load().ecmc_g1_track(self._h, int(P), int(K)))

    def g1_table(self, cap=1024):
        """(lags, g1, origin counts) of the current g1 table."""
        lag = np.zeros(cap, dtype=np.int64)
        g1 = np.zeros(cap)
        cnt = np.zeros(cap, dtype=np.int64)
        n = C.c_int32(0)
        _check(load().ecmc_g1_table(self._h, _p(lag, C.c_int64), _p(g1, C.c_double),
                                    _p(cnt, C.c_int64), int(cap), C.byref(n)))
        return lag[: n.value], g1[: n.value], cnt[: n.value]

    def records(self, cap):
        dig = np.zeros(cap, dtype=np.uint64)
        lift = np.zeros(cap)
        ev = np.zeros(cap, dtype=np.int64)
        n = C.c_int64(cap)
        _check(load().ecmc_records(self._h, _p(dig, C.c_uint64), _p(lift, C.c_double),
                                   _p(ev, C.c_int64), C.byref(n)))
        return dig[: n.value], lift[: n.value], ev[: n.value]

    def log_reserve(self, cap):
        _check(load().ecmc_log_reserve(self._h, int(cap)))

    def event_log(self, cap):
        buf = np.zeros(cap, dtype=EVENT_DTYPE)
        n = C.c_int64()
        _check(load().ecmc_event_log(self._h, buf.ctypes.data, int(cap), C.byref(n)))
        out = buf[: n.value]
        return out[np.lexsort((out["seq"], out["unit"]))]

    def domain_tags(self, seed, sweep):
        tags = np.zeros(self.n, dtype=np.int32)
        shift = np.zeros(3)
        _check(load().ecmc_domain_tags(self._h, int(seed) & (2**64 - 1), int(sweep),
                                       _p(tags, C.c_int32), _p(shift, C.c_double)))
        return tags, shift

    def checkpoint(self, path):
        _check(load().ecmc_checkpoint(self._h, str(path).encode()))

    def restore(self, path):
        _check(load().ecmc_restore(self._h, str(path).encode()))


def cells_static(d_r, n, box, tiles, joint, cell_side, seed, sweep, d_tags, d_cell_start,
                 d_cell_ids, stream=0):
    """ecmc_cells_static on caller-owned device buffers (device pointers as
    ints); returns the tile shift.  Allocates nothing on the device."""
    b = np.ascontiguousarray(box, dtype=np.float64)
    t = np.ascontiguousarray(tiles, dtype=np.int32)
    shift = np.zeros(3)
    _check(load().ecmc_cells_static(C.c_void_p(d_r), int(n), _p(b, C.c_double),
                                    _p(t, C.c_int32), float(joint), float(cell_side),
                                    int(seed) & (2**64 - 1), int(sweep), C.c_void_p(d_tags),
                                    C.c_void_p(d_cell_start), C.c_void_p(d_cell_ids),
                                    _p(shift, C.c_double), C.c_void_p(stream)))
    return shift


class Batch:
    """Many independent melts advanced together (wraps an ecmc_batch)."""

    def __init__(self, specs, jitter=0.0, seed=0):
        arr = (ReplicaSpec * len(specs))()
        for i, sp in enumerate(specs):
            for a in range(3):
                arr[i].dims[a] = int(sp["dims"][a])
            arr[i].spacing = float(sp["spacing"])
            arr[i].N = int(sp["N"])
            arr[i].sigma = float(sp.get("sigma", 1.0))
            arr[i].b_max = float(sp.get("b_max", 1.2))
        self._h = C.c_void_p()
        _check(load().ecmc_batch_create(arr, len(specs), float(jitter), int(seed) & (2**64 - 1),
                                        C.byref(self._h)))
        self.n = len(specs)

    def close(self):
        if self._h:
            load().ecmc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def configure(self, **kw):
        kw.setdefault("mode", MODE_DOMAIN)
        kw.setdefault("tiles", (0, 0, 0))
        o = opts(**kw)
        _check(load().ecmc_batch_configure(self._h, C.byref(o)))

    def run(self, ell, seed=0, n_sweeps=1, graph=True):
        _check(load().ecmc_batch_run(self._h, float(ell), int(seed) & (2**64 - 1), int(n_sweeps),
                                     1 if graph else 0))

    def autotune(self, ell, seed=0, trial_sweeps=2):
        """As Context.autotune, over the whole batch (per-replica tiles follow
        the chosen tile side)."""
        t = Tuning()
        _check(load().ecmc_batch_autotune(self._h, float(ell), int(seed) & (2**64 - 1),
                                          int(trial_sweeps), C.byref(t)))
        return t.as_dict()

    def info(self, r):
        t = np.zeros(3, dtype=np.int32)
        off = C.c_int64()
        nb = C.c_int64()
        _check(load().ecmc_batch_info(self._h, int(r), _p(t, C.c_int32), C.byref(off),
                                      C.byref(nb)))
        return tuple(int(x) for x in t), off.value, nb.value

    def get_positions(self, r):
        _, _, nb = self.info(r)
        x = np.zeros((nb, 3))
        img = np.zeros((nb, 3), dtype=np.int32)
        _check(load().ecmc_batch_get_positions(self._h, int(r), _p(x, C.c_double),
                                               _p(img, C.c_int32)))
        return x, img

    def stats(self):
        ev = C.c_int64()
        ecs = C.c_int64()
        sec = C.c_double()
        _check(load().ecmc_batch_stats(self._h, C.byref(ev), C.byref(ecs), C.byref(sec)))
        return {"events_total": ev.value, "ecs": ecs.value, "device_seconds": sec.value}

    def records(self, cap):
        dig = np.zeros(cap, dtype=np.uint64)
        lift = np.zeros(cap)
        ev = np.zeros(cap, dtype=np.int64)
        n = C.c_int64(cap)
        _check(load().ecmc_batch_records(self._h, _p(dig, C.c_uint64), _p(lift, C.c_double),
                                         _p(ev, C.c_int64), C.byref(n)))
        return dig[: n.value], lift[: n.value], ev[: n.value]
