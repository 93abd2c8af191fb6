"""Oracle for the event-chain (EC) Monte Carlo move of tethered hard-sphere
bead chains (arXiv:1502.06447, Sec. II and Sec. II.A-D).

TEST INFRASTRUCTURE ONLY.  This is the plain, serial, FP64 checker that the
CUDA library is compared against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  It shares no code with the CUDA library (own Philox4x64-10, own geometry,
own cell list) and neither side imports the other.

The arithmetic lives in ``ecmc_oracle.c`` (compiled with
``-O2 -ffp-contract=off``: every FP64 expression evaluated as written; the
only fused multiply-adds are explicit C99 ``fma`` calls, one rounding each).
This module is ctypes marshalling only.

Functions and the passage each follows:
  run_serial / run_domain   EC move, Sec. II (four-step rule, min over
                            partners); tile-joint decomposition and
                            reflections, Sec. II.A, Fig. 2c; swap, Sec. II.C
  domain_tags               tile-joint partition, Sec. II.A
  lattice                   initial lattice melt (a reading: the paper grows
                            random walks instead; the lattice start is the
                            workload's stated synthetic input)
  chain_obs                 end-to-end distance R_e^2 (Sec. IV), bond lengths
  min_pair                  hard-sphere constraint check, Eq. 1
  chain_struct              gyration tensor and centre of mass (R_g and g2,
                            Sec. IV; moment of inertia tensor, Appendix A),
                            internal distances R^2(n) (Sec. II.B), end-to-end
                            distance histogram W(R) (Appendix A)
  shape_descriptors         eigenvalues of the gyration tensor, asphericity,
                            acylindricity, shape anisotropy (Appendix A)
  phantom_chains            non-reversal random walks without excluded volume,
                            the first stage of the initial configuration
                            (Sec. II.B)
  k_spring (System)         bead-spring chains: harmonic bonds with Boltzmann
                            energies per event instead of tethers (Sec. II)
  pushoff, overlap_flags    slow push-off of overlapping chains: the
                            diameter grows in stages, ECs start at the
                            overlapping beads and ignore their pivot's
                            overlaps (Sec. II.B)
  g1_table                  the middle bead's mean-square displacement g1
                            (Sec. IV, Eq. 3) over log-spaced lags, averaged
                            over chains and time origins
All functions are pinned by the ``tests/test_oracle_*.py`` files.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "ecmc_oracle.c")]
_HDR = [os.path.join(_HERE, "orc.h")]
_SO = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_SERIAL, MODE_DOMAIN = 0, 1
DIR_CART3, DIR_ISO, DIR_PLUSX = 0, 1, 2
OUT_NAMES = ("end", "pass", "wall", "hs_lift", "hs_reflect", "te_lift",
             "te_reflect", "swap")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE FP64, no implicit contraction)."""
    newest = max(os.path.getmtime(p) for p in _SRC + _HDR)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp] + _SRC + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class Params(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("N", C.c_int32), ("mode", C.c_int32),
        ("L", C.c_double * 3), ("sigma", C.c_double), ("b_max", C.c_double),
        ("s_cap", C.c_double), ("dir_mode", C.c_int32), ("D", C.c_int32 * 3),
        ("w", C.c_double), ("p_swap", C.c_double), ("event_cap", C.c_int64),
        ("use_cells", C.c_int32), ("ecs_per_tile", C.c_int32),
        ("seed", C.c_uint64), ("replica", C.c_uint64),
        ("pushoff", C.c_int32), ("pad_po", C.c_int32), ("po_flag", C.c_void_p),
        ("k_spring", C.c_double), ("tile_mod", C.c_int32), ("tile_rem", C.c_int32),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("ecs", C.c_int64), ("events", C.c_int64), ("out", C.c_int64 * 8),
        ("swap_tried", C.c_int64), ("lift_sum", C.c_double),
        ("refl_sum", C.c_double), ("disp_sum", C.c_double),
        ("status", C.c_int64),
    ]

    def as_dict(self) -> dict:
        d = {"ecs": self.ecs, "events": self.events,
             "swap_tried": self.swap_tried, "lift_sum": self.lift_sum,
             "refl_sum": self.refl_sum, "disp_sum": self.disp_sum,
             "status": self.status}
        for k, name in enumerate(OUT_NAMES):
            d[name] = self.out[k]
        return d


EVENT_DTYPE = np.dtype([("unit", "<i8"), ("pivot", "<i4"), ("kind", "<i4"),
                        ("partner", "<i8"), ("x", "<f8")])


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER
            lib.orc_philox4x64_10.argtypes = [P(C.c_uint64), P(C.c_uint64), P(C.c_uint64)]
            lib.orc_philox4x64_10.restype = None
            run_args = [P(Params), P(C.c_double), P(C.c_int32), C.c_int64, C.c_int64,
                        C.c_double, P(Stats), P(C.c_uint64), P(C.c_double),
                        P(C.c_int64), C.c_void_p, C.c_int64, P(C.c_int64)]
            lib.orc_run_serial.argtypes = run_args
            lib.orc_run_domain.argtypes = run_args
            lib.orc_run_serial.restype = C.c_int
            lib.orc_run_domain.restype = C.c_int
            lib.orc_domain_tags.argtypes = [P(Params), P(C.c_double), C.c_uint64,
                                            P(C.c_int32), P(C.c_double)]
            lib.orc_lattice.argtypes = [P(C.c_int32), C.c_double, C.c_double, C.c_uint64,
                                        C.c_uint64, P(C.c_double)]
            lib.orc_chain_obs.argtypes = [P(Params), P(C.c_double), P(C.c_double),
                                          P(C.c_double)]
            lib.orc_min_pair.argtypes = [P(Params), P(C.c_double), P(C.c_double),
                                         P(C.c_int64)]
            lib.orc_min_pair_cells.argtypes = lib.orc_min_pair.argtypes
            lib.orc_spring_x.argtypes = [P(C.c_double), P(C.c_double), C.c_double, C.c_double,
                                         C.c_double]
            lib.orc_spring_x.restype = C.c_double
            lib.orc_log.argtypes = [C.c_double]
            lib.orc_log.restype = C.c_double
            lib.orc_overlap_flags.argtypes = [P(Params), P(C.c_double), C.c_double, C.c_void_p]
            lib.orc_overlap_flags.restype = C.c_int64
            lib.orc_pushoff.argtypes = [P(Params), P(C.c_double), P(C.c_int32), C.c_double,
                                        C.c_int32, C.c_double, C.c_int64, C.c_int64,
                                        P(C.c_int64), P(Stats)]
            lib.orc_phantom.argtypes = [P(C.c_double), C.c_int64, C.c_int32, C.c_double,
                                        C.c_double, C.c_uint64, P(C.c_double), P(C.c_int32)]
            lib.orc_chain_struct.argtypes = [P(Params), P(C.c_double), C.c_void_p, C.c_void_p,
                                             C.c_void_p, C.c_double, C.c_int64, C.c_void_p]
            lib.orc_contacts.argtypes = [P(Params), P(C.c_double), C.c_double, P(C.c_int64),
                                         P(C.c_int64)]
            lib.orc_start_draws.argtypes = [P(Params), C.c_int64, C.c_int64, P(C.c_int64),
                                            P(C.c_double)]
            _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def philox4x64_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib.orc_philox4x64_10(_ptr(c, C.c_uint64), _ptr(k, C.c_uint64), _ptr(out, C.c_uint64))
    return out


def lattice(dims, a: float, jitter: float = 0.0, seed: int = 0, replica: int = 0) -> np.ndarray:
    """Snake-ordered simple-cubic lattice, optionally jittered (Philox tag 4)."""
    lib = _load()
    d = np.asarray(dims, dtype=np.int32)
    r = np.zeros((int(np.prod(d)), 3), dtype=np.float64)
    lib.orc_lattice(_ptr(d, C.c_int32), float(a), float(jitter), int(seed) & (2**64 - 1),
                    int(replica) & (2**64 - 1), _ptr(r, C.c_double))
    return r


class System:
    """One melt: positions (n,3) wrapped in [0,L), image counters, parameters."""

    def __init__(self, r, L, N, sigma=1.0, b_max=1.2, s_cap=0.25, mode=MODE_SERIAL,
                 dir_mode=DIR_CART3, D=(1, 1, 1), w=None, p_swap=0.0,
                 event_cap=10_000_000, use_cells=1, ecs_per_tile=1, seed=0,
                 replica=0, img=None, k_spring=0.0, tile_mod=0, tile_rem=0):
        self.r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1, 3).copy()
        self.img = (np.zeros_like(self.r, dtype=np.int32) if img is None
                    else np.ascontiguousarray(img, dtype=np.int32).reshape(-1, 3).copy())
        p = Params()
        p.n = self.r.shape[0]
        p.N = int(N)
        p.mode = int(mode)
        Lv = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
        for a in range(3):
            p.L[a] = float(Lv[a])
            p.D[a] = int(np.broadcast_to(np.asarray(D), (3,))[a])
        p.sigma = float(sigma)
        p.b_max = float(b_max)
        p.s_cap = float(s_cap)
        p.dir_mode = int(dir_mode)
        p.w = float(b_max if w is None else w)
        p.p_swap = float(p_swap)
        p.event_cap = int(event_cap)
        p.use_cells = int(use_cells)
        p.ecs_per_tile = int(ecs_per_tile)
        p.seed = int(seed) & (2**64 - 1)
        p.replica = int(replica) & (2**64 - 1)
        p.k_spring = float(k_spring)
        p.tile_mod, p.tile_rem = int(tile_mod), int(tile_rem)
        self.P = p

    @property
    def L(self) -> np.ndarray:
        return np.array([self.P.L[0], self.P.L[1], self.P.L[2]])

    def _run(self, fn, start, count, ell, digests, log_cap, units):
        lib = _load()
        st = Stats()
        dig = np.zeros(units, dtype=np.uint64) if digests else None
        lift = np.zeros(units, dtype=np.float64) if digests else None
        nev = np.zeros(units, dtype=np.int64) if digests else None
        log = np.zeros(max(log_cap, 1), dtype=EVENT_DTYPE) if log_cap else None
        log_n = C.c_int64(0)
        rc = fn(C.byref(self.P), _ptr(self.r, C.c_double), _ptr(self.img, C.c_int32),
                int(start), int(count), float(ell), C.byref(st),
                _ptr(dig, C.c_uint64) if dig is not None else None,
                _ptr(lift, C.c_double) if lift is not None else None,
                _ptr(nev, C.c_int64) if nev is not None else None,
                log.ctypes.data if log is not None else None, int(log_cap),
                C.byref(log_n))
        res = {"rc": rc, "stats": st.as_dict()}
        if digests:
            res.update(digest=dig, ec_lift=lift, ec_events=nev)
        if log is not None:
            res["log"] = log[: log_n.value]
        return res

    def run_serial(self, n_ec, ell, ec0=0, digests=False, log_cap=0):
        """n_ec serial ECs of length ell (Sec. II); ECs numbered from ec0."""
        return self._run(_load().orc_run_serial, ec0, n_ec, ell, digests, log_cap,
                         int(n_ec))

    def run_domain(self, n_sweeps, ell, sweep0=0, digests=False, log_cap=0):
        """Domain-decomposed sweeps (Sec. II.A), one EC per tile per sweep x
        ecs_per_tile; sweeps numbered from sweep0."""
        nt = self.P.D[0] * self.P.D[1] * self.P.D[2]
        units = int(n_sweeps) * nt * self.P.ecs_per_tile
        return self._run(_load().orc_run_domain, sweep0, n_sweeps, ell, digests,
                         log_cap, units)

    def domain_tags(self, sweep):
        lib = _load()
        tags = np.zeros(self.r.shape[0], dtype=np.int32)
        shift = np.zeros(3, dtype=np.float64)
        lib.orc_domain_tags(C.byref(self.P), _ptr(self.r, C.c_double), int(sweep),
                            _ptr(tags, C.c_int32), _ptr(shift, C.c_double))
        return tags, shift

    def chain_obs(self):
        lib = _load()
        nch = self.r.shape[0] // self.P.N
        re2 = np.zeros(nch)
        bonds = np.zeros(max(nch * (self.P.N - 1), 1))
        lib.orc_chain_obs(C.byref(self.P), _ptr(self.r, C.c_double), _ptr(re2, C.c_double),
                          _ptr(bonds, C.c_double))
        return re2, bonds[: nch * (self.P.N - 1)]

    def min_pair(self, cells=None):
        lib = _load()
        dmin = C.c_double(0)
        cnt = C.c_int64(0)
        use_cells = self.r.shape[0] > 3000 if cells is None else cells
        fn = lib.orc_min_pair_cells if use_cells else lib.orc_min_pair
        fn(C.byref(self.P), _ptr(self.r, C.c_double), C.byref(dmin), C.byref(cnt))
        return dmin.value, cnt.value

    def contacts(self, delta):
        """Pair counts in the two shells of width delta above sigma and bond
        counts in the two shells below b_max (every pair, brute force)."""
        lib = _load()
        pairs = np.zeros(2, dtype=np.int64)
        bonds = np.zeros(2, dtype=np.int64)
        lib.orc_contacts(C.byref(self.P), _ptr(self.r, C.c_double), float(delta),
                         _ptr(pairs, C.c_int64), _ptr(bonds, C.c_int64))
        return pairs, bonds

    def contact_pressure(self, delta):
        """betaP/rho from the contact values (virial theorem for hard
        constraints): 1 + [sigma f(sigma+) - b_max f_b(b_max-)] / (3 n), with
        f, f_b the pair and bond counts per unit distance at contact, each
        extrapolated linearly from its two shells."""
        pairs, bonds = self.contacts(delta)
        fs = (1.5 * pairs[0] - 0.5 * pairs[1]) / delta
        fb = (1.5 * bonds[0] - 0.5 * bonds[1]) / delta
        return 1.0 + (self.P.sigma * fs - self.P.b_max * fb) / (3.0 * self.P.n)

    def start_draws(self, n, ec0=0):
        """Start bead and direction of serial ECs ec0..ec0+n-1."""
        lib = _load()
        idx = np.zeros(int(n), dtype=np.int64)
        v = np.zeros((int(n), 3), dtype=np.float64)
        lib.orc_start_draws(C.byref(self.P), int(ec0), int(n), _ptr(idx, C.c_int64),
                            _ptr(v, C.c_double))
        return idx, v

    def unwrapped(self):
        return self.r + self.img * self.L

    def overlap_flags(self, d):
        """Beads overlapping another bead at diameter d (flags, count)."""
        lib = _load()
        flag = np.zeros(self.r.shape[0], dtype=np.uint8)
        m = lib.orc_overlap_flags(C.byref(self.P), _ptr(self.r, C.c_double), float(d),
                                  flag.ctypes.data_as(C.c_void_p))
        return flag, int(m)

    def pushoff(self, f0, stages, ell, max_sweeps, sweep0=0):
        """Slow push-off in the domain mode with this system's tiles, seed
        and key; returns (rc, sweeps, stats)."""
        lib = _load()
        st = Stats()
        n_sw = C.c_int64(0)
        rc = lib.orc_pushoff(C.byref(self.P), _ptr(self.r, C.c_double), _ptr(self.img, C.c_int32),
                             float(f0), int(stages), float(ell), int(max_sweeps), int(sweep0),
                             C.byref(n_sw), C.byref(st))
        return rc, n_sw.value, st.as_dict()

    def chain_struct(self, dR=0.5, nbins=0, r2n=True):
        """Gyration tensor per chain (S_xx, S_xy, S_xz, S_yy, S_yz, S_zz),
        the middle bead relative to the centre of mass, R^2(n) for n < N
        and the end-to-end distance histogram (bins of width dR, the last
        taking the rest), all from positions along each chain built from
        minimum-image bonds."""
        lib = _load()
        nch = self.r.shape[0] // self.P.N
        gyr = np.zeros((nch, 6))
        mid = np.zeros((nch, 3))
        rn = np.zeros(self.P.N) if r2n else None
        hist = np.zeros(max(int(nbins), 1), dtype=np.int64)
        vp = lambda a: a.ctypes.data_as(C.c_void_p) if a is not None else None
        rc = lib.orc_chain_struct(C.byref(self.P), _ptr(self.r, C.c_double), vp(gyr), vp(mid),
                                  vp(rn), float(dR), int(nbins), vp(hist) if nbins else None)
        if rc != 0:
            raise RuntimeError(f"orc_chain_struct: {rc}")
        return {"gyr": gyr, "mid": mid, "r2n": rn, "hist": hist[: int(nbins)]}


def phantom_chains(L, n_chains, N, bond=1.0, c=1.9, seed=0):
    """Phantom chains (Sec. II.B): wrapped positions (n_chains N x 3) and
    image counters of non-reversal random walks with stiffness c."""
    lib = _load()
    n = int(n_chains) * int(N)
    r = np.zeros((n, 3))
    img = np.zeros((n, 3), dtype=np.int32)
    Lc = np.ascontiguousarray(L, dtype=np.float64)
    lib.orc_phantom(_ptr(Lc, C.c_double), int(n_chains), int(N), float(bond), float(c),
                    int(seed) & (2**64 - 1), _ptr(r, C.c_double), _ptr(img, C.c_int32))
    return r, img


def spring_x(d, v, sigma, k, dE) -> float:
    """Spring event distance of a pivot at separation d (pivot minus
    bonded bead) moving along unit v with consumable energy dE."""
    dd = np.ascontiguousarray(d, dtype=np.float64)
    vv = np.ascontiguousarray(v, dtype=np.float64)
    return float(_load().orc_spring_x(_ptr(dd, C.c_double), _ptr(vv, C.c_double), float(sigma),
                                      float(k), float(dE)))


def own_log(u: float) -> float:
    """The oracle's own natural logarithm (behind the springs' Boltzmann
    energies)."""
    return float(_load().orc_log(float(u)))


def g1_table(traj, P, K):
    """g1 of Sec. IV, Eq. 3, over the log-spaced lags j P^k (k < K,
    1 <= j < P): traj[t] holds the unwrapped middle beads (chains x 3) after
    sweep t (t = 0 the start).  The origins of lag j P^k are the sweeps t0
    that are multiples of P^k with t0 + j P^k <= T.  Returns (lags, g1,
    counts, sums): for every end sweep t in increasing order and every lag
    whose origin t - lag qualifies, the chains' (dx^2 + dy^2) + dz^2 are
    added in chain order and that sum is added to the lag's total; g1 =
    total / (origins x chains)."""
    traj = np.asarray(traj, dtype=np.float64)
    T = traj.shape[0] - 1
    nch = traj.shape[1]
    lags, sums, cnts = [], [], []
    pks = [P ** k for k in range(K)]
    for k in range(K):
        for j in range(1, P):
            lags.append(j * pks[k])
    sums = [0.0] * len(lags)
    cnts = [0] * len(lags)
    for t in range(1, T + 1):
        for k in range(K):
            pk = pks[k]
            if t % pk != 0:
                continue
            for j in range(1, P):
                if t // pk < j:
                    continue
                q = k * (P - 1) + (j - 1)
                a, b = traj[t], traj[t - j * pk]
                s = 0.0
                for ch in range(nch):
                    d0 = float(a[ch, 0]) - float(b[ch, 0])
                    d1 = float(a[ch, 1]) - float(b[ch, 1])
                    d2 = float(a[ch, 2]) - float(b[ch, 2])
                    s = s + ((d0 * d0 + d1 * d1) + d2 * d2)
                sums[q] = sums[q] + s
                cnts[q] += 1
    g1 = [sums[q] / (cnts[q] * nch) if cnts[q] else 0.0 for q in range(len(lags))]
    return (np.array(lags, dtype=np.int64), np.array(g1), np.array(cnts, dtype=np.int64),
            np.array(sums))


def seq_sum(x) -> float:
    """Left-to-right sum in index order (the order the library sums chains in)."""
    x = np.asarray(x, dtype=np.float64)
    return float(np.cumsum(x)[-1]) if x.size else 0.0


def shape_descriptors(gyr):
    """Per-chain shape from the gyration tensor S (Appendix A): T = Tr S =
    R_g^2; P = lam1 lam2 + lam2 lam3 + lam3 lam1 (the sum of the principal
    2x2 minors); eigenvalues lam1 <= lam2 <= lam3 (numpy.linalg.eigvalsh);
    asphericity b = lam3 - (lam1 + lam2)/2; acylindricity c = lam2 - lam1;
    shape anisotropy kappa2 = 1 - 3 P / T^2; 4 b^2 + 3 c^2 = 4 (T^2 - 3 P).
    The moment of inertia tensor of a chain is N (T 1 - S): its eigenvalues
    taken in descending order I1 >= I2 >= I3 are N (T - lam1) ... so that
    I1 + I2 - I3 = 2 N lam3, I1 - I2 + I3 = 2 N lam2, -I1 + I2 + I3 = 2 N lam1
    and Tr I = 2 N T (the reading under which the paper's ratios and limits
    hold)."""
    g = np.asarray(gyr, dtype=np.float64)
    sxx, sxy, sxz, syy, syz, szz = (g[:, k] for k in range(6))
    T = (sxx + syy) + szz
    P = ((sxx * syy - sxy * sxy) + (sxx * szz - sxz * sxz)) + (syy * szz - syz * syz)
    M = np.empty((g.shape[0], 3, 3))
    M[:, 0, 0], M[:, 0, 1], M[:, 0, 2] = sxx, sxy, sxz
    M[:, 1, 0], M[:, 1, 1], M[:, 1, 2] = sxy, syy, syz
    M[:, 2, 0], M[:, 2, 1], M[:, 2, 2] = sxz, syz, szz
    lam = np.linalg.eigvalsh(M)  # ascending
    b = lam[:, 2] - 0.5 * (lam[:, 0] + lam[:, 1])
    c = lam[:, 1] - lam[:, 0]
    kappa2 = 1.0 - 3.0 * P / (T * T)
    bc = 4.0 * (T * T - 3.0 * P)
    return {"T": T, "P": P, "lam": lam, "b": b, "c": c, "kappa2": kappa2, "bc": bc}


def g2_terms(mid_ref, mid):
    """Per-chain squared displacement of the middle bead relative to the
    centre of mass (the summand of g2, Sec. IV)."""
    d = np.asarray(mid, dtype=np.float64) - np.asarray(mid_ref, dtype=np.float64)
    return (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
