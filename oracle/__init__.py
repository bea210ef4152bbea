"""ctypes front end of the CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline and
reference legs may import this package. It wraps ``ocmc_oracle.c`` (plain C,
double precision), which shares no code with the CUDA engine.

``run`` splits a history range over host threads (ctypes releases the GIL
during the C call); every thread owns its tally, and the int64 tallies are
summed, so the result does not depend on the thread count.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ocmc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

N_COUNTERS = 24
N_LEDGER = 12
COUNTERS = ["flights", "fictitious", "compton", "photo", "pair", "esteps", "moller", "brems",
            "hard_fict", "escaped", "viol_photon", "viol_electron", "stack_overflow",
            "transmitted", "geo_cross", "annih", "missed"]
LEDGER = ["e_in", "e_dep", "e_esc", "e_miss", "pair_mass", "annih_mass", "e_killed",
          "e_path", "e_trans"]

NO_HARD, NO_MS, KILL_FIRST_REAL, KERMA, CROSS_VOXELS = 1, 2, 4, 8, 16
TALLY_SCALE = 2.0 ** 28


def build(force=False):
    """Compile the oracle with gcc (portable flags, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ocmc_oracle.h"))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"],
                   check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("e_abs_e", C.c_double), ("e_abs_g", C.c_double), ("w_cc", C.c_double),
                ("w_cb", C.c_double), ("d_maxs", C.c_double), ("f_maxe", C.c_double),
                ("s_min", C.c_double), ("n_batches", C.c_int32), ("flags", C.c_int32)]


MAX_MAT, MAX_ELEM = 16, 16


class _Material(C.Structure):
    _fields_ = [("n_elements", C.c_int32), ("Z", C.c_int32 * MAX_ELEM), ("A", C.c_double * MAX_ELEM),
                ("mass_fraction", C.c_double * MAX_ELEM), ("I_eV", C.c_double), ("density", C.c_double)]


class _Phantom(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("density", C.POINTER(C.c_float)), ("material", C.POINTER(C.c_uint8))]


class _Source(C.Structure):
    _fields_ = [("particle", C.c_int32), ("n_bins", C.c_int32),
                ("edges", C.POINTER(C.c_float)), ("weights", C.POINTER(C.c_float)),
                ("field_x", C.c_double), ("field_y", C.c_double), ("ssd", C.c_double),
                ("iso", C.c_double * 3), ("dir", C.c_double * 3)]


def params(e_abs_e=0.2, e_abs_g=0.01, w_cc=None, w_cb=None, d_maxs=0.5, f_maxe=0.05,
           s_min=1e-4, n_batches=10, flags=0):
    """Default cutoffs: electrons 200 keV, photons 10 keV; hard-event thresholds
    equal to the absorption energies (W_cc = E_abs,e, W_cb = E_abs,gamma)."""
    return Params(e_abs_e, e_abs_g, e_abs_e if w_cc is None else w_cc,
                  e_abs_g if w_cb is None else w_cb, d_maxs, f_maxe, s_min, n_batches, flags)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            d, i, u64 = C.c_double, C.c_int, C.c_uint64
            for name, res, args in [
                ("orc_init", None, []),
                ("orc_mu", d, [i, d, i]), ("orc_sigma_kn", d, [d]),
                ("orc_L_col", d, [i, d, d]), ("orc_L_rad", d, [i, d, d]),
                ("orc_sigma_moller", d, [i, d, d]), ("orc_sigma_brems", d, [i, d, d]),
                ("orc_lambda1_inv", d, [i, d]), ("orc_density_effect", d, [i, d]),
                ("orc_material_const", d, [i, i]), ("orc_ms_mean_u", d, [d]),
                ("orc_ms_solve_A", d, [d]),
                ("orc_csda_loss", d, [i, d, d, C.POINTER(Params)]),
                ("orc_philox", None, [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]),
                ("orc_sample", i, [i, i, d, d, u64, u64, C.POINTER(Params), C.POINTER(d)]),
                ("orc_event", i, [i, i, d, d, C.POINTER(d), u64, u64, C.POINTER(Params), C.POINTER(d)]),
                ("orc_rotate", None, [C.POINTER(d), d, d, C.POINTER(d)]),
                ("orc_stratify", i, [i, C.POINTER(C.c_float), C.POINTER(C.c_float), u64,
                                     C.POINTER(u64), C.POINTER(C.c_int32)]),
                ("orc_source_sample", i, [C.POINTER(_Phantom), C.POINTER(_Source), u64, u64, u64, u64,
                                          C.POINTER(d)]),
                ("orc_run", i, [C.POINTER(_Phantom), C.POINTER(_Source), C.POINTER(Params), u64, u64, u64,
                                u64, C.POINTER(C.c_int64), C.POINTER(d), C.POINTER(u64)]),
                ("orc_set_materials", i, [i, C.c_void_p]),
                ("orc_reset_materials", None, []), ("orc_n_materials", i, []),
                ("orc_ps_sample", i, [C.POINTER(_Phantom), C.c_void_p, u64, u64, u64, C.POINTER(d)]),
                ("orc_run_ps", i, [C.POINTER(_Phantom), C.c_void_p, u64, C.POINTER(Params), u64, u64, u64,
                                   C.POINTER(C.c_int64), C.POINTER(d), C.POINTER(u64)]),
            ]:
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            L.orc_init()
            _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


# ---- physics accessors (vectorised over E) -----------------------------------------
def _vec(fn, *args):
    E = args[-1]
    if np.ndim(E) == 0:
        return fn(*args)
    return np.array([fn(*args[:-1], float(e)) for e in np.ravel(E)]).reshape(np.shape(E))


def mu(m, E, channel=0):
    L = lib()
    return _vec(lambda mm, e: L.orc_mu(mm, e, channel), m, E)


def sigma_kn(E):
    return _vec(lib().orc_sigma_kn, E)


def L_col(m, T, w_cc=0.2):
    L = lib()
    return _vec(lambda mm, t: L.orc_L_col(mm, t, w_cc), m, T)


def L_rad(m, T, w_cb=0.01):
    L = lib()
    return _vec(lambda mm, t: L.orc_L_rad(mm, t, w_cb), m, T)


def sigma_moller(m, T, w_cc=0.2):
    L = lib()
    return _vec(lambda mm, t: L.orc_sigma_moller(mm, t, w_cc), m, T)


def sigma_brems(m, T, w_cb=0.01):
    L = lib()
    return _vec(lambda mm, t: L.orc_sigma_brems(mm, t, w_cb), m, T)


def lambda1_inv(m, T):
    return _vec(lib().orc_lambda1_inv, m, T)


def density_effect(m, T):
    return _vec(lib().orc_density_effect, m, T)


def material_const(m, which):
    return lib().orc_material_const(m, which)


def ms_mean_u(A):
    return lib().orc_ms_mean_u(A)


def ms_solve_A(G1):
    return lib().orc_ms_solve_A(G1)


def csda_loss(m, T, X, p=None):
    p = p or params()
    return lib().orc_csda_loss(m, T, X, C.byref(p))


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox(c, k, o)
    return np.array(list(o), dtype=np.uint32)


SAMPLE_KN_MU, SAMPLE_MOLLER_EPS, SAMPLE_BREMS_K, SAMPLE_MS_MU = 0, 1, 2, 3


EVENT_KINDS = {"compton": 0, "moller": 1, "brems": 2, "annihilation": 3, "rotation": 4}


def event(kind, E, d0, n, seed=1, m=0, aux=0.0, p=None):
    """n single interactions of one kind from unit direction d0 (see orc_event). Returns
    (Ea, da, Eb, db): energies (n,) and unit directions (n, 3) of the two outgoing particles."""
    p = params() if p is None else p
    out = np.zeros((n, 8), np.float64)
    d = np.ascontiguousarray(np.asarray(d0, np.float64).reshape(3))
    rc = lib().orc_event(EVENT_KINDS[kind], m, float(E), float(aux), _ptr(d, C.c_double), n, seed,
                         C.byref(p), _ptr(out, C.c_double))
    if rc != 0:
        raise ValueError("orc_event failed")
    return out[:, 0], out[:, 1:4], out[:, 4], out[:, 5:8]


def rotate(dirs, mu, phi):
    """Rows of dirs turned by polar cosine mu and azimuth phi (the rotation every event uses)."""
    dirs = np.asarray(dirs, np.float64).reshape(-1, 3)
    mu = np.broadcast_to(np.asarray(mu, np.float64), (len(dirs),))
    phi = np.broadcast_to(np.asarray(phi, np.float64), (len(dirs),))
    out = np.empty_like(dirs)
    L = lib()
    o = np.empty(3, np.float64)
    for j in range(len(dirs)):
        dj = np.ascontiguousarray(dirs[j])
        L.orc_rotate(_ptr(dj, C.c_double), float(mu[j]), float(phi[j]), _ptr(o, C.c_double))
        out[j] = o
    return out


def sample(kind, E, n, seed=1, m=0, aux=0.0, p=None):
    p = p or params()
    out = np.empty(n, np.float64)
    rc = lib().orc_sample(kind, m, float(E), float(aux), n, seed, C.byref(p), _ptr(out, C.c_double))
    if rc != 0:
        raise ValueError("orc_sample failed")
    return out


def stratify(edges, weights, n_total):
    edges = np.ascontiguousarray(edges, np.float32)
    weights = np.ascontiguousarray(weights, np.float32)
    nb = len(weights)
    bounds = np.empty(nb + 1, np.uint64)
    order = np.empty(nb, np.int32)
    rc = lib().orc_stratify(nb, _ptr(edges, C.c_float), _ptr(weights, C.c_float), n_total,
                            _ptr(bounds, C.c_uint64), _ptr(order, C.c_int32))
    if rc != 0:
        raise ValueError("bad spectrum")
    return bounds, order


class _Keep:
    """Keeps numpy buffers alive for the duration of a C call."""

    def __init__(self, ph, beam):
        self.density = np.ascontiguousarray(ph.density, np.float32)
        self.material = np.ascontiguousarray(ph.material, np.uint8)
        self.edges = np.ascontiguousarray(beam.edges, np.float32)
        self.weights = np.ascontiguousarray(beam.weights, np.float32)
        nx, ny, nz = ph.shape_xyz
        self.ph = _Phantom(nx, ny, nz, ph.voxel[0], ph.voxel[1], ph.voxel[2],
                           _ptr(self.density, C.c_float), _ptr(self.material, C.c_uint8))
        self.src = _Source(beam.particle, len(self.weights), _ptr(self.edges, C.c_float),
                           _ptr(self.weights, C.c_float), float(beam.field[0]), float(beam.field[1]),
                           float(beam.ssd), (C.c_double * 3)(*beam.iso), (C.c_double * 3)(*beam.direction))


def source_sample(ph, beam, n_total, first=0, count=None, seed=1):
    count = n_total - first if count is None else count
    k = _Keep(ph, beam)
    out = np.empty((count, 8), np.float64)
    rc = lib().orc_source_sample(C.byref(k.ph), C.byref(k.src), seed, n_total, first, count,
                                 _ptr(out, C.c_double))
    if rc != 0:
        raise ValueError("orc_source_sample failed")
    return out


class Result:
    def __init__(self, tally, ledger, counters, n_hist, ph):
        self.tally = tally              # int64 (B, nz, ny, nx), units 2^-28 MeV
        self.ledger = dict(zip(LEDGER, ledger[:len(LEDGER)]))
        self.counters = dict(zip(COUNTERS, counters[:len(COUNTERS)].tolist()))
        self.n_hist = n_hist
        self.ph = ph

    def dose(self):
        """Dose in MeV/g per source particle and its batch standard error
        (Sec. 3.1: sigma_D of the local dose; batch method)."""
        return finalize(self.tally, self.ph, self.n_hist)


def finalize(tally, ph, n_hist):
    """D_v = sum_b tally_bv / (2^28 rho_v V N); sigma from the B batch means."""
    B = tally.shape[0]
    V = ph.voxel[0] * ph.voxel[1] * ph.voxel[2]
    rho = ph.density.astype(np.float64)
    mass = np.where(rho > 0, rho * V, np.inf)
    E = tally.astype(np.float64) / TALLY_SCALE            # MeV per batch
    nb = np.array([(n_hist - b + B - 1) // B for b in range(B)], np.float64)
    Db = E / mass[None] / np.maximum(nb, 1)[(...,) + (None,) * 3]
    D = E.sum(0) / mass / max(n_hist, 1)
    if B > 1:
        sig = np.sqrt(((Db - D[None]) ** 2).sum(0) / (B * (B - 1)))
    else:
        sig = np.zeros_like(D)
    return D, sig


def run(ph, beam, n_hist, seed=1, p=None, first=0, count=None, threads=None, n_total=None):
    """Transport histories [first, first+count) of a run of n_total histories."""
    p = p or params()
    n_total = n_hist if n_total is None else n_total
    count = n_hist - first if count is None else count
    threads = threads or os.cpu_count() or 1
    threads = max(1, min(threads, count if count > 0 else 1))
    k = _Keep(ph, beam)
    nvox = ph.density.size
    B = p.n_batches
    chunks = np.linspace(first, first + count, threads + 1).astype(np.int64)
    L = lib()

    def work(t):
        tally = np.zeros(B * nvox, np.int64)
        ledger = np.zeros(N_LEDGER, np.float64)
        cnt = np.zeros(N_COUNTERS, np.uint64)
        a, b = int(chunks[t]), int(chunks[t + 1])
        if b > a:
            rc = L.orc_run(C.byref(k.ph), C.byref(k.src), C.byref(p), seed, n_total, a, b - a,
                           _ptr(tally, C.c_int64), _ptr(ledger, C.c_double), _ptr(cnt, C.c_uint64))
            if rc != 0:
                raise ValueError(f"orc_run failed ({rc})")
        return tally, ledger, cnt

    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(work, range(threads)))
    tally = sum(p_[0] for p_ in parts).reshape((B,) + ph.density.shape)
    ledger = sum(p_[1] for p_ in parts)
    cnt = sum(p_[2] for p_ in parts)
    return Result(tally, ledger, cnt, count, ph)


# ---- phase-space source (Sec. 2.2 "Materials": particles from a file or a user's model) -----
def _ps_records(records):
    r = np.ascontiguousarray(records)
    if r.dtype.itemsize != 32 or len(r) == 0:
        raise ValueError("records: 32-byte structured array (x, y, z, u, v, w, E float32; type int32)")
    return r


def ps_sample(ph, records, first=0, count=None):
    """Entry state of histories [first, first+count) of a phase-space source: rows
    (x, y, z, u, v, w, E, entered)."""
    r = _ps_records(records)
    count = len(r) - first if count is None else count
    k = _Keep(ph, _NoBeam)
    out = np.empty((count, 8), np.float64)
    rc = lib().orc_ps_sample(C.byref(k.ph), C.c_void_p(r.ctypes.data), len(r), first, count,
                             _ptr(out, C.c_double))
    if rc != 0:
        raise ValueError("orc_ps_sample failed (invalid records)")
    return out


def run_ps(ph, records, n_hist, seed=1, p=None, first=0, count=None, threads=None):
    """Transport histories [first, first+count) of a phase-space source (history h starts
    from record h mod len(records))."""
    p = p or params()
    r = _ps_records(records)
    count = n_hist - first if count is None else count
    threads = threads or os.cpu_count() or 1
    threads = max(1, min(threads, count if count > 0 else 1))
    k = _Keep(ph, _NoBeam)
    nvox = ph.density.size
    B = p.n_batches
    chunks = np.linspace(first, first + count, threads + 1).astype(np.int64)
    L = lib()

    def work(t):
        tally = np.zeros(B * nvox, np.int64)
        ledger = np.zeros(N_LEDGER, np.float64)
        cnt = np.zeros(N_COUNTERS, np.uint64)
        a, b = int(chunks[t]), int(chunks[t + 1])
        if b > a:
            rc = L.orc_run_ps(C.byref(k.ph), C.c_void_p(r.ctypes.data), len(r), C.byref(p), seed, a, b - a,
                              _ptr(tally, C.c_int64), _ptr(ledger, C.c_double), _ptr(cnt, C.c_uint64))
            if rc != 0:
                raise ValueError(f"orc_run_ps failed ({rc})")
        return tally, ledger, cnt

    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(work, range(threads)))
    tally = sum(p_[0] for p_ in parts).reshape((B,) + ph.density.shape)
    ledger = sum(p_[1] for p_ in parts)
    cnt = sum(p_[2] for p_ in parts)
    return Result(tally, ledger, cnt, count, ph)


class _NoBeam:
    """Placeholder beam for the phantom-only ctypes structure of the phase-space calls."""
    particle, edges, weights = 0, np.zeros(2, np.float32), np.ones(1, np.float32)
    field, ssd, iso, direction = (0.0, 0.0), 0.0, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0)


# ---- user-defined materials (the paper's material database, generalised) ----------------------
def _material_array(defs):
    arr = (_Material * len(defs))()
    for k, d in enumerate(defs):
        n = len(d["Z"])
        arr[k].n_elements = n
        for i in range(n):
            arr[k].Z[i] = int(d["Z"][i])
            arr[k].A[i] = float(d["A"][i])
            arr[k].mass_fraction[i] = float(d["w"][i])
        arr[k].I_eV = float(d["I"])
        arr[k].density = float(d["density"])
    return arr


def set_materials(defs):
    """Replace the materials (process-wide) by compositions: dicts with Z, A (g/mol), w (mass
    fractions), I (eV) and density (g/cm^3). Material m of a phantom is defs[m]."""
    arr = _material_array(defs)
    if lib().orc_set_materials(len(defs), C.cast(arr, C.c_void_p)) != 0:
        raise ValueError("bad material definition")


def reset_materials():
    lib().orc_reset_materials()


def n_materials():
    return lib().orc_n_materials()
