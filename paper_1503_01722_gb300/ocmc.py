"""Thin ctypes binding of the engine's C ABI (include/ocmc.h).

Argument marshalling only: every step of the transport runs in the CUDA
library libocmc.so. Importing this module loads the library and raises if it
is missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# OCMC_CHECKS=1 selects the checks build (bounds checks on voxel indices, tally addresses and
# stack slots; build it with paper_1503_01722_gb300.build.build(checks=True))
_LIB_PATH = os.path.join(_HERE, "libocmc_checks.so" if os.environ.get("OCMC_CHECKS") == "1" else "libocmc.so")

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_OVERFLOW, ERR_TIMEOUT, ERR_STATE, ERR_BOUNDS = range(8)
FLAG_NO_HARD, FLAG_NO_MS, FLAG_KILL_FIRST_REAL, FLAG_KERMA, FLAG_CROSS_VOXELS = 1, 2, 4, 8, 16
TALLY_SCALE = 2.0 ** 28


class OcmcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"ocmc status {status}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("e_abs_e", C.c_float), ("e_abs_g", C.c_float), ("w_cc", C.c_float), ("w_cb", C.c_float),
                ("d_maxs", C.c_float), ("f_maxe", C.c_float), ("s_min", C.c_float),
                ("n_batches", C.c_int32), ("flags", C.c_int32),
                ("block_threads", C.c_int32), ("blocks_per_sm", C.c_int32), ("stack_capacity", C.c_int32),
                ("switch_high", C.c_int32), ("switch_low", C.c_int32), ("stream_tag", C.c_uint32),
                ("beamlet_capacity_scale", C.c_float), ("refill_min", C.c_int32), ("max_registers", C.c_int32),
                ("e_class_split", C.c_float)]


class Beamlet(C.Structure):
    _fields_ = [("field_x", C.c_float), ("field_y", C.c_float), ("ssd", C.c_float), ("iso", C.c_float * 3),
                ("dir", C.c_float * 3), ("n_histories", C.c_uint64)]


class Material(C.Structure):
    _fields_ = [("n_elements", C.c_int32), ("Z", C.c_int32 * 16), ("A", C.c_double * 16),
                ("mass_fraction", C.c_double * 16), ("I_eV", C.c_double), ("density", C.c_double)]


class Stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in (
        "histories", "photon_flights", "fictitious", "compton", "photo", "pair", "electron_steps", "moller",
        "brems", "hard_fictitious", "annihilations", "escaped", "missed", "geo_crossings",
        "majorant_violations", "dropped", "transmitted", "warp_iterations", "lane_steps")] + \
        [(n, C.c_double) for n in ("e_in", "e_dep", "e_esc", "e_miss", "pair_mass", "annih_mass", "e_killed",
                                   "e_trans", "e_dropped", "last_run_ms", "warp_ms", "tail_warp_ms", "span_ms",
                                   "tail_span_ms")] + [("warps", C.c_uint64)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} not found: build it with paper_1503_01722_gb300.build.build()")
    L = C.CDLL(_LIB_PATH)
    P = C.c_void_p
    sig = {
        "ocmc_default_params": (None, [C.POINTER(Params)]),
        "ocmc_init": (C.c_int, [C.POINTER(P), C.c_int, C.POINTER(Params)]),
        "ocmc_set_params": (C.c_int, [P, C.POINTER(Params)]),
        "ocmc_create_phantom": (C.c_int, [P, C.c_int, C.c_int, C.c_int, P, P, C.c_float, C.c_float, C.c_float]),
        "ocmc_set_source": (C.c_int, [P, C.c_int, C.c_int, P, P, C.c_float, C.c_float, C.c_float,
                                      C.POINTER(C.c_float), C.POINTER(C.c_float)]),
        "ocmc_run": (C.c_int, [P, C.c_uint64, C.c_uint64, P]),
        "ocmc_run_range": (C.c_int, [P, C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64, P]),
        "ocmc_get_dose": (C.c_int, [P, P, P, C.c_int]),
        "ocmc_get_raw_tally": (C.c_int, [P, P, C.c_int]),
        "ocmc_add_raw_tally": (C.c_int, [P, P, C.c_int, C.c_uint64, C.c_uint64]),
        "ocmc_reset_tally": (C.c_int, [P]),
        "ocmc_get_stats": (C.c_int, [P, C.POINTER(Stats)]),
        "ocmc_get_shape": (C.c_int, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
        "ocmc_last_error": (C.c_char_p, [P]),
        "ocmc_destroy": (None, [P]),
        "ocmc_test_philox": (C.c_int, [C.c_int, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                       C.c_uint32, C.c_uint32, P]),
        "ocmc_test_rotate": (C.c_int, [C.c_int, P, P, P, C.c_int, P]),
        "ocmc_test_source": (C.c_int, [P, C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64, P]),
        "ocmc_test_sample": (C.c_int, [P, C.c_int, C.c_int, C.c_float, C.c_float, C.c_uint64, C.c_uint64, P]),
        "ocmc_test_tables": (C.c_int, [P, C.c_int, P, C.c_int, P]),
        "ocmc_test_csda": (C.c_int, [P, C.c_int, P, P, C.c_int, P]),
        "ocmc_set_beamlets": (C.c_int, [P, C.c_int, C.c_int, P, P, C.c_int, P]),
        "ocmc_run_beamlets": (C.c_int, [P, C.c_uint64, P]),
        "ocmc_get_beamlet_dose": (C.c_int, [P, C.c_int, P, P, P, C.c_int64, C.POINTER(C.c_int64)]),
        "ocmc_autotune": (C.c_int, [P, C.c_uint64, C.POINTER(Params)]),
        "ocmc_set_phase_space": (C.c_int, [P, P, C.c_uint64, C.c_int]),
        "ocmc_set_materials": (C.c_int, [P, C.c_int, P]),
        "ocmc_load_phase_space": (C.c_int, [P, C.c_char_p]),
        "ocmc_unet_create": (C.c_int, [C.POINTER(P), C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64]),
        "ocmc_unet_destroy": (None, [P]),
        "ocmc_unet_last_error": (C.c_char_p, [P]),
        "ocmc_unet_num_params": (C.c_int, [P, C.POINTER(C.c_int64)]),
        "ocmc_unet_get_params": (C.c_int, [P, P, C.c_int]),
        "ocmc_unet_set_params": (C.c_int, [P, P]),
        "ocmc_unet_forward": (C.c_int, [P, P, P, P, P, P]),
        "ocmc_unet_train_step": (C.c_int, [P, P, P, P, P, C.c_float, C.POINTER(C.c_float), P]),
        "ocmc_unet_layer_times": (C.c_int, [P, P, P, P, C.c_int, P, C.POINTER(C.c_int)]),
        "ocmc_unet_test_layer": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                           P, P, P, P, P, P]),
        "ocmc_denoise": (C.c_int, [P, P, C.c_float, P, P, C.c_int]),
        "ocmc_unet_test_stall": (C.c_int, [C.c_int, C.c_uint64]),
        "ocmc_run_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, P, P, C.c_float, C.c_float, C.c_float,
                                       C.c_int, C.c_int, P, P, C.c_float, C.c_float, C.c_float,
                                       C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(Params),
                                       C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64, P, P, C.c_char_p,
                                       C.c_size_t]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()


def default_params(**kw) -> Params:
    p = Params()
    lib.ocmc_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    if "e_abs_e" in kw and "w_cc" not in kw:
        p.w_cc = p.e_abs_e
    if "e_abs_g" in kw and "w_cb" not in kw:
        p.w_cb = p.e_abs_g
    return p


def _ptr(a):
    """Host numpy array or CUDA tensor -> (void*, on_device)."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(a.ctypes.data), 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    raise TypeError(type(a))


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


class Engine:
    """One engine context on one GPU (ocmc_ctx)."""

    def __init__(self, device: int = 0, params: Params | None = None, **kw):
        self._c = C.c_void_p()
        p = params if params is not None else default_params(**kw)
        self._check(lib.ocmc_init(C.byref(self._c), device, C.byref(p)), init=True)
        self.params = p
        self.device = device
        self.shape = None

    def _check(self, status, init=False):
        if status != OK:
            msg = lib.ocmc_last_error(None if init else self._c).decode()
            raise OcmcError(status, msg)

    def close(self):
        if getattr(self, "_c", None) and self._c.value:
            lib.ocmc_destroy(self._c)
            self._c = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_params(self, params: Params | None = None, **kw):
        if params is None:
            params = Params.from_buffer_copy(self.params)
            for k, v in kw.items():
                setattr(params, k, v)
        self._check(lib.ocmc_set_params(self._c, C.byref(params)))
        self.params = params

    def set_materials(self, defs):
        """Define the materials: dicts with Z, A (g/mol), w (mass fractions), I (eV) and
        density (g/cm^3); voxel material m is defs[m]. Drops the current phantom."""
        arr = (Material * len(defs))()
        for k, d in enumerate(defs):
            n = len(d["Z"])
            arr[k].n_elements = n
            for i in range(n):
                arr[k].Z[i] = int(d["Z"][i])
                arr[k].A[i] = float(d["A"][i])
                arr[k].mass_fraction[i] = float(d["w"][i])
            arr[k].I_eV = float(d["I"])
            arr[k].density = float(d["density"])
        self._check(lib.ocmc_set_materials(self._c, len(defs), C.cast(arr, C.c_void_p)))

    def create_phantom(self, phantom=None, *, density=None, material=None, voxel=None):
        """phantom: object with .density (nz,ny,nx) float32, .material uint8, .voxel (dx,dy,dz)."""
        if phantom is not None:
            density, material, voxel = phantom.density, phantom.material, phantom.voxel
        d = np.ascontiguousarray(density, np.float32)
        m = np.ascontiguousarray(material, np.uint8)
        nz, ny, nx = d.shape
        self._check(lib.ocmc_create_phantom(self._c, nx, ny, nz, C.c_void_p(d.ctypes.data),
                                            C.c_void_p(m.ctypes.data), *map(float, voxel)))
        self.shape = (nz, ny, nx)

    def set_source(self, beam=None, *, particle=None, edges=None, weights=None, field=None, ssd=None,
                   iso=None, direction=None):
        if beam is not None:
            particle, edges, weights = beam.particle, beam.edges, beam.weights
            field, ssd, iso, direction = beam.field, beam.ssd, beam.iso, beam.direction
        e = np.ascontiguousarray(edges, np.float32)
        w = np.ascontiguousarray(weights, np.float32)
        iso_c = (C.c_float * 3)(*iso)
        dir_c = (C.c_float * 3)(*direction)
        self._check(lib.ocmc_set_source(self._c, int(particle), len(w), C.c_void_p(e.ctypes.data),
                                        C.c_void_p(w.ctypes.data), float(field[0]), float(field[1]),
                                        float(ssd), iso_c, dir_c))

    def set_phase_space(self, records):
        """Phase-space source: a structured array of 32-byte records (x, y, z, u, v, w, E as
        float32, type as int32; see ocmc_inputs.PS_DTYPE) in host memory, or a CUDA uint8/
        int32/float32 tensor holding the same bytes."""
        if isinstance(records, np.ndarray):
            r = np.ascontiguousarray(records)
            if r.dtype.itemsize != 32:
                raise ValueError("records must be 32-byte structured records")
            self._check(lib.ocmc_set_phase_space(self._c, C.c_void_p(r.ctypes.data), len(r), 0))
        else:
            pt, dev = _ptr(records)
            nbytes = records.numel() * records.element_size()
            if nbytes % 32:
                raise ValueError("tensor size must be a multiple of 32 bytes")
            self._check(lib.ocmc_set_phase_space(self._c, pt, nbytes // 32, dev))

    def load_phase_space(self, path):
        self._check(lib.ocmc_load_phase_space(self._c, os.fsencode(str(path))))

    def run(self, n_histories: int, seed: int = 1, stream=None):
        self._check(lib.ocmc_run(self._c, int(n_histories), int(seed), _stream_ptr(stream)))

    def run_range(self, first: int, count: int, n_total: int, seed: int = 1, stream=None):
        self._check(lib.ocmc_run_range(self._c, int(first), int(count), int(n_total), int(seed),
                                       _stream_ptr(stream)))

    def dose(self, out=None, sigma=True):
        """Dose (MeV/g per source particle) and batch sigma as (nz,ny,nx) arrays.
        `out` may be a (dose, sigma) pair of CUDA tensors to write on the device."""
        if out is not None:
            d, s = out
            pd, dev = _ptr(d)
            ps = _ptr(s)[0] if s is not None else None
            self._check(lib.ocmc_get_dose(self._c, pd, ps, dev))
            return d, s
        d = np.empty(self.shape, np.float32)
        s = np.empty(self.shape, np.float32) if sigma else None
        self._check(lib.ocmc_get_dose(self._c, C.c_void_p(d.ctypes.data),
                                      C.c_void_p(s.ctypes.data) if sigma else None, 0))
        return d, s

    def raw_tally(self, out=None):
        nvox, B = C.c_int64(), C.c_int32()
        self._check(lib.ocmc_get_shape(self._c, C.byref(nvox), C.byref(B)))
        if out is not None:
            p, dev = _ptr(out)
            self._check(lib.ocmc_get_raw_tally(self._c, p, dev))
            return out
        t = np.empty((B.value,) + self.shape, np.int64)
        self._check(lib.ocmc_get_raw_tally(self._c, C.c_void_p(t.ctypes.data), 0))
        return t

    def add_raw_tally(self, tally, first: int, count: int):
        p, dev = _ptr(tally if not isinstance(tally, np.ndarray) else np.ascontiguousarray(tally, np.int64))
        self._check(lib.ocmc_add_raw_tally(self._c, p, dev, int(first), int(count)))

    def reset(self):
        self._check(lib.ocmc_reset_tally(self._c))

    def stats(self) -> dict:
        s = Stats()
        self._check(lib.ocmc_get_stats(self._c, C.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    # ---- batched beamlets ----
    def set_beamlets(self, particle, edges, weights, beamlets):
        """beamlets: sequence of dicts/objects with field (fx, fy), ssd, iso, direction, n_histories."""
        e = np.ascontiguousarray(edges, np.float32)
        w = np.ascontiguousarray(weights, np.float32)
        arr = (Beamlet * len(beamlets))()
        for i, b in enumerate(beamlets):
            g = b if isinstance(b, dict) else b.__dict__
            arr[i].field_x, arr[i].field_y = map(float, g["field"])
            arr[i].ssd = float(g["ssd"])
            arr[i].iso[:] = [float(v) for v in g["iso"]]
            arr[i].dir[:] = [float(v) for v in g["direction"]]
            arr[i].n_histories = int(g["n_histories"])
        self._check(lib.ocmc_set_beamlets(self._c, int(particle), len(w), C.c_void_p(e.ctypes.data),
                                          C.c_void_p(w.ctypes.data), len(beamlets), arr))
        self.n_beamlets = len(beamlets)

    def run_beamlets(self, seed=1, stream=None):
        self._check(lib.ocmc_run_beamlets(self._c, int(seed), _stream_ptr(stream)))

    def beamlet_dose(self, b):
        """(voxel indices int32, dose float32 MeV/g per history, raw int64) in voxel order."""
        nnz = C.c_int64()
        self._check(lib.ocmc_get_beamlet_dose(self._c, int(b), None, None, None, 0, C.byref(nnz)))
        n = nnz.value
        idx = np.empty(n, np.int32)
        dose = np.empty(n, np.float32)
        raw = np.empty(n, np.int64)
        self._check(lib.ocmc_get_beamlet_dose(self._c, int(b), C.c_void_p(idx.ctypes.data),
                                              C.c_void_p(dose.ctypes.data), C.c_void_p(raw.ctypes.data), n,
                                              C.byref(nnz)))
        return idx, dose, raw

    def beamlet_doses(self, raw=False):
        """Every beamlet's sparse dose, [(voxel indices int32, dose float32 MeV/g per history
        [, raw int64])] in beamlet order: one extraction per beamlet into reusable pinned host
        buffers of one phantom's size (no size query, no pageable copies)."""
        import torch
        if self.shape is None:
            raise OcmcError(ERR_STATE, "no phantom")
        nvox = int(np.prod(self.shape))
        if getattr(self, "_bl_buf", None) is None or self._bl_buf[0].numel() < nvox:
            self._bl_buf = (torch.empty(nvox, dtype=torch.int32).pin_memory(),
                            torch.empty(nvox, dtype=torch.float32).pin_memory(),
                            torch.empty(nvox, dtype=torch.int64).pin_memory())
        bi, bd, br = self._bl_buf
        nnz = C.c_int64()
        out = []
        for b in range(self.n_beamlets):
            self._check(lib.ocmc_get_beamlet_dose(self._c, b, C.c_void_p(bi.data_ptr()), C.c_void_p(bd.data_ptr()),
                                                  C.c_void_p(br.data_ptr()) if raw else None, nvox, C.byref(nnz)))
            n = nnz.value
            item = (bi[:n].numpy().copy(), bd[:n].numpy().copy())
            out.append(item + (br[:n].numpy().copy(),) if raw else item)
        return out

    def autotune(self, pilot_histories):
        p = Params()
        self._check(lib.ocmc_autotune(self._c, int(pilot_histories), C.byref(p)))
        self.params = p
        return p

    # ---- building blocks for the tests ----
    def test_source(self, n_total, first=0, count=None, seed=1):
        count = n_total - first if count is None else count
        out = np.empty((count, 8), np.float32)
        self._check(lib.ocmc_test_source(self._c, n_total, first, count, seed, C.c_void_p(out.ctypes.data)))
        return out

    def test_sample(self, kind, E, n, seed=1, material=0, aux=0.0):
        out = np.empty(n, np.float32)
        self._check(lib.ocmc_test_sample(self._c, kind, material, float(E), float(aux), n, seed,
                                         C.c_void_p(out.ctypes.data)))
        return out

    def test_tables(self, material, E):
        E = np.ascontiguousarray(E, np.float32)
        out = np.empty((len(E), 8), np.float32)
        self._check(lib.ocmc_test_tables(self._c, material, C.c_void_p(E.ctypes.data), len(E),
                                         C.c_void_p(out.ctypes.data)))
        return out

    def test_csda(self, material, T, X):
        T = np.ascontiguousarray(T, np.float32)
        X = np.ascontiguousarray(X, np.float32)
        out = np.empty(len(T), np.float32)
        self._check(lib.ocmc_test_csda(self._c, material, C.c_void_p(T.ctypes.data), C.c_void_p(X.ctypes.data),
                                       len(T), C.c_void_p(out.ctypes.data)))
        return out


def test_philox(key, c1, c2, c3, first_block, n_blocks, device=0):
    out = np.empty((n_blocks, 4), np.uint32)
    st = lib.ocmc_test_philox(device, key[0], key[1], c1, c2, c3, first_block, n_blocks,
                              C.c_void_p(out.ctypes.data))
    if st != OK:
        raise OcmcError(st, lib.ocmc_last_error(None).decode())
    return out


def unet_test_stall(tile=-1, wait_ns=0):
    """Test hook of the tensor-memory convolution's bounded waits (ocmc_unet_test_stall):
    tile >= 0 makes every later launch time out at that block-local tile; -1 turns it off."""
    st = lib.ocmc_unet_test_stall(int(tile), int(wait_ns))
    if st != OK:
        raise OcmcError(st, "ocmc_unet_test_stall failed")


def test_rotate(dirs, mu, xi, device=0):
    """The transport kernel's rotation (ocmc_test_rotate): rows of `dirs` turned by polar cosine
    `mu` and azimuth 2 pi `xi`."""
    d = np.ascontiguousarray(dirs, np.float32).reshape(-1, 3)
    m = np.ascontiguousarray(mu, np.float32).reshape(-1)
    x = np.ascontiguousarray(xi, np.float32).reshape(-1)
    if not (len(d) == len(m) == len(x)):
        raise ValueError("dirs, mu and xi must have the same length")
    out = np.empty_like(d)
    st = lib.ocmc_test_rotate(device, C.c_void_p(d.ctypes.data), C.c_void_p(m.ctypes.data),
                              C.c_void_p(x.ctypes.data), len(d), C.c_void_p(out.ctypes.data))
    if st != OK:
        raise OcmcError(st, lib.ocmc_last_error(None).decode())
    return out


SAMPLE_COMPTON, SAMPLE_MOLLER, SAMPLE_BREMS, SAMPLE_MS = 0, 1, 2, 3


def run_noalloc(density, material, voxel, beam, tally, first, count, n_total, seed=1, params=None, device=0,
                stream=None):
    """Allocation-free transport (ocmc_run_noalloc) for callers that cannot allocate
    device memory: `density` (float32), `material` (uint8) and `tally` (int64,
    n_batches x nz x ny x nx, added into) are CUDA tensors the caller owns; every
    scratch buffer is the library's fixed static device array. Calls that overlap on
    the GPU share that array and must be serialised by the caller."""
    import torch
    p = params if params is not None else default_params()
    for name, t, dtype in (("density", density, torch.float32), ("material", material, torch.uint8),
                           ("tally", tally, torch.int64)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.device.index != device:
            raise ValueError(f"{name} must be a CUDA tensor on device {device}")
        if t.dtype != dtype or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {dtype} tensor")
    if density.dim() != 3 or tuple(material.shape) != tuple(density.shape):
        raise ValueError("density and material must have the same shape (nz, ny, nx)")
    nz, ny, nx = density.shape
    if tuple(tally.shape) != (int(p.n_batches), nz, ny, nx):
        raise ValueError(f"tally must have shape (n_batches={int(p.n_batches)}, {nz}, {ny}, {nx})")
    pd, _ = _ptr(density)
    pm, _ = _ptr(material)
    pt, _ = _ptr(tally)
    e = np.ascontiguousarray(beam.edges, np.float32)
    w = np.ascontiguousarray(beam.weights, np.float32)
    msg = C.create_string_buffer(256)
    st = lib.ocmc_run_noalloc(device, nx, ny, nz, pd, pm, *map(float, voxel), int(beam.particle), len(w),
                              C.c_void_p(e.ctypes.data), C.c_void_p(w.ctypes.data), float(beam.field[0]),
                              float(beam.field[1]), float(beam.ssd), (C.c_float * 3)(*beam.iso),
                              (C.c_float * 3)(*beam.direction), C.byref(p), int(first), int(count), int(n_total),
                              int(seed), pt, _stream_ptr(stream), msg, 256)
    if st != OK:
        raise OcmcError(st, msg.value.decode())


class UNet:
    """The 3D U-Net dose denoiser (ocmc_unet). Dose/density/target arguments are
    CUDA tensors of the network's grid shape (nz, ny, nx), float32."""

    def __init__(self, shape, device=0, seed=1):
        nz, ny, nx = shape
        self._u = C.c_void_p()
        st = lib.ocmc_unet_create(C.byref(self._u), device, nx, ny, nz, int(seed))
        if st != OK:
            raise OcmcError(st, "ocmc_unet_create failed")
        self.shape = tuple(shape)
        n = C.c_int64()
        self._check(lib.ocmc_unet_num_params(self._u, C.byref(n)))
        self.num_params = n.value

    def _check(self, st):
        if st != OK:
            raise OcmcError(st, lib.ocmc_unet_last_error(self._u).decode())

    def close(self):
        if getattr(self, "_u", None) and self._u.value:
            lib.ocmc_unet_destroy(self._u)
            self._u = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self, grads=False):
        out = np.empty(self.num_params, np.float32)
        self._check(lib.ocmc_unet_get_params(self._u, C.c_void_p(out.ctypes.data), 1 if grads else 0))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        self._check(lib.ocmc_unet_set_params(self._u, C.c_void_p(p.ctypes.data)))

    def forward(self, dose, density, out, stream=None, sigma=None):
        sg = _ptr(sigma)[0] if sigma is not None else None
        self._check(lib.ocmc_unet_forward(self._u, _ptr(dose)[0], sg, _ptr(density)[0], _ptr(out)[0],
                                          _stream_ptr(stream)))
        return out

    def layer_times(self, dose, density, repeats=10, sigma=None):
        """Mean forward time of each layer in ms (CUDA events around every layer)."""
        n = C.c_int()
        sg = _ptr(sigma)[0] if sigma is not None else None
        self._check(lib.ocmc_unet_layer_times(self._u, _ptr(dose)[0], sg, _ptr(density)[0], 1, None, C.byref(n)))
        out = np.empty(n.value, np.float32)
        self._check(lib.ocmc_unet_layer_times(self._u, _ptr(dose)[0], sg, _ptr(density)[0], int(repeats),
                                              C.c_void_p(out.ctypes.data), C.byref(n)))
        return out

    def train_step(self, dose, density, target, lr, stream=None, sigma=None):
        loss = C.c_float()
        sg = _ptr(sigma)[0] if sigma is not None else None
        self._check(lib.ocmc_unet_train_step(self._u, _ptr(dose)[0], sg, _ptr(density)[0], _ptr(target)[0],
                                             float(lr), C.byref(loss), _stream_ptr(stream)))
        return loss.value


def unet_test_layer(mode, fine_shape, cin, cout, x, w, dy, device=0):
    """One layer through the denoiser's kernels: returns (y, dx, dw)."""
    nz, ny, nx = fine_shape
    x = np.ascontiguousarray(x, np.float32)
    w = np.ascontiguousarray(w, np.float32)
    dy = np.ascontiguousarray(dy, np.float32)
    y = np.empty(dy.shape, np.float32)
    dx = np.empty(x.shape, np.float32)
    dw = np.empty(w.shape, np.float32)
    st = lib.ocmc_unet_test_layer(device, mode, nx, ny, nz, cin, cout, *(C.c_void_p(a.ctypes.data)
                                                                        for a in (x, w, dy, y, dx, dw)))
    if st != OK:
        raise OcmcError(st, "ocmc_unet_test_layer failed")
    return y, dx, dw


def denoise(engine, net, k_sigma, out, flag=None):
    """ocmc_denoise: denoised dose of the engine's current tally with plain-MC fallback."""
    po, dev = _ptr(out)
    pf = _ptr(flag)[0] if flag is not None else None
    engine._check(lib.ocmc_denoise(engine._c, net._u, float(k_sigma), po, pf, dev))
    return out, flag
