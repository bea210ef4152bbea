"""Seeded synthetic inputs shared by the CUDA engine's tests/bench and the oracle.

This module holds none of the transport method's arithmetic: it only builds
phantoms (density + material grids) and beam descriptions (energy bin edges
and weights, field, SSD, direction) shaped like the workloads of Tian et al.
(oclMC), Sec. 2.2 "Materials": a homogeneous water phantom, a water/bone/lung
slab phantom and a half-slab phantom irradiated by a 15 MeV electron beam or
a 6 MV photon beam from a point source at SSD 100 cm.

Material indices: 0 water, 1 cortical bone (ICRP, 1.85 g/cm^3),
2 lung (ICRP, 0.26 g/cm^3). Arrays are x-fastest: index = x + nx*(y + ny*z),
stored as numpy arrays of shape (nz, ny, nx).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

WATER, BONE, LUNG = 0, 1, 2
RHO = {WATER: 1.0, BONE: 1.85, LUNG: 0.26}

# Public compositions (ICRU Report 46 / ICRP tissue compositions and common physics materials):
# elements Z, standard atomic masses A (g/mol), mass fractions w, mean excitation energy I (eV)
# and nominal density (g/cm^3). Inputs for user-defined material sets; no method arithmetic.
_A = {1: 1.008, 6: 12.011, 7: 14.007, 8: 15.999, 11: 22.990, 12: 24.305, 13: 26.982, 15: 30.974,
      16: 32.06, 17: 35.45, 19: 39.098, 20: 40.078, 26: 55.845, 29: 63.546, 30: 65.38, 53: 126.90}


def _mat(zw, I, rho):
    Z = [z for z, _ in zw]
    return {"Z": Z, "A": [_A[z] for z in Z], "w": [w for _, w in zw], "I": I, "density": rho}


MATERIALS = {
    "water": _mat([(1, 0.111894), (8, 0.888106)], 75.0, 1.0),
    "bone_cortical": _mat([(1, 0.047234), (6, 0.144330), (7, 0.041990), (8, 0.446096), (12, 0.002200),
                           (15, 0.104970), (16, 0.003150), (20, 0.209930), (30, 0.000100)], 106.4, 1.85),
    "lung": _mat([(1, 0.101278), (6, 0.102310), (7, 0.028650), (8, 0.757072), (11, 0.001840), (12, 0.000730),
                  (15, 0.000800), (16, 0.002250), (17, 0.002660), (19, 0.001940), (20, 0.000090),
                  (26, 0.000370), (30, 0.000010)], 75.3, 0.26),
    "adipose": _mat([(1, 0.114), (6, 0.598), (7, 0.007), (8, 0.278), (11, 0.001), (16, 0.001), (17, 0.001)],
                    63.2, 0.95),
    "muscle": _mat([(1, 0.102), (6, 0.143), (7, 0.034), (8, 0.710), (11, 0.001), (15, 0.002), (16, 0.003),
                    (17, 0.001), (19, 0.004)], 75.3, 1.05),
    "pmma": _mat([(1, 0.080538), (6, 0.599848), (8, 0.319614)], 74.0, 1.19),
    "aluminium": _mat([(13, 1.0)], 166.0, 2.699),
    "copper": _mat([(29, 1.0)], 322.0, 8.96),
    "hydrogen_rich_gel": _mat([(1, 0.14), (6, 0.10), (8, 0.76)], 70.0, 1.02),
}
MATERIAL_ORDER = ["water", "bone_cortical", "lung", "adipose", "muscle", "pmma", "aluminium", "copper",
                  "hydrogen_rich_gel"]


def material_set(names):
    return [MATERIALS[n] for n in names]


@dataclasses.dataclass
class Phantom:
    density: np.ndarray   # float32 (nz, ny, nx), g/cm^3
    material: np.ndarray  # uint8 (nz, ny, nx)
    voxel: tuple          # (dx, dy, dz) cm

    @property
    def shape_xyz(self):
        nz, ny, nx = self.density.shape
        return nx, ny, nz

    @property
    def size_cm(self):
        nx, ny, nz = self.shape_xyz
        return nx * self.voxel[0], ny * self.voxel[1], nz * self.voxel[2]


@dataclasses.dataclass
class Beam:
    particle: int            # 0 photon, 1 electron
    edges: np.ndarray        # float32 (n_bins+1,) MeV
    weights: np.ndarray      # float32 (n_bins,)
    field: tuple             # (fx, fy) cm, in the plane through iso normal to dir
    ssd: float               # cm; <= 0 means a parallel beam
    iso: tuple               # field centre (cm)
    direction: tuple         # beam axis (unit vector)


def homogeneous(n, voxel, material=WATER, density=None):
    nx, ny, nz = n
    rho = RHO[material] if density is None else density
    d = np.full((nz, ny, nx), rho, dtype=np.float32)
    m = np.full((nz, ny, nx), material, dtype=np.uint8)
    return Phantom(d, m, tuple(float(v) for v in voxel))


def _layered(n, voxel, layers, half=False):
    """layers: list of (z0, z1, material) in cm from the entrance surface z=0.
    With half=True the layers cover only x < Lx/2 for bone and x >= Lx/2 for
    lung (the half-slab phantom); elsewhere water."""
    nx, ny, nz = n
    ph = homogeneous(n, voxel, WATER)
    zc = (np.arange(nz) + 0.5) * voxel[2]
    xc = (np.arange(nx) + 0.5) * voxel[0]
    lx = nx * voxel[0]
    for z0, z1, mat in layers:
        zsel = (zc >= z0) & (zc < z1)
        if not half:
            ph.material[zsel] = mat
            ph.density[zsel] = RHO[mat]
        else:
            xsel = xc < lx / 2 if mat == BONE else xc >= lx / 2
            sel = zsel[:, None, None] & np.ones((1, ny, 1), bool) & xsel[None, None, :]
            ph.material[sel] = mat
            ph.density[sel] = RHO[mat]
    return ph


def slab(n=(120, 120, 120), voxel=(0.25, 0.25, 0.25), layers=((3.0, 5.0, BONE), (5.0, 12.0, LUNG))):
    """Water with a bone layer and a lung layer along z (water beyond)."""
    return _layered(n, voxel, layers)


def half_slab(n=(120, 120, 120), voxel=(0.25, 0.25, 0.25)):
    """Bone for x < Lx/2 and lung for x >= Lx/2 over depths 3-10 cm; water elsewhere."""
    return _layered(n, voxel, ((3.0, 10.0, BONE), (3.0, 10.0, LUNG)), half=True)


def ct_like(n=(256, 256, 128), voxel=(0.2, 0.2, 0.2), seed=1):
    """Synthetic CT-like phantom: water-body ellipsoid with 3-8 random inserts,
    densities uniform in [0.2, 1.9]; density thresholds pick the material
    (< 0.6 lung, 0.6-1.3 water, > 1.3 bone). Outside the body: air-like 0.0012 water."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    lx, ly, lz = nx * voxel[0], ny * voxel[1], nz * voxel[2]
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) * voxel[2], (np.arange(ny) + 0.5) * voxel[1],
                          (np.arange(nx) + 0.5) * voxel[0], indexing="ij")
    dens = np.full((nz, ny, nx), 0.0012, np.float32)
    body = ((x - lx / 2) / (0.45 * lx)) ** 2 + ((y - ly / 2) / (0.35 * ly)) ** 2 + ((z - lz / 2) / (0.48 * lz)) ** 2 <= 1
    dens[body] = 1.0
    for _ in range(int(rng.integers(3, 9))):
        c = rng.uniform([0.3 * lx, 0.35 * ly, 0.2 * lz], [0.7 * lx, 0.65 * ly, 0.8 * lz])
        r = rng.uniform([1.0, 1.0, 1.0], [0.12 * lx, 0.1 * ly, 0.2 * lz])
        sel = (((x - c[0]) / r[0]) ** 2 + ((y - c[1]) / r[1]) ** 2 + ((z - c[2]) / r[2]) ** 2 <= 1) & body
        dens[sel] = np.float32(rng.uniform(0.2, 1.9))
    mat = np.full(dens.shape, WATER, np.uint8)
    mat[dens < 0.6] = LUNG
    mat[dens > 1.3] = BONE
    mat[~body] = WATER
    return Phantom(dens, mat, tuple(float(v) for v in voxel))


def spectrum_6mv(n_bins=24, lo=0.25, hi=6.0):
    """Closed-form stand-in for a 6 MV bremsstrahlung spectrum,
    phi(E) ~ ((6 - E)/E) (1 - exp(-(E/1.3)^2)) on [0.25, 6] MeV (mean ~2.0 MeV),
    integrated over n_bins equal-width bins (Simpson, 64 panels per bin)."""
    edges = np.linspace(lo, hi, n_bins + 1)
    w = np.empty(n_bins)
    for i in range(n_bins):
        e = np.linspace(edges[i], edges[i + 1], 129)
        f = ((6.0 - e) / e) * (1.0 - np.exp(-(e / 1.3) ** 2))
        h = (e[-1] - e[0]) / 128
        w[i] = h / 3 * (f[0] + f[-1] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum())
    w = np.maximum(w, 0)
    return edges.astype(np.float32), (w / w.sum()).astype(np.float32)


def mono(E):
    return np.array([E, E], np.float32), np.array([1.0], np.float32)


def beam_on(ph: Phantom, particle, spectrum, field=(10.0, 10.0), ssd=100.0):
    """Beam normal to the entrance surface z=0, centred on the phantom's x-y centre."""
    lx, ly, _ = ph.size_cm
    edges, w = spectrum
    return Beam(particle, edges, w, tuple(field), float(ssd), (lx / 2, ly / 2, 0.0), (0.0, 0.0, 1.0))


# ---- named workloads ---------------------------------------------------------------
def electron_water_61():
    """15 MeV e-, 10x10 parallel field, water 30.5x30.5x30 cm at 0.5 cm (61x61x60)."""
    ph = homogeneous((61, 61, 60), (0.5, 0.5, 0.5))
    return ph, beam_on(ph, 1, mono(15.0), (10.0, 10.0), ssd=0.0)


def photon_slab_120():
    """6 MV photons, 10x10 at SSD 100 cm, slab phantom 120^3 at 0.25 cm."""
    ph = slab()
    return ph, beam_on(ph, 0, spectrum_6mv(), (10.0, 10.0), ssd=100.0)


def photon_half_slab_120():
    ph = half_slab()
    return ph, beam_on(ph, 0, spectrum_6mv(), (10.0, 10.0), ssd=100.0)


def electron_half_slab_120():
    ph = half_slab()
    return ph, beam_on(ph, 1, mono(15.0), (10.0, 10.0), ssd=100.0)


def paper_phantom(kind="water"):
    """Phantoms of the paper's experiments (Sec. 2.2 "Materials"): 32x32x32 cm^3 at 0.25 cm
    (128^3); slab: water, bone and lung layers of 2 cm each along z (0-2, 2-4, 4-6 cm),
    then water; half-slab: the bone and lung layers cover half of the x-y plane."""
    n, v = (128, 128, 128), (0.25, 0.25, 0.25)
    if kind == "water":
        return homogeneous(n, v)
    if kind == "slab":
        return _layered(n, v, ((2.0, 4.0, BONE), (4.0, 6.0, LUNG)))
    return _layered(n, v, ((2.0, 4.0, BONE), (4.0, 6.0, LUNG)), half=True)


def paper_preset(particle, kind="water"):
    """The paper's beams: 2x2 cm^2 at the surface, point source at SSD 100 cm,
    15 MeV electrons or the 6 MV spectrum."""
    ph = paper_phantom(kind)
    spec = mono(15.0) if particle == 1 else spectrum_6mv()
    return ph, beam_on(ph, particle, spec, (2.0, 2.0), 100.0)


def scaled(ph: Phantom, factor):
    """Coarsen a phantom by an integer factor (nearest sample) for oracle-sized cases."""
    f = int(factor)
    d = ph.density[f // 2::f, f // 2::f, f // 2::f].copy()
    m = ph.material[f // 2::f, f // 2::f, f // 2::f].copy()
    return Phantom(d, m, tuple(v * f for v in ph.voxel))


def random_phantom(n=(24, 20, 28), voxel=(0.5, 0.5, 0.5), seed=0):
    """Small random heterogeneous phantom for parity tests: random materials with
    nominal densities, scaled by a random factor in [0.7, 1.3], ~5% vacuum-free."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    mat = rng.integers(0, 3, size=(nz, ny, nx)).astype(np.uint8)
    base = np.vectorize(RHO.get)(mat).astype(np.float32)
    dens = (base * rng.uniform(0.7, 1.3, size=base.shape)).astype(np.float32)
    return Phantom(dens, mat, tuple(float(v) for v in voxel))


def beamlets(ph: Phantom, n_beamlets=512, seed=1, log10_mean=5.0, log10_sd=0.5, lo=10_000, hi=1_000_000,
             field=(0.5, 0.5), sad=100.0, offset=4.0):
    """Pencil beamlets at random gantry angles about the y axis through the phantom centre:
    field 0.5x0.5 cm^2 in the isocentre plane, point source at SAD, beam's-eye-view
    offsets uniform in [-offset, offset] cm, histories 10^N(log10_mean, log10_sd)
    clipped to [lo, hi]. Returns a list of dicts for Engine.set_beamlets."""
    rng = np.random.default_rng(seed)
    lx, ly, lz = ph.size_cm
    c = np.array([lx / 2, ly / 2, lz / 2])
    out = []
    for _ in range(n_beamlets):
        th = rng.uniform(0.0, 2.0 * math.pi)
        d = np.array([math.sin(th), 0.0, math.cos(th)])
        e1 = np.array([d[2], 0.0, -d[0]])
        e2 = np.array([0.0, 1.0, 0.0])
        a, b = rng.uniform(-offset, offset, 2)
        n = int(np.clip(round(10.0 ** rng.normal(log10_mean, log10_sd)), lo, hi))
        out.append({"field": tuple(field), "ssd": float(sad), "iso": tuple(c + a * e1 + b * e2),
                    "direction": tuple(d), "n_histories": n})
    return out


def beamlets_ct():
    """512 6 MV pencil beamlets on the CT-like phantom 256x256x128 at 0.2 cm."""
    ph = ct_like()
    return ph, spectrum_6mv(), beamlets(ph)


def denoiser_case(seed, n=(128, 128, 128), voxel=(0.25, 0.25, 0.25)):
    """One random case for training or judging the dose denoiser: the CT-like phantom
    generator at 128^3 x 0.25 cm with this seed, and a random beam: 6 MV photons or
    mono-energetic electrons with E ~ U(6, 20) MeV (equal odds), field sides U(2, 20) cm each
    in the plane through the phantom centre, gantry angle U(0, 2 pi) about the y axis through
    the centre, point source at SAD 100 cm."""
    ph = ct_like(n, voxel, seed)
    rng = np.random.default_rng([int(seed), 5])
    particle = int(rng.integers(0, 2))
    edges, w = spectrum_6mv() if particle == 0 else mono(float(rng.uniform(6.0, 20.0)))
    fx, fy = (float(v) for v in rng.uniform(2.0, 20.0, 2))
    th = float(rng.uniform(0.0, 2.0 * math.pi))
    lx, ly, lz = ph.size_cm
    beam = Beam(particle, edges, w, (fx, fy), 100.0, (lx / 2, ly / 2, lz / 2),
                (math.sin(th), 0.0, math.cos(th)))
    return ph, beam


# ---- phase-space sources ---------------------------------------------------------------
# One record per source particle, 32 bytes: position (cm, phantom frame), direction (any
# length), kinetic energy (MeV), type (0 photon, 1 electron, 2 positron).
PS_DTYPE = np.dtype([("x", "<f4"), ("y", "<f4"), ("z", "<f4"), ("u", "<f4"), ("v", "<f4"), ("w", "<f4"),
                     ("E", "<f4"), ("type", "<i4")])


def phase_space_linac(ph: Phantom, n, seed=1, field=(10.0, 10.0), ssd=100.0, z_plane=-2.0,
                      f_electron=0.05, f_positron=0.01, spread_deg=0.5):
    """A user-side source model written out as phase-space records: particles on the plane
    z = z_plane (cm, above the entrance surface z = 0) inside the beam's projection of a
    field x field rectangle at the surface from a point source at SSD, directions from the
    source point blurred by a Gaussian angle (spread_deg), centred on the phantom's x-y
    centre. Photons (energies from the closed-form 6 MV spectrum, uniform within a bin),
    contaminant electrons (fraction f_electron, U(0.5, 6) MeV) and positrons (f_positron,
    U(0.5, 4) MeV)."""
    rng = np.random.default_rng(seed)
    lx, ly, _ = ph.size_cm
    edges, w = spectrum_6mv()
    rec = np.zeros(n, PS_DTYPE)
    S = np.array([lx / 2, ly / 2, -ssd])
    a = rng.uniform(-0.5, 0.5, n) * field[0]
    b = rng.uniform(-0.5, 0.5, n) * field[1]
    P = np.stack([lx / 2 + a, ly / 2 + b, np.zeros(n)], 1)             # point in the surface field
    d = P - S
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d += rng.normal(0.0, np.radians(spread_deg), (n, 3))
    t = (z_plane - S[2]) / d[:, 2]
    X = S + t[:, None] * d
    kind = rng.random(n)
    typ = np.where(kind < f_positron, 2, np.where(kind < f_positron + f_electron, 1, 0)).astype(np.int32)
    bins = rng.choice(len(w), size=n, p=w / w.sum())
    E = edges[bins] + rng.random(n) * (edges[bins + 1] - edges[bins])
    E = np.where(typ == 1, rng.uniform(0.5, 6.0, n), np.where(typ == 2, rng.uniform(0.5, 4.0, n), E))
    rec["x"], rec["y"], rec["z"] = X[:, 0], X[:, 1], X[:, 2]
    rec["u"], rec["v"], rec["w"] = d[:, 0], d[:, 1], d[:, 2]
    rec["E"], rec["type"] = E, typ
    return rec


PS_MAGIC = b"OCMCPS01"


def write_phase_space(path, records):
    """Phase-space file: 8-byte magic 'OCMCPS01', uint64 record count (little endian), then
    the 32-byte records of PS_DTYPE."""
    r = np.ascontiguousarray(records, PS_DTYPE)
    with open(path, "wb") as f:
        f.write(PS_MAGIC)
        f.write(np.uint64(len(r)).tobytes())
        f.write(r.tobytes())


def read_phase_space(path):
    with open(path, "rb") as f:
        if f.read(8) != PS_MAGIC:
            raise ValueError("not a phase-space file")
        n = int(np.frombuffer(f.read(8), "<u8")[0])
        return np.frombuffer(f.read(32 * n), PS_DTYPE).copy()


def pencil(ph: Phantom, particle, E, direction=(0.0, 0.0, 1.0)):
    """Infinitely thin parallel beam along +z through the x-y centre."""
    lx, ly, _ = ph.size_cm
    edges, w = mono(E)
    return Beam(particle, edges, w, (0.0, 0.0), 0.0, (lx / 2 + 1e-3, ly / 2 + 1e-3, 0.0), direction)


__all__ = [n for n in dir() if not n.startswith("_") and n not in ("annotations", "dataclasses", "math", "np")]
