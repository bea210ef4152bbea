"""The seeded synthetic inputs against the configurations they stand for: grid sizes and voxel
sizes, layer depths and densities of the slab and half-slab phantoms, the 6 MV spectrum, the
CT-like phantom's body, inserts and density-to-material rule, the 512 beamlets' history counts
and geometry, the denoiser cases' beams, and the paper's own setups (Sec. 2.2 "Materials"). Every
generator is deterministic for a given seed."""
import math

import numpy as np
import pytest

import ocmc_inputs as I


def depth_centres(ph):
    return (np.arange(ph.density.shape[0]) + 0.5) * ph.voxel[2]


def test_material_densities():
    assert I.RHO[I.WATER] == pytest.approx(1.0)
    assert I.RHO[I.BONE] == pytest.approx(1.85)
    assert I.RHO[I.LUNG] == pytest.approx(0.26)


def test_electron_water_61():
    ph, beam = I.electron_water_61()
    assert ph.density.shape == (60, 61, 61) and ph.voxel == (0.5, 0.5, 0.5)
    assert ph.size_cm == pytest.approx((30.5, 30.5, 30.0))
    assert np.all(ph.material == I.WATER) and np.all(ph.density == np.float32(1.0))
    assert beam.particle == 1 and np.all(beam.edges == 15.0) and beam.weights.tolist() == [1.0]
    assert beam.field == (10.0, 10.0) and beam.ssd <= 0           # parallel field
    assert beam.direction == (0.0, 0.0, 1.0) and beam.iso[:2] == pytest.approx((15.25, 15.25))


def test_photon_slab_120_layers():
    ph, beam = I.photon_slab_120()
    assert ph.density.shape == (120, 120, 120) and ph.voxel == (0.25, 0.25, 0.25)
    z = depth_centres(ph)
    want = np.where(z < 3.0, I.WATER, np.where(z < 5.0, I.BONE, np.where(z < 12.0, I.LUNG, I.WATER)))
    # every voxel of a depth slice has that slice's material and nominal density
    assert np.all(ph.material == want[:, None, None])
    assert np.all(ph.density == np.vectorize(I.RHO.get)(want).astype(np.float32)[:, None, None])
    assert beam.particle == 0 and beam.ssd == 100.0 and beam.field == (10.0, 10.0)
    assert beam.direction == (0.0, 0.0, 1.0)


def test_half_slab_layers():
    for ph, beam, particle in ((*I.photon_half_slab_120(), 0), (*I.electron_half_slab_120(), 1)):
        assert beam.particle == particle and beam.ssd == 100.0 and beam.field == (10.0, 10.0)
        z = depth_centres(ph)
        x = (np.arange(ph.density.shape[2]) + 0.5) * ph.voxel[0]
        inner = (z >= 3.0) & (z < 10.0)
        left = x < ph.size_cm[0] / 2
        want = np.full(ph.material.shape, I.WATER, np.uint8)
        want[np.ix_(inner, np.ones(ph.material.shape[1], bool), left)] = I.BONE
        want[np.ix_(inner, np.ones(ph.material.shape[1], bool), ~left)] = I.LUNG
        assert np.array_equal(ph.material, want)
        assert np.array_equal(ph.density, np.vectorize(I.RHO.get)(want).astype(np.float32))


def test_spectrum_6mv():
    edges, w = I.spectrum_6mv()
    assert len(edges) == 25 and len(w) == 24
    assert edges[0] == pytest.approx(0.25) and edges[-1] == pytest.approx(6.0)
    assert np.allclose(np.diff(edges), (6.0 - 0.25) / 24, rtol=1e-5)
    assert w.sum() == pytest.approx(1.0, rel=1e-6) and np.all(w >= 0)
    # energies are drawn uniformly within a bin: the sampled mean is the weighted bin centre,
    # against the closed-form shape integrated on a fine grid (mean 2.0 MeV)
    e = np.linspace(0.25, 6.0, 200001)
    f = ((6.0 - e) / e) * (1.0 - np.exp(-(e / 1.3) ** 2))
    exact = np.trapezoid(e * f, e) / np.trapezoid(f, e)
    mean = float(np.sum(w * 0.5 * (edges[1:] + edges[:-1])))
    assert mean == pytest.approx(exact, rel=2e-3) and exact == pytest.approx(2.0, abs=0.05)


def test_ct_like_phantom():
    ph = I.ct_like()
    assert ph.density.shape == (128, 256, 256) and ph.voxel == (0.2, 0.2, 0.2)
    d, m = ph.density, ph.material
    outside = d == np.float32(0.0012)
    body = ~outside
    assert 0.2 < body.mean() < 0.8                                   # an ellipsoidal body inside the box
    assert np.all(m[outside] == I.WATER)                             # air-like low-density water around it
    inserts = np.unique(d[body & (d != np.float32(1.0))])
    assert 1 <= len(inserts) <= 8 and np.all((inserts >= 0.2) & (inserts <= 1.9))
    # density thresholds pick the material inside the body
    db, mb = d[body], m[body]
    assert np.all(mb[db < 0.6] == I.LUNG) and np.all(mb[db > 1.3] == I.BONE)
    assert np.all(mb[(db >= 0.6) & (db <= 1.3)] == I.WATER)
    again = I.ct_like()
    assert np.array_equal(d, again.density) and np.array_equal(m, again.material)
    small = [I.ct_like(n=(64, 64, 32), seed=k).density for k in (1, 1, 2)]
    assert np.array_equal(small[0], small[1]) and not np.array_equal(small[0], small[2])


def test_beamlets_ct_recipe():
    ph, spec, bl = I.beamlets_ct()
    assert len(bl) == 512
    n = np.array([b["n_histories"] for b in bl])
    assert n.min() >= 10_000 and n.max() <= 1_000_000
    lg = np.log10(n)
    # 10^N(5, 0.5) clipped at 4 and 6 (two standard deviations, symmetric): the mean stays at 5
    assert abs(lg.mean() - 5.0) < 0.1 and 0.38 < lg.std() < 0.55
    c = np.array(ph.size_cm) / 2
    for b in bl:
        d = np.array(b["direction"])
        assert abs(np.linalg.norm(d) - 1.0) < 1e-12 and d[1] == 0.0        # gantry about the y axis
        assert b["field"] == (0.5, 0.5) and b["ssd"] == 100.0
        off = np.array(b["iso"]) - c
        assert abs(off @ d) < 1e-9 and np.all(np.abs(off) <= 4.0 + 1e-9)     # beam's-eye-view offsets
    ang = np.array([math.atan2(b["direction"][0], b["direction"][2]) % (2 * math.pi) for b in bl])
    counts, _ = np.histogram(ang, bins=8, range=(0, 2 * math.pi))
    assert counts.min() > 0.5 * 512 / 8                              # angles cover the whole circle
    assert spec[0][0] == pytest.approx(0.25) and len(spec[1]) == 24


def test_denoiser_cases():
    seen = set()
    for seed in range(40):
        ph, beam = I.denoiser_case(900_000 + seed, n=(48, 48, 48))   # inserts need a body of ~10 cm
        assert 2.0 <= beam.field[0] <= 20.0 and 2.0 <= beam.field[1] <= 20.0
        assert beam.ssd == 100.0 and abs(np.linalg.norm(beam.direction) - 1.0) < 1e-12 and beam.direction[1] == 0.0
        if beam.particle == 0:
            assert len(beam.weights) == 24
        else:
            assert 6.0 <= float(beam.edges[0]) <= 20.0 and beam.edges[0] == beam.edges[1]
        seen.add(beam.particle)
        # the beam does not depend on the grid: same seed, same beam at the full size
        if seed < 2:
            _, full = I.denoiser_case(900_000 + seed)
            assert full.particle == beam.particle and full.field == beam.field
            assert full.direction == beam.direction
    assert seen == {0, 1}
    ph, _ = I.denoiser_case(910_001)
    assert ph.density.shape == (128, 128, 128) and ph.voxel == (0.25, 0.25, 0.25)


@pytest.mark.parametrize("kind", ["water", "slab", "half"])
def test_paper_presets(kind):
    for particle in (0, 1):
        ph, beam = I.paper_preset(particle, kind)
        assert ph.density.shape == (128, 128, 128) and ph.size_cm == pytest.approx((32.0, 32.0, 32.0))
        assert beam.field == (2.0, 2.0) and beam.ssd == 100.0
        assert (beam.particle, len(beam.weights)) == ((0, 24) if particle == 0 else (1, 1))
    z = depth_centres(ph)
    mats = set(np.unique(ph.material[(z >= 2.0) & (z < 4.0)]).tolist())
    if kind == "water":
        assert np.all(ph.material == I.WATER)
    elif kind == "slab":
        assert mats == {I.BONE} and np.all(ph.material[(z >= 4.0) & (z < 6.0)] == I.LUNG)
        assert np.all(ph.material[(z < 2.0) | (z >= 6.0)] == I.WATER)
    else:
        assert mats == {I.WATER, I.BONE}
