"""User-defined materials on the GPU (Sec. 2.1: per-material cross-section data; the paper's
database has 16 materials): tables against the oracle's closed forms, dose parity, the
built-in set reproduced, and the staging of at most 10 materials per phantom."""
import numpy as np
import pytest

import ocmc_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

USER = ["adipose", "muscle", "aluminium", "copper", "pmma"]


@pytest.fixture(scope="module")
def ocmc():
    from paper_1503_01722_gb300 import build
    build.build()
    from paper_1503_01722_gb300 import ocmc as m
    return m


@pytest.fixture(autouse=True)
def _restore():
    yield
    O.reset_materials()


def phantom_of(defs, seed=1, shape=(24, 20, 28), voxel=0.5):
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    mat = rng.integers(0, len(defs), size=(nz, ny, nx)).astype(np.uint8)
    rho = np.array([d["density"] for d in defs], np.float32)[mat] * rng.uniform(0.8, 1.2, mat.shape).astype(np.float32)
    return I.Phantom(rho.astype(np.float32), mat, (voxel, voxel, voxel))


def test_user_material_tables_match_closed_forms(ocmc):
    defs = I.material_set(USER)
    O.set_materials(defs)
    E = np.geomspace(0.0105, 29.0, 401).astype(np.float32)
    Ed = E.astype(np.float64)
    with ocmc.Engine(0) as e:
        e.set_materials(defs)
        e.create_phantom(phantom_of(defs))
        for m in range(len(defs)):
            t = e.test_tables(m, E).astype(np.float64)
            for col, ref in ((0, O.mu(m, Ed)), (1, O.mu(m, Ed, 1)), (2, O.mu(m, Ed, 2))):
                assert np.max(np.abs(t[:, col] / ref - 1)) < 1e-3, (m, col)
            sel = Ed > 0.05
            assert np.max(np.abs(t[sel, 4] / O.lambda1_inv(m, Ed[sel]) - 1)) < 1e-3, m
            far = Ed > 0.45
            sm, sb = O.sigma_moller(m, Ed), O.sigma_brems(m, Ed)
            assert np.max(np.abs(t[far, 5] / sm[far] - 1)) < 2e-3, m
            assert np.max(np.abs(t[:, 6][sb > 0] / sb[sb > 0] - 1)) < 2e-3, m


def test_dose_parity_with_user_materials(ocmc):
    defs = I.material_set(USER)
    O.set_materials(defs)
    ph = phantom_of(defs, seed=3)
    beam = I.beam_on(ph, 0, I.mono(15.0), (6, 5), 100.0)
    n, B = 60_000, 50
    with ocmc.Engine(0, n_batches=B) as e:
        e.set_materials(defs)
        e.create_phantom(ph)
        e.set_source(beam)
        e.run(n, seed=5)
        D, S = e.dose()
        st = e.stats()
    r = O.run(ph, beam, n, seed=5, p=O.params(n_batches=B))
    Dr, Sr = r.dose()
    m = Dr >= 0.1 * Dr.max()
    z = np.abs(D - Dr)[m] / np.sqrt(S ** 2 + Sr ** 2)[m]
    assert np.mean(z <= 3) >= 0.99, np.mean(z <= 3)
    assert abs((D - Dr)[m].mean()) < 0.005 * Dr.max()
    bal = st["e_in"] + st["annih_mass"] - st["e_dep"] - st["e_esc"] - st["pair_mass"] - st["e_killed"]
    assert abs(bal) <= 2e-5 * st["e_in"] and st["majorant_violations"] == 0


def test_builtin_set_reproduced_bit_for_bit(ocmc):
    ph = I.random_phantom()
    beam = I.beam_on(ph, 1, I.mono(12.0), (6, 5), 100.0)
    out = []
    for user in (False, True):
        with ocmc.Engine(0) as e:
            if user:
                e.set_materials(I.material_set(["water", "bone_cortical", "lung"]))
            e.create_phantom(ph)
            e.set_source(beam)
            e.run(20_000, seed=2)
            out.append(e.raw_tally())
    assert np.array_equal(out[0], out[1])


def test_more_than_ten_defined_materials_are_staged_per_phantom(ocmc):
    names = I.MATERIAL_ORDER
    defs = [dict(I.MATERIALS[names[k % len(names)]], I=I.MATERIALS[names[k % len(names)]]["I"] + k)
            for k in range(14)]                        # 14 distinct definitions
    used = [1, 3, 4, 6, 7, 8, 9, 11, 12, 13]            # ten of them
    sub = phantom_of([defs[u] for u in used], seed=4)
    full = I.Phantom(sub.density, np.array(used, np.uint8)[sub.material], sub.voxel)
    beam = I.beam_on(sub, 0, I.mono(8.0), (6, 5), 100.0)
    tallies = []
    for ds, ph in ((defs, full), ([defs[u] for u in used], sub)):
        with ocmc.Engine(0) as e:
            e.set_materials(ds)
            e.create_phantom(ph)
            e.set_source(beam)
            e.run(15_000, seed=7)
            tallies.append(e.raw_tally())
    assert np.array_equal(tallies[0], tallies[1])      # compacted indices: the same tables
    bad = I.Phantom(full.density, full.material.copy(), full.voxel)
    bad.material[0, 0, 0] = 0                           # an eleventh material
    with ocmc.Engine(0) as e:
        e.set_materials(defs)
        with pytest.raises(ocmc.OcmcError):
            e.create_phantom(bad)
        with pytest.raises(ocmc.OcmcError):
            e.set_materials(defs + defs[:3])            # 17 materials


def test_set_materials_drops_the_phantom(ocmc):
    ph = I.random_phantom()
    with ocmc.Engine(0) as e:
        e.create_phantom(ph)
        e.set_source(I.beam_on(ph, 0, I.mono(2.0), (4, 4), 100.0))
        e.set_materials(I.material_set(["water", "pmma"]))
        with pytest.raises(ocmc.OcmcError):
            e.run(10)
        with pytest.raises(ocmc.OcmcError):
            e.create_phantom(ph)                        # index 2 is not defined any more
