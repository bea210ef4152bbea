"""Pins of the oracle's phase-space source (Sec. 2.2 "Materials": source particles loaded
from a phase-space file or made by a user's own source model)."""
import numpy as np
import pytest

import ocmc_inputs as I
import oracle as O


def _box_contains(P, L, eps=0.0):
    return np.all((P >= -eps) & (P <= np.array(L) + eps), axis=-1)


def test_entry_points_by_brute_force():
    ph = I.homogeneous((20, 16, 24), (0.5, 0.5, 0.5))
    L = ph.size_cm
    rng = np.random.default_rng(4)
    n = 400
    rec = np.zeros(n, I.PS_DTYPE)
    rec["x"], rec["y"], rec["z"] = rng.uniform(-6, 16, n), rng.uniform(-6, 14, n), rng.uniform(-6, 18, n)
    d = rng.normal(size=(n, 3))
    rec["u"], rec["v"], rec["w"] = d[:, 0], d[:, 1], d[:, 2]
    rec["E"], rec["type"] = 1.0, 0
    out = O.ps_sample(ph, rec)
    t = np.linspace(0.0, 60.0, 60001)
    for i in range(n):
        S = np.array([rec["x"][i], rec["y"][i], rec["z"][i]], np.float64)
        D = d[i] / np.linalg.norm(d[i])
        pts = S[None] + t[:, None] * D[None]
        inside = _box_contains(pts, L)
        hit = out[i, 7] == 1
        if not hit:
            assert not inside[1:].any(), i                  # the ray never enters
            continue
        E = out[i, :3]
        if _box_contains(S, L):
            assert np.allclose(E, S, atol=1e-12), i         # starts where it is
        else:
            t0 = np.argmax(inside)                          # first sampled point inside
            assert np.linalg.norm(E - S) <= t[t0] + 1e-9 and np.linalg.norm(E - S) >= t[t0] - 1.1e-3
            assert np.min(np.abs(np.concatenate([E, np.array(L) - E]))) < 1e-9   # on a face
        assert np.allclose(out[i, 3:6], D, atol=1e-12) and out[i, 6] == 1.0


def test_same_particles_as_the_analytic_source_give_the_same_dose():
    """Records made from the analytic source's own entry states reproduce its dose
    (different random streams: statistical agreement)."""
    ph = I.scaled(I.slab(), 4)
    beam = I.beam_on(ph, 1, I.mono(12.0), (8, 8), 100.0)
    n = 30_000
    src = O.source_sample(ph, beam, n)
    hit = src[:, 7] == 1
    rec = np.zeros(int(hit.sum()), I.PS_DTYPE)
    for k, name in enumerate(("x", "y", "z", "u", "v", "w", "E")):
        rec[name] = src[hit, k]
    rec["type"] = 1
    B = 20
    a = O.run(ph, beam, n, seed=3, p=O.params(n_batches=B))
    b = O.run_ps(ph, rec, len(rec), seed=5, p=O.params(n_batches=B))
    Da, Sa = a.dose()
    Db, Sb = b.dose()
    Db = Db * len(rec) / n                    # per source particle of the analytic run
    Sb = Sb * len(rec) / n
    m = Da >= 0.1 * Da.max()
    z = np.abs(Da - Db)[m] / np.sqrt(Sa ** 2 + Sb ** 2)[m]
    assert np.mean(z <= 3) >= 0.98, np.mean(z <= 3)
    assert abs((Da - Db)[m].mean()) < 0.01 * Da.max()


def test_mixed_types_conserve_energy_and_recycle_records():
    ph = I.random_phantom()
    rec = I.phase_space_linac(ph, 500, seed=7, field=(6, 5))
    r = O.run_ps(ph, rec, 1000, seed=2, threads=4)
    L = r.ledger
    bal = L["e_in"] + L["annih_mass"] - L["e_dep"] - L["e_esc"] - L["pair_mass"]
    assert abs(bal) < 1e-9 * L["e_in"]
    # every record used twice: entering + missed energy = 2 x the records' energy
    assert np.isclose(L["e_in"] + L["e_miss"], 2 * rec["E"].astype(np.float64).sum(), rtol=1e-12)
    assert r.counters["annih"] > 0


def test_positron_below_cutoff_annihilates():
    ph = I.homogeneous((10, 10, 10), (1.0, 1.0, 1.0))
    rec = np.zeros(1, I.PS_DTYPE)
    rec["x"], rec["y"], rec["z"], rec["w"], rec["E"], rec["type"] = 5.0, 5.0, 5.0, 1.0, 0.1, 2
    r = O.run_ps(ph, rec, 200, seed=1, threads=1)
    assert r.counters["annih"] == 200
    assert np.isclose(r.ledger["annih_mass"], 200 * 2 * 0.51099895, rtol=1e-6)


def test_invalid_records_are_rejected():
    ph = I.homogeneous((4, 4, 4), (1.0, 1.0, 1.0))
    rec = np.zeros(2, I.PS_DTYPE)
    rec["w"], rec["E"] = 1.0, 1.0
    rec["type"][1] = 3
    with pytest.raises(ValueError):
        O.ps_sample(ph, rec)
    rec["type"][1] = 0
    rec["E"][0] = 0.0
    with pytest.raises(ValueError):
        O.run_ps(ph, rec, 2)


def test_file_round_trip(tmp_path):
    ph = I.homogeneous((8, 8, 8), (1.0, 1.0, 1.0))
    rec = I.phase_space_linac(ph, 100, seed=1)
    f = tmp_path / "beam.ps"
    I.write_phase_space(f, rec)
    assert np.array_equal(I.read_phase_space(f), rec)
    assert f.stat().st_size == 16 + 32 * 100
