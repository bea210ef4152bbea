"""Pins of the oracle's user-defined materials (Sec. 2.1: cross-section data per material
type; the paper's database has 16). Per-gram cross sections are sums over the atoms per gram,
so they are mass-fraction-weighted sums of the pure elements' values; the collision stopping
power obeys Bragg additivity where the density effect vanishes."""
import math

import numpy as np
import pytest

import ocmc_inputs as I
import oracle as O


@pytest.fixture(autouse=True)
def _restore():
    yield
    O.reset_materials()


def pure(z, A, I_eV, rho=1.0):
    return {"Z": [z], "A": [A], "w": [1.0], "I": I_eV, "density": rho}


def test_user_water_reproduces_builtin_water_exactly():
    ph = I.homogeneous((12, 12, 14), (0.5, 0.5, 0.5))
    beam = I.beam_on(ph, 0, I.mono(8.0), (4, 4), 100.0)
    a = O.run(ph, beam, 2000, seed=3, threads=2)
    O.set_materials([I.MATERIALS["water"], I.MATERIALS["aluminium"]])
    b = O.run(ph, beam, 2000, seed=3, threads=2)
    assert np.array_equal(a.tally, b.tally)


def test_cross_sections_are_mass_fraction_sums_of_elements():
    mix = I.MATERIALS["muscle"]
    els = [pure(z, A, 75.0) for z, A in zip(mix["Z"], mix["A"])]
    wsum = sum(mix["w"])
    O.set_materials([mix] + els)
    for E in (0.03, 0.3, 3.0, 25.0):
        for ch in (1, 2, 3):
            lhs = O.mu(0, E, ch)
            rhs = sum(w / wsum * O.mu(1 + i, E, ch) for i, w in enumerate(mix["w"]))
            assert math.isclose(lhs, rhs, rel_tol=1e-12), (E, ch)
    for T in (0.5, 2.0, 15.0):
        for fn in (lambda m, t: O.sigma_moller(m, t, 0.2), lambda m, t: O.L_rad(m, t, 0.01),
                   lambda m, t: O.sigma_brems(m, t, 0.01)):
            lhs = fn(0, T)
            rhs = sum(w / wsum * fn(1 + i, T) for i, w in enumerate(mix["w"]))
            assert math.isclose(lhs, rhs, rel_tol=1e-12), T


def test_collision_stopping_power_bragg_additivity_below_density_effect():
    """With ln I_mix = sum_i n_e,i ln I_i / sum_i n_e,i and no density effect (small T), the
    restricted collision stopping power per gram of the mixture is the mass-fraction sum."""
    zs, As, ws, Is = [1, 8, 20], [1.008, 15.999, 40.078], [0.2, 0.5, 0.3], [19.2, 95.0, 191.0]
    ne = [w * z / A for z, A, w in zip(zs, As, ws)]
    I_mix = math.exp(sum(n * math.log(i) for n, i in zip(ne, Is)) / sum(ne))
    mix = {"Z": zs, "A": As, "w": ws, "I": I_mix, "density": 1.0}
    O.set_materials([mix] + [pure(z, A, i) for z, A, i in zip(zs, As, Is)])
    for T in (0.25, 0.4):
        for m in range(4):
            assert O.density_effect(m, T) == 0.0
        lhs = O.L_col(0, T, 0.2)
        rhs = sum(w * O.L_col(1 + i, T, 0.2) for i, w in enumerate(ws))
        assert math.isclose(lhs, rhs, rel_tol=1e-10), T


def test_sixteen_materials_conserve_energy_and_bad_indices_fail():
    names = I.MATERIAL_ORDER
    defs = [I.MATERIALS[names[k % len(names)]] for k in range(16)]
    O.set_materials(defs)
    rng = np.random.default_rng(2)
    ph = I.random_phantom()
    ph.material = rng.integers(0, 16, size=ph.material.shape).astype(np.uint8)
    ph.density = np.array([defs[m]["density"] for m in ph.material.ravel()], np.float32).reshape(ph.material.shape)
    beam = I.beam_on(ph, 0, I.mono(15.0), (6, 5), 100.0)
    r = O.run(ph, beam, 1500, seed=1, threads=4)
    L = r.ledger
    assert abs(L["e_in"] + L["annih_mass"] - L["e_dep"] - L["e_esc"] - L["pair_mass"]) < 1e-9 * L["e_in"]
    O.set_materials(defs[:4])
    with pytest.raises(ValueError):
        O.run(ph, beam, 10, seed=1, threads=1)
    with pytest.raises(ValueError):
        O.set_materials([{"Z": [1], "A": [1.008], "w": [1.0], "I": -1.0, "density": 1.0}])
