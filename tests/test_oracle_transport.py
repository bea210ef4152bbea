"""Transport-level pins of the oracle: conservation, Woodcock transmission,
CSDA range, first-collision energy transfer, special cases, determinism."""
import math

import numpy as np
import pytest
from scipy import integrate

import ocmc_inputs as I
import oracle as O

MC2 = 0.51099895


def balance(r):
    L = r.ledger
    return L["e_in"] + L["annih_mass"] - L["e_dep"] - L["e_esc"] - L["pair_mass"] - L["e_killed"]


@pytest.mark.parametrize("case", ["e_water", "g_slab", "g_half_high"])
def test_energy_conservation(case):
    if case == "e_water":
        ph, beam = I.electron_water_61()
        n = 300
    elif case == "g_slab":
        ph, beam = I.photon_slab_120()
        ph = I.scaled(ph, 3)
        n = 3000
    else:   # 20 MeV photons make pairs and annihilations in bone
        ph = I.scaled(I.half_slab(), 3)
        beam = I.beam_on(ph, 0, I.mono(20.0), (10, 10), 100.0)
        n = 2000
    r = O.run(ph, beam, n, seed=3, threads=4)
    assert r.ledger["e_in"] > 0
    assert abs(balance(r)) <= 1e-6 * r.ledger["e_in"]
    # the int64 tally holds the deposited energy to the 2^-29 MeV rounding bound per deposit
    assert abs(r.tally.sum() / 2 ** 28 - r.ledger["e_dep"]) < 1e-6 * r.ledger["e_in"]
    assert r.counters["viol_photon"] == 0 and r.counters["viol_electron"] == 0
    assert r.counters["stack_overflow"] == 0
    if case == "g_half_high":
        assert r.counters["pair"] > 0 and r.counters["annih"] > 0


@pytest.mark.parametrize("layers", ["water", "slab"])
def test_narrow_beam_transmission(layers):
    """Unscattered transmission of a pencil beam equals exp(-sum mu_i rho_i x_i):
    Woodcock tracking against the majorant gives the analogue result (Sec. 2.1)."""
    E = 1.25
    n = 60_000
    if layers == "water":
        ph = I.homogeneous((9, 9, 40), (1.0, 1.0, 0.25))
        segs = [(0, 10.0, 0)]
    else:
        ph = I.slab((9, 9, 48), (1.0, 1.0, 0.25), layers=((3.0, 5.0, I.BONE), (5.0, 9.0, I.LUNG)))
        segs = [(0, 3.0, 0), (3.0, 5.0, 1), (5.0, 9.0, 2), (9.0, 12.0, 0)]
    beam = I.pencil(ph, 0, E)
    r = O.run(ph, beam, n, seed=5, p=O.params(flags=O.KILL_FIRST_REAL), threads=4)
    tau = sum(I.RHO[m] * O.mu(m, E) * (z1 - z0) for z0, z1, m in segs)
    p = math.exp(-tau)
    got = r.counters["transmitted"] / n
    assert abs(got - p) < 3.5 * math.sqrt(p * (1 - p) / n), (got, p)
    if layers == "slab":
        # majorant = bone: most sampled events in water/lung are fictitious (Sec. 3.2)
        assert r.counters["fictitious"] > 0.3 * r.counters["flights"]


@pytest.mark.parametrize("E0", [2.0, 10.0])
def test_csda_range(E0):
    """With hard events and deflections off, the path length to the absorption
    energy is the CSDA range integral of 1/L(E) (to within 1%)."""
    p = O.params(flags=O.NO_HARD | O.NO_MS)
    ph = I.homogeneous((5, 5, 200), (4.0, 4.0, 0.1))
    beam = I.pencil(ph, 1, E0)
    n = 20
    r = O.run(ph, beam, n, seed=2, p=p, threads=2)
    L = lambda t: O.L_col(0, t, p.w_cc) + O.L_rad(0, t, p.w_cb)
    R, _ = integrate.quad(lambda t: 1 / L(t), p.e_abs_e, E0, epsrel=1e-10)
    path = r.ledger["e_path"] / n
    assert abs(path / R - 1) < 0.01, (path, R)
    assert r.counters["moller"] == 0 and r.counters["brems"] == 0


def test_first_collision_energy_transfer():
    """Thin water slab, photons with electrons deposited where they are created:
    deposited energy per photon ~ E (mu_C tau) <T>/E with <T>/E from the
    Klein-Nishina energy-transfer integral (thin-target limit)."""
    E = 1.0
    ph = I.homogeneous((20, 20, 1), (1.0, 1.0, 0.1))
    beam = I.pencil(ph, 0, E)
    n = 400_000
    r = O.run(ph, beam, n, seed=9, p=O.params(flags=O.KERMA), threads=8)
    k = E / MC2

    def dsig(m):
        e = 1 / (1 + k * (1 - m))
        return e * e * (e + 1 / e - (1 - m * m))

    s_tot = integrate.quad(dsig, -1, 1, epsrel=1e-12)[0]
    s_tr = integrate.quad(lambda m: (1 - 1 / (1 + k * (1 - m))) * dsig(m), -1, 1, epsrel=1e-12)[0]
    mu = O.mu(0, E)
    first = (1 - math.exp(-mu * 0.1)) * (O.mu(0, E, 1) / mu) * E * s_tr / s_tot
    got = r.ledger["e_dep"] / n
    # statistical error ~1% at this n; second collisions add < 1%
    assert abs(got / first - 1) < 0.03, (got, first)


def test_vacuum_phantom_deposits_nothing():
    ph = I.homogeneous((10, 10, 10), (1.0, 1.0, 1.0), density=0.0)
    for particle, E in ((0, 2.0), (1, 10.0)):
        beam = I.beam_on(ph, particle, I.mono(E), (4, 4), 100.0)
        r = O.run(ph, beam, 500, seed=1, threads=2)
        assert r.tally.sum() == 0
        assert abs(r.ledger["e_esc"] - r.ledger["e_in"]) < 1e-9 * r.ledger["e_in"]


def test_thread_count_does_not_change_result():
    ph, beam = I.photon_slab_120()
    ph = I.scaled(ph, 4)
    a = O.run(ph, beam, 3000, seed=7, threads=1)
    b = O.run(ph, beam, 3000, seed=7, threads=5)
    assert np.array_equal(a.tally, b.tally)
    c = O.run(ph, beam, 3000, seed=8, threads=5)
    assert not np.array_equal(a.tally, c.tally)


def test_heterogeneity_costs_more_events():
    """Sec. 3.2: slab phantoms take more photon events (fictitious, under a bone
    majorant) and more electron steps than water."""
    ph_w = I.homogeneous((40, 40, 40), (0.75, 0.75, 0.75))
    ph_s = I.scaled(I.slab(), 3)
    beam = I.beam_on(ph_w, 0, I.spectrum_6mv(), (10, 10), 100.0)
    rw = O.run(ph_w, beam, 4000, seed=1, threads=8)
    rs = O.run(ph_s, beam, 4000, seed=1, threads=8)
    assert rs.counters["flights"] > 1.2 * rw.counters["flights"]
    assert rw.counters["fictitious"] == 0 and rs.counters["fictitious"] > 0


def test_source_geometry_point_and_parallel():
    ph, beam = I.photon_slab_120()
    s = O.source_sample(ph, beam, 20000, seed=4)
    assert np.all(s[:, 7] == 1)
    lx, ly, _ = ph.size_cm
    # entering at z=0 inside the 10x10 field, directions from the point source
    assert np.allclose(s[:, 2], 0.0)
    assert np.all(np.abs(s[:, 0] - lx / 2) <= 5.0) and np.all(np.abs(s[:, 1] - ly / 2) <= 5.0)
    src = np.array([lx / 2, ly / 2, -100.0])
    d = s[:, :3] - src
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    assert np.allclose(d, s[:, 3:6], atol=1e-12)
    # energies follow the stratified spectrum
    b, order = O.stratify(beam.edges, beam.weights, 20000)
    for q in range(len(order)):
        j = order[q]
        e = s[int(b[q]):int(b[q + 1]), 6]
        assert np.all((e >= beam.edges[j]) & (e <= beam.edges[j + 1]))
    ph, beam = I.electron_water_61()
    s = O.source_sample(ph, beam, 5000, seed=4)
    assert np.all(s[:, 5] == 1.0) and np.all(s[:, 6] == np.float32(15.0))
    assert abs(s[:, 0].mean() - 61 * 0.5 / 2) < 0.1
