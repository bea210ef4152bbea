"""Pins of the oracle's interaction kinematics: the directions and energies that leave an event
(paper Sec. 2.1: Compton electron and Moller directions from kinematics, bremsstrahlung photon
angle, positron annihilation).

What fixes them here is mechanics, not the oracle: relativistic energy and momentum
conservation (p c = sqrt(T (T + 2 mc^2)) for an electron of kinetic energy T, p c = E for a
photon), the Compton relation between the scattered energy and the angle, the fixed
bremsstrahlung angle mc^2 / (T + mc^2), isotropy of the annihilation pair, and uniform azimuths.
Every event is checked from several incoming directions, including the poles +-z (where the
rotation changes frame) and directions a hair away from them. The azimuth of an outgoing
direction is measured in a frame built here, independently of the oracle's rotation.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle as O

MC2 = 0.51099895

DIRECTIONS = {
    "+z": (0.0, 0.0, 1.0),
    "-z": (0.0, 0.0, -1.0),
    "near+z": (3e-11, -2e-11, 1.0),
    "near-z": (1e-6, 2e-6, -1.0),
    "+x": (1.0, 0.0, 0.0),
    "oblique": (0.3, -0.5, 0.81),
    "oblique-back": (-0.62, 0.2, -0.35),
}


def unit(d):
    d = np.asarray(d, np.float64)
    return d / np.linalg.norm(d)


def momentum(T):
    return np.sqrt(T * (T + 2 * MC2))


def azimuth(d0, d):
    """Azimuth of the rows of d about d0, in a frame (e1, e2, d0) made from the coordinate axis
    least aligned with d0."""
    d0 = unit(d0)
    a = np.zeros(3)
    a[np.argmin(np.abs(d0))] = 1.0
    e1 = unit(a - a.dot(d0) * d0)
    e2 = np.cross(d0, e1)
    return np.arctan2(d @ e2, d @ e1)


def uniform_p(x, lo, hi, bins=24):
    counts, _ = np.histogram(x, bins=np.linspace(lo, hi, bins + 1))
    return stats.chisquare(counts).pvalue


def bin_probs(pdf, edges):
    return np.array([integrate.quad(pdf, a, b, epsrel=1e-10)[0] for a, b in zip(edges[:-1], edges[1:])])


def chi2_p(samples, edges, probs):
    counts, _ = np.histogram(samples, bins=edges)
    exp = probs / probs.sum() * len(samples)
    keep = exp > 5
    chi2 = ((counts[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    return stats.chi2.sf(chi2, keep.sum() - 1)


def cos_tol(d0):
    """Tolerance of a polar cosine about d0: rounding, plus, within 1e-10 of a pole, the
    distance sin(theta_0) from the pole, whose own axis the rotation then takes."""
    s0 = math.hypot(d0[0], d0[1])
    return 1e-12 + (s0 if s0 < 1e-10 else 0.0)


def assert_unit(d, tol=1e-12):
    assert np.max(np.abs(np.linalg.norm(d, axis=1) - 1.0)) < tol


# ---- rotation ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", list(DIRECTIONS))
@pytest.mark.parametrize("mu", [-1.0, -0.5, 0.0, 0.3, 0.999999, 1.0])
def test_rotation_polar_cosine(name, mu):
    d0 = unit(DIRECTIONS[name])
    a, d, phi, _ = O.event("rotation", 1.0, d0, 2000, seed=3, aux=mu)
    assert_unit(d)
    assert np.max(np.abs(d @ d0 - mu)) < cos_tol(d0)
    assert phi.min() > 0 and phi.max() <= 2 * math.pi


@pytest.mark.parametrize("name", list(DIRECTIONS))
def test_rotation_azimuth_uniform(name):
    d0 = unit(DIRECTIONS[name])
    _, d, phi, _ = O.event("rotation", 1.0, d0, 100_000, seed=4, aux=0.2)
    az = azimuth(d0, d)
    assert uniform_p(az, -math.pi, math.pi) > 0.01
    # the azimuth the rotation was given and the one measured differ by a constant (mod 2 pi)
    # whose sign is one handedness for every event
    off = np.angle(np.exp(1j * (az - phi)) * np.exp(-1j * (az[0] - phi[0])))
    off2 = np.angle(np.exp(1j * (az + phi)) * np.exp(-1j * (az[0] + phi[0])))
    assert min(np.max(np.abs(off)), np.max(np.abs(off2))) < 1e-9


# ---- Compton ----------------------------------------------------------------------------

@pytest.mark.parametrize("name", list(DIRECTIONS))
@pytest.mark.parametrize("E0", [0.1, 1.0, 10.0])
def test_compton_conservation(name, E0):
    d0 = unit(DIRECTIONS[name])
    E1, d1, T, de = O.event("compton", E0, d0, 20_000, seed=5)
    assert_unit(d1)
    assert_unit(de[T > 0])
    assert np.max(np.abs(E1 + T - E0)) < 1e-12 * E0
    # Compton relation: 1/E1 - 1/E0 = (1 - cos theta)/mc^2, theta the angle between d0 and d1
    mu_from_energy = 1.0 - MC2 * (1.0 / E1 - 1.0 / E0)
    assert np.max(np.abs(d1 @ d0 - mu_from_energy)) < 1e-9
    # momentum: E0 d0 = E1 d1 + p_e de, with p_e from the electron's kinetic energy
    bal = E0 * d0[None, :] - E1[:, None] * d1 - momentum(T)[:, None] * de
    assert np.max(np.abs(bal)) < 1e-9 * E0


@pytest.mark.parametrize("name", ["+z", "near-z", "oblique"])
def test_compton_angles(name):
    """The angle between the incoming and the scattered photon follows Klein-Nishina, and the
    azimuth is uniform with the electron on the opposite side."""
    E0, n = 1.0, 200_000
    d0 = unit(DIRECTIONS[name])
    E1, d1, T, de = O.event("compton", E0, d0, n, seed=6)
    k = E0 / MC2

    def pdf(m):
        e = 1 / (1 + k * (1 - m))
        return e * e * (e + 1 / e - (1 - m * m))

    edges = np.linspace(-1, 1, 41)
    assert chi2_p(d1 @ d0, edges, bin_probs(pdf, edges)) > 0.01
    az = azimuth(d0, d1)
    assert uniform_p(az, -math.pi, math.pi) > 0.01
    sel = (T > 1e-6) & (np.abs(d1 @ d0) < 0.999)
    dphi = np.angle(np.exp(1j * (azimuth(d0, de[sel]) - az[sel] - math.pi)))
    assert np.max(np.abs(dphi)) < 1e-6


# ---- Moller -----------------------------------------------------------------------------

@pytest.mark.parametrize("name", list(DIRECTIONS))
@pytest.mark.parametrize("T0", [0.6, 3.0, 15.0])
def test_moller_conservation(name, T0):
    d0 = unit(DIRECTIONS[name])
    p = O.params(w_cc=0.2)
    T1, d1, W, d2 = O.event("moller", T0, d0, 20_000, seed=7, p=p)
    assert_unit(d1)
    assert_unit(d2)
    assert np.max(np.abs(T1 + W - T0)) < 1e-12 * T0
    assert W.min() >= 0.2 * (1 - 1e-12) and np.all(W <= T1 * (1 + 1e-12))
    # the target electron is at rest: p0 d0 = p1 d1 + p2 d2
    bal = momentum(T0) * d0[None, :] - momentum(T1)[:, None] * d1 - momentum(W)[:, None] * d2
    assert np.max(np.abs(bal)) < 1e-9 * momentum(T0)
    # both leave forward, the knock-on at the wider angle
    assert np.all(d1 @ d0 >= d2 @ d0 - 1e-12) and np.all(d2 @ d0 > 0)


@pytest.mark.parametrize("name", ["-z", "near+z", "oblique-back"])
def test_moller_azimuth(name):
    d0 = unit(DIRECTIONS[name])
    T1, d1, W, d2 = O.event("moller", 5.0, d0, 100_000, seed=8, p=O.params(w_cc=0.2))
    az1, az2 = azimuth(d0, d1), azimuth(d0, d2)
    assert uniform_p(az1, -math.pi, math.pi) > 0.01
    dphi = np.angle(np.exp(1j * (az2 - az1 - math.pi)))
    assert np.max(np.abs(dphi)) < 1e-6


# ---- bremsstrahlung ---------------------------------------------------------------------

@pytest.mark.parametrize("name", list(DIRECTIONS))
@pytest.mark.parametrize("T0,m", [(0.5, 0), (5.0, 1), (15.0, 2)])
def test_brems_photon_angle(name, T0, m):
    d0 = unit(DIRECTIONS[name])
    Te, de, k, dg = O.event("brems", T0, d0, 20_000, seed=9, m=m, p=O.params(w_cb=0.01))
    assert_unit(dg)
    assert np.max(np.abs(de - d0[None, :])) == 0.0
    assert np.max(np.abs(Te + k - T0)) < 1e-12 * T0
    assert k.min() >= 0.01 * (1 - 1e-12) and k.max() <= T0 * (1 + 1e-12)
    theta = MC2 / (T0 + MC2)
    assert np.max(np.abs(dg @ d0 - math.cos(theta))) < cos_tol(d0)
    assert uniform_p(azimuth(d0, dg), -math.pi, math.pi) > 0.01


# ---- annihilation -----------------------------------------------------------------------

@pytest.mark.parametrize("name", ["+z", "oblique"])
def test_annihilation_back_to_back_isotropic(name):
    n = 200_000
    Ea, d1, Eb, d2 = O.event("annihilation", 0.0, DIRECTIONS[name], n, seed=10)
    assert np.all(Ea == MC2) and np.all(Eb == MC2)
    assert_unit(d1)
    assert np.max(np.abs(d1 + d2)) == 0.0
    # isotropy: every Cartesian component of a uniform direction on the sphere is uniform on
    # [-1, 1] (Archimedes), and the azimuth about each axis is uniform
    for a in range(3):
        assert uniform_p(d1[:, a], -1.0, 1.0) > 0.01
    assert uniform_p(np.arctan2(d1[:, 1], d1[:, 0]), -math.pi, math.pi) > 0.01
    assert uniform_p(np.arctan2(d1[:, 0], d1[:, 2]), -math.pi, math.pi) > 0.01


def test_rotation_accessor_is_the_events_rotation():
    """orc_rotate (used to compare the engine's rotation direction by direction) is the rotation
    pinned above: the same polar cosine about the incoming direction, unit length."""
    rng = np.random.default_rng(2)
    d0 = np.vstack([[0, 0, 1], [0, 0, -1], [1e-7, 0, 1], rng.normal(size=(200, 3))])
    mu = rng.uniform(-1, 1, len(d0))
    phi = rng.uniform(0, 2 * math.pi, len(d0))
    out = O.rotate(d0, mu, phi)
    d0n = d0 / np.linalg.norm(d0, axis=1)[:, None]
    assert np.max(np.abs(np.linalg.norm(out, axis=1) - 1)) < 1e-12
    assert np.max(np.abs(np.sum(out * d0n, axis=1) - mu)) < 1e-12
