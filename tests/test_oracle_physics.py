"""Pins of the oracle's closed-form physics (CPU only).

Each closed form is checked against something other than itself: numerical
quadrature of the textbook differential cross section, published reference
data (tests/golden/reference_data.txt), continuity of piecewise published
expansions, or limits that reduce to textbook constants.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle as O

MC2 = 0.51099895
RE = 2.8179403262e-13
ALPHA = 1 / 137.035999084
NA = 6.02214076e23
WATER, BONE, LUNG = 0, 1, 2
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "reference_data.txt")


def golden_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            q, mat, E, val, unit, tol, *src = line.split()
            rows.append((q, mat, float(E), float(val), float(tol), " ".join(src)))
    return rows


@pytest.mark.parametrize("row", golden_rows(), ids=lambda r: f"{r[0]}-{r[1]}-{r[2]}")
def test_reference_values(row):
    q, mat, E, val, tol, src = row
    if q == "mu_total":
        got = O.mu(WATER, E)
    elif q == "mu_compton":
        got = O.mu(WATER, E, 1)
    elif q == "S_col":
        got = O.L_col(WATER, E, 1e9)          # unrestricted: threshold above T/2
    elif q == "X0":
        got = 1.0 / (4 * ALPHA * RE ** 2 * O.material_const(WATER, 3))
    elif q == "sigma_thomson":
        k = E / MC2                            # Klein-Nishina -> Thomson as k -> 0
        got = O.sigma_kn(E) / 1e-24 / (1 - 2 * k + 26 / 5 * k * k)
    else:
        raise AssertionError(q)
    assert abs(got / val - 1) < tol, (q, got, val, src)


def kn_dsig_dmu(E, mu):
    """Klein-Nishina d(sigma)/d(cos theta) per electron (textbook form)."""
    k = E / MC2
    e = 1.0 / (1.0 + k * (1.0 - mu))
    return math.pi * RE ** 2 * e ** 2 * (e + 1.0 / e - (1.0 - mu ** 2))


@pytest.mark.parametrize("E", [0.01, 0.1, 0.5, 1.0, 2.0, 6.0, 20.0])
def test_klein_nishina_total_is_integral_of_differential(E):
    num, _ = integrate.quad(lambda m: kn_dsig_dmu(E, m), -1, 1, epsabs=0, epsrel=1e-12, limit=200)
    assert abs(O.sigma_kn(E) / num - 1) < 1e-9


def test_compton_mu_is_electron_density_times_kn():
    for m in (WATER, BONE, LUNG):
        for E in (0.05, 1.0, 10.0):
            assert abs(O.mu(m, E, 1) / (O.material_const(m, 0) * O.sigma_kn(E)) - 1) < 1e-14


def test_water_electron_density():
    # H2O: 10 electrons per 18.015 g/mol (composition by mass fractions)
    assert abs(O.material_const(WATER, 0) / (10 * NA / 18.015) - 1) < 2e-3


def test_photoelectric_scaling_laws():
    # K-shell Born form: E^(-7/2) at fixed material, Z^5 weighting across materials
    r = O.mu(WATER, 0.05, 2) / O.mu(WATER, 0.1, 2)
    assert abs(r / 2 ** 3.5 - 1) < 1e-12
    sigT = 8 * math.pi / 3 * RE ** 2
    per_z5 = 4 * math.sqrt(2) * ALPHA ** 4 * sigT * (MC2 / 0.1) ** 3.5
    # water: sum over H (Z=1) and O (Z=8) by mass fraction
    atoms = NA * np.array([0.111894 / 1.008, 0.888106 / 15.999])
    assert abs(O.mu(WATER, 0.1, 2) / (per_z5 * (atoms * np.array([1, 8 ** 5])).sum()) - 1) < 1e-3
    # magnitude against NIST XCOM water photoelectric at 100 keV (2.76e-3 cm2/g)
    assert 0.7 < O.mu(WATER, 0.1, 2) / 2.76e-3 < 1.5


def test_pair_threshold_and_continuity():
    assert O.mu(WATER, 2 * MC2, 3) == 0.0
    assert O.mu(WATER, 1.0, 3) == 0.0
    assert O.mu(WATER, 2 * MC2 * 1.01, 3) > 0.0
    k4 = 4 * MC2
    lo, hi = O.mu(BONE, k4 * (1 - 1e-12), 3), O.mu(BONE, k4 * (1 + 1e-12), 3)
    # Maximon's near-threshold and high-energy expansions meet at k = 4 mc^2
    assert abs(lo / hi - 1) < 1e-3
    # monotone growth and the asymptotic (28/9) ln(2k) slope
    Es = np.geomspace(1.1, 1000, 60)
    v = O.mu(WATER, Es, 3)
    assert np.all(np.diff(v) > 0)
    d = (O.mu(WATER, 2000.0, 3) - O.mu(WATER, 1000.0, 3)) / (ALPHA * RE ** 2 * O.material_const(WATER, 2))
    assert abs(d / (28 / 9 * math.log(2)) - 1) < 1e-3


def moller_dsig_dW(T, W, ne):
    tau = T / MC2
    g = tau + 1
    b2 = 1 - 1 / g ** 2
    e = W / T
    return (2 * math.pi * RE ** 2 * MC2 * ne / (b2 * T ** 2)) * (
        1 / e ** 2 + 1 / (1 - e) ** 2 + (tau / g) ** 2 - (2 * tau + 1) / g ** 2 / (e * (1 - e)))


@pytest.mark.parametrize("T", [0.5, 1.0, 5.0, 15.0])
@pytest.mark.parametrize("m", [WATER, BONE, LUNG])
def test_moller_total_is_integral_of_differential(T, m):
    ne = O.material_const(m, 0)
    wcc = 0.2
    num, _ = integrate.quad(lambda W: moller_dsig_dW(T, W, ne), wcc, T / 2, epsrel=1e-12, limit=200)
    assert abs(O.sigma_moller(m, T, wcc) / num - 1) < 1e-9


@pytest.mark.parametrize("T", [0.5, 1.0, 5.0, 15.0])
def test_restricted_collision_power_plus_hard_losses_is_unrestricted(T):
    """L(T; unrestricted) - L(T; Delta) = integral over W in [Delta, T/2] of W dsigma/dW."""
    ne = O.material_const(WATER, 0)
    wcc = 0.2
    hard, _ = integrate.quad(lambda W: W * moller_dsig_dW(T, W, ne), wcc, T / 2, epsrel=1e-12, limit=200)
    diff = O.L_col(WATER, T, 1e9) - O.L_col(WATER, T, wcc)
    assert abs(diff / hard - 1) < 1e-8


def test_collision_power_below_twice_threshold_is_unrestricted():
    assert O.L_col(WATER, 0.3, 0.2) == O.L_col(WATER, 0.3, 1e9)


def brems_dsig_dk(m, T, k):
    E = T + MC2
    y = k / E
    return 4 * ALPHA * RE ** 2 / k * ((4 / 3 - 4 / 3 * y + y * y) * O.material_const(m, 3)
                                      + (1 - y) * O.material_const(m, 4))


@pytest.mark.parametrize("T", [0.3, 2.0, 15.0])
@pytest.mark.parametrize("m", [WATER, BONE])
def test_brems_integrals(T, m):
    kc = 0.01
    sig, _ = integrate.quad(lambda k: brems_dsig_dk(m, T, k), kc, T, epsrel=1e-12, limit=200)
    assert abs(O.sigma_brems(m, T, kc) / sig - 1) < 1e-9
    lr, _ = integrate.quad(lambda k: k * brems_dsig_dk(m, T, k), 0, kc, epsrel=1e-12, limit=200)
    assert abs(O.L_rad(m, T, kc) / lr - 1) < 1e-9
    # the unrestricted radiative power is the full-spectrum energy integral
    lf, _ = integrate.quad(lambda k: k * brems_dsig_dk(m, T, k), 0, T, epsrel=1e-12, limit=200)
    assert abs(O.L_rad(m, T, 1e9) / lf - 1) < 1e-9


def test_brems_screening_constant_matches_composition():
    # S1 = N_A sum_i (w_i/A_i) Z(Z+1) ln(183 Z^-1/3) for water
    w = {1: (0.111894, 1.008), 8: (0.888106, 15.999)}
    s1 = sum(NA * wi / Ai * Z * (Z + 1) * math.log(183 * Z ** (-1 / 3)) for Z, (wi, Ai) in w.items())
    s1 /= (0.111894 + 0.888106)
    assert abs(O.material_const(WATER, 3) / s1 - 1) < 1e-12


def test_density_effect_limits_and_continuity():
    for m in (WATER, BONE, LUNG):
        C, x0, x1, a = (O.material_const(m, i) for i in (7, 8, 9, 10))
        tx = lambda x: MC2 * (math.sqrt(1 + 10 ** (2 * x)) - 1)   # T with log10(beta gamma) = x
        assert O.density_effect(m, tx(x0 - 0.05)) == 0.0
        # continuous at x0 (by construction of a) and at x1
        assert abs(O.density_effect(m, tx(x0 + 1e-9))) < 1e-6
        assert abs(O.density_effect(m, tx(x1 - 1e-9)) - O.density_effect(m, tx(x1 + 1e-9))) < 1e-6
        # asymptote 2 ln(10) x - C
        x = 4.0
        assert abs(O.density_effect(m, tx(x)) - (2 * math.log(10) * x - C)) < 1e-9
        # Sternheimer-Peierls: C = 2 ln(I / (h w_p)) + 1, h w_p = 28.816 sqrt(rho Z/A) eV
        hw = 28.816 * math.sqrt(O.material_const(m, 6) * O.material_const(m, 0) / NA)
        assert abs(C - (2 * math.log(O.material_const(m, 5) / hw) + 1)) < 1e-12


def lambda1_water_by_quadrature(T):
    """First transport cross section of the screened Rutherford model, by
    quadrature over cos(theta) of (1 - mu) d sigma / d mu for H and O."""
    pc = math.sqrt(T * (T + 2 * MC2))
    b = pc / (T + MC2)
    tot = 0.0
    for Z, w, A in ((1, 0.111894, 1.008), (8, 0.888106, 15.999)):
        eta = 0.25 * (ALPHA * Z ** (1 / 3) * MC2 / (0.885 * pc)) ** 2 * (1.13 + 3.76 * (ALPHA * Z / b) ** 2)
        pref = 2 * math.pi * Z * (Z + 1) * RE ** 2 * (MC2 / (pc * b)) ** 2
        f = lambda u: u / (u + 2 * eta) ** 2                        # u = 1 - mu
        val, _ = integrate.quad(f, 0, 2, points=[eta, 10 * eta, 100 * eta], epsrel=1e-11, limit=400)
        tot += NA * w / A * pref * val
    return tot


@pytest.mark.parametrize("T", [0.2, 1.0, 15.0])
def test_lambda1_is_integral_of_screened_rutherford(T):
    assert abs(O.lambda1_inv(WATER, T) / lambda1_water_by_quadrature(T) - 1) < 1e-7


@pytest.mark.parametrize("A", [1e-8, 1e-4, 0.01, 0.3, 3.0, 50.0, 2e3, 1e6])
def test_wentzel_mean_by_quadrature(A):
    # p(u) = 2A(1+A)/(u+2A)^2 on [0,2]; integrate in v = ln(u + 2A), du = e^v dv
    a, b = math.log(2 * A), math.log(2 + 2 * A)
    norm, _ = integrate.quad(lambda v: 2 * A * (1 + A) * math.exp(-v), a, b, epsrel=1e-13, limit=400)
    mean, _ = integrate.quad(lambda v: 2 * A * (1 + A) * (math.exp(v) - 2 * A) * math.exp(-v), a, b,
                             epsrel=1e-13, limit=400)
    assert abs(norm - 1) < 1e-9
    assert abs(O.ms_mean_u(A) / mean - 1) < 1e-8


@pytest.mark.parametrize("G1", [1e-9, 1e-5, 1e-2, 0.3, 2.0, 10.0])
def test_wentzel_screening_solves_first_moment(G1):
    A = O.ms_solve_A(G1)
    assert abs(O.ms_mean_u(A) / (-math.expm1(-G1)) - 1) < 1e-10


@pytest.mark.parametrize("m,T,X", [(WATER, 15.0, 1.0), (WATER, 1.0, 0.02), (BONE, 5.0, 0.3), (LUNG, 0.4, 0.005)])
def test_csda_rk4_against_ode_solver(m, T, X):
    p = O.params()
    L = lambda t: O.L_col(m, t, p.w_cc) + O.L_rad(m, t, p.w_cb)
    sol = integrate.solve_ivp(lambda x, y: [-L(y[0])], (0, X), [T], rtol=1e-12, atol=1e-14, method="DOP853")
    assert abs(O.csda_loss(m, T, X, p) / sol.y[0, -1] - 1) < 1e-9


def test_stratified_bins_exact():
    import ocmc_inputs as I
    edges, w = I.spectrum_6mv()
    for n in (1, 7, 1000, 12345, 10 ** 9 + 7):
        b, order = O.stratify(edges, w, n)
        assert b[0] == 0 and b[-1] == n and np.all(np.diff(b.astype(np.int64)) >= 0)
        # highest-energy bin first
        assert list(order) == list(range(len(w) - 1, -1, -1))
        counts = np.diff(b.astype(np.int64))
        assert np.all(np.abs(counts - n * w[order].astype(np.float64) / w.astype(np.float64).sum()) <= 1.0 + 1e-9)
