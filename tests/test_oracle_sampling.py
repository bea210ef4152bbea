"""Chi-square pins of the oracle's samplers against analytic distributions.

Bin probabilities come from quadrature of the textbook differential cross
sections (written out here), not from the oracle. Seeds are fixed, so the
statistics are deterministic; the bound p > 0.01 is the acceptance level
required of the Klein-Nishina test and is reused for the other samplers.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle as O

MC2 = 0.51099895


def chi2_p(samples, edges, probs):
    counts, _ = np.histogram(samples, bins=edges)
    exp = probs / probs.sum() * len(samples)
    keep = exp > 5
    chi2 = ((counts[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    return stats.chi2.sf(chi2, keep.sum() - 1)


def bin_probs(pdf, edges):
    return np.array([integrate.quad(pdf, a, b, epsrel=1e-10)[0] for a, b in zip(edges[:-1], edges[1:])])


@pytest.mark.parametrize("E", [0.1, 1.0, 10.0])
def test_klein_nishina_angles(E):
    n = 200_000
    mu = O.sample(O.SAMPLE_KN_MU, E, n, seed=11)
    k = E / MC2

    def pdf(m):
        e = 1 / (1 + k * (1 - m))
        return e * e * (e + 1 / e - (1 - m * m))

    edges = np.linspace(-1, 1, 41)
    if E >= 10:
        edges = np.concatenate([np.linspace(-1, 0.9, 20), np.linspace(0.9, 1, 21)[1:]])
    assert chi2_p(mu, edges, bin_probs(pdf, edges)) > 0.01


@pytest.mark.parametrize("T", [0.6, 3.0, 15.0])
def test_moller_energy_transfer(T):
    n = 200_000
    wcc = 0.2
    eps = O.sample(O.SAMPLE_MOLLER_EPS, T, n, seed=12, p=O.params(w_cc=wcc))
    tau = T / MC2
    g = tau + 1
    pdf = lambda e: 1 / e ** 2 + 1 / (1 - e) ** 2 + (tau / g) ** 2 - (2 * tau + 1) / g ** 2 / (e * (1 - e))
    e0 = wcc / T
    edges = np.geomspace(e0, 0.5, 41)
    assert eps.min() >= e0 and eps.max() <= 0.5
    assert chi2_p(eps, edges, bin_probs(pdf, edges)) > 0.01


@pytest.mark.parametrize("T,m", [(0.5, 0), (5.0, 1), (15.0, 0)])
def test_brems_photon_energy(T, m):
    n = 200_000
    kc = 0.01
    k = O.sample(O.SAMPLE_BREMS_K, T, n, seed=13, m=m, p=O.params(w_cb=kc))
    S1, S2 = O.material_const(m, 3), O.material_const(m, 4)
    E = T + MC2
    pdf = lambda x: ((4 / 3 - 4 / 3 * x / E + (x / E) ** 2) * S1 + (1 - x / E) * S2) / x
    edges = np.geomspace(kc, T, 41)
    assert k.min() >= kc and k.max() <= T
    assert chi2_p(k, edges, bin_probs(pdf, edges)) > 0.01


@pytest.mark.parametrize("G1", [1e-3, 0.05, 0.5, 3.0])
def test_multiple_scattering_angle(G1):
    n = 200_000
    mu = O.sample(O.SAMPLE_MS_MU, 1.0, n, seed=14, aux=G1)
    u = 1 - mu
    # first moment: <1 - cos theta> = 1 - exp(-G1) (Goudsmit-Saunderson / Lewis)
    target = -math.expm1(-G1)
    assert abs(u.mean() - target) < 4 * u.std() / math.sqrt(n)
    # full shape: Wentzel p(u) ~ (u + 2A)^-2 with the solved A
    A = O.ms_solve_A(G1)
    cdf = lambda x: (1 + A) * x / (x + 2 * A)
    edges = np.concatenate([[0], np.geomspace(A * 1e-2, 2, 40)])
    probs = np.diff([cdf(x) for x in edges])
    assert chi2_p(u, edges, probs) > 0.01
