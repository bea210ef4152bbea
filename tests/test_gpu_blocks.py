"""GPU building blocks against the oracle and analytic distributions, through the C ABI.

RNG and source sampling are compared element by element (same Philox stream,
same uniform-variate definition); tables against the oracle's closed forms;
samplers by chi-square against the analytic distributions.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import ocmc_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu
MC2 = 0.51099895


@pytest.fixture(scope="module")
def ocmc():
    from paper_1503_01722_gb300 import build
    build.build()
    from paper_1503_01722_gb300 import ocmc as m
    return m


@pytest.fixture(scope="module")
def eng(ocmc):
    e = ocmc.Engine(0)
    ph = I.slab((40, 40, 40), (0.75, 0.75, 0.75))
    e.create_phantom(ph)
    yield e
    e.close()


def test_philox_bit_exact(ocmc):
    rng = np.random.default_rng(3)
    for _ in range(6):
        key = [int(x) for x in rng.integers(0, 2 ** 32, 2)]
        c1, c2, c3 = (int(x) for x in rng.integers(0, 2 ** 32, 3))
        first = int(rng.integers(0, 2 ** 31))
        got = ocmc.test_philox(key, c1, c2, c3, first, 257)
        ref = np.stack([O.philox((first + j, c1, c2, c3), key) for j in range(257)])
        assert np.array_equal(got, ref)


def test_rotation_vs_oracle(ocmc):
    """The kernel's FP32 rotation against the oracle's (pinned by momentum and angle tests),
    direction by direction, including the poles and FP32 directions a hair away from them."""
    rng = np.random.default_rng(17)
    n = 20000
    d = rng.normal(size=(n, 3))
    d[:8] = [[0, 0, 1], [0, 0, -1], [1e-7, 0, 1], [0, -3e-6, -1], [2e-4, 1e-4, 1], [-1e-3, 0, -1],
             [1, 0, 0], [0, 1, 1e-6]]
    d = (d / np.linalg.norm(d, axis=1)[:, None]).astype(np.float32)
    mu = rng.uniform(-1, 1, n).astype(np.float32)
    mu[:4000:7] = 1.0 - rng.uniform(0, 1e-3, len(mu[:4000:7])).astype(np.float32)   # small deflections
    xi = rng.uniform(0, 1, n).astype(np.float32)
    got = ocmc.test_rotate(d, mu, xi).astype(np.float64)
    ref = O.rotate(d.astype(np.float64), mu.astype(np.float64), 2 * math.pi * xi.astype(np.float64))
    assert np.max(np.abs(np.linalg.norm(got, axis=1) - 1)) < 1e-6
    assert np.max(np.abs(got - ref)) < 2e-5


@pytest.mark.parametrize("case", ["photon_point", "electron_parallel", "oblique_miss"])
def test_source_elementwise(ocmc, case):
    if case == "photon_point":
        ph, beam = I.photon_slab_120()
    elif case == "electron_parallel":
        ph, beam = I.electron_water_61()
    else:
        ph = I.homogeneous((30, 20, 10), (0.5, 0.5, 0.5))
        beam = I.Beam(0, *I.spectrum_6mv(), (40.0, 40.0), 60.0, (7.5, 5.0, 2.5), (0.6, 0.0, 0.8))
    n = 20011
    with ocmc.Engine(0) as e:
        e.create_phantom(ph)
        e.set_source(beam)
        g = e.test_source(n, seed=77)
    r = O.source_sample(ph, beam, n, seed=77)
    hit = r[:, 7] == 1
    assert np.array_equal(g[:, 7] == 1, hit)
    if case == "oblique_miss":
        assert 0 < hit.sum() < n
    # identical energies up to FP32 rounding: the same draw and the same bin for every history
    assert np.allclose(g[:, 6], r[:, 6], rtol=2e-7, atol=0)
    assert np.allclose(g[hit, :3], r[hit, :3], rtol=0, atol=2e-4)
    assert np.allclose(g[hit, 3:6], r[hit, 3:6], rtol=0, atol=2e-6)


def test_tables_against_closed_forms(eng):
    E = np.geomspace(0.0105, 29.0, 997).astype(np.float32)
    for m in range(3):
        t = eng.test_tables(m, E).astype(np.float64)
        Ed = E.astype(np.float64)
        for col, ref in ((0, O.mu(m, Ed)), (1, O.mu(m, Ed, 1)), (2, O.mu(m, Ed, 2))):
            assert np.max(np.abs(t[:, col] / ref - 1)) < 1e-3, (m, col)
        sel = Ed > 0.05
        assert np.max(np.abs(t[sel, 4] / O.lambda1_inv(m, Ed[sel]) - 1)) < 1e-3
        sm = O.sigma_moller(m, Ed)
        sb = O.sigma_brems(m, Ed)
        ok = sm > 0
        # Moller rises steeply from zero at 2 w_cc; compare away from threshold
        far = Ed > 0.45
        assert np.max(np.abs(t[far, 5] / sm[far] - 1)) < 2e-3
        assert np.max(np.abs(t[:, 6][sb > 0] / sb[sb > 0] - 1)) < 2e-3
        # the hard-event majorant bounds the exact cross section over the step's energy window
        for j in range(0, len(E), 37):
            w = np.linspace(E[j] * 0.95, E[j], 9)
            exact = O.sigma_moller(m, w) + O.sigma_brems(m, w)
            assert t[j, 7] >= exact.max() * (1 - 1e-6), (m, E[j])
        assert ok.any()
        # range differences against the integral of 1/L
        L = lambda x: O.L_col(m, x, 0.2) + O.L_rad(m, x, 0.01)
        for a, b in ((0.2, 1.0), (1.0, 6.0), (6.0, 20.0)):
            ia, ib = np.searchsorted(E, a), np.searchsorted(E, b)
            num = integrate.quad(lambda x: 1 / L(x), E[ia], E[ib], epsrel=1e-10)[0]
            assert abs((t[ib, 3] - t[ia, 3]) / num - 1) < 2e-3, (m, a, b)


def test_csda_step_against_rk4(eng):
    rng = np.random.default_rng(5)
    p = O.params()
    for m in range(3):
        T = np.exp(rng.uniform(np.log(0.21), np.log(20.0), 200)).astype(np.float32)
        frac = rng.uniform(0.0, 1.0, 200)
        X = np.empty(200, np.float32)
        for j, t in enumerate(T):
            L = O.L_col(m, float(t), 0.2) + O.L_rad(m, float(t), 0.01)
            X[j] = frac[j] * 0.05 * float(t) / L          # up to ~5 % energy loss
        got = eng.test_csda(m, T, X).astype(np.float64)
        ref = np.array([O.csda_loss(m, float(t), float(x), p) for t, x in zip(T, X)])
        dE_got, dE_ref = T - got, T - ref
        big = dE_ref > 1e-3 * T
        assert np.max(np.abs(dE_got[big] / dE_ref[big] - 1)) < 5e-3, m
        assert np.all(got <= T)


def _chi2(samples, edges, probs):
    counts, _ = np.histogram(samples, bins=edges)
    exp = probs / probs.sum() * len(samples)
    keep = exp > 5
    chi2 = ((counts[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    return stats.chi2.sf(chi2, keep.sum() - 1)


def _bin_probs(pdf, edges):
    return np.array([integrate.quad(pdf, a, b, epsrel=1e-10)[0] for a, b in zip(edges[:-1], edges[1:])])


@pytest.mark.parametrize("E", [0.1, 1.0, 10.0])
def test_compton_sampler(eng, ocmc, E):
    mu = eng.test_sample(ocmc.SAMPLE_COMPTON, E, 400_000, seed=21).astype(np.float64)
    k = E / MC2

    def pdf(m):
        e = 1 / (1 + k * (1 - m))
        return e * e * (e + 1 / e - (1 - m * m))

    edges = np.linspace(-1, 1, 41) if E < 10 else np.concatenate([np.linspace(-1, 0.9, 20), np.linspace(0.9, 1, 21)[1:]])
    assert _chi2(mu, edges, _bin_probs(pdf, edges)) > 1e-3


@pytest.mark.parametrize("T", [0.6, 3.0, 15.0])
def test_moller_sampler(eng, ocmc, T):
    eps = eng.test_sample(ocmc.SAMPLE_MOLLER, T, 400_000, seed=22).astype(np.float64)
    tau = T / MC2
    g = tau + 1
    pdf = lambda e: 1 / e ** 2 + 1 / (1 - e) ** 2 + (tau / g) ** 2 - (2 * tau + 1) / g ** 2 / (e * (1 - e))
    edges = np.geomspace(0.2 / T, 0.5, 41)
    assert _chi2(eps, edges, _bin_probs(pdf, edges)) > 1e-3


@pytest.mark.parametrize("T,m", [(0.5, 0), (5.0, 1), (15.0, 2)])
def test_brems_sampler(eng, ocmc, T, m):
    k = eng.test_sample(ocmc.SAMPLE_BREMS, T, 400_000, seed=23, material=m).astype(np.float64)
    S1, S2 = O.material_const(m, 3), O.material_const(m, 4)
    E = T + MC2
    pdf = lambda x: ((4 / 3 - 4 / 3 * x / E + (x / E) ** 2) * S1 + (1 - x / E) * S2) / x
    edges = np.geomspace(0.01, T, 41)
    assert _chi2(k, edges, _bin_probs(pdf, edges)) > 1e-3


@pytest.mark.parametrize("G1", [1e-3, 0.05, 0.5, 3.0])
def test_ms_sampler(eng, ocmc, G1):
    n = 400_000
    mu = eng.test_sample(ocmc.SAMPLE_MS, 1.0, n, seed=24, aux=G1).astype(np.float64)
    u = 1 - mu
    assert abs(u.mean() + math.expm1(-G1)) < 4 * u.std() / math.sqrt(n) + 2e-4 * (-math.expm1(-G1))
    A = O.ms_solve_A(G1)
    cdf = lambda x: (1 + A) * x / (x + 2 * A)
    edges = np.concatenate([[0], np.geomspace(A * 0.05, 2, 40)])
    assert _chi2(u, edges, np.diff([cdf(x) for x in edges])) > 1e-3
