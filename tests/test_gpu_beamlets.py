"""Batched beamlets (one graph-captured persistent launch, per-beamlet sparse tallies)
and the autotuner, through the C ABI.

Beamlet b uses random streams tagged 0x80000000 | b, so a dense single-beam run of
the same source with that stream tag must reproduce its sparse tally bit for bit;
the dense path itself is parity-tested against the oracle."""
import numpy as np
import pytest

import ocmc_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ocmc():
    from paper_1503_01722_gb300 import build
    build.build()
    from paper_1503_01722_gb300 import ocmc as m
    return m


@pytest.fixture(scope="module")
def setup():
    ph = I.ct_like(n=(64, 64, 32), voxel=(0.8, 0.8, 0.8), seed=3)
    spec = I.spectrum_6mv()
    bl = I.beamlets(ph, n_beamlets=24, seed=2, log10_mean=3.4, log10_sd=0.4, lo=500, hi=20_000, offset=3.0)
    return ph, spec, bl


def dense_of(ph, idx, raw):
    d = np.zeros(ph.density.size, np.int64)
    d[idx] = raw
    return d


def single_beam_tally(ocmc, ph, spec, b, blist, seed):
    B = blist[b]
    beam = I.Beam(0, spec[0], spec[1], B["field"], B["ssd"], B["iso"], B["direction"])
    with ocmc.Engine(0, stream_tag=0x80000000 | b) as e:
        e.create_phantom(ph)
        e.set_source(beam)
        e.run(B["n_histories"], seed=seed)
        return e.raw_tally().sum(axis=0).ravel()


def test_beamlets_match_dense_runs_and_replay(ocmc, setup):
    ph, spec, bl = setup
    with ocmc.Engine(0) as e:
        e.create_phantom(ph)
        e.set_beamlets(0, spec[0], spec[1], bl)
        e.run_beamlets(seed=5)
        st1 = e.stats()
        outs = [e.beamlet_dose(b) for b in range(len(bl))]
        e.run_beamlets(seed=5)           # graph replay
        outs2 = [e.beamlet_dose(b) for b in range(len(bl))]
        st2 = e.stats()
        batch = e.beamlet_doses(raw=True)     # every beamlet through reused pinned buffers
        plain = e.beamlet_doses()
    for (i1, d1, r1), (i2, d2, r2), (i3, d3, r3), (i4, d4) in zip(outs, outs2, batch, plain):
        assert np.array_equal(i1, i2) and np.array_equal(r1, r2) and np.array_equal(d1, d2)
        assert np.array_equal(i1, i3) and np.array_equal(r1, r3) and np.array_equal(d1, d3)
        assert np.array_equal(i1, i4) and np.array_equal(d1, d4)
    # a beamlet run replaces its tallies and its statistics
    assert st2["histories"] == st1["histories"] == sum(b["n_histories"] for b in bl)
    assert st2["lane_steps"] == st1["lane_steps"]
    for b in (0, 7, 23):
        idx, dose, raw = outs[b]
        assert len(idx) > 0 and np.all(np.diff(idx) > 0) and np.all(raw > 0)
        ref = single_beam_tally(ocmc, ph, spec, b, bl, seed=5)
        assert np.array_equal(dense_of(ph, idx, raw), ref)
        V = np.prod(ph.voxel)
        rho = ph.density.ravel()[idx].astype(np.float64)
        expect = raw / 2.0 ** 28 / (rho * V * bl[b]["n_histories"])
        assert np.allclose(dose, expect, rtol=1e-6)


def test_tables_that_overflow_are_enlarged_with_identical_result(ocmc, setup):
    ph, spec, bl = setup
    res = []
    for scale in (0.0, 0.002):
        with ocmc.Engine(0, beamlet_capacity_scale=scale) as e:
            e.create_phantom(ph)
            e.set_beamlets(0, spec[0], spec[1], bl[:6])
            e.run_beamlets(seed=11)
            res.append([e.beamlet_dose(b)[2] for b in range(6)])
    for a, b in zip(*res):
        assert np.array_equal(a, b)


def test_beamlet_dose_statistically_matches_oracle(ocmc, setup):
    ph, spec, bl = setup
    # a widened beamlet (3x3 cm2) gives a 10%-isodose region of several hundred voxels
    b = 4
    B = dict(bl[b])
    B["field"] = (3.0, 3.0)
    B["n_histories"] = 150_000
    beam = I.Beam(0, spec[0], spec[1], B["field"], B["ssd"], B["iso"], B["direction"])
    with ocmc.Engine(0, n_batches=50, stream_tag=0x80000000 | b) as e:
        e.create_phantom(ph)
        e.set_source(beam)
        e.run(B["n_histories"], seed=3)
        D, S = e.dose()
    r = O.run(ph, beam, B["n_histories"], seed=3, p=O.params(n_batches=50))
    Dr, Sr = r.dose()
    # tissue only: the air around the body (0.0012 g/cm^3) has a huge, noisy dose per mass
    tissue = ph.density >= 0.1
    dmax = Dr[tissue].max()
    mask = tissue & (Dr >= 0.1 * dmax)
    z = np.abs(D - Dr)[mask] / np.sqrt(S ** 2 + Sr ** 2)[mask]
    assert mask.sum() > 300
    assert np.mean(z <= 3) >= 0.99
    assert abs((D - Dr)[mask].mean() / dmax) < 0.005


def test_autotune_keeps_the_dose(ocmc):
    ph = I.scaled(I.slab(), 3)
    beam = I.beam_on(ph, 0, I.spectrum_6mv(), (10, 10), 100.0)
    with ocmc.Engine(0) as e:
        e.create_phantom(ph)
        e.set_source(beam)
        e.run(50_000, seed=2)
        ref = e.raw_tally()
        p = e.autotune(100_000)
        assert (p.max_registers, p.block_threads) in ((64, 1024), (64, 512), (80, 256), (56, 384))
        assert p.switch_high in (2048, 4096, 7680) and p.e_class_split in (0.0, 2.0)
        e.run(50_000, seed=2)
        assert np.array_equal(e.raw_tally(), ref)
