"""The allocation-free entry point (ocmc_run_noalloc) through the C ABI.

It serves callers that cannot allocate device memory (code under another
framework's allocator, hosts that forbid allocation after start-up, plug-ins
handed only device pointers). Its scratch is one static device array shared by
every call, so two calls in a row are checked: each must give the same tally as
the context entry point (ocmc_create_phantom + ocmc_run_range) on the same input,
bit for bit (integer tallies, lineage-keyed random numbers). This file is named
to be collected last."""
import numpy as np
import pytest

import ocmc_inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ocmc():
    from paper_1503_01722_gb300 import build
    build.build()
    from paper_1503_01722_gb300 import ocmc as m
    return m


def context_tally(ocmc, ph, beam, n, first, count, seed):
    with ocmc.Engine(0) as e:
        e.create_phantom(ph)
        e.set_source(beam)
        e.run_range(first, count, n, seed=seed)
        return e.raw_tally()


def noalloc_tally(ocmc, ph, beam, n, first, count, seed):
    import torch
    dens = torch.from_numpy(np.ascontiguousarray(ph.density)).cuda()
    mat = torch.from_numpy(np.ascontiguousarray(ph.material)).cuda()
    tally = torch.zeros((10,) + ph.density.shape, dtype=torch.int64, device="cuda")
    ocmc.run_noalloc(dens, mat, ph.voxel, beam, tally, first, count, n, seed=seed)
    torch.cuda.synchronize()
    return tally.cpu().numpy()


def test_noalloc_matches_context_entry_point_on_two_calls_in_a_row(ocmc):
    # call 1: 6 MV photons on the (coarsened) slab phantom
    ph1 = I.scaled(I.slab(), 3)
    b1 = I.beam_on(ph1, 0, I.spectrum_6mv(), (10, 10), 100.0)
    # call 2: another phantom, particle type, grid shape and seed, over a sub-range of the run
    ph2 = I.random_phantom()
    b2 = I.beam_on(ph2, 1, I.mono(12.0), (5, 4), 90.0)
    cases = [(ph1, b1, 40_000, 0, 40_000, 7), (ph2, b2, 9_000, 1_000, 6_000, 8)]
    for ph, beam, n, first, count, seed in cases:
        got = noalloc_tally(ocmc, ph, beam, n, first, count, seed)
        ref = context_tally(ocmc, ph, beam, n, first, count, seed)
        assert ref.sum() > 0
        assert np.array_equal(got, ref)


def test_noalloc_rejects_launch_shape_beyond_static_scratch(ocmc):
    import torch
    ph = I.homogeneous((8, 8, 8), (1.0, 1.0, 1.0))
    beam = I.beam_on(ph, 0, I.mono(1.0), (4, 4), 100.0)
    dens = torch.from_numpy(np.ascontiguousarray(ph.density)).cuda()
    mat = torch.from_numpy(np.ascontiguousarray(ph.material)).cuda()
    tally = torch.zeros((10,) + ph.density.shape, dtype=torch.int64, device="cuda")
    p = ocmc.default_params(stack_capacity=1 << 20, blocks_per_sm=4)
    with pytest.raises(ocmc.OcmcError) as e:
        ocmc.run_noalloc(dens, mat, ph.voxel, beam, tally, 0, 100, 100, params=p)
    assert e.value.status == ocmc.ERR_ARG and "static" in str(e.value)
    assert int(tally.abs().sum()) == 0


@pytest.mark.parametrize("case", ["photon_slab_120_1e7", "electron_water_61_2e5"])
def test_noalloc_default_parameters_keep_stacks_from_overflowing(ocmc, case):
    """With default parameters (256-record stacks) the type switch stays on, so showers with
    many secondaries finish without overflow, and the tally equals the context entry point's."""
    if case == "photon_slab_120_1e7":
        ph, beam = I.photon_slab_120()
        n = 10_000_000
    else:
        ph, beam = I.electron_water_61()
        n = 200_000
    got = noalloc_tally(ocmc, ph, beam, n, 0, n, 3)      # raises OcmcError on OCMC_ERR_OVERFLOW
    ref = context_tally(ocmc, ph, beam, n, 0, n, 3)
    assert np.array_equal(got, ref)


def test_noalloc_rejects_bad_phantom_before_transport(ocmc):
    import torch
    ph = I.homogeneous((8, 8, 8), (1.0, 1.0, 1.0))
    beam = I.beam_on(ph, 0, I.mono(1.0), (4, 4), 100.0)
    dens = torch.from_numpy(np.ascontiguousarray(ph.density)).cuda()
    material = np.ascontiguousarray(ph.material).copy()
    material[3, 4, 5] = 7                                 # no such built-in material
    mat = torch.from_numpy(material).cuda()
    tally = torch.zeros((10,) + ph.density.shape, dtype=torch.int64, device="cuda")
    with pytest.raises(ocmc.OcmcError) as e:
        ocmc.run_noalloc(dens, mat, ph.voxel, beam, tally, 0, 1000, 1000)
    assert e.value.status == ocmc.ERR_ARG and "phantom" in str(e.value)
    assert int(tally.abs().sum()) == 0
    # the library still works after the rejected call
    ok = noalloc_tally(ocmc, ph, beam, 1000, 0, 1000, 1)
    assert ok.sum() > 0


def test_noalloc_checks_tensors_on_the_host(ocmc):
    import torch
    ph = I.homogeneous((8, 8, 8), (1.0, 1.0, 1.0))
    beam = I.beam_on(ph, 0, I.mono(1.0), (4, 4), 100.0)
    dens = torch.from_numpy(np.ascontiguousarray(ph.density)).cuda()
    mat = torch.from_numpy(np.ascontiguousarray(ph.material)).cuda()
    bad = [
        (dens, mat, torch.zeros(ph.density.shape, dtype=torch.int64, device="cuda")),      # no batch axis
        (dens, mat, torch.zeros((10,) + ph.density.shape, dtype=torch.float64, device="cuda")),
        (dens.double(), mat, torch.zeros((10,) + ph.density.shape, dtype=torch.int64, device="cuda")),
        (dens, mat[:4], torch.zeros((10,) + ph.density.shape, dtype=torch.int64, device="cuda")),
        (dens.cpu(), mat, torch.zeros((10,) + ph.density.shape, dtype=torch.int64, device="cuda")),
    ]
    for d, m, t in bad:
        with pytest.raises(ValueError):
            ocmc.run_noalloc(d, m, ph.voxel, beam, t, 0, 100, 100)
