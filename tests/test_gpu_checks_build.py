"""The checks build (libocmc_checks.so, -DOCMC_CHECKS=1): voxel indices, tally addresses and
stack slots are checked before every access in the transport kernel. On valid inputs no check
may fire, and the tallies must equal the normal build's bit for bit (the checks add branches,
no arithmetic). The checks library runs in a child process (OCMC_CHECKS=1 selects it)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import ocmc_inputs as I

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import ocmc_inputs as I
from paper_1503_01722_gb300 import ocmc
assert ocmc._LIB_PATH.endswith("libocmc_checks.so")
out = {}
for name, (ph, beam, n, kw) in {
        "photon_slab": (*(lambda ph: (ph, I.beam_on(ph, 0, I.spectrum_6mv(), (10, 10), 100.0)))(I.scaled(I.slab(), 3)),
                        200_000, {}),
        "electron_half_slab": (*(lambda ph: (ph, I.beam_on(ph, 1, I.mono(15.0), (10, 10), 100.0)))(
            I.scaled(I.half_slab(), 3)), 20_000, {}),
        "electron_random_cross": (*(lambda ph: (ph, I.beam_on(ph, 1, I.mono(12.0), (5, 4), 90.0)))(I.random_phantom()),
                                  20_000, {"flags": 16}),
}.items():
    with ocmc.Engine(0, **kw) as e:
        e.create_phantom(ph)
        e.set_source(beam)
        e.run(n, seed=7)
        e.dose()                         # raises on OCMC_ERR_BOUNDS
        t = e.raw_tally()
        np.save(sys.argv[2] + "_" + name + ".npy", t)
        out[name] = int(t.sum())
print(json.dumps(out))
"""


@pytest.fixture(scope="module")
def ocmc():
    from paper_1503_01722_gb300 import build
    build.build()
    from paper_1503_01722_gb300 import ocmc as m
    return m


def test_checks_build_matches_normal_build(ocmc, tmp_path):
    from paper_1503_01722_gb300 import build
    build.build(checks=True)
    prefix = str(tmp_path / "t")
    env = dict(os.environ, OCMC_CHECKS="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, prefix], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    cases = {
        "photon_slab": ((lambda ph: (ph, I.beam_on(ph, 0, I.spectrum_6mv(), (10, 10), 100.0)))(I.scaled(I.slab(), 3)),
                        200_000, {}),
        "electron_half_slab": ((lambda ph: (ph, I.beam_on(ph, 1, I.mono(15.0), (10, 10), 100.0)))(
            I.scaled(I.half_slab(), 3)), 20_000, {}),
        "electron_random_cross": ((lambda ph: (ph, I.beam_on(ph, 1, I.mono(12.0), (5, 4), 90.0)))(I.random_phantom()),
                                  20_000, {"flags": 16}),
    }
    for name, ((ph, beam), n, kw) in cases.items():
        with ocmc.Engine(0, **kw) as e:
            e.create_phantom(ph)
            e.set_source(beam)
            e.run(n, seed=7)
            ref = e.raw_tally()
        got = np.load(prefix + "_" + name + ".npy")
        assert ref.sum() > 0
        assert np.array_equal(got, ref), name
