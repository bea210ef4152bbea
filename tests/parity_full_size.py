"""Full-size dose parity of the engine with the CPU oracle: the 6 MV slab workload (120^3 at
0.25 cm, 10x10 cm^2 at SSD 100) at 10^8 histories each, on independent seeds (GPU 2, oracle 1),
the history count at which the agreement
criterion is stated (|D_gpu - D_oracle| <= 3 sigma_combined in >= 99 % of the voxels above the
10 % isodose, mean difference < 0.5 % of D_max there).

Not a pytest module (the oracle needs hours of CPU time for 10^8 histories). Three steps:

    python tests/parity_full_size.py gpu --out gpu.npz          # on a GB300: dose and sigma
    python tests/parity_full_size.py oracle --out oracle.npz    # host cores, resumable chunks
    python tests/parity_full_size.py compare gpu.npz oracle.npz # prints the statistics (JSON)
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import ocmc_inputs as I  # noqa: E402

N_HIST = 100_000_000
SEED = 1          # the oracle leg
GPU_SEED = 2      # the GPU leg: an independent sample, so sigma_combined is the right yardstick
BATCHES = 10


def run_gpu(out):
    from paper_1503_01722_gb300 import build
    build.build()
    from paper_1503_01722_gb300 import ocmc
    ph, beam = I.photon_slab_120()
    with ocmc.Engine(0, n_batches=BATCHES) as e:
        e.create_phantom(ph)
        e.set_source(beam)
        e.run(N_HIST, seed=GPU_SEED)
        D, S = e.dose()
        st = e.stats()
    np.savez_compressed(out, dose=D, sigma=S, n=N_HIST, seed=GPU_SEED, stats=json.dumps(st))


def run_oracle(out, chunks=20, threads=None):
    """Histories [k N/chunks, (k+1) N/chunks) per chunk; the summed int64 tally is saved after
    every chunk, so a stopped run resumes where it stopped."""
    import oracle as O
    ph, beam = I.photon_slab_120()
    p = O.params(n_batches=BATCHES)
    bounds = np.linspace(0, N_HIST, chunks + 1).astype(np.int64)
    done, tally = 0, None
    if os.path.exists(out):
        z = np.load(out)
        done, tally = int(z["chunks_done"]), z["tally"]
    for k in range(done, chunks):
        t = time.perf_counter()
        r = O.run(ph, beam, N_HIST, seed=SEED, p=p, first=int(bounds[k]), count=int(bounds[k + 1] - bounds[k]),
                  threads=threads, n_total=N_HIST)
        tally = r.tally if tally is None else tally + r.tally
        np.savez(out + ".tmp.npz", tally=tally, chunks_done=k + 1)
        os.replace(out + ".tmp.npz", out)
        print(f"chunk {k + 1}/{chunks}: {time.perf_counter() - t:.0f} s", flush=True)


def compare(gpu_file, oracle_file):
    import oracle as O
    ph, _ = I.photon_slab_120()
    g = np.load(gpu_file)
    z = np.load(oracle_file)
    D, S = g["dose"], g["sigma"]
    Dr, Sr = O.finalize(z["tally"], ph, N_HIST)
    m = Dr >= 0.1 * Dr.max()
    comb = np.sqrt(S ** 2 + Sr ** 2)[m]
    diff = (D - Dr)[m]
    res = {"histories": N_HIST, "gpu_seed": int(g["seed"]) if "seed" in g else None, "oracle_seed": SEED,
           "voxels_in_10pct_isodose": int(m.sum()),
           "within_3_sigma": float(np.mean(np.abs(diff) <= 3 * comb)),
           "within_2_sigma": float(np.mean(np.abs(diff) <= 2 * comb)),
           "mean_signed_diff_over_dmax": float(diff.mean() / Dr.max()),
           "mean_abs_diff_over_dmax": float(np.abs(diff).mean() / Dr.max()),
           "mean_sigma_over_d": float(np.mean(Sr[m] / Dr[m])),
           "oracle_chunks": int(z["chunks_done"])}
    print(json.dumps(res))
    return res


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    a = sub.add_parser("gpu")
    a.add_argument("--out", required=True)
    b = sub.add_parser("oracle")
    b.add_argument("--out", required=True)
    b.add_argument("--threads", type=int, default=None)
    c = sub.add_parser("compare")
    c.add_argument("gpu")
    c.add_argument("oracle")
    args = ap.parse_args()
    if args.cmd == "gpu":
        run_gpu(args.out)
    elif args.cmd == "oracle":
        run_oracle(args.out, threads=args.threads)
    else:
        compare(args.gpu, args.oracle)


if __name__ == "__main__":
    main()
