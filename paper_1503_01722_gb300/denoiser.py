"""Learned dose denoiser: training data made by the engine, the training loop, and the
comparison of plain and denoised Monte Carlo by the time each needs to reach a target error.

Training pairs. For every random case (phantom + beam) the engine runs n_low histories (the
network's input: the dose and its batch standard error) and, with an independent seed, n_high
histories (the target). The maps and the density stay on the device.

Error. The error of a dose D against a reference R is the mean of |D - R| / max(R) over the
voxels with R >= 0.1 max(R) (the 10% isodose), the agreement statistic of the paper's Sec. 3.1.

Time to a target error. Plain: the engine runs N histories for N on a geometric grid until the
dose reaches the target; the time is the wall time of ocmc_run + ocmc_get_dose for that N.
Denoised: the same with ocmc_denoise (network inference with the plain-MC fallback) in place of
ocmc_get_dose. Both are wall times through the public calls, synchronised on both sides.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import ocmc


def dose_error(dose: torch.Tensor, ref: torch.Tensor, iso: float = 0.1) -> float:
    """Mean |dose - ref| / max(ref) over the voxels with ref >= iso * max(ref)."""
    m = ref.max()
    sel = ref >= iso * m
    return float(((dose - ref).abs()[sel]).mean() / m)


def _dose(engine, shape, device):
    d = torch.empty(shape, dtype=torch.float32, device=device)
    engine.dose(out=(d, None))
    return d


def _dose_sigma(engine, shape, device):
    d = torch.empty(shape, dtype=torch.float32, device=device)
    s = torch.empty_like(d)
    engine.dose(out=(d, s))
    return d, s


def make_pairs(cases, n_low, n_high, seed=1, device=0, engine=None, log=None):
    """Engine-generated (input, input sigma, density, target) on the device, one per case.
    Seeds: input 2 k + seed, target 2 k + seed + 1 for case k (independent histories)."""
    own = engine is None
    eng = ocmc.Engine(device) if own else engine
    dev = torch.device("cuda", device)
    out = []
    try:
        for k, (ph, beam) in enumerate(cases):
            eng.create_phantom(ph)
            eng.set_source(beam)
            eng.reset()
            eng.run(n_low, seed=2 * k + seed)
            low, low_sigma = _dose_sigma(eng, ph.density.shape, dev)
            eng.reset()
            eng.run(n_high, seed=2 * k + seed + 1)
            high = _dose(eng, ph.density.shape, dev)
            dens = torch.from_numpy(np.ascontiguousarray(ph.density)).to(dev)
            out.append((low, low_sigma, dens, high))
            if log:
                log(f"pair {k + 1}/{len(cases)}")
    finally:
        if own:
            eng.close()
    return out


def train(net: ocmc.UNet, pairs, steps: int, lr: float = 5e-4, lr_final: float = 2e-5, warmup: int = 300,
          seed: int = 0, log_every: int = 0, log=print, flips: bool = False):
    """Adam on one pair per step, pairs drawn in shuffled epochs; the learning rate rises
    linearly over `warmup` steps to lr, then decays to lr_final along a cosine (a high rate
    from the start can silence every ReLU of a layer, after which the network only returns its
    input). With flips, each step mirrors its pair (all four grids alike) along a random
    subset of the three axes: a mirrored case is another valid geometry, so the network sees
    eight times as many distinct cases. Returns the per-step losses."""
    rng = np.random.default_rng(seed)
    order, losses = [], []
    for t in range(steps):
        if not order:
            order = list(rng.permutation(len(pairs)))
        low, low_sigma, dens, high = pairs[order.pop()]
        if flips:
            bits = int(rng.integers(0, 8))
            dims = [d for d in range(3) if bits >> d & 1]
            if dims:
                low, low_sigma, dens, high = (torch.flip(x, dims).contiguous() for x in (low, low_sigma, dens, high))
        if t < warmup:
            a = lr * (t + 1) / warmup
        else:
            x = (t - warmup) / max(steps - warmup - 1, 1)
            a = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * x))
        losses.append(net.train_step(low, dens, high, a, sigma=low_sigma))
        if log_every and (t + 1) % log_every == 0:
            log(f"step {t + 1}/{steps} loss {np.mean(losses[-log_every:]):.4e} lr {a:.2e}")
    return losses


def _sync_time(fn):
    torch.cuda.synchronize()
    t = time.perf_counter()
    fn()
    torch.cuda.synchronize()
    return time.perf_counter() - t


def time_to_error(engine, net, ph, beam, ref, target=0.01, n0=10_000, factor=math.sqrt(2.0),
                  n_max=2_000_000_000, k_sigma=4.0, seed=12345, device=0):
    """Plain and denoised Monte Carlo on one case: for N = n0 * factor^j, the error of each
    against `ref` and the wall time. Returns a dict with, per method, the first N that
    reaches `target`, its time, and the whole curve."""
    dev = torch.device("cuda", device)
    engine.create_phantom(ph)
    engine.set_source(beam)
    shape = ph.density.shape
    out = torch.empty(shape, dtype=torch.float32, device=dev)
    flag = torch.empty_like(out)
    plain = torch.empty_like(out)
    res = {"plain": None, "denoised": None, "curve": []}
    n = float(n0)
    while n <= n_max and (res["plain"] is None or res["denoised"] is None):
        N = int(round(n))

        def run():
            engine.reset()
            engine.run(N, seed=seed)

        t_mc = _sync_time(run)
        t_plain = _sync_time(lambda: engine.dose(out=(plain, None)))
        t_dn = _sync_time(lambda: ocmc.denoise(engine, net, k_sigma, out, flag))
        e_plain, e_dn = dose_error(plain, ref), dose_error(out, ref)
        sel = ref >= 0.1 * ref.max()
        row = {"n": N, "err_plain": e_plain, "err_denoised": e_dn, "t_mc": t_mc, "t_dose": t_plain,
               "t_denoise": t_dn, "flagged": float(flag[sel].mean())}
        ocmc.denoise(engine, net, 3.0e38, out, flag)          # the network alone, for the record
        row["err_network"] = dose_error(out, ref)
        res["curve"].append(row)
        if res["plain"] is None and e_plain <= target:
            res["plain"] = {"n": N, "time_s": t_mc + t_plain, "err": e_plain}
        if res["denoised"] is None and e_dn <= target:
            res["denoised"] = {"n": N, "time_s": t_mc + t_dn, "err": e_dn}
        n *= factor
    return res


# ---- layer shapes and work ----------------------------------------------------------------
CHANNELS = (16, 32, 64, 128)


def layer_shapes(shape):
    """(kind, cin, cout, output voxels) of every layer, in the network's order: per encoder
    level two 3x3x3 convolutions and a 2x2x2 stride-2 convolution, then per decoder level a
    transposed 2x2x2 convolution and two 3x3x3 convolutions (the first over the concatenated
    skip). The input has 16 channels (dose, density, zero padding)."""
    nz, ny, nx = shape
    vox = [(nz >> l) * (ny >> l) * (nx >> l) for l in range(len(CHANNELS))]
    out, cin = [], 16
    for l, c in enumerate(CHANNELS):
        out += [("conv3", cin, c, vox[l]), ("conv3", c, c, vox[l])]
        if l < len(CHANNELS) - 1:
            out.append(("down", c, CHANNELS[l + 1], vox[l + 1]))
            cin = CHANNELS[l + 1]
    for l in range(len(CHANNELS) - 2, -1, -1):
        c = CHANNELS[l]
        out += [("up", CHANNELS[l + 1], c, vox[l]), ("conv3", 2 * c, c, vox[l]), ("conv3", c, c, vox[l])]
    return out


def forward_flops(shape):
    """Multiply-add work of one forward pass (2 FLOP per MAC): 27 taps for 3x3x3
    convolutions, 8 for stride-2 convolutions per coarse voxel, 1 per fine voxel for the
    transposed convolution, plus the 16-weight head."""
    taps = {"conv3": 27, "down": 8, "up": 1}
    f = sum(2 * taps[k] * ci * co * v for k, ci, co, v in layer_shapes(shape))
    return f + 2 * 16 * shape[0] * shape[1] * shape[2]


# ---- the full study -------------------------------------------------------------------------
def _cases(seeds, shape, voxel, workers=8):
    import ocmc_inputs as inputs
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(workers) as ex:
        return list(ex.map(lambda s: inputs.denoiser_case(s, shape, voxel), seeds))


def judge(engine, ph, beam, n_ref, seed, shape, device=0, max_err=None, n_cap=2 * 10**11):
    """The reference dose of one case: plain MC at n_ref histories; with max_err, more
    histories (independent seeds, accumulated in the same tally) until the judge's own error
    estimate (mean sigma / max over the 10 % isodose, times sqrt(2/pi)) is at most max_err, or
    n_cap. Returns (reference dose, its error estimate, histories)."""
    dev = torch.device("cuda", device)
    engine.create_phantom(ph)
    engine.set_source(beam)
    engine.reset()
    done, k = 0, 0
    want = int(n_ref)
    while True:
        engine.run(want - done, seed=seed + 7919 * k)
        done, k = want, k + 1
        ref = torch.empty(shape, dtype=torch.float32, device=dev)
        sig = torch.empty_like(ref)
        engine.dose(out=(ref, sig))
        m = ref.max()
        sel = ref >= 0.1 * m
        err = float(sig[sel].mean() / m * math.sqrt(2 / math.pi))
        if max_err is None or err <= max_err or done >= n_cap:
            return ref, err, done
        want = min(n_cap, int(math.ceil(done * (err / max_err) ** 2 * 1.1)))


def train_on_cases(eng, net, cases, lows, n_high, steps, lr, warmup, seed, flips, shape, device, log, rep):
    """Training data from the engine (several input noise levels per case, one target of
    n_high histories), then Adam on the network; timings and losses go into rep."""
    dev = torch.device("cuda", device)
    t0 = time.perf_counter()
    pairs = []
    for k, (ph, beam) in enumerate(cases):
        eng.create_phantom(ph)
        eng.set_source(beam)
        dens = torch.from_numpy(np.ascontiguousarray(ph.density)).to(dev)
        eng.reset()
        eng.run(n_high, seed=7 * k + seed)
        high = _dose(eng, shape, dev)
        for j, n in enumerate(lows):
            eng.reset()
            eng.run(n, seed=7 * k + seed + 1 + j)
            low, low_sigma = _dose_sigma(eng, shape, dev)
            pairs.append((low, low_sigma, dens, high))
        if (k + 1) % 25 == 0:
            log(f"pairs: case {k + 1}/{len(cases)} ({time.perf_counter() - t0:.0f} s)")
    torch.cuda.synchronize()
    rep["t_pairs_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = train(net, pairs, steps, lr=lr, warmup=warmup, seed=seed, log_every=max(steps // 10, 1), log=log,
                   flips=flips)
    torch.cuda.synchronize()
    rep["t_train_s"] = time.perf_counter() - t0
    rep["loss_first_100"] = float(np.mean(losses[:100]))
    rep["loss_last_100"] = float(np.mean(losses[-100:]))


def run_study(n_train=200, n_eval=8, lows=(10**5, 10**6, 10**7), n_high=10**9,
              n_ref=(10**10, 10**9), steps=12000, lr=5e-4, shape=(128, 128, 128),
              voxel=(0.25, 0.25, 0.25), target=0.01, k_sigma=4.0, device=0, seed=1, log=print,
              weights_out=None, warmup=300, flips=True, weights_in=None, judge_max_err=None):
    """Generate training pairs on random cases, train the network, then on held-out cases
    compare plain and denoised Monte Carlo by the wall time each needs to reach `target`
    against a reference of n_ref histories (photon, electron beams; with judge_max_err, more
    until the reference's own error estimate is at most that). With weights_in the training is
    skipped and the given weights are evaluated. Returns a report dict."""
    t0 = time.perf_counter()
    train_cases = [] if weights_in is not None else _cases([100_000 + seed * 10_000 + k for k in range(n_train)],
                                                            shape, voxel)
    eval_cases = _cases([900_000 + seed * 10_000 + k for k in range(n_eval)], shape, voxel)
    t_cases = time.perf_counter() - t0
    eng = ocmc.Engine(device)
    net = ocmc.UNet(shape, device=device, seed=seed)
    rep = {"shape": list(shape), "voxel_cm": list(voxel), "n_train": n_train, "n_eval": n_eval,
           "lows": list(lows), "n_high": n_high, "n_ref": list(n_ref), "steps": steps, "flips": flips, "target": target,
           "k_sigma": k_sigma, "t_case_generation_s": t_cases, "judge_max_err": judge_max_err,
           "weights_in": weights_in}
    try:
        if weights_in is not None:
            net.set_params(np.load(weights_in))
        else:
            train_on_cases(eng, net, train_cases, lows, n_high, steps, lr, warmup, seed, flips, shape, device, log,
                           rep)
            if weights_out:
                np.save(weights_out, net.params())
        # evaluation on held-out cases
        rows = []
        for k, (ph, beam) in enumerate(eval_cases):
            t1 = time.perf_counter()
            ref, ref_err, nr = judge(eng, ph, beam, n_ref[0] if beam.particle == 0 else n_ref[1], 99_991 + k,
                                     shape, device=device, max_err=judge_max_err)
            t_ref = time.perf_counter() - t1
            r = time_to_error(eng, net, ph, beam, ref, target=target, k_sigma=k_sigma, seed=31 + k,
                              device=device)
            row = {"particle": "photon" if beam.particle == 0 else "electron",
                   "energy_MeV": float(beam.edges[0]) if beam.particle == 1 else "6MV",
                   "field_cm": [round(v, 2) for v in beam.field], "n_ref": nr, "t_ref_s": t_ref,
                   "ref_err_est": ref_err, "plain": r["plain"], "denoised": r["denoised"],
                   "curve": r["curve"]}
            if r["plain"] and r["denoised"]:
                row["speedup"] = r["plain"]["time_s"] / r["denoised"]["time_s"]
            rows.append(row)
            log(f"eval {k}: {row['particle']} field {row['field_cm']} judge {nr:.2e} ({100 * ref_err:.3f} %) "
                f"plain {r['plain']} denoised {r['denoised']}")
        rep["cases"] = rows
        tp = [r["plain"]["time_s"] for r in rows if r["plain"]]
        td = [r["denoised"]["time_s"] for r in rows if r["denoised"]]
        rep["median_time_plain_s"] = float(np.median(tp)) if tp else None
        rep["median_time_denoised_s"] = float(np.median(td)) if td else None
        sp = [r["speedup"] for r in rows if "speedup" in r]
        rep["median_speedup"] = float(np.median(sp)) if sp else None
    finally:
        net.close()
        eng.close()
    return rep


def time_training(shape=(128, 128, 128), steps=5, warmup=2, seed=1):
    """Mean CUDA-event time (ms) of one training step (forward, loss, backward, Adam) on seeded
    synthetic inputs of the given grid; the study's pairs are not needed for timing."""
    import torch
    from . import ocmc
    rng = np.random.default_rng(seed)
    dose = torch.from_numpy(rng.random(shape, dtype=np.float32)).cuda()
    sig = torch.from_numpy((0.1 * rng.random(shape)).astype(np.float32)).cuda()
    dens = torch.from_numpy(rng.uniform(0.3, 1.8, shape).astype(np.float32)).cuda()
    net = ocmc.UNet(shape, seed=seed)
    ms = []
    for k in range(warmup + steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        net.train_step(dose, dens, dose, 1e-4, sigma=sig)
        e1.record()
        e1.synchronize()
        if k >= warmup:
            ms.append(e0.elapsed_time(e1))
    net.close()
    return float(np.mean(ms)) if ms else 0.0


def main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser(description="train the dose denoiser on engine-made pairs and compare "
                                             "plain and denoised Monte Carlo by time to a target error")
    ap.add_argument("--train", type=int, default=200)
    ap.add_argument("--eval", type=int, default=8)
    ap.add_argument("--steps", type=int, default=12000)
    ap.add_argument("--no-flips", action="store_true", help="train without mirrored copies of the pairs")
    ap.add_argument("--n-high", type=float, default=1e9, help="histories of each training target")
    ap.add_argument("--n-ref-photon", type=float, default=1e10, help="histories of a photon case's judge")
    ap.add_argument("--n-ref-electron", type=float, default=1e9, help="histories of an electron case's judge")
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--voxel", type=float, default=0.25)
    ap.add_argument("--lr", type=float, default=5e-4)
    ap.add_argument("--weights-out", default=None)
    ap.add_argument("--weights-in", default=None, help="evaluate these weights (.npy) instead of training")
    ap.add_argument("--judge-max-err", type=float, default=None,
                    help="raise a judge's histories until its own error estimate is at most this (e.g. 0.001)")
    ap.add_argument("--report", default=None)
    ap.add_argument("--time-steps", type=int, default=0,
                    help="only time this many training steps on synthetic input (after two warm-up steps)")
    a = ap.parse_args(argv)
    g = a.grid
    if a.time_steps:
        print(json.dumps({"grid": g, "train_step_ms": time_training((g, g, g), steps=a.time_steps)}))
        return
    rep = run_study(n_train=a.train, n_eval=a.eval, n_high=int(a.n_high), steps=a.steps, lr=a.lr, flips=not a.no_flips,
                    n_ref=(int(a.n_ref_photon), int(a.n_ref_electron)), weights_in=a.weights_in,
                    judge_max_err=a.judge_max_err,
                    shape=(g, g, g), voxel=(a.voxel,) * 3, weights_out=a.weights_out,
                    log=lambda m: print(m, flush=True))
    s = json.dumps(rep)
    if a.report:
        with open(a.report, "w") as f:
            f.write(s)
    print(json.dumps({k: v for k, v in rep.items() if k != "cases"}))


if __name__ == "__main__":
    main()
