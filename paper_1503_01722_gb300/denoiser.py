"""Learned dose denoiser: training data made by the engine, the training loop, and the
comparison of plain and denoised Monte Carlo by the time each needs to reach a target error.

Training pairs. For every random case (phantom + beam) the engine runs n_low histories (the
network's input) and, with an independent seed, n_high histories (the target). Both dose maps
and the density stay on the device.

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


def make_pairs(cases, n_low, n_high, seed=1, device=0, engine=None, log=None):
    """Engine-generated (input, density, target) triples on the device, one per case.
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
            low = _dose(eng, ph.density.shape, dev)
            eng.reset()
            eng.run(n_high, seed=2 * k + seed + 1)
            high = _dose(eng, ph.density.shape, dev)
            dens = torch.from_numpy(np.ascontiguousarray(ph.density)).to(dev)
            out.append((low, dens, high))
            if log:
                log(f"pair {k + 1}/{len(cases)}")
    finally:
        if own:
            eng.close()
    return out


def train(net: ocmc.UNet, pairs, steps: int, lr: float = 1e-3, lr_final: float = 1e-4, seed: int = 0,
          log_every: int = 0, log=print):
    """Adam on one pair per step, pairs drawn in shuffled epochs; cosine learning-rate decay
    from lr to lr_final. Returns the per-step losses."""
    rng = np.random.default_rng(seed)
    order, losses = [], []
    for t in range(steps):
        if not order:
            order = list(rng.permutation(len(pairs)))
        low, dens, high = pairs[order.pop()]
        a = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * t / max(steps - 1, 1)))
        losses.append(net.train_step(low, dens, high, a))
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
        row = {"n": N, "err_plain": e_plain, "err_denoised": e_dn, "t_mc": t_mc, "t_dose": t_plain,
               "t_denoise": t_dn, "flagged": float(flag.mean())}
        res["curve"].append(row)
        if res["plain"] is None and e_plain <= target:
            res["plain"] = {"n": N, "time_s": t_mc + t_plain, "err": e_plain}
        if res["denoised"] is None and e_dn <= target:
            res["denoised"] = {"n": N, "time_s": t_mc + t_dn, "err": e_dn}
        n *= factor
    return res
