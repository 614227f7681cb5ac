"""Learned proposal vs plain walk on the same GPU and the same walkers.

1. Data: a plain walk at length L with the log armed (one record per walker and chunk).
2. Training: `train_steps` AdamW steps of batch `batch` on those records.
3. Comparison: walks of `walkers` walkers from the same seed: plain, in the learned
   mode, and (restart_arm) in the restart-only learned mode (the plain kernels, the
   network picking restart states only), each advanced in segments of `segment` steps up to `steps`, or until
   `seconds` of wall time have passed (whichever comes first).  After every segment the
   best ISL so far is read back, so each threshold F >= f gets the wall time and step
   count of the segment in which some walker first reached it (None when the run ends
   first: a time censored at the run's length).
Every step of every phase runs in the library's kernels.
"""
from __future__ import annotations

import time

import torch

from . import Search
from . import learned as lrn
from ._native import LABS_FLAG_LEARNED, LABS_FLAG_LEARNED_RESTARTS

THRESHOLDS = (7.0, 7.5, 8.0, 8.25, 8.5)


def train_flop_per_sample(n: int) -> int:
    """Multiply-add FLOPs of one training sample's products over its n positions: the
    forward convolutions (3 real input channels padded to 16, then 64 -> 64, 7 taps)
    and the 64 -> 64 MLP; backward, the data gradients of conv3, conv2 and the MLP and
    the weight gradients of all four (each as many FLOPs as its forward product); the
    heads and the loss are left out (linear in n)."""
    conv1, conv, mlp = 2 * n * 64 * 16 * 7, 2 * n * 64 * 64 * 7, 2 * n * 64 * 64
    forward = conv1 + 2 * conv + mlp
    backward = (2 * conv + mlp) + (conv1 + 2 * conv + mlp)
    return forward + backward


def _run(L, walkers, seed, steps, segment, params=None, tau=0, candidates=4, chunk=1024, device=None,
         seconds=None, restarts_only=False):
    flags = 0 if params is None else (LABS_FLAG_LEARNED_RESTARTS if restarts_only else LABS_FLAG_LEARNED)
    s = Search(L, walkers, seed, device=device, chunk_steps=chunk, flags=flags)
    if params is not None:
        s.learned(params, tau=tau, candidates=candidates)
    hits = {f: None for f in THRESHOLDS}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done = 0
    curve = []
    while done < steps and (seconds is None or time.perf_counter() - t0 < seconds):
        k = min(segment, steps - done)
        s.walk(k)
        done += k
        b = s.best()
        el = time.perf_counter() - t0
        curve.append((done, el, b["isl"]))
        for f in THRESHOLDS:
            if hits[f] is None and 2 * f * b["isl"] <= L * L:
                hits[f] = {"steps": done, "seconds": el}
    el = time.perf_counter() - t0
    st = s.stats()
    b = s.best()
    s.close()
    return {"seconds": el, "steps": done, "flips_per_s": st["flip_evaluations"] / el, "best_isl": b["isl"],
            "best_F": b["F"], "best_hex": b["hex"], "restarts": st["restarts"],
            "time_to_F": {str(f): hits[f] for f in THRESHOLDS}, "curve": curve}


def run(L=255, walkers=32768, steps=20000, segment=1024, seed=11, train_walkers=16384, train_chunks=32,
        train_chunk_steps=256, train_steps=20000, batch=4096, lr=1e-3, tau=None, candidates=4, device=None,
        seconds=None, restart_arm=False, full_arm=True):
    n = (L + 1) // 2
    tau = 8 * L if tau is None else tau
    t0 = time.perf_counter()
    recs = lrn.collect(L, train_walkers, train_chunks, seed + 1, chunk_steps=train_chunk_steps, device=device)
    t_collect = time.perf_counter() - t0
    tr = lrn.Trainer(L, batch=batch, seed=seed + 2, device=device, lr=lr)
    t0 = time.perf_counter()
    losses = tr.fit(recs, steps=train_steps, seed=seed + 3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    plain = _run(L, walkers, seed, steps, segment, device=device, seconds=seconds)
    learned = (_run(L, walkers, seed, steps, segment, params=tr.params, tau=tau, candidates=candidates,
                    device=device, seconds=seconds) if full_arm else None)
    restarts = (_run(L, walkers, seed, steps, segment, params=tr.params, candidates=candidates, device=device,
                     seconds=seconds, restarts_only=True) if restart_arm else None)
    return {"L": L, "n": n, "walkers": walkers, "steps": steps, "seed": seed,
            "train": {"records": int(recs.shape[0]), "steps": train_steps, "batch": batch, "lr": lr,
                      "collect_s": t_collect, "train_s": t_train,
                      "samples_per_s": train_steps * batch / t_train,
                      "tflops": train_steps * batch * train_flop_per_sample(n) / t_train / 1e12,
                      "loss_first": sum(losses[:50]) / min(50, len(losses)),
                      "loss_last": sum(losses[-50:]) / min(50, len(losses))},
            "tau": tau, "candidates": candidates, "seconds_cap": seconds, "plain": plain, "learned": learned,
            "learned_restarts": restarts}
