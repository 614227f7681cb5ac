"""Learned proposal vs plain walk on the same GPU and the same walkers.

1. Data: a plain walk at length L with the log armed (one record per walker and chunk).
2. Training: `train_steps` AdamW steps of batch `batch` on those records.
3. Comparison: two walks of `walkers` walkers from the same seed, one plain and one in
   the learned mode, each advanced in segments of `segment` steps up to `steps`.  After
   every segment the best ISL so far is read back, so each threshold F >= f gets the
   wall time and step count of the segment in which some walker first reached it
   (None when the run ends first: a censored time).
Every step of every phase runs in the library's kernels.
"""
from __future__ import annotations

import time

import torch

from . import Search
from . import learned as lrn
from ._native import LABS_FLAG_LEARNED

THRESHOLDS = (7.0, 7.5, 8.0, 8.5)


def _run(L, walkers, seed, steps, segment, params=None, tau=0, candidates=4, chunk=1024, device=None):
    flags = LABS_FLAG_LEARNED if params is not None else 0
    s = Search(L, walkers, seed, device=device, chunk_steps=chunk, flags=flags)
    if params is not None:
        s.learned(params, tau=tau, candidates=candidates)
    hits = {f: None for f in THRESHOLDS}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done = 0
    curve = []
    while done < steps:
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
    return {"seconds": el, "steps": steps, "flips_per_s": st["flip_evaluations"] / el, "best_isl": b["isl"],
            "best_F": b["F"], "best_hex": b["hex"], "restarts": st["restarts"],
            "time_to_F": {str(f): hits[f] for f in THRESHOLDS}, "curve": curve}


def run(L=255, walkers=32768, steps=20000, segment=1024, seed=11, train_walkers=16384, train_chunks=32,
        train_chunk_steps=256, train_steps=20000, batch=4096, lr=1e-3, tau=None, candidates=4, device=None):
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
    plain = _run(L, walkers, seed, steps, segment, device=device)
    learned = _run(L, walkers, seed, steps, segment, params=tr.params, tau=tau, candidates=candidates, device=device)
    return {"L": L, "n": n, "walkers": walkers, "steps": steps, "seed": seed,
            "train": {"records": int(recs.shape[0]), "steps": train_steps, "batch": batch, "lr": lr,
                      "collect_s": t_collect, "train_s": t_train,
                      "samples_per_s": train_steps * batch / t_train,
                      "loss_first": sum(losses[:50]) / min(50, len(losses)),
                      "loss_last": sum(losses[-50:]) / min(50, len(losses))},
            "tau": tau, "candidates": candidates, "plain": plain, "learned": learned}
