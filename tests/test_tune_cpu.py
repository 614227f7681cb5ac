"""Host logic of the launch-shape autotuner (paper_2011_00068_gb300/tune.py) on CPU: a
fake Search whose walk advances a fake stream clock by a per-shape cost, and fake CUDA
events that read that clock, stand in for the GPU.  Checked: every candidate shape is
timed once, the fastest is returned and cached under a key of the GPU name, lengths,
walker counts, table size and flags; a second call is served from the cache without
timing; refresh times again."""
from __future__ import annotations

import json

import pytest
import torch

import paper_2011_00068_gb300 as labs
from paper_2011_00068_gb300 import tune


class FakeStream:
    def __init__(self):
        self.t = 0.0


class FakeEvent:
    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream):
        self.t = stream.t

    def elapsed_time(self, other):
        return other.t - self.t


def make_search(cost, made):
    class FakeSearch:
        def __init__(self, L, walkers, seed, *, device=None, tabu_log2=16, warps_per_cta=0, chunk_steps=0,
                     flags=0):
            self.shape = (warps_per_cta, chunk_steps)
            self.stream = FakeStream()
            made.append((L, walkers, tabu_log2, self.shape, flags))

        def walk(self, steps):
            self.stream.t += cost(*self.shape) * steps

        def sync(self):
            pass

        def close(self):
            pass

    return FakeSearch


@pytest.fixture
def fake_gpu(tmp_path, monkeypatch):
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "tune_cache.json"))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda dev=None: "FakeGPU")
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    made = []
    # (4 warps, 1024 steps) is the fastest shape; the rest cost more per step
    cost = lambda wpc, chunk: 1.0 if (wpc, chunk) == (4, 1024) else 2.0 + wpc / 8 + chunk / 4096
    monkeypatch.setattr(labs, "Search", make_search(cost, made))
    return made


def test_tune_picks_the_fastest_shape_and_caches_it(fake_gpu):
    made = fake_gpu
    best = tune.tune(201, 16384, steps=100)
    assert (best["warps_per_cta"], best["chunk_steps"]) == (4, 1024)
    shapes = [m[3] for m in made]
    assert sorted(shapes) == sorted((w, c) for w in tune.WARPS for c in tune.CHUNKS)
    assert all(m[:3] == (201, 16384, 16) for m in made)
    assert best["ms"] == pytest.approx(100.0)
    assert len(best["all"]) == len(tune.WARPS) * len(tune.CHUNKS)
    with open(tune.CACHE) as f:
        cache = json.load(f)
    assert list(cache) == ["FakeGPU|201|16384|16"]
    # served from the cache: no Search is made
    n = len(made)
    again = tune.tune(201, 16384, steps=100)
    assert len(made) == n and (again["warps_per_cta"], again["chunk_steps"]) == (4, 1024)
    # refresh times every shape again
    tune.tune(201, 16384, steps=100, refresh=True)
    assert len(made) == 2 * n


def test_tune_keys_separate_mixes_tables_and_flags(fake_gpu):
    made = fake_gpu
    tune.tune([201, 203], [2048, 2048], steps=10)
    assert all(m[0] == [201, 203] and m[1] == [2048, 2048] for m in made)
    tune.tune(201, 16384, steps=10, tabu_log2=12)
    tune.tune(201, 16384, steps=10, flags=64)
    assert {m[4] for m in made} == {0, 64}
    with open(tune.CACHE) as f:
        keys = sorted(json.load(f))
    assert keys == ["FakeGPU|201,203|2048,2048|16", "FakeGPU|201|16384|12", "FakeGPU|201|16384|16/flags64"]
