"""Autotuner and CUDA-graph runner for batched multi-view rendering.

The batched path renders every view of every scene in one launch sequence:
one preprocess launch per scene, one sort and one blend launch for the whole
batch.  The persistent blends keep one resident wave of CTAs pulling tiles, in
longest-first order (views of uneven size share the GPU without tail effects)
or in tile order (neighbouring tiles' records stay in L2, and no CTA waits to be
launched).  The sequence is allocation
and synchronisation free, so it can be captured once in a CUDA graph and
replayed every frame.

The tuner times candidate plans on the caller's own batch and caches the
fastest under a key of (GPU name, view sizes, scene sizes):
  - blend schedule: one CTA per tile, or a persistent grid in longest-first
    or in tile order, whose CTAs claim 1 or 4 tiles of the work order per
    atomic (the batch-per-block knob);
  - sort: tile buckets, or the global LSD radix sort with the minimal key
    width (tile-id bits + 32) or the full 64 bits;
  - tile edge 8 / 16 / 32 only when ``allow_tile_change`` is set, because the
    tile size changes which splats a pixel sees (pixels also see a splat
    beyond its 3-sigma ellipse inside the tiles it touches).
All other choices give bit-identical images.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os
from typing import Dict, List, Optional, Sequence

import torch

from .render import Rasterizer, SceneTensors

CACHE_PATH = os.environ.get("VRS_AUTOTUNE_CACHE",
                            os.path.join(os.path.expanduser("~"), ".cache", "vrs_autotune.json"))


def _key(scenes: Sequence[SceneTensors], views: Sequence, allow_tile_change: bool) -> str:
    dev = torch.cuda.get_device_name()
    sig = json.dumps(["v3", dev, [(v.width, v.height, v.scene) for v in views],
                      [(s.n, s.sh_degree) for s in scenes], allow_tile_change])
    return hashlib.sha1(sig.encode()).hexdigest()


class CallableGraph:
    """Captures a launch sequence (a callable that only enqueues work on the current stream,
    allocates nothing and does not synchronise, e.g. a training step's forward_async and
    backward_params) in a CUDA graph and replays it."""

    def __init__(self, fn, warmup: int = 2):
        self.fn = fn
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                fn()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            fn()
        torch.cuda.synchronize()

    def replay(self):
        self.graph.replay()


class GraphRunner:
    """Captures Rasterizer.forward_async in a CUDA graph and replays it."""

    def __init__(self, ras: Rasterizer, warmup: int = 2):
        self.ras = ras
        ras.forward()                       # sizes the instance list outside the capture
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                ras.forward_async()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            ras.forward_async()
        torch.cuda.synchronize()

    def replay(self):
        self.graph.replay()


def time_ms(fn, iters: int = 20, warmup: int = 3) -> float:
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(iters):
        fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / iters


def candidates(allow_tile_change: bool, tile: int = 16) -> List[Dict]:
    tiles = (8, 16, 32) if allow_tile_change else (tile,)
    out = []
    for t, p, s in itertools.product(tiles, (0, 1, 2), (0, 1)):
        for pull in ((1, 4) if p else (1,)):
            for kb in ((0, 64) if s == 1 and pull == 1 else (0,)):
                out.append(dict(tile=t, persistent=p, sort=s, tiles_per_pull=pull, key_bits=kb))
    return out


def tune(scenes: Sequence[SceneTensors], views: Sequence, allow_tile_change: bool = False,
         tile: int = 16, iters: int = 10, use_cache: bool = True, verbose: bool = False,
         timings_out: Optional[list] = None) -> Dict:
    """Returns the fastest plan options {tile, persistent, sort, tiles_per_pull, key_bits} for
    this batch (cached); timings_out, when given, receives every (ms, options) measured."""
    key = _key(scenes, views, allow_tile_change)
    cache = {}
    if use_cache and os.path.exists(CACHE_PATH):
        try:
            with open(CACHE_PATH) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        return cache[key]["best"]
    results = []
    for c in candidates(allow_tile_change, tile):
        ras = Rasterizer(scenes, views, **c)
        runner = GraphRunner(ras)
        ms = time_ms(runner.replay, iters=iters)
        results.append((ms, c))
        if verbose:
            print(f"autotune {c}: {ms:.4f} ms")
        del runner, ras
    results.sort(key=lambda x: x[0])
    best = results[0][1]
    if timings_out is not None:
        timings_out.extend(results)
    if use_cache:
        cache[key] = {"best": best, "timings": [(ms, c) for ms, c in results]}
        try:
            os.makedirs(os.path.dirname(CACHE_PATH), exist_ok=True)
            with open(CACHE_PATH, "w") as f:
                json.dump(cache, f)
        except OSError:
            pass
    return best


class ViewsGraphRunner:
    """One CUDA graph replaying several rasterizers' forward passes one after another
    (the per-view baseline of a batch, captured the same way as the batched frame)."""

    def __init__(self, rasterizers: Sequence[Rasterizer], warmup: int = 2):
        self.rasterizers = list(rasterizers)
        for r in self.rasterizers:
            r.forward()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                for r in self.rasterizers:
                    r.forward_async()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            for r in self.rasterizers:
                r.forward_async()
        torch.cuda.synchronize()

    def replay(self):
        self.graph.replay()
