"""Seeded synthetic inputs shaped like the paper's workloads.

This module is the one piece shared by the CUDA engine's tests/bench and the
CPU oracle's tests: it only draws random numbers and lays out launch
descriptions (extents, machine sizes, chain draws, distribution kinds).  It
holds none of the mapping arithmetic: a random transform chain is handed out
as a list of raw 64-bit draws, and each side builds the chain from the draws
with its own copy of the canonical op alphabet.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), seeded per query with
0x2507170870000000 + query_index.
"""
from __future__ import annotations

import math

MASK = (1 << 64) - 1
SEED_BASE = 0x2507170870000000


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & MASK

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform in [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (modulo draw; bias is irrelevant here)."""
        return lo + self.next() % (hi - lo + 1)

    def choice(self, seq):
        return seq[self.next() % len(seq)]


def rng(query_index: int) -> SplitMix64:
    return SplitMix64(SEED_BASE + query_index)


# ----------------------------------------------------------------- launches
#
# A launch is a dict:
#   L        task-space extents (tuple, rank 1..4)
#   machine  (nodes, procs_per_node)
#   chain    explicit chain tuples, or None when the chain comes from draws
#   draws    list of 64-bit draws for a random canonical chain (or [])
#   dist     ("block",) / ("cyclic",) / ("block_cyclic", b) / ("hier",) /
#            ("linear_cyclic",)
#   face     per-dimension face bytes of the nearest-neighbour stencil

DIST_KINDS = ("block", "cyclic", "block_cyclic", "hier", "linear_cyclic")


def plain_config():
    """64x64 tiles of 256x256 float64 on 2 nodes x 4 GPUs, block mapping via
    decompose, 5-point stencil (one 256-element edge of float64 per face)."""
    return {
        "name": "plain-64x64-on-2x4",
        "L": (64, 64),
        "machine": (2, 4),
        "chain": [("merge", 0, 1), ("decompose", 0, (64, 64))],
        "draws": [],
        "dist": ("block",),
        "face": (256 * 8, 256 * 8),
    }


def large_config(variant: str, query_index: int = 1):
    """1024x1024x512 points on 64 nodes x 8 procs, a seeded random
    split/merge/swap chain of depth 4, 7-point stencil with 8-byte elements."""
    r = rng(query_index)
    draws = [r.next() for _ in range(4)]
    dist = {"block": ("block",), "cyclic": ("cyclic",),
            "block_cyclic": ("block_cyclic", 4)}[variant]
    return {
        "name": f"large-1024x1024x512-on-64x8-{variant}",
        "L": (1024, 1024, 512),
        "machine": (64, 8),
        "chain": None,
        "draws": draws,
        "dist": dist,
        "face": (8, 8, 8),
    }


def scaled_launch(L, machine, variant, query_index, depth=4):
    """Same recipe as large_config at other sizes (for parity tests)."""
    r = rng(query_index)
    draws = [r.next() for _ in range(depth)]
    dist = {"block": ("block",), "cyclic": ("cyclic",), "block_cyclic": ("block_cyclic", 4),
            "hier": ("hier",), "linear_cyclic": ("linear_cyclic",)}[variant]
    return {"name": f"scaled-{variant}-{query_index}", "L": tuple(L), "machine": tuple(machine),
            "chain": None, "draws": draws, "dist": dist, "face": tuple([8] * len(L))}


def _split_extents(r: SplitMix64, total: int, rank: int):
    """Extents of a rank-`rank` box with about `total` points: random
    log-weights, each extent at least 1."""
    if rank == 1:
        return (max(1, total),)
    w = [r.uniform() + 0.05 for _ in range(rank)]
    s = sum(w)
    logt = math.log(total)
    ext = [max(1, int(round(math.exp(logt * wi / s)))) for wi in w]
    return tuple(ext)


def batched_queries(count: int = 10000, first_index: int = 1000, max_points: int = 1 << 24):
    """Uneven mapping queries: rank U{1..4}, point count log-uniform in
    [16, max_points], machine U{1..256} x U{1..8}, chain depth U{1..5},
    distribution uniform over the five kinds."""
    out = []
    lo, hi = math.log(16), math.log(max_points)
    for q in range(count):
        r = rng(first_index + q)
        rank = r.randint(1, 4)
        total = int(round(math.exp(lo + (hi - lo) * r.uniform())))
        L = _split_extents(r, total, rank)
        machine = (r.randint(1, 256), r.randint(1, 8))
        depth = r.randint(1, 5)
        draws = [r.next() for _ in range(depth)]
        kind = r.choice(DIST_KINDS)
        dist = ("block_cyclic", r.choice((2, 3, 4, 8))) if kind == "block_cyclic" else (kind,)
        face = tuple(r.choice((4, 8, 16, 64)) for _ in range(rank))
        out.append({"name": f"batched-{q}", "L": L, "machine": machine, "chain": None,
                    "draws": draws, "dist": dist, "face": face})
    return out


SEARCH_EXTENTS = (256, 1024, 4096)
SEARCH_PROCS = (512, 2520, 3600, 4096)


def search_queries(count: int, first_index: int = 5000):
    """3-D matmul decompose-search queries: tile-grid extents (M, N, K) from
    {256, 1024, 4096}, P from {512, 2520, 3600, 4096}, machine (P/8, 8),
    chains of depth <= 3, float32 512x512 tiles (1 MiB)."""
    out = []
    for q in range(count):
        r = rng(first_index + q)
        M, N, K = (r.choice(SEARCH_EXTENTS) for _ in range(3))
        P = r.choice(SEARCH_PROCS)
        out.append({"name": f"search-{q}", "MNK": (M, N, K), "machine": (P // 8, 8),
                    "max_depth": 3, "tile_bytes": 512 * 512 * 4})
    return out


def search_query_small(first_index: int = 7000, count: int = 8):
    """Smaller search queries (P <= 64) for full exhaustive parity tests."""
    out = []
    for q in range(count):
        r = rng(first_index + q)
        M, N, K = (r.choice((3, 8, 16, 64, 256)) for _ in range(3))
        n = r.choice((1, 2, 3, 4, 6, 8))
        g = r.choice((1, 2, 4, 8))
        out.append({"name": f"search-small-{q}", "MNK": (M, N, K), "machine": (n, g),
                    "max_depth": r.choice((1, 2, 3)), "tile_bytes": 512 * 512 * 4})
    return out


TRAIN_EXTENTS = (128, 256, 512, 1024, 2048, 4096, 8192)
TRAIN_PROCS = (256, 512, 720, 1024, 1440, 2048, 2520, 3600, 4096)


def search_training_queries(count: int, first_index: int = 20000):
    """Training queries for the learned cost model: a wider generator than
    the evaluation queries (extents from {128, ..., 8192}, P from a set of
    highly composite counts, seeds disjoint from the evaluation seeds)."""
    out = []
    for q in range(count):
        r = rng(first_index + q)
        M, N, K = (r.choice(TRAIN_EXTENTS) for _ in range(3))
        P = r.choice(TRAIN_PROCS)
        out.append({"name": f"train-{q}", "MNK": (M, N, K), "machine": (P // 8, 8),
                    "max_depth": 3, "tile_bytes": 512 * 512 * 4})
    return out


# ------------------------------------------------------ decompose vs greedy
#
# The stencil grid of the paper's decompose study (Sec. 6, "Performance Study
# of the Decompose Primitive"): six aspect ratios 1:1 .. 1:32, five task-space
# sizes per node (1e6 .. 4e8 points), 4 .. 128 GPUs in powers of two at four
# GPUs per node -- 180 configurations of a 2-D task space.

STUDY_RATIOS = (1, 2, 4, 8, 16, 32)
STUDY_AREAS = (10 ** 6, 10 ** 7, 10 ** 8, 2 * 10 ** 8, 4 * 10 ** 8)
STUDY_GPUS = (4, 8, 16, 32, 64, 128)
STUDY_GPUS_PER_NODE = 4


def stencil_study_configs():
    """(X, r X) task spaces with about area x nodes points on (G / 4, 4)."""
    out = []
    for r in STUDY_RATIOS:
        for area in STUDY_AREAS:
            for G in STUDY_GPUS:
                nodes = G // STUDY_GPUS_PER_NODE
                X = max(1, int(round(math.sqrt(area * nodes / r))))
                out.append({"name": f"stencil-1:{r}-{area}-{G}", "L": (X, r * X),
                            "machine": (nodes, STUDY_GPUS_PER_NODE), "ratio": r, "area": area, "gpus": G})
    return out


# ------------------------------------------------------ application shapes
#
# Launch shapes of the paper's applications (Sec. 6: Circuit, PENNANT,
# Stencil, Cannon, SUMMA, PUMMA, Johnson, COSMA), at 2^28-2^29 points on
# 64 nodes x 8 processors; the applications' own sizes are not given, so the
# piece counts are powers of two chosen to fill 1-2 GB of ids.

def application_shapes():
    n, g = 64, 8
    P = n * g
    return [
        # Circuit: a 1-D launch of pieces, c per processor, block over P
        {"name": "circuit-1d-block", "L": (P * (1 << 20),), "machine": (n, g), "chain": [],
         "dist": ("block",), "face": (8,)},
        # PENNANT-like: 1-D zone chunks dealt block-cyclically
        {"name": "pennant-1d-block-cyclic", "L": (P * (1 << 20),), "machine": (n, g), "chain": [],
         "dist": ("block_cyclic", 1024), "face": (8,)},
        # 2-D stencil: block mapping through decompose (Sec. 4)
        {"name": "stencil-2d-decompose", "L": (16384, 32768), "machine": (n, g),
         "chain": [("merge", 0, 1), ("decompose", 0, (16384, 32768))], "dist": ("block",), "face": (8, 8)},
        # Cannon: the hierarchical block / cyclic mapper of Appendix A.1
        {"name": "cannon-2d-hier", "L": (16384, 16384), "machine": (n, g), "chain": [],
         "dist": ("hier",), "face": (8, 8)},
        # SUMMA: block over an explicit 16 x 32 processor grid
        {"name": "summa-2d-block", "L": (16384, 16384), "machine": (n, g),
         "chain": [("merge", 0, 1), ("split", 0, 16)], "dist": ("block",), "face": (8, 8)},
        # PUMMA: block-cyclic over the same grid
        {"name": "pumma-2d-block-cyclic", "L": (16384, 16384), "machine": (n, g),
         "chain": [("merge", 0, 1), ("split", 0, 16)], "dist": ("block_cyclic", 256), "face": (8, 8)},
        # Johnson / COSMA: a cubic 8 x 8 x 8 grid over a 3-D launch
        {"name": "johnson-3d-cubic", "L": (512, 1024, 512), "machine": (n, g),
         "chain": [("merge", 0, 1), ("split", 0, 8), ("split", 1, 8)], "dist": ("block",), "face": (8, 8, 8)},
    ]
