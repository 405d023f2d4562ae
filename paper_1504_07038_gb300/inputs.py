"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds random-number generation only -- none of the Mojette
arithmetic. Pixels are uniform 64-bit words from a counter-based SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014; finaliser constants from Vigna's public-domain splitmix64.c):

    word(seed, i) = mix(seed + (i + 1) * 0x9E3779B97F4A7C15)   (mod 2^64)
    mix(z): z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
            z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31

with i the global word index ``stripe * Q * P + l * P + x``. Any stripe can
therefore be regenerated on its own, which is how parity tests at full size
check sampled stripes.

The paper benchmarks single 4 KB / 8 KB blocks "filled with random data"
(Sec. 3.1); these generators stand in for that data.
"""
from __future__ import annotations

import itertools

import numpy as np

DEFAULT_SEED = 1504070381
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK_STREAM = np.uint64(0xD1B54A32D192ED03)   # separates erasure draws from pixels


def _mix(z: np.ndarray) -> np.ndarray:
    z = z ^ (z >> np.uint64(30))
    z = z * _M1
    z = z ^ (z >> np.uint64(27))
    z = z * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, index: np.ndarray) -> np.ndarray:
    """Counter-based SplitMix64 at the given uint64 indices."""
    with np.errstate(over="ignore"):
        idx = np.asarray(index, dtype=np.uint64)
        return _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx + np.uint64(1)) * _GAMMA)


def stripes(S: int, Q: int, P: int, seed: int = DEFAULT_SEED, first: int = 0,
            chunk_words: int = 1 << 24) -> np.ndarray:
    """``uint64[S, Q, P]``: stripes ``first .. first + S - 1`` of the stream."""
    words = Q * P
    out = np.empty(S * words, dtype=np.uint64)
    base = first * words
    for a in range(0, S * words, chunk_words):
        b = min(S * words, a + chunk_words)
        out[a:b] = splitmix64(seed, np.arange(base + a, base + b, dtype=np.uint64))
    return out.reshape(S, Q, P)


def stripe_rows(idx: np.ndarray, Q: int, P: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """The stripes with the given global indices, ``uint64[len(idx), Q, P]``."""
    idx = np.asarray(idx, dtype=np.uint64)
    w = np.arange(Q * P, dtype=np.uint64)
    g = idx[:, None] * np.uint64(Q * P) + w[None, :]
    return splitmix64(seed, g).reshape(len(idx), Q, P)


def erasure_masks(S: int, n: int, erasures, seed: int = DEFAULT_SEED,
                  first: int = 0) -> np.ndarray:
    """One seeded erasure mask per stripe (bit i set: projection i lost).

    ``erasures`` is a count for every stripe or an array of per-stripe counts.
    Each stripe draws n keys and loses the projections holding its smallest
    keys, so every subset of the given size is equally likely.
    """
    s = np.arange(first, first + S, dtype=np.uint64)
    keys = splitmix64(seed ^ int(_MASK_STREAM),
                      s[:, None] * np.uint64(n) + np.arange(n, dtype=np.uint64)[None, :])
    order = np.argsort(keys, axis=1, kind="stable")
    e = np.broadcast_to(np.asarray(erasures, dtype=np.int64), (S,))
    rank = np.empty_like(order)
    np.put_along_axis(rank, order, np.arange(n)[None, :].repeat(S, 0), axis=1)
    lost = rank < e[:, None]
    bits = (lost.astype(np.uint64) << np.arange(n, dtype=np.uint64)[None, :]).sum(axis=1)
    return bits.astype(np.uint32)


def erasure_counts(S: int, max_erasures: int, seed: int = DEFAULT_SEED,
                   first: int = 0) -> np.ndarray:
    """Per-stripe erasure counts uniform on 0..max_erasures (seeded)."""
    s = np.arange(first, first + S, dtype=np.uint64)
    k = splitmix64(seed ^ int(_MASK_STREAM) ^ 0x5555, s)
    return (k % np.uint64(max_erasures + 1)).astype(np.int64)


def categories(S: int, k: int, seed: int = DEFAULT_SEED, first: int = 0) -> np.ndarray:
    """Per-stripe category in 0..k-1, uniform and seeded (e.g. which geometry
    a stripe of a mixed batch uses)."""
    s = np.arange(first, first + S, dtype=np.uint64)
    c = splitmix64(seed ^ int(_MASK_STREAM) ^ 0xA5A5, s)
    return (c % np.uint64(k)).astype(np.int64)


def permutation(S: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """A seeded permutation of 0..S-1 (stripes sorted by a counter-based key)."""
    keys = splitmix64(seed ^ int(_MASK_STREAM) ^ 0x3C3C, np.arange(S, dtype=np.uint64))
    return np.argsort(keys, kind="stable")


def all_masks(n: int, erasures: int):
    """Every mask of n projections with exactly ``erasures`` bits set."""
    out = []
    for lost in itertools.combinations(range(n), erasures):
        m = 0
        for i in lost:
            m |= 1 << i
        out.append(m)
    return out
