"""Philox4x32-10 and the draw mappings used by every random decision.

The paper leaves the random number generator unspecified (it only says genes,
random trees and mutation steps are "determined randomly", Sec. 2.2).  Both the
oracle and the CUDA library therefore implement the same counter-based
generator independently from its published definition:

  Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
  SC'11.  Philox-4x32 with R = 10 rounds: each round multiplies counter words
  0 and 2 by the constants M0, M1 and mixes the high/low halves with words 1
  and 3 and the round key; the key is bumped by the Weyl constants W0, W1
  between rounds.

Stream layout (shared contract, restated on both sides):
  key     = (seed mod 2^32, seed div 2^32)
  counter = (block, individual, generation_or_purpose, run)
  word w of a stream = lane (w mod 4) of block (w div 4)
  generation_or_purpose = g for evolution generation g, or
                          0x80000000 | purpose at initialisation.

Mappings (integer only, so every platform agrees bit for bit):
  idx(w, n) = floor(w * n / 2^32)             -> uniform index in [0, n)
  u24(w)    = (w >> 8) * 2^-24                -> exact float in [0, 1)
  erc(w)    = float32(lo + (hi - lo) * u24(w)) with the product and the sum
              each rounded once in float64 (no fused multiply-add).
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
_MASK = 0xFFFFFFFF

PURPOSE_POP = 1
PURPOSE_RT = 2
INIT_FLAG = 0x80000000


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32 with 10 rounds on arrays of counters.

    ctr: (..., 4) unsigned 32-bit words; key: (..., 2) or (2,).
    Returns (..., 4) uint32.
    """
    c = np.asarray(ctr, dtype=np.uint64)
    k = np.asarray(key, dtype=np.uint64)
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0 = np.broadcast_to(k[..., 0], c0.shape).copy()
    k1 = np.broadcast_to(k[..., 1], c0.shape).copy()
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & _MASK
            k1 = (k1 + W1) & _MASK
        p0 = c0 * np.uint64(M0)          # 32 x 32 -> 64 bit, no overflow
        p1 = c2 * np.uint64(M1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(_MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(_MASK)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def seed_key(seed: int):
    return (seed & _MASK, (seed >> 32) & _MASK)


def stream_words(seed: int, run: int, gen_or_purpose: int, individual: int,
                 n_words: int) -> np.ndarray:
    """First ``n_words`` words of the stream (individual, gen_or_purpose, run)."""
    nb = (n_words + 3) // 4
    ctr = np.zeros((nb, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(nb, dtype=np.uint64)
    ctr[:, 1] = individual
    ctr[:, 2] = gen_or_purpose
    ctr[:, 3] = run
    out = philox4x32_10(ctr, np.array(seed_key(seed), dtype=np.uint64))
    return out.reshape(-1)[:n_words]


def streams_words(seed: int, run: int, gen_or_purpose: int, n_individuals: int,
                  n_words: int) -> np.ndarray:
    """Words [0, n_words) of the streams of individuals 0..n_individuals-1.
    Returns (n_individuals, n_words) uint32."""
    nb = (n_words + 3) // 4
    ctr = np.zeros((n_individuals, nb, 4), dtype=np.uint64)
    ctr[:, :, 0] = np.arange(nb, dtype=np.uint64)[None, :]
    ctr[:, :, 1] = np.arange(n_individuals, dtype=np.uint64)[:, None]
    ctr[:, :, 2] = gen_or_purpose
    ctr[:, :, 3] = run
    out = philox4x32_10(ctr, np.array(seed_key(seed), dtype=np.uint64))
    return out.reshape(n_individuals, nb * 4)[:, :n_words]


def idx(w, n: int):
    """Multiply-shift index in [0, n) (bias at most n / 2^32)."""
    if isinstance(w, np.ndarray):
        return ((w.astype(np.uint64) * np.uint64(n)) >> np.uint64(32)).astype(np.int64)
    return (int(w) * int(n)) >> 32


def u24(w):
    """Top 24 bits of a word as an exact float in [0, 1)."""
    if isinstance(w, np.ndarray):
        return (w >> np.uint32(8)).astype(np.float64) * 2.0 ** -24
    return float(int(w) >> 8) * 2.0 ** -24


def erc(w, lo: float, hi: float) -> np.float32:
    """Ephemeral random constant in [lo, hi): float64 product and sum, each
    rounded once, then rounded to float32."""
    lo64 = float(np.float32(lo))
    hi64 = float(np.float32(hi))
    span = hi64 - lo64            # rounded once
    prod = span * u24(w)          # rounded once (Python floats never fuse)
    return np.float32(lo64 + prod)


class WordStream:
    """Sequential reader of one Philox stream (words drawn in order)."""

    def __init__(self, seed: int, run: int, gen_or_purpose: int, individual: int,
                 chunk: int = 64):
        self.seed, self.run, self.gp, self.ind = seed, run, gen_or_purpose, individual
        self.chunk = chunk
        self.buf = stream_words(seed, run, gen_or_purpose, individual, chunk)
        self.pos = 0

    def next(self) -> int:
        if self.pos >= len(self.buf):
            self.chunk *= 2
            self.buf = stream_words(self.seed, self.run, self.gp, self.ind, self.chunk)
        w = int(self.buf[self.pos])
        self.pos += 1
        return w
