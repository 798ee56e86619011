"""Bucket hash and fingerprint of a cell descriptor (Section 2.2.1).

The paper hashes the descriptor twice: a first hash picks the bucket, a
second one gives the fingerprint used to recognise the cell while probing
linearly, the pair chosen from the Jarzynski & Olano (2020) study of GPU
hash functions without naming them.  This reading takes two functions from
that study:

* the PCG hash (one LCG step, multiplier 747796405, increment 2891336453,
  followed by PCG's RXS-M-XS output permutation) for the bucket;
* the xxHash32 mixing of one 4-byte word (xxHash specification: seed +
  PRIME5 + length, word * PRIME3, rotate 17, * PRIME4, then the avalanche)
  for the fingerprint.

A 64-bit descriptor is folded as h(lo ^ h(hi)) for the bucket and as
xxh(lo, seed = xxh(hi, seed 0)) for the fingerprint.

Cell identity: the bucket ("home" slot) is h1 mod N; the fingerprint is the
top 24 bits of h2 (0 is reserved for empty slots and is remapped to 1).  The
stored 32-bit tag is fingerprint << 8 | (home mod 256); with probe runs
shorter than 256 slots a tag can only ever be matched from its own home, so a
cell is exactly the pair (home, fingerprint), whatever the insertion order.
"""
from __future__ import annotations

import numpy as np

U32 = np.uint32

PCG_MUL = U32(747796405)
PCG_INC = U32(2891336453)
PCG_OUT = U32(277803737)

XXH_P1 = U32(0x9E3779B1)
XXH_P2 = U32(0x85EBCA77)
XXH_P3 = U32(0xC2B2AE3D)
XXH_P4 = U32(0x27D4EB2F)
XXH_P5 = U32(0x165667B1)


def _u32(a):
    return np.atleast_1d(np.asarray(a)).astype(np.uint32)


def pcg_hash(v):
    """PCG hash of 32-bit words (LCG step then RXS-M-XS output permutation)."""
    v = _u32(v)
    state = v * PCG_MUL + PCG_INC
    shift = (state >> U32(28)) + U32(4)
    word = ((state >> shift) ^ state) * PCG_OUT
    return (word >> U32(22)) ^ word


def _rotl(x, r):
    return (x << U32(r)) | (x >> U32(32 - r))


def xxh32_word(w, seed):
    """xxHash32 of one 4-byte little-endian word with the given seed."""
    w = _u32(w)
    h = _u32(seed) + XXH_P5 + U32(4)
    h = h + w * XXH_P3
    h = _rotl(h, 17) * XXH_P4
    h = h ^ (h >> U32(15))
    h = h * XXH_P2
    h = h ^ (h >> U32(13))
    h = h * XXH_P3
    h = h ^ (h >> U32(16))
    return h


def cell_identity(key, log2_slots: int):
    """(home slot, 24-bit fingerprint) of 64-bit descriptors."""
    key = np.atleast_1d(np.asarray(key, np.uint64))
    lo = (key & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    hi = (key >> np.uint64(32)).astype(np.uint32)
    h1 = pcg_hash(lo ^ pcg_hash(hi))
    home = h1 & U32((1 << log2_slots) - 1)
    h2 = xxh32_word(lo, xxh32_word(hi, 0))
    fp = h2 >> U32(8)
    fp = np.where(fp == 0, U32(1), fp).astype(np.uint32)
    return home, fp


def identity_u64(home, fp):
    """Packed identity home << 24 | fingerprint, as sorted and compared by the tests."""
    return (np.asarray(home, np.uint64) << np.uint64(24)) | np.asarray(fp, np.uint64)


def tag_of(home, fp):
    """32-bit word stored in the slot array: fingerprint << 8 | (home mod 256)."""
    return ((np.asarray(fp, np.uint32) << U32(8)) | (np.asarray(home, np.uint32) & U32(0xFF))).astype(np.uint32)
