"""Pins for oracle/hashing.py: the two hash functions against their published
definitions (a byte-oriented XXH32 written from the xxHash specification and
its reference test vector; PCG values worked step by step from its published definition
and its permutation property), and the identity /
tag construction of Section 2.2.1's bucket + fingerprint scheme."""
import json
import os

import numpy as np

from oracle import hashing

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "sequences.json")))
M32 = 0xFFFFFFFF
P1, P2, P3, P4, P5 = 0x9E3779B1, 0x85EBCA77, 0xC2B2AE3D, 0x27D4EB2F, 0x165667B1


def _rotl(x, r):
    return ((x << r) | (x >> (32 - r))) & M32


def xxh32_bytes(data: bytes, seed: int) -> int:
    """General XXH32 over a byte string (inputs shorter than 16 bytes take the short path:
    seed + PRIME5 + length, then 4-byte lanes, then single bytes, then the avalanche)."""
    assert len(data) < 16
    h = (seed + P5 + len(data)) & M32
    i = 0
    while i + 4 <= len(data):
        w = int.from_bytes(data[i:i + 4], "little")
        h = (h + w * P3) & M32
        h = (_rotl(h, 17) * P4) & M32
        i += 4
    while i < len(data):
        h = (h + data[i] * P5) & M32
        h = (_rotl(h, 11) * P1) & M32
        i += 1
    h ^= h >> 15
    h = (h * P2) & M32
    h ^= h >> 13
    h = (h * P3) & M32
    h ^= h >> 16
    return h


def test_xxh32_reference_vector():
    assert xxh32_bytes(b"", 0) == int(GOLDEN["xxh32_empty_seed0"], 16)


def test_xxh32_word_matches_byte_definition():
    rng = np.random.default_rng(1)
    w = rng.integers(0, 2 ** 32, 300, dtype=np.uint64).astype(np.uint32)
    s = rng.integers(0, 2 ** 32, 300, dtype=np.uint64).astype(np.uint32)
    got = hashing.xxh32_word(w, s)
    for a, b, g in zip(w, s, got):
        assert int(g) == xxh32_bytes(int(a).to_bytes(4, "little"), int(b))


def test_pcg_is_a_permutation_on_a_large_sample():
    # an LCG step, a data-dependent xorshift and an odd multiply are each bijective on 32-bit words
    rng = np.random.default_rng(2)
    v = np.unique(rng.integers(0, 2 ** 32, 1 << 20, dtype=np.uint64)).astype(np.uint32)
    h = hashing.pcg_hash(v)
    assert np.unique(h).size == v.size
    # consecutive integers too
    v = np.arange(1 << 20, dtype=np.uint32)
    assert np.unique(hashing.pcg_hash(v)).size == v.size


def test_pcg_worked_values():
    # values worked step by step from the published definition (golden file lists every step)
    for row in GOLDEN["pcg_worked"]:
        assert int(hashing.pcg_hash(int(row["v"], 16))[0]) == int(row["out"], 16), row["v"]


def test_pcg_worked_values_are_self_consistent():
    # each listed intermediate follows from the previous one: a typo in the golden file fails here,
    # not silently in the oracle test above
    for row in GOLDEN["pcg_worked"]:
        v, st = int(row["v"], 16), int(row["state"], 16)
        assert st == (v * 747796405 + 2891336453) % 2 ** 32
        assert row["shift"] == (st >> 28) + 4
        assert int(row["xorshift"], 16) == (st >> row["shift"]) ^ st
        w = int(row["word"], 16)
        assert w == int(row["xorshift"], 16) * 277803737 % 2 ** 32
        assert int(row["out"], 16) == (w >> 22) ^ w


def test_cell_identity_worked_fold():
    # bucket h(lo ^ h(hi)) and fingerprint xxh(lo, xxh(hi)) >> 8 of one descriptor, worked by hand:
    # a swapped fold (hi and lo exchanged, or the seed chain reversed) gives other values
    g = GOLDEN["fold_worked"]
    key = int(g["key"], 16)
    home, fp = hashing.cell_identity(np.uint64(key), 16)
    assert int(home[0]) == int(g["home_log2_16"], 16)
    assert int(fp[0]) == int(g["fingerprint"], 16)
    # the intermediates agree with the byte-oriented XXH32 pinned to its reference vector
    assert xxh32_bytes((1).to_bytes(4, "little"), 0) == int(g["xxh_hi_seed0"]["avalanche"][-1], 16)
    assert xxh32_bytes((2).to_bytes(4, "little"), int(g["xxh_hi_seed0"]["avalanche"][-1], 16)) == \
        int(g["xxh_lo_seed"]["avalanche"][-1], 16)
    assert int(g["xxh_lo_seed"]["avalanche"][-1], 16) >> 8 == int(g["fingerprint"], 16)


def test_identity_fingerprint_never_zero_and_tag_layout():
    rng = np.random.default_rng(3)
    keys = rng.integers(0, 2 ** 63, 200000, dtype=np.uint64)
    home, fp = hashing.cell_identity(keys, 16)
    assert home.max() < (1 << 16)
    assert fp.min() >= 1 and fp.max() < (1 << 24)
    tag = hashing.tag_of(home, fp)
    assert np.all(tag != 0)
    assert np.all((tag & 0xFF) == (home & 0xFF))
    assert np.all((tag >> 8) == fp)
    # identity packs and unpacks losslessly
    ident = hashing.identity_u64(home, fp)
    assert np.all((ident >> np.uint64(24)) == home)
    assert np.all((ident & np.uint64(0xFFFFFF)) == fp)


def test_identity_spreads_over_buckets():
    # the bucket hash of consecutive keys fills buckets like a uniform draw (chi-square bound)
    keys = np.arange(1 << 18, dtype=np.uint64)
    home, _ = hashing.cell_identity(keys, 10)
    cnt = np.bincount(home, minlength=1024)
    exp = keys.size / 1024
    chi2 = ((cnt - exp) ** 2 / exp).sum()
    assert chi2 < 1024 + 6 * np.sqrt(2 * 1024)
