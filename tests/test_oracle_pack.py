"""Pins for oracle.pack: the serialisation contract of Sec. III.B.2-3.

The paper fixes three properties: the size is known before serialising, the
parts form one contiguous stream that deserialises into an identical object,
and each part is self-contained, so parts may be reassembled in any order.
"""
import struct

import numpy as np
import pytest

import inputs
from oracle import pack as P


def test_checksum_closed_form():
    # words 1.0 = 0x3FF0..., 2.0 = 0x4000...: 1*w0 + 3*w1 mod 2^64 = 0xFFF0...
    assert P.checksum(struct.pack("<dd", 1.0, 2.0)) == 0xFFF0000000000000
    assert P.checksum(b"") == 0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_round_trip_bit_exact_and_size_prediction(seed):
    cls = inputs.make_env_blocks(6, seed, empty_every=3)
    blocks, arena_n = P.canonical_blocks(cls)
    sizes, offsets, total = P.predicted_sizes(cls)
    s = P.pack(cls, side=1, length=9)
    assert len(s) == total
    assert all(o % 16 == 0 for o in offsets)
    arena = P.unpack(s, arena_n)
    assert arena.tobytes() == P.arena(cls).tobytes()
    assert all(b[7] % 2 == 0 for b in blocks)


def test_order_independent_reassembly():
    cls = inputs.make_env_blocks(8, 5)
    _, arena_n = P.canonical_blocks(cls)
    s = P.pack(cls, side=0, length=4)
    pk = P.split_packages(s)
    rng = np.random.default_rng(1)
    shuffled = b"".join(pk[i] for i in rng.permutation(len(pk)))
    assert P.unpack(shuffled, arena_n).tobytes() == P.unpack(s, arena_n).tobytes()


def test_corruption_detected():
    cls = inputs.make_env_blocks(3, 9)
    _, arena_n = P.canonical_blocks(cls)
    s = bytearray(P.pack(cls, side=0, length=4))
    # flip one payload byte of the first non-empty package
    off = 0
    for pk in P.split_packages(bytes(s)):
        if len(pk) > 64:
            break
        off += len(pk)
    s[off + 64] ^= 0x01
    with pytest.raises(ValueError):
        P.unpack(bytes(s), arena_n)
    s[off + 64] ^= 0x01
    s[off] ^= 0xFF
    with pytest.raises(ValueError):
        P.unpack(bytes(s), arena_n)
