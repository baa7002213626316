"""Serialisation of block-sparse environments (Sec. III.B.2-3, Fig. 4, Fig. 5).

Test infrastructure.  The paper's serialiser (i) predicts the exact
serialised size before writing, (ii) lets every worker write its part at an
offset fixed in advance, so the parts form one contiguous byte stream, and
(iii) makes every part self-contained: it carries the metadata that locates
it in the whole object, so parts can arrive in any order and still
deserialise into an object identical to the input.

Format (little-endian).  One package per stored block of an operator class
(all layers of the block together, Fig. 4a):

    off  type  field
    0    u32   magic 0x50444247 ("GBDP")
    4    u16   version (1)
    6    u8    dtype (1 = float64)
    7    u8    side (0 = left block, 1 = right block)
    8    u32   block length (orbitals in the block)
    12   u32   number of packages in the environment
    16   u32   package index (position in canonical order)
    20   u32   class index
    24   u32   reserved (0)
    28   u32   layers
    32   i16   q_out.n, i16 q_out.tsz, i16 q_in.n, i16 q_in.tsz
    40   u32   rows
    44   u32   cols
    48   u64   element offset of the block in the unpacked arena (blocks
               follow each other in canonical order, each padded to an even
               number of float64 so that every block starts 16-byte aligned)
    56   u64   checksum
    64   ...   payload: layers*rows*cols float64, row-major per layer,
               zero-padded to a multiple of 16 bytes

checksum = sum_i w_i * (2 i + 1) mod 2^64 over the payload read as u64 words
(padding included; it is zero).  Packages follow each other at 16-byte
aligned offsets given by the exclusive prefix sum of their sizes.
"""
from __future__ import annotations

import struct

import numpy as np

MAGIC = 0x50444247
HEADER = struct.Struct("<IHBBIIIIII hhhh II QQ")
assert HEADER.size == 64
MASK = (1 << 64) - 1


def pad16(n: int) -> int:
    return (n + 15) // 16 * 16


def checksum(payload: bytes) -> int:
    w = np.frombuffer(payload, dtype="<u8")
    i = np.arange(len(w), dtype=np.uint64)
    with np.errstate(over="ignore"):
        return int(np.sum(w * (2 * i + np.uint64(1)), dtype=np.uint64)) & MASK


def canonical_blocks(classes):
    """Flatten classes into (class index, block) in canonical order with arena offsets.

    Returns the list and the arena length in float64 elements.
    """
    out = []
    off = 0
    for ci, cl in enumerate(classes):
        nl = len(cl["layers"])
        for (qo, qi, r, c, data) in cl["blocks"]:
            out.append((ci, nl, qo, qi, r, c, data, off))
            off += (nl * r * c + 1) // 2 * 2
    return out, off


def predicted_sizes(classes):
    """Exact package sizes and offsets before serialising (the size prediction)."""
    blocks, _ = canonical_blocks(classes)
    sizes = [64 + pad16(nl * r * c * 8) for (_, nl, _, _, r, c, _, _) in blocks]
    offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64) if sizes else np.zeros(0, np.int64)
    return sizes, offsets, int(sum(sizes))


def pack(classes, side: int, length: int) -> bytes:
    blocks, _ = canonical_blocks(classes)
    sizes, offsets, total = predicted_sizes(classes)
    buf = bytearray(total)
    n = len(blocks)
    for k, (ci, nl, qo, qi, r, c, data, aoff) in enumerate(blocks):
        payload = np.ascontiguousarray(data, dtype="<f8").tobytes()
        payload += b"\0" * (pad16(len(payload)) - len(payload))
        hdr = HEADER.pack(MAGIC, 1, 1, side, length, n, k, ci, 0, nl,
                          qo[0], qo[1], qi[0], qi[1], r, c, aoff, checksum(payload))
        o = int(offsets[k])
        buf[o:o + 64] = hdr
        buf[o + 64:o + 64 + len(payload)] = payload
    return bytes(buf)


def split_packages(stream: bytes):
    """Walk a stream and return the list of package byte strings."""
    out = []
    o = 0
    while o < len(stream):
        f = HEADER.unpack_from(stream, o)
        nl, r, c = f[9], f[14], f[15]
        size = 64 + pad16(nl * r * c * 8)
        out.append(stream[o:o + size])
        o += size
    return out


def arena(classes):
    """The unpacked arena of an environment: blocks in canonical order, padded."""
    blocks, n = canonical_blocks(classes)
    out = np.zeros(n)
    for (_, nl, _, _, r, c, data, off) in blocks:
        out[off:off + nl * r * c] = np.asarray(data, dtype=np.float64).ravel()
    return out


def unpack(stream: bytes, arena_elems: int):
    """Deserialise packages in any order into a flat float64 arena.

    Raises ValueError on a bad magic number or checksum.
    """
    arena = np.zeros(arena_elems)
    o = 0
    seen = 0
    while o < len(stream):
        f = HEADER.unpack_from(stream, o)
        if f[0] != MAGIC or f[1] != 1:
            raise ValueError("bad package header")
        nl, r, c, aoff, cs = f[9], f[14], f[15], f[16], f[17]
        nbytes = nl * r * c * 8
        payload = stream[o + 64:o + 64 + pad16(nbytes)]
        if checksum(payload) != cs:
            raise ValueError("checksum mismatch")
        arena[aoff:aoff + nl * r * c] = np.frombuffer(payload[:nbytes], dtype="<f8")
        o += 64 + pad16(nbytes)
        seen += 1
    return arena
