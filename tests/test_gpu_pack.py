"""GPU pack/unpack (Sec. III.B.2-3) against the oracle serialiser: byte-exact.

The library's packed stream of an imported environment must equal the
oracle's stream byte for byte; packages reassemble in any order; a flipped
byte is caught by the checksum; a computed environment round-trips exactly.
"""
import numpy as np
import pytest

import inputs
import paper_2412_04676_gb300 as g
from gpu_common import build_lib, heff_case
from oracle import pack as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build_lib()


def _ctx():
    c = g.Context(4, 4, 0)
    h, eri = inputs.make_integrals(4, 1)
    c.load_integrals(h, eri)
    return c


@pytest.mark.parametrize("seed,ncls,maxd", [(0, 6, 40), (1, 10, 3), (2, 4, 300)])
def test_pack_bytes_equal_oracle(seed, ncls, maxd):
    cls = inputs.make_env_blocks(ncls, seed, max_dim=maxd, empty_every=4)
    c = _ctx()
    c.env_import(0, 2, cls)
    want = P.pack(cls, side=0, length=2)
    assert c.pack_size(0, 2) == len(want)
    got = c.pack_env(0, 2)
    assert got.tobytes() == want
    assert c.env_export(0, 2).tobytes() == P.arena(cls).tobytes()


def test_unpack_any_order_and_device_buffers():
    import torch
    cls = inputs.make_env_blocks(8, 7, max_dim=120)
    c = _ctx()
    c.env_import(1, 1, cls)
    stream = P.pack(cls, side=1, length=3)
    pk = P.split_packages(stream)
    order = np.random.default_rng(2).permutation(len(pk))
    shuffled = np.frombuffer(b"".join(pk[i] for i in order), dtype=np.uint8).copy()
    c.env_import(1, 1, [dict(dq=x["dq"], layers=x["layers"],
                             blocks=[(a, b_, r, cc, np.zeros_like(d)) for (a, b_, r, cc, d) in x["blocks"]])
                        for x in cls])
    c.unpack_env(1, 1, shuffled)
    assert c.env_export(1, 1).tobytes() == P.arena(cls).tobytes()
    # device-resident stream in and out
    dev = torch.empty(len(stream), dtype=torch.uint8, device="cuda")
    c.pack_env(1, 1, dev)
    assert dev.cpu().numpy().tobytes() == stream
    c.unpack_env(1, 1, dev)
    assert c.env_export(1, 1).tobytes() == P.arena(cls).tobytes()


def test_corrupt_package_rejected():
    cls = inputs.make_env_blocks(5, 11, max_dim=30)
    c = _ctx()
    c.env_import(0, 3, cls)
    s = np.frombuffer(P.pack(cls, side=0, length=3), dtype=np.uint8).copy()
    first = next(len(x) for x in P.split_packages(s.tobytes()))
    off = 0
    for x in P.split_packages(s.tobytes()):
        if len(x) > 64:
            break
        off += len(x)
    s[off + 70] ^= 0x10
    with pytest.raises(g.GbdError) as e:
        c.unpack_env(0, 3, s)
    assert e.value.code == -6
    s[off + 70] ^= 0x10
    s[4] = 9  # version
    with pytest.raises(g.GbdError) as e:
        c.unpack_env(0, 3, s)
    assert e.value.code == -6
    assert first >= 64


def test_computed_environment_round_trip():
    c = heff_case(10, 10, 0, 64, 400, 5, oracle=False)
    ctx = c["ctx"]
    before = ctx.env_export(0, 5)
    s = ctx.pack_env(0, 5)
    assert len(s) == ctx.pack_size(0, 5)
    ctx.unpack_env(0, 5, s)
    assert ctx.env_export(0, 5).tobytes() == before.tobytes()


def test_offload_round_trip_is_byte_exact():
    # an environment a step saved (pack kernel into mapped pinned host memory
    # on the IO stream), that the next step released from the device after
    # using it, is loaded back through the offload path (unpack from pinned
    # memory, package checksums verified) with the bytes it had before the save
    L, N, D, b = 8, 8, 40, 2
    h, eri = inputs.make_integrals(L, 51)
    sites, dims = inputs.make_mps(L, N, 0, D, 52, n_left=b)
    c = g.Context(L, N, 0, D=D, offload=True)
    c.load_integrals(h, eri)
    c.import_mps(sites, [0] * b + [1] * (L - b))
    c.build_envs(b)
    c.step(b, 1, D)                 # creates the left environment at cut b+1 and saves it
    before = c.env_export(0, b + 1)
    c.step(b + 1, 1, D)             # consumes it; afterwards it lives only in pinned host memory
    h2d0 = c.io_stats()["bytes_h2d"]
    after = c.env_export(0, b + 1)  # loaded back through the offload path
    assert c.io_stats()["bytes_h2d"] > h2d0
    assert after.tobytes() == before.tobytes()
    c.close()
