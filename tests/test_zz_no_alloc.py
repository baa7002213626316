"""The allocation-free pack entry point (gbd_pack_noalloc) against gbd_pack_env.

Some callers cannot allocate device memory: a host runtime whose GPU memory
is entirely owned by another allocator (a framework's caching allocator that
reserved the whole device), or a latency-critical offload thread that must not
take the device synchronisation cudaMalloc/cudaFree can cause.  For them the
library packs an environment that lives in the caller's device memory into
the caller's device buffer, with its scratch in a fixed device array inside
the library.  Its output must equal, byte for byte, what the allocating entry
point produces for the same environment, on consecutive calls (the shared
scratch keeps the previous call's contents, so anything that must start at
zero has to be cleared by each call).
"""
import numpy as np
import pytest

import inputs
import paper_2412_04676_gb300 as g

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_04676_gb300 import build
    build.build()


def _ctx():
    c = g.Context(4, 4, 0)
    h, eri = inputs.make_integrals(4, 1)
    c.load_integrals(h, eri)
    return c


def test_noalloc_pack_equals_pack_env_on_consecutive_calls():
    import torch
    ctx = _ctx()
    for seed in (3, 3, 4):  # the same environment twice, then another one
        cls = inputs.make_env_blocks(9, seed, max_dim=70, empty_every=3)
        ctx.env_import(0, 2, cls)
        want = ctx.pack_env(0, 2).tobytes()
        cm, bm, _ = g.env_metadata(cls)
        arena = torch.from_numpy(ctx.env_export(0, 2)).to("cuda")
        dst = torch.full((len(want) + 64,), 0xAB, dtype=torch.uint8, device="cuda")
        n = g.pack_noalloc(0, 2, arena, cm, bm, dst)
        assert n == len(want)
        out = dst.cpu().numpy()
        assert out[:n].tobytes() == want
        assert np.all(out[n:] == 0xAB)  # nothing written past the stream


def test_noalloc_pack_rejects_small_destination_and_oversize():
    import torch
    cls = inputs.make_env_blocks(4, 9, max_dim=20)
    cm, bm, data = g.env_metadata(cls)
    arena = torch.zeros(max(1, data.size + len(bm)), dtype=torch.float64, device="cuda")
    dst = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(g.GbdError) as e:
        g.pack_noalloc(1, 3, arena, cm, bm, dst)
    assert e.value.code == -1 and e.value.required > 16
    big_cm = np.array([[0, 0, 1]], dtype=np.int32)
    big_bm = np.zeros((40000, 7), dtype=np.int32)
    big_bm[:, 5] = 1
    big_bm[:, 6] = 1
    big_arena = torch.zeros(2 * 40000, dtype=torch.float64, device="cuda")
    with pytest.raises(g.GbdError) as e:
        g.pack_noalloc(0, 1, big_arena, big_cm, big_bm, dst)
    assert e.value.code == -1


def test_noalloc_pack_rejects_misaligned_buffers():
    # a view one double into the arena is only 8-byte aligned: refused before any launch
    import torch
    cls = inputs.make_env_blocks(3, 5, max_dim=10)
    cm, bm, data = g.env_metadata(cls)
    arena = torch.zeros(data.size + 2 * len(bm) + 2, dtype=torch.float64, device="cuda")
    dst = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(g.GbdError) as e:
        g.pack_noalloc(0, 1, arena[1:], cm, bm, dst)
    assert e.value.code == -1
    with pytest.raises(g.GbdError) as e:
        g.pack_noalloc(0, 1, arena, cm, bm, dst[8:])
    assert e.value.code == -1
