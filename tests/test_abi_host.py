"""C-ABI checks that need no GPU: the library loads, exports every symbol
declared in include/gbdmrg.h, validates arguments, and its host-side
operator sets (Eq. 1 split at every cut, Sec. II.B) contract to the
Jordan-Wigner matrix of Eq. 1."""
import numpy as np
import pytest

import inputs
import paper_2412_04676_gb300 as g
from oracle import hamiltonian as H


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_04676_gb300 import build
    build.build()


def test_every_declared_symbol_is_exported():
    names = g.declared_symbols()
    assert len(names) >= 20
    L = g.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert missing == []


def test_argument_validation():
    with pytest.raises(g.GbdError):
        g.Context(3, 3, 0)   # odd N with even 2Sz
    with pytest.raises(g.GbdError):
        g.Context(3, 7, 1)   # too many electrons
    c = g.Context(4, 4, 0)
    h, eri = inputs.make_integrals(4, 3)
    hb = h.copy()
    hb[0, 1] += 1e-6
    with pytest.raises(g.GbdError):
        c.load_integrals(hb, eri)
    eb = eri.copy()
    eb[0, 1, 2, 3] += 1e-6
    with pytest.raises(g.GbdError):
        c.load_integrals(h, eb)


@pytest.mark.parametrize("L,seed", [(2, 4), (3, 5), (4, 6), (5, 7)])
def test_library_operator_sets_contract_to_eq1(L, seed):
    h, eri = inputs.make_integrals(L, seed)
    c = g.Context(L, L, L % 2)
    c.load_integrals(h, eri)
    Hd = c.mpo_dense()
    Hj = H.jw_hamiltonian(h, eri).toarray()
    assert np.abs(Hd - Hj).max() <= 1e-12 * max(1.0, np.abs(Hj).max())


@pytest.mark.parametrize("switch", [2, 3, 4])
def test_switch_position_does_not_change_hamiltonian(switch):
    L = 5
    h, eri = inputs.make_integrals(L, 21)
    c = g.Context(L, 4, 0, switch_cut=switch)
    c.load_integrals(h, eri)
    assert np.abs(c.mpo_dense() - H.jw_hamiltonian(h, eri).toarray()).max() < 1e-12


def test_bond_dimension_is_symmetric_and_quadratic():
    L = 12
    h, eri = inputs.make_integrals(L, 5)
    c = g.Context(L, L, 0, switch_cut=L // 2 + 1)
    c.load_integrals(h, eri)
    d = [c.mpo_bond_dim(k) for k in range(L + 1)]
    assert d[0] == 1 and d[L] == 1
    assert d == d[::-1]
    assert max(d) == d[L // 2]
    # default switch one cut left of the centre: the centre cut is unchanged
    c2 = g.Context(L, L, 0)
    c2.load_integrals(h, eri)
    d2 = [c2.mpo_bond_dim(k) for k in range(L + 1)]
    assert d2[L // 2] == d[L // 2] and d2[L // 2 + 1:] == d[L // 2 + 1:]


def test_config_defaults_and_validation():
    # the mixed form's documented defaults, and the ranges the ABI accepts
    cfg = g.Config()
    assert g.lib().gbd_config_default(g.C.byref(cfg)) == 0
    assert cfg.precision == g.FP64 and cfg.mixed_polish == 2 and cfg.mixed_fp64_blocks == 0
    with pytest.raises(g.GbdError):
        g.Context(4, 4, 0, mixed_polish=3)
    with pytest.raises(g.GbdError):
        g.Context(4, 4, 0, precision=g.SLICED_BF16)  # a product form, not a context precision
    # the two-kernel BF16x3 form is the default; the fused kernel is an option
    assert cfg.bf16x3_fused == 0 and cfg.autotune == 1 and cfg.low_memory == 0
    with pytest.raises(g.GbdError):
        g.Context(4, 4, 0, bf16x3_fused=2)
    g.Context(4, 4, 0, bf16x3_fused=True).close()
    # comparison forms are product forms only
    with pytest.raises(g.GbdError):
        g.Context(4, 4, 0, precision=g.BF16X3_FUSED)
    # the binding's constants are the header's
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "gbdmrg.h")).read()
    val = lambda name: int(re.search(r"\b%s\s*=?\s*(\d+)" % name, hdr).group(1))
    assert g.BF16X3_TWO_PHASE == val("GBD_BF16X3_TWO_PHASE") and g.BF16X3_FUSED == val("GBD_BF16X3_FUSED")
    assert g.MAX_ANCHORS == int(re.search(r"#define GBD_MAX_ANCHORS (\d+)", hdr).group(1))


def test_timers_match_the_documented_list():
    # gbd_timers reports exactly the entries the binding names, all zero
    # before any work (no device needed)
    c = g.Context(4, 4, 0)
    t = c.timers()
    assert list(t) == g.Context.TIMERS
    assert all(v == 0.0 for v in t.values())


def test_export_site_returns_the_imported_blocks():
    # before the sites reach the device, export is the exact inverse of import
    L, N, D = 6, 6, 20
    h, eri = inputs.make_integrals(L, 11)
    sites, dims = inputs.make_mps(L, N, 0, D, 12)
    c = g.Context(L, N, 0, D=D)
    c.load_integrals(h, eri)
    c.import_mps(sites, [1] * L)
    for k in range(L):
        kind, site = c.export_site(k)
        assert kind == 1 and set(site) == set(sites[k])
        for key, blk in sites[k].items():
            assert np.array_equal(site[key], blk)


class _FakeTensor:
    """Stands in for a torch tensor in the binding's checks; its pointer is never used."""

    def __init__(self, n, dtype, is_cuda=True):
        self._n, self.dtype, self.is_cuda = n, dtype, is_cuda

    def data_ptr(self):
        return 0x1000

    def is_contiguous(self):
        return True

    def numel(self):
        return self._n


def test_pack_noalloc_binding_rejects_bad_buffers_before_the_library():
    # the C entry point cannot see the arena's length or which memory a
    # pointer belongs to, so the binding refuses these before any call
    torch = pytest.importorskip("torch")
    cls = inputs.make_env_blocks(4, 9, max_dim=20)
    cm, bm, data = g.env_metadata(cls)
    need = sum((cm[r[0], 2] * r[5] * r[6] + 1) // 2 * 2 for r in bm)
    good_arena = _FakeTensor(need, torch.float64)
    good_dst = _FakeTensor(1 << 20, torch.uint8)
    with pytest.raises(TypeError):      # host (numpy) arena
        g.pack_noalloc(0, 1, np.zeros(need), cm, bm, good_dst)
    with pytest.raises(TypeError):      # CPU tensor
        g.pack_noalloc(0, 1, torch.zeros(need, dtype=torch.float64), cm, bm, good_dst)
    with pytest.raises(TypeError):      # wrong dtype
        g.pack_noalloc(0, 1, _FakeTensor(need, torch.float32), cm, bm, good_dst)
    with pytest.raises(ValueError):     # shorter than the blocks
        g.pack_noalloc(0, 1, _FakeTensor(need - 1, torch.float64), cm, bm, good_dst)
    with pytest.raises(TypeError):      # dst not uint8
        g.pack_noalloc(0, 1, good_arena, cm, bm, _FakeTensor(1 << 20, torch.float64))
    with pytest.raises(TypeError):      # dst on the host
        g.pack_noalloc(0, 1, good_arena, cm, bm, _FakeTensor(1 << 20, torch.uint8, is_cuda=False))
