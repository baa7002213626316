"""Python binding of libgbdmrg (ctypes): argument marshalling only.

Every step of the two-site DMRG hot path runs inside the library's CUDA
kernels; this module converts numpy arrays / torch tensors to plain pointers
and status codes to exceptions.  The library must have been built in-tree
(``paper_2412_04676_gb300/build.py``); there is no fallback of any kind.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libgbdmrg.so")
HEADER = os.path.join(HERE, "..", "include", "gbdmrg.h")

FP64, MIXED_BF16X3, SLICED_BF16, FP64_PER_BLOCK, BF16X3_TWO_PHASE, BF16X3_FUSED = 0, 1, 2, 3, 4, 5
FAULT_PINNED_ALLOC, FAULT_IO_NEVER_READY, FAULT_CORRUPT_HOST_COPY = 1, 2, 4
ERRORS = {-1: "GBD_ERR_ARG", -2: "GBD_ERR_DEVICE_OOM", -3: "GBD_ERR_HOST_OOM", -4: "GBD_ERR_CUDA",
          -5: "GBD_ERR_TIMEOUT", -6: "GBD_ERR_CORRUPT", -7: "GBD_ERR_STATE"}
WARN_NOT_CONVERGED, WARN_PRECISION_FLOOR = 1, 2
MAX_ANCHORS = 6  # GBD_MAX_ANCHORS


class GbdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [("L", C.c_int), ("N", C.c_int), ("tsz", C.c_int), ("D", C.c_int), ("precision", C.c_int),
                ("dav_tol", C.c_double), ("dav_max_sub", C.c_int), ("dav_keep", C.c_int),
                ("dav_max_matvec", C.c_int), ("offload", C.c_int), ("device", C.c_int),
                ("switch_cut", C.c_int), ("io_timeout_ms", C.c_int), ("seed", C.c_ulonglong),
                ("mixed_fp64_blocks", C.c_int), ("mixed_polish", C.c_int), ("fault_inject", C.c_int),
                ("autotune", C.c_int), ("env_recompute", C.c_int), ("host_store_bytes", C.c_longlong),
                ("low_memory", C.c_int), ("bf16x3_fused", C.c_int)]


class SectorInfo(C.Structure):
    _fields_ = [("n", C.c_int), ("tsz", C.c_int), ("rows", C.c_int), ("cols", C.c_int), ("offset", C.c_longlong)]


class HeffInfo(C.Structure):
    _fields_ = [("dim", C.c_longlong), ("n_sectors", C.c_int), ("n_terms", C.c_int), ("n_classes", C.c_int),
                ("n_gemm", C.c_longlong), ("useful_flops", C.c_double), ("operator_bytes", C.c_double),
                ("mixed_bytes", C.c_double), ("mixed_x_bytes", C.c_double), ("mem_operators", C.c_double),
                ("mem_planes_bf16x3", C.c_double), ("mem_planes_sliced", C.c_double), ("mem_x_fp64", C.c_double),
                ("mem_x_tensor", C.c_double)]


class StepStats(C.Structure):
    _fields_ = [("energy", C.c_double), ("trunc_weight", C.c_double), ("resid", C.c_double), ("matvecs", C.c_int),
                ("ms_total", C.c_double), ("ms_matvec", C.c_double), ("ms_davidson", C.c_double),
                ("ms_truncate", C.c_double), ("ms_renorm", C.c_double), ("ms_io_exposed", C.c_double),
                ("useful_flops", C.c_double), ("bytes_packed", C.c_double), ("ms_device", C.c_double),
                ("dav_status", C.c_int), ("anchors", C.c_int), ("anchor_resid", C.c_double * MAX_ANCHORS)]


class TuneInfo(C.Structure):
    _fields_ = [("position", C.c_int), ("active", C.c_int), ("n_candidates", C.c_int), ("chosen", C.c_int),
                ("current", C.c_int),
                ("from_cache", C.c_int), ("default_index", C.c_int), ("split_per_sm", C.c_int * 8),
                ("order", C.c_int * 8), ("ms", C.c_double * 8), ("hist", C.c_int * 16), ("key", C.c_ulonglong)]


class DavStats(C.Structure):
    _fields_ = [("energy", C.c_double), ("resid", C.c_double), ("matvecs", C.c_int), ("iterations", C.c_int),
                ("ms_matvec", C.c_double), ("anchors", C.c_int), ("anchor_resid", C.c_double * MAX_ANCHORS)]


class SweepStats(C.Structure):
    _fields_ = [("energy_last", C.c_double), ("energy_min", C.c_double), ("max_trunc", C.c_double),
                ("matvecs", C.c_int), ("ms_total", C.c_double), ("ms_matvec", C.c_double),
                ("ms_davidson", C.c_double), ("ms_truncate", C.c_double), ("ms_renorm", C.c_double),
                ("ms_io_exposed", C.c_double), ("bytes_packed", C.c_double), ("ms_pack", C.c_double),
                ("useful_flops", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

_P = C.c_void_p
_SIGS = {
    "gbd_version": (C.c_int, []),
    "gbd_last_error": (C.c_char_p, []),
    "gbd_config_default": (C.c_int, [C.POINTER(Config)]),
    "gbd_create": (C.c_int, [C.POINTER(Config), C.POINTER(_P)]),
    "gbd_destroy": (None, [_P]),
    "gbd_load_integrals": (C.c_int, [_P, C.c_int, _P, _P, C.c_double]),
    "gbd_mpo_bond_dim": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int)]),
    "gbd_mpo_dense": (C.c_int, [_P, _P, C.c_size_t]),
    "gbd_import_site": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P]),
    "gbd_export_site": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), _P, C.c_int, _P, C.c_size_t,
                                  C.POINTER(C.c_size_t)]),
    "gbd_build_envs": (C.c_int, [_P, C.c_int]),
    "gbd_build_tables": (C.c_int, [_P, C.c_int, _P, C.c_int, C.POINTER(C.c_int), C.POINTER(HeffInfo)]),
    "gbd_apply_heff": (C.c_int, [_P, C.c_int, _P, _P, C.c_int, C.c_int]),
    "gbd_heff_diagonal": (C.c_int, [_P, C.c_int, _P, C.c_int]),
    "gbd_davidson": (C.c_int, [_P, C.c_int, _P, C.POINTER(C.c_double), C.POINTER(DavStats)]),
    "gbd_truncate": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "gbd_sweep": (C.c_int, [_P, C.c_int, C.c_int, _P]),
    "gbd_step_energies": (C.c_int, [_P, _P, C.c_int, C.POINTER(C.c_int)]),
    "gbd_step": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.POINTER(StepStats)]),
    "gbd_get_psi": (C.c_int, [_P, _P, C.c_size_t, C.POINTER(C.c_longlong), C.POINTER(C.c_int)]),
    "gbd_launch_count": (C.c_int, [C.POINTER(C.c_ulonglong)]),
    "gbd_set_psi": (C.c_int, [_P, C.c_int, _P, C.c_longlong, C.c_int]),
    "gbd_pack_env": (C.c_int, [_P, C.c_int, C.c_int, _P, C.c_size_t, C.POINTER(C.c_size_t), C.c_int]),
    "gbd_unpack_env": (C.c_int, [_P, C.c_int, C.c_int, _P, C.c_size_t, C.c_int]),
    "gbd_env_import": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, C.c_int, _P, _P]),
    "gbd_env_export": (C.c_int, [_P, C.c_int, C.c_int, _P, C.c_size_t, C.POINTER(C.c_size_t)]),
    "gbd_io_stats": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                               C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "gbd_timers": (C.c_int, [_P, _P, C.c_int, C.POINTER(C.c_int)]),
    "gbd_tune_info_get": (C.c_int, [_P, C.POINTER(TuneInfo)]),
    "gbd_tune_reset": (C.c_int, []),
    "gbd_pack_noalloc": (C.c_int, [C.c_int, C.c_int, _P, C.c_int, _P, C.c_int, _P, _P, C.c_size_t,
                                   C.POINTER(C.c_size_t), _P]),
}


def tune_reset():
    """Forget every cached autotuner choice (shared by all contexts of the process)."""
    _check(lib().gbd_tune_reset())


def launch_count():
    v = C.c_ulonglong()
    _check(lib().gbd_launch_count(C.byref(v)))
    return v.value


def declared_symbols():
    """Names of the functions declared in include/gbdmrg.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_ ]+\*?\s*\**\s*(gbd_[a-z_]+)\s*\(", txt, re.M)))


def lib():
    """Load the in-tree library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgbdmrg.so not built ({LIB_PATH}); run paper_2412_04676_gb300/build.py")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc < 0:
        raise GbdError(rc, lib().gbd_last_error().decode())
    return rc


def _ptr(a):
    """Pointer of a contiguous numpy array or torch tensor (host or device)."""
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return C.c_void_p(a.data_ptr())
    assert a.flags["C_CONTIGUOUS"]
    return C.c_void_p(a.ctypes.data)


def _on_device(a):
    return int(bool(getattr(a, "is_cuda", False)))


def site_arrays(site):
    """Flatten a dict site tensor {(q_left, s): block} into (meta, data)."""
    keys = sorted(site.keys())
    meta = np.array([[q[0], q[1], s, site[(q, s)].shape[0], site[(q, s)].shape[1]] for (q, s) in keys],
                    dtype=np.int32).reshape(-1, 5)
    data = np.concatenate([np.ascontiguousarray(site[k], dtype=np.float64).ravel() for k in keys]) \
        if keys else np.zeros(0)
    return np.ascontiguousarray(meta), np.ascontiguousarray(data)


def env_metadata(classes):
    """(class_meta, block_meta, data) arrays of an environment in canonical order."""
    cm = np.array([[c["dq"][0], c["dq"][1], len(c["layers"])] for c in classes], dtype=np.int32).reshape(-1, 3)
    bm, data = [], []
    for ci, c in enumerate(classes):
        for (qo, qi, r, cc, d) in c["blocks"]:
            bm.append([ci, qo[0], qo[1], qi[0], qi[1], r, cc])
            data.append(np.ascontiguousarray(d, dtype=np.float64).ravel())
    bm = np.array(bm, dtype=np.int32).reshape(-1, 7)
    data = np.concatenate(data) if data else np.zeros(0)
    return np.ascontiguousarray(cm), np.ascontiguousarray(bm), np.ascontiguousarray(data)


def pack_noalloc(side, length, arena, class_meta, block_meta, dst, stream=None):
    """Allocation-free pack of a caller-owned device arena into a caller-owned device buffer.

    Returns the number of bytes written; raises GbdError (with the required size
    in ``.required``) when dst is too small or a limit is exceeded.
    """
    # the C side cannot see the arena's length or where the buffers live:
    # check here, before anything reaches the device
    for name, t in (("arena", arena), ("dst", dst)):
        if not (hasattr(t, "data_ptr") and getattr(t, "is_cuda", False)):
            raise TypeError(f"pack_noalloc: {name} must be a CUDA tensor")
        if not t.is_contiguous():
            raise ValueError(f"pack_noalloc: {name} must be contiguous")
    import torch
    if arena.dtype != torch.float64:
        raise TypeError("pack_noalloc: arena must be float64")
    if dst.dtype != torch.uint8:
        raise TypeError("pack_noalloc: dst must be uint8")
    class_meta = np.ascontiguousarray(class_meta, dtype=np.int32).reshape(-1, 3)
    block_meta = np.ascontiguousarray(block_meta, dtype=np.int32).reshape(-1, 7)
    need_elems = 0
    for row in block_meta:
        ci = int(row[0])
        if not 0 <= ci < class_meta.shape[0]:
            raise ValueError("pack_noalloc: block class index out of range")
        n = int(class_meta[ci, 2]) * int(row[5]) * int(row[6])
        need_elems += (n + 1) // 2 * 2
    if arena.numel() < need_elems:
        raise ValueError(f"pack_noalloc: arena holds {arena.numel()} doubles, the blocks need {need_elems}")
    need = C.c_size_t()
    nbytes = dst.numel()
    rc = lib().gbd_pack_noalloc(side, length, _ptr(arena), class_meta.shape[0], _ptr(class_meta),
                                block_meta.shape[0], _ptr(block_meta), _ptr(dst), nbytes, C.byref(need),
                                C.c_void_p(stream))
    if rc < 0:
        err = GbdError(rc, lib().gbd_last_error().decode())
        err.required = need.value
        raise err
    return need.value


class Context:
    """One library context: integrals, MPS, environments, two-site position."""

    def __init__(self, L, N, tsz, D=256, precision=FP64, offload=False, device=0, dav_tol=1e-8,
                 dav_max_sub=24, dav_keep=4, dav_max_matvec=200, switch_cut=0, io_timeout_ms=120000, seed=12345,
                 mixed_fp64_blocks=False, mixed_polish=2, fault_inject=0, low_memory=0, autotune=True,
                 env_recompute=0, host_store_bytes=0, bf16x3_fused=False):
        cfg = Config()
        _check(lib().gbd_config_default(C.byref(cfg)))
        cfg.L, cfg.N, cfg.tsz, cfg.D, cfg.precision = L, N, tsz, D, precision
        cfg.offload, cfg.device, cfg.dav_tol = int(offload), device, dav_tol
        cfg.dav_max_sub, cfg.dav_keep, cfg.dav_max_matvec = dav_max_sub, dav_keep, dav_max_matvec
        cfg.switch_cut, cfg.io_timeout_ms, cfg.seed = switch_cut, io_timeout_ms, seed
        cfg.mixed_fp64_blocks, cfg.mixed_polish = int(mixed_fp64_blocks), int(mixed_polish)
        cfg.fault_inject = int(fault_inject)
        cfg.low_memory = int(low_memory)
        cfg.autotune = int(autotune)
        cfg.env_recompute = int(env_recompute)
        cfg.host_store_bytes = int(host_store_bytes)
        cfg.bf16x3_fused = int(bf16x3_fused)
        h = C.c_void_p()
        _check(lib().gbd_create(C.byref(cfg), C.byref(h)))
        self.h = h
        self.L, self.N, self.tsz = L, N, tsz

    def close(self):
        if getattr(self, "h", None):
            lib().gbd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- model
    def load_integrals(self, h, eri, e_core=0.0):
        h = np.ascontiguousarray(h, dtype=np.float64)
        eri = np.ascontiguousarray(eri, dtype=np.float64)
        _check(lib().gbd_load_integrals(self.h, h.shape[0], _ptr(h), _ptr(eri), e_core))

    def mpo_bond_dim(self, cut):
        d = C.c_int()
        _check(lib().gbd_mpo_bond_dim(self.h, cut, C.byref(d)))
        return d.value

    def mpo_dense(self):
        n = 4 ** self.L
        out = np.zeros((n, n))
        _check(lib().gbd_mpo_dense(self.h, _ptr(out), out.size))
        return out

    def import_mps(self, sites, kinds):
        for k, (site, kind) in enumerate(zip(sites, kinds)):
            meta, data = site_arrays(site)
            _check(lib().gbd_import_site(self.h, k, kind, meta.shape[0], _ptr(meta), _ptr(data)))

    def export_site(self, k):
        """(kind, {(q_left, s): block}) of site k, the inverse of import_mps's format."""
        kind, nb, nd = C.c_int(), C.c_int(), C.c_size_t()
        _check(lib().gbd_export_site(self.h, k, C.byref(kind), C.byref(nb), None, 0, None, 0, C.byref(nd)))
        meta = np.zeros((max(nb.value, 1), 5), dtype=np.int32)
        data = np.zeros(max(nd.value, 1))
        _check(lib().gbd_export_site(self.h, k, C.byref(kind), C.byref(nb), _ptr(meta), nb.value, _ptr(data), data.size,
                                     C.byref(nd)))
        site, off = {}, 0
        for (qn, qt, s, r, c) in meta[:nb.value]:
            site[((int(qn), int(qt)), int(s))] = data[off:off + r * c].reshape(r, c).copy()
            off += r * c
        return kind.value, site

    def build_envs(self, b):
        _check(lib().gbd_build_envs(self.h, b))

    # ---------------------------------------------------------------- tables
    def tables(self, b):
        n = C.c_int()
        info = HeffInfo()
        _check(lib().gbd_build_tables(self.h, b, None, 0, C.byref(n), C.byref(info)))
        arr = (SectorInfo * max(n.value, 1))()
        _check(lib().gbd_build_tables(self.h, b, C.cast(arr, C.c_void_p), n.value, C.byref(n), C.byref(info)))
        secs = [dict(q=(a.n, a.tsz), rows=a.rows, cols=a.cols, offset=a.offset) for a in arr[:n.value]]
        return secs, {k: getattr(info, k) for k, _ in HeffInfo._fields_}

    # ---------------------------------------------------------------- hot path
    def apply_heff(self, b, x, out=None, precision=FP64):
        if out is None:
            out = np.zeros_like(x) if not hasattr(x, "data_ptr") else x.new_zeros(x.shape)
        _check(lib().gbd_apply_heff(self.h, b, _ptr(x), _ptr(out), _on_device(x), precision))
        return out

    def heff_diagonal(self, b, dim):
        d = np.zeros(dim)
        _check(lib().gbd_heff_diagonal(self.h, b, _ptr(d), 0))
        return d

    def davidson(self, b, psi=None):
        e = C.c_double()
        st = DavStats()
        p = None
        if psi is not None:
            psi = np.ascontiguousarray(psi, dtype=np.float64)
            p = _ptr(psi)
        rc = _check(lib().gbd_davidson(self.h, b, p, C.byref(e), C.byref(st)))
        out = {k: getattr(st, k) for k, _ in DavStats._fields_}
        out["anchor_resid"] = list(st.anchor_resid)
        return e.value, psi, out, rc

    def truncate(self, b, direction, Dmax):
        w = C.c_double()
        _check(lib().gbd_truncate(self.h, b, direction, Dmax, C.byref(w)))
        return w.value

    def sweep(self, nsweeps, D):
        st = (SweepStats * nsweeps)()
        _check(lib().gbd_sweep(self.h, nsweeps, D, C.cast(st, C.c_void_p)))
        return [s.as_dict() for s in st]

    def step(self, b, direction, D):
        """One two-site iteration; 'dav_status' is 1 when Davidson stopped at its product limit."""
        st = StepStats()
        _check(lib().gbd_step(self.h, b, direction, D, C.byref(st)))
        out = {k: getattr(st, k) for k, _ in StepStats._fields_}
        out["anchor_resid"] = list(st.anchor_resid)
        return out

    def get_psi(self, out=None):
        n = C.c_longlong()
        b = C.c_int()
        _check(lib().gbd_get_psi(self.h, None, 0, C.byref(n), C.byref(b)))
        if out is None:
            out = np.zeros(n.value)
        _check(lib().gbd_get_psi(self.h, _ptr(out), out.size, C.byref(n), C.byref(b)))
        return out, b.value

    def set_psi(self, b, psi):
        n = psi.numel() if hasattr(psi, "numel") else psi.size
        _check(lib().gbd_set_psi(self.h, b, _ptr(psi), n, _on_device(psi)))

    def step_energies(self):
        n = C.c_int()
        _check(lib().gbd_step_energies(self.h, None, 0, C.byref(n)))
        out = np.zeros(max(n.value, 1))
        _check(lib().gbd_step_energies(self.h, _ptr(out), n.value, C.byref(n)))
        return out[:n.value]

    # ---------------------------------------------------------------- pack
    def pack_size(self, side, cut):
        need = C.c_size_t()
        rc = lib().gbd_pack_env(self.h, side, cut, None, 0, C.byref(need), 0)
        if rc not in (0, -1):
            _check(rc)
        return need.value

    def pack_env(self, side, cut, dst=None):
        n = self.pack_size(side, cut)
        if dst is None:
            dst = np.zeros(n, dtype=np.uint8)
        need = C.c_size_t()
        nbytes = dst.numel() if hasattr(dst, "numel") else dst.nbytes
        _check(lib().gbd_pack_env(self.h, side, cut, _ptr(dst), nbytes, C.byref(need), _on_device(dst)))
        return dst

    def unpack_env(self, side, cut, src):
        nbytes = src.numel() if hasattr(src, "numel") else src.nbytes
        _check(lib().gbd_unpack_env(self.h, side, cut, _ptr(src), nbytes, _on_device(src)))

    def env_import(self, side, cut, classes):
        """classes as produced by inputs.make_env_blocks (canonical order)."""
        cm, bm, data = env_metadata(classes)
        _check(lib().gbd_env_import(self.h, side, cut, cm.shape[0], _ptr(cm), bm.shape[0], _ptr(bm), _ptr(data)))

    def env_export(self, side, cut):
        n = C.c_size_t()
        rc = lib().gbd_env_export(self.h, side, cut, None, 0, C.byref(n))
        if rc not in (0, -1):
            _check(rc)
        out = np.zeros(max(n.value, 1))
        _check(lib().gbd_env_export(self.h, side, cut, _ptr(out), out.size, C.byref(n)))
        return out[:n.value]

    TIMERS = ["enlarge_host", "enlarge_dev", "renorm_host", "renorm_dev", "eigensolve", "polish", "tc_prepare",
              "davidson_host", "enlarge_gflop", "renorm_gflop", "tc_issued_gflop_p1", "tc_issued_gflop_p2",
              "products_fp64_ms", "products_bf16x3_ms", "products_sliced_ms", "products_fp64_n", "products_bf16x3_n",
              "products_sliced_n", "tc_sliced_issued_gflop", "tc_prep_split", "tc_prep_plan", "tc_prep_upload",
              "products_fp64_gflop", "products_bf16x3_gflop", "products_sliced_gflop", "renorm_tc_gflop",
              "enlarge_tc_gflop", "step_resident", "step_enlarge", "step_davidson", "step_rho_eig", "step_renorm",
              "step_next", "step_io", "enlarge_host_links", "enlarge_host_subs", "enlarge_host_items",
              "products_bf16x3_gbytes", "products_bf16x3_x_gbytes", "products_fp64_per_block_ms",
              "products_fp64_per_block_n", "recompute_ms", "recompute_n", "spill_gbytes", "restore_gbytes",
              "spill_wait_ms", "products_bf16x3_two_phase_ms", "products_bf16x3_two_phase_n",
              "products_bf16x3_fused_ms", "products_bf16x3_fused_n"]

    def timers(self):
        out = np.zeros(64)
        n = C.c_int()
        _check(lib().gbd_timers(self.h, _ptr(out), 64, C.byref(n)))
        return dict(zip(self.TIMERS, out[:n.value]))

    def tune_info(self):
        """Autotuner state of the BF16x3 product at the current position (see gbd_tune_info)."""
        t = TuneInfo()
        _check(lib().gbd_tune_info_get(self.h, C.byref(t)))
        n = t.n_candidates
        return dict(position=t.position, active=bool(t.active), chosen=t.chosen, current=t.current,
                    from_cache=bool(t.from_cache),
                    default_index=t.default_index, key=t.key, hist=list(t.hist),
                    candidates=[dict(split_per_sm=t.split_per_sm[i], order=t.order[i], ms=t.ms[i]) for i in range(n)])

    def io_stats(self):
        v = [C.c_double() for _ in range(5)]
        _check(lib().gbd_io_stats(self.h, *[C.byref(x) for x in v]))
        return dict(bytes_d2h=v[0].value, bytes_h2d=v[1].value, ms_exposed=v[2].value, ms_pack=v[3].value,
                    ms_save=v[4].value)
