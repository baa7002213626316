// capi.cu -- the extern "C" boundary of libgbdmrg (declared in include/gbdmrg.h).
// Every entry point converts internal exceptions into status codes and a
// thread-local message; nothing throws across the ABI.
#include <cstring>
#include <string>

#include "engine.h"

using namespace gbd;

struct gbd_ctx {
    Ctx C;
};

namespace {
thread_local std::string g_err;

template <class F> int guard(F&& f) {
    try {
        return f();
    } catch (const Error& e) {
        g_err = e.what();
        return e.code;
    } catch (const std::bad_alloc&) {
        g_err = "host allocation failed";
        return GBD_ERR_HOST_OOM;
    } catch (const std::exception& e) {
        g_err = e.what();
        return GBD_ERR_CUDA;
    }
}

}  // namespace

void gbd::set_last_error(const char* msg) { g_err = msg; }

namespace {
Ctx& ctx(gbd_ctx* c) {
    if (!c) throw Error(GBD_ERR_ARG, "null context");
    return c->C;
}
}  // namespace

extern "C" {

int gbd_version(void) { return 1; }

const char* gbd_last_error(void) { return g_err.c_str(); }

int gbd_config_default(gbd_config* cfg) {
    if (!cfg) { g_err = "null config"; return GBD_ERR_ARG; }
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->D = 256;
    cfg->precision = GBD_FP64;
    cfg->dav_tol = 1e-8;
    cfg->dav_max_sub = 24;
    cfg->dav_keep = 4;
    cfg->dav_max_matvec = 200;
    cfg->offload = 0;
    cfg->device = 0;
    cfg->switch_cut = 0;
    cfg->io_timeout_ms = 120000;
    cfg->seed = 12345;
    cfg->mixed_fp64_blocks = 0;
    cfg->mixed_polish = 2;
    cfg->fault_inject = 0;
    cfg->low_memory = 0;
    cfg->autotune = 1;
    cfg->env_recompute = 0;
    cfg->host_store_bytes = 0;
    cfg->bf16x3_fused = 0;
    return GBD_OK;
}

int gbd_create(const gbd_config* cfg, gbd_ctx** out) {
    return guard([&] {
        GBD_REQUIRE(cfg && out, GBD_ERR_ARG, "null argument");
        GBD_REQUIRE(cfg->L >= 2 && cfg->L <= 16000, GBD_ERR_ARG, "L out of range");
        GBD_REQUIRE(cfg->N >= 0 && cfg->N <= 2 * cfg->L, GBD_ERR_ARG, "N out of range");
        GBD_REQUIRE(((cfg->N + cfg->tsz) % 2 == 0) && std::abs(cfg->tsz) <= cfg->N, GBD_ERR_ARG, "inconsistent (N, 2Sz)");
        GBD_REQUIRE((cfg->N + cfg->tsz) / 2 <= cfg->L && (cfg->N - cfg->tsz) / 2 <= cfg->L, GBD_ERR_ARG,
                    "too many electrons of one spin");
        GBD_REQUIRE(cfg->precision == GBD_FP64 || cfg->precision == GBD_MIXED_BF16X3, GBD_ERR_ARG, "bad precision");
        GBD_REQUIRE(cfg->D >= 1 && cfg->dav_max_sub >= 3 && cfg->dav_max_sub <= 36 && cfg->dav_keep >= 1 &&
                        cfg->dav_max_matvec >= 1 && cfg->dav_tol > 0 && cfg->io_timeout_ms > 0,
                    GBD_ERR_ARG, "bad solver settings");
        GBD_REQUIRE(cfg->mixed_polish >= 0 && cfg->mixed_polish <= 2, GBD_ERR_ARG, "mixed_polish must be 0, 1 or 2");
        GBD_REQUIRE(cfg->low_memory >= -1 && cfg->low_memory <= 1, GBD_ERR_ARG, "low_memory must be -1, 0 or 1");
        GBD_REQUIRE(cfg->autotune == 0 || cfg->autotune == 1, GBD_ERR_ARG, "autotune must be 0 or 1");
        GBD_REQUIRE(cfg->env_recompute == 0 || cfg->env_recompute >= 2, GBD_ERR_ARG, "env_recompute must be 0 or >= 2");
        GBD_REQUIRE(cfg->host_store_bytes >= 0, GBD_ERR_ARG, "host_store_bytes must be >= 0");
        GBD_REQUIRE(cfg->bf16x3_fused == 0 || cfg->bf16x3_fused == 1, GBD_ERR_ARG, "bf16x3_fused must be 0 or 1");
        auto* c = new gbd_ctx();
        c->C.cfg = *cfg;
        *out = c;
        return GBD_OK;
    });
}

void gbd_destroy(gbd_ctx* c) {
    if (!c) return;
    try {
        destroy_ctx(c->C);
    } catch (...) {
    }
    delete c;
}

int gbd_load_integrals(gbd_ctx* c, int L, const double* h, const double* eri, double e_core) {
    return guard([&] {
        GBD_REQUIRE(h && eri, GBD_ERR_ARG, "null integrals");
        load_integrals(ctx(c), L, h, eri, e_core);
        return GBD_OK;
    });
}

int gbd_mpo_bond_dim(gbd_ctx* c, int cut, int* dim) {
    return guard([&] {
        Ctx& C = ctx(c);
        GBD_REQUIRE(C.have_ints, GBD_ERR_STATE, "load integrals first");
        GBD_REQUIRE(dim && cut >= 0 && cut <= C.L, GBD_ERR_ARG, "bad cut");
        *dim = C.mpo.bond_dim(cut);
        return GBD_OK;
    });
}

int gbd_mpo_dense(gbd_ctx* c, double* out, size_t cap) {
    return guard([&] {
        Ctx& C = ctx(c);
        GBD_REQUIRE(C.have_ints, GBD_ERR_STATE, "load integrals first");
        std::vector<double> H = C.mpo.dense();
        GBD_REQUIRE(out && cap >= H.size(), GBD_ERR_ARG, "output too small");
        std::memcpy(out, H.data(), H.size() * sizeof(double));
        return GBD_OK;
    });
}

int gbd_import_site(gbd_ctx* c, int site, int kind, int nblocks, const int* meta, const double* data) {
    return guard([&] {
        GBD_REQUIRE(nblocks == 0 || (meta && data), GBD_ERR_ARG, "null block arrays");
        import_site(ctx(c), site, kind, nblocks, meta, data);
        return GBD_OK;
    });
}

int gbd_export_site(gbd_ctx* c, int site, int* kind, int* nblocks, int* meta, int meta_cap, double* data,
                    size_t data_cap, size_t* data_len) {
    return guard([&] {
        std::vector<int> m;
        std::vector<double> d;
        int k = -1;
        export_site(ctx(c), site, &k, m, d);
        const int nb = int(m.size() / 5);
        if (kind) *kind = k;
        if (nblocks) *nblocks = nb;
        if (data_len) *data_len = d.size();
        if (meta || data) {
            GBD_REQUIRE(meta && data && meta_cap >= nb && data_cap >= d.size(), GBD_ERR_ARG,
                        "export buffers too small (sizes written to *nblocks and *data_len)");
            std::copy(m.begin(), m.end(), meta);
            std::copy(d.begin(), d.end(), data);
        }
        return GBD_OK;
    });
}

int gbd_build_envs(gbd_ctx* c, int b) {
    return guard([&] {
        build_envs(ctx(c), b);
        return GBD_OK;
    });
}

static void ensure_heff(Ctx& C, int b) {
    GBD_REQUIRE(C.have_ints, GBD_ERR_STATE, "load integrals first");
    ensure_cuda(C);
    if (C.H.b != b) setup_heff(C, b);
}

int gbd_build_tables(gbd_ctx* c, int b, gbd_sector_info* out, int cap, int* n, gbd_heff_info* info) {
    return guard([&] {
        Ctx& C = ctx(c);
        ensure_heff(C, b);
        const Heff& H = C.H;
        int ns = int(H.sq.size());
        if (n) *n = ns;
        if (out) {
            GBD_REQUIRE(cap >= ns, GBD_ERR_ARG, "sector table too small");
            for (int i = 0; i < ns; ++i) {
                out[i].n = H.sq[i].n;
                out[i].tsz = H.sq[i].t;
                out[i].rows = H.bL.dim[H.sL[i]];
                out[i].cols = H.bR.dim[H.sR[i]];
                out[i].offset = H.soff[i];
            }
        }
        if (info) {
            info->dim = H.dim;
            info->n_sectors = ns;
            info->n_terms = C.mpo.bond_dim(b + 1);
            info->n_classes = int(H.OL.cls.size());
            info->n_gemm = H.ngemm;
            info->useful_flops = H.flops;
            info->operator_bytes = H.op_bytes;
            info->mixed_bytes = H.mixed_bytes;
            info->mixed_x_bytes = H.mixed_x_bytes;
            info->mem_operators = H.mem_ops;
            info->mem_planes_bf16x3 = H.mem_bf16x3;
            info->mem_planes_sliced = H.mem_sliced;
            info->mem_x_fp64 = H.mem_x64;
            info->mem_x_tensor = H.mem_xtc;
        }
        return GBD_OK;
    });
}

int gbd_apply_heff(gbd_ctx* c, int b, const double* psi_in, double* psi_out, int on_device, int precision) {
    return guard([&] {
        Ctx& C = ctx(c);
        GBD_REQUIRE(psi_in && psi_out && psi_in != psi_out, GBD_ERR_ARG, "bad vectors");
        GBD_REQUIRE(precision == GBD_FP64 || precision == GBD_MIXED_BF16X3 || precision == GBD_SLICED_BF16 ||
                        precision == GBD_FP64_PER_BLOCK || precision == GBD_BF16X3_TWO_PHASE ||
                        precision == GBD_BF16X3_FUSED, GBD_ERR_ARG,
                    "bad precision");
        ensure_heff(C, b);
        Heff& H = C.H;
        if (on_device) {
            apply_heff_dev(C, psi_in, psi_out, precision);
        } else {
            C.dav_x.ensure(size_t(H.dim) * sizeof(double));
            C.dav_ax.ensure(size_t(H.dim) * sizeof(double));
            GBD_CHECK_CUDA(cudaMemcpyAsync(C.dav_x.p, psi_in, size_t(H.dim) * 8, cudaMemcpyHostToDevice, C.cs));
            apply_heff_dev(C, C.dav_x.as<double>(), C.dav_ax.as<double>(), precision);
            GBD_CHECK_CUDA(cudaMemcpyAsync(psi_out, C.dav_ax.p, size_t(H.dim) * 8, cudaMemcpyDeviceToHost, C.cs));
            GBD_CHECK_CUDA(cudaStreamSynchronize(C.cs));
        }
        return GBD_OK;
    });
}

int gbd_heff_diagonal(gbd_ctx* c, int b, double* diag, int on_device) {
    return guard([&] {
        Ctx& C = ctx(c);
        GBD_REQUIRE(diag, GBD_ERR_ARG, "null output");
        ensure_heff(C, b);
        heff_diag(C);
        GBD_CHECK_CUDA(cudaMemcpyAsync(diag, C.H.diag.p, size_t(C.H.dim) * 8,
                                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, C.cs));
        GBD_CHECK_CUDA(cudaStreamSynchronize(C.cs));
        return GBD_OK;
    });
}

int gbd_davidson(gbd_ctx* c, int b, double* psi, double* energy, gbd_dav_stats* stats) {
    return guard([&] {
        Ctx& C = ctx(c);
        ensure_heff(C, b);
        return davidson(C, psi, energy, stats);
    });
}

int gbd_truncate(gbd_ctx* c, int b, int dir, int Dmax, double* trunc_weight) {
    return guard([&] {
        Ctx& C = ctx(c);
        ensure_heff(C, b);
        double w = truncate_step(C, dir, Dmax);
        if (trunc_weight) *trunc_weight = w;
        return GBD_OK;
    });
}

int gbd_sweep(gbd_ctx* c, int nsweeps, int D, gbd_sweep_stats* stats) {
    return guard([&] {
        GBD_REQUIRE(nsweeps >= 1 && D >= 1, GBD_ERR_ARG, "bad sweep arguments");
        return sweep(ctx(c), nsweeps, D, stats);
    });
}

int gbd_step(gbd_ctx* c, int b, int dir, int D, gbd_step_stats* stats) {
    return guard([&] {
        GBD_REQUIRE(dir == 1 || dir == -1, GBD_ERR_ARG, "dir must be +1 or -1");
        GBD_REQUIRE(D >= 1, GBD_ERR_ARG, "D must be >= 1");
        return run_step(ctx(c), b, dir, D, stats);
    });
}

int gbd_get_psi(gbd_ctx* c, double* out, size_t cap, long long* n, int* b) {
    return guard([&] {
        Ctx& C = ctx(c);
        GBD_REQUIRE(C.psi_valid, GBD_ERR_STATE, "no two-site vector");
        size_t len = C.psi.bytes / sizeof(double);
        // the vector length is that of the layout at psi_b
        if (C.H.b == C.psi_b) len = size_t(C.H.dim);
        else {
            const Bond& bl = C.bonds[C.psi_b];
            const Bond& br = C.bonds[C.psi_b + 2];
            EBasis eL = left_enlarged(bl), eR = right_enlarged(br);
            len = 0;
            for (size_t i = 0; i < eL.q.size(); ++i) {
                int j = eR.find(eL.q[i]);
                if (j >= 0) len += size_t(eL.dim[i]) * eR.dim[j];
            }
        }
        if (n) *n = (long long)len;
        if (b) *b = C.psi_b;
        if (out) {
            GBD_REQUIRE(cap >= len, GBD_ERR_ARG, "output too small");
            GBD_CHECK_CUDA(cudaMemcpy(out, C.psi.p, len * sizeof(double), cudaMemcpyDeviceToHost));
        }
        return GBD_OK;
    });
}

int gbd_set_psi(gbd_ctx* c, int b, const double* psi, long long n, int on_device) {
    return guard([&] {
        Ctx& C = ctx(c);
        GBD_REQUIRE(psi, GBD_ERR_ARG, "null vector");
        ensure_heff(C, b);
        GBD_REQUIRE(n == C.H.dim, GBD_ERR_ARG, "vector length does not match the layout at b");
        C.psi.ensure(size_t(n) * sizeof(double));
        GBD_CHECK_CUDA(cudaMemcpyAsync(C.psi.p, psi, size_t(n) * sizeof(double),
                                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, C.cs));
        GBD_CHECK_CUDA(cudaStreamSynchronize(C.cs));
        C.psi_valid = true;
        C.psi_b = b;
        return GBD_OK;
    });
}

int gbd_launch_count(unsigned long long* count) {
    if (!count) { g_err = "null output"; return GBD_ERR_ARG; }
    *count = launch_count();
    return GBD_OK;
}

int gbd_step_energies(gbd_ctx* c, double* out, int cap, int* n) {
    return guard([&] {
        Ctx& C = ctx(c);
        int m = int(C.step_energy.size());
        if (n) *n = m;
        if (out) {
            GBD_REQUIRE(cap >= m, GBD_ERR_ARG, "output too small");
            std::memcpy(out, C.step_energy.data(), size_t(m) * sizeof(double));
        }
        return GBD_OK;
    });
}

int gbd_pack_env(gbd_ctx* c, int side, int cut, void* dst, size_t cap, size_t* bytes, int dst_on_device) {
    return guard([&] {
        Ctx& C = ctx(c);
        GBD_REQUIRE(C.have_ints, GBD_ERR_STATE, "load integrals first");
        OpSet* E = env_of(C, side, cut, false);
        GBD_REQUIRE(E && E->resident(), GBD_ERR_STATE, "environment not resident");
        size_t need = pack_size(*E);
        if (bytes) *bytes = need;
        GBD_REQUIRE(dst && cap >= need, GBD_ERR_ARG, "destination too small (required size written to *bytes)");
        ensure_cuda(C);
        pack_env(C, *E, reinterpret_cast<unsigned char*>(dst), dst_on_device != 0, C.cs);
        return GBD_OK;
    });
}

int gbd_unpack_env(gbd_ctx* c, int side, int cut, const void* src, size_t bytes, int src_on_device) {
    return guard([&] {
        Ctx& C = ctx(c);
        GBD_REQUIRE(C.have_ints, GBD_ERR_STATE, "load integrals first");
        OpSet* E = env_of(C, side, cut, false);
        GBD_REQUIRE(E && E->resident(), GBD_ERR_STATE, "environment not resident");
        GBD_REQUIRE(src || bytes == 0, GBD_ERR_ARG, "null source");
        ensure_cuda(C);
        unpack_env(C, *E, reinterpret_cast<const unsigned char*>(src), bytes, src_on_device != 0, C.cs);
        return GBD_OK;
    });
}

int gbd_env_import(gbd_ctx* c, int side, int cut, int ncls, const int* class_meta, int nblk, const int* block_meta,
                   const double* data) {
    return guard([&] {
        Ctx& C = ctx(c);
        GBD_REQUIRE(C.have_ints, GBD_ERR_STATE, "load integrals first");
        GBD_REQUIRE(ncls >= 0 && nblk >= 0 && (ncls == 0 || class_meta) && (nblk == 0 || (block_meta && data)),
                    GBD_ERR_ARG, "bad environment arrays");
        ensure_cuda(C);
        OpSet* E = env_of(C, side, cut, true);
        *E = OpSet();
        E->side = side;
        E->cut = cut;
        int sid = 0;
        for (int i = 0; i < ncls; ++i) {
            OpClass oc;
            oc.dq = Q{class_meta[3 * i], class_meta[3 * i + 1]};
            GBD_REQUIRE(class_meta[3 * i + 2] >= 1, GBD_ERR_ARG, "class needs >= 1 layer");
            for (int l = 0; l < class_meta[3 * i + 2]; ++l) oc.states.push_back(sid++);
            E->cls.push_back(oc);
        }
        int prev = -1;
        for (int j = 0; j < nblk; ++j) {
            const int* m = block_meta + 7 * j;
            GBD_REQUIRE(m[0] >= 0 && m[0] < ncls && m[0] >= prev && m[5] >= 0 && m[6] >= 0, GBD_ERR_ARG,
                        "blocks must be class-major with valid dims");
            prev = m[0];
            OpBlock b{};
            b.qo = b.qi = -1;
            b.Qo = Q{m[1], m[2]};
            b.Qi = Q{m[3], m[4]};
            b.rows = m[5];
            b.cols = m[6];
            E->cls[m[0]].blocks.push_back(b);
        }
        E->layout();
        size_t n = size_t(std::max<long long>(E->total, 2));
        std::vector<double> host(n, 0.0);
        long long src = 0;
        for (auto& oc : E->cls)
            for (auto& b : oc.blocks) {
                long long cnt = (long long)oc.states.size() * b.rows * b.cols;
                std::memcpy(host.data() + b.off, data + src, size_t(cnt) * sizeof(double));
                src += cnt;
            }
        E->data.ensure(n * sizeof(double));
        GBD_CHECK_CUDA(cudaMemcpy(E->data.p, host.data(), n * sizeof(double), cudaMemcpyHostToDevice));
        return GBD_OK;
    });
}

int gbd_env_export(gbd_ctx* c, int side, int cut, double* out, size_t cap, size_t* elems) {
    return guard([&] {
        Ctx& C = ctx(c);
        OpSet* E = env_of(C, side, cut, false);
        GBD_REQUIRE(E, GBD_ERR_STATE, "environment never built");
        if (!E->resident()) make_resident(C, side, cut);
        if (elems) *elems = size_t(E->total);
        GBD_REQUIRE(out && cap >= size_t(E->total), GBD_ERR_ARG, "output too small");
        GBD_CHECK_CUDA(cudaMemcpy(out, E->data.p, size_t(E->total) * sizeof(double), cudaMemcpyDeviceToHost));
        return GBD_OK;
    });
}

int gbd_tune_info_get(gbd_ctx* c, gbd_tune_info* out) {
    return guard([&] {
        Ctx& C = ctx(c);
        GBD_REQUIRE(out, GBD_ERR_ARG, "null output");
        tc_tune_info(C, out);
        return GBD_OK;
    });
}

int gbd_tune_reset(void) {
    return guard([&] {
        tc_tune_reset();
        return GBD_OK;
    });
}

int gbd_timers(gbd_ctx* c, double* out, int cap, int* n) {
    return guard([&] {
        Ctx& C = ctx(c);
        if (n) *n = Ctx::T_COUNT;
        if (out) {
            GBD_REQUIRE(cap >= Ctx::T_COUNT, GBD_ERR_ARG, "output too small");
            for (int i = 0; i < Ctx::T_COUNT; ++i) out[i] = C.timers[i];
        }
        return GBD_OK;
    });
}

int gbd_io_stats(gbd_ctx* c, double* bytes_d2h, double* bytes_h2d, double* ms_exposed, double* ms_pack,
                 double* ms_save) {
    return guard([&] {
        Ctx& C = ctx(c);
        if (C.cuda_ready) collect_saves(C, true);
        if (ms_save) *ms_save = C.save_ms;
        if (bytes_d2h) *bytes_d2h = C.io_d2h;
        if (bytes_h2d) *bytes_h2d = C.io_h2d;
        if (ms_exposed) *ms_exposed = C.io_exposed_ms;
        if (ms_pack) *ms_pack = C.pack_ms;
        return GBD_OK;
    });
}

}  // extern "C"
