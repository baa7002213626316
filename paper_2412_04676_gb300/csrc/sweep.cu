// sweep.cu -- serialisation of environments (Sec. III.B.2-3 of
// arXiv:2412.04676), their asynchronous save to pinned host RAM and load on
// demand (Sec. III.A strategy 2, Sec. III.B.4 ordering), and the sweep.
//
// Package format (little-endian), one package per stored block of an
// operator class with all its layers (Fig. 4a):
//   u32 magic 0x50444247 | u16 version 1 | u8 dtype 1 (f64) | u8 side |
//   u32 block length (orbitals) | u32 packages in the environment |
//   u32 package index | u32 class index | u32 reserved | u32 layers |
//   i16 q_out.n, q_out.tsz, q_in.n, q_in.tsz | u32 rows | u32 cols |
//   u64 element offset in the arena | u64 checksum | payload (f64, padded to
//   16 bytes).  checksum = sum_i w_i (2i+1) mod 2^64 over the payload words.
// Packages sit at 16-byte aligned offsets, the exclusive prefix sum of their
// exactly predicted sizes, so every CTA of the pack kernel knows where to
// write before it starts (no locks, no inter-thread talk; Sec. III.B.2).
#include <chrono>
#include <cmath>
#include <cstring>
#include <thread>

#include "engine.h"

namespace gbd {

#pragma pack(push, 1)
struct PkgHeader {
    uint32_t magic;
    uint16_t version;
    uint8_t dtype;
    uint8_t side;
    uint32_t length;
    uint32_t npk;
    uint32_t index;
    uint32_t cls;
    uint32_t reserved;
    uint32_t layers;
    int16_t qon, qot, qin, qit;
    uint32_t rows, cols;
    uint64_t aoff;
    uint64_t checksum;
};
#pragma pack(pop)
static_assert(sizeof(PkgHeader) == 64, "package header must be 64 bytes");

static constexpr uint32_t kMagic = 0x50444247u;
static constexpr unsigned long long kChunkWords = 8192;  // 64 KB per CTA

static inline size_t pad16(size_t n) { return (n + 15) / 16 * 16; }

size_t pack_size(const OpSet& E) {
    size_t s = 0;
    for (const auto& c : E.cls)
        for (const auto& b : c.blocks) s += 64 + pad16(size_t(c.states.size()) * b.rows * b.cols * 8);
    return s;
}

namespace {

struct PackHost {
    std::vector<unsigned char> headers;
    std::vector<PackItem> items;
    std::vector<PackChunk> chunks;
    size_t total = 0;
};

int env_length(const Ctx& C, const OpSet& E) { return E.side == 0 ? E.cut : C.L - E.cut; }

void build_pack(const Ctx& C, const OpSet& E, PackHost& P) {
    int npk = 0;
    for (const auto& c : E.cls) npk += int(c.blocks.size());
    P.headers.assign(size_t(npk) * 64, 0);
    P.items.clear();
    P.chunks.clear();
    size_t off = 0;
    int k = 0;
    const double* base = E.data.as<double>();
    for (size_t ci = 0; ci < E.cls.size(); ++ci) {
        const OpClass& c = E.cls[ci];
        for (const auto& b : c.blocks) {
            size_t bytes = size_t(c.states.size()) * b.rows * b.cols * 8;
            PkgHeader h{};
            h.magic = kMagic;
            h.version = 1;
            h.dtype = 1;
            h.side = uint8_t(E.side);
            h.length = uint32_t(env_length(C, E));
            h.npk = uint32_t(npk);
            h.index = uint32_t(k);
            h.cls = uint32_t(ci);
            h.layers = uint32_t(c.states.size());
            h.qon = int16_t(b.Qo.n); h.qot = int16_t(b.Qo.t);
            h.qin = int16_t(b.Qi.n); h.qit = int16_t(b.Qi.t);
            h.rows = uint32_t(b.rows);
            h.cols = uint32_t(b.cols);
            h.aoff = uint64_t(b.off);
            h.checksum = 0;
            std::memcpy(P.headers.data() + size_t(k) * 64, &h, 64);
            unsigned long long words = pad16(bytes) / 8;
            P.items.push_back({base ? base + b.off : nullptr, nullptr, off, words});
            for (unsigned long long w0 = 0; w0 < words; w0 += kChunkWords)
                P.chunks.push_back({k, w0, std::min(words, w0 + kChunkWords)});
            off += 64 + pad16(bytes);
            ++k;
        }
    }
    P.total = off;
}

// device copies of pack metadata (grow-only)
struct MetaBufs {
    DevBuf headers, items, chunks, cks;
};

void upload_meta(const PackHost& P, MetaBufs& M, bool with_headers, cudaStream_t st) {
    if (with_headers) {
        M.headers.ensure(std::max<size_t>(P.headers.size(), 64));
        GBD_CHECK_CUDA(cudaMemcpyAsync(M.headers.p, P.headers.data(), P.headers.size(), cudaMemcpyHostToDevice, st));
    }
    M.items.ensure(std::max<size_t>(P.items.size(), 1) * sizeof(PackItem));
    M.chunks.ensure(std::max<size_t>(P.chunks.size(), 1) * sizeof(PackChunk));
    M.cks.ensure(std::max<size_t>(P.items.size(), 1) * sizeof(unsigned long long));
    if (!P.items.empty())
        GBD_CHECK_CUDA(cudaMemcpyAsync(M.items.p, P.items.data(), P.items.size() * sizeof(PackItem), cudaMemcpyHostToDevice, st));
    if (!P.chunks.empty())
        GBD_CHECK_CUDA(cudaMemcpyAsync(M.chunks.p, P.chunks.data(), P.chunks.size() * sizeof(PackChunk),
                                       cudaMemcpyHostToDevice, st));
}

MetaBufs& meta_for(Ctx& C, int slot) {
    static thread_local std::vector<std::unique_ptr<MetaBufs>> pool;
    (void)C;
    while ((int)pool.size() <= slot) pool.push_back(std::make_unique<MetaBufs>());
    return *pool[slot];
}

}  // namespace

// Serialises E into dst.  dst_gpu: dst is device memory or mapped pinned host
// memory the kernels may write; otherwise a device staging buffer is used.
void pack_env(Ctx& C, const OpSet& E, unsigned char* dst, bool dst_gpu, cudaStream_t st) {
    GBD_REQUIRE(E.resident(), GBD_ERR_STATE, "environment not resident");
    PackHost P;
    build_pack(C, E, P);
    if (P.total == 0) return;
    MetaBufs& M = meta_for(C, 0);
    upload_meta(P, M, true, st);
    unsigned char* base = dst;
    if (!dst_gpu) {
        C.stage.ensure(P.total);
        base = C.stage.as<unsigned char>();
    }
    cudaEvent_t a, b;
    GBD_CHECK_CUDA(cudaEventCreate(&a));
    GBD_CHECK_CUDA(cudaEventCreate(&b));
    GBD_CHECK_CUDA(cudaEventRecord(a, st));
    pack_launch(base, M.headers.as<unsigned char>(), M.items.as<PackItem>(), int(P.items.size()),
                M.chunks.as<PackChunk>(), int(P.chunks.size()), M.cks.as<unsigned long long>(), st);
    GBD_CHECK_CUDA(cudaEventRecord(b, st));
    if (!dst_gpu) GBD_CHECK_CUDA(cudaMemcpyAsync(dst, base, P.total, cudaMemcpyDefault, st));
    GBD_CHECK_CUDA(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    C.pack_ms += ms;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
}

// Deserialises packages in any order into E (block structure must match).
// src_host: a host-readable copy of the stream (for the header walk);
// src_gpu: the stream as the kernels may read it (device or mapped pinned),
// or nullptr to stage src_host through device memory.
static void unpack_core(Ctx& C, OpSet& E, const unsigned char* src_host, const unsigned char* src_gpu, size_t bytes,
                        cudaStream_t st) {
    GBD_REQUIRE(E.resident(), GBD_ERR_STATE, "environment not resident");
    std::vector<const OpBlock*> blk;
    std::vector<int> blk_cls;
    for (size_t ci = 0; ci < E.cls.size(); ++ci)
        for (const auto& b : E.cls[ci].blocks) { blk.push_back(&b); blk_cls.push_back(int(ci)); }
    const int npk = int(blk.size());
    PackHost P;
    std::vector<uint64_t> want(npk, 0);
    std::vector<int> seen(npk, 0);
    size_t off = 0;
    int len = env_length(C, E);
    while (off < bytes) {
        GBD_REQUIRE(off + 64 <= bytes, GBD_ERR_CORRUPT, "truncated package header");
        PkgHeader h;
        std::memcpy(&h, src_host + off, 64);
        GBD_REQUIRE(h.magic == kMagic && h.version == 1 && h.dtype == 1, GBD_ERR_CORRUPT, "bad package magic/version");
        GBD_REQUIRE(h.side == E.side && int(h.length) == len && int(h.npk) == npk && int(h.index) < npk,
                    GBD_ERR_CORRUPT, "package belongs to another environment");
        const OpBlock& b = *blk[h.index];
        const OpClass& c = E.cls[blk_cls[h.index]];
        GBD_REQUIRE(int(h.cls) == blk_cls[h.index] && int(h.layers) == int(c.states.size()) && int(h.rows) == b.rows &&
                        int(h.cols) == b.cols && h.qon == b.Qo.n && h.qot == b.Qo.t && h.qin == b.Qi.n &&
                        h.qit == b.Qi.t && (long long)h.aoff == b.off,
                    GBD_ERR_CORRUPT, "package metadata disagrees with the environment");
        GBD_REQUIRE(!seen[h.index], GBD_ERR_CORRUPT, "duplicate package");
        seen[h.index] = 1;
        size_t pb = size_t(h.layers) * h.rows * h.cols * 8;
        GBD_REQUIRE(off + 64 + pad16(pb) <= bytes, GBD_ERR_CORRUPT, "truncated package payload");
        unsigned long long words = pad16(pb) / 8;
        int item = int(P.items.size());
        P.items.push_back({nullptr, E.data.as<double>() + b.off, off, words});
        want[item] = h.checksum;
        for (unsigned long long w0 = 0; w0 < words; w0 += kChunkWords)
            P.chunks.push_back({item, w0, std::min(words, w0 + kChunkWords)});
        off += 64 + pad16(pb);
    }
    for (int i = 0; i < npk; ++i) GBD_REQUIRE(seen[i], GBD_ERR_CORRUPT, "missing package");
    MetaBufs& M = meta_for(C, 1);
    upload_meta(P, M, false, st);
    const unsigned char* base = src_gpu;
    if (!base) {
        C.stage.ensure(bytes);
        GBD_CHECK_CUDA(cudaMemcpyAsync(C.stage.p, src_host, bytes, cudaMemcpyDefault, st));
        base = C.stage.as<unsigned char>();
    }
    GBD_CHECK_CUDA(cudaMemsetAsync(M.cks.p, 0, std::max<size_t>(P.items.size(), 1) * 8, st));
    unpack_launch(base, M.items.as<PackItem>(), M.chunks.as<PackChunk>(), int(P.chunks.size()),
                  M.cks.as<unsigned long long>(), st);
    std::vector<uint64_t> got(P.items.size());
    if (!got.empty())
        GBD_CHECK_CUDA(cudaMemcpyAsync(got.data(), M.cks.p, got.size() * 8, cudaMemcpyDeviceToHost, st));
    GBD_CHECK_CUDA(cudaStreamSynchronize(st));
    for (size_t i = 0; i < got.size(); ++i) GBD_REQUIRE(got[i] == want[i], GBD_ERR_CORRUPT, "package checksum mismatch");
}

void unpack_env(Ctx& C, OpSet& E, const unsigned char* src, size_t bytes, bool src_device, cudaStream_t st) {
    if (src_device) {
        std::vector<unsigned char> h(bytes);
        GBD_CHECK_CUDA(cudaMemcpyAsync(h.data(), src, bytes, cudaMemcpyDeviceToHost, st));
        GBD_CHECK_CUDA(cudaStreamSynchronize(st));
        unpack_core(C, E, h.data(), src, bytes, st);
    } else {
        unpack_core(C, E, src, nullptr, bytes, st);
    }
}

// ============================================================== offload
namespace {

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// bounded host wait on an event; the elapsed time counts as exposed IO
void wait_event(Ctx& C, cudaEvent_t e) {
    if (!e) return;
    double t0 = now_ms();
    const bool never = (C.cfg.fault_inject & GBD_FAULT_IO_NEVER_READY) != 0;
    while (true) {
        cudaError_t r = never ? cudaErrorNotReady : cudaEventQuery(e);
        if (r == cudaSuccess) break;
        if (r != cudaErrorNotReady) GBD_CHECK_CUDA(r);
        if (now_ms() - t0 > C.cfg.io_timeout_ms) throw Error(GBD_ERR_TIMEOUT, "IO event wait timed out");
        std::this_thread::yield();
    }
    C.io_exposed_ms += now_ms() - t0;
}

HostEnv& host_of(Ctx& C, int side, int cut) { return side == 0 ? C.hostL[cut] : C.hostR[cut]; }

void pinned_grow(const Ctx& C, unsigned char*& p, size_t& cap, size_t need) {
    if (need <= cap && p) return;
    if (p) cudaFreeHost(p);
    p = nullptr;
    size_t c = std::max(need, cap + cap / 4);
    if ((C.cfg.fault_inject & GBD_FAULT_PINNED_ALLOC) ||
        cudaHostAlloc((void**)&p, c, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        cap = 0;
        throw Error(GBD_ERR_HOST_OOM, "pinned host allocation failed");
    }
    cap = c;
}

// ---- bounded host store (host_store_bytes) and its spill file

SpillStore& spill_of(Ctx& C) {
    if (!C.spill) C.spill = std::make_unique<SpillStore>();
    return *C.spill;
}

// Waits for h's spill job (bounded by io_timeout_ms, counted as exposed IO);
// a finished write frees the pinned copy, a finished read makes it valid.
void finish_job(Ctx& C, HostEnv& h) {
    if (!h.job) return;
    const double t0 = now_ms();
    const int st = SpillStore::wait(h.job, C.cfg.io_timeout_ms);
    const double dt = now_ms() - t0;
    C.io_exposed_ms += dt;
    C.timers[Ctx::T_SPILL_WAIT_MS] += dt;
    if (st == 0) throw Error(GBD_ERR_TIMEOUT, "spill file job wait timed out");
    if (st < 0) throw Error(GBD_ERR_HOST_OOM, "spill file read or write failed");
    if (h.job->write) {
        cudaFreeHost(h.host);
        C.pinned_bytes -= h.cap;
        h.host = nullptr;
        h.cap = 0;
        h.spilled = true;
        C.timers[Ctx::T_SPILL_GB] += double(h.bytes) * 1e-9;
    } else {
        h.spilled = false;
        h.restoring = false;
        C.timers[Ctx::T_RESTORE_GB] += double(h.bytes) * 1e-9;
    }
    h.job.reset();
}

// Frees the pinned copies whose spill writes have finished (no wait).
void reap_spills(Ctx& C) {
    for (auto* v : {&C.hostL, &C.hostR})
        for (auto& h : *v)
            if (h.job && h.job->write && h.job->state.load() != 0) finish_job(C, h);
}

// Makes room for `need` more pinned bytes: the least recently used saved
// environments whose saves have finished are written to the spill file;
// their pinned copies go once the writes finish.  The bound is soft: with
// nothing left to spill the store grows past it.
void make_room(Ctx& C, size_t need, const HostEnv* self) {
    const long long budget = C.cfg.host_store_bytes;
    if (budget <= 0) return;
    reap_spills(C);
    while ((long long)(C.pinned_bytes + need) > budget) {
        HostEnv* victim = nullptr;
        for (auto* v : {&C.hostL, &C.hostR})
            for (auto& h : *v) {
                if (&h == self || !h.host || !h.valid || h.job || h.pending || h.restoring) continue;
                if (h.done && cudaEventQuery(h.done) != cudaSuccess) { cudaGetLastError(); continue; }  // save running
                if (!victim || h.stamp < victim->stamp) victim = &h;
            }
        if (victim) {
            size_t cap = 0;
            victim->file_off = spill_of(C).region(victim->file_off, victim->file_cap, victim->bytes, &cap);
            victim->file_cap = cap;
            victim->job = spill_of(C).submit(true, victim->host, victim->bytes, victim->file_off);
        }
        // the oldest write in flight frees its copy
        HostEnv* oldest = nullptr;
        for (auto* v : {&C.hostL, &C.hostR})
            for (auto& h : *v)
                if (h.job && h.job->write && (!oldest || h.stamp < oldest->stamp)) oldest = &h;
        if (!oldest) break;
        finish_job(C, *oldest);
    }
}

// The pinned buffer of h's packed stream, within the store's bound.
void host_alloc(Ctx& C, HostEnv& h, size_t need) {
    if (h.host && need <= h.cap) return;
    if (h.host) {
        cudaFreeHost(h.host);
        C.pinned_bytes -= h.cap;
        h.host = nullptr;
        h.cap = 0;
    }
    const size_t c = C.cfg.host_store_bytes > 0 ? need : std::max<size_t>(need, 64);
    make_room(C, c, &h);
    pinned_grow(C, h.host, h.cap, c);
    C.pinned_bytes += h.cap;
}

template <class T> T* dev_view(void* host) {
    void* d = nullptr;
    GBD_CHECK_CUDA(cudaHostGetDevicePointer(&d, host, 0));
    return reinterpret_cast<T*>(d);
}

// item + chunk tables copied into the id's mapped pinned buffer
void stage_tables(const Ctx& C, HostEnv& h, const PackHost& P, PackItem** d_items, PackChunk** d_chunks) {
    size_t ib = P.items.size() * sizeof(PackItem), cb = P.chunks.size() * sizeof(PackChunk);
    size_t ib16 = pad16(ib);
    pinned_grow(C, h.meta, h.meta_cap, ib16 + cb + 16);
    if (ib) std::memcpy(h.meta, P.items.data(), ib);
    if (cb) std::memcpy(h.meta + ib16, P.chunks.data(), cb);
    unsigned char* d = dev_view<unsigned char>(h.meta);
    *d_items = reinterpret_cast<PackItem*>(d);
    *d_chunks = reinterpret_cast<PackChunk*>(d + ib16);
    size_t nk = std::max<size_t>(P.items.size(), 1);
    if (nk > h.cks_cap) {
        if (h.cks_dev) cudaFree(h.cks_dev);
        if (h.cks_host) cudaFreeHost(h.cks_host);
        h.cks_dev = nullptr;
        h.cks_host = nullptr;
        GBD_CHECK_CUDA(cudaMalloc((void**)&h.cks_dev, nk * 8));
        GBD_CHECK_CUDA(cudaHostAlloc((void**)&h.cks_host, nk * 8, cudaHostAllocDefault));
        h.cks_cap = nk;
    }
}

// Asynchronous save (Sec. III.A strategy 2): the pack kernel writes straight
// into mapped pinned host memory on the IO stream once the compute stream
// has produced E; no device staging copy, so no device memory peak.
void save_async(Ctx& C, int side, int cut) {
    OpSet* E = env_of(C, side, cut, false);
    if (!E || !E->resident()) return;
    HostEnv& h = host_of(C, side, cut);
    wait_event(C, h.done);
    if (h.pending) wait_event(C, h.loaded);
    finish_job(C, h);  // a spill or restore of the old content in flight
    PackHost P;
    build_pack(C, *E, P);
    h.spilled = false;
    h.restoring = false;
    h.stamp = ++C.io_stamp;
    host_alloc(C, h, std::max<size_t>(P.total, 64));
    if (!h.done) GBD_CHECK_CUDA(cudaEventCreateWithFlags(&h.done, cudaEventDisableTiming));
    h.bytes = P.total;
    h.npk = int(P.items.size());
    for (size_t i = 0; i < P.items.size(); ++i) std::memcpy(h.host + P.items[i].pkg, P.headers.data() + i * 64, 64);
    PackItem* di = nullptr;
    PackChunk* dc = nullptr;
    stage_tables(C, h, P, &di, &dc);
    cudaEvent_t ready;
    GBD_CHECK_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    GBD_CHECK_CUDA(cudaEventRecord(ready, C.cs));
    GBD_CHECK_CUDA(cudaStreamWaitEvent(C.ios, ready, 0));
    cudaEventDestroy(ready);
    Ctx::PendingSave ps{};
    GBD_CHECK_CUDA(cudaEventCreate(&ps.a));
    GBD_CHECK_CUDA(cudaEventCreate(&ps.b));
    GBD_CHECK_CUDA(cudaEventRecord(ps.a, C.ios));
    pack_launch(dev_view<unsigned char>(h.host), nullptr, di, int(P.items.size()), dc, int(P.chunks.size()), h.cks_dev,
                C.ios);
    GBD_CHECK_CUDA(cudaEventRecord(ps.b, C.ios));
    C.saves.push_back(ps);
    GBD_CHECK_CUDA(cudaEventRecord(h.done, C.ios));
    h.valid = true;
    C.io_d2h += double(P.total);
}

// Release the device arena after every use already enqueued on the compute
// stream and the pending save (both ordered before the free on the IO stream).
void release_async(Ctx& C, int side, int cut) {
    OpSet* E = env_of(C, side, cut, false);
    if (!E || !E->resident()) return;
    HostEnv& h = host_of(C, side, cut);
    if (!h.valid) return;  // never drop the only copy
    cudaEvent_t used;
    GBD_CHECK_CUDA(cudaEventCreateWithFlags(&used, cudaEventDisableTiming));
    GBD_CHECK_CUDA(cudaEventRecord(used, C.cs));
    GBD_CHECK_CUDA(cudaStreamWaitEvent(C.ios, used, 0));
    cudaEventDestroy(used);
    E->data.release_async(C.ios);
}

// Releases the device arena of an environment that has no host copy; it is
// rebuilt when needed (env_recompute).
void drop_async(Ctx& C, int side, int cut) {
    OpSet* E = env_of(C, side, cut, false);
    if (!E || !E->resident()) return;
    cudaEvent_t used;
    GBD_CHECK_CUDA(cudaEventCreateWithFlags(&used, cudaEventDisableTiming));
    GBD_CHECK_CUDA(cudaEventRecord(used, C.cs));
    GBD_CHECK_CUDA(cudaStreamWaitEvent(C.ios, used, 0));
    cudaEventDestroy(used);
    E->data.release_async(C.ios);
}

// A new environment goes to the host store, or (env_recompute, not a
// checkpoint) any older host copy of its id is invalidated.
void store_env(Ctx& C, int side, int cut) {
    if (env_checkpoint(C, side, cut)) {
        save_async(C, side, cut);
    } else {
        HostEnv& h = host_of(C, side, cut);
        wait_event(C, h.done);
        h.valid = false;
    }
}

// Releases an environment after its last use: kept in the host store, or
// (env_recompute) dropped to be rebuilt.
void retire_env(Ctx& C, int side, int cut) {
    if (C.cfg.env_recompute && !env_checkpoint(C, side, cut)) drop_async(C, side, cut);
    else release_async(C, side, cut);
}

// Load on demand (Sec. III.B.4): walk the self-contained headers on the host,
// then unpack from mapped pinned memory on the IO stream; the checksums are
// verified when the environment is first used.
void load_async(Ctx& C, int side, int cut) {
    OpSet* E = env_of(C, side, cut, false);
    GBD_REQUIRE(E, GBD_ERR_STATE, "environment never built");
    if (E->resident()) return;
    HostEnv& h = host_of(C, side, cut);
    GBD_REQUIRE(h.valid, GBD_ERR_STATE, "environment neither resident nor saved");
    h.stamp = ++C.io_stamp;
    if (h.job && h.job->write) finish_job(C, h);  // a spill of it in flight
    if (h.spilled) {
        // read back into pinned memory on the IO thread; the unpack follows
        // when the step needs it (ensure_resident)
        if (!h.restoring) {
            host_alloc(C, h, h.bytes);
            h.job = spill_of(C).submit(false, h.host, h.bytes, h.file_off);
            h.restoring = true;
        }
        return;
    }
    wait_event(C, h.done);  // "fetching": the save must have finished
    size_t n = size_t(std::max<long long>(E->total, 2)) * sizeof(double);
    E->data.alloc_async(n, C.ios);
    GBD_CHECK_CUDA(cudaMemsetAsync(E->data.p, 0, n, C.ios));
    std::vector<const OpBlock*> blk;
    for (const auto& c : E->cls)
        for (const auto& b : c.blocks) blk.push_back(&b);
    PackHost P;
    h.want.assign(blk.size(), 0);
    size_t off = 0;
    while (off < h.bytes) {
        PkgHeader hd;
        std::memcpy(&hd, h.host + off, 64);
        GBD_REQUIRE(hd.magic == kMagic && hd.index < blk.size() && (long long)hd.aoff == blk[hd.index]->off,
                    GBD_ERR_CORRUPT, "bad package in host copy");
        size_t pb = size_t(hd.layers) * hd.rows * hd.cols * 8;
        unsigned long long words = pad16(pb) / 8;
        int item = int(P.items.size());
        P.items.push_back({nullptr, E->data.as<double>() + hd.aoff, off, words});
        h.want[item] = hd.checksum;
        for (unsigned long long w0 = 0; w0 < words; w0 += kChunkWords)
            P.chunks.push_back({item, w0, std::min(words, w0 + kChunkWords)});
        off += 64 + pad16(pb);
    }
    h.want.resize(P.items.size());
    if (C.cfg.fault_inject & GBD_FAULT_CORRUPT_HOST_COPY) {
        // one payload byte of the first non-empty package is flipped in host
        // memory after its save finished: the checksum must catch it
        for (const auto& it : P.items)
            if (it.words > 0) { h.host[it.pkg + 64] ^= 0x01; break; }
    }
    PackItem* di = nullptr;
    PackChunk* dc = nullptr;
    stage_tables(C, h, P, &di, &dc);
    GBD_CHECK_CUDA(cudaMemsetAsync(h.cks_dev, 0, std::max<size_t>(P.items.size(), 1) * 8, C.ios));
    unpack_launch(dev_view<unsigned char>(h.host), di, dc, int(P.chunks.size()), h.cks_dev, C.ios);
    if (!P.items.empty())
        GBD_CHECK_CUDA(cudaMemcpyAsync(h.cks_host, h.cks_dev, P.items.size() * 8, cudaMemcpyDeviceToHost, C.ios));
    if (!h.loaded) GBD_CHECK_CUDA(cudaEventCreateWithFlags(&h.loaded, cudaEventDisableTiming));
    GBD_CHECK_CUDA(cudaEventRecord(h.loaded, C.ios));
    h.pending = true;
    C.io_h2d += double(h.bytes);
}

void ensure_resident(Ctx& C, int side, int cut) {
    OpSet* E = env_of(C, side, cut, false);
    GBD_REQUIRE(E, GBD_ERR_STATE, "environment never built");
    HostEnv& h = host_of(C, side, cut);
    if (!E->resident() && !h.valid && C.cfg.env_recompute) {
        rebuild_env(C, side, cut);  // recomputation instead of IO
        return;
    }
    if (!E->resident()) {
        load_async(C, side, cut);
        if (h.restoring) {  // residency checkpoint: the restore must have finished
            finish_job(C, h);
            load_async(C, side, cut);
        }
    }
    if (h.pending) {
        wait_event(C, h.loaded);
        for (size_t i = 0; i < h.want.size(); ++i)
            GBD_REQUIRE(h.cks_host[i] == h.want[i], GBD_ERR_CORRUPT, "package checksum mismatch on load");
        h.pending = false;
    }
}

}  // namespace

// Saves an environment to the pinned host store and releases its device
// arena once the save and every use already enqueued have finished (with
// env_recompute, only checkpoints are saved; the others are dropped).
void offload_env(Ctx& C, int side, int cut) {
    store_env(C, side, cut);
    retire_env(C, side, cut);
}

bool env_checkpoint(const Ctx& C, int side, int cut) {
    (void)side;
    const int k = C.cfg.env_recompute;
    return k < 2 || cut == 0 || cut == C.L || cut % k == 0;
}

// An environment made resident for the caller: if it lives only in the
// pinned host store it is loaded back through the offload path (unpack from
// mapped pinned memory, checksums verified).
void make_resident(Ctx& C, int side, int cut) {
    ensure_cuda(C);
    ensure_resident(C, side, cut);
}

// collect the device time of finished asynchronous saves
void collect_saves(Ctx& C, bool wait) {
    std::vector<Ctx::PendingSave> keep;
    for (auto& ps : C.saves) {
        if (wait) GBD_CHECK_CUDA(cudaEventSynchronize(ps.b));
        if (cudaEventQuery(ps.b) == cudaSuccess) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ps.a, ps.b);
            C.save_ms += ms;
            cudaEventDestroy(ps.a);
            cudaEventDestroy(ps.b);
        } else {
            keep.push_back(ps);
        }
    }
    C.saves.swap(keep);
}

// ============================================================== step / sweep
// One DMRG iteration of Sec. II.B at position b, moving towards dir.
int run_step(Ctx& C, int b, int dir, int D, gbd_step_stats* out) {
    GBD_REQUIRE(C.have_ints, GBD_ERR_STATE, "load integrals first");
    GBD_REQUIRE(b >= 0 && b + 1 < C.L, GBD_ERR_ARG, "two-site position out of range");
    ensure_cuda(C);
    const bool off = C.cfg.offload != 0;
    const int L = C.L;
    collect_saves(C, false);
    double t0 = now_ms();
    double io0 = C.io_exposed_ms, d2h0 = C.io_d2h, mv0 = C.ms_matvec_acc;
    cudaEvent_t ea, eb;
    GBD_CHECK_CUDA(cudaEventCreate(&ea));
    GBD_CHECK_CUDA(cudaEventCreate(&eb));
    GBD_CHECK_CUDA(cudaEventRecord(ea, C.cs));
    C.marks.clear();
    step_mark(C, Ctx::T_PH_RESIDENT);
    // pre-processing: environments resident, enlarged operators
    ensure_resident(C, 0, b);
    ensure_resident(C, 1, b + 2);
    step_mark(C, Ctx::T_PH_ENLARGE);
    if (C.H.b != b || !C.H.OL.resident()) setup_heff(C, b);
    if (off) {  // both environments are consumed by the enlargement
        retire_env(C, 0, b);
        retire_env(C, 1, b + 2);
    }
    double t1 = now_ms();
    double e = 0.0;
    gbd_dav_stats ds{};
    step_mark(C, Ctx::T_PH_DAVIDSON);
    const int dav_status = davidson(C, nullptr, &e, &ds);
    double flops = C.H.flops * ds.matvecs;
    double t2 = now_ms();
    double w = truncate_step(C, dir, D);
    step_mark(C, Ctx::T_PH_IO);
    if (off) {
        // Sec. III.B.4: the next environment is loaded right after the
        // renormalisation, then the new one is saved asynchronously
        int nb = b + dir;
        if (nb >= 0 && nb + 1 < L) {
            int need_side = dir == 1 ? 1 : 0;
            int need_cut = dir == 1 ? nb + 2 : nb;
            OpSet* nE = env_of(C, need_side, need_cut, false);
            if (nE && !nE->resident() && host_of(C, need_side, need_cut).valid) load_async(C, need_side, need_cut);
        }
        if (dir == 1) store_env(C, 0, b + 1);
        else store_env(C, 1, b + 1);
    }
    step_mark(C, Ctx::T_PH_IO);  // closing mark
    GBD_CHECK_CUDA(cudaEventRecord(eb, C.cs));
    GBD_CHECK_CUDA(cudaEventSynchronize(eb));
    step_marks_flush(C);
    float msd = 0.f;
    cudaEventElapsedTime(&msd, ea, eb);
    cudaEventDestroy(ea);
    cudaEventDestroy(eb);
    double t3 = now_ms();
    C.step_energy.push_back(e);
    if (out) {
        out->ms_device = msd;
        out->energy = e;
        out->trunc_weight = w;
        out->resid = ds.resid;
        out->matvecs = ds.matvecs;
        out->ms_total = t3 - t0;
        out->ms_matvec = C.ms_matvec_acc - mv0;
        out->ms_davidson = (t2 - t1) - out->ms_matvec;
        out->ms_truncate = t3 - t2;
        out->ms_renorm = t1 - t0;
        out->ms_io_exposed = C.io_exposed_ms - io0;
        out->useful_flops = flops;
        out->bytes_packed = C.io_d2h - d2h0;
        out->dav_status = dav_status;
        out->anchors = ds.anchors;
        for (int i = 0; i < GBD_MAX_ANCHORS; ++i) out->anchor_resid[i] = ds.anchor_resid[i];
    }
    return dav_status;
}

int sweep(Ctx& C, int nsweeps, int D, gbd_sweep_stats* stats) {
    GBD_REQUIRE(C.have_ints, GBD_ERR_STATE, "load integrals first");
    const int L = C.L;
    GBD_REQUIRE(L >= 3, GBD_ERR_ARG, "a sweep needs L >= 3");
    for (int k = 0; k < L; ++k)
        GBD_REQUIRE(C.site_kind[k] == 1, GBD_ERR_STATE, "import a right-isometric MPS (all sites) before sweeping");
    ensure_cuda(C);
    build_envs(C, 0);  // right environments for cuts L..2, left at cut 0
    const bool off = C.cfg.offload != 0;
    if (off)
        for (int c = 2; c <= L; ++c) store_env(C, 1, c);
    // start vector on (0, 1) from B_0 B_1 (host, from the imported blocks)
    setup_heff(C, 0);
    {
        Heff& H = C.H;
        std::vector<double> psi(size_t(H.dim), 0.0);
        const Iso& B0 = C.sites[0];
        const Iso& B1 = C.sites[1];
        // Psi[Q][seg s0][seg s1] = B0[(0,0), s0] B1[(q_s0, s1)] with B = V^T
        for (size_t si = 0; si < H.sq.size(); ++si) {
            Q Qs = H.sq[si];
            int eL = H.sL[si], eR = H.sR[si];
            int ncol = H.bR.dim[eR];
            for (const auto& sl : H.bL.segs[eL]) {  // s0 with bond-0 sector (0,0)
                int e0 = B0.basis.find(Q{0, 0});
                if (e0 < 0) continue;
                const Seg* g0 = nullptr;
                for (const auto& g : B0.basis.segs[e0]) if (g.s == sl.s) g0 = &g;
                if (!g0) continue;
                int o1 = B1.out.find(Qs);
                int e1 = B1.basis.find(Qs);
                if (o1 < 0 || e1 < 0) continue;
                int d1 = B1.out.dim[o1];
                for (const auto& sr : H.bR.segs[eR]) {
                    const Seg* g1 = nullptr;
                    for (const auto& g : B1.basis.segs[e1]) if (g.s == sr.s) g1 = &g;
                    if (!g1) continue;
                    for (int j = 0; j < g1->size; ++j) {
                        double v = 0.0;
                        for (int a = 0; a < d1; ++a)
                            v += B0.host[B0.off[0] + (g0->off + a)] * B1.host[B1.off[o1] + (long long)(g1->off + j) * d1 + a];
                        psi[H.soff[si] + (long long)sl.off * ncol + sr.off + j] = v;
                    }
                }
            }
        }
        C.psi.ensure(psi.size() * sizeof(double));
        GBD_CHECK_CUDA(cudaMemcpy(C.psi.p, psi.data(), psi.size() * sizeof(double), cudaMemcpyHostToDevice));
        C.psi_valid = true;
        C.psi_b = 0;
    }
    C.step_energy.clear();
    for (int sw = 0; sw < nsweeps; ++sw) {
        gbd_sweep_stats st{};
        st.energy_min = 1e300;
        double t_start = now_ms();
        double pk0 = C.pack_ms;
        auto step = [&](int b, int dir) {
            gbd_step_stats ss{};
            run_step(C, b, dir, D, &ss);
            st.max_trunc = std::max(st.max_trunc, ss.trunc_weight);
            st.matvecs += ss.matvecs;
            st.energy_last = ss.energy;
            st.energy_min = std::min(st.energy_min, ss.energy);
            st.ms_matvec += ss.ms_matvec;
            st.ms_davidson += ss.ms_davidson;
            st.ms_truncate += ss.ms_truncate;
            st.ms_renorm += ss.ms_renorm;
            st.ms_io_exposed += ss.ms_io_exposed;
            st.bytes_packed += ss.bytes_packed;
            st.useful_flops += ss.useful_flops;
        };
        for (int b = 0; b <= L - 3; ++b) step(b, 1);
        for (int b = L - 2; b >= 1; --b) step(b, -1);
        GBD_CHECK_CUDA(cudaStreamSynchronize(C.cs));
        st.ms_total = now_ms() - t_start;
        st.ms_pack = C.pack_ms - pk0;
        if (stats) stats[sw] = st;
    }
    GBD_CHECK_CUDA(cudaStreamSynchronize(C.ios));
    return GBD_OK;
}

}  // namespace gbd
