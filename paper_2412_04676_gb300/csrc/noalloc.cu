// noalloc.cu -- an allocation-free variant of the environment pack.
//
// gbd_pack_env works on environments the library owns and uses device
// scratch that the library allocates (package tables and per-package checksum
// accumulators).  gbd_pack_noalloc serves callers that cannot allocate device
// memory at all: a host runtime whose device memory is entirely owned by
// another allocator (for example a framework caching allocator that has
// reserved the whole GPU, so a fresh cudaMalloc fails or fragments its pool),
// or a latency-critical offload thread that must not take the implicit
// device-wide synchronisation cudaMalloc / cudaFree can cause.  Such a caller
// passes the block-sparse environment and the output buffer in its own device
// memory; the scratch lives in the fixed file-scope array below, which every
// GPU that loads this library holds until the process exits.
#include <cstring>
#include <mutex>
#include <string>

#include "engine.h"

namespace gbd {

// Scratch of the allocation-free pack: headers, item and chunk tables and the
// checksum accumulators of at most kNoallocMaxPackages packages.
constexpr size_t kNoallocScratchBytes = size_t(8) << 20;  // 8 MiB per device
constexpr int kNoallocMaxPackages = 32768;
constexpr int kNoallocMaxChunks = 65536;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {

constexpr size_t kHdrOff = 0;
constexpr size_t kItemOff = kHdrOff + size_t(kNoallocMaxPackages) * 64;
constexpr size_t kChunkOff = kItemOff + size_t(kNoallocMaxPackages) * sizeof(PackItem);
constexpr size_t kCksOff = kChunkOff + size_t(kNoallocMaxChunks) * sizeof(PackChunk);
static_assert(kCksOff + size_t(kNoallocMaxPackages) * 8 <= kNoallocScratchBytes, "scratch layout exceeds the array");
static_assert(sizeof(PackItem) % 16 == 0 || sizeof(PackItem) % 8 == 0, "table alignment");

std::mutex g_mu;
unsigned char* g_addr[64] = {nullptr};  // device address of the array, per device ordinal

// Host code may not use the array's name as a device address; resolve it
// once per device, with that device current.
unsigned char* scratch_address() {
    int dev = 0;
    GBD_CHECK_CUDA(cudaGetDevice(&dev));
    GBD_REQUIRE(dev >= 0 && dev < 64, GBD_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        GBD_CHECK_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_addr[dev] = reinterpret_cast<unsigned char*>(p);
    }
    return g_addr[dev];
}

}  // namespace

}  // namespace gbd

using namespace gbd;

extern "C" int gbd_pack_noalloc(int side, int length, const double* arena, int ncls, const int* class_meta, int nblk,
                                const int* block_meta, void* dst, size_t cap, size_t* bytes, void* stream) {
    try {
        GBD_REQUIRE(ncls >= 0 && nblk >= 0 && (ncls == 0 || class_meta) && (nblk == 0 || block_meta), GBD_ERR_ARG,
                    "bad environment metadata");
        GBD_REQUIRE(side == 0 || side == 1, GBD_ERR_ARG, "side must be 0 or 1");
        GBD_REQUIRE(nblk <= kNoallocMaxPackages, GBD_ERR_ARG,
                    "too many blocks for the allocation-free pack (maximum 32768 packages)");
        // canonical layout: blocks class-major, each padded to an even count
        std::vector<long long> aoff(nblk);
        std::vector<size_t> pkg(nblk);
        long long a = 0;
        size_t total = 0;
        long long nchunks = 0;
        int prev = -1;
        for (int j = 0; j < nblk; ++j) {
            const int* m = block_meta + 7 * j;
            GBD_REQUIRE(m[0] >= 0 && m[0] < ncls && m[0] >= prev && m[5] >= 0 && m[6] >= 0, GBD_ERR_ARG,
                        "blocks must be class-major with valid dims");
            prev = m[0];
            const long long layers = class_meta[3 * m[0] + 2];
            GBD_REQUIRE(layers >= 1, GBD_ERR_ARG, "class needs >= 1 layer");
            const long long n = layers * m[5] * m[6];
            aoff[j] = a;
            a += (n + 1) / 2 * 2;
            pkg[j] = total;
            const size_t payload = (size_t(n) * 8 + 15) / 16 * 16;
            total += 64 + payload;
            nchunks += (long long)((payload / 8 + 8191) / 8192);
        }
        if (bytes) *bytes = total;
        GBD_REQUIRE(nchunks <= kNoallocMaxChunks, GBD_ERR_ARG,
                    "environment too large for the allocation-free pack (maximum 65536 chunks of 64 KB)");
        GBD_REQUIRE(dst && cap >= total, GBD_ERR_ARG, "destination too small (required size written to *bytes)");
        GBD_REQUIRE(nblk == 0 || arena, GBD_ERR_ARG, "null arena");
        if (nblk == 0) return GBD_OK;
        // the kernels move 16-byte vectors and run on the device: both
        // buffers must be 16-byte aligned memory the device can address
        GBD_REQUIRE((reinterpret_cast<uintptr_t>(arena) & 15) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0,
                    GBD_ERR_ARG, "arena and dst must be 16-byte aligned");
        for (const void* p : {static_cast<const void*>(arena), static_cast<const void*>(dst)}) {
            cudaPointerAttributes at{};
            const cudaError_t r = cudaPointerGetAttributes(&at, p);
            if (r != cudaSuccess) {
                cudaGetLastError();
                throw Error(GBD_ERR_ARG, "arena and dst must be device memory");
            }
            GBD_REQUIRE(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged, GBD_ERR_ARG,
                        "arena and dst must be device memory");
        }
        // headers and tables on the host, copied into the file-scope scratch
        std::vector<unsigned char> hdr(size_t(nblk) * 64, 0);
        std::vector<PackItem> items(nblk);
        std::vector<PackChunk> chunks;
        chunks.reserve(size_t(nchunks));
        for (int j = 0; j < nblk; ++j) {
            const int* m = block_meta + 7 * j;
            const uint32_t layers = uint32_t(class_meta[3 * m[0] + 2]);
            unsigned char* h = hdr.data() + size_t(j) * 64;
            auto put32 = [&](int off, uint32_t v) { std::memcpy(h + off, &v, 4); };
            auto put16 = [&](int off, int16_t v) { std::memcpy(h + off, &v, 2); };
            auto put64 = [&](int off, uint64_t v) { std::memcpy(h + off, &v, 8); };
            put32(0, 0x50444247u);
            uint16_t ver = 1;
            std::memcpy(h + 4, &ver, 2);
            h[6] = 1;
            h[7] = uint8_t(side);
            put32(8, uint32_t(length));
            put32(12, uint32_t(nblk));
            put32(16, uint32_t(j));
            put32(20, uint32_t(m[0]));
            put32(24, 0);
            put32(28, layers);
            put16(32, int16_t(m[1]));
            put16(34, int16_t(m[2]));
            put16(36, int16_t(m[3]));
            put16(38, int16_t(m[4]));
            put32(40, uint32_t(m[5]));
            put32(44, uint32_t(m[6]));
            put64(48, uint64_t(aoff[j]));
            put64(56, 0);
            const unsigned long long words = ((unsigned long long)layers * m[5] * m[6] * 8 + 15) / 16 * 2;
            items[j] = {arena + aoff[j], nullptr, (unsigned long long)pkg[j], words};
            for (unsigned long long w0 = 0; w0 < words; w0 += 8192)
                chunks.push_back({j, w0, std::min(words, w0 + 8192)});
        }
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        unsigned char* base = scratch_address();
        GBD_CHECK_CUDA(cudaMemcpyAsync(base + kHdrOff, hdr.data(), hdr.size(), cudaMemcpyHostToDevice, st));
        GBD_CHECK_CUDA(cudaMemcpyAsync(base + kItemOff, items.data(), items.size() * sizeof(PackItem),
                                       cudaMemcpyHostToDevice, st));
        if (!chunks.empty())
            GBD_CHECK_CUDA(cudaMemcpyAsync(base + kChunkOff, chunks.data(), chunks.size() * sizeof(PackChunk),
                                           cudaMemcpyHostToDevice, st));
        // pack_launch zeroes the checksum accumulators before it adds to them
        pack_launch(reinterpret_cast<unsigned char*>(dst), base + kHdrOff, reinterpret_cast<const PackItem*>(base + kItemOff),
                    nblk, reinterpret_cast<const PackChunk*>(base + kChunkOff), int(chunks.size()),
                    reinterpret_cast<unsigned long long*>(base + kCksOff), st);
        GBD_CHECK_CUDA(cudaStreamSynchronize(st));
        return GBD_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return GBD_ERR_CUDA;
    }
}
