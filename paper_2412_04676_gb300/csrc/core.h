// core.h -- shared host types of the GB300 two-site DMRG library.
//
// Quantum numbers, bond sector lists, enlarged-block bases, block-sparse
// operator-set layout, error handling and device buffers.  Sector and
// operator layouts follow Sec. II.B / Fig. 4a of arXiv:2412.04676: dense
// sector blocks of a quantum-number block-sparse matrix, with operators that
// share one block structure stacked as layers.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/gbdmrg.h"

namespace gbd {

struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define GBD_CHECK_CUDA(x)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (x);                                                               \
        if (e_ != cudaSuccess) {                                                            \
            int code_ = (e_ == cudaErrorMemoryAllocation) ? GBD_ERR_DEVICE_OOM : GBD_ERR_CUDA; \
            throw ::gbd::Error(code_, std::string(#x) + ": " + cudaGetErrorString(e_));     \
        }                                                                                   \
    } while (0)

// Device allocation failure with the size asked for and the device's free memory.
[[noreturn]] void throw_device_oom(size_t bytes, const char* what);

#define GBD_REQUIRE(cond, code, msg)                                   \
    do {                                                               \
        if (!(cond)) throw ::gbd::Error((code), std::string(msg));     \
    } while (0)

// ---------------------------------------------------------------- quantum numbers
struct Q {
    int n = 0, t = 0;
    bool operator<(const Q& o) const { return n < o.n || (n == o.n && t < o.t); }
    bool operator==(const Q& o) const { return n == o.n && t == o.t; }
    bool operator!=(const Q& o) const { return !(*this == o); }
    Q operator+(const Q& o) const { return {n + o.n, t + o.t}; }
    Q operator-(const Q& o) const { return {n - o.n, t - o.t}; }
};

// (n, tsz) of the local states |0>, |up>, |dn>, |updn>
static const Q kQS[4] = {{0, 0}, {1, 1}, {1, -1}, {2, 0}};

// Sectors of one bond, ascending (n, tsz).
struct Bond {
    std::vector<Q> q;
    std::vector<int> dim;
    int find(const Q& x) const {
        auto it = std::lower_bound(q.begin(), q.end(), x);
        if (it == q.end() || *it != x) return -1;
        return int(it - q.begin());
    }
    int dim_of(const Q& x) const {
        int i = find(x);
        return i < 0 ? 0 : dim[i];
    }
    long long total() const {
        long long s = 0;
        for (int d : dim) s += d;
        return s;
    }
    void add(const Q& x, int d) {  // keeps order
        auto it = std::lower_bound(q.begin(), q.end(), x);
        size_t i = it - q.begin();
        if (it != q.end() && *it == x) {
            dim[i] += d;
            return;
        }
        q.insert(it, x);
        dim.insert(dim.begin() + i, d);
    }
};

// One local-state segment of an enlarged-block sector.
struct Seg {
    int s;     // local state of the added orbital
    int bq;    // index of the sector in the underlying bond
    int off;   // first row of the segment inside the enlarged sector
    int size;  // rows
};

// Basis of an enlarged block: (bond at cut b) + orbital b on the left, or
// orbital b+1 + (bond at cut b+2) on the right, labelled from the left.
struct EBasis {
    std::vector<Q> q;
    std::vector<int> dim;
    std::vector<std::vector<Seg>> segs;
    int find(const Q& x) const {
        auto it = std::lower_bound(q.begin(), q.end(), x);
        if (it == q.end() || *it != x) return -1;
        return int(it - q.begin());
    }
};

EBasis left_enlarged(const Bond& b);    // Q = q + q_s
EBasis right_enlarged(const Bond& b1);  // Q = q - q_s

// ------------------------------------------------------------- operator sets
// A block-sparse operator set (Fig. 4a): layers (MPO states) that share one
// quantum-number change dq form a class; every block of a class stores all
// its layers contiguously, [layer][rows][cols] row-major.  Blocks are padded
// to an even number of doubles so every block starts 16-byte aligned.
struct OpBlock {
    int qo, qi;          // sector indices in the basis (output, input)
    int rows, cols;
    long long off;       // element offset in the arena
    Q Qo, Qi;            // the sectors' quantum numbers
};

struct OpClass {
    Q dq;
    std::vector<int> states;     // MPO state index at the cut, per layer
    std::vector<OpBlock> blocks; // ascending qi
    int find_block(int qi) const {
        for (size_t i = 0; i < blocks.size(); ++i)
            if (blocks[i].qi == qi) return int(i);
        return -1;
    }
};

// Cache of device blocks for the large per-position buffers (enlarged
// operator arenas, tensor-core slice planes): every position allocates blocks
// of similar sizes, and cudaFree synchronises the device and unmaps memory.
// A released block keeps an event recorded on the stream that used it; the
// next user's stream waits for that event, so reuse needs no host wait.
void* devcache_get(size_t n, cudaStream_t st, size_t* got);
void devcache_put(void* p, size_t bytes, cudaStream_t st);  // never throws
void devcache_trim();                                        // cudaFree every cached block
size_t devcache_bytes();                                     // bytes held in cached blocks

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaStream_t cst = nullptr;  // stream of a cached block's users
    bool cached = false;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes), cst(o.cst), cached(o.cached) {
        o.p = nullptr; o.bytes = 0; o.cst = nullptr; o.cached = false;
    }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p; bytes = o.bytes; cst = o.cst; cached = o.cached;
            o.p = nullptr; o.bytes = 0; o.cst = nullptr; o.cached = false;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void release() {
        if (p) {
            if (cached) devcache_put(p, bytes, cst);
            else cudaFree(p);
        }
        p = nullptr;
        bytes = 0;
        cst = nullptr;
        cached = false;
    }
    void ensure(size_t n) {  // grow-only, contents not kept
        if (n <= bytes && p) return;
        release();
        if (n == 0) n = 16;
        if (cudaMalloc(&p, n) != cudaSuccess) {  // blocks held by the cache go back first
            cudaGetLastError();
            p = nullptr;
            devcache_trim();
            if (cudaMalloc(&p, n) != cudaSuccess) {
                cudaGetLastError();
                p = nullptr;
                throw_device_oom(n, "cudaMalloc");
            }
        }
        bytes = n;
    }
    // grow-only from the block cache; the block is used on stream st
    void ensure_cached(size_t n, cudaStream_t st) {
        if (n <= bytes && p && cached && cst == st) return;
        release();
        if (n == 0) n = 16;
        p = devcache_get(n, st, &bytes);
        cached = true;
        cst = st;
    }
    // stream-ordered allocation / release (cudaMallocAsync pool)
    void alloc_async(size_t n, cudaStream_t st) {
        release();
        if (n == 0) n = 16;
        if (cudaMallocAsync(&p, n, st) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            devcache_trim();
            if (cudaMallocAsync(&p, n, st) != cudaSuccess) {
                cudaGetLastError();
                p = nullptr;
                throw_device_oom(n, "cudaMallocAsync");
            }
        }
        bytes = n;
    }
    void release_async(cudaStream_t st) {
        if (p) {
            if (cached) devcache_put(p, bytes, cst);
            else cudaFreeAsync(p, st);
        }
        p = nullptr;
        bytes = 0;
        cst = nullptr;
        cached = false;
    }
    template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

struct OpSet {
    int side = 0;            // 0 left, 1 right
    int cut = 0;             // cut index of the MPO states
    std::vector<OpClass> cls;
    long long total = 0;     // arena elements
    DevBuf data;             // device arena (double)
    std::vector<int> state_class, state_layer;  // per MPO state at the cut
    bool resident() const { return data.p != nullptr; }
    int find_class(const Q& dq) const {
        for (size_t i = 0; i < cls.size(); ++i)
            if (cls[i].dq == dq) return int(i);
        return -1;
    }
    void layout() {  // assigns block offsets in canonical order
        long long off = 0;
        for (auto& c : cls)
            for (auto& b : c.blocks) {
                b.off = off;
                long long n = (long long)c.states.size() * b.rows * b.cols;
                off += (n + 1) / 2 * 2;
            }
        total = off;
    }
};

inline long long pad2(long long n) { return (n + 1) / 2 * 2; }

}  // namespace gbd
