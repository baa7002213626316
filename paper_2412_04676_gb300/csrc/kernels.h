// kernels.h -- launchers of the library's own CUDA kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace gbd {

// ------------------------------------------------------------------ grouped GEMM
// One reduction segment: sum_{t<T} coef * op(A + t sA) op(B + t sB), K inner.
// op(A) is M x K: A[m*lda + k] (transA = 0) or A[k*lda + m] (transA = 1).
// op(B) is K x N: B[k*ldb + n] (transB = 0) or B[n*ldb + k] (transB = 1).
struct GemmSeg {
    const double* A;
    const double* B;
    long long lda, ldb, sA, sB;
    int K, T, transA, transB;
    double coef;
};

// C (M x N) = sum over the task's segments + beta * C, for nbatch independent
// items (A, B, C advanced by bA, bB, bC per item).  Output column n maps to
// C[m*ldc + (n / ncols) * ldr + n % ncols] so a strided 3-D region can be
// written as one matrix.
struct GemmTask {
    double* C;
    long long ldc, ldr, bA, bB, bC;
    int M, N, ncols;
    int seg0, nseg, nbatch;
    double beta;
};

struct GemmTile {
    int task, batch, m0, n0;
};

// Device-resident task list.  upload() copies host vectors to the device
// (reusing its buffers); launch() runs all tiles on `stream`.
struct GemmPlan {
    std::vector<GemmTask> tasks;
    std::vector<GemmSeg> segs;
    std::vector<GemmTile> tiles;
    void* d_tasks = nullptr;
    void* d_segs = nullptr;
    void* d_tiles = nullptr;
    size_t cap_tasks = 0, cap_segs = 0, cap_tiles = 0;
    cudaStream_t st_last = nullptr;  // stream of the last upload (the tables' users)
    double flops = 0.0;  // 2*M*N*K summed (useful)
    void clear() { tasks.clear(); segs.clear(); tiles.clear(); task_tile0.clear(); flops = 0.0; }
    void add_task(GemmTask t, const std::vector<GemmSeg>& s);
    void upload(cudaStream_t st);
    void launch(cudaStream_t st) const;
    // the same tiles, one launch per task (comparison against batching)
    void launch_per_task(cudaStream_t st) const;
    std::vector<int> task_tile0;  // first tile of each task
    // Host-side check, before any launch, that every address a task reads or
    // writes lies inside one of the given buffers (base, bytes).
    void check(const std::vector<std::pair<const void*, size_t>>& bufs, const char* what) const;
    void free();
    GemmPlan() = default;
    GemmPlan(const GemmPlan&) = delete;
    GemmPlan& operator=(const GemmPlan&) = delete;
    GemmPlan(GemmPlan&& o) noexcept { take(o); }
    GemmPlan& operator=(GemmPlan&& o) noexcept {
        if (this != &o) { free(); take(o); }
        return *this;
    }
    ~GemmPlan() { free(); }

  private:
    void take(GemmPlan& o) {
        tasks = std::move(o.tasks);
        segs = std::move(o.segs);
        tiles = std::move(o.tiles);
        task_tile0 = std::move(o.task_tile0);
        d_tasks = o.d_tasks; d_segs = o.d_segs; d_tiles = o.d_tiles;
        cap_tasks = o.cap_tasks; cap_segs = o.cap_segs; cap_tiles = o.cap_tiles;
        st_last = o.st_last;
        flops = o.flops;
        o.d_tasks = o.d_segs = o.d_tiles = nullptr;
        o.cap_tasks = o.cap_segs = o.cap_tiles = 0;
        o.st_last = nullptr;
    }
};

// ------------------------------------------------------------------ vectors
// out[i] = V_i . x (i < k, V_i = V + i*ldv), deterministic two-stage reduction.
void multi_dot(const double* V, long long ldv, int k, const double* x, long long n, double* out,
               double* partial, cudaStream_t st);
// y = beta*y + alpha * sum_i c[i] V_i  (c on the device)
void combine(const double* V, long long ldv, int k, const double* c, double* y, long long n, double alpha,
             double beta, cudaStream_t st);
// t = -r / (diag - theta), |diag - theta| floored at 1e-12
void precondition(const double* r, const double* diag, double theta, double* t, long long n, cudaStream_t st);
void axpby(const double* x, double* y, long long n, double a, double b, cudaStream_t st);  // y = a x + b y
void scale(double* x, long long n, double a, cudaStream_t st);
size_t multi_dot_partial_elems(int k);

// ------------------------------------------------------------------ H_eff diagonal
// diag[Q][i][k] = sum over (segments) sum_t OL[t][i][i] * OR[t][k][k]
struct DiagSeg {
    const double* OL;  // [T][mL][mL]
    const double* OR;  // [T][mR][mR]
    int T;
};
struct DiagTask {
    double* out;  // mL x mR
    int mL, mR, seg0, nseg;
};
void heff_diagonal(const std::vector<DiagTask>& tasks, const std::vector<DiagSeg>& segs, cudaStream_t st);

// ------------------------------------------------------------------ pack / unpack
// One package of the serialised stream: a 64-byte header then the payload.
struct PackItem {
    const double* src;          // pack: arena block (device); unpack: unused
    double* dst_arena;          // unpack: arena block (device); pack: unused
    unsigned long long pkg;     // byte offset of the package in the stream
    unsigned long long words;   // payload u64 words (padded to 16 bytes)
};
struct PackChunk {
    int item;
    unsigned long long w0, w1;  // word range [w0, w1) of the payload
};
// Writes headers (host-built, 64 bytes each, checksum 0; skipped when
// d_headers is null because the caller already placed them) and payloads
// into `stream_base` (device or mapped pinned host memory), then the
// checksums.  All metadata pointers must be readable by the device.
void pack_launch(unsigned char* stream_base, const unsigned char* d_headers, const PackItem* d_items, int n_items,
                 const PackChunk* d_chunks, int n_chunks, unsigned long long* d_cks, cudaStream_t st);
// Copies payloads from `stream_base` to their arena blocks and accumulates
// each package's checksum into d_cks (zeroed by the caller).
void unpack_launch(const unsigned char* stream_base, const PackItem* d_items, const PackChunk* d_chunks,
                   int n_chunks, unsigned long long* d_cks, cudaStream_t st);

// ------------------------------------------------------------------ scaled copies
// Enlargement pass-through links (Sec. II.B step 1): output layer c of a
// sub-block (rows x cols, row stride ldr, layer stride out_pitch) +=
// sum over the sub-block's links l of sum_(a, coef) in cols(l, c) of
// coef * input layer a of l's input block (contiguous rows x cols, layer
// stride in_pitch).  cols(l, c) depends on the link only, so it is stored
// once per link and shared by every sub-block the link feeds.
struct CopyCoef {
    int a;           // input layer
    double coef;
};
struct CopyCol {
    int c0, n;       // CopyCoef range of one (link, output layer)
};
struct CopyLink {
    const double* src;   // input block, layer 0
    long long in_pitch;  // elements between input layers
    int col0;            // CopyCol index of output layer 0 of this link
};
struct CopyItem {
    double* dst;          // output sub-block, layer 0
    long long out_pitch;  // elements between output layers
    long long ldr;
    int rows, cols, tout; // sub-block shape, output layers
    int link0, nlink;     // CopyLink range
    int overwrite;        // 1: no GEMM writes this sub-block, so the copy-sum stores (the
                          // arena is zero-filled) instead of adding to what is there
};
// grid: (items, ceil(max tout / kCopyLayers)); each (item, layer) has one writer
constexpr int kCopyLayers = 8;
void copy_sum(const CopyItem* d_items, int n_items, int max_tout, const CopyLink* d_links, const CopyCol* d_cols,
              const CopyCoef* d_coefs, cudaStream_t st);

// ------------------------------------------------------------------ padded slots
// Writes value on the diagonal entries m..n-1 of the column-major n x n slot
// at p (the rest of the slot is set by the caller).
struct PadSeg {
    double* p;
    int n, m;
};
void pad_identity(const std::vector<PadSeg>& segs, double value, cudaStream_t st);

// ------------------------------------------------------------------ misc
// Count of this library's kernel launches (incremented by every launcher).
unsigned long long launch_count();
void count_launch(unsigned n = 1);
void fill_zero(double* p, long long n, cudaStream_t st);

}  // namespace gbd
