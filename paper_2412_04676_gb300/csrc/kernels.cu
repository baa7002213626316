// kernels.cu -- FP64 grouped GEMM, Davidson vector kernels, H_eff diagonal and
// the pack/unpack (serialise/deserialise) kernels of the GB300 DMRG library.
//
// The grouped GEMM is the FP64 ("plain") engine behind every block product
// of Sec. II.B: H_eff psi, environment enlargement and renormalisation.  It
// runs one launch over a host-built tile list; a task may sum many
// segments (a long K split over operator layers and sector pairs) into one
// output, so no output is written by two tiles and no atomics are needed.
//
// The pack kernel is the single-GPU form of the parallel serialiser of
// Sec. III.B.2: every package's byte offset is known before the launch
// (exclusive prefix sum of exactly predicted sizes), every CTA copies one
// 64 KB chunk with 16-byte loads and stores, independently of all others,
// and the checksum of each self-contained package (Sec. III.B.3) is an
// order-free sum so chunks never talk to each other.
#include "core.h"
#include "kernels.h"

#include <atomic>
#include <cstdio>
#include <iterator>
#include <map>
#include <mutex>

namespace gbd {

static std::atomic<unsigned long long> g_launches{0};
unsigned long long launch_count() { return g_launches.load(); }
void count_launch(unsigned n) { g_launches += n; }

// ============================================================== grouped GEMM
namespace {
// 32 x 32 CTA tiles of eight warps; each warp owns a 16 x 8 sub-tile (two
// rows x two columns per lane) and skips the FMA loop when its sub-tile lies
// outside the task, and the K loop stops at the task's true K.  GB300's FP64
// pipe retires about 2 FMA/clk/SM, so padded FMAs cost as much as useful ones.
constexpr int BM = 32, BN = 32, BK = 16, NT = 256;

__global__ void __launch_bounds__(NT) gemm_f64_kernel(const GemmTask* __restrict__ tasks,
                                                      const GemmSeg* __restrict__ segs,
                                                      const GemmTile* __restrict__ tiles) {
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const GemmTile tl = tiles[blockIdx.x];
    const GemmTask tk = tasks[tl.task];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wr = (warp >> 2) * 16, wc = (warp & 3) * 8;   // warp sub-tile origin
    const int lr = lane >> 2, lc = lane & 3;                // lane: rows lr, lr+8; cols lc, lc+4
    const bool active = (tl.m0 + wr < tk.M) && (tl.n0 + wc < tk.N);
    double acc00 = 0.0, acc01 = 0.0, acc10 = 0.0, acc11 = 0.0;

    for (int s = tk.seg0; s < tk.seg0 + tk.nseg; ++s) {
        const GemmSeg sg = segs[s];
        const double* A0 = sg.A + (long long)tl.batch * tk.bA;
        const double* B0 = sg.B + (long long)tl.batch * tk.bB;
        for (int t = 0; t < sg.T; ++t) {
            const double* A = A0 + (long long)t * sg.sA;
            const double* B = B0 + (long long)t * sg.sB;
            for (int k0 = 0; k0 < sg.K; k0 += BK) {
#pragma unroll
                for (int r = 0; r < (BM * BK) / NT; ++r) {
                    int idx = threadIdx.x + r * NT;
                    int m, k;
                    if (sg.transA) { k = idx / BM; m = idx % BM; }
                    else { m = idx / BK; k = idx % BK; }
                    int gm = tl.m0 + m, gk = k0 + k;
                    double v = 0.0;
                    if (gm < tk.M && gk < sg.K)
                        v = sg.transA ? A[(long long)gk * sg.lda + gm] : A[(long long)gm * sg.lda + gk];
                    As[k][m] = v * sg.coef;
                }
#pragma unroll
                for (int r = 0; r < (BN * BK) / NT; ++r) {
                    int idx = threadIdx.x + r * NT;
                    int n, k;
                    if (sg.transB) { n = idx / BK; k = idx % BK; }
                    else { k = idx / BN; n = idx % BN; }
                    int gn = tl.n0 + n, gk = k0 + k;
                    double v = 0.0;
                    if (gn < tk.N && gk < sg.K)
                        v = sg.transB ? B[(long long)gn * sg.ldb + gk] : B[(long long)gk * sg.ldb + gn];
                    Bs[k][n] = v;
                }
                __syncthreads();
                if (active) {
                    const int kend = min(BK, sg.K - k0);
                    for (int kk = 0; kk < kend; ++kk) {
                        const double a0 = As[kk][wr + lr], a1 = As[kk][wr + lr + 8];
                        const double b0 = Bs[kk][wc + lc], b1 = Bs[kk][wc + lc + 4];
                        acc00 = fma(a0, b0, acc00);
                        acc01 = fma(a0, b1, acc01);
                        acc10 = fma(a1, b0, acc10);
                        acc11 = fma(a1, b1, acc11);
                    }
                }
                __syncthreads();
            }
        }
    }
    if (!active) return;
    double* C = tk.C + (long long)tl.batch * tk.bC;
    auto store = [&](int m, int n, double v) {
        if (m >= tk.M || n >= tk.N) return;
        long long off = (long long)m * tk.ldc + (long long)(n / tk.ncols) * tk.ldr + (n % tk.ncols);
        if (tk.beta != 0.0) v += tk.beta * C[off];
        C[off] = v;
    };
    const int m0 = tl.m0 + wr + lr, n0 = tl.n0 + wc + lc;
    store(m0, n0, acc00);
    store(m0, n0 + 4, acc01);
    store(m0 + 8, n0, acc10);
    store(m0 + 8, n0 + 4, acc11);
}

template <class T>
void upload_vec(const std::vector<T>& v, void*& d, size_t& cap, cudaStream_t st) {
    // grow-only device table from the block cache (the plan is launched on st)
    size_t bytes = v.size() * sizeof(T);
    if (bytes == 0) return;
    if (bytes > cap) {
        const size_t nb = std::max(bytes, cap * 2);
        if (d) devcache_put(d, cap, st);
        d = devcache_get(nb, st, &cap);
    }
    GBD_CHECK_CUDA(cudaMemcpyAsync(d, v.data(), bytes, cudaMemcpyHostToDevice, st));
}
}  // namespace

void GemmPlan::add_task(GemmTask t, const std::vector<GemmSeg>& s) {
    if (t.M <= 0 || t.N <= 0 || t.nbatch <= 0) return;
    t.seg0 = int(segs.size());
    t.nseg = 0;
    for (const auto& x : s) {
        if (x.K <= 0 || x.T <= 0) continue;
        segs.push_back(x);
        ++t.nseg;
        flops += 2.0 * t.M * double(t.N) * x.K * x.T * t.nbatch;
    }
    if (t.ncols <= 0) t.ncols = t.N;
    if (t.nseg == 0 && t.beta != 0.0) return;  // nothing to add, C unchanged
    int id = int(tasks.size());
    tasks.push_back(t);
    task_tile0.push_back(int(tiles.size()));
    for (int b = 0; b < t.nbatch; ++b)
        for (int m0 = 0; m0 < t.M; m0 += BM)
            for (int n0 = 0; n0 < t.N; n0 += BN) tiles.push_back({id, b, m0, n0});
}

namespace {
bool inside(const std::vector<std::pair<const void*, size_t>>& bufs, const double* p, long long max_off) {
    if (max_off < 0) return true;
    const char* a = reinterpret_cast<const char*>(p);
    const char* e = reinterpret_cast<const char*>(p + max_off + 1);
    for (const auto& b : bufs) {
        const char* lo = reinterpret_cast<const char*>(b.first);
        if (a >= lo && e <= lo + b.second) return true;
    }
    return false;
}
}  // namespace

void GemmPlan::check(const std::vector<std::pair<const void*, size_t>>& bufs, const char* what) const {
    for (size_t ti = 0; ti < tasks.size(); ++ti) {
        const GemmTask& t = tasks[ti];
        long long cmax = (long long)(t.M - 1) * t.ldc + (long long)((t.N - 1) / t.ncols) * t.ldr +
                         std::min(t.N, t.ncols) - 1 + (long long)(t.nbatch - 1) * t.bC;
        if (!inside(bufs, t.C, cmax))
            throw Error(GBD_ERR_STATE, std::string(what) + ": task output outside its buffer (task " + std::to_string(ti) + ")");
        for (int si = t.seg0; si < t.seg0 + t.nseg; ++si) {
            const GemmSeg& g = segs[si];
            long long amax = (g.transA ? (long long)(g.K - 1) * g.lda + (t.M - 1) : (long long)(t.M - 1) * g.lda + (g.K - 1)) +
                             (long long)(g.T - 1) * g.sA + (long long)(t.nbatch - 1) * t.bA;
            long long bmax = (g.transB ? (long long)(t.N - 1) * g.ldb + (g.K - 1) : (long long)(g.K - 1) * g.ldb + (t.N - 1)) +
                             (long long)(g.T - 1) * g.sB + (long long)(t.nbatch - 1) * t.bB;
            if (!inside(bufs, g.A, amax))
                throw Error(GBD_ERR_STATE, std::string(what) + ": operand A outside its buffer (task " + std::to_string(ti) + ")");
            if (!inside(bufs, g.B, bmax))
                throw Error(GBD_ERR_STATE, std::string(what) + ": operand B outside its buffer (task " + std::to_string(ti) + ")");
        }
    }
}

void GemmPlan::upload(cudaStream_t st) {
    if (st_last && st_last != st) free();  // the tables' users move to another stream
    st_last = st;
    upload_vec(tasks, d_tasks, cap_tasks, st);
    upload_vec(segs, d_segs, cap_segs, st);
    upload_vec(tiles, d_tiles, cap_tiles, st);
}

void GemmPlan::launch(cudaStream_t st) const {
    if (tiles.empty()) return;
    size_t n = tiles.size();
    const size_t maxgrid = 0x7FFFFFFF;
    GBD_REQUIRE(n <= maxgrid, GBD_ERR_ARG, "too many GEMM tiles");
    gemm_f64_kernel<<<unsigned(n), NT, 0, st>>>((const GemmTask*)d_tasks, (const GemmSeg*)d_segs,
                                                (const GemmTile*)d_tiles);
    count_launch();
    GBD_CHECK_CUDA(cudaGetLastError());
}

void GemmPlan::launch_per_task(cudaStream_t st) const {
    for (size_t k = 0; k < task_tile0.size(); ++k) {
        const int t0 = task_tile0[k];
        const int t1 = k + 1 < task_tile0.size() ? task_tile0[k + 1] : int(tiles.size());
        if (t1 <= t0) continue;
        gemm_f64_kernel<<<unsigned(t1 - t0), NT, 0, st>>>((const GemmTask*)d_tasks, (const GemmSeg*)d_segs,
                                                          (const GemmTile*)d_tiles + t0);
        count_launch();
    }
    GBD_CHECK_CUDA(cudaGetLastError());
}

void GemmPlan::free() {
    auto rel = [&](void* d, size_t cap) {
        if (!d) return;
        if (st_last) devcache_put(d, cap, st_last);
        else cudaFree(d);
    };
    rel(d_tasks, cap_tasks);
    rel(d_segs, cap_segs);
    rel(d_tiles, cap_tiles);
    d_tasks = d_segs = d_tiles = nullptr;
    cap_tasks = cap_segs = cap_tiles = 0;
}

// ============================================================== vectors
namespace {
constexpr int VT = 256;
constexpr int DOT_BLOCKS = 304;  // 2 per SM on 152 SMs
constexpr int MAXK = 40;

__global__ void __launch_bounds__(VT) multi_dot_partial_kernel(const double* __restrict__ V, long long ldv, int k,
                                                               const double* __restrict__ x, long long n,
                                                               double* __restrict__ partial) {
    __shared__ double red[VT / 32][MAXK];
    double acc[MAXK];
    for (int i = 0; i < k; ++i) acc[i] = 0.0;
    for (long long j = blockIdx.x * (long long)VT + threadIdx.x; j < n; j += (long long)gridDim.x * VT) {
        double xv = x[j];
        for (int i = 0; i < k; ++i) acc[i] = fma(V[i * ldv + j], xv, acc[i]);
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = 0; i < k; ++i) {
        double v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[w][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < k) {
        double v = 0.0;
        for (int ww = 0; ww < VT / 32; ++ww) v += red[ww][threadIdx.x];
        partial[(long long)blockIdx.x * k + threadIdx.x] = v;
    }
}

__global__ void multi_dot_final_kernel(const double* __restrict__ partial, int nb, int k, double* __restrict__ out) {
    int i = threadIdx.x;
    if (i >= k) return;
    double v = 0.0;
    for (int b = 0; b < nb; ++b) v += partial[(long long)b * k + i];
    out[i] = v;
}

__global__ void combine_kernel(const double* __restrict__ V, long long ldv, int k, const double* __restrict__ c,
                               double* __restrict__ y, long long n, double alpha, double beta) {
    __shared__ double cs[MAXK];
    if (threadIdx.x < k) cs[threadIdx.x] = c[threadIdx.x];
    __syncthreads();
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < k; ++i) s = fma(cs[i], V[i * ldv + j], s);
        y[j] = (beta == 0.0 ? 0.0 : beta * y[j]) + alpha * s;
    }
}

__global__ void precond_kernel(const double* __restrict__ r, const double* __restrict__ d, double theta,
                               double* __restrict__ t, long long n) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        double den = d[j] - theta;
        if (fabs(den) < 1e-12) den = den < 0 ? -1e-12 : 1e-12;
        t[j] = -r[j] / den;
    }
}

__global__ void axpby_kernel(const double* __restrict__ x, double* __restrict__ y, long long n, double a, double b) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
        y[j] = a * x[j] + (b == 0.0 ? 0.0 : b * y[j]);
}

__global__ void scale_kernel(double* __restrict__ x, long long n, double a) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
        x[j] *= a;
}

__global__ void zero_kernel(double* __restrict__ x, long long n) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
        x[j] = 0.0;
}

inline unsigned grid_for(long long n) {
    long long g = (n + VT - 1) / VT;
    if (g > 152 * 8) g = 152 * 8;
    if (g < 1) g = 1;
    return unsigned(g);
}
}  // namespace

size_t multi_dot_partial_elems(int k) { return size_t(DOT_BLOCKS) * k; }

void multi_dot(const double* V, long long ldv, int k, const double* x, long long n, double* out, double* partial,
               cudaStream_t st) {
    GBD_REQUIRE(k >= 1 && k <= MAXK, GBD_ERR_ARG, "multi_dot: k out of range");
    multi_dot_partial_kernel<<<DOT_BLOCKS, VT, 0, st>>>(V, ldv, k, x, n, partial);
    multi_dot_final_kernel<<<1, 64, 0, st>>>(partial, DOT_BLOCKS, k, out);
    count_launch(2);
    GBD_CHECK_CUDA(cudaGetLastError());
}

void combine(const double* V, long long ldv, int k, const double* c, double* y, long long n, double alpha,
             double beta, cudaStream_t st) {
    GBD_REQUIRE(k >= 1 && k <= MAXK, GBD_ERR_ARG, "combine: k out of range");
    combine_kernel<<<grid_for(n), VT, 0, st>>>(V, ldv, k, c, y, n, alpha, beta);
    count_launch();
    GBD_CHECK_CUDA(cudaGetLastError());
}

void precondition(const double* r, const double* diag, double theta, double* t, long long n, cudaStream_t st) {
    precond_kernel<<<grid_for(n), VT, 0, st>>>(r, diag, theta, t, n);
    count_launch();
    GBD_CHECK_CUDA(cudaGetLastError());
}

void axpby(const double* x, double* y, long long n, double a, double b, cudaStream_t st) {
    axpby_kernel<<<grid_for(n), VT, 0, st>>>(x, y, n, a, b);
    count_launch();
    GBD_CHECK_CUDA(cudaGetLastError());
}

void scale(double* x, long long n, double a, cudaStream_t st) {
    scale_kernel<<<grid_for(n), VT, 0, st>>>(x, n, a);
    count_launch();
    GBD_CHECK_CUDA(cudaGetLastError());
}

void fill_zero(double* p, long long n, cudaStream_t st) {
    if (n <= 0) return;
    zero_kernel<<<grid_for(n), VT, 0, st>>>(p, n);
    count_launch();
    GBD_CHECK_CUDA(cudaGetLastError());
}

// ============================================================== scaled copies
namespace {
__global__ void copy_sum_kernel(const CopyItem* __restrict__ items, const CopyLink* __restrict__ links,
                                const CopyCol* __restrict__ cols, const CopyCoef* __restrict__ coefs) {
    const CopyItem it = items[blockIdx.x];
    const int n = it.rows * it.cols;
    const int c_end = min(it.tout, int(blockIdx.y + 1) * kCopyLayers);
    for (int c = blockIdx.y * kCopyLayers; c < c_end; ++c) {
        double* dst = it.dst + (long long)c * it.out_pitch;
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            double v = 0.0;
            bool any = false;
            for (int l = it.link0; l < it.link0 + it.nlink; ++l) {
                const CopyLink L = links[l];
                const CopyCol col = cols[L.col0 + c];
                for (int k = col.c0; k < col.c0 + col.n; ++k) {
                    v = fma(coefs[k].coef, L.src[(long long)coefs[k].a * L.in_pitch + e], v);
                    any = true;
                }
            }
            if (!any) continue;
            const int r = e / it.cols, cc = e - r * it.cols;
            double* o = dst + (long long)r * it.ldr + cc;
            if (it.overwrite) *o = v;  // no other writer: skip the read
            else *o += v;
        }
    }
}
}  // namespace

void copy_sum(const CopyItem* d_items, int n_items, int max_tout, const CopyLink* d_links, const CopyCol* d_cols,
              const CopyCoef* d_coefs, cudaStream_t st) {
    if (n_items <= 0 || max_tout <= 0) return;
    const unsigned gy = unsigned((max_tout + kCopyLayers - 1) / kCopyLayers);
    GBD_REQUIRE(gy <= 65535, GBD_ERR_ARG, "copy_sum: too many output layers");
    for (int i0 = 0; i0 < n_items; i0 += 0x7FFFFFF) {
        int n = std::min(n_items - i0, 0x7FFFFFF);
        copy_sum_kernel<<<dim3(n, gy), 128, 0, st>>>(d_items + i0, d_links, d_cols, d_coefs);
        count_launch();
    }
    GBD_CHECK_CUDA(cudaGetLastError());
}

// ============================================================== H_eff diagonal
namespace {
__global__ void diag_kernel(const DiagTask* __restrict__ tasks, const DiagSeg* __restrict__ segs) {
    const DiagTask tk = tasks[blockIdx.y];
    long long n = (long long)tk.mL * tk.mR;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        int i = int(e / tk.mR), k = int(e % tk.mR);
        double v = 0.0;
        for (int s = tk.seg0; s < tk.seg0 + tk.nseg; ++s) {
            const DiagSeg sg = segs[s];
            long long sl = (long long)tk.mL * tk.mL, sr = (long long)tk.mR * tk.mR;
            for (int t = 0; t < sg.T; ++t)
                v = fma(sg.OL[t * sl + (long long)i * tk.mL + i], sg.OR[t * sr + (long long)k * tk.mR + k], v);
        }
        tk.out[e] = v;
    }
}
}  // namespace

void heff_diagonal(const std::vector<DiagTask>& tasks, const std::vector<DiagSeg>& segs, cudaStream_t st) {
    if (tasks.empty()) return;
    DiagTask* dt = nullptr;
    DiagSeg* ds = nullptr;
    GBD_CHECK_CUDA(cudaMallocAsync(&dt, tasks.size() * sizeof(DiagTask), st));
    GBD_CHECK_CUDA(cudaMallocAsync(&ds, std::max<size_t>(1, segs.size()) * sizeof(DiagSeg), st));
    GBD_CHECK_CUDA(cudaMemcpyAsync(dt, tasks.data(), tasks.size() * sizeof(DiagTask), cudaMemcpyHostToDevice, st));
    if (!segs.empty())
        GBD_CHECK_CUDA(cudaMemcpyAsync(ds, segs.data(), segs.size() * sizeof(DiagSeg), cudaMemcpyHostToDevice, st));
    GBD_REQUIRE(tasks.size() < 65536, GBD_ERR_ARG, "too many diagonal tasks");
    dim3 grid(64, unsigned(tasks.size()));
    diag_kernel<<<grid, 256, 0, st>>>(dt, ds);
    count_launch();
    GBD_CHECK_CUDA(cudaGetLastError());
    GBD_CHECK_CUDA(cudaFreeAsync(dt, st));
    GBD_CHECK_CUDA(cudaFreeAsync(ds, st));
}

// ============================================================== pack / unpack
namespace {
constexpr int PT = 256;

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v) {
    __shared__ unsigned long long red[PT / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    unsigned long long s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < PT / 32; ++i) s += red[i];
    return s;  // valid in thread 0
}

__global__ void pack_headers_kernel(unsigned char* __restrict__ base, const unsigned char* __restrict__ headers,
                                    const PackItem* __restrict__ items, int n) {
    int i = blockIdx.x * 64 + (threadIdx.x >> 2);  // 4 threads x 16 bytes per header, 64 headers per block
    if (i >= n) return;
    int part = threadIdx.x & 3;
    const uint4* src = reinterpret_cast<const uint4*>(headers + (size_t)i * 64) + part;
    uint4* dst = reinterpret_cast<uint4*>(base + items[i].pkg) + part;
    *dst = *src;
}

// payload copy: word index w of package item; checksum term w_i * (2i + 1)
__global__ void __launch_bounds__(PT) pack_payload_kernel(unsigned char* __restrict__ base,
                                                          const PackItem* __restrict__ items,
                                                          const PackChunk* __restrict__ chunks,
                                                          unsigned long long* __restrict__ cks) {
    const PackChunk ch = chunks[blockIdx.x];
    const PackItem it = items[ch.item];
    const ulonglong2* src = reinterpret_cast<const ulonglong2*>(it.src);
    ulonglong2* dst = reinterpret_cast<ulonglong2*>(base + it.pkg + 64);
    unsigned long long s = 0;
    for (unsigned long long p = ch.w0 / 2 + threadIdx.x; p < ch.w1 / 2; p += PT) {
        ulonglong2 v = src[p];
        dst[p] = v;
        unsigned long long i0 = 2 * p;
        s += v.x * (2 * i0 + 1) + v.y * (2 * i0 + 3);
    }
    unsigned long long tot = block_sum_u64(s);
    if (threadIdx.x == 0) atomicAdd(cks + ch.item, tot);
}

__global__ void pack_checksums_kernel(unsigned char* __restrict__ base, const PackItem* __restrict__ items,
                                      const unsigned long long* __restrict__ cks, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    *reinterpret_cast<unsigned long long*>(base + items[i].pkg + 56) = cks[i];
}

__global__ void __launch_bounds__(PT) unpack_payload_kernel(const unsigned char* __restrict__ base,
                                                            const PackItem* __restrict__ items,
                                                            const PackChunk* __restrict__ chunks,
                                                            unsigned long long* __restrict__ cks) {
    const PackChunk ch = chunks[blockIdx.x];
    const PackItem it = items[ch.item];
    const ulonglong2* src = reinterpret_cast<const ulonglong2*>(base + it.pkg + 64);
    ulonglong2* dst = reinterpret_cast<ulonglong2*>(it.dst_arena);
    unsigned long long s = 0;
    for (unsigned long long p = ch.w0 / 2 + threadIdx.x; p < ch.w1 / 2; p += PT) {
        ulonglong2 v = src[p];
        dst[p] = v;
        unsigned long long i0 = 2 * p;
        s += v.x * (2 * i0 + 1) + v.y * (2 * i0 + 3);
    }
    unsigned long long tot = block_sum_u64(s);
    if (threadIdx.x == 0) atomicAdd(cks + ch.item, tot);
}
}  // namespace

void pack_launch(unsigned char* base, const unsigned char* d_headers, const PackItem* d_items, int n_items,
                 const PackChunk* d_chunks, int n_chunks, unsigned long long* d_cks, cudaStream_t st) {
    if (n_items == 0) return;
    GBD_CHECK_CUDA(cudaMemsetAsync(d_cks, 0, sizeof(unsigned long long) * n_items, st));
    if (d_headers) { pack_headers_kernel<<<(n_items + 63) / 64, 256, 0, st>>>(base, d_headers, d_items, n_items); count_launch(); }
    if (n_chunks > 0) { pack_payload_kernel<<<n_chunks, PT, 0, st>>>(base, d_items, d_chunks, d_cks); count_launch(); }
    pack_checksums_kernel<<<(n_items + 255) / 256, 256, 0, st>>>(base, d_items, d_cks, n_items);
    count_launch();
    GBD_CHECK_CUDA(cudaGetLastError());
}

void unpack_launch(const unsigned char* base, const PackItem* d_items, const PackChunk* d_chunks, int n_chunks,
                   unsigned long long* d_cks, cudaStream_t st) {
    if (n_chunks > 0) { unpack_payload_kernel<<<n_chunks, PT, 0, st>>>(base, d_items, d_chunks, d_cks); count_launch(); }
    GBD_CHECK_CUDA(cudaGetLastError());
}

// ============================================================== padded slots
namespace {
__global__ void pad_identity_kernel(const PadSeg* __restrict__ segs, int n, double value) {
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const PadSeg sg = segs[i];
        for (int d = sg.m + threadIdx.x; d < sg.n; d += blockDim.x) sg.p[(long long)d * sg.n + d] = value;
    }
}
}  // namespace

void pad_identity(const std::vector<PadSeg>& segs, double value, cudaStream_t st) {
    if (segs.empty()) return;
    PadSeg* d = nullptr;
    GBD_CHECK_CUDA(cudaMallocAsync(&d, segs.size() * sizeof(PadSeg), st));
    GBD_CHECK_CUDA(cudaMemcpyAsync(d, segs.data(), segs.size() * sizeof(PadSeg), cudaMemcpyHostToDevice, st));
    pad_identity_kernel<<<unsigned(std::min<size_t>(segs.size(), 4096)), 128, 0, st>>>(d, int(segs.size()), value);
    count_launch();
    GBD_CHECK_CUDA(cudaGetLastError());
    GBD_CHECK_CUDA(cudaFreeAsync(d, st));
}

// ============================================================== device block cache
namespace {
struct CacheBlock {
    void* p;
    size_t bytes;
    cudaEvent_t ev;
    int dev;
};
std::mutex g_cache_mu;
std::multimap<size_t, CacheBlock> g_cache;
size_t g_cache_bytes = 0;
constexpr size_t kCacheMax = size_t(96) << 30;  // cached bytes kept at most
}  // namespace

void* devcache_get(size_t n, cudaStream_t st, size_t* got) {
    int dev = 0;
    GBD_CHECK_CUDA(cudaGetDevice(&dev));
    {
        std::unique_lock<std::mutex> lk(g_cache_mu);
        // best fit within 1.5x of the request, on this device
        for (auto it = g_cache.lower_bound(n); it != g_cache.end() && it->first <= n + n / 2 + (size_t(1) << 20); ++it) {
            if (it->second.dev != dev) continue;
            CacheBlock b = it->second;
            g_cache.erase(it);
            g_cache_bytes -= b.bytes;
            lk.unlock();
            GBD_CHECK_CUDA(cudaStreamWaitEvent(st, b.ev, 0));
            cudaEventDestroy(b.ev);
            *got = b.bytes;
            return b.p;
        }
    }
    void* p = nullptr;
    if (cudaMalloc(&p, n) != cudaSuccess) {
        cudaGetLastError();
        devcache_trim();
        if (cudaMalloc(&p, n) != cudaSuccess) {
            cudaGetLastError();
            throw_device_oom(n, "cudaMalloc (block cache)");
        }
    }
    *got = n;
    return p;
}

void throw_device_oom(size_t bytes, const char* what) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) cudaGetLastError();
    char buf[200];
    snprintf(buf, sizeof(buf), "%s of %.2f GB failed: device has %.2f GB free of %.2f GB", what, bytes * 1e-9,
             fr * 1e-9, tot * 1e-9);
    throw Error(GBD_ERR_DEVICE_OOM, buf);
}

void devcache_put(void* p, size_t bytes, cudaStream_t st) {
    if (!p) return;
    int dev = 0;
    cudaEvent_t ev = nullptr;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ev, st) != cudaSuccess) {
        if (ev) cudaEventDestroy(ev);
        cudaGetLastError();
        cudaFree(p);  // synchronises: safe without the event
        return;
    }
    std::vector<CacheBlock> evict;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        g_cache.insert({bytes, {p, bytes, ev, dev}});
        g_cache_bytes += bytes;
        while (g_cache_bytes > kCacheMax && !g_cache.empty()) {
            auto it = std::prev(g_cache.end());  // the largest
            evict.push_back(it->second);
            g_cache_bytes -= it->second.bytes;
            g_cache.erase(it);
        }
    }
    for (auto& b : evict) {
        cudaEventSynchronize(b.ev);
        cudaEventDestroy(b.ev);
        cudaFree(b.p);
    }
}

size_t devcache_bytes() {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    return g_cache_bytes;
}

void devcache_trim() {
    std::vector<CacheBlock> all;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        for (auto& kv : g_cache) all.push_back(kv.second);
        g_cache.clear();
        g_cache_bytes = 0;
    }
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto& b : all) {
        cudaSetDevice(b.dev);
        cudaEventSynchronize(b.ev);
        cudaEventDestroy(b.ev);
        cudaFree(b.p);
    }
    cudaSetDevice(cur);
}

}  // namespace gbd
