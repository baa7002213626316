// tc.cu -- H_eff products on the GB300 tensor cores.
//
// The product of Sec. II.B step 2 is two grouped GEMM phases over the
// symmetry sectors (X = O^Lx_stacked psi, then Y += sum_t X_t (O^xR_t)^T with
// one long K over layers t and inner index j).  Both run here as BF16
// tcgen05.mma (kind::f16, FP32 accumulation in TMEM) on split operands, in
// one of two forms (see tc.h): BF16x3 (hi + lo elementwise, three products)
// for the cheap Davidson products, and four row-scaled slices with ten
// products for the anchor products.  The TMEM accumulators are promoted into
// FP32 (hi, lo) two-sum pairs (about 48 significant bits) through two
// ping-pong buffers, so long phase-2 reductions add no FP32 rounding; FP64
// appears only in the split-K reduction.  Operands reach shared memory
// through TMA (cp.async.bulk.tensor, 128-byte swizzle) into a two-stage
// mbarrier ring; one thread issues TMA, one issues MMA, sixteen warps drain
// TMEM.  The kernel is persistent (one CTA per SM walking the work list), so
// loads and MMAs of the next tile overlap the epilogue of the last.  Zero
// fill of TMA boxes handles ragged sector edges.  Every spin-wait is
// bounded: on expiry the CTA records an error code in a device word, stops
// issuing, waits (bounded) for its copies and frees TMEM.
// The BF16x3 product also runs as one fused kernel (tc_fused_kernel, an
// option): each chunk of X is formed in TMEM, split there and multiplied
// into the output tile at once, so X never reaches HBM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <cmath>
#include <cstring>

#include "engine.h"
#include "split.h"
#include "tc.h"

namespace gbd {
namespace tc {

constexpr long long kSpinCycles = 4000000000LL;  // ~2 s at 2 GHz

// PH 1: phase-1 kernel (BF16 output planes through a staging tile); PH 2:
// phase-2 kernel (split-K partial tiles straight from registers, so its
// shared memory goes to pipeline stages); PH 3: FP64 output tiles (one work
// item per tile, no split-K).
template <int MODE, int PH> struct KT {
    static constexpr int NS = ModeCfg<MODE>::NS;
    static constexpr int BN = PH == 2 ? ModeCfg<MODE>::BN2 : ModeCfg<MODE>::BN;
    static constexpr int BUFCOLS = PH == 2 ? ModeCfg<MODE>::BUFCOLS2 : ModeCfg<MODE>::BUFCOLS;
    static constexpr int TMEM_COLS = PH == 2 ? ModeCfg<MODE>::TMEM_COLS2 : ModeCfg<MODE>::TMEM_COLS;
    static constexpr int NB = TMEM_COLS / BUFCOLS;  // TMEM accumulator buffers (the MMA runs NB - 1 fills ahead)
    static_assert(NB == 2 || NB == 4, "two or four accumulator buffers");
    // BF16x3 phase 2 sums its promotions in plain FP32 (the form's own error
    // is 2^-16); the sliced form keeps error-free (hi, lo) pairs
    static constexpr bool PAIRS = !(PH == 2 && MODE == 0);
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE_BYTES = NS * (A_BYTES + B_BYTES);
    static constexpr int CP = BN / 4;                        // accumulator columns per epilogue thread
    static constexpr int ST = 2;  // PH 2 / 3: output straight from registers
    static constexpr int RS = BN * 2;                        // row stride of a BF16 staging plane (XOR-swizzled)
    static constexpr int NPL = PH == 1 ? (MODE == 0 ? 2 : 1) : 0;  // staging planes
    static constexpr int EPI_BYTES = NPL * BM * RS;
    static constexpr int RMAX_BYTES = (MODE == 1 && PH == 1) ? 4 * BM * 4 : 0;  // row maxima of the four column parts
    static constexpr int SMEM_BYTES = ST * STAGE_BYTES + EPI_BYTES + RMAX_BYTES + 1024;
    static_assert(ST <= MAX_STAGES, "barrier arrays");
    // instruction descriptor: BF16 x BF16 -> FP32, both K-major, M = BM, N = BN
    static constexpr uint32_t IDESC =
        (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(BN >> 3) << 17) | (uint32_t(BM >> 4) << 24);
    static_assert(SMEM_BYTES <= 227 * 1024, "shared memory per CTA");
    static_assert(CP % 16 == 0, "TMEM loads of 16 columns");
};

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; returns false on expiry
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (clock64() - t0 > kSpinCycles) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_2d(uint32_t dst, const void* map, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_3d(uint32_t dst, const void* map, int c0, int c1, int c2, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_4d(uint32_t dst, const void* map, int c0, int c1, int c2, int c3, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// TMA tile store shared -> global (bulk group of the issuing thread)
__device__ __forceinline__ void tma_store_4d(const void* map, uint32_t src, int c0, int c1, int c2, int c3) {
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(map),
                 "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    uint64_t d = 0;
    d |= uint64_t((addr >> 4) & 0x3FFF);
    d |= uint64_t(1) << 16;             // leading byte offset (unused for swizzled K-major)
    d |= uint64_t(1024 >> 4) << 32;     // stride byte offset
    d |= uint64_t(1) << 46;             // descriptor version
    d |= uint64_t(2) << 61;             // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// OR of a flag over the epilogue warps (named barrier 1, the barrier of the
// staging planes): every epilogue warp gets the same answer
__device__ __forceinline__ bool epi_any(bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred q, p;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, 1, %2, q;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(r)
        : "r"(uint32_t(v)), "n"(EPI_THREADS)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ int vload(const int& x) { return *reinterpret_cast<const volatile int*>(&x); }
__device__ __forceinline__ void vstore(int& x, int v) { *reinterpret_cast<volatile int*>(&x) = v; }

// MMA width of a work item: its valid columns rounded up to 16, at most BN
template <int BN_> __device__ __forceinline__ int tile_n_of(int N, int n0) {
    const int v = N - n0;
    return v >= BN_ ? BN_ : ((v + 15) & ~15);
}

// position (segment, layer, inner offset) of global chunk c
__device__ __forceinline__ void locate(const KSeg* segs, int seg0, int nseg, int c, int& s, int& t, int& j0) {
    s = seg0;
    while (s < seg0 + nseg && c >= segs[s].nchunk) { c -= segs[s].nchunk; ++s; }
    if (s >= seg0 + nseg) { t = 0; j0 = 0; return; }
    int kch = (segs[s].K + BK - 1) / BK;
    t = c / kch;
    j0 = (c % kch) * BK;
}

// ------------------------------------------------------------------ the kernel
// Persistent: CTA c handles work items c, c + gridDim.x, ...  The TMA
// producer runs ahead across items through the stage ring, the MMA issuer
// alternates two TMEM accumulator buffers (a new one per item and per
// promotion), and the epilogue warps drain one while the MMA fills the other.

// (hi, lo) += x without rounding error (two-sum; hi keeps the FP32 sum)
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
    const float sum = hi + x;
    const float bb = sum - hi;
    lo += (hi - (sum - bb)) + (x - bb);
    hi = sum;
}

template <int MODE, int PH>
__global__ void __launch_bounds__(THREADS, 1) tc_gemm_kernel(const Work* __restrict__ works, int nworks,
                                                             const KSeg* __restrict__ segs,
                                                             const CUtensorMap* __restrict__ maps, int* __restrict__ err) {
    using K_ = KT<MODE, PH>;
    auto tile_n = [](const Work& w) { return tile_n_of<K_::BN>(w.N, w.n0); };
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[MAX_STAGES], empty_bar[MAX_STAGES], tfull[4], tempty[4];
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* epi = smem + K_::ST * K_::STAGE_BYTES;
    float* rmax = reinterpret_cast<float*>(epi + K_::EPI_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < K_::ST; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int b = 0; b < K_::NB; ++b) {
            mbar_init(smem_u32(&tfull[b]), 1);
            mbar_init(smem_u32(&tempty[b]), EPI_WARPS);
        }
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(K_::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer
        long long g = 0;  // chunks issued by this CTA
        for (int wi = blockIdx.x; wi < nworks && !vload(abort_s); wi += gridDim.x) {
            const Work w = works[wi];
            const int n = w.c1 - w.c0;
            if (n <= 0) continue;
            int s, t, j0;
            locate(segs, w.seg0, w.nseg, w.c0, s, t, j0);
            for (int i = 0; i < n; ++i, ++g) {
                const int st = int(g % K_::ST);
                if (g >= K_::ST && !mbar_wait(smem_u32(&empty_bar[st]), uint32_t(((g / K_::ST) & 1) ^ 1))) {
                    atomicExch(err, 1);
                    vstore(abort_s, 1);
                    break;
                }
                if (vload(abort_s)) break;
                const KSeg sg = segs[s];
                const uint32_t bar = smem_u32(&full_bar[st]);
                uint8_t* base = smem + st * K_::STAGE_BYTES;
                mbar_expect_tx(bar, K_::STAGE_BYTES);
                const CUtensorMap* mA = maps + sg.mapA;
                const CUtensorMap* mB = maps + sg.mapB;
                // the slice planes are the outermost dimension of each map
#pragma unroll
                for (int q = 0; q < K_::NS; ++q) {
                    const uint32_t da = smem_u32(base + q * K_::A_BYTES);
                    const uint32_t db = smem_u32(base + K_::NS * K_::A_BYTES + q * K_::B_BYTES);
                    if (sg.rank == 3) {
                        tma_4d(da, mA, j0, sg.a_row + w.m0, t, q, bar);
                        tma_4d(db, mB, j0, sg.b_row + w.n0, t, q, bar);
                    } else {
                        tma_3d(da, mA, j0, sg.a_row + w.m0, q, bar);
                        tma_3d(db, mB, j0, sg.b_row + w.n0, q, bar);
                    }
                }
                j0 += BK;
                if (j0 >= sg.K) {
                    j0 = 0;
                    if (++t >= sg.T) { t = 0; ++s; }
                }
            }
        }
        // on abort: let the loads already issued land before the CTA may exit
        if (vload(abort_s))
            for (long long i = (g > K_::ST ? g - K_::ST : 0); i < g; ++i)
                mbar_wait(smem_u32(&full_bar[i % K_::ST]), uint32_t((i / K_::ST) & 1));
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        long long g = 0;   // chunks consumed
        int D = 0;         // accumulator fills started (buffer D % NB)
        for (int wi = blockIdx.x; wi < nworks && !vload(abort_s); wi += gridDim.x) {
            const Work w = works[wi];
            const int n = w.c1 - w.c0;
            if (n <= 0) continue;
            const int promote = w.promote > 0 ? w.promote : (1 << 30);
            // MMA width: the tile's valid columns rounded up to 16 (M = 128 needs N % 16 == 0)
            const uint32_t idesc = (K_::IDESC & ~(0x3Fu << 17)) | (uint32_t(tile_n(w) >> 3) << 17);
            int inbuf = 0;
            // the chunk's position, as the producer walks it: K steps of 16
            // wholly past the segment's K read zero fill and are skipped
            int ks, kt, kj0;
            locate(segs, w.seg0, w.nseg, w.c0, ks, kt, kj0);
            for (int i = 0; i < n; ++i, ++g) {
                int kst = BK / 16;
                if (ks < w.seg0 + w.nseg) {
                    const int kk = segs[ks].K;
                    kst = (max(1, min(BK, kk - kj0)) + 15) / 16;  // at least one step: the buffer's first MMA clears it
                    kj0 += BK;
                    if (kj0 >= kk) {
                        kj0 = 0;
                        if (++kt >= segs[ks].T) { kt = 0; ++ks; }
                    }
                }
                const int st = int(g % K_::ST);
                if (!mbar_wait(smem_u32(&full_bar[st]), uint32_t((g / K_::ST) & 1))) {
                    atomicExch(err, 2);
                    vstore(abort_s, 1);
                    break;
                }
                if (vload(abort_s)) break;
                tc_fence_after();
                const int buf = D % K_::NB;
                if (inbuf == 0 && D / K_::NB > 0) {
                    if (!mbar_wait(smem_u32(&tempty[buf]), uint32_t((D / K_::NB - 1) & 1))) {
                        atomicExch(err, 3);
                        vstore(abort_s, 1);
                        break;
                    }
                    tc_fence_after();
                }
                const uint32_t a0 = smem_u32(smem + st * K_::STAGE_BYTES);
                const uint32_t b0 = a0 + K_::NS * K_::A_BYTES;
                const uint32_t d = tmem + uint32_t(buf * K_::BUFCOLS);
#pragma unroll
                for (int k = 0; k < BK / 16; ++k) {
                    if (k >= kst) break;
                    const uint32_t off = k * 32;  // 16 BF16 = 32 bytes along K inside the swizzle row
                    const uint32_t acc = (inbuf > 0 || k > 0) ? 1u : 0u;
                    if constexpr (MODE == 0) {
                        const uint64_t ah = sdesc(a0 + off), al = sdesc(a0 + K_::A_BYTES + off);
                        const uint64_t bh = sdesc(b0 + off), bl = sdesc(b0 + K_::B_BYTES + off);
                        umma(d, ah, bh, idesc, acc);
                        umma(d, ah, bl, idesc, 1u);
                        umma(d, al, bh, idesc, 1u);
                    } else {
                        // slice products by order: a1 b1 | a1 b2 + a2 b1 | orders 3 and 4
                        uint64_t sa[4], sb[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            sa[q] = sdesc(a0 + q * K_::A_BYTES + off);
                            sb[q] = sdesc(b0 + q * K_::B_BYTES + off);
                        }
                        const uint32_t d2 = d + 64, d3 = d + 128;
                        umma(d, sa[0], sb[0], idesc, acc);
                        umma(d2, sa[0], sb[1], idesc, acc);
                        umma(d2, sa[1], sb[0], idesc, 1u);
                        umma(d3, sa[0], sb[2], idesc, acc);
                        umma(d3, sa[1], sb[1], idesc, 1u);
                        umma(d3, sa[2], sb[0], idesc, 1u);
                        umma(d3, sa[0], sb[3], idesc, 1u);
                        umma(d3, sa[1], sb[2], idesc, 1u);
                        umma(d3, sa[2], sb[1], idesc, 1u);
                        umma(d3, sa[3], sb[0], idesc, 1u);
                    }
                }
                umma_commit(smem_u32(&empty_bar[st]));
                ++inbuf;
                if (inbuf == promote || i == n - 1) {
                    umma_commit(smem_u32(&tfull[buf]));
                    ++D;
                    inbuf = 0;
                }
            }
        }
    } else if (warp >= 2) {
        // ---------------- epilogue: TMEM -> FP32 (hi, lo) pairs
        // GB300's FP64 pipe is narrow, so each promotion is an error-free FP32
        // two-sum into a (hi, lo) pair (about 48 significant bits).
        constexpr int CP = K_::CP;
        const int quad = warp & 3;          // TMEM lane quadrant this warp may access
        const int part = (warp - 2) >> 2;   // column slice of CP columns
        const int row = quad * 32 + lane;
        int D = 0;
        // Phase 1 stages its output through named barrier 1, so its epilogue
        // warps leave the item loop only together: the loop does not test
        // the abort flag, and after each item's drains every epilogue warp,
        // one that gave up on a wait included, votes before the staging
        // barriers.  The other phases use no named barrier and leave alone.
        for (int wi = blockIdx.x; wi < nworks && (PH == 1 || !vload(abort_s)); wi += gridDim.x) {
            int ndrain, nn;
            {
                const int n = works[wi].c1 - works[wi].c0;
                const int promote = works[wi].promote > 0 ? works[wi].promote : (1 << 30);
                ndrain = n > 0 ? (n + promote - 1) / promote : 0;
                nn = tile_n_of<K_::BN>(works[wi].N, works[wi].n0);  // TMEM columns the MMAs wrote
            }
            float ah[CP], al[K_::PAIRS ? CP : 1];
#pragma unroll
            for (int i = 0; i < CP; ++i) ah[i] = 0.f;
#pragma unroll
            for (int i = 0; i < (K_::PAIRS ? CP : 1); ++i) al[i] = 0.f;
            bool gave_up = false;
            for (int dd = 0; dd < ndrain; ++dd, ++D) {
                const int buf = D % K_::NB;
                // warp-uniform outcome: the TMEM loads below are .sync.aligned
                if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&tfull[buf]), uint32_t((D / K_::NB) & 1)))) {
                    if (lane == 0) atomicExch(err, 4);
                    vstore(abort_s, 1);
                    gave_up = true;
                    break;
                }
                tc_fence_after();
                const uint32_t tb = tmem + (uint32_t(quad * 32) << 16) + uint32_t(buf * K_::BUFCOLS + part * CP);
                if constexpr (MODE == 0) {
#pragma unroll
                    for (int c = 0; c < CP / 16; ++c) {
                        if (part * CP + c * 16 >= nn) continue;  // warp-uniform: columns the MMAs did not write
                        uint32_t r[16];
                        tmem_ld16(tb + c * 16, r);
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            // phase 1 drains once (K = one block dimension), phase 2
                            // promotes every few chunks: plain FP32 sums
                            ah[c * 16 + i] += __uint_as_float(r[i]);
                        }
                    }
                } else {
                    // order 1 and order 2 are exact FP32 sums; orders 3-4 are
                    // 2^-16 of order 1, so one rounded add joins them to order 2
                    if (part * CP < nn) {  // warp-uniform: columns the MMAs wrote
                        uint32_t r1[16], r2[16], r3[16];
                        tmem_ld16(tb, r1);
                        tmem_ld16(tb + 64, r2);
                        tmem_ld16(tb + 128, r3);
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            two_sum_acc(ah[i], al[i], __uint_as_float(r1[i]));
                            two_sum_acc(ah[i], al[i], __uint_as_float(r2[i]) + __uint_as_float(r3[i]));
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&tempty[buf]));
            }
            if constexpr (PH == 1) {
                if (epi_any(gave_up || vload(abort_s))) break;
            } else {
                if (gave_up || vload(abort_s)) break;
            }
            const Work w = works[wi];  // loaded after the drains: keeps registers free for ah / al
            if constexpr (PH == 3) {
                const int gr = w.m0 + row;
                const int gc0 = w.n0 + part * CP;
                if (gr < w.M) {
                    double* o = reinterpret_cast<double*>(w.out) + (long long)gr * w.ldo;
                    if (w.ncols > 0) {
                        int q = gc0 / w.ncols, rcol = gc0 - q * w.ncols;
#pragma unroll
                        for (int i = 0; i < CP; ++i) {
                            if (gc0 + i < w.N) o[(long long)q * w.ldr + rcol] = double(ah[i]) + double(al[i]);
                            if (++rcol == w.ncols) { rcol = 0; ++q; }
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < CP; ++i)
                            if (gc0 + i < w.N) o[gc0 + i] = double(ah[i]) + double(al[i]);
                    }
                }
            } else if constexpr (PH == 2) {
                if constexpr (K_::PAIRS) {
                    // partial tile of (hi, lo) pairs, column-pair-major: a warp
                    // writes 512 contiguous bytes per store
                    float4* out = reinterpret_cast<float4*>(w.out);
#pragma unroll
                    for (int i = 0; i < CP; i += 2)
                        out[(long long)(part * (CP / 2) + i / 2) * BM + row] = make_float4(ah[i], al[i], ah[i + 1], al[i + 1]);
                } else {
                    // partial tile of FP32 sums, column-pair-major (256 contiguous bytes per warp store)
                    float2* out = reinterpret_cast<float2*>(w.out);
#pragma unroll
                    for (int i = 0; i < CP; i += 2)
                        out[(long long)(part * (CP / 2) + i / 2) * BM + row] = make_float2(ah[i], ah[i + 1]);
                }
            } else {
                __nv_bfloat16* o0 = reinterpret_cast<__nv_bfloat16*>(w.out);
                const long long ldo = w.ldo;
                const int et = threadIdx.x - 64;  // 0 .. EPI_THREADS - 1
                constexpr int vpr = K_::BN / 8;   // 16-byte vectors per row
                if constexpr (MODE == 0) {
                    // BF16 hi / lo through four staging tiles (plane x 64-column
                    // half, 128 rows of 128 bytes in the TMA 128-byte swizzle:
                    // chunk c of row r at chunk c ^ (r & 7)).  The rows of the
                    // tile's first layer go out as four TMA tile stores (rows
                    // past the layer's end fall outside the store map and are
                    // not written); rows of later layers (sectors shorter than
                    // the tile) are stored by the epilogue threads.
                    uint32_t ph[CP / 2], pl[CP / 2];
#pragma unroll
                    for (int i = 0; i < CP; i += 2) {
                        // x - bf16(x) is exact in FP32, so the split needs no FP64
                        const float x0 = ah[i], x1 = ah[i + 1];  // phase 1: no lo part
                        const __nv_bfloat16 h0 = __float2bfloat16_rn(x0);
                        const __nv_bfloat16 h1 = __float2bfloat16_rn(x1);
                        const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
                        const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
                        ph[i / 2] = uint32_t(__bfloat16_as_ushort(h0)) | (uint32_t(__bfloat16_as_ushort(h1)) << 16);
                        pl[i / 2] = uint32_t(__bfloat16_as_ushort(l0)) | (uint32_t(__bfloat16_as_ushort(l1)) << 16);
                    }
                    constexpr int SUB = BM * 128;  // one staging tile: 128 rows x 64 BF16
                    auto soff = [](int r, int v) {  // byte offset of 16-byte vector v (0..15) of row r in plane 0
                        return (v >> 3) * SUB + r * 128 + (((v & 7) ^ (r & 7)) << 4);
                    };
                    if (et == 0) bulk_wait_read();  // the previous tile's stores have read the staging tiles
                    asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory");  // earlier readers are done
#pragma unroll
                    for (int j = 0; j < CP / 8; ++j) {
                        const int off = soff(row, part * (CP / 8) + j);
                        *reinterpret_cast<uint4*>(epi + off) = make_uint4(ph[4 * j], ph[4 * j + 1], ph[4 * j + 2], ph[4 * j + 3]);
                        *reinterpret_cast<uint4*>(epi + 2 * SUB + off) =
                            make_uint4(pl[4 * j], pl[4 * j + 1], pl[4 * j + 2], pl[4 * j + 3]);
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the TMA unit
                    asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory");
                    // rows of the first layer: [0, kfirst)
                    const int t0 = w.m0 / w.lay_rows, lo0 = w.m0 - t0 * w.lay_rows;
                    const int kfirst = min(BM, w.lay_rows - lo0);
                    if (et == 0) {
                        const CUtensorMap* om = maps + w.omap;
#pragma unroll
                        for (int q = 0; q < 2; ++q)
#pragma unroll
                            for (int h = 0; h < 2; ++h)
                                if (w.n0 + h * 64 < w.colcap)
                                    tma_store_4d(om, smem_u32(epi + (2 * q + h) * SUB), w.n0 + h * 64, t0, lo0, q);
                        bulk_commit();
                    }
                    // later layers: thread et copies vector et % vpr of rows
                    // kfirst + et / vpr + k * rstep; stacked row t * lay_rows + rr
                    // goes to row rr at column offset t * lay_pitch
                    constexpr int rstep = EPI_THREADS / vpr;
                    const int cv = et % vpr;
                    const int gcol = w.n0 + cv * 8;
                    int r = kfirst + et / vpr;
                    int grow = w.m0 + r;
                    int t = grow / w.lay_rows, rr = grow - t * w.lay_rows;
                    for (; r < BM; r += rstep) {
                        if (grow < w.M && gcol < w.colcap) {
                            const long long at = (long long)rr * ldo + (long long)t * w.lay_pitch + gcol;
                            const int so = soff(r, cv);
                            *reinterpret_cast<uint4*>(o0 + at) = *reinterpret_cast<const uint4*>(epi + so);
                            *reinterpret_cast<uint4*>(o0 + w.plane + at) = *reinterpret_cast<const uint4*>(epi + 2 * SUB + so);
                        }
                        grow += rstep;
                        rr += rstep;
                        while (rr >= w.lay_rows) { rr -= w.lay_rows; ++t; }
                    }
                } else {
                    // four slices on the grid of this row's maximum over the
                    // tile's 64 columns (the K block of the next phase)
                    float m = 0.f;
#pragma unroll
                    for (int i = 0; i < CP; ++i) m = fmaxf(m, fabsf(ah[i]));
                    asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory");  // previous item's readers are done
                    rmax[part * BM + row] = m;
                    asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory");
                    m = fmaxf(fmaxf(rmax[row], rmax[BM + row]), fmaxf(rmax[2 * BM + row], rmax[3 * BM + row]));
                    int ex = 0;
                    frexpf(m, &ex);  // |x| <= m < 2^ex for every x of the row
                    uint32_t pk[4][CP / 2];
#pragma unroll
                    for (int i = 0; i < CP; i += 2) {
                        __nv_bfloat16 q0[4], q1[4];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            // s_k = round(x 2^(8k - ex)) 2^(ex - 8k) of the remainder;
                            // each difference is exact, each slice has <= 8 bits
                            float r = ah[i + h];
                            const float s1 = ldexpf(rintf(ldexpf(r, 8 - ex)), ex - 8);
                            r = (r - s1) + al[i + h];
                            const float s2 = ldexpf(rintf(ldexpf(r, 16 - ex)), ex - 16);
                            r -= s2;
                            const float s3 = ldexpf(rintf(ldexpf(r, 24 - ex)), ex - 24);
                            r -= s3;
                            const float s4 = ldexpf(rintf(ldexpf(r, 32 - ex)), ex - 32);
                            __nv_bfloat16* q = h == 0 ? q0 : q1;
                            q[0] = __float2bfloat16_rn(s1);
                            q[1] = __float2bfloat16_rn(s2);
                            q[2] = __float2bfloat16_rn(s3);
                            q[3] = __float2bfloat16_rn(s4);
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            pk[q][i / 2] = uint32_t(__bfloat16_as_ushort(q0[q])) | (uint32_t(__bfloat16_as_ushort(q1[q])) << 16);
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (q > 0) asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory");  // plane q-1 copied out
#pragma unroll
                        for (int i = 0; i < CP / 2; i += 4) {
                            const int v = (part * CP * 2 + i * 4) >> 4;
                            *reinterpret_cast<uint4*>(epi + row * K_::RS + ((v ^ (row & (vpr - 1))) << 4)) =
                                make_uint4(pk[q][i], pk[q][i + 1], pk[q][i + 2], pk[q][i + 3]);
                        }
                        asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory");
                        for (int v = et; v < BM * vpr; v += EPI_THREADS) {
                            const int r = v / vpr, c8 = (v % vpr) * 8;
                            const int grow = w.m0 + r, gcol = w.n0 + c8;
                            if (grow >= w.M || gcol >= w.colcap) continue;
                            *reinterpret_cast<uint4*>(o0 + q * w.plane + grow * ldo + gcol) =
                                *reinterpret_cast<const uint4*>(epi + r * K_::RS + (((c8 >> 3) ^ (r & (vpr - 1))) << 4));
                        }
                    }
                }
            }
        }
    }
    // the phase-1 tile stores have landed before the CTA exits
    if (PH == 1 && MODE == 0 && threadIdx.x == 64) bulk_wait_all();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(K_::TMEM_COLS) : "memory");
    }
}

// ------------------------------------------------------------------ the fused BF16x3 product
// One kernel for both phases of the BF16x3 product.  A work item is an output
// tile (128 rows of the output left sector x up to 256 columns of the output
// right sector) and a range of chunks of its segments (FSeg).  Per chunk:
//   P1: Xacc (TMEM, FP32) = O^Lx_t[tile rows, :] psi[:, FN columns]   (K = mLi)
//   split: the epilogue warps read Xacc, split it into BF16 hi / lo and store
//          both back into TMEM, where the next MMAs take them as operand A;
//   P2: Y (TMEM, FP32) += X_t(hi, lo) O^xR_t[tile columns, FN columns]^T (K = FN)
// Xacc and the split X are double-buffered and the MMA thread issues P1 of
// chunk g before P2 of chunk g - 1, so the tensor pipe runs P1(g) while the
// epilogue splits chunk g - 1 and never waits for a split younger than one
// chunk.  Operands come through one TMA ring of 64 KB stages in the MMA
// thread's consumption order (the P1 stages of chunk g, then the P2 stage of
// chunk g - 1).  At the end of an item the epilogue drains Y into an FP32
// split-K partial tile (the layout of the two-kernel form's partials, summed
// by reduce_kernel).
// TMEM columns: Y 0-255; buffer b: Xacc 256 + 64 b, X hi 384 + 64 b, X lo
// 416 + 64 b (two BF16 per 32-bit column).  Every wait is bounded; on expiry
// the CTA records an error code, stops, waits (bounded) for its copies and
// MMAs, frees TMEM.

// Chunks of one fused split-K item: its FP32 sum in TMEM runs over at most
// 32 * FN = 2048 terms of K per output element (3 * 128 accumulation steps
// of K = 16, each rounded to FP32).
constexpr int kFusedChunks = 32;

struct KF {
    static constexpr int BN = 256;                // output tile columns
    static constexpr int STAGES = 3;
    static constexpr int PL = BM * BK * 2;        // one plane of an O^Lx tile: 128 rows x 64 (16 KB)
    static constexpr int PP = FN * BK * 2;        // one plane of a psi^T tile: 64 rows x 64 (8 KB)
    static constexpr int RPL = BN * BK * 2;       // one plane of an O^xR tile: 256 rows x 64 (32 KB)
    static constexpr int P1_BYTES = 2 * PL + 2 * PP;  // P1 stage: O^Lx hi, lo, psi^T hi, lo
    static constexpr int P2_BYTES = 2 * RPL;          // P2 stage: O^xR hi, lo
    static constexpr int STAGE_BYTES = P2_BYTES;
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
    static constexpr uint32_t Y = 0, XACC = 256, XHI = 384, XLO = 416, XSTEP = 64, TMEM_COLS = 512;
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(BM >> 4) << 24);
    static_assert(P1_BYTES <= STAGE_BYTES, "a P1 stage fits a ring stage");
    static_assert(SMEM_BYTES <= 227 * 1024, "shared memory per CTA");
    static_assert(FN == BK && FN == 64 && BN % 64 == 0, "one P2 stage per chunk, four epilogue column parts");
};

__device__ __forceinline__ uint32_t idesc_n(uint32_t base, int n) { return (base & ~(0x3Fu << 17)) | (uint32_t(n >> 3) << 17); }

// D (TMEM) += A (TMEM, K-major, two BF16 per column) x B (shared memory descriptor)
__device__ __forceinline__ void umma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr), "r"(r[0]),
                 "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// One chunk of the CTA's chunk stream (items blockIdx.x, + gridDim.x, ...).
struct FChunk {
    int wi, s, t, j0;
    int n1;          // MMA width of the X chunk: valid columns rounded up to 16
    int n2;          // MMA width of the output tile
    int m0, n0;
    int item;        // ordinal of the item within this CTA
    bool first, last;
};
struct FIter {
    int wi = -1, c = 0, c1 = 0, s = 0, t = 0, jb = 0, item = -1;
    bool first = false;
};

// Every role walks the same stream with the same code, so the TMA ring and
// the barriers see one order.
__device__ __forceinline__ bool fnext(const Work* __restrict__ works, int nworks, const FSeg* __restrict__ segs, FIter& it,
                                      FChunk& ch) {
    while (it.c >= it.c1) {
        it.wi = it.wi < 0 ? int(blockIdx.x) : it.wi + int(gridDim.x);
        if (it.wi >= nworks) return false;
        const Work& w = works[it.wi];
        it.c = w.c0;
        it.c1 = w.c1;
        if (it.c >= it.c1) continue;
        int c = it.c, s = w.seg0;
        while (s < w.seg0 + w.nseg && c >= segs[s].nchunk) { c -= segs[s].nchunk; ++s; }
        if (s >= w.seg0 + w.nseg) { it.c = it.c1; continue; }  // range past its segments: nothing to do
        ++it.item;
        it.s = s;
        it.t = c / segs[s].ncol;
        it.jb = c - it.t * segs[s].ncol;
        it.first = true;
    }
    const Work& w = works[it.wi];
    const FSeg& sg = segs[it.s];
    ch.wi = it.wi;
    ch.s = it.s;
    ch.t = it.t;
    ch.j0 = it.jb * FN;
    ch.n1 = tile_n_of<FN>(sg.mRi, ch.j0);
    ch.n2 = tile_n_of<KF::BN>(w.N, w.n0);
    ch.m0 = w.m0;
    ch.n0 = w.n0;
    ch.item = it.item;
    ch.first = it.first;
    it.first = false;
    ++it.c;
    ch.last = it.c >= it.c1;
    if (++it.jb >= sg.ncol) {
        it.jb = 0;
        if (++it.t >= sg.T) { it.t = 0; ++it.s; }
    }
    // a range that runs past its item's segments ends here
    if (!ch.last && it.s >= w.seg0 + w.nseg) { it.c = it.c1; ch.last = true; }
    return true;
}

__global__ void __launch_bounds__(THREADS, 1) tc_fused_kernel(const Work* __restrict__ works, int nworks,
                                                              const FSeg* __restrict__ segs,
                                                              const CUtensorMap* __restrict__ maps, int* __restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[KF::STAGES], empty_bar[KF::STAGES];
    __shared__ __align__(8) uint64_t xacc_full[2], xacc_free[2], xbf_full[2], xbf_free[2], y_full, y_empty, mma_done;
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < KF::STAGES; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&xacc_full[b]), 1);
            mbar_init(smem_u32(&xacc_free[b]), EPI_WARPS);
            mbar_init(smem_u32(&xbf_full[b]), EPI_WARPS);
            mbar_init(smem_u32(&xbf_free[b]), 1);
        }
        mbar_init(smem_u32(&y_full), 1);
        mbar_init(smem_u32(&y_empty), EPI_WARPS);
        mbar_init(smem_u32(&mma_done), 1);
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(KF::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer: P1 stages of chunk g, then the P2 stage of chunk g - 1
        long long g = 0;  // stages issued
        auto stage = [&](uint32_t bytes, uint32_t& bar, uint8_t*& base) -> bool {
            const int st = int(g % KF::STAGES);
            if (g >= KF::STAGES && !mbar_wait(smem_u32(&empty_bar[st]), uint32_t(((g / KF::STAGES) & 1) ^ 1))) {
                atomicExch(err, 11);
                vstore(abort_s, 1);
                return false;
            }
            if (vload(abort_s)) return false;
            bar = smem_u32(&full_bar[st]);
            base = smem + st * KF::STAGE_BYTES;
            mbar_expect_tx(bar, bytes);
            ++g;
            return true;
        };
        auto load_p2 = [&](const FChunk& p) -> bool {
            uint32_t bar;
            uint8_t* base;
            if (!stage(KF::P2_BYTES, bar, base)) return false;
#pragma unroll
            for (int q = 0; q < 2; ++q) tma_4d(smem_u32(base + q * KF::RPL), maps + segs[p.s].mapR, p.j0, p.t, p.n0, q, bar);
            return true;
        };
        FIter it;
        FChunk cur, prev;
        bool hp = false, ok = true;
        while (ok && fnext(works, nworks, segs, it, cur)) {
            const FSeg& sg = segs[cur.s];
            for (int k1 = 0; k1 < sg.nk1 && ok; ++k1) {
                uint32_t bar;
                uint8_t* base;
                if (!(ok = stage(KF::P1_BYTES, bar, base))) break;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    tma_4d(smem_u32(base + q * KF::PL), maps + sg.mapL, k1 * BK, cur.m0, cur.t, q, bar);
                    tma_3d(smem_u32(base + 2 * KF::PL + q * KF::PP), maps + sg.mapP, k1 * BK, cur.j0, q, bar);
                }
            }
            if (ok && hp) ok = load_p2(prev);
            prev = cur;
            hp = true;
        }
        if (ok && hp) load_p2(prev);
        // on abort: let the loads already issued land before the CTA may exit
        if (vload(abort_s))
            for (long long i = (g > KF::STAGES ? g - KF::STAGES : 0); i < g; ++i)
                mbar_wait(smem_u32(&full_bar[i % KF::STAGES]), uint32_t((i / KF::STAGES) & 1));
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        long long g = 0;  // stages consumed
        int gc = 0;       // chunks whose P1 was issued
        auto fail = [&](int code) {
            atomicExch(err, code);
            vstore(abort_s, 1);
            return false;
        };
        auto take = [&](uint32_t& base) -> bool {
            const int st = int(g % KF::STAGES);
            if (!mbar_wait(smem_u32(&full_bar[st]), uint32_t((g / KF::STAGES) & 1))) return fail(12);
            if (vload(abort_s)) return false;
            tc_fence_after();
            base = smem_u32(smem + st * KF::STAGE_BYTES);
            return true;
        };
        auto release = [&]() { umma_commit(smem_u32(&empty_bar[int(g % KF::STAGES)])); ++g; };
        // P2 of chunk p (the pc-th chunk of the stream)
        auto issue_p2 = [&](const FChunk& p, int pc) -> bool {
            const int b = pc & 1;
            if (p.first && p.item > 0) {
                if (!mbar_wait(smem_u32(&y_empty), uint32_t((p.item - 1) & 1))) return fail(13);
                tc_fence_after();
            }
            if (!mbar_wait(smem_u32(&xbf_full[b]), uint32_t((pc >> 1) & 1))) return fail(14);
            tc_fence_after();
            const uint32_t idesc = idesc_n(KF::IDESC, p.n2);
            uint32_t b0;
            if (!take(b0)) return false;
            const uint32_t xh = tmem + KF::XHI + b * KF::XSTEP, xl = tmem + KF::XLO + b * KF::XSTEP;
            for (int k = 0; k < p.n1 / 16; ++k) {
                const uint64_t bh = sdesc(b0 + k * 32), bl = sdesc(b0 + KF::RPL + k * 32);
                const uint32_t acc = (!p.first || k > 0) ? 1u : 0u;
                umma_ts(tmem + KF::Y, xh + k * 8, bh, idesc, acc);  // 16 BF16 of K = 8 TMEM columns
                umma_ts(tmem + KF::Y, xh + k * 8, bl, idesc, 1u);
                umma_ts(tmem + KF::Y, xl + k * 8, bh, idesc, 1u);
            }
            release();
            umma_commit(smem_u32(&xbf_free[b]));
            if (p.last) umma_commit(smem_u32(&y_full));
            return true;
        };
        FIter it;
        FChunk cur, prev;
        bool hp = false, ok = true;
        while (ok && fnext(works, nworks, segs, it, cur)) {
            const FSeg& sg = segs[cur.s];
            const int b = gc & 1;
            if (gc >= 2) {
                if (!(ok = mbar_wait(smem_u32(&xacc_free[b]), uint32_t(((gc >> 1) - 1) & 1)) || fail(15))) break;
                tc_fence_after();
            }
            const uint32_t idesc = idesc_n(KF::IDESC, cur.n1);
            const uint32_t xa = tmem + KF::XACC + b * KF::XSTEP;
            for (int k1 = 0; k1 < sg.nk1 && ok; ++k1) {
                uint32_t a0;
                if (!(ok = take(a0))) break;
                const uint32_t b0 = a0 + 2 * KF::PL;
                const int kst = (max(1, min(BK, sg.mLi - k1 * BK)) + 15) / 16;  // K steps past mLi read zero fill
#pragma unroll
                for (int k = 0; k < BK / 16; ++k) {
                    if (k >= kst) break;
                    const uint32_t off = k * 32;
                    const uint64_t ah = sdesc(a0 + off), al = sdesc(a0 + KF::PL + off);
                    const uint64_t bh = sdesc(b0 + off), bl = sdesc(b0 + KF::PP + off);
                    const uint32_t acc = (k1 > 0 || k > 0) ? 1u : 0u;
                    umma(xa, ah, bh, idesc, acc);
                    umma(xa, ah, bl, idesc, 1u);
                    umma(xa, al, bh, idesc, 1u);
                }
                release();
            }
            if (!ok) break;
            umma_commit(smem_u32(&xacc_full[b]));
            if (hp && !(ok = issue_p2(prev, gc - 1))) break;
            prev = cur;
            hp = true;
            ++gc;
        }
        if (ok && hp) issue_p2(prev, gc - 1);
        // every MMA of this thread has completed before TMEM may be freed
        umma_commit(smem_u32(&mma_done));
        mbar_wait(smem_u32(&mma_done), 0u);
    } else if (warp >= 2) {
        // ---------------- epilogue: split each X chunk, drain Y per item
        const int quad = warp & 3;          // TMEM lane quadrant this warp may access
        const int part = (warp - 2) >> 2;   // column part: 16 X columns, 64 Y columns
        const int row = quad * 32 + lane;
        const uint32_t lane_off = uint32_t(quad * 32) << 16;
        auto wait_all = [&](uint64_t& bar, uint32_t parity, int code) -> bool {
            if (__all_sync(0xffffffffu, mbar_wait(smem_u32(&bar), parity))) return true;
            if (lane == 0) atomicExch(err, code);
            vstore(abort_s, 1);
            return false;
        };
        auto arrive = [&](uint64_t& bar) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bar));
        };
        FIter it;
        FChunk ch;
        int gc = 0;
        while (!vload(abort_s) && fnext(works, nworks, segs, it, ch)) {
            // X chunk: TMEM FP32 -> BF16 (hi, lo) pairs back into TMEM
            const int b = gc & 1;
            if (!wait_all(xacc_full[b], uint32_t((gc >> 1) & 1), 16)) break;
            tc_fence_after();
            const bool act = part * 16 < ch.n1;  // warp-uniform: columns P1 wrote
            uint32_t ph[8], pl[8];
            if (act) {
                uint32_t r[16];
                tmem_ld16(tmem + lane_off + KF::XACC + b * KF::XSTEP + part * 16, r);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    // x - bf16(x) is exact in FP32, so the split needs no FP64
                    const float x0 = __uint_as_float(r[2 * i]), x1 = __uint_as_float(r[2 * i + 1]);
                    const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
                    const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
                    const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
                    ph[i] = uint32_t(__bfloat16_as_ushort(h0)) | (uint32_t(__bfloat16_as_ushort(h1)) << 16);
                    pl[i] = uint32_t(__bfloat16_as_ushort(l0)) | (uint32_t(__bfloat16_as_ushort(l1)) << 16);
                }
            }
            arrive(xacc_free[b]);
            if (gc >= 2 && !wait_all(xbf_free[b], uint32_t(((gc >> 1) - 1) & 1), 17)) break;
            tc_fence_after();
            if (act) {
                tmem_st8(tmem + lane_off + KF::XHI + b * KF::XSTEP + part * 8, ph);
                tmem_st8(tmem + lane_off + KF::XLO + b * KF::XSTEP + part * 8, pl);
                tmem_st_wait();
            }
            arrive(xbf_full[b]);
            ++gc;
            if (!ch.last) continue;
            // end of the item: Y -> FP32 partial tile
            if (!wait_all(y_full, uint32_t(ch.item & 1), 18)) break;
            tc_fence_after();
            float y[64];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (part * 64 + c * 16 < ch.n2) {  // warp-uniform: columns the MMAs wrote
                    uint32_t r[16];
                    tmem_ld16(tmem + lane_off + KF::Y + part * 64 + c * 16, r);
#pragma unroll
                    for (int i = 0; i < 16; ++i) y[c * 16 + i] = __uint_as_float(r[i]);
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) y[c * 16 + i] = 0.f;
                }
            }
            arrive(y_empty);
            // column-pair-major partial tile (256 contiguous bytes per warp store)
            float2* out = reinterpret_cast<float2*>(works[ch.wi].out);
#pragma unroll
            for (int i = 0; i < 64; i += 2) out[(long long)(part * 32 + i / 2) * BM + row] = make_float2(y[i], y[i + 1]);
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(KF::TMEM_COLS) : "memory");
    }
}

// partial tiles hold FP32 (hi, lo) pairs (or FP32 sums), column-pair-major:
// element (i, j) at index ((j / 2) * BM + i) * 2 + (j % 2)
// grid (tiles, kReduceSplit): CTA y sums rows y, y + kReduceSplit, ... of its tile
constexpr int kReduceSplit = 16;

__global__ void reduce_kernel(const Reduce* __restrict__ red, const float2* __restrict__ partial) {
    const Reduce r = red[blockIdx.x];
    for (int i = blockIdx.y; i < BM; i += kReduceSplit) {
        const int gi = r.m0 + i;
        if (gi >= r.M) break;
        for (int j = threadIdx.x; j < r.bn; j += blockDim.x) {
            const int gj = r.n0 + j;
            if (gj >= r.N) break;
            const long long idx = ((long long)(j / 2) * BM + i) * 2 + (j % 2);
            double v = 0.0;
            if (r.pairs) {
                for (int p = r.p0; p < r.p1; ++p) {
                    const float2 x = partial[(long long)p * BM * r.bn + idx];
                    v += double(x.x) + double(x.y);
                }
            } else {
                const float* pf = reinterpret_cast<const float*>(partial);
                for (int p = r.p0; p < r.p1; ++p) v += double(pf[(long long)p * BM * r.bn + idx]);
            }
            r.out[(long long)gi * r.ldo + gj] = v;
        }
    }
}

// ------------------------------------------------------------------ tensor maps
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                                const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        GBD_CHECK_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        GBD_REQUIRE(p && q == cudaDriverEntryPointSuccess, GBD_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
        fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

// BF16 K-major operand: inner extent K (elements), rows, optional layers,
// then the slice planes; row pitch ld elements (multiple of 8), layer and
// plane pitches in elements (multiples of 8).
CUtensorMap make_map(const void* base, int K, long long rows, int layers, int ld, long long layer_pitch, int planes,
                     long long plane_pitch, int box_rows) {
    CUtensorMap m;
    std::memset(&m, 0, sizeof(m));
    GBD_REQUIRE((reinterpret_cast<uintptr_t>(base) & 15) == 0 && ld % 8 == 0 && layer_pitch % 8 == 0 &&
                    plane_pitch % 8 == 0,
                GBD_ERR_STATE, "TMA operand misaligned");
    cuuint64_t dims[4];
    cuuint64_t strides[3];
    cuuint32_t box[4];
    cuuint32_t estr[4] = {1, 1, 1, 1};
    cuuint32_t rank = 0;
    dims[rank] = cuuint64_t(std::max(K, 1));
    box[rank++] = cuuint32_t(BK);
    dims[rank] = cuuint64_t(std::max<long long>(rows, 1));
    strides[rank - 1] = cuuint64_t(ld) * 2;
    box[rank++] = cuuint32_t(box_rows);
    if (layers > 0) {
        dims[rank] = cuuint64_t(layers);
        strides[rank - 1] = cuuint64_t(layer_pitch) * 2;
        box[rank++] = 1;
    }
    dims[rank] = cuuint64_t(std::max(planes, 1));
    strides[rank - 1] = cuuint64_t(std::max<long long>(plane_pitch, 8)) * 2;
    box[rank++] = 1;
    CUresult r = encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, const_cast<void*>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    GBD_REQUIRE(r == CUDA_SUCCESS, GBD_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    return m;
}

// BF16 K-major operand with up to two outer dimensions of any element
// strides (multiples of 8), then the slice planes; box BK x box1 x box2.
CUtensorMap make_map_n(const void* base, int K, int nd, const long long* dims, const long long* strides, const int* box,
                       int planes, long long plane_pitch) {
    CUtensorMap m;
    std::memset(&m, 0, sizeof(m));
    GBD_REQUIRE((reinterpret_cast<uintptr_t>(base) & 15) == 0 && plane_pitch % 8 == 0 && nd >= 1 && nd <= 2,
                GBD_ERR_STATE, "TMA operand misaligned");
    cuuint64_t gd[4], gs[3];
    cuuint32_t bx[4], es[4] = {1, 1, 1, 1};
    gd[0] = cuuint64_t(std::max(K, 1));
    bx[0] = cuuint32_t(BK);
    for (int i = 0; i < nd; ++i) {
        GBD_REQUIRE(strides[i] % 8 == 0 && box[i] >= 1 && box[i] <= 256, GBD_ERR_STATE, "TMA operand misaligned");
        gd[1 + i] = cuuint64_t(std::max<long long>(dims[i], 1));
        gs[i] = cuuint64_t(strides[i]) * 2;
        bx[1 + i] = cuuint32_t(box[i]);
    }
    gd[1 + nd] = cuuint64_t(std::max(planes, 1));
    gs[nd] = cuuint64_t(std::max<long long>(plane_pitch, 8)) * 2;
    bx[1 + nd] = 1;
    CUresult r = encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, cuuint32_t(nd + 2), const_cast<void*>(base), gd, gs, bx, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    GBD_REQUIRE(r == CUDA_SUCCESS, GBD_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    return m;
}

inline int pad8(int x) { return (x + 7) / 8 * 8; }

}  // namespace tc

using namespace tc;

namespace {

// Operator blocks laid out class by class, rows padded to 8 elements.
long long op_layout(const OpSet& O, std::vector<std::vector<long long>>& off) {
    long long tot = 0;
    off.assign(O.cls.size(), {});
    for (size_t c = 0; c < O.cls.size(); ++c)
        for (const auto& b : O.cls[c].blocks) {
            off[c].push_back(tot);
            tot += (long long)O.cls[c].states.size() * b.rows * pad8(b.cols);
        }
    return tot;
}

template <class T> void upload_vec(DevBuf& d, const std::vector<T>& v, cudaStream_t st) {
    d.ensure_cached(std::max<size_t>(v.size() * sizeof(T), 16), st);
    if (!v.empty()) GBD_CHECK_CUDA(cudaMemcpyAsync(d.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
}

// FP64 path of the two block-Hamiltonian terms (mode 0, optional): their
// layers are zeroed in the BF16 copies and applied in FP64 after each product.
void build_block_terms(Ctx& C, TcPlan& P, const std::vector<std::vector<long long>>& offL,
                       const std::vector<std::vector<long long>>& offR) {
    Heff& H = C.H;
    TcHeff& T = H.tc;
    cudaStream_t st = C.cs;
    const int cut = H.b + 1;
    const int sI = C.mpo.idxI[cut], sF = C.mpo.idxF[cut];
    T.blk = C.cfg.mixed_fp64_blocks && sI >= 0 && sF >= 0;
    if (!T.blk) return;
    int c0 = H.OL.state_class[sI];
    GBD_REQUIRE(c0 == H.OL.state_class[sF], GBD_ERR_STATE, "block terms in different classes");
    const int lay[2] = {H.OL.state_layer[sI], H.OL.state_layer[sF]};
    std::vector<long long> xoff(H.sq.size() * 2);
    long long xt = 0;
    for (size_t q = 0; q < H.sq.size(); ++q)
        for (int k = 0; k < 2; ++k) {
            xoff[q * 2 + k] = xt;
            xt += (long long)H.bL.dim[H.sL[q]] * H.bR.dim[H.sR[q]];
        }
    T.blk_x.ensure(size_t(std::max(xt, 1LL)) * 8);
    T.blk_a.clear();
    T.blk_b.clear();
    const int Tn = int(H.OL.cls[c0].states.size());
    for (int side = 0; side < 2; ++side) {
        const OpSet& O = side == 0 ? H.OL : H.OR;
        __nv_bfloat16* base = side == 0 ? P.ol.as<__nv_bfloat16>() : P.orr.as<__nv_bfloat16>();
        const long long plane = side == 0 ? P.nL : P.nR;
        const auto& off = side == 0 ? offL : offR;
        for (size_t i = 0; i < O.cls[c0].blocks.size(); ++i) {
            const OpBlock& bb = O.cls[c0].blocks[i];
            const long long ldk = pad8(bb.cols);
            const long long per = (long long)bb.rows * ldk;
            for (int k = 0; k < 2; ++k)
                for (int q = 0; q < 2; ++q) {
                    if (side == 0) {  // layer-stacked
                        GBD_CHECK_CUDA(cudaMemsetAsync(base + q * plane + off[c0][i] + lay[k] * per, 0, size_t(per) * 2, st));
                    } else if (bb.rows > 0) {  // layers side by side along each row
                        GBD_CHECK_CUDA(cudaMemset2DAsync(base + q * plane + off[c0][i] + lay[k] * ldk, size_t(Tn * ldk) * 2, 0,
                                                         size_t(ldk) * 2, size_t(bb.rows), st));
                    }
                }
        }
    }
    for (size_t q = 0; q < H.sq.size(); ++q) {
        int bl = -1, br = -1;
        for (size_t x = 0; x < H.OL.cls[c0].blocks.size(); ++x)
            if (H.OL.cls[c0].blocks[x].Qo == H.sq[q] && H.OL.cls[c0].blocks[x].Qi == H.sq[q]) bl = int(x);
        for (size_t x = 0; x < H.OR.cls[c0].blocks.size(); ++x)
            if (H.OR.cls[c0].blocks[x].Qo == H.sq[q] && H.OR.cls[c0].blocks[x].Qi == H.sq[q]) br = int(x);
        if (bl < 0 || br < 0) continue;
        const int mL = H.bL.dim[H.sL[q]], mR = H.bR.dim[H.sR[q]];
        std::vector<GemmSeg> segB;
        for (int k = 0; k < 2; ++k) {
            GemmTask ta{};
            ta.C = T.blk_x.as<double>() + xoff[q * 2 + k];
            ta.ldc = mR; ta.M = mL; ta.N = mR; ta.nbatch = 1;
            GemmSeg ga{};
            ga.A = H.OL.data.as<double>() + H.OL.cls[c0].blocks[bl].off + (long long)lay[k] * mL * mL;
            ga.lda = mL;
            ga.B = H.xin.as<double>() + H.soff[q];
            ga.ldb = mR; ga.K = mL; ga.T = 1; ga.coef = 1.0;
            T.blk_a.add_task(ta, {ga});
            GemmSeg gb{};
            gb.A = T.blk_x.as<double>() + xoff[q * 2 + k];
            gb.lda = mR;
            gb.B = H.OR.data.as<double>() + H.OR.cls[c0].blocks[br].off + (long long)lay[k] * mR * mR;
            gb.ldb = mR; gb.transB = 1; gb.K = mR; gb.T = 1; gb.coef = 1.0;
            segB.push_back(gb);
        }
        GemmTask tb{};
        tb.C = H.yout.as<double>() + H.soff[q];
        tb.ldc = mR; tb.M = mL; tb.N = mR; tb.nbatch = 1; tb.beta = 1.0;
        T.blk_b.add_task(tb, segB);
    }
    std::vector<std::pair<const void*, size_t>> bufs = {{H.OL.data.p, size_t(H.OL.total) * 8},
                                                        {H.OR.data.p, size_t(H.OR.total) * 8},
                                                        {T.blk_x.p, T.blk_x.bytes}, {H.xin.p, H.xin.bytes},
                                                        {H.yout.p, H.yout.bytes}};
    T.blk_a.check(bufs, "mixed/block-a");
    T.blk_b.check(bufs, "mixed/block-b");
    T.blk_a.upload(st);
    T.blk_b.upload(st);
}

// tensor-core GFLOP a work list issues (whole 128-row tiles at the MMA width,
// every split or slice product): the gap to the useful flops is padding
template <int MODE, int PH> double issued_gflop(const std::vector<Work>& ws, const std::vector<KSeg>& segs) {
    constexpr int TBN = PH == 2 ? ModeCfg<MODE>::BN2 : ModeCfg<MODE>::BN;
    double f = 0.0;
    for (const auto& w : ws) {
        const int v = w.N - w.n0;
        const int nn = v >= TBN ? TBN : ((v + 15) & ~15);  // the kernel's MMA width
        // K steps of 16 the kernel issues over the item's chunks: per
        // segment, BK / 16 for every chunk but a layer's last, which takes
        // its remaining K rounded up to 16 (chunk j is a layer's last when
        // (j + 1) is a multiple of the chunks per layer)
        long long ksteps = 0;
        int s = w.seg0, a = w.c0;
        while (s < w.seg0 + w.nseg && a >= segs[s].nchunk) { a -= segs[s].nchunk; ++s; }
        for (int rem = w.c1 - w.c0; rem > 0 && s < w.seg0 + w.nseg; ++s, a = 0) {
            const KSeg& g = segs[s];
            const int b = std::min(g.nchunk, a + rem);
            const int kch = (g.K + BK - 1) / BK;
            const int lst = (std::max(1, std::min(BK, g.K - (kch - 1) * BK)) + 15) / 16;
            ksteps += (long long)(BK / 16) * (b - a) - (long long)(BK / 16 - lst) * (b / kch - a / kch);
            rem -= b - a;
        }
        f += double(ksteps) * 16.0 * BM * nn * 2.0 * (MODE == 0 ? 3.0 : 10.0);
    }
    return f * 1e-9;
}

// ---- autotuner of the BF16x3 phase-2 work list over the sector sizes.
// Candidates: split-K items per SM (chunks per item = total / (k * SMs)) and
// the listing order of the items (K range by K range across the tiles of a
// sector, so tiles reading the same chunks run together, or tile by tile).
struct TuneCand { int split_per_sm, order; };
constexpr TuneCand kTuneCands[] = {{2, 0}, {4, 0}, {8, 0}, {2, 1}, {4, 1}, {8, 1}};
constexpr int kTuneN = int(sizeof(kTuneCands) / sizeof(kTuneCands[0]));
constexpr int kTuneDefault = 1;  // the fixed shape: 4 items per SM, K-range order
static_assert(kTuneN <= 8, "gbd_tune_info holds 8 candidates");

std::mutex g_tune_mu;
std::map<unsigned long long, int> g_tune_cache;  // sector-size histogram key -> chosen candidate

TuneParams tune_params(const TcTune& t) {
    const int i = t.cur >= 0 ? t.cur : kTuneDefault;
    return TuneParams{kTuneCands[i].split_per_sm, kTuneCands[i].order};
}

// Histogram of the position's sector sizes (max(rows, cols) in bins of 64,
// the last bin open) and the operator count bucket: the tuning key.
void tune_begin(Ctx& C) {
    Heff& H = C.H;
    TcTune& t = H.tc.tune;
    t = TcTune();
    for (size_t q = 0; q < H.sq.size(); ++q) {
        const int m = std::max(H.bL.dim[H.sL[q]], H.bR.dim[H.sR[q]]);
        t.hist[std::min(m / 64, 15)] += 1;
    }
    // the key is coarse on purpose: positions of one sweep region, whose
    // bond dimensions change a little at every truncation, share it.  It
    // takes the largest sector (in 64-row bins), the total of the histogram
    // weighted by bin (a size moment, within 25%) and the layer count (within
    // 512).
    unsigned long long k = 1469598103934665603ULL;  // FNV-1a
    auto mix = [&](unsigned long long v) { k = (k ^ v) * 1099511628211ULL; };
    int top = 0;
    double moment = 0.0;
    for (int i = 0; i < 16; ++i)
        if (t.hist[i]) { top = i; moment += double(t.hist[i]) * (i + 1) * (i + 1); }
    mix((unsigned long long)top);
    mix((unsigned long long)std::lround(std::log(std::max(moment, 1.0)) / std::log(1.25)));
    mix((unsigned long long)C.mpo.bond_dim(H.b + 1) / 512);
    t.key = k;
    if (!C.cfg.autotune) { t.cur = -1; return; }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(k);
    if (it != g_tune_cache.end()) {
        t.cur = t.chosen = it->second;
        t.from_cache = true;
        C.last_tune = t;
        C.last_tune_b = H.b;
    } else {
        t.active = true;
        t.cur = 0;
    }
}

// Operator slice planes for one side (0: O^Lx, 1: O^xR), split from the FP64
// enlarged arena of that side: FORM 0 the BF16x3 planes, FORM 1 the sliced
// planes, FORM 2 both in one pass over the FP64 arena.
template <int FORM> void build_ops(Ctx& C, int side) {
    Heff& H = C.H;
    cudaStream_t st = C.cs;
    const OpSet& O = side == 0 ? H.OL : H.OR;
    GBD_REQUIRE(O.resident(), GBD_ERR_STATE, "enlarged operators not resident for the operator planes");
    std::vector<std::vector<long long>> off;
    const long long n = std::max(op_layout(O, off), 8LL);
    constexpr int mlo = FORM == 1 ? 1 : 0, mhi = FORM == 0 ? 0 : 1;  // the forms built
    const int NSm[2] = {ModeCfg<0>::NS, ModeCfg<1>::NS};
    __nv_bfloat16* dst[2] = {nullptr, nullptr};
    for (int m = mlo; m <= mhi; ++m) {
        TcPlan& P = H.tc.pl[m];
        DevBuf& d = side == 0 ? P.ol : P.orr;
        (side == 0 ? P.nL : P.nR) = n;
        d.ensure_cached(size_t(n) * NSm[m] * 2, st);
        dst[m] = d.as<__nv_bfloat16>();
    }
    // BF16x3 O^xR: layers side by side along each row ([row][layer][col]),
    // the phase-2 B operand; otherwise layer-stacked rows
    std::vector<SplitDesc> sd[2];
    for (size_t c = 0; c < O.cls.size(); ++c)
        for (size_t i = 0; i < O.cls[c].blocks.size(); ++i) {
            const OpBlock& b = O.cls[c].blocks[i];
            const long long Tn = (long long)O.cls[c].states.size();
            const long long rows = Tn * b.rows;
            const int ldd = pad8(b.cols);
            const long long per = std::max<long long>(1, kSplitUnits / ((ldd + 63) / 64));
            for (long long r0 = 0; r0 < rows; r0 += per)
                for (int m = mlo; m <= mhi; ++m) {
                    SplitDesc q{O.data.as<double>() + b.off + r0 * b.cols, b.cols, 1, std::min(per, rows - r0),
                                b.cols, ldd, dst[m] + off[c][i], n, 1LL << 62, 0, ldd, r0};
                    if (m == 0 && side == 1) { q.R = std::max(b.rows, 1); q.lpitch = ldd; q.rpitch = Tn * ldd; }
                    sd[m].push_back(q);
                }
        }
    if (!sd[mlo].empty()) {
        DevBuf d0, d1;
        upload_vec(d0, sd[mlo], st);
        if (FORM == 2) upload_vec(d1, sd[1], st);
        for (size_t i0 = 0; i0 < sd[mlo].size(); i0 += (1u << 30)) {
            const unsigned nb = unsigned(std::min<size_t>(1u << 30, sd[mlo].size() - i0));
            launch_split(FORM, d0.as<SplitDesc>() + i0, FORM == 2 ? d1.as<SplitDesc>() + i0 : nullptr, nb, st);
        }
        GBD_CHECK_CUDA(cudaGetLastError());
        GBD_CHECK_CUDA(cudaStreamSynchronize(st));  // the descriptor buffers are freed on return
    }
    for (int m = mlo; m <= mhi; ++m) {
        TcPlan& P = H.tc.pl[m];
        P.bytes_ops = double(P.nL + P.nR) * NSm[m] * 2.0;
        (side == 0 ? P.ops_l : P.ops_r) = true;
    }
}

// Both forms' operator planes are needed at this position: the mixed
// Davidson with sliced anchors (which also renormalise from the sliced planes).
bool both_forms(const Ctx& C) {
    return C.cfg.precision == GBD_MIXED_BF16X3 && C.cfg.mixed_polish == 2;
}

// Split-K work list over the output sector tiles: per tile (BM x TBN) the K
// chunks of all its segments (Seg: KSeg of the phase-2 kernel or FSeg of the
// fused kernel) split into near-equal ranges, one FP64 reduction per tile;
// max_chunks > 0 caps the chunks of one item.
template <class Seg>
void build_items(Ctx& C, const std::vector<Seg>& segs, const std::vector<std::vector<int>>& seg_of_out, int TBN,
                 bool pairs, int promote, int max_chunks, const TuneParams& tp, std::vector<Work>& w2,
                 std::vector<Reduce>& red, std::vector<Seg>& s2o, long long& npart) {
    Heff& H = C.H;
    long long total_chunks = 0;
    for (size_t q = 0; q < H.sq.size(); ++q) {
        long long c = 0;
        for (int si : seg_of_out[q]) c += segs[si].nchunk;
        int tiles = ((H.bL.dim[H.sL[q]] + BM - 1) / BM) * ((H.bR.dim[H.sR[q]] + TBN - 1) / TBN);
        total_chunks += c * tiles;
    }
    long long target = std::max<long long>(16, total_chunks / ((long long)tp.split_per_sm * H.tc.n_sm) + 1);
    if (max_chunks > 0) target = std::min<long long>(target, max_chunks);
    npart = 0;
    for (size_t q = 0; q < H.sq.size(); ++q) {
        int seg0 = int(s2o.size());
        int nchunk = 0;
        for (int si : seg_of_out[q]) { s2o.push_back(segs[si]); nchunk += segs[si].nchunk; }
        int nseg = int(s2o.size()) - seg0;
        const int mL = H.bL.dim[H.sL[q]], mR = H.bR.dim[H.sR[q]];
        // one reduction (and a run of partials) per output tile; order 0 lists
        // the items K range by K range, so the tiles of one sector that read
        // the same K chunks run side by side and share them in L2; order 1
        // lists them tile by tile
        const int nrange = int((nchunk + target - 1) / target);
        const size_t r0 = red.size();
        for (int m0 = 0; m0 < mL; m0 += BM)
            for (int n0 = 0; n0 < mR; n0 += TBN) {
                Reduce r{};
                r.out = H.yout.as<double>() + H.soff[q];
                r.ldo = mR;
                r.m0 = m0;
                r.n0 = n0;
                r.M = mL;
                r.N = mR;
                r.bn = TBN;
                r.pairs = pairs ? 1 : 0;
                r.p0 = int(npart);
                npart += nrange;
                r.p1 = int(npart);
                red.push_back(r);
            }
        const size_t r1 = red.size();
        auto item = [&](size_t ti, int k) {
            const Reduce& r = red[ti];
            const int c0 = int(k * target);
            Work w{};
            w.m0 = r.m0;
            w.n0 = r.n0;
            w.M = mL;
            w.N = mR;
            w.seg0 = seg0;
            w.nseg = nseg;
            w.c0 = c0;
            w.c1 = int(std::min<long long>(nchunk, c0 + target));
            w.out_kind = 0;
            w.promote = promote;
            w.ldo = TBN;
            w.colcap = TBN;
            w.out = reinterpret_cast<void*>((long long)r.p0 + k);  // patched to a pointer by the caller
            w2.push_back(w);
        };
        if (tp.order == 0) {
            for (int k = 0; k < nrange; ++k)
                for (size_t ti = r0; ti < r1; ++ti) item(ti, k);
        } else {
            for (size_t ti = r0; ti < r1; ++ti)
                for (int k = 0; k < nrange; ++k) item(ti, k);
        }
    }
}

// tensor-core GFLOP the fused work list issues per product (P1 and P2 of
// every chunk at their MMA widths, three split products each)
void issued_fused(const std::vector<Work>& ws, const std::vector<FSeg>& segs, double& p1, double& p2) {
    p1 = p2 = 0.0;
    for (const auto& w : ws) {
        const int v2 = w.N - w.n0;
        const int n2 = v2 >= KF::BN ? KF::BN : ((v2 + 15) & ~15);
        int s = w.seg0, c = w.c0;
        while (s < w.seg0 + w.nseg && c >= segs[s].nchunk) { c -= segs[s].nchunk; ++s; }
        for (int k = w.c0; k < w.c1 && s < w.seg0 + w.nseg; ++k) {
            const FSeg& g = segs[s];
            const int j0 = (c % g.ncol) * FN, v1 = g.mRi - j0;
            const int n1 = v1 >= FN ? FN : ((v1 + 15) & ~15);
            p1 += double(BM) * n1 * ((g.mLi + 15) / 16 * 16) * 2.0 * 3.0;
            p2 += double(BM) * n2 * n1 * 2.0 * 3.0;
            if (++c >= g.nchunk) { c = 0; ++s; }
        }
    }
    p1 *= 1e-9;
    p2 *= 1e-9;
}

// Phase-2 work list of one product form (BF16x3 fused: the fused kernel's).
template <int MODE> void build_p2(Ctx& C, const TuneParams& tp) {
    constexpr int TBN = ModeCfg<MODE>::BN2;
    constexpr bool pairs = KT<MODE, 2>::PAIRS;
    TcPlan& P = C.H.tc.pl[MODE];
    cudaStream_t st = C.cs;
    const bool fused = MODE == 0 && P.fused;
    const int bn = fused ? KF::BN : TBN;
    std::vector<Work> w2;
    std::vector<Reduce> red;
    long long npart = 0;
    if (fused) {
        std::vector<FSeg> s2o;
        // an item accumulates at most kFusedChunks chunks (K = 2048) in TMEM
        build_items(C, P.f_host, P.seg_of_out, bn, false, 0, kFusedChunks, tp, w2, red, s2o, npart);
        issued_fused(w2, s2o, P.issued_p1, P.issued_p2);
        upload_vec(P.s2, s2o, st);
    } else {
        std::vector<KSeg> s2o;
        build_items(C, P.s2_host, P.seg_of_out, bn, pairs, MODE == 0 ? 8 : 1, 0, tp, w2, red, s2o, npart);
        P.issued_p2 = issued_gflop<MODE, 2>(w2, s2o);
        upload_vec(P.s2, s2o, st);
    }
    // partial tiles: float2 (hi, lo) per element, or one float per element
    P.partial.ensure_cached(size_t(std::max<long long>(npart, 1)) * BM * bn * sizeof(float2), st);
    for (auto& w : w2)
        w.out = reinterpret_cast<float*>(P.partial.p) + reinterpret_cast<long long>(w.out) * BM * bn * (pairs ? 2 : 1);
    upload_vec(P.w2, w2, st);
    upload_vec(P.red, red, st);
    P.n_w2 = int(w2.size());
    P.n_red = int(red.size());
    GBD_CHECK_CUDA(cudaStreamSynchronize(st));  // the host vectors are freed on return
}

// Slice planes, tensor maps and work lists of one product form.
template <int MODE> void build_plan(Ctx& C) {
    constexpr int NS = ModeCfg<MODE>::NS, TBN = ModeCfg<MODE>::BN;
    Heff& H = C.H;
    TcHeff& T = H.tc;
    TcPlan& P = T.pl[MODE];
    cudaStream_t st = C.cs;
    const double t0 = wall_ms();
    // ---- operator slice planes (already built when the FP64 arenas were released)
    for (int side = 0; side < 2; ++side) {
        if (P.ops(side)) continue;
        // one pass writes both forms' planes when both are needed and the
        // other form's are not there yet
        if (both_forms(C) && !T.pl[1 - MODE].ops(side)) build_ops<2>(C, side);
        else build_ops<MODE>(C, side);
    }
    std::vector<std::vector<long long>> offL, offR;
    op_layout(H.OL, offL);
    op_layout(H.OR, offR);
    const double t1 = wall_ms();
    if (MODE == 0) build_block_terms(C, P, offL, offR);
    // ---- psi^T slice planes
    P.np = 8;
    for (const auto& ps : T.psec) P.np = std::max(P.np, ps.dst + (long long)ps.mR * ps.ldp);
    P.psi.ensure_cached(size_t(P.np) * NS * 2, st);
    {
        // psi^T per sector: row n of the operand is column n of psi
        std::vector<SplitDesc> sd;
        for (const auto& ps : T.psec) {
            // psi is small and read transposed: many short descriptors keep enough loads in flight
            const long long per = std::max<long long>(1, 32 / ((ps.ldp + 63) / 64));
            for (long long r0 = 0; r0 < ps.mR; r0 += per)
                sd.push_back({H.xin.as<double>() + ps.src + r0, 1, ps.mR, std::min<long long>(per, ps.mR - r0), ps.mL,
                              ps.ldp, P.psi.as<__nv_bfloat16>() + ps.dst, P.np, 1LL << 62, 0, ps.ldp, r0});
        }
        upload_vec(P.psi_split, sd, st);
        P.n_psi = int(sd.size());
    }
    // ---- pairs (class, block) with their phase-1 outputs X
    // (the position's (class, left block, right block) pairs, longest phase-1
    // K first so the phase-1 work list comes out longest first)
    struct Pair { int c, bl, br, so, si; long long x; };
    std::vector<Pair> pairs;
    pairs.reserve(H.pairs.size());
    long long nx = 0;
    for (const auto& hp : H.pairs) {
        pairs.push_back({hp.c, hp.bl, hp.br, hp.s_out, hp.s_in, nx});
        nx += (long long)H.OL.cls[hp.c].states.size() * H.bL.dim[H.sL[hp.s_out]] * pad8(H.bR.dim[H.sR[hp.s_in]]);
    }
    std::stable_sort(pairs.begin(), pairs.end(), [&](const Pair& a, const Pair& b) {
        return H.bL.dim[H.sL[a.si]] > H.bL.dim[H.sL[b.si]];
    });
    P.nx = std::max(nx, 8LL);
    // the fused BF16x3 kernel keeps X on the SM: no phase-1 buffer
    P.fused = MODE == 0 && T.want_fused;
    P.f_host.clear();
    // one phase-1 buffer serves both forms (they never run at the same time):
    // sized for the four slice planes of the sliced form
    if (!P.fused) T.x.ensure_cached(size_t(P.nx) * ModeCfg<1>::NS * 2, st);
    __nv_bfloat16* const xbase = P.fused ? nullptr : T.x.as<__nv_bfloat16>();
    // ---- tensor maps: one per operand, the NS slice planes as outer dimension
    std::vector<CUtensorMap> maps;
    auto add_maps = [&](const __nv_bfloat16* base, long long plane, int K, long long rows, int layers, int ld,
                        long long lp, int box_rows) {
        int id = int(maps.size());
        maps.push_back(make_map(base, K, rows, layers, ld, lp, NS, plane, box_rows));
        return id;
    };
    std::vector<int> psi_map(H.sq.size());
    for (size_t s = 0; s < H.sq.size(); ++s) {
        const auto& ps = T.psec[s];
        // box rows: the phase-1 tile columns, or one X chunk of the fused kernel
        psi_map[s] = add_maps(P.psi.as<__nv_bfloat16>() + ps.dst, P.np, ps.mL, ps.mR, 0, ps.ldp, 0, P.fused ? FN : TBN);
    }
    std::vector<KSeg> s1, s2;
    std::vector<Work> w1;
    std::vector<std::vector<int>> seg_of_out(H.sq.size());
    for (const auto& p : pairs) {
        const OpClass& cl = H.OL.cls[p.c];
        const int Tn = int(cl.states.size());
        const int mLo = H.bL.dim[H.sL[p.so]], mLi = H.bL.dim[H.sL[p.si]];
        const int mRo = H.bR.dim[H.sR[p.so]], mRi = H.bR.dim[H.sR[p.si]];
        const long long ol = offL[p.c][p.bl];
        const long long orr = offR[p.c][p.br];
        if (MODE == 0 && P.fused) {
            // O^Lx block (mLi, mLo, Tn) and O^xR block (mRi, Tn, mRo), both K-major
            const long long dl[2] = {mLo, Tn}, sl[2] = {pad8(mLi), (long long)mLo * pad8(mLi)};
            const long long dr[2] = {Tn, mRo}, sr[2] = {pad8(mRi), (long long)Tn * pad8(mRi)};
            const int bl[2] = {BM, 1}, br[2] = {1, KF::BN};
            const int mL_ = int(maps.size());
            maps.push_back(make_map_n(P.ol.as<__nv_bfloat16>() + ol, mLi, 2, dl, sl, bl, NS, P.nL));
            const int mR_ = int(maps.size());
            maps.push_back(make_map_n(P.orr.as<__nv_bfloat16>() + orr, mRi, 2, dr, sr, br, NS, P.nR));
            FSeg f{};
            f.mapL = mL_;
            f.mapP = psi_map[p.si];
            f.mapR = mR_;
            f.mLi = mLi;
            f.mRi = mRi;
            f.T = Tn;
            f.nk1 = (mLi + BK - 1) / BK;
            f.ncol = (mRi + FN - 1) / FN;
            f.nchunk = Tn * f.ncol;
            seg_of_out[p.so].push_back(int(P.f_host.size()));
            P.f_host.push_back(f);
            continue;
        }
        // phase 1: X (Tn*mLo x mRi) = OL_stacked (Tn*mLo x mLi) psi (mLi x mRi), psi^T K-major
        int mA = add_maps(P.ol.as<__nv_bfloat16>() + ol, P.nL, mLi, (long long)Tn * mLo, 0, pad8(mLi), 0, BM);
        int sidx = int(s1.size());
        s1.push_back({mA, psi_map[p.si], 0, 0, mLi, 1, 2, (mLi + BK - 1) / BK});
        int xmap = -1;
        if (MODE == 0) {
            // tile stores of X ([row][layer][col]): dims (col, layer, row), box 64 x 1 x 128
            const long long dx[2] = {Tn, mLo}, sx[2] = {pad8(mRi), (long long)Tn * pad8(mRi)};
            const int bx[2] = {1, BM};
            xmap = int(maps.size());
            maps.push_back(make_map_n(xbase + p.x, pad8(mRi), 2, dx, sx, bx, NS, P.nx));
        }
        for (long long m0 = 0; m0 < (long long)Tn * mLo; m0 += BM)
            for (int n0 = 0; n0 < mRi; n0 += TBN) {
                Work w{};
                w.m0 = int(m0);
                w.n0 = n0;
                w.M = Tn * mLo;
                w.N = mRi;
                w.seg0 = sidx;
                w.nseg = 1;
                w.c0 = 0;
                w.c1 = s1[sidx].nchunk;
                w.out_kind = 1;
                w.promote = MODE == 0 ? (1 << 30) : 1;
                w.plane = P.nx;
                w.colcap = pad8(mRi);
                if (MODE == 0) {  // X stored [row][layer][col] for the concatenated phase-2 K
                    w.lay_rows = mLo;
                    w.lay_pitch = pad8(mRi);
                    w.ldo = (long long)Tn * pad8(mRi);
                } else {
                    w.lay_rows = 0;
                    w.ldo = pad8(mRi);
                }
                w.out = xbase + p.x;
                w.omap = xmap;
                w1.push_back(w);
            }
        seg_of_out[p.so].push_back(int(s2.size()));
        if (MODE == 0) {
            // phase 2 operands with layers side by side: X (mLo x Tn*ldk),
            // OR (mRo x Tn*ldk); one K of Tn * ldk, padded only at its end
            const int Kc = Tn * pad8(mRi);
            int mX = add_maps(xbase + p.x, P.nx, Kc, mLo, 0, Kc, 0, BM);
            int mO = add_maps(P.orr.as<__nv_bfloat16>() + orr, P.nR, Kc, mRo, 0, Kc, 0, ModeCfg<MODE>::BN2);
            s2.push_back({mX, mO, 0, 0, Kc, 1, 2, (Kc + BK - 1) / BK});
        } else {
            // phase 2 operands: X_t (mLo x mRi), OR_t (mRo x mRi), layers Tn; K
            // chunks stay inside one layer (the slices' grid is per layer row)
            int mX = add_maps(xbase + p.x, P.nx, mRi, mLo, Tn, pad8(mRi), (long long)mLo * pad8(mRi), BM);
            int mO = add_maps(P.orr.as<__nv_bfloat16>() + orr, P.nR, mRi, mRo, Tn, pad8(mRi), (long long)mRo * pad8(mRi),
                              ModeCfg<MODE>::BN2);
            s2.push_back({mX, mO, 0, 0, mRi, Tn, 3, Tn * ((mRi + BK - 1) / BK)});
        }
    }
    P.s2_host = s2;
    P.seg_of_out = seg_of_out;
    // tensor-core work issued per product (whole 128-row tiles at the MMA
    // width, every slice product): the gap to the useful flops is padding
    if (!P.fused) P.issued_p1 = issued_gflop<MODE, 1>(w1, s1);
    if (MODE == 0) tune_begin(C);
    build_p2<MODE>(C, MODE == 0 ? tune_params(H.tc.tune) : TuneParams{});
    // persistent CTAs take items round-robin: w1 is longest first by
    // construction (pairs sorted by K), w2 keeps its K-range grouping
    const double t2 = wall_ms();
    // ---- upload
    upload_vec(P.maps, maps, st);
    upload_vec(P.w1, w1, st);
    upload_vec(P.s1, s1, st);
    P.n_w1 = int(w1.size());
    GBD_CHECK_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<MODE, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        KT<MODE, 1>::SMEM_BYTES));
    GBD_CHECK_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<MODE, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        KT<MODE, 2>::SMEM_BYTES));
    if (P.fused)
        GBD_CHECK_CUDA(cudaFuncSetAttribute(tc_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, KF::SMEM_BYTES));
    GBD_CHECK_CUDA(cudaStreamSynchronize(st));
    P.built = true;
    C.timers[Ctx::T_PREP_SPLIT] += t1 - t0;
    C.timers[Ctx::T_PREP_PLAN] += t2 - t1;
    C.timers[Ctx::T_PREP_UPLOAD] += wall_ms() - t2;
}

}  // namespace

// Builds the slice planes, tensor maps and work lists of one product form
// (0: BF16x3, 1: sliced) for the current position.
void tc_prepare(Ctx& C, int mode) {
    GBD_REQUIRE(mode == 0 || mode == 1, GBD_ERR_ARG, "tensor-core product form must be 0 or 1");
    Heff& H = C.H;
    TcHeff& T = H.tc;
    cudaStream_t st = C.cs;
    if (!H.tc_ready) {
        // shared by both forms: psi^T sector layout, error word, SM count
        T.psec.clear();
        long long np = 0;
        for (size_t s = 0; s < H.sq.size(); ++s) {
            int mL = H.bL.dim[H.sL[s]], mR = H.bR.dim[H.sR[s]];
            T.psec.push_back({H.soff[s], np, mL, mR, pad8(mL)});
            np += (long long)mR * pad8(mL);
        }
        T.err.ensure_cached(sizeof(int), st);
        GBD_CHECK_CUDA(cudaMemsetAsync(T.err.p, 0, sizeof(int), st));
        int dev = 0;
        GBD_CHECK_CUDA(cudaGetDevice(&dev));
        GBD_CHECK_CUDA(cudaDeviceGetAttribute(&T.n_sm, cudaDevAttrMultiProcessorCount, dev));
        T.n_sm = std::max(T.n_sm, 1);
        T.pl[0] = TcPlan();
        T.pl[1] = TcPlan();
        // the mixed form with sliced anchors needs the FP64 enlarged arenas only
        // to build the operator planes (and the diagonal): when the planes and
        // the shared phase-1 buffer would not fit beside them, both forms'
        // planes are built side by side and each side's FP64 arena released
        T.low_mem = false;
        if (C.cfg.precision == GBD_MIXED_BF16X3 && C.cfg.mixed_polish == 2 && !C.cfg.mixed_fp64_blocks &&
            C.cfg.low_memory >= 0) {
            size_t fr = 0, tot = 0;
            GBD_CHECK_CUDA(cudaMemGetInfo(&fr, &tot));
            const double avail = double(fr) + double(devcache_bytes());
            const double need = H.mem_bf16x3 + H.mem_sliced + H.mem_xtc;
            T.low_mem = C.cfg.low_memory == 1 || need > 0.85 * avail;
        }
        H.tc_ready = true;
    }
    if (T.low_mem && (H.OL.resident() || H.OR.resident())) {
        heff_diag(C);  // the diagonal reads the FP64 arenas
        const double t0 = wall_ms();
        for (int side = 0; side < 2; ++side) {
            if (!T.pl[0].ops(side) && !T.pl[1].ops(side)) {
                build_ops<2>(C, side);
            } else {
                if (!T.pl[0].ops(side)) build_ops<0>(C, side);
                if (!T.pl[1].ops(side)) build_ops<1>(C, side);
            }
            (side == 0 ? H.OL : H.OR).data.release();
        }
        C.timers[Ctx::T_PREP_SPLIT] += wall_ms() - t0;
    }
    if (!T.pl[mode].built) {
        if (mode == 0) {
            build_plan<0>(C);
            C.timers[Ctx::T_TC_ISSUE1] = T.pl[0].issued_p1;
            C.timers[Ctx::T_TC_ISSUE2] = T.pl[0].issued_p2;
        } else {
            build_plan<1>(C);
            C.timers[Ctx::T_TC_ISSUE_SL] = T.pl[1].issued_p1 + T.pl[1].issued_p2;
        }
    }
}

// After each BF16x3 product: while the tuner is trying candidates, record
// this product's device time and move to the next candidate; after the last
// one, keep the fastest (cached under the sector-size histogram key).
void tc_tune_step(Ctx& C, double ms) {
    TcTune& t = C.H.tc.tune;
    if (!t.active) return;
    t.ms[t.cur] = ms;
    int next = t.cur + 1;
    if (next < kTuneN) {
        t.cur = next;
    } else {
        int best = 0;
        for (int i = 1; i < kTuneN; ++i)
            if (t.ms[i] < t.ms[best]) best = i;
        t.chosen = best;
        t.cur = best;
        t.active = false;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[t.key] = best;
        C.last_tune = t;
        C.last_tune_b = C.H.b;
    }
    build_p2<0>(C, tune_params(t));
    C.timers[Ctx::T_TC_ISSUE2] = C.H.tc.pl[0].issued_p2;
}

void tc_tune_reset() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache.clear();
}

void tc_tune_info(Ctx& C, gbd_tune_info* out) {
    // the current position's state while it has one, else the last finished choice
    const bool cur = C.H.tc_ready && C.H.tc.tune.key != 0;
    const TcTune& t = cur ? C.H.tc.tune : C.last_tune;
    std::memset(out, 0, sizeof(*out));
    out->position = cur ? C.H.b : C.last_tune_b;
    out->active = t.active ? 1 : 0;
    out->n_candidates = kTuneN;
    out->chosen = t.chosen;
    out->current = t.cur;
    out->from_cache = t.from_cache ? 1 : 0;
    out->default_index = kTuneDefault;
    out->key = t.key;
    for (int i = 0; i < kTuneN; ++i) {
        out->split_per_sm[i] = kTuneCands[i].split_per_sm;
        out->order[i] = kTuneCands[i].order;
        out->ms[i] = t.ms[i];
    }
    for (int i = 0; i < 16; ++i) out->hist[i] = t.hist[i];
}

// Frees the BF16x3 operands, the shared phase-1 buffer and the split-K
// partials of the position: after its Davidson, only the sliced operator
// planes are still read (by the renormalisation).
void tc_release_products(Ctx& C) {
    TcHeff& T = C.H.tc;
    T.pl[0] = TcPlan();
    T.pl[1].psi.release();
    T.pl[1].partial.release();
    T.pl[1].built = false;
    T.x.release();
}

namespace {
template <int MODE> void run_plan(Ctx& C) {
    Heff& H = C.H;
    TcHeff& T = H.tc;
    TcPlan& P = T.pl[MODE];
    cudaStream_t st = C.cs;
    if (P.n_psi > 0) {
        launch_split(MODE, P.psi_split.as<SplitDesc>(), nullptr, unsigned(P.n_psi), st);
    }
    if (P.n_w1 > 0) {
        tc_gemm_kernel<MODE, 1><<<std::min(P.n_w1, T.n_sm), THREADS, KT<MODE, 1>::SMEM_BYTES, st>>>(
            P.w1.as<Work>(), P.n_w1, P.s1.as<KSeg>(), P.maps.as<CUtensorMap>(), T.err.as<int>());
        count_launch();
    }
    if (P.n_red > 0) {
        if (P.n_w2 > 0 && MODE == 0 && P.fused) {
            tc_fused_kernel<<<std::min(P.n_w2, T.n_sm), THREADS, KF::SMEM_BYTES, st>>>(
                P.w2.as<Work>(), P.n_w2, P.s2.as<FSeg>(), P.maps.as<CUtensorMap>(), T.err.as<int>());
            count_launch();
        } else if (P.n_w2 > 0) {
            tc_gemm_kernel<MODE, 2><<<std::min(P.n_w2, T.n_sm), THREADS, KT<MODE, 2>::SMEM_BYTES, st>>>(
                P.w2.as<Work>(), P.n_w2, P.s2.as<KSeg>(), P.maps.as<CUtensorMap>(), T.err.as<int>());
            count_launch();
        }
        reduce_kernel<<<dim3(P.n_red, kReduceSplit), 128, 0, st>>>(P.red.as<Reduce>(), P.partial.as<float2>());
        count_launch();
    }
    if (MODE == 0 && T.blk) {
        T.blk_a.launch(st);
        T.blk_b.launch(st);
    }
    GBD_CHECK_CUDA(cudaGetLastError());
}
}  // namespace

// One tensor-core product: H.xin (FP64) -> H.yout (FP64).
void tc_apply(Ctx& C, int mode) {
    GBD_REQUIRE(C.H.tc_ready && C.H.tc.pl[mode].built, GBD_ERR_STATE, "tensor-core plan not prepared");
    if (mode == 0) run_plan<0>(C); else run_plan<1>(C);
}

// The renormalisation (Sec. II.B step 3) on the tensor cores in the sliced
// form, for every kept block j of out (class order):
//   phase A: tmp_j (T*dimO x k_i) = O_stacked (T*dimO x dimI) U_i, O read from
//            the sliced planes of the current enlarged set (built for the
//            anchor products), U^T sliced here; tmp_j at tmp + toff[j] (FP64);
//   phase B: new_j[t] (k_o x k_i) = U_o^T tmp_j[t] for all layers t at once as
//            U_o^T [tmp_j[0] | tmp_j[1] | ...], with tmp_j transposed and
//            sliced per layer, written into out's arena.
// Returns false (nothing launched) when the sliced planes of O are not built.
bool tc_renormalize(Ctx& C, const OpSet& O, const Iso& U, OpSet& out, const std::vector<long long>& toff,
                    double* tmp) {
    Heff& H = C.H;
    TcHeff& T = H.tc;
    if (!H.tc_ready || !T.pl[1].ops_l || !T.pl[1].ops_r) return false;
    const bool left = &O == &H.OL;
    if (!left && &O != &H.OR) return false;
    constexpr int NS = ModeCfg<1>::NS, TBN = ModeCfg<1>::BN;
    TcPlan& P = T.pl[1];
    cudaStream_t st = C.cs;
    std::vector<std::vector<long long>> off;
    op_layout(O, off);
    const __nv_bfloat16* arena = left ? P.ol.as<__nv_bfloat16>() : P.orr.as<__nv_bfloat16>();
    const long long plane = left ? P.nL : P.nR;
    // U_Q^T per kept sector Q (k rows, K = basis dimension), sliced
    std::vector<long long> uoff(U.out.q.size(), -1);
    long long nu = 0;
    for (size_t q = 0; q < U.out.q.size(); ++q) {
        if (U.off[q] < 0) continue;
        const int e = U.basis.find(U.out.q[q]);
        uoff[q] = nu;
        nu += (long long)U.out.dim[q] * pad8(U.basis.dim[e]);
    }
    nu = std::max(nu, 8LL);
    T.ren_u.ensure_cached(size_t(nu) * NS * 2, st);
    std::vector<SplitDesc> sd;
    for (size_t q = 0; q < U.out.q.size(); ++q) {
        if (uoff[q] < 0) continue;
        const int k = U.out.dim[q];
        const int dim = U.basis.dim[U.basis.find(U.out.q[q])];
        // element (r = kept state, c = basis state) of U^T is U[c][r]
        const long long per = std::max<long long>(1, 32 / ((pad8(dim) + 63) / 64));
        for (long long r0 = 0; r0 < k; r0 += per)
            sd.push_back({U.data.as<double>() + U.off[q] + r0, 1, k, std::min<long long>(per, k - r0), dim, pad8(dim),
                          T.ren_u.as<__nv_bfloat16>() + uoff[q], nu, 1LL << 62, 0, pad8(dim), r0});
    }
    DevBuf dsd;
    upload_vec(dsd, sd, st);
    if (!sd.empty()) {
        launch_split(1, dsd.as<SplitDesc>(), nullptr, unsigned(sd.size()), st);
    }
    std::vector<CUtensorMap> maps;
    std::vector<KSeg> segs;
    std::vector<Work> works;
    size_t j = 0;
    for (size_t c = 0; c < out.cls.size(); ++c) {
        const int Tn = int(out.cls[c].states.size());
        for (const auto& nb : out.cls[c].blocks) {
            const int eo = U.basis.find(nb.Qo), ei = U.basis.find(nb.Qi);
            const int dimO = U.basis.dim[eo], dimI = U.basis.dim[ei];
            int bi = -1;
            for (size_t x = 0; x < O.cls[c].blocks.size(); ++x)
                if (O.cls[c].blocks[x].qo == eo && O.cls[c].blocks[x].qi == ei) bi = int(x);
            GBD_REQUIRE(bi >= 0, GBD_ERR_STATE, "renormalisation: missing enlarged block");
            const int mA = int(maps.size());
            maps.push_back(make_map(arena + off[c][bi], dimI, (long long)Tn * dimO, 0, pad8(dimI), 0, NS, plane, BM));
            maps.push_back(make_map(T.ren_u.as<__nv_bfloat16>() + uoff[nb.qi], dimI, nb.cols, 0, pad8(dimI), 0, NS, nu,
                                    TBN));
            const int sidx = int(segs.size());
            segs.push_back({mA, mA + 1, 0, 0, dimI, 1, 2, (dimI + BK - 1) / BK});
            for (long long m0 = 0; m0 < (long long)Tn * dimO; m0 += BM)
                for (int n0 = 0; n0 < nb.cols; n0 += TBN) {
                    Work w{};
                    w.m0 = int(m0);
                    w.n0 = n0;
                    w.M = Tn * dimO;
                    w.N = nb.cols;
                    w.seg0 = sidx;
                    w.nseg = 1;
                    w.c0 = 0;
                    w.c1 = segs[sidx].nchunk;
                    w.out_kind = 2;
                    w.promote = 1;
                    w.ldo = nb.cols;
                    w.colcap = nb.cols;
                    w.out = tmp + toff[j];
                    works.push_back(w);
                }
            ++j;
        }
    }
    auto longer = [](const Work& x, const Work& y) { return x.c1 - x.c0 > y.c1 - y.c0; };
    std::stable_sort(works.begin(), works.end(), longer);
    DevBuf dmaps, dsegs, dworks;
    upload_vec(dmaps, maps, st);
    upload_vec(dsegs, segs, st);
    upload_vec(dworks, works, st);
    GBD_CHECK_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<1, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        KT<1, 3>::SMEM_BYTES));
    const int nw = int(works.size());
    if (nw > 0) {
        tc_gemm_kernel<1, 3><<<std::min(nw, T.n_sm), THREADS, KT<1, 3>::SMEM_BYTES, st>>>(
            dworks.as<Work>(), nw, dsegs.as<KSeg>(), dmaps.as<CUtensorMap>(), T.err.as<int>());
        count_launch();
    }
    GBD_CHECK_CUDA(cudaGetLastError());
    // ---- phase B: tmp_j^T per layer, sliced: rows (t, k_i), K = dimO
    std::vector<long long> toffT;
    long long nt = 0;
    for (size_t c = 0; c < out.cls.size(); ++c) {
        const int Tn = int(out.cls[c].states.size());
        for (const auto& nb : out.cls[c].blocks) {
            const int dimO = U.basis.dim[U.basis.find(nb.Qo)];
            toffT.push_back(nt);
            nt += (long long)Tn * nb.cols * pad8(dimO);
        }
    }
    nt = std::max(nt, 8LL);
    T.ren_t.ensure_cached(size_t(nt) * NS * 2, st);
    std::vector<SplitDesc> sdB;
    std::vector<CUtensorMap> mapsB;
    std::vector<KSeg> segsB;
    std::vector<Work> worksB;
    j = 0;
    double* dN = out.data.as<double>();
    for (size_t c = 0; c < out.cls.size(); ++c) {
        const int Tn = int(out.cls[c].states.size());
        for (const auto& nb : out.cls[c].blocks) {
            const int dimO = U.basis.dim[U.basis.find(nb.Qo)];
            const int ki = nb.cols, ko = nb.rows;
            // element (row kk, col r) of tmp_j[t]^T is tmp_j[(t*dimO + r)*ki + kk]
            const long long per = std::max<long long>(1, kSplitUnits / ((pad8(dimO) + 63) / 64));
            for (int t = 0; t < Tn; ++t)
                for (long long r0 = 0; r0 < ki; r0 += per)
                    sdB.push_back({tmp + toff[j] + (long long)t * dimO * ki + r0, 1, ki, std::min<long long>(per, ki - r0),
                                   dimO, pad8(dimO), T.ren_t.as<__nv_bfloat16>() + toffT[j] + (long long)t * ki * pad8(dimO),
                                   nt, 1LL << 62, 0, pad8(dimO), r0});
            const int mA = int(mapsB.size());
            mapsB.push_back(make_map(T.ren_u.as<__nv_bfloat16>() + uoff[nb.qo], dimO, ko, 0, pad8(dimO), 0, NS, nu, BM));
            mapsB.push_back(make_map(T.ren_t.as<__nv_bfloat16>() + toffT[j], dimO, (long long)Tn * ki, 0, pad8(dimO), 0, NS,
                                     nt, TBN));
            const int sidx = int(segsB.size());
            segsB.push_back({mA, mA + 1, 0, 0, dimO, 1, 2, (dimO + BK - 1) / BK});
            for (int m0 = 0; m0 < ko; m0 += BM)
                for (long long n0 = 0; n0 < (long long)Tn * ki; n0 += TBN) {
                    Work w{};
                    w.m0 = m0;
                    w.n0 = int(n0);
                    w.M = ko;
                    w.N = Tn * ki;
                    w.seg0 = sidx;
                    w.nseg = 1;
                    w.c0 = 0;
                    w.c1 = segsB[sidx].nchunk;
                    w.out_kind = 2;
                    w.promote = 1;
                    w.ldo = ki;           // row pitch inside a layer
                    w.ncols = ki;         // column t*ki + kk -> layer t, column kk
                    w.ldr = (long long)ko * ki;
                    w.out = dN + nb.off;
                    worksB.push_back(w);
                }
            ++j;
        }
    }
    DevBuf dsdB, dmapsB, dsegsB, dworksB;
    upload_vec(dsdB, sdB, st);
    for (size_t i0 = 0; i0 < sdB.size(); i0 += (1u << 30)) {
        const unsigned n = unsigned(std::min<size_t>(1u << 30, sdB.size() - i0));
        launch_split(1, dsdB.as<SplitDesc>() + i0, nullptr, n, st);
    }
    if (!worksB.empty()) {
        std::stable_sort(worksB.begin(), worksB.end(), longer);
        upload_vec(dmapsB, mapsB, st);
        upload_vec(dsegsB, segsB, st);
        upload_vec(dworksB, worksB, st);
        const int nwB = int(worksB.size());
        tc_gemm_kernel<1, 3><<<std::min(nwB, T.n_sm), THREADS, KT<1, 3>::SMEM_BYTES, st>>>(
            dworksB.as<Work>(), nwB, dsegsB.as<KSeg>(), dmapsB.as<CUtensorMap>(), T.err.as<int>());
        count_launch();
    }
    GBD_CHECK_CUDA(cudaGetLastError());
    GBD_CHECK_CUDA(cudaStreamSynchronize(st));  // the tables above are freed on return
    T.ren_u.release();
    T.ren_t.release();
    const int e = tc_error(C);
    GBD_REQUIRE(e == 0, GBD_ERR_CUDA, "tensor-core renormalisation stopped on a bounded wait (code " + std::to_string(e) + ")");
    return true;
}

// Dense enlargement GEMMs in the sliced form: A = W^T (Tout x Tin) per
// segment, B = E^T (n x Tin) per input block, both sliced (transposed) here;
// one FP64 output tile per work item, written with the sub-block strides.
void tc_enlarge_dense(Ctx& C, const std::vector<TcEnlTask>& tasks, const std::vector<TcEnlSeg>& segs) {
    constexpr int NS = ModeCfg<1>::NS, TBN = ModeCfg<1>::BN;
    cudaStream_t st = C.cs;
    // distinct operands
    std::map<const double*, std::pair<long long, int>> wmap, emap;  // -> (offset in the slice planes, index)
    std::vector<const TcEnlSeg*> wlist, elist;
    long long nw = 0, ne = 0;
    for (const auto& sg : segs) {
        if (!wmap.count(sg.W)) {
            wmap[sg.W] = {nw, int(wlist.size())};
            wlist.push_back(&sg);
            nw += (long long)sg.Tout * pad8(sg.Tin);
        }
        if (!emap.count(sg.E)) {
            emap[sg.E] = {ne, int(elist.size())};
            elist.push_back(&sg);
            ne += sg.n * pad8(sg.Tin);
        }
    }
    nw = std::max(nw, 8LL);
    ne = std::max(ne, 8LL);
    C.env_sl_w.ensure_cached(size_t(nw) * NS * 2, st);
    C.env_sl_e.ensure_cached(size_t(ne) * NS * 2, st);
    C.env_err.ensure(sizeof(int));
    GBD_CHECK_CUDA(cudaMemsetAsync(C.env_err.p, 0, sizeof(int), st));
    // slicing: W^T row c = column c of W; E^T row e = column e of E
    std::vector<SplitDesc> sd;
    auto add = [&](const double* src, long long rows, int K, long long src_rowstep, __nv_bfloat16* dst, long long plane) {
        const long long per = std::max<long long>(1, kSplitUnits / ((pad8(K) + 63) / 64));
        for (long long r0 = 0; r0 < rows; r0 += per)
            sd.push_back({src + r0, 1, src_rowstep, std::min(per, rows - r0), K, pad8(K), dst, plane, 1LL << 62, 0, pad8(K),
                          r0});
    };
    for (const auto* sg : wlist)
        add(sg->W, sg->Tout, sg->Tin, sg->Tout, C.env_sl_w.as<__nv_bfloat16>() + wmap[sg->W].first, nw);
    for (const auto* sg : elist)
        add(sg->E, sg->n, sg->Tin, sg->n, C.env_sl_e.as<__nv_bfloat16>() + emap[sg->E].first, ne);
    DevBuf dsd;
    upload_vec(dsd, sd, st);
    for (size_t i0 = 0; i0 < sd.size(); i0 += (1u << 30)) {
        const unsigned n = unsigned(std::min<size_t>(1u << 30, sd.size() - i0));
        launch_split(1, dsd.as<SplitDesc>() + i0, nullptr, n, st);
    }
    // tensor maps (one per distinct operand), segments, work items
    std::vector<CUtensorMap> maps;
    std::vector<int> wmi(wlist.size()), emi(elist.size());
    for (size_t i = 0; i < wlist.size(); ++i) {
        wmi[i] = int(maps.size());
        maps.push_back(make_map(C.env_sl_w.as<__nv_bfloat16>() + wmap[wlist[i]->W].first, wlist[i]->Tin, wlist[i]->Tout, 0,
                                pad8(wlist[i]->Tin), 0, NS, nw, BM));
    }
    for (size_t i = 0; i < elist.size(); ++i) {
        emi[i] = int(maps.size());
        maps.push_back(make_map(C.env_sl_e.as<__nv_bfloat16>() + emap[elist[i]->E].first, elist[i]->Tin, elist[i]->n, 0,
                                pad8(elist[i]->Tin), 0, NS, ne, TBN));
    }
    std::vector<KSeg> ks;
    ks.reserve(segs.size());
    for (const auto& sg : segs)
        ks.push_back({wmi[wmap[sg.W].second], emi[emap[sg.E].second], 0, 0, sg.Tin, 1, 2, (sg.Tin + BK - 1) / BK});
    std::vector<Work> works;
    for (const auto& tk : tasks) {
        int nchunk = 0;
        for (int i = tk.seg0; i < tk.seg0 + tk.nseg; ++i) nchunk += ks[i].nchunk;
        for (int m0 = 0; m0 < tk.M; m0 += BM)
            for (int n0 = 0; n0 < tk.N; n0 += TBN) {
                Work w{};
                w.m0 = m0;
                w.n0 = n0;
                w.M = tk.M;
                w.N = tk.N;
                w.seg0 = tk.seg0;
                w.nseg = tk.nseg;
                w.c0 = 0;
                w.c1 = nchunk;
                w.out_kind = 2;
                w.promote = 1;
                w.ldo = tk.ldc;
                w.ncols = tk.ncols;
                w.ldr = tk.ldr;
                w.out = tk.C;
                works.push_back(w);
            }
    }
    if (works.empty()) return;
    auto longer = [](const Work& x, const Work& y) { return x.c1 - x.c0 > y.c1 - y.c0; };
    std::stable_sort(works.begin(), works.end(), longer);
    DevBuf dmaps, dsegs, dworks;
    upload_vec(dmaps, maps, st);
    upload_vec(dsegs, ks, st);
    upload_vec(dworks, works, st);
    int dev = 0, nsm = 152;
    GBD_CHECK_CUDA(cudaGetDevice(&dev));
    GBD_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    GBD_CHECK_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<1, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        KT<1, 3>::SMEM_BYTES));
    const int nwk = int(works.size());
    tc_gemm_kernel<1, 3><<<std::min(nwk, std::max(nsm, 1)), THREADS, KT<1, 3>::SMEM_BYTES, st>>>(
        dworks.as<Work>(), nwk, dsegs.as<KSeg>(), dmaps.as<CUtensorMap>(), C.env_err.as<int>());
    count_launch();
    GBD_CHECK_CUDA(cudaGetLastError());
    GBD_CHECK_CUDA(cudaStreamSynchronize(st));  // the tables above are freed on return
    C.env_sl_w.release();  // sliced operands go back to the block cache
    C.env_sl_e.release();
    int e = 0;
    GBD_CHECK_CUDA(cudaMemcpy(&e, C.env_err.p, sizeof(int), cudaMemcpyDeviceToHost));
    GBD_REQUIRE(e == 0, GBD_ERR_CUDA, "tensor-core enlargement stopped on a bounded wait (code " + std::to_string(e) + ")");
}

int tc_error(Ctx& C) {
    int e = 0;
    if (C.H.tc.err.p) GBD_CHECK_CUDA(cudaMemcpy(&e, C.H.tc.err.p, sizeof(int), cudaMemcpyDeviceToHost));
    return e;
}

}  // namespace gbd
