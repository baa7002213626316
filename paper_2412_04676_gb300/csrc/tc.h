// tc.h -- mixed-precision (BF16x3 split, FP32 accumulate, FP64 promotion)
// H_eff products on the fifth-generation tensor cores (tcgen05 + TMEM, TMA).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "core.h"
#include "kernels.h"

namespace gbd {

struct Heff;
struct Ctx;

namespace tc {

constexpr int BM = 128;       // tile rows (UMMA M)
constexpr int BN = 128;       // tile cols (UMMA N)
constexpr int BK = 64;        // K elements per pipeline stage (one 128-byte swizzle row)
constexpr int STAGES = 2;
constexpr int EPI_WARPS = 16;                // four per TMEM lane quadrant
constexpr int EPI_THREADS = EPI_WARPS * 32;
constexpr int CP = BN / (EPI_WARPS / 4);     // accumulator columns per epilogue thread
constexpr int THREADS = 64 + EPI_THREADS;    // warp 0 TMA, warp 1 MMA, then the epilogue warps
constexpr int TMEM_COLS = 2 * BN;

// One K segment: chunks over layers t < T and inner offsets j0 < K step BK.
struct KSeg {
    int mapA, mapB;   // tensor-map index of the hi operand; lo is index + 1
    int a_row, b_row; // row coordinate of the tile origin's operand rows
    int K, T;
    int rank;         // 2 (no layer dimension) or 3
    int nchunk;       // T * ceil(K / BK)
};

// One CTA's work: an output tile and a contiguous range of K chunks.
struct Work {
    int m0, n0;
    int M, N;          // valid rows / cols of the whole output (bounds)
    int seg0, nseg;
    int c0, c1;        // chunk range over the concatenated segments
    int out_kind;      // 0: FP64 partial tile, 1: BF16 hi/lo matrix, 2: FP64 matrix
    int promote;       // chunks between FP32 -> FP64 promotions
    long long ldo;
    void* out_hi;
    void* out_lo;
};

// Sum of split-K partial tiles into one FP64 output tile.
struct Reduce {
    double* out;
    long long ldo;
    int m0, n0, M, N;
    int p0, p1;        // partial tiles [p0, p1)
};

}  // namespace tc

struct TcHeff {
    bool built = false;
    DevBuf ol_hi, ol_lo, or_hi, or_lo;      // BF16 operator arenas (rows padded to 8 elements)
    DevBuf psi_hi, psi_lo;                  // BF16 psi^T per sector
    DevBuf x_hi, x_lo;                      // BF16 phase-1 output
    DevBuf maps;                            // CUtensorMap array (64-byte aligned entries)
    DevBuf w1, s1, w2, s2, red, partial;    // work lists, segments, reductions, split-K partials
    DevBuf err;                             // device error word
    int n_w1 = 0, n_w2 = 0, n_red = 0, n_sm = 152;
    // psi split plan: per sector source / destination offsets
    struct PsiSec { long long src, dst; int mL, mR, ldp; };
    std::vector<PsiSec> psec;
    DevBuf psec_dev;
    double bytes_ops = 0.0;                 // BF16 operator bytes (hi + lo)
    GemmPlan blk_a, blk_b;                  // FP64 block-Hamiltonian terms (optional)
    DevBuf blk_x;
    bool blk = false;
};

void tc_prepare(Ctx& C);
void tc_apply(Ctx& C);
int tc_error(Ctx& C);

}  // namespace gbd
