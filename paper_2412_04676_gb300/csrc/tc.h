// tc.h -- H_eff products on the fifth-generation tensor cores (tcgen05 +
// TMEM, TMA) in two forms:
//   mode 0 (BF16x3): x = hi + lo elementwise, products hh + hl + lh, FP32
//                    accumulation, ~1e-5 relative accuracy; the cheap product
//                    of the mixed-precision Davidson iterations.
//   mode 1 (sliced): error-free splitting of every operand row, per 64-wide K
//                    block, into four BF16 slices on a common power-of-two
//                    grid (the splitting of Ozaki et al., as used for tensor
//                    cores by Mukunoki et al.); the ten slice products of
//                    orders <= 4 go to three TMEM accumulators, the two
//                    leading orders of which add up exactly in FP32.  About
//                    2^-30 relative to the row maxima: the anchor products of
//                    the mixed-precision Davidson.
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
constexpr int BK = 64;        // K elements per pipeline stage (one 128-byte swizzle row)
constexpr int MAX_STAGES = 3;
constexpr int EPI_WARPS = 16;                // four per TMEM lane quadrant
constexpr int EPI_THREADS = EPI_WARPS * 32;
constexpr int THREADS = 64 + EPI_THREADS;    // warp 0 TMA, warp 1 MMA, then the epilogue warps

// per-mode tile shape: slices per operand, tile columns, TMEM columns per
// buffer, pipeline stages (as many as fit in shared memory)
// BN2 / BUFCOLS2 / TMEM_COLS2: the phase-2 tile of the form (BF16x3: 256
// columns, so a sector of up to 256 columns reads its X rows once).
template <int MODE> struct ModeCfg;
template <> struct ModeCfg<0> {
    static constexpr int NS = 2, BN = 128, BUFCOLS = 128, TMEM_COLS = 256, STAGES = 3;
    static constexpr int BN2 = 256, BUFCOLS2 = 256, TMEM_COLS2 = 512;
};
template <> struct ModeCfg<1> {
    static constexpr int NS = 4, BN = 64, BUFCOLS = 256, TMEM_COLS = 512, STAGES = 2;
    static constexpr int BN2 = 64, BUFCOLS2 = 256, TMEM_COLS2 = 512;
};

// One K segment: chunks over layers t < T and inner offsets j0 < K step BK.
struct KSeg {
    int mapA, mapB;   // tensor-map index of each operand (slice planes are its outer dimension)
    int a_row, b_row; // row coordinate of the tile origin's operand rows
    int K, T;
    int rank;         // 2 (no layer dimension) or 3, not counting the slice-plane dimension
    int nchunk;       // T * ceil(K / BK)
};

// One work item: an output tile and a contiguous range of K chunks.
struct Work {
    int m0, n0;
    int M, N;          // valid rows / cols of the whole output (bounds)
    int seg0, nseg;
    int c0, c1;        // chunk range over the concatenated segments
    int out_kind;      // 0: FP32-pair partial tile, 1: BF16 slice planes, 2: FP64 matrix (phase kernels 2, 1, 3)
    int promote;       // chunks between promotions of the TMEM accumulators
    long long ldo;     // output row pitch (elements)
    long long plane;   // element distance between BF16 slice planes (kind 1)
    // kind 1 with layer-concatenated output: output row t * lay_rows + r goes
    // to row r at column offset t * lay_pitch (lay_rows = 0: plain rows)
    int lay_rows;
    int colcap;        // kind 1: columns written per row (per layer)
    long long lay_pitch;
    // kind 2: column e of a row goes to (e / ncols) * ldr + e % ncols (ncols = 0: e)
    int ncols;
    long long ldr;
    int omap;          // kind 1, BF16x3: tensor map of the output X for the tile stores
    void* out;
};

// One segment of the fused BF16x3 product: a (class, left block, right
// block) pair feeding one output sector.  Its chunks run over the layers
// t < T and over column blocks of FN columns of the input right sector; a
// chunk computes X_t(rows of the tile, FN columns) = O^Lx_t psi on the
// tensor cores (K = mLi) and multiplies it at once into the output tile
// (K = FN), so X never leaves the SM.
constexpr int FN = 64;
struct FSeg {
    int mapL;          // O^Lx block: dims (mLi, mLo, T), layer-stacked rows
    int mapP;          // psi^T of the input sector: dims (mLi, mRi)
    int mapR;          // O^xR block: dims (mRi, T, mRo), layers side by side along each row
    int mLi, mRi, T;
    int nk1;           // ceil(mLi / BK): K chunks of one X chunk
    int ncol;          // ceil(mRi / FN): column blocks per layer
    int nchunk;        // T * ncol
};

// Sum of split-K partial tiles into one FP64 output tile.
struct Reduce {
    double* out;
    long long ldo;
    int m0, n0, M, N;
    int p0, p1;        // partial tiles [p0, p1)
    int bn;            // tile columns
    int pairs;         // 1: partial elements are FP32 (hi, lo) pairs; 0: FP32 sums
};

}  // namespace tc

// Phase-2 work-list shape (autotuned for the BF16x3 form).
struct TuneParams {
    int split_per_sm = 4;  // split-K work items per SM
    int order = 0;         // 0: items K range by K range across a sector's tiles, 1: tile by tile
};

// Autotuner state of the position: candidate times, choice, histogram key.
struct TcTune {
    bool active = false;     // still trying candidates
    bool from_cache = false; // choice taken from an earlier position with the same key
    int cur = -1;            // candidate the current work list uses (-1: fixed default)
    int chosen = -1;
    double ms[8] = {0};
    int hist[16] = {0};      // sectors per max(rows, cols) / 64 bin
    unsigned long long key = 0;
};

// Device data of one product form: slice planes, tensor maps, work lists.
struct TcPlan {
    bool built = false;                         // work lists, tensor maps, psi planes
    bool ops_l = false, ops_r = false;          // operator planes of O^Lx / O^xR
    bool ops(int side) const { return side == 0 ? ops_l : ops_r; }
    long long nL = 0, nR = 0, np = 0, nx = 0;  // plane strides (elements) of the operator / psi / X slices
    DevBuf ol, orr, psi;                        // BF16 slice planes
    DevBuf maps;                                // CUtensorMap array (64-byte aligned entries)
    DevBuf w1, s1, w2, s2, red, partial;        // work lists, segments, reductions, split-K partials
    DevBuf psi_split;                           // splitting descriptors of psi^T (one per sector)
    int n_w1 = 0, n_w2 = 0, n_red = 0, n_psi = 0;
    double bytes_ops = 0.0;                     // operator slice bytes
    double issued_p1 = 0.0, issued_p2 = 0.0;    // tensor-core GFLOP issued per product
    bool fused = false;                         // BF16x3: one fused kernel (s2 holds FSeg), no phase 1
    std::vector<tc::KSeg> s2_host;              // phase-2 segments per pair (host, for re-planning)
    std::vector<tc::FSeg> f_host;               // fused segments per pair (host, for re-planning)
    std::vector<std::vector<int>> seg_of_out;   // phase-2 segments of each output sector
};

struct TcHeff {
    TcPlan pl[2];
    DevBuf x;                               // phase-1 output X, shared by both forms
    TcTune tune;                            // BF16x3 phase-2 autotuner
    bool low_mem = false;                   // FP64 enlarged arenas released after the planes were built
    bool want_fused = false;                // the next BF16x3 plan: the fused kernel (set per product)
    // psi split plan: per sector source / destination offsets
    struct PsiSec { long long src, dst; int mL, mR, ldp; };
    std::vector<PsiSec> psec;
    DevBuf err;                             // device error word
    int n_sm = 152;
    DevBuf ren_u, ren_t;                    // sliced U^T and tmp^T of the renormalisation
    GemmPlan blk_a, blk_b;                  // FP64 block-Hamiltonian terms (mode 0, optional)
    DevBuf blk_x;
    bool blk = false;
};

struct OpSet;
struct Iso;

// Dense enlargement GEMMs (Sec. II.B step 1) for the sliced tensor-core form:
// C[c][e] = sum over segments of sum_a W[a][c] E[a][e], W: [Tin][Tout] and
// E: [Tin][n] FP64 (device); element e of the output row c sits at
// C + c * ldc + (e / ncols) * ldr + e % ncols.
struct TcEnlSeg { const double* W; int Tin, Tout; const double* E; long long n; };
struct TcEnlTask { double* C; long long ldc, ldr; int M, N, ncols; int seg0, nseg; };

void tc_prepare(Ctx& C, int mode);
void tc_release_products(Ctx& C);
void tc_tune_step(Ctx& C, double ms);       // after each BF16x3 product
void tc_tune_info(Ctx& C, gbd_tune_info* out);
void tc_tune_reset();                       // forgets every cached choice
void tc_apply(Ctx& C, int mode);
int tc_error(Ctx& C);
bool tc_renormalize(Ctx& C, const OpSet& O, const Iso& U, OpSet& out, const std::vector<long long>& toff, double* tmp);
void tc_enlarge_dense(Ctx& C, const std::vector<TcEnlTask>& tasks, const std::vector<TcEnlSeg>& segs);

}  // namespace gbd
