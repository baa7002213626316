// split.cu -- operand splitting kernel of the tensor-core product forms.
#include "split.h"

#include <cstdint>

#include "core.h"
#include "kernels.h"

namespace gbd {
namespace tc {

namespace {

__device__ __forceinline__ float pow2f(int e) {
    return (e >= -126 && e <= 127) ? __int_as_float((e + 127) << 23) : ldexpf(1.f, e);
}

// Two adjacent BF16 values: one 4-byte store where the address allows it.
__device__ __forceinline__ void store_pair(__nv_bfloat16* p, __nv_bfloat16 a, __nv_bfloat16 b) {
    if ((reinterpret_cast<uintptr_t>(p) & 3) == 0) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __halves2bfloat162(a, b);
    } else {
        p[0] = a;
        p[1] = b;
    }
}

// MODE 0: BF16x3 planes, MODE 1: sliced planes, MODE 2: both from one read
// of the source (blocks: the BF16x3 destinations, blocks2: the sliced ones,
// descriptor i of both over the same source units).  Lane gl of a group
// handles columns c0 + 2 gl and c0 + 2 gl + 1 of its unit (ldd is a
// multiple of 8, so both are valid or neither).
template <int MODE>
__global__ void split_kernel(const SplitDesc* __restrict__ blocks, const SplitDesc* __restrict__ blocks2) {
    const SplitDesc b = blocks[blockIdx.x];
    const int nb64 = (b.ldd + 63) >> 6;
    const int G = b.ldd > 16 ? 32 : (b.ldd > 8 ? 16 : 8);
    const int upw = 32 / G;  // units per warp and iteration
    const int units = int(b.rows) * nb64;  // a descriptor covers at most max(kSplitUnits, nb64) units
    const int lane = threadIdx.x & 31, sub = lane / G, gl = lane % G;
    const int nw = blockDim.x >> 5;
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(b.src);
    // destination row offset of source row r of a descriptor (regrouped rows: block rows < 2^31)
    auto dest = [](const SplitDesc& d, int r) {
        const long long ra = d.rbase + r;
        if (d.lpitch != 0) {
            const int t = int(ra) / int(d.R);
            return d.dst + (long long)t * d.lpitch + (ra - (long long)t * d.R) * d.rpitch;
        }
        return d.dst + ra * d.rpitch;
    };
    // kInflight units per lane group and iteration: all their loads are
    // issued before any is processed, so each warp keeps several 512-byte
    // row segments in flight
    constexpr int kInflight = 4;
    for (int ub = (threadIdx.x >> 5) * upw * kInflight; ub < units; ub += nw * upw * kInflight) {
        unsigned long long bw[kInflight][2];
        int rf[kInflight], cf[kInflight];  // row and column block of each unit (one division per group)
        {
            const int u = ub + sub;
            int r = u / nb64, cb = u - r * nb64;
#pragma unroll
            for (int f = 0; f < kInflight; ++f) {
                rf[f] = r;
                cf[f] = cb;
                cb += upw;  // the next unit of this lane group: upw units further
                while (cb >= nb64) { cb -= nb64; ++r; }
            }
        }
#pragma unroll
        for (int f = 0; f < kInflight; ++f) {
            const int u = ub + f * upw + sub;
            const bool uv = u < units;
            const int r = uv ? rf[f] : 0;
            const int c0 = uv ? cf[f] * 64 : 0;
            const int c = c0 + 2 * gl;
            const bool cv = uv && c < c0 + 64 && c < b.ldd;
#pragma unroll
            for (int h = 0; h < 2; ++h) bw[f][h] = (cv && c + h < b.cols) ? src[r * b.rs + (long long)(c + h) * b.cs] : 0ULL;
        }
#pragma unroll
        for (int f = 0; f < kInflight; ++f) {
            const int u = ub + f * upw + sub;
            const bool uv = u < units;
            const int r = uv ? rf[f] : 0;
            const int c0 = uv ? cf[f] * 64 : 0;
            const int c = c0 + 2 * gl;
            const bool cv = uv && c < c0 + 64 && c < b.ldd;
            const unsigned long long* bits = bw[f];
            if constexpr (MODE == 0 || MODE == 2) {
                if (cv) {
                    __nv_bfloat16 hi[2], lo[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float x = __double2float_rn(__longlong_as_double((long long)bits[h]));
                        hi[h] = __float2bfloat16_rn(x);
                        lo[h] = __float2bfloat16_rn(x - __bfloat162float(hi[h]));
                    }
                    __nv_bfloat16* d = dest(b, r) + c;
                    store_pair(d, hi[0], hi[1]);
                    store_pair(d + b.plane, lo[0], lo[1]);
                }
            }
            if constexpr (MODE == 1 || MODE == 2) {
                const SplitDesc& e = MODE == 2 ? blocks2[blockIdx.x] : b;
                // block maximum: non-negative doubles order like their bit
                // patterns; only its exponent is used, and that sits in the
                // high 32 bits, so the group reduces those
                unsigned int mag = max(unsigned(bits[0] >> 32) & 0x7FFFFFFFu, unsigned(bits[1] >> 32) & 0x7FFFFFFFu);
                for (int o = G / 2; o > 0; o >>= 1) mag = max(mag, __shfl_xor_sync(0xffffffffu, mag, o));
                const int emax = int(mag >> 20);  // biased exponent of the maximum
                const int ex = emax - 1022;       // max < 2^ex
                if (cv) {
                    float sc[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) sc[k] = pow2f(ex - 8 * (k + 1));
                    __nv_bfloat16 sl[4][2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const unsigned long long w = bits[h];
                        const int E = int((w >> 52) & 0x7FF);
                        long long q = 0;
                        if (emax > 0 && E > 0) {
                            // x = M 2^(E-1075), q = round(M 2^-s) with s = 21 + (emax - E) >= 21
                            const unsigned long long M = (w & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
                            const int sh = 21 + (emax - E);
                            q = sh >= 64 ? 0 : (long long)((M + (1ULL << (sh - 1))) >> sh);
                            if (w >> 63) q = -q;
                        }
                        // |q| <= 2^32: the digits and every remainder after
                        // the first fit in 32-bit integers
                        const int m1 = int((q + (1LL << 23)) >> 24);
                        int rem = int(q - ((long long)m1 << 24));
                        const int m2 = (rem + (1 << 15)) >> 16;
                        rem -= m2 << 16;
                        const int m3 = (rem + (1 << 7)) >> 8;
                        const int m4 = rem - (m3 << 8);
                        sl[0][h] = __float2bfloat16_rn(float(m1) * sc[0]);
                        sl[1][h] = __float2bfloat16_rn(float(m2) * sc[1]);
                        sl[2][h] = __float2bfloat16_rn(float(m3) * sc[2]);
                        sl[3][h] = __float2bfloat16_rn(float(m4) * sc[3]);
                    }
                    __nv_bfloat16* d = dest(e, r) + c;
#pragma unroll
                    for (int k = 0; k < 4; ++k) store_pair(d + k * e.plane, sl[k][0], sl[k][1]);
                }
            }
        }
    }
}

}  // namespace

void launch_split(int form, const SplitDesc* d0, const SplitDesc* d1, unsigned nblocks, cudaStream_t st) {
    if (nblocks == 0) return;
    if (form == 0) split_kernel<0><<<nblocks, 256, 0, st>>>(d0, nullptr);
    else if (form == 1) split_kernel<1><<<nblocks, 256, 0, st>>>(d0, nullptr);
    else split_kernel<2><<<nblocks, 256, 0, st>>>(d0, d1);
    count_launch();
}

}  // namespace tc
}  // namespace gbd
