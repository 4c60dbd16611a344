// fft_split.cuh -- split-precision radix-16 passes on the tensor cores.
//
// A radix-16 Stockham pass applies the 16-point DFT matrix F (F[s][r] =
// exp(S 2 pi i s r / 16)) to 16-element columns x (after the inter-pass
// twiddles).  Written over reals, with the 16 complex inputs of a butterfly
// interleaved (k = 2r + {re, im}) and the outputs split into a block of real
// parts (rows s) and a block of imaginary parts, this is a 32x32 real matrix
// A times a 32 x (butterflies) matrix B:
//
//   re block: A[s][2r] =  cos t,   A[s][2r+1] = -S sin t      (t = 2 pi s r / 16)
//   im block: A[s][2r] =  S sin t, A[s][2r+1] =  cos t
//
// Each warp multiplies 8 butterflies at a time with mma.m16n8k16 (FP16 inputs,
// FP32 accumulation): 2 row blocks x 2 k-steps.  To keep about 22 significant
// bits, both operands are split into FP16 hi + lo parts and the product is
// A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped A_lo B_lo term is ~2^-22
// relative).  Before the split, every butterfly's 16 values are scaled by a
// power of two that puts their largest component in [2^12, 2^13) (FP16 holds
// up to 65504), and the outputs are scaled back exactly.
//
// Fragment layout of mma.m16n8k16 (lane = 4 g + q): A regs i = 0..3 hold
// rows g + 8 (i & 1), columns 2q + 8 (i >> 1) + {0, 1}; B regs hold rows
// 2q + {0, 1} and 2q + 8 + {0, 1} of column g; D holds rows g, g + 8 of
// columns 2q, 2q + 1.  With the interleaved k, lane (g, q) therefore loads the
// complex inputs r = q, q + 4, q + 8, q + 12 of butterfly g and receives the
// outputs s = g, g + 8 of butterflies 2q and 2q + 1.
#pragma once

#include <cuda_fp16.h>

#include "fft_access.cuh"

namespace afft {

// Per-lane A fragments of one direction: 16 hi words then 16 lo words, word
// (mt * 2 + ks) * 4 + i for row block mt (0 re, 1 im), k-step ks, register i.
constexpr int kMmaWordsPerLane = 32;
constexpr int kMmaTableWords = 2 * 32 * kMmaWordsPerLane;   // [direction][lane][word]

__device__ __forceinline__ void mma_f16_16816(float d[4], const unsigned a[4], unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned pack_half2(__half2 h) { return *reinterpret_cast<unsigned *>(&h); }

// hi + lo FP16 split of a (scaled) complex value, packed (re low, im high).
__device__ __forceinline__ void split_half2(float2 v, unsigned &hi, unsigned &lo)
{
    const __half2 h = __floats2half2_rn(v.x, v.y);
    const float2 f = __half22float2(h);
    hi = pack_half2(h);
    lo = pack_half2(__floats2half2_rn(v.x - f.x, v.y - f.y));
}

// Power-of-two scale putting m (the largest |component|, m >= 0) into
// [2^12, 2^13), and its inverse; exponents are clamped to the normal range.
__device__ __forceinline__ void split_scale(float m, float &sc, float &inv)
{
    int e = ((__float_as_int(m) >> 23) & 0xff) - 127;
    e = m > 0.f ? max(-114, min(e, 127)) : 0;
    sc = __int_as_float((127 + 12 - e) << 23);
    inv = __int_as_float((127 + e - 12) << 23);
}

// One in-place radix-16 pass over the tile behind `sm` (src and dst may alias:
// every read of the CTA precedes the barrier, every write follows it).  The
// CTA covers all lines * n / 16 butterflies with at most 4 groups of 8 per
// warp (the host sizes CTAs so that threads >= butterflies).  frag: the
// fragment table of this direction (32 words per lane).
template <int S, class Map, class Src, class Dst>
__device__ __forceinline__ void mma16_pass(int n, int Ns, const float2 *__restrict__ tw, int lines, const Map &map,
                                           const Src &src, const Dst &dst, const unsigned *__restrict__ frag)
{
    constexpr int G = 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int g = lane >> 2, q = lane & 3;
    const int nb = n / 16;
    const int total = lines * nb;
    unsigned ahi[16], alo[16];
    {
        const uint4 *f4 = reinterpret_cast<const uint4 *>(frag + lane * kMmaWordsPerLane);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint4 h = __ldg(f4 + k), l = __ldg(f4 + 4 + k);
            ahi[4 * k] = h.x, ahi[4 * k + 1] = h.y, ahi[4 * k + 2] = h.z, ahi[4 * k + 3] = h.w;
            alo[4 * k] = l.x, alo[4 * k + 1] = l.y, alo[4 * k + 2] = l.z, alo[4 * k + 3] = l.w;
        }
    }
    float2 y[G][4];
    int ol[G][2], oo[G][2];
#pragma unroll
    for (int gi = 0; gi < G; ++gi) {
        ol[gi][0] = ol[gi][1] = -1;
        oo[gi][0] = oo[gi][1] = 0;
        const int grp = warp + gi * nwarps;
        if (grp * 8 >= total) continue;            // warp-uniform
        // inputs of butterfly g of this group
        const int idx = grp * 8 + g;
        float2 x[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        if (idx < total) {
            int l, j;
            map(idx, nb, l, j);
#pragma unroll
            for (int t = 0; t < 4; ++t) x[t] = src(l, j + (q + 4 * t) * nb);
            if (Ns > 1) {
                const float2 *w = tw + (j % Ns) * 15;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int r = q + 4 * t;
                    if (r > 0) x[t] = ctw<S>(x[t], ldgc(w + r - 1));
                }
            }
        }
        float m = 0.f;
#pragma unroll
        for (int t = 0; t < 4; ++t) m = fmaxf(m, fmaxf(fabsf(x[t].x), fabsf(x[t].y)));
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
        float sc, inv;
        split_scale(m, sc, inv);
        unsigned bh[4], bl[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) split_half2(make_float2(x[t].x * sc, x[t].y * sc), bh[t], bl[t]);
        float d[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
            for (int e = 0; e < 4; ++e) d[mt][e] = 0.f;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const unsigned *ah = ahi + (mt * 2 + ks) * 4, *al = alo + (mt * 2 + ks) * 4;
                mma_f16_16816(d[mt], ah, bh[2 * ks], bh[2 * ks + 1]);
                mma_f16_16816(d[mt], ah, bl[2 * ks], bl[2 * ks + 1]);
                mma_f16_16816(d[mt], al, bh[2 * ks], bh[2 * ks + 1]);
            }
        }
        // outputs s = g, g + 8 of butterflies 2q, 2q + 1 (their scales live in lanes 8q, 8q + 4)
        const float i0 = __shfl_sync(0xffffffffu, inv, 8 * q), i1 = __shfl_sync(0xffffffffu, inv, 8 * q + 4);
        y[gi][0] = make_float2(d[0][0] * i0, d[1][0] * i0);
        y[gi][1] = make_float2(d[0][1] * i1, d[1][1] * i1);
        y[gi][2] = make_float2(d[0][2] * i0, d[1][2] * i0);
        y[gi][3] = make_float2(d[0][3] * i1, d[1][3] * i1);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int bidx = grp * 8 + 2 * q + c;
            if (bidx < total) {
                int l, j;
                map(bidx, nb, l, j);
                const int k = j % Ns;
                ol[gi][c] = l;
                oo[gi][c] = (j - k) * 16 + k;
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int gi = 0; gi < G; ++gi) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (ol[gi][c] >= 0) {
                dst(ol[gi][c], oo[gi][c] + g * Ns, y[gi][c]);
                dst(ol[gi][c], oo[gi][c] + (g + 8) * Ns, y[gi][2 + c]);
            }
        }
    }
}

}  // namespace afft
