// fft_tc.cuh -- split-precision radix-16 passes on the fifth-generation tensor
// cores (tcgen05, sm_103a).
//
// One radix-16 pass over B butterflies is a real matrix product
//
//     D[m][n] = sum_k X[m][k] F[n][k],   m < B,  k, n < 32,
//
// with row m the 16 complex inputs of butterfly m (after the inter-pass
// twiddles) as 32 reals, k = 2 r + {re, im}, and F the 32 x 32 real form of
// the 16-point DFT (n < 16: real part of output s = n, n >= 16: imaginary part
// of output s = n - 16; see split_b_matrix in kernels_split.cu).  Both X and F
// are split into FP16 hi + lo parts and D = X_hi F_hi + X_hi F_lo + X_lo F_hi
// accumulates in FP32 (about 22 significant bits), each butterfly's inputs
// first scaled by a power of two into [2^12, 2^13).
//
// Thread t of the CTA owns butterfly t: it reads and scales its inputs, writes
// row t of X_hi and X_lo into shared memory in the tensor cores' canonical
// K-major layout (8-row x 16-byte core matrices; core (row group g, k group c)
// at g * 512 + c * 128 bytes, so the leading-dimension offset -- between k
// groups -- is 128 B and the stride offset -- between row groups -- 512 B), one
// thread issues the MMAs (M = 128 rows per block, N = 32, K = 16 per
// instruction: 2 k-steps x 3 products), tcgen05.commit signals an mbarrier,
// and each warp reads its 32 rows of D from tensor memory (warp w: lanes
// 32 (w mod 4) .., columns 32 (w div 4) ..).  X is staged in a shared tile the
// pass no longer needs (its source after every thread has read its inputs),
// which holds exactly 128 bytes per butterfly.
#pragma once

#include <cuda_fp16.h>

#include "fft_split.cuh"

namespace afft {

constexpr int kTcBBytes = 2 * 32 * 64;          // F_hi then F_lo, 32 rows x 64 bytes each
constexpr int kTcTableBytes = 2 * kTcBBytes;    // both directions (forward, then backward)

// Per-CTA state of the tensor-core passes (static shared memory of the kernels that use them).
struct TcState {
    unsigned long long bar;      // signalled by tcgen05.commit when a pass's MMAs are done
    unsigned tmem;               // tensor memory base (lane 0, first allocated column)
    unsigned ncols;              // columns allocated (0: none; the passes fall back to mma.sync)
    unsigned phase;              // parity of the next completion of `bar`
    unsigned ok;                 // 0 after a wait that ran out
    unsigned char b[kTcBBytes] __attribute__((aligned(128)));   // this direction's F_hi, F_lo
};

__device__ __forceinline__ TcState &tc_state()
{
    __shared__ __align__(128) TcState s;
    return s;
}

__device__ __forceinline__ unsigned tc_smem_addr(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: canonical K-major layout without swizzle, start address,
// leading-dimension (k group) and stride (row group) byte offsets in 16-byte units, the
// descriptor version 1 of this architecture at bits 46-47.
__device__ __forceinline__ unsigned long long tc_desc(unsigned saddr, unsigned lbo, unsigned sbo)
{
    return (unsigned long long)((saddr & 0x3FFFFu) >> 4) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), FP16 A and B (bits
// 7-12 = 0), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr unsigned tc_idesc(int M, int N)
{
    return (1u << 4) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(unsigned dtmem, unsigned long long adesc, unsigned long long bdesc,
                                       unsigned idesc, unsigned accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned long long *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     tc_smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_proxy() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's lane (the load and its wait in one statement,
// so that nothing reads the registers before they are written).
__device__ __forceinline__ void tc_ld32(unsigned taddr, float (&d)[32])
{
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) d[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ bool tc_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(tc_smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait (about 2 s of %globaltimer) for the given phase of the MMA barrier.
__device__ __forceinline__ bool tc_wait(unsigned long long *bar, unsigned parity)
{
    if (tc_try_wait(bar, parity)) return true;
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (unsigned it = 1;; ++it) {
        if (tc_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0) {
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t - t0 > 2000000000ull) return false;
        }
    }
}

// Kernel prologue of CTAs whose radix-16 passes may run on the tensor cores: warp 0 allocates
// `ncols` tensor-memory columns (a power of two from 32 to 512; 0: none, the passes then use
// mma.sync), the mbarrier is initialised and this direction's F_hi, F_lo (kTcBBytes, already
// in the canonical layout) are copied into shared memory.  Every thread of the CTA must call
// it; it ends with a barrier.
__device__ __forceinline__ void tc_setup(const unsigned char *btab, unsigned ncols)
{
    TcState &st = tc_state();
    if (ncols != 0 && threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_addr(&st.tmem)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem_addr(&st.bar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        st.ncols = ncols;
        st.phase = 0;
        st.ok = 1;
    }
    const uint4 *src = reinterpret_cast<const uint4 *>(btab);
    uint4 *dst = reinterpret_cast<uint4 *>(st.b);
    for (int i = threadIdx.x; i < kTcBBytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    tc_fence_proxy();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// Kernel epilogue: every thread calls it once its tensor-core passes are done (or abandoned);
// warp 0 frees the columns.
__device__ __forceinline__ void tc_teardown()
{
    TcState &st = tc_state();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32 && st.ncols)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(st.tmem), "r"(st.ncols) : "memory");
}

// Whether a pass over `total` butterflies can run here: the CTA holds tensor memory, has a
// whole number of 128-thread groups covering every butterfly, and the butterflies fill whole
// 128-row blocks (the staging tile holds 128 bytes per butterfly).
__device__ __forceinline__ bool tc_usable(int total)
{
    const TcState &st = tc_state();
    return st.ncols != 0 && st.ok && (blockDim.x & 127) == 0 && total <= (int)blockDim.x && (total & 127) == 0 &&
           (unsigned)(total / 128) * 32u <= st.ncols;
}

// One radix-16 pass (Stockham: butterfly j of line l reads positions j + r nb, r < 16, and
// writes (j - j mod Ns) 16 + j mod Ns + s Ns) with the products on the tensor cores.  stage:
// shared memory of at least total * 128 bytes that may be overwritten once every thread has
// read its inputs (the source tile itself is fine).
template <int S, bool TwSmem = false, class Map, class Src, class Dst>
__device__ __forceinline__ void tc16_pass(int n, int Ns, const float2 *__restrict__ tw, int lines, const Map &map,
                                          const Src &src, const Dst &dst, void *stage)
{
    TcState &st = tc_state();
    const int tid = threadIdx.x;
    const int nb = n / 16, total = lines * nb;
    const unsigned phase = st.phase;
    unsigned hi[16], lo[16];
    float inv = 1.f;
    int l = -1, j = 0;
    if (tid < total) {
        map(tid, nb, l, j);
        float2 x[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) x[r] = src(l, j + r * nb);
        if (Ns > 1) {
            const float2 *w = tw + (j % Ns) * 15;
#pragma unroll
            for (int r = 1; r < 16; ++r) x[r] = ctw<S>(x[r], tw_ld<TwSmem>(w + r - 1));
        }
        float m = 0.f;
#pragma unroll
        for (int r = 0; r < 16; ++r) m = fmaxf(m, fmaxf(fabsf(x[r].x), fabsf(x[r].y)));
        float sc;
        split_scale(m, sc, inv);
#pragma unroll
        for (int r = 0; r < 16; ++r) split_half2(make_float2(x[r].x * sc, x[r].y * sc), hi[r], lo[r]);
    } else {
#pragma unroll
        for (int r = 0; r < 16; ++r) hi[r] = lo[r] = 0u;
    }
    __syncthreads();   // every input is read: the stage may be overwritten
    if (tid == 0) st.phase = phase ^ 1u;   // every thread has its copy of the current parity
    // row tid of X_hi (block b at stage + b 16 KB) and of X_lo (8 KB after it)
    if (tid < total) {
        unsigned char *blk = reinterpret_cast<unsigned char *>(stage) + (tid >> 7) * 16384;
        const int m = tid & 127;
        unsigned char *row = blk + (m >> 3) * 512 + (m & 7) * 16;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            *reinterpret_cast<uint4 *>(row + c * 128) = make_uint4(hi[4 * c], hi[4 * c + 1], hi[4 * c + 2], hi[4 * c + 3]);
            *reinterpret_cast<uint4 *>(row + 8192 + c * 128) =
                make_uint4(lo[4 * c], lo[4 * c + 1], lo[4 * c + 2], lo[4 * c + 3]);
        }
    }
    tc_fence_proxy();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const int nblk = total >> 7;
    if (tid == 0) {
        constexpr unsigned idesc = tc_idesc(128, 32);
        const unsigned sa = tc_smem_addr(stage), sb = tc_smem_addr(st.b);
        for (int b = 0; b < nblk; ++b) {
            const unsigned d = st.tmem + 32u * (unsigned)b;
            const unsigned ah = sa + 16384u * (unsigned)b, al = ah + 8192u;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const unsigned long long a_hi = tc_desc(ah + 256u * ks, 128, 512), a_lo = tc_desc(al + 256u * ks, 128, 512);
                const unsigned long long b_hi = tc_desc(sb + 256u * ks, 128, 512),
                                         b_lo = tc_desc(sb + 2048u + 256u * ks, 128, 512);
                tc_mma(d, a_hi, b_hi, idesc, ks > 0);
                tc_mma(d, a_hi, b_lo, idesc, 1u);
                tc_mma(d, a_lo, b_hi, idesc, 1u);
            }
        }
        tc_commit(&st.bar);
    }
    const bool done = tc_wait(&st.bar, phase);
    tc_fence_after();
    if (!done && tid == 0) st.ok = 0;
    const int warp = tid >> 5;
    float d[32];
    if ((warp >> 2) < nblk) {   // warp-uniform: warp w reads lanes 32 (w mod 4) of block w div 4
        tc_ld32(st.tmem + ((unsigned)(32 * (warp & 3)) << 16) + 32u * (unsigned)(warp >> 2), d);
    }
    if (tid < total) {
        const int k = j % Ns;
        const int o = (j - k) * 16 + k;
#pragma unroll
        for (int s = 0; s < 16; ++s) dst(l, o + s * Ns, make_float2(d[s] * inv, d[16 + s] * inv));
    }
    tc_fence_before();
    __syncthreads();   // the tensor memory and the stage are free again
    tc_fence_after();
}

// Columns a CTA of `threads` threads needs: 32 per 128-thread group, as a power of two; 0 when
// the CTA is not a whole number of such groups.
__host__ __device__ constexpr unsigned tc_cols_for(int threads)
{
    return (threads % 128 != 0 || threads > 512) ? 0u
           : threads <= 128                      ? 32u
           : threads <= 256                      ? 64u
                                                 : 128u;
}

}  // namespace afft
