// fft_access.cuh -- tile accessors of the stage kernels.
//
// A tile element is addressed by (l, p): line l of the CTA's tile, position p
// along the line.  Sources return a value (operator()(l, p)), sinks take one
// (operator()(l, p, v)).  Global accessors read and write the caller's arrays;
// shared-memory accessors hold the tile between radix passes.
#pragma once

#include "fft_math.cuh"

namespace afft {

// Shared-memory address and per-thread asynchronous global -> shared copies
// (cp.async; a zero-byte source fills the destination with zeros).
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

template <int BYTES>
__device__ __forceinline__ void cp_async_zfill(void *dst, const void *src, bool valid)
{
    static_assert(BYTES == 8 || BYTES == 16, "cp.async size");
    const int n = valid ? BYTES : 0;
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(n)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(n)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// mbarriers (shared::cta) for the asynchronous copies of the tensor-memory
// accelerator: initialisation, the expected byte count of a phase, and waits
// bounded by %globaltimer.
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the given phase of the barrier for at most limit_ns (default ~2 s).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity,
                                                  unsigned long long limit_ns = 2000000000ull)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0 && global_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void fence_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One-dimensional bulk copy (TMA, no tensor map) of `bytes` from global to
// shared memory, completing on `bar`; both addresses 16-byte aligned, `bytes`
// a multiple of 16.
__device__ __forceinline__ void bulk_load_1d(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// CTA-wide decision after a float-float first pass: keep float-float only if no
// value of the tile was too large and some value was >= 2^-50 (two votes, so
// every thread of the CTA must call it).
__device__ __forceinline__ bool df_tile_ok(const DfFlags &f)
{
    const int large = __syncthreads_or(f.large);
    const int normal = __syncthreads_or(f.normal);
    return !large && normal;
}

template <typename V> __device__ __forceinline__ V czero()
{
    V v{};
    return v;
}

// Shared-memory tile of a strided stage: [n][lines], one 128-byte row per
// line position (conflict-free for line-fast thread maps).
template <typename V> struct SmemRows {
    V *sm;
    int log2_lines;
    __device__ __forceinline__ V operator()(int l, int p) const { return sm[(p << log2_lines) + l]; }
    __device__ __forceinline__ void operator()(int l, int p, V v) const { sm[(p << log2_lines) + l] = v; }
};

// Shared-memory tile of a contiguous stage: [lines][n] with the offset
// XOR-swizzled inside 128-byte rows, so strided pass writes spread over banks.
template <typename V> struct SmemLines {
    V *sm;
    int n;
    static constexpr int kRow = 128 / sizeof(V);
    __device__ __forceinline__ int at(int l, int p) const
    {
        const int e = l * n + p;
        return e ^ ((e / kRow) & (kRow - 1));
    }
    __device__ __forceinline__ V operator()(int l, int p) const { return sm[at(l, p)]; }
    __device__ __forceinline__ void operator()(int l, int p, V v) const { sm[at(l, p)] = v; }
};

// Global accessors store type V and compute in CT (the same, or float-float
// for FP64 data): sources convert on load and record out-of-range values in
// *bad, sinks convert on store.  CG sources load through L2 only (ld.global.cg):
// the persistent executor reads data that other CTAs of the same launch wrote,
// which a copy cached in L1 (or read through the non-coherent path) could miss.
template <bool CG, typename V> __device__ __forceinline__ V ld_data(const V *p)
{
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// Global columns c0 .. c0+lines-1 of a [outer][n][W] slab (strided stage).
template <typename V, typename CT = V, bool CG = false> struct GlobalCols {
    const V *base;                 // &x[o][0][c0]
    long long W;
    int valid;                     // columns of the tile inside the array
    DfFlags *bad;
    __device__ __forceinline__ CT operator()(int l, int p) const
    {
        return l < valid ? Conv<CT, V>::in(ld_data<CG>(base + (long long)p * W + l), bad) : czero<CT>();
    }
};
template <typename V, typename CT = V> struct GlobalColsOut {
    V *base;
    long long W;
    int valid;
    __device__ __forceinline__ void operator()(int l, int p, CT v) const
    {
        if (l < valid) base[(long long)p * W + l] = Conv<CT, V>::out(v);
    }
};

// Output side of a strided tile for passes whose every call comes from the
// thread that owns one column (line-fast maps with a CTA size that is a
// multiple of the tile width): the destination column `col` (or -1 for "not
// stored") is resolved once per tile per thread.
template <typename V, typename CT = V> struct GlobalColFixedOut {
    V *base;                       // &y[o][0][0]
    long long W;                   // output row pitch
    long long col;                 // this thread's output column, -1 to drop
    __device__ __forceinline__ void operator()(int, int p, CT v) const
    {
        if (col >= 0) base[(long long)p * W + col] = Conv<CT, V>::out(v);
    }
};

// Shared-memory rows holding storage values V, read as compute values CT
// (the first pass of a float-float tile that a TMA copy brought in as FP64).
template <typename V, typename CT, int LG> struct SmemRowsConvIn {
    const V *sm;
    DfFlags *bad;
    __device__ __forceinline__ CT operator()(int l, int p) const { return Conv<CT, V>::in(sm[(p << LG) + l], bad); }
};

// Global contiguous lines b0 .. b0+lines-1 of length n (contiguous stage).
template <typename V, typename CT = V> struct GlobalLines {
    const V *base;                 // &x[b0][0]
    int n;                         // line stride in complex elements
    int valid;
    DfFlags *bad;
    __device__ __forceinline__ CT operator()(int l, int p) const
    {
        return l < valid ? Conv<CT, V>::in(base[l * n + p], bad) : czero<CT>();
    }
};
template <typename V, typename CT = V> struct GlobalLinesOut {
    V *base;
    int n;
    int valid;
    typename RealOf<CT>::T scale;  // 1 forward, 1/N for the last backward store
    __device__ __forceinline__ void operator()(int l, int p, CT v) const
    {
        if (l < valid) base[l * n + p] = Conv<CT, V>::out(cscale(v, scale));
    }
};

// c2r: builds Z[k] = E[k] + i O[k] of the half-length complex sequence from
// the half spectrum X[0..M] of a real line of length 2M:
//   E[k] = X[k] + conj(X[M-k]),  O[k] = (X[k] - conj(X[M-k])) w_{2M}^{+k},
// with the imaginary parts of the self-conjugate bins X[0], X[M] dropped.
// (The factor 1/2 of the textbook identity is folded into the 1/N scale.)
template <typename V, typename CT = V, bool CG = false> struct C2RPre {
    const V *base;                 // &X[b0][0]
    const CT *post_tw;             // w_{2M}^k forward, k = 0..M
    int M;
    int ld;                        // line stride (M + 1 for the compact layout)
    int valid;
    DfFlags *bad;
    __device__ __forceinline__ CT operator()(int l, int k) const
    {
        if (l >= valid) return czero<CT>();
        const V *x = base + l * ld;
        CT a = Conv<CT, V>::in(ld_data<CG>(x + k), bad);
        CT b = cconj(Conv<CT, V>::in(ld_data<CG>(x + M - k), bad));
        if (k == 0) {
            a.y = typename RealOf<CT>::T();
            b.y = typename RealOf<CT>::T();
        }
        const CT e = cadd(a, b);
        const CT o = cmulc(csub(a, b), ldgc(post_tw + k));
        return cmk<CT>(e.x - o.y, e.y + o.x);
    }
};


// Four-step split of a line of n = n_a n_b points (j = n_a j_b + j_a,
// k = k_b + n_b k_a): after length-n_b DFTs along j_b, element (j_a, k_b) is
// multiplied by w_n^{j_a k_b} and length-n_a DFTs run along j_a.  FourStepSrc
// reads row j_a of the tile for one k_b and applies that twiddle (conjugated
// for the backward transform); FourStepDst stores DFT output k_a to row
// k_b + n_b k_a of the destination line (the transpose back to natural order).
template <int S, typename V> struct FourStepSrc {
    const V *base;                 // &t[o'][0][c0], o' = (o, k_b)
    long long W;
    int valid;
    const V *wn;                   // w_n^m, m < n (forward sign)
    int kb;
    __device__ __forceinline__ V operator()(int l, int p) const
    {
        if (l >= valid) return czero<V>();
        const V v = base[(long long)p * W + l];
        const V w = ldgc(wn + p * kb);   // p * kb < n_a n_b = n
        return S < 0 ? cmul(v, w) : cmulc(v, w);
    }
};
template <typename V> struct FourStepDst {
    V *base;                       // &y[o][k_b][c0]
    long long Wrow;                // n_b * W: distance between rows k_a and k_a + 1
    int valid;
    typename RealOf<V>::T scale;
    __device__ __forceinline__ void operator()(int l, int p, V v) const
    {
        if (l < valid) base[(long long)p * Wrow + l] = cscale(v, scale);
    }
};

}  // namespace afft
