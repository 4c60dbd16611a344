// fft_stage.cuh -- the kernels of one axis stage of the 3-D FFT.
//
// A stage runs batched 1-D DFTs of length n along one axis: one FFT row of
// Algorithm 1 of AccFFT with P0 = P1 = 1.  Each CTA owns a tile of `lines`
// lines, computes their DFTs with a Stockham autosort FFT and writes them
// back in natural order.  One radix-R pass over a line of n points, with Ns
// the product of the radices already applied and nb = n / R:
//
//   for each butterfly j < nb:  k = j mod Ns
//     v[r] = x[j + r nb] * w_{R Ns}^{r k}                      r = 0..R-1
//     y[(j - k) R + k + s Ns] = sum_r v[r] w_R^{r s}           s = 0..R-1
//
// with w_L = exp(-2 pi i / L) forward and its conjugate backward.  The
// paper's transposes never materialise: a strided stage loads a tile of
// adjacent columns (the paper's "pack" before the exchange is the tile load)
// and stores it back where it came from, so the frequency-domain array keeps
// the spatial xyz layout (the paper's local transpose back to xyz is free).
//
// Two implementations:
//  * specialised kernels, one per line length in AFFT_LINE_PLANS: the radix
//    sequence is a compile-time list, the first pass reads the tile straight
//    from global memory and the last pass writes it straight back (both
//    coalesced), and the passes in between exchange through shared memory;
//  * a generic kernel for every other length: the tile is staged through
//    shared memory and each pass is a separate (non-inlined) function chosen
//    at run time by its radix.
#pragma once

#include <type_traits>

#include "afft_internal.h"
#include "fft_access.cuh"
#include "fft_split.cuh"
#include "fft_tc.cuh"

namespace afft {

// Thread -> (line, butterfly) maps, also used as (line, position) maps by the
// load/store loops of the generic kernel.
struct MapLineFast {   // strided stage: consecutive threads take adjacent columns
    int log2_lines;
    __device__ __forceinline__ void operator()(int idx, int, int &l, int &j) const
    {
        l = idx & ((1 << log2_lines) - 1);
        j = idx >> log2_lines;
    }
};
struct MapButterflyFast {  // contiguous stage: consecutive threads walk along a line
    __device__ __forceinline__ void operator()(int idx, int nb, int &l, int &j) const
    {
        l = idx / nb;
        j = idx - l * nb;
    }
};

// ------------------------------------------------------ one radix pass ------
// Thread t handles butterflies idx = t, t + blockDim.x, ... (at most
// bmax_for_radix(R) of them; the host sizes the CTA so that suffices).  With
// InPlace the pass reads everything into registers, waits for the whole CTA,
// then writes.

template <int R, int S, bool InPlace, int NT = 0, int BM = 0, bool TwSmem = false, typename V, class Map, class Src,
          class Dst>
__device__ __forceinline__ void radix_pass(int n, int Ns, const V *__restrict__ tw, int lines,
                                           const Map &map, const Src &src, const Dst &dst)
{
    constexpr int B = BM > 0 ? BM : bmax_for_radix(R);   // BM: fewer butterflies per thread (larger CTAs)
    const int nthr = NT > 0 ? NT : (int)blockDim.x;  // NT: compile-time CTA size, when known
    const int nb = n / R;
    const int total = lines * nb;
    V v[B][R];
    int lb[B], jb[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int idx = threadIdx.x + b * nthr;
        lb[b] = -1;
        jb[b] = 0;
        if (idx < total) {
            int l, j;
            map(idx, nb, l, j);
            lb[b] = l;
            jb[b] = j;
#pragma unroll
            for (int r = 0; r < R; ++r) v[b][r] = src(l, j + r * nb);
            if (Ns > 1) {
                const V *t = tw + (j % Ns) * (R - 1);
#pragma unroll
                for (int r = 1; r < R; ++r) v[b][r] = ctw<S>(v[b][r], tw_ld<TwSmem>(t + r - 1));
            }
            Dft<R, S, V>::run(v[b]);
        }
    }
    if (InPlace) __syncthreads();
#pragma unroll
    for (int b = 0; b < B; ++b) {
        if (lb[b] >= 0) {
            const int j = jb[b];
            const int k = j % Ns;
            const int o = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) dst(lb[b], o + r * Ns, cnorm(v[b][r]));
        }
    }
}

// ------------------------------------------- specialised pass sequences -----

template <int... Rs> struct Seq {};

template <int N, int... Rs> struct LinePlan {
    static constexpr int n = N;
    static constexpr int npass = sizeof...(Rs);
    using seq = Seq<Rs...>;
};

// One pass of a specialised sequence: radix_pass, or with Split (complex64
// split-precision families) a radix-16 pass on the tensor cores: tcgen05 (fft_tc.cuh) in
// kernels that set up tensor memory, staging in `stage` -- TC = 1: when the tile allows it
// (checked at run time), else mma.sync (fft_split.cuh); TC = 2: always (the kernel's tile
// shape qualifies at compile time).  TwSmem: twiddles from a shared-memory table.
template <int R, int S, bool InPlace, bool Split, int NT = 0, int BM = 0, int TC = 0, bool TwSmem = false,
          typename V, class Map, class Src, class Dst>
__device__ __forceinline__ void spec_pass(int n, int Ns, const V *__restrict__ tw, int lines, const Map &map,
                                          const Src &src, const Dst &dst, const unsigned *mma, void *stage = nullptr)
{
    if constexpr (Split && R == 16 && std::is_same<V, float2>::value) {
        if constexpr (TC == 2) {
            tc16_pass<S, TwSmem>(n, Ns, tw, lines, map, src, dst, stage);
        } else {
            if constexpr (TC == 1) {
                if (tc_usable(lines * (n / 16))) {
                    tc16_pass<S, TwSmem>(n, Ns, tw, lines, map, src, dst, stage);
                    return;
                }
            }
            mma16_pass<S>(n, Ns, tw, lines, map, src, dst, mma + (S < 0 ? 0 : 32 * 32));
        }
    } else {
        radix_pass<R, S, InPlace, NT, BM, TwSmem>(n, Ns, tw, lines, map, src, dst);
    }
}

// Runs passes Seq<R, Rest...> with Ns = product of the earlier radices and
// TwOff = the table offset of this pass (the host lays tables out the same
// way: Ns (R - 1) entries per pass with Ns > 1, in pass order).
template <int S, bool First, bool LastToSmem, int N, int Ns, int TwOff, bool Split, int TC = 0, typename V,
          class Map, class Src, class Sm, class Dst, int R, int... Rest>
__device__ __forceinline__ void run_passes(Seq<R, Rest...>, const V *tw, int lines, const Map &map,
                                           const Src &src, const Sm &sm, const Dst &dst, const unsigned *mma)
{
    constexpr bool Last = sizeof...(Rest) == 0;
    // tensor-core passes stage their operands in the CTA's shared tile (lines * n elements)
    void *stage = nullptr;
    if constexpr (TC) stage = sm.sm;
    if (!First) __syncthreads();
    if constexpr (First && Last) {
        if constexpr (LastToSmem) spec_pass<R, S, false, Split, 0, 0, TC>(N, Ns, tw + TwOff, lines, map, src, sm, mma, stage);
        else spec_pass<R, S, false, Split, 0, 0, TC>(N, Ns, tw + TwOff, lines, map, src, dst, mma, stage);
    } else if constexpr (First) {
        spec_pass<R, S, false, Split, 0, 0, TC>(N, Ns, tw + TwOff, lines, map, src, sm, mma, stage);
    } else if constexpr (Last && !LastToSmem) {
        spec_pass<R, S, false, Split, 0, 0, TC>(N, Ns, tw + TwOff, lines, map, sm, dst, mma, stage);
    } else {
        spec_pass<R, S, true, Split, 0, 0, TC>(N, Ns, tw + TwOff, lines, map, sm, sm, mma, stage);
    }
    if constexpr (!Last) {
        constexpr int next = TwOff + (Ns > 1 ? Ns * (R - 1) : 0);
        run_passes<S, false, LastToSmem, N, Ns * R, next, Split, TC>(Seq<Rest...>{}, tw, lines, map, src, sm, dst, mma);
    }
}

template <class P, int S, bool LastToSmem, bool Split = false, int TC = 0, typename V, class Map, class Src,
          class Sm, class Dst>
__device__ __forceinline__ void run_plan(const V *tw, int lines, const Map &map, const Src &src,
                                         const Sm &sm, const Dst &dst, const unsigned *mma = nullptr)
{
    if constexpr (P::npass == 0) {  // n == 1: a copy
        for (int idx = threadIdx.x; idx < lines; idx += blockDim.x) {
            if constexpr (LastToSmem) sm(idx, 0, src(idx, 0));
            else dst(idx, 0, src(idx, 0));
        }
    } else {
        run_passes<S, true, LastToSmem, P::n, 1, 0, Split, TC>(typename P::seq{}, tw, lines, map, src, sm, dst, mma);
    }
}

// Float-float stage for FP64 data (see dfl): the first pass converts the
// FP64 input on load and records any value outside float-float range; a
// CTA-wide vote then either continues in float-float or reports failure, in
// which case the caller redoes the tile in FP64 (the first pass wrote only
// shared memory, so the input is untouched).  Plans with one pass are not
// eligible (their only pass writes the output).
template <class P, int S, bool LastToSmem, typename CT, class Map, class Src, class Sm, class Dst, int R0,
          int... Rest>
__device__ __forceinline__ bool df_stage_impl(Seq<R0, Rest...>, const CT *tw, int lines, const Map &map,
                                              const Src &src, const Sm &sm, const Dst &dst, const DfFlags &bad)
{
    radix_pass<R0, S, false>(P::n, 1, tw, lines, map, src, sm);
    if (!df_tile_ok(bad)) return false;
    run_passes<S, false, LastToSmem, P::n, R0, 0, false>(Seq<Rest...>{}, tw, lines, map, sm, sm, dst, nullptr);
    return true;
}
template <class P, int S, bool LastToSmem, typename CT, class Map, class Src, class Sm, class Dst>
__device__ __forceinline__ bool df_stage(const CT *tw, int lines, const Map &map, const Src &src, const Sm &sm,
                                         const Dst &dst, const DfFlags &bad)
{
    return df_stage_impl<P, S, LastToSmem>(typename P::seq{}, tw, lines, map, src, sm, dst, bad);
}

// Specialised FP64 kernels with at least two passes compute in float-float.
template <class F, typename V> struct UseDf {
    static constexpr bool value = !F::generic && std::is_same<V, double2>::value && F::plan::npass >= 2;
};

// ------------------------------------------------- generic pass sequence ----
// One non-inlined function per (radix, direction, layout): the tile lives in
// shared memory, so each takes only scalars and keeps its registers to itself.

template <int R, int S, bool Rows, typename V>
__device__ __noinline__ void smem_pass(V *sm, int n, int Ns, const V *tw, int lines, int log2_lines)
{
    if constexpr (Rows) {
        const SmemRows<V> t{sm, log2_lines};
        radix_pass<R, S, true>(n, Ns, tw, lines, MapLineFast{log2_lines}, t, t);
    } else {
        const SmemLines<V> t{sm, n};
        radix_pass<R, S, true>(n, Ns, tw, lines, MapButterflyFast{}, t, t);
    }
}

// Split-precision radix-16 pass (tensor cores, see fft_split.cuh) on the tile.
template <int S, bool Rows>
__device__ __noinline__ void smem_mma16(float2 *sm, int n, int Ns, const float2 *tw, int lines, int log2_lines,
                                        const unsigned *frag)
{
    if constexpr (Rows) {
        const SmemRows<float2> t{sm, log2_lines};
        mma16_pass<S>(n, Ns, tw, lines, MapLineFast{log2_lines}, t, t, frag);
    } else {
        const SmemLines<float2> t{sm, n};
        mma16_pass<S>(n, Ns, tw, lines, MapButterflyFast{}, t, t, frag);
    }
}

template <int S, bool Rows, bool Split, typename V>
__device__ __forceinline__ void smem_pass_any(int R, V *sm, int n, int Ns, const V *tw, int lines,
                                              int log2_lines, const unsigned *mma)
{
    switch (R) {
    case 16:
        if constexpr (Split && std::is_same<V, float2>::value)
            smem_mma16<S, Rows>(sm, n, Ns, tw, lines, log2_lines, mma + (S < 0 ? 0 : 32 * 32));
        else
            smem_pass<16, S, Rows>(sm, n, Ns, tw, lines, log2_lines);
        break;
    case 8: smem_pass<8, S, Rows>(sm, n, Ns, tw, lines, log2_lines); break;
    case 4: smem_pass<4, S, Rows>(sm, n, Ns, tw, lines, log2_lines); break;
    case 2: smem_pass<2, S, Rows>(sm, n, Ns, tw, lines, log2_lines); break;
    case 3: smem_pass<3, S, Rows>(sm, n, Ns, tw, lines, log2_lines); break;
    case 5: smem_pass<5, S, Rows>(sm, n, Ns, tw, lines, log2_lines); break;
    default: break;  // the plan emits only the radices above
    }
}

// Generic stage body: load src -> smem, all passes in smem, store smem -> dst
// (skipped with LastToSmem).  Split: radix-16 passes on the tensor cores.
template <int S, bool Rows, bool LastToSmem, bool Split = false, typename V, class Map, class Src, class Dst>
__device__ __forceinline__ void run_generic(const StageDesc &d, const V *tw, V *sm, int lines,
                                            int log2_lines, const Map &map, const Src &src,
                                            const Dst &dst)
{
    const int n = d.n;
    const int total = lines * n;
    const SmemRows<V> rows{sm, log2_lines};
    const SmemLines<V> cols{sm, n};
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int l, p;
        map(idx, n, l, p);
        if constexpr (Rows) rows(l, p, src(l, p));
        else cols(l, p, src(l, p));
    }
    for (int p = 0; p < d.npass; ++p) {
        __syncthreads();
        smem_pass_any<S, Rows, Split>(d.radix[p], sm, n, d.ns[p], tw + d.tw_off[p], lines, log2_lines, d.mma);
    }
    if constexpr (LastToSmem) return;
    __syncthreads();
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int l, p;
        map(idx, n, l, p);
        if constexpr (Rows) dst(l, p, rows(l, p));
        else dst(l, p, cols(l, p));
    }
}

// ------------------------------------------------------- kernel families ----

// Specialised kernels keep two CTAs per SM resident: 512 threads x 64
// registers for FP32, 256 x 128 for FP64.  Generic kernels use 256 threads
// with the full register file.
template <typename V> struct SpecThreads;
template <> struct SpecThreads<float2> { static constexpr int value = 512; };
template <> struct SpecThreads<double2> { static constexpr int value = 256; };

template <class Plan, bool Split = false> struct Spec {
    static constexpr bool generic = false;
    static constexpr bool split = Split;
    using plan = Plan;
    template <typename V> static constexpr int threads() { return SpecThreads<V>::value; }
    static constexpr int min_blocks = Split ? 1 : 2;   // split: the DFT-16 fragments need 128 registers
};
struct Generic {
    static constexpr bool generic = true;
    static constexpr bool split = false;
    using plan = LinePlan<0>;
    template <typename V> static constexpr int threads() { return 256; }
    static constexpr int min_blocks = 2;
};
// Generic complex64 kernels of split-precision plans: radix-16 passes on the
// tensor cores, otherwise as Generic.
struct GenericSplit {
    static constexpr bool generic = true;
    static constexpr bool split = true;
    using plan = LinePlan<0>;
    template <typename V> static constexpr int threads() { return 256; }
    static constexpr int min_blocks = 1;
};

// ------------------------------------------------------------- kernels ------

// Strided axis: lines run along a [outer][n][W] slab with stride W; the CTA
// takes `lines` adjacent columns of one outer slab.
template <class F, int S, typename V>
__global__ void __launch_bounds__(F::template threads<V>(), F::min_blocks)
    k_strided(const V *__restrict__ in, V *out, const __grid_constant__ StageDesc d,
              const V *__restrict__ tw, long long W, long long tiles_per_outer, int log2_lines)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *sm = reinterpret_cast<V *>(smem_raw);
    const int n = F::generic ? d.n : F::plan::n;
    const int lines = 1 << log2_lines;
    const long long tile = stage_order(blockIdx.x, gridDim.x, d.rev);
    const long long o = tile / tiles_per_outer;
    const long long c0 = (tile - o * tiles_per_outer) * lines;
    const long long off = o * (long long)n * W + c0;
    const int valid = (int)min((long long)lines, W - c0);
    const GlobalCols<V> src{in + off, W, valid};
    const GlobalColsOut<V> dst{out + off, W, valid};
    const MapLineFast map{log2_lines};
    if constexpr (F::generic) {
        run_generic<S, true, false, F::split>(d, tw, sm, lines, log2_lines, map, src, dst);
    } else {
        if constexpr (UseDf<F, V>::value) {
            if (d.twdf) {
                DfFlags bad;
                const GlobalCols<V, dcx> sdf{in + off, W, valid, &bad};
                const GlobalColsOut<V, dcx> ddf{out + off, W, valid};
                const SmemRows<dcx> tdf{reinterpret_cast<dcx *>(sm), log2_lines};
                if (df_stage<typename F::plan, S, false>((const dcx *)d.twdf, lines, map, sdf, tdf, ddf, bad)) return;
            }
        }
        const SmemRows<V> tile{sm, log2_lines};
        run_plan<typename F::plan, S, false, F::split>(tw, lines, map, src, tile, dst, d.mma);
    }
}

// Contiguous axis, complex to complex (x scale at the store).
template <class F, int S, typename V>
__global__ void __launch_bounds__(F::template threads<V>(), F::min_blocks)
    k_contig(const V *__restrict__ in, V *out, const __grid_constant__ StageDesc d,
             const V *__restrict__ tw, long long nlines, int lines, typename RealOf<V>::T scale)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *sm = reinterpret_cast<V *>(smem_raw);
    const int n = F::generic ? d.n : F::plan::n;
    const long long b0 = stage_order(blockIdx.x, gridDim.x, d.rev) * lines;
    const int valid = (int)min((long long)lines, nlines - b0);
    // a blocked layout on either side keeps the CTA's lines consecutive (the host makes `lines`
    // divide the block), so only the first line's position changes
    const long long lb = d.blk ? blocked_line(d, b0) : b0;
    const V *in0 = in + (d.blk && d.blk_in ? lb : b0) * n;
    V *out0 = out + (d.blk && d.blk_out ? lb : b0) * n;
    const GlobalLines<V> src{in0, n, valid};
    const GlobalLinesOut<V> dst{out0, n, valid, scale};
    const MapButterflyFast map{};
    if constexpr (F::generic) {
        run_generic<S, false, false, F::split>(d, tw, sm, lines, 0, map, src, dst);
    } else {
        if constexpr (UseDf<F, V>::value) {
            if (d.twdf) {
                DfFlags bad;
                const GlobalLines<V, dcx> sdf{in0, n, valid, &bad};
                const GlobalLinesOut<V, dcx> ddf{out0, n, valid, dfl(scale)};
                const SmemLines<dcx> tdf{reinterpret_cast<dcx *>(sm), n};
                if (df_stage<typename F::plan, S, false>((const dcx *)d.twdf, lines, map, sdf, tdf, ddf, bad)) return;
            }
        }
        const SmemLines<V> tile{sm, n};
        if constexpr (F::split && std::is_same<V, float2>::value) {
            // split precision: radix-16 passes on tcgen05 (fft_tc.cuh) where the CTA allows
            tc_setup(reinterpret_cast<const unsigned char *>(d.mma) + kMmaTableWords * 4 + (S < 0 ? 0 : kTcBBytes),
                     tc_cols_for((int)blockDim.x));
            run_plan<typename F::plan, S, false, true, 1>(tw, lines, map, src, tile, dst, d.mma);
            tc_teardown();
        } else {
            run_plan<typename F::plan, S, false, F::split>(tw, lines, map, src, tile, dst, d.mma);
        }
    }
}

// The passes of a tile whose input was staged in the work tile itself (src
// reads shared memory): the first pass in place (all reads, a barrier, all
// writes), the rest as usual, the last one writing dst.
template <class P, int S, typename V, class Map, class Src, class Sm, class Dst, int R0, int... Rest>
__device__ __forceinline__ void run_plan_staged(Seq<R0, Rest...>, const V *tw, int lines, const Map &map,
                                                const Src &src, const Sm &sm, const Dst &dst)
{
    if constexpr (sizeof...(Rest) == 0) {
        radix_pass<R0, S, true>(P::n, 1, tw, lines, map, src, dst);
    } else {
        radix_pass<R0, S, true>(P::n, 1, tw, lines, map, src, sm);
        run_passes<S, false, false, P::n, R0, 0, false>(Seq<Rest...>{}, tw, lines, map, sm, sm, dst, nullptr);
    }
}

// Copies `elems` complex values (complex64 or complex128) from global memory
// (16-byte aligned) into shared memory with one bulk copy (an 8-byte load for
// an odd complex64 tail) and waits for them (all threads of the CTA; a
// one-shot mbarrier, the wait bounded).  Returns false, on every thread, if
// the copy did not land in time.
template <typename V>
__device__ __forceinline__ bool stage_contiguous(V *sm, const V *src, int elems)
{
    static_assert(sizeof(V) == 8 || sizeof(V) == 16, "complex64 or complex128");
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned bytes = (unsigned)((size_t)elems * sizeof(V) / 16) * 16u;
        mbar_expect_tx(&bar, bytes);
        bulk_load_1d(sm, src, bytes, &bar);
        if (sizeof(V) == 8 && (elems & 1)) sm[elems - 1] = __ldcg(src + elems - 1);
    }
    const bool ok = mbar_wait_bounded(&bar, 0);
    return __syncthreads_or(!ok) == 0;
}

// The launch's dynamic shared memory in bytes.
__device__ __forceinline__ unsigned dynamic_smem_bytes()
{
    unsigned b;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(b));
    return b;
}

// r2c post-processing of the DFT_M lines in shared memory into M+1 bins per
// line (compute type CT, stored as V):
//   X[k] = E[k] + w_{2M}^k O[k],  E = (Z[k] + conj Z[M-k]) / 2,
//   O = (Z[k] - conj Z[M-k]) / (2i),  Z[M] = Z[0].
// Bins k and M - k share E and O up to conjugation (E[M-k] = conj E[k],
// O[M-k] = conj O[k], w_{2M}^{M-k} = -conj w_{2M}^k), so one thread reads
// Z[k] and Z[M-k] once and writes X[k] = E + t and X[M-k] = conj(E - t) with
// t = w_{2M}^k O[k]; k = 0 gives X[0] and X[M].
template <typename V, typename CT, class Tile>
__device__ __forceinline__ void r2c_post(const Tile &tile, V *o, const CT *post_tw, int M, int ld, int valid)
{
    using T = typename RealOf<CT>::T;
    const int half = M / 2 + 1;
    for (int idx = threadIdx.x; idx < valid * half; idx += blockDim.x) {
        const int l = idx / half;
        const int k = idx - l * half;
        const CT zk = tile(l, k);
        const CT zm = cconj(tile(l, k == 0 ? 0 : M - k));
        const CT e = cscale(cadd(zk, zm), T(0.5));
        const CT dd = csub(zk, zm);
        const CT od = cmk<CT>(T(0.5) * dd.y, T(-0.5) * dd.x);  // (zk - zm) / (2i)
        const CT t = cmul(od, ldgc(post_tw + k));
        V *line = o + l * ld;
        line[k] = Conv<CT, V>::out(cnorm(cadd(e, t)));
        if (2 * k != M) line[k == 0 ? M : M - k] = Conv<CT, V>::out(cnorm(cconj(csub(e, t))));
    }
}

// r2c_post for a compile-time M when the CTA size is a multiple of M/2: thread
// t owns the bin pair k = t mod M/2 (k and M - k) of lines t div M/2, +step,
// ..., so its twiddle is loaded once and no index is divided; k = 0 also
// writes X[M] and X[M/2] = conj Z[M/2] (E = Re Z, O = Im Z, w^{M/2} = -i).
// Returns false, doing nothing, when the CTA size does not fit.
template <int M, typename V, typename CT, class Tile>
__device__ __forceinline__ bool r2c_post_fixed_k(const Tile &tile, V *o, const CT *post_tw, int ld, int valid)
{
    if constexpr (M < 2) {
        return false;
    } else {
        using T = typename RealOf<CT>::T;
        constexpr int H = M / 2;
        const int nthr = blockDim.x;
        if (H > nthr || nthr % H != 0) return false;
        const int k = threadIdx.x % H;
        const int step = nthr / H;
        const CT w = ldgc(post_tw + k);
        for (int l = threadIdx.x / H; l < valid; l += step) {
            V *line = o + l * ld;
            const CT zk = tile(l, k);
            const CT zm = cconj(tile(l, k == 0 ? 0 : M - k));
            const CT e = cscale(cadd(zk, zm), T(0.5));
            const CT dd = csub(zk, zm);
            const CT od = cmk<CT>(T(0.5) * dd.y, T(-0.5) * dd.x);  // (zk - zm) / (2i)
            const CT t = cmul(od, w);
            line[k] = Conv<CT, V>::out(cnorm(cadd(e, t)));
            line[k == 0 ? M : M - k] = Conv<CT, V>::out(cnorm(cconj(csub(e, t))));
            if (k == 0) line[H] = Conv<CT, V>::out(cnorm(cconj(tile(l, H))));
        }
        return true;
    }
}

// Contiguous axis, real line of 2M points -> M+1 bins (forward).  The line is
// read as M complex z[m] = x[2m] + i x[2m+1]; Z = DFT_M(z) is left in shared
// memory and post-processed:
//   X[k] = E[k] + w_{2M}^k O[k],  E = (Z[k] + conj Z[M-k]) / 2,
//   O = (Z[k] - conj Z[M-k]) / (2i),  Z[M] = Z[0].
template <class F, typename V>
__global__ void __launch_bounds__(F::template threads<V>(), F::min_blocks)
    k_r2c(const typename RealOf<V>::T *__restrict__ in, V *out, const __grid_constant__ StageDesc d,
          const V *__restrict__ tw, const V *__restrict__ post_tw, long long nlines, int lines)
{
    using T = typename RealOf<V>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *sm = reinterpret_cast<V *>(smem_raw);
    const int M = F::generic ? d.n : F::plan::n;
    const long long b0 = stage_order(blockIdx.x, gridDim.x, d.rev) * lines;
    const int valid = (int)min((long long)lines, nlines - b0);
    const GlobalLines<V> src{reinterpret_cast<const V *>(in) + b0 * M, M, valid};
    const SmemLines<V> tile{sm, M};
    const MapButterflyFast map{};
    const int ld = d.ld > 0 ? d.ld : M + 1;  // output line stride (d.ld > 0: lines further apart)
    V *o = out + b0 * ld;
    if constexpr (UseDf<F, V>::value) {
        if (d.twdf) {
            DfFlags bad;
            const GlobalLines<V, dcx> sdf{reinterpret_cast<const V *>(in) + b0 * M, M, valid, &bad};
            const SmemLines<dcx> tdf{reinterpret_cast<dcx *>(sm), M};
            if (df_stage<typename F::plan, -1, true>((const dcx *)d.twdf, lines, map, sdf, tdf, tdf, bad)) {
                __syncthreads();
                // (float-float tiles keep the general loop: the fixed-bin form measured no faster)
                r2c_post<V, dcx>(tdf, o, (const dcx *)d.post_df, M, ld, valid);
                return;
            }
        }
    }
    // (the input is read from global memory in the first pass: staging it in shared memory as
    // k_c2r does measured 12% slower here, the 16 loads of a thread being in flight together)
    if constexpr (F::generic) run_generic<-1, false, true, F::split>(d, tw, sm, lines, 0, map, src, tile);
    else run_plan<typename F::plan, -1, true, F::split>(tw, lines, map, src, tile, tile, d.mma);
    __syncthreads();
    if constexpr (!F::generic && sizeof(V) == 8) {
        if (r2c_post_fixed_k<F::plan::n, V, V>(tile, o, post_tw, ld, valid)) return;
    }
    r2c_post<V, V>(tile, o, post_tw, M, ld, valid);
    (void)sizeof(T);
}

// Contiguous axis, M+1 bins -> real line of 2M points (backward, last stage):
// C2RPre builds Z from the half spectrum, an inverse DFT_M gives z, and z[m]
// is stored as the real pair (x[2m], x[2m+1]) times `scale`.
template <class F, typename V>
__global__ void __launch_bounds__(F::template threads<V>(), F::min_blocks)
    k_c2r(const V *__restrict__ in, typename RealOf<V>::T *out, const __grid_constant__ StageDesc d,
          const V *__restrict__ tw, const V *__restrict__ post_tw, long long nlines, int lines,
          typename RealOf<V>::T scale)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *sm = reinterpret_cast<V *>(smem_raw);
    const int M = F::generic ? d.n : F::plan::n;
    const long long b0 = stage_order(blockIdx.x, gridDim.x, d.rev) * lines;
    const int valid = (int)min((long long)lines, nlines - b0);
    const int ld = d.ld > 0 ? d.ld : M + 1;  // input line stride
    const C2RPre<V> src{in + b0 * ld, post_tw, M, ld, valid};
    const GlobalLinesOut<V> dst{reinterpret_cast<V *>(out) + b0 * M, M, valid, scale};
    const MapButterflyFast map{};
    if constexpr (F::generic) {
        run_generic<+1, false, false, F::split>(d, tw, sm, lines, 0, map, src, dst);
    } else {
        // complex64 (not split): the CTA's lines are one contiguous run of valid * (M + 1)
        // elements; when it starts 16-byte aligned it is copied by one bulk copy (TMA) into the
        // work tile itself (the host sizes it for lines * (M + 1) elements) and the first pass runs
        // in place: every thread reads its X[k], X[M - k] from shared memory, a barrier, then
        // the DFT outputs overwrite the tile.  Each element is read from HBM once, with the
        // whole run in flight and no thread issuing per-element copies (measured on the 512^3
        // stage: 0.192 ms with 16-byte cp.async per thread, 0.183 ms with the bulk copy).
        if constexpr (sizeof(V) == 8 && !F::split && F::plan::npass >= 1) {
            const V *xin = in + b0 * ld;
            // staging needs lines * (M + 1) elements of shared memory
            if (ld == M + 1 && (reinterpret_cast<unsigned long long>(xin) & 15) == 0 &&
                dynamic_smem_bytes() >= (unsigned)lines * (unsigned)(M + 1) * (unsigned)sizeof(V)) {
                if (!stage_contiguous(sm, xin, valid * (M + 1))) {
                    if (threadIdx.x == 0 && d.err) atomicExch(d.err, 1u);
                    return;
                }
                const C2RPre<V> sx{sm, post_tw, M, M + 1, valid};
                run_plan_staged<typename F::plan, +1>(typename F::plan::seq{}, tw, lines, map, sx, SmemLines<V>{sm, M},
                                                      dst);
                return;
            }
        }
        // complex128: the tile's half spectra are staged with cp.async behind the work tile (the
        // host adds lines * (M + 1) elements to the launch's shared memory), so the float-float
        // first pass reads shared memory; other complex64 tiles read them from global memory in
        // the first pass
        constexpr bool kStage = sizeof(V) == 16;
        constexpr int kRow = 128 / (int)sizeof(V);
        V *xs = sm + (lines * M + kRow - 1) / kRow * kRow;
        if constexpr (kStage) {
            const V *xin = in + b0 * ld;
            const int per = M + 1;
            if (ld == per) {
                // one contiguous run: one bulk copy
                if (!stage_contiguous(xs, xin, valid * per)) {
                    if (threadIdx.x == 0 && d.err) atomicExch(d.err, 1u);
                    return;
                }
            } else {
                for (int idx = threadIdx.x; idx < valid * per; idx += blockDim.x) {
                    const int l = idx / per;
                    cp_async_zfill<(int)sizeof(V)>(xs + idx, xin + (long long)l * ld + (idx - l * per), true);
                }
                cp_async_commit();
                cp_async_wait<0>();
                __syncthreads();
            }
        }
        const V *xsrc = kStage ? xs : in + b0 * ld;
        const int xld = kStage ? M + 1 : ld;
        if constexpr (UseDf<F, V>::value) {
            if (d.twdf) {
                DfFlags bad;
                const C2RPre<V, dcx> sdf{xsrc, (const dcx *)d.post_df, M, xld, valid, &bad};
                const GlobalLinesOut<V, dcx> ddf{reinterpret_cast<V *>(out) + b0 * M, M, valid, dfl(scale)};
                const SmemLines<dcx> tdf{reinterpret_cast<dcx *>(sm), M};
                if (df_stage<typename F::plan, +1, false>((const dcx *)d.twdf, lines, map, sdf, tdf, ddf, bad)) return;
            }
        }
        const SmemLines<V> tile{sm, M};
        const C2RPre<V> sx{xsrc, post_tw, M, xld, valid};
        run_plan<typename F::plan, +1, false, F::split>(tw, lines, map, sx, tile, dst, d.mma);
    }
}

// Second half of a four-step line (see FourStepSrc): the input is
// [outer * n_b][n_a][W] (row k_b of each outer line group holds the length-n_b
// DFT outputs, laid out as n_a rows), the output [outer][n_a n_b][W].  Generic
// family only: the split serves lines longer than one CTA holds.
template <int S, typename V, bool Split>
__global__ void __launch_bounds__(256, 1)
    k_fourstep(const V *__restrict__ in, V *out, const __grid_constant__ StageDesc d, const V *__restrict__ tw,
               const V *__restrict__ wn, long long W, long long tiles_per_outer, int log2_lines, int nb,
               typename RealOf<V>::T scale)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *sm = reinterpret_cast<V *>(smem_raw);
    const int na = d.n;
    const int lines = 1 << log2_lines;
    const long long op = blockIdx.x / tiles_per_outer;            // (o, k_b)
    const long long c0 = (blockIdx.x - op * tiles_per_outer) * lines;
    const long long o = op / nb;
    const int kb = (int)(op - o * nb);
    const int valid = (int)min((long long)lines, W - c0);
    const FourStepSrc<S, V> src{in + op * (long long)na * W + c0, W, valid, wn, kb};
    const FourStepDst<V> dst{out + (o * (long long)na * nb + kb) * W + c0, (long long)nb * W, valid, scale};
    run_generic<S, true, false, Split>(d, tw, sm, lines, log2_lines, MapLineFast{log2_lines}, src, dst);
}

// Spectral Poisson multiply on a half spectrum [planes][n1][nhp] (rows of nhp >= nh elements; planes =
// batch * n0): bin (k0, k1, k2) times 1/|k|^2 with wrapped integer wavenumbers,
// k = 0 and pad columns (k2 >= nh) set to zero.  Used when the N0 stage of a
// plan cannot run the fused pipelined operator.
template <typename V>
__global__ void k_poisson_mult(V *x, long long planes, int n0, int n1, int nhp, int nh)
{
    using T = typename RealOf<V>::T;
    const long long total = planes * n1 * nhp;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k2 = (int)(i % nhp);
        const long long r = i / nhp;
        const int k1 = (int)(r % n1);
        const int k0 = (int)((r / n1) % n0);
        const int a = 2 * k0 > n0 ? k0 - n0 : k0, b = 2 * k1 > n1 ? k1 - n1 : k1;
        const int K = a * a + b * b + k2 * k2;
        x[i] = (K > 0 && k2 < nh) ? cscale(x[i], T(1) / T(K)) : czero<V>();
    }
}

// Line lengths with specialised kernels and their radix sequences (n first,
// then the radices in pass order).  Split-precision plans use the sequences of
// AFFT_SPLIT_LINE_PLANS (as many radix-16 passes as the length allows), and
// the FP32 kernels for the other lengths of AFFT_LINE_PLANS (no radix-16 pass).
// (Groups A-E only split the complex128 instantiations over translation units
// that compile in parallel.)
#define AFFT_LINE_PLANS_A(X)                                                                        \
    X(1) X(2, 2) X(4, 4) X(8, 8) X(16, 16) X(24, 8, 3) X(32, 8, 4) X(48, 16, 3) X(60, 4, 3, 5) X(64, 8, 8)
#define AFFT_LINE_PLANS_B(X) X(80, 16, 5) X(96, 8, 4, 3) X(120, 8, 3, 5) X(128, 16, 8) X(160, 8, 4, 5) X(192, 8, 8, 3)
#define AFFT_LINE_PLANS_C(X) X(256, 16, 16) X(384, 16, 8, 3)
#define AFFT_LINE_PLANS_D(X) X(512, 8, 8, 8) X(1024, 16, 8, 8)
#define AFFT_LINE_PLANS_E(X) X(2048, 16, 16, 8) X(4096, 16, 16, 16)
#define AFFT_LINE_PLANS(X)                                                                          \
    AFFT_LINE_PLANS_A(X) AFFT_LINE_PLANS_B(X) AFFT_LINE_PLANS_C(X) AFFT_LINE_PLANS_D(X) AFFT_LINE_PLANS_E(X)
#define AFFT_SPLIT_LINE_PLANS(X)                                                                    \
    X(16, 16) X(32, 16, 2) X(48, 16, 3) X(64, 16, 4) X(80, 16, 5) X(96, 16, 3, 2) X(128, 16, 8)     \
    X(160, 16, 5, 2) X(192, 16, 4, 3) X(256, 16, 16) X(384, 16, 8, 3) X(512, 16, 16, 2)             \
    X(1024, 16, 16, 4) X(2048, 16, 16, 8) X(4096, 16, 16, 16)

}  // namespace afft
