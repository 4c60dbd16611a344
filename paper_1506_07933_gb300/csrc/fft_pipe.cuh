// fft_pipe.cuh -- persistent, double-buffered strided stage for GB300.
//
// The strided stages (N1 and N0 of Algorithm 1) move each element through
// HBM once in and once out; to keep HBM busy the next tile must already be
// in flight while the current one is transformed.  Each CTA therefore walks
// a sequence of tiles (tile t, t + gridDim.x, ...) with two shared-memory
// tile buffers:
//
//   load(tile 0 -> buf 0)
//   loop: load(next tile -> other buf);  wait(current buf);
//         radix passes in shared memory (the first one in place), the last
//         pass storing straight to global memory;  barrier.
//
// A tile is LINES adjacent columns x N rows ([N][LINES], LINES*C = 64 or 128
// bytes per row).  Loads are TMA tensor copies (cp.async.bulk.tensor.3d,
// completion on an mbarrier, one elected thread) when the array's row pitch
// is a multiple of 16 bytes, and per-element cp.async copies with zero fill
// otherwise (e.g. the N1 stage of an FP32 r2c plan, row pitch (n2/2+1)*8 B).
// Columns past the array's edge read as zero (TMA out-of-bounds fill, or a
// zero-byte cp.async) and are not stored.
//
// Every wait on an mbarrier is bounded (about two seconds of %globaltimer);
// on timeout the CTA sets *err and returns, after a CTA-wide vote so that no
// thread is left at a barrier.
#pragma once

#include <cuda.h>

#include <initializer_list>

#include "fft_stage.cuh"

namespace afft {

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int x, int y, int z, int w,
                                            unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}



// Shared-memory rows of a compile-time width: [N][1 << LG].
template <typename V, int LG> struct SmemRowsC {
    V *sm;
    __device__ __forceinline__ V operator()(int l, int p) const { return sm[(p << LG) + l]; }
    __device__ __forceinline__ void operator()(int l, int p, V v) const { sm[(p << LG) + l] = v; }
};

template <int LG> struct MapLineFastC {
    __device__ __forceinline__ void operator()(int idx, int, int &l, int &j) const
    {
        l = idx & ((1 << LG) - 1);
        j = idx >> LG;
    }
};

// ------------------------------------------------------------------ shape ---
// Compile-time shape of the pipelined strided kernel for line length N and
// complex type V.  A tile is LINES columns x N rows with 128-byte rows
// (LINES = 16 for complex64, 8 for complex128), halved while three tile
// buffers (two load targets and one scratch for out-of-place passes) exceed
// kPipeSmemCap.  FP32 passes of radix <= 8 give each thread two adjacent
// columns ("pairs": 16-byte shared-memory and global accesses, one twiddle
// load for both); other passes give each thread one column.  Every thread
// carries at most 16 complex values per pass.
constexpr int kPipeSmemCap = 200 * 1024;

template <class P, typename V> struct PipeShape {
    static constexpr int row_lines = 128 / (int)sizeof(V);
    __host__ __device__ static constexpr int lines_for(int l)
    {
        return (l > 1 && 3 * P::n * l * (int)sizeof(V) > kPipeSmemCap) ? lines_for(l / 2) : l;
    }
    static constexpr int lines = lines_for(row_lines);
    static constexpr int lg = lines == 16 ? 4 : lines == 8 ? 3 : lines == 4 ? 2 : lines == 2 ? 1 : 0;
    __host__ __device__ static constexpr bool pairs(int r) { return sizeof(V) == 8 && lines >= 2 && 2 * r <= 16; }
    template <int... Rs> __host__ __device__ static constexpr int max_radix(Seq<Rs...>)
    {
        int m = 1;
        for (int r : {Rs...}) m = r > m ? r : m;
        return m;
    }
    // butterflies (or butterfly pairs) per thread; complex128 tiles (float-float arithmetic, twice
    // the registers per value) of plans without a radix-16 pass carry at most 8 values per thread,
    // for more warps per SM
    __host__ __device__ static constexpr int per_thread(int r)
    {
        return pairs(r) ? (16 / (2 * r) > 0 ? 16 / (2 * r) : 1)
               : (sizeof(V) == 16 && max_radix(typename P::seq{}) <= 8) ? (8 / r > 1 ? 8 / r : 1)
                                                                      : bmax_for_radix(r);
    }
    __host__ __device__ static constexpr int units(int r) { return (pairs(r) ? lines / 2 : lines) * (P::n / r); }
    template <int... Rs> __host__ __device__ static constexpr int threads_for(Seq<Rs...>)
    {
        int req = lines;
        for (int r : {Rs...}) {
            const int t = (units(r) + per_thread(r) - 1) / per_thread(r);
            req = t > req ? t : req;
        }
        return (req + 31) / 32 * 32;
    }
    static constexpr int threads = threads_for(typename P::seq{});
    static_assert(threads % lines == 0, "each thread must own fixed columns of the tile");
    // butterflies (or pairs) per thread that cover a radix-r pass with `threads` threads: in-place
    // passes hold all of them in registers across the barrier, so no more than needed
    __host__ __device__ static constexpr int covering(int r) { return (units(r) + threads - 1) / threads; }
    using seq = typename P::seq;
    static constexpr int npass = P::npass;
    static constexpr int tile = P::n * lines;                       // complex elements per tile
    // twiddle entries of the line's passes (Ns (R - 1) per pass with Ns > 1, in pass order)
    template <int... Rs> __host__ __device__ static constexpr int tw_count(Seq<Rs...>)
    {
        int ns = 1, c = 0;
        for (int r : {Rs...}) {
            if (ns > 1) c += ns * (r - 1);
            ns *= r;
        }
        return c;
    }
    // complex64 tiles stage the table in shared memory (behind the mbarriers), once per CTA
    static constexpr int tw_smem = sizeof(V) == 8 ? tw_count(seq{}) : 0;
    static constexpr int smem = 3 * tile * (int)sizeof(V) + 16 + tw_smem * 8;   // 3 buffers, mbarriers, table
    // odd-width complex64 rows read as row pairs (k_strided_pipe_rp): load buffers of two
    // [n/2][lines + 2] boxes, then the scratch tile and the mbarriers
    static constexpr int lw = lines + 2;
    static constexpr int tile_rp = P::n * lw;
    static constexpr int smem_rp = (2 * tile_rp + tile) * (int)sizeof(V) + 16 + tw_smem * 8;
    static constexpr bool rp_ok = sizeof(V) == 8 && lines == 16 && P::n % 16 == 0 && P::n / 2 <= 256;
    static constexpr int box_rows = tma_box_rows(P::n);
    // split precision: the radix-16 passes' butterflies (tile / 16) fill whole 128-row blocks and
    // one 128-thread group per block covers them -- the tcgen05 pass runs unconditionally
    static constexpr bool tc_tile = sizeof(V) == 8 && (tile / 16) % 128 == 0 && threads % 128 == 0 &&
                                    tile / 16 <= threads && threads <= 512;
    // CTAs per SM the launch bounds ask for: two when two such CTAs' shared memory fits (tiles,
    // table and the tensor-core state, about 5 KB of static shared memory)
    static constexpr int min_blocks_split = 2 * (smem + 6 * 1024) <= 226 * 1024 ? 2 : 1;
    static_assert((box_rows * lines * (int)sizeof(V)) % 128 == 0 || box_rows == P::n,
                  "TMA boxes must start 128-byte aligned in shared memory");
};

// ---------------------------------------------------------- pair passes ---

// Writes of a pair pass: shared memory rows, or the stage's global output.
template <int LG> struct PairSmemOut {
    float2 *sm;
    __device__ __forceinline__ void operator()(int lp, int p, float2 lo, float2 hi) const
    {
        reinterpret_cast<float4 *>(sm)[(p << (LG - 1)) + lp] = make_float4(lo.x, lo.y, hi.x, hi.y);
    }
};
struct PairGlobalOut {
    float2 *base;                  // &y[o][0][0]
    long long W;                   // output row pitch
    long long oc0, oc1;            // this thread's two output columns (-1: not stored)
    bool vec;                      // adjacent, 16-byte aligned: one 16-byte store
    __device__ __forceinline__ void operator()(int, int p, float2 lo, float2 hi) const
    {
        float2 *row = base + (long long)p * W;
        if (vec) {
            *reinterpret_cast<float4 *>(row + oc0) = make_float4(lo.x, lo.y, hi.x, hi.y);
        } else {
            if (oc0 >= 0) row[oc0] = lo;
            if (oc1 >= 0) row[oc1] = hi;
        }
    }
};

// One radix-R Stockham pass over a [N][2^LG] float2 tile; the thread's
// butterflies are (column pair lp, butterfly j), reading both columns' R
// values with 16-byte loads and sharing the twiddles.  InPlace: every read of
// the CTA precedes a barrier, every write follows it (src and dst may alias).
template <int R, int S, int N, int Ns, int LG, int NT, int B, bool InPlace = false, bool TwSmem = false, class Dst>
__device__ __forceinline__ void pair_pass(const float2 *src, const float2 *__restrict__ tw, const Dst &dst)
{
    constexpr int PAIRS = (1 << LG) / 2, NB = N / R, TOTAL = PAIRS * NB;
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    float2 lo[B][R], hi[B][R];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int idx = threadIdx.x + b * NT;
        if (B * NT == TOTAL || idx < TOTAL) {
            const int lp = idx % PAIRS, j = idx / PAIRS;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float4 q = s4[(j + r * NB) * PAIRS + lp];
                lo[b][r] = make_float2(q.x, q.y);
                hi[b][r] = make_float2(q.z, q.w);
            }
            const int k = j % Ns;
            if (Ns > 1) {
                const float2 *t = tw + k * (R - 1);
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const float2 w = tw_ld<TwSmem>(t + r - 1);
                    lo[b][r] = ctw<S>(lo[b][r], w);
                    hi[b][r] = ctw<S>(hi[b][r], w);
                }
            }
            Dft<R, S, float2>::run(lo[b]);
            Dft<R, S, float2>::run(hi[b]);
        }
    }
    if constexpr (InPlace) __syncthreads();
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int idx = threadIdx.x + b * NT;
        if (B * NT == TOTAL || idx < TOTAL) {
            const int lp = idx % PAIRS, j = idx / PAIRS;
            const int k = j % Ns;
            const int o = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) dst(lp, o + r * Ns, lo[b][r], hi[b][r]);
        }
    }
}

// Output of a tile's column l (tile columns start at c0), for passes whose
// threads do not own fixed columns (the tensor-core radix-16 pass).
template <typename V> struct PipeColOut {
    V *base;                          // &y[o][0][0]
    long long c0, W;
    __device__ __forceinline__ void operator()(int l, int p, V v) const
    {
        const long long c = c0 + l;
        if (c < W) base[(long long)p * W + c] = v;
    }
};

// The stage's global output for the pass kinds, resolved per thread per tile
// (stored as V, computed as CT).
template <typename V, typename CT = V> struct TileOut {
    GlobalColFixedOut<V, CT> single;  // one column per thread
    PairGlobalOut pair;               // two columns per thread (float2 only)
    PipeColOut<V> cols;               // any column (split-precision radix-16 passes)
};

// Passes Seq<R, Rest...>: pass number Q reads buffer X (Q even) or C (Q odd)
// and writes the other one; the last pass writes the stage's output.  Split:
// radix-16 passes of complex64 tiles on the tensor cores (fft_split.cuh, table
// `mma` of both directions).
template <class Sh, int S, int N, int Ns, int TwOff, int Q, bool Split = false, bool TwSmem = false, int TC = 0,
          typename V, class Out, int R, int... Rest>
__device__ __forceinline__ void pipe_passes(Seq<R, Rest...>, V *X, V *C, const V *tw, const Out &out,
                                            const unsigned *mma = nullptr)
{
    constexpr bool Last = sizeof...(Rest) == 0;
    constexpr int LG = Sh::lg, NT = Sh::threads;
    V *src = (Q % 2 == 0) ? X : C;
    V *dst = (Q % 2 == 0) ? C : X;
    if constexpr (Sh::pairs(R)) {
        constexpr int B = Sh::per_thread(R);
        if constexpr (Last) pair_pass<R, S, N, Ns, LG, NT, B, false, TwSmem>(src, tw + TwOff, out.pair);
        else pair_pass<R, S, N, Ns, LG, NT, B, false, TwSmem>(src, tw + TwOff, PairSmemOut<LG>{dst});
    } else {
        const SmemRowsC<V, LG> in_rows{src};
        constexpr int B = Sh::per_thread(R);
        if constexpr (Last && Split && R == 16)
            spec_pass<R, S, false, Split, NT, B, TC, TwSmem>(N, Ns, tw + TwOff, Sh::lines, MapLineFastC<LG>{}, in_rows,
                                                             out.cols, mma, src);
        else if constexpr (Split && R == 16)
            spec_pass<R, S, false, Split, NT, B, TC, TwSmem>(N, Ns, tw + TwOff, Sh::lines, MapLineFastC<LG>{}, in_rows,
                                                             SmemRowsC<V, LG>{dst}, mma, src);
        else if constexpr (Last && TwSmem)
            radix_pass<R, S, false, NT, B, true>(N, Ns, tw + TwOff, Sh::lines, MapLineFastC<LG>{}, in_rows, out.single);
        else if constexpr (TwSmem)
            radix_pass<R, S, false, NT, B, true>(N, Ns, tw + TwOff, Sh::lines, MapLineFastC<LG>{}, in_rows,
                                                 SmemRowsC<V, LG>{dst});
        else if constexpr (Last)
            spec_pass<R, S, false, Split, NT, B>(N, Ns, tw + TwOff, Sh::lines, MapLineFastC<LG>{}, in_rows,
                                                 out.single, mma);
        else
            spec_pass<R, S, false, Split, NT, B>(N, Ns, tw + TwOff, Sh::lines, MapLineFastC<LG>{}, in_rows,
                                                 SmemRowsC<V, LG>{dst}, mma);
    }
    if constexpr (!Last) {
        __syncthreads();
        constexpr int next = TwOff + (Ns > 1 ? Ns * (R - 1) : 0);
        pipe_passes<Sh, S, N, Ns * R, next, Q + 1, Split, TwSmem, TC>(Seq<Rest...>{}, X, C, tw, out, mma);
    }
}

// Passes Seq<R, Rest...> after the first (Ns: the product of the radices
// before them), all on the scratch tile C in place, the last one writing the
// stage's output (complex64, no split).
template <class Sh, int S, int N, int Ns, int TwOff, class Out, int R, int... Rest>
__device__ __forceinline__ void scratch_passes(Seq<R, Rest...>, float2 *C, const float2 *tw, const Out &out)
{
    constexpr bool Global = sizeof...(Rest) == 0;
    constexpr int LG = Sh::lg, NT = Sh::threads, B = Sh::covering(R);
    if constexpr (Sh::pairs(R)) {
        if constexpr (Global) pair_pass<R, S, N, Ns, LG, NT, B, false, true>(C, tw + TwOff, out.pair);
        else pair_pass<R, S, N, Ns, LG, NT, B, true, true>(C, tw + TwOff, PairSmemOut<LG>{C});
    } else {
        const SmemRowsC<float2, LG> rows{C};
        if constexpr (Global)
            radix_pass<R, S, false, NT, B, true>(N, Ns, tw + TwOff, Sh::lines, MapLineFastC<LG>{}, rows, out.single);
        else radix_pass<R, S, true, NT, B, true>(N, Ns, tw + TwOff, Sh::lines, MapLineFastC<LG>{}, rows, rows);
    }
    if constexpr (sizeof...(Rest) > 0) {
        __syncthreads();
        scratch_passes<Sh, S, N, Ns * R, TwOff + (Ns > 1 ? Ns * (R - 1) : 0)>(Seq<Rest...>{}, C, tw, out);
    }
}

// A complex64 tile of at least two passes whose load buffer X is released
// after the first pass (X -> C), so that the next load into it can start
// while the other passes run in place on C: `released` issues that load.
template <class Sh, int S, int N, class Out, class Released, int R0, int... Rest>
__device__ __forceinline__ void early_release_passes(Seq<R0, Rest...>, const float2 *X, float2 *C,
                                                     const float2 *tw, const Out &out, const Released &released)
{
    static_assert(sizeof...(Rest) >= 1, "the first pass must not be the last");
    constexpr int LG = Sh::lg, NT = Sh::threads, B = Sh::per_thread(R0);
    if constexpr (Sh::pairs(R0))
        pair_pass<R0, S, N, 1, LG, NT, B>(X, tw, PairSmemOut<LG>{C});
    else
        radix_pass<R0, S, false, NT, B>(N, 1, tw, Sh::lines, MapLineFastC<LG>{}, SmemRowsC<float2, LG>{const_cast<float2 *>(X)},
                                        SmemRowsC<float2, LG>{C});
    __syncthreads();
    released();
    scratch_passes<Sh, S, N, R0, 0>(Seq<Rest...>{}, C, tw, out);
}

// FP64 tile in float-float: the first pass converts the FP64 tile X (as the
// TMA copy left it) into float-float values in C and votes on range; the
// remaining passes continue in float-float (Q = 1: C -> X -> ...).  Returns
// false, with X untouched, when some value was out of float-float range.
template <class Sh, int S, int N, class Out, int R0, int... Rest>
__device__ __forceinline__ bool pipe_df(Seq<R0, Rest...>, double2 *X, double2 *C, const dcx *tw, const Out &out)
{
    constexpr int LG = Sh::lg, NT = Sh::threads;
    DfFlags bad;
    const SmemRowsConvIn<double2, dcx, LG> src{X, &bad};
    radix_pass<R0, S, false, NT, Sh::per_thread(R0)>(N, 1, tw, Sh::lines, MapLineFastC<LG>{}, src,
                                 SmemRowsC<dcx, LG>{reinterpret_cast<dcx *>(C)});
    if (!df_tile_ok(bad)) return false;
    pipe_passes<Sh, S, N, R0, 0, 1>(Seq<Rest...>{}, reinterpret_cast<dcx *>(X), reinterpret_cast<dcx *>(C), tw, out);
    return true;
}

// ---------------------------------------------------------------- kernel ---

template <class P, int S, typename V, bool TMA, bool Split = false, bool Blocked = false>
__global__ void __launch_bounds__(PipeShape<P, V>::threads, Split ? PipeShape<P, V>::min_blocks_split : 1)
    k_strided_pipe(const V *__restrict__ in, V *out, const __grid_constant__ CUtensorMap tmap,
                   const V *__restrict__ tw, long long W, long long tiles_per_outer, long long ntiles,
                   unsigned *err, const void *twdf, const unsigned *mma, int rev)
{
    using Sh = PipeShape<P, V>;
    constexpr int N = P::n, LINES = Sh::lines, LG = Sh::lg, NT = Sh::threads, TILE = Sh::tile;
    constexpr unsigned TILE_BYTES = TILE * sizeof(V);
    extern __shared__ __align__(1024) unsigned char pipe_smem_raw[];
    V *const buf0 = reinterpret_cast<V *>(pipe_smem_raw);   // load buffer b at buf0 + b * TILE
    V *const scratch = buf0 + 2 * TILE;                  // out-of-place passes
    unsigned long long *const bars = reinterpret_cast<unsigned long long *>(pipe_smem_raw + 3 * TILE_BYTES);
    const int tid = threadIdx.x;

    long long t = blockIdx.x;
    if (t >= ntiles) return;
    // Complex64 TMA tiles of two or more passes release their load buffer after
    // the first pass, so two loads are in flight while the rest runs; otherwise
    // the next tile's load is issued once this one has landed.
    constexpr bool Early = TMA && !Split && sizeof(V) == 8 && P::npass >= 2;
    // those tiles read their twiddles from a copy of the line's table in shared memory, staged
    // once per CTA (the factors of a pass are the same for every tile)
    float2 *const tw_s = reinterpret_cast<float2 *>(pipe_smem_raw + 3 * TILE_BYTES + 16);
    constexpr bool StageTw = Early || (Split && sizeof(V) == 8);
    if constexpr (StageTw) {
        for (int e = tid; e < Sh::tw_smem; e += NT) tw_s[e] = ldgc(reinterpret_cast<const float2 *>(tw) + e);
    }
    if (TMA && tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // split precision: radix-16 passes on tcgen05 where the tile allows (fft_tc.cuh)
    constexpr bool TC = Split && sizeof(V) == 8;
    if constexpr (TC)
        tc_setup(reinterpret_cast<const unsigned char *>(mma) + kMmaTableWords * 4 + (S < 0 ? 0 : kTcBBytes),
                 tc_cols_for(NT));

    auto issue = [&](long long tile_i, int b) {
        const long long tile = stage_order(tile_i, ntiles, rev);
        const long long o = tile / tiles_per_outer;
        const long long c0 = (tile - o * tiles_per_outer) * LINES;
        if constexpr (TMA) {
            if (tid == 0) {
                fence_async_shared();
                mbar_expect_tx(&bars[b], TILE_BYTES);
                constexpr int rows = Sh::box_rows;
                constexpr int per = (int)sizeof(V) / 8;  // 8-byte elements per complex value
                if constexpr (Blocked) {
                    // a 4-D map [N / R groups][outer lines][R rows][W] (the blocked workspace, or rows
                    // grouped by R): one box (all groups of line o) brings the tile in natural row order
                    tma_load_4d(buf0 + b * TILE, &tmap, (int)(c0 * per), 0, (int)o, 0, &bars[b]);
                } else {
                    // boxes of at most 256 rows (measured on the 512^3 N0 stage: 0.175 ms with two
                    // 256-row boxes, 0.178 ms with one 4-D box of 512 rows)
#pragma unroll
                    for (int r0 = 0; r0 < N; r0 += rows)
                        tma_load_3d(buf0 + b * TILE + r0 * LINES, &tmap, (int)(c0 * per), r0, (int)o, &bars[b]);
                }
            }
        } else {
            const V *src = in + o * (long long)N * W + c0;
            const int valid = (int)min((long long)LINES, W - c0);
            for (int e = tid; e < TILE; e += NT) {
                const int p = e >> LG, l = e & (LINES - 1);
                const bool ok = l < valid;
                cp_async_zfill<(int)sizeof(V)>(buf0 + b * TILE + e,
                                               ok ? (const void *)(src + (long long)p * W + l) : (const void *)src,
                                               ok);
            }
            cp_async_commit();
        }
    };
    auto out_col = [&](long long c) -> long long { return c < W ? c : -1; };

    issue(t, 0);
    if (Early && t + gridDim.x < ntiles) issue(t + gridDim.x, 1);
    for (int i = 0;; ++i) {
        const int b = i & 1;
        const long long tn = t + gridDim.x;
        // wait for this tile; the barrier also retires every read of the other buffer
        if constexpr (TMA) {
            const bool ok = mbar_wait_bounded(&bars[b], (unsigned)((i >> 1) & 1));
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    atomicExch(err, 1u);
                    // the other buffer's load, if one was issued, must land before the CTA exits
                    if (Early && tn < ntiles) mbar_wait_bounded(&bars[b ^ 1], (unsigned)(((i + 1) >> 1) & 1));
                }
                if constexpr (TC) tc_teardown();
                return;
            }
        } else {
            cp_async_wait<0>();
            __syncthreads();
        }
        if (!Early && tn < ntiles) issue(tn, b ^ 1);   // next tile flies while this one is transformed

        const long long tile = stage_order(t, ntiles, rev);
        const long long o = tile / tiles_per_outer;
        const long long c0 = (tile - o * tiles_per_outer) * LINES;
        TileOut<V> to;
        to.single = GlobalColFixedOut<V>{out + o * (long long)N * W, W, out_col(c0 + (tid & (LINES - 1)))};
        to.cols = PipeColOut<V>{out + o * (long long)N * W, c0, W};
        if constexpr (sizeof(V) == 8) {
            const int lp = tid % (LINES / 2 > 0 ? LINES / 2 : 1);
            const long long a = out_col(c0 + 2 * lp), bcol = out_col(c0 + 2 * lp + 1);
            float2 *base = reinterpret_cast<float2 *>(out + o * (long long)N * W);
            const bool vec = a >= 0 && bcol == a + 1 && (a % 2) == 0 && (W % 2) == 0 &&
                             (reinterpret_cast<unsigned long long>(base) & 15) == 0;
            to.pair = PairGlobalOut{base, W, a, bcol, vec};
        }
        bool done = false;
        if constexpr (std::is_same<V, double2>::value && P::npass >= 2) {
            if (twdf) {
                TileOut<V, dcx> tdf;
                tdf.single = GlobalColFixedOut<V, dcx>{to.single.base, to.single.W, to.single.col};
                done = pipe_df<Sh, S, N>(typename P::seq{}, buf0 + b * TILE, scratch, (const dcx *)twdf, tdf);
            }
        }
        if constexpr (Early) {
            const float2 *x = reinterpret_cast<const float2 *>(buf0 + b * TILE);
            early_release_passes<Sh, S, N>(typename P::seq{}, x, reinterpret_cast<float2 *>(scratch), tw_s, to, [&] {
                                               if (tn + gridDim.x < ntiles) issue(tn + gridDim.x, b);
                                           });
        } else if (!done) {
            if constexpr (TC)
                pipe_passes<Sh, S, N, 1, 0, 0, Split, true, Sh::tc_tile ? 2 : 1>(
                    typename P::seq{}, buf0 + b * TILE, scratch, reinterpret_cast<const V *>(tw_s), to, mma);
            else
                pipe_passes<Sh, S, N, 1, 0, 0, Split>(typename P::seq{}, buf0 + b * TILE, scratch, tw, to, mma);
        }
        if (tn >= ntiles) break;
        t = tn;
    }
    if constexpr (TC) {
        if (tid == 0 && !tc_state().ok) atomicExch(err, 1u);   // a tensor-core wait ran out
        tc_teardown();
    }
}

// ----------------------------------------------- odd-width complex64 rows ---
// A strided stage over rows of W complex64 with W odd (the N1 stage of an r2c
// plan whose half spectrum has n2/2 + 1 bins, n2/2 even) cannot use TMA on
// single rows: their pitch, 8 W bytes, is not a multiple of 16.  Two rows
// are: the array is viewed as [outer][n/2][2W] and a tile of 16 columns c0..
// of all n rows is two boxes of lines + 2 = 18 columns and n/2 row pairs,
// A at x = c0 (even rows, column l at offset l) and B at x = W + c0 - 1 (odd
// rows, column l at offset l + 1); both x are even, as TMA requires.  The
// first pass reads the rows from the boxes, the others use the 16-wide tiles.

// First-pass source for threads owning one fixed column l.
template <int LW> struct RowPairIn {
    const float2 *A, *B;
    int l;
    __device__ __forceinline__ float2 operator()(int, int p) const
    {
        const int h = p >> 1;
        return (p & 1) ? B[h * LW + l + 1] : A[h * LW + l];
    }
};

// Column-pair first pass (Ns = 1) over the row-pair boxes.
template <int R, int S, int N, int LW, int LG, int NT, int B, class Dst>
__device__ __forceinline__ void pair_pass_rp(const float2 *A, const float2 *Bx, const Dst &dst)
{
    constexpr int PAIRS = (1 << LG) / 2, NB = N / R, TOTAL = PAIRS * NB;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int idx = threadIdx.x + b * NT;
        if (B * NT == TOTAL || idx < TOTAL) {
            const int lp = idx % PAIRS, j = idx / PAIRS;
            float2 lo[R], hi[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int p = j + r * NB, odd = p & 1;
                const float2 *row = (odd ? Bx : A) + (p >> 1) * LW + 2 * lp + odd;
                lo[r] = row[0];
                hi[r] = row[1];
            }
            Dft<R, S, float2>::run(lo);
            Dft<R, S, float2>::run(hi);
#pragma unroll
            for (int r = 0; r < R; ++r) dst(lp, j * R + r, lo[r], hi[r]);   // Ns = 1: output j R + r
        }
    }
}

// Stores of the column-pair passes into rows of odd pitch: a 16-byte store
// where row p puts the pair on a 16-byte boundary, else two 8-byte stores.
struct PairGlobalOutOdd {
    float2 *base;
    long long W;
    long long oc0, oc1;            // this thread's two output columns (-1: not stored)
    bool vec;                      // adjacent columns and a 16-byte aligned base
    __device__ __forceinline__ void operator()(int, int p, float2 lo, float2 hi) const
    {
        const long long e = (long long)p * W;
        float2 *row = base + e;
        if (vec && ((e + oc0) & 1) == 0) {
            *reinterpret_cast<float4 *>(row + oc0) = make_float4(lo.x, lo.y, hi.x, hi.y);
        } else {
            if (oc0 >= 0) row[oc0] = lo;
            if (oc1 >= 0) row[oc1] = hi;
        }
    }
};
struct TileOutOdd {
    GlobalColFixedOut<float2> single;
    PairGlobalOutOdd pair;
};

// The first pass from the row-pair boxes (into C, or to the output when it is
// the only pass), then the other passes ping-pong between C and X (Q = 1).
template <class Sh, int S, int N, class Out, int R0, int... Rest>
__device__ __forceinline__ void rp_passes(Seq<R0, Rest...>, float2 *X, float2 *C, const float2 *tw, const Out &out,
                                          int l)
{
    constexpr int LG = Sh::lg, NT = Sh::threads, LW = Sh::lw;
    constexpr bool Last = sizeof...(Rest) == 0;
    const float2 *A = X, *Bx = X + (N / 2) * LW;
    if constexpr (Sh::pairs(R0)) {
        constexpr int B = Sh::per_thread(R0);
        if constexpr (Last) pair_pass_rp<R0, S, N, LW, LG, NT, B>(A, Bx, out.pair);
        else pair_pass_rp<R0, S, N, LW, LG, NT, B>(A, Bx, PairSmemOut<LG>{C});
    } else {
        constexpr int B = Sh::per_thread(R0);
        const RowPairIn<LW> in{A, Bx, l};
        if constexpr (Last)
            radix_pass<R0, S, false, NT, B>(N, 1, tw, Sh::lines, MapLineFastC<LG>{}, in, out.single);
        else
            radix_pass<R0, S, false, NT, B>(N, 1, tw, Sh::lines, MapLineFastC<LG>{}, in, SmemRowsC<float2, LG>{C});
    }
    if constexpr (!Last) {
        __syncthreads();
        pipe_passes<Sh, S, N, R0, 0, 1, false, true>(Seq<Rest...>{}, X, C, tw, out);
    }
}

// Early release for row-pair tiles: the first pass reads the boxes (X -> C), then
// `released` issues the load of the tile after next into X while the other
// passes run in place on C.
template <class Sh, int S, int N, class Out, class Released, int R0, int... Rest>
__device__ __forceinline__ void rp_early_passes(Seq<R0, Rest...>, const float2 *X, float2 *C, const float2 *tw,
                                                const Out &out, int l, const Released &released)
{
    static_assert(sizeof...(Rest) >= 1, "the first pass must not be the last");
    constexpr int LG = Sh::lg, NT = Sh::threads, LW = Sh::lw;
    const float2 *A = X, *Bx = X + (N / 2) * LW;
    if constexpr (Sh::pairs(R0))
        pair_pass_rp<R0, S, N, LW, LG, NT, Sh::per_thread(R0)>(A, Bx, PairSmemOut<LG>{C});
    else
        radix_pass<R0, S, false, NT, Sh::per_thread(R0)>(N, 1, tw, Sh::lines, MapLineFastC<LG>{}, RowPairIn<LW>{A, Bx, l},
                                                        SmemRowsC<float2, LG>{C});
    __syncthreads();
    released();
    scratch_passes<Sh, S, N, R0, 0>(Seq<Rest...>{}, C, tw, out);
}

// Persistent, double-buffered strided stage over odd-width complex64 rows (the
// arguments of k_strided_pipe; the tensor map views [outer][n/2][2W] with boxes
// of 18 x n/2).  Early: the load buffer is released after the first pass
// (two tile loads in flight during the other passes), as k_strided_pipe does.
template <class P, int S, bool Early = false>
__global__ void __launch_bounds__(PipeShape<P, float2>::threads, 1)
    k_strided_pipe_rp(const float2 *__restrict__, float2 *out, const __grid_constant__ CUtensorMap tmap,
                      const float2 *__restrict__ tw, long long W, long long tiles_per_outer, long long ntiles,
                      unsigned *err, const void *, const unsigned *, int rev)
{
    using V = float2;
    using Sh = PipeShape<P, V>;
    constexpr int N = P::n, LINES = Sh::lines, LW = Sh::lw, TILE_RP = Sh::tile_rp;
    constexpr unsigned BOX_BYTES = (N / 2) * LW * sizeof(V);
    static_assert(Sh::rp_ok, "row-pair tiles: 16 complex64 columns, n a multiple of 16, at most 512");
    extern __shared__ __align__(1024) unsigned char pipe_smem_raw[];
    V *const buf0 = reinterpret_cast<V *>(pipe_smem_raw);   // load buffer b at buf0 + b * TILE_RP
    V *const scratch = buf0 + 2 * TILE_RP;
    unsigned long long *const bars =
        reinterpret_cast<unsigned long long *>(pipe_smem_raw + (2 * TILE_RP + Sh::tile) * sizeof(V));
    // the line's twiddle table, staged once per CTA behind the mbarriers
    float2 *const tw_s = reinterpret_cast<float2 *>(pipe_smem_raw + (2 * TILE_RP + Sh::tile) * sizeof(V) + 16);
    const int tid = threadIdx.x;

    long long t = blockIdx.x;
    if (t >= ntiles) return;
    for (int e = tid; e < Sh::tw_smem; e += Sh::threads) tw_s[e] = ldgc(tw + e);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    auto issue = [&](long long tile_i, int b) {
        if (tid != 0) return;
        const long long tile = stage_order(tile_i, ntiles, rev);
        const long long o = tile / tiles_per_outer;
        const long long c0 = (tile - o * tiles_per_outer) * LINES;
        fence_async_shared();
        mbar_expect_tx(&bars[b], 2 * BOX_BYTES);
        tma_load_3d(buf0 + b * TILE_RP, &tmap, (int)c0, 0, (int)o, &bars[b]);
        tma_load_3d(buf0 + b * TILE_RP + (N / 2) * LW, &tmap, (int)(W + c0 - 1), 0, (int)o, &bars[b]);
    };

    // Without Early the next tile's load is issued once this one has landed.
    issue(t, 0);
    if (Early && t + gridDim.x < ntiles) issue(t + gridDim.x, 1);
    for (int i = 0;; ++i) {
        const int b = i & 1;
        const long long tn = t + gridDim.x;
        const bool ok = mbar_wait_bounded(&bars[b], (unsigned)((i >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(err, 1u);
                // the other buffer's load, if one was issued, must land before the CTA exits
                if (Early && tn < ntiles) mbar_wait_bounded(&bars[b ^ 1], (unsigned)(((i + 1) >> 1) & 1));
            }
            return;
        }
        if (!Early && tn < ntiles) issue(tn, b ^ 1);

        const long long tile = stage_order(t, ntiles, rev);
        const long long o = tile / tiles_per_outer;
        const long long c0 = (tile - o * tiles_per_outer) * LINES;
        const int l = tid & (LINES - 1), lp = tid % (LINES / 2);
        V *obase = out + o * (long long)N * W;
        const long long a = c0 + 2 * lp;
        TileOutOdd to;
        to.single = GlobalColFixedOut<V>{obase, W, c0 + l < W ? c0 + l : -1};
        to.pair = PairGlobalOutOdd{obase, W, a < W ? a : -1, a + 1 < W ? a + 1 : -1,
                                   a + 1 < W && (reinterpret_cast<unsigned long long>(obase) & 15) == 0};
        if constexpr (Early && P::npass >= 2)
            rp_early_passes<Sh, S, N>(typename P::seq{}, buf0 + b * TILE_RP, scratch, tw_s, to, l, [&] {
                if (tn + gridDim.x < ntiles) issue(tn + gridDim.x, b);
            });
        else
            rp_passes<Sh, S, N>(typename P::seq{}, buf0 + b * TILE_RP, scratch, tw_s, to, l);
        if (tn >= ntiles) break;
        t = tn;
    }
}

// ------------------------------------------------------ Poisson operator ---
// The spectral Poisson solve -Lap u = f on [0, 2 pi)^3 divides each bin of
// the r2c spectrum by |k|^2 (integer wavenumbers k_i = m for m <= n_i/2, else
// m - n_i) and zeroes k = 0.  Its N0 stage is fused: forward N0 DFTs, the
// division, inverse N0 DFTs, all on the tile in shared memory, so the
// spectrum makes one HBM round trip instead of three.

template <typename T> __device__ __forceinline__ T inv_int(int K);
template <> __device__ __forceinline__ float inv_int<float>(int K) { return 1.0f / (float)K; }
template <> __device__ __forceinline__ double inv_int<double>(int K) { return 1.0 / (double)K; }
template <> __device__ __forceinline__ dfl inv_int<dfl>(int K)
{
    // K < 2^24 is exact in float; the FMA residual gives the low part
    const float k = (float)K, r = 1.0f / k;
    return dfl(r, fmaf(-r, k, 1.0f) * r);
}

// Writes of the forward half's last pass into a shared tile (both pass kinds).
template <typename V, int LG> struct SmemTileOut {
    SmemRowsC<V, LG> single;
    PairSmemOut<LG> pair;
};

// Forward N0 DFTs (tile A, scratch Bf), the 1/|k|^2 scaling, inverse N0 DFTs,
// the last pass storing through `gout`.  The thread's column is fixed
// (tid mod LINES), so its (k1, k2) are resolved once: col1 = k1, col2 = k2,
// keep = false for pad columns.
template <class Sh, int N, typename CT, class GOut>
__device__ __forceinline__ void poisson_tile(CT *A, CT *Bf, const CT *tw, const GOut &gout, int n1, int k1,
                                             int k2, bool keep)
{
    using T = typename RealOf<CT>::T;
    constexpr int LG = Sh::lg, NT = Sh::threads, TILE = Sh::tile;
    constexpr int NP = Sh::npass;
    CT *D = (NP - 1) % 2 == 0 ? Bf : A;       // where the forward half's last pass writes
    CT *E = D == Bf ? A : Bf;
    SmemTileOut<CT, LG> mid;
    mid.single = SmemRowsC<CT, LG>{D};
    mid.pair = PairSmemOut<LG>{reinterpret_cast<float2 *>(D)};
    pipe_passes<Sh, -1, N, 1, 0, 0>(typename Sh::seq{}, A, Bf, tw, mid);
    __syncthreads();
    const int k1w = 2 * k1 > n1 ? k1 - n1 : k1;
    for (int e = threadIdx.x; e < TILE; e += NT) {
        const int p = e >> LG;                 // k0 (natural order after the forward passes)
        const int k0w = 2 * p > N ? p - N : p;
        const int K = k0w * k0w + k1w * k1w + k2 * k2;
        D[e] = (keep && K > 0) ? cscale(D[e], inv_int<T>(K)) : czero<CT>();
    }
    __syncthreads();
    pipe_passes<Sh, +1, N, 1, 0, 0>(typename Sh::seq{}, D, E, tw, gout);
}

template <class P, typename V, bool TMA>
__global__ void __launch_bounds__(PipeShape<P, V>::threads, 1)
    k_poisson_pipe(const V *__restrict__ in, V *out, const __grid_constant__ CUtensorMap tmap,
                   const V *__restrict__ tw, long long W, long long tiles_per_outer, long long ntiles,
                   unsigned *err, const void *twdf, int n1, int nhp, int nh, int rev)
{
    using Sh = PipeShape<P, V>;
    constexpr int N = P::n, LINES = Sh::lines, LG = Sh::lg, NT = Sh::threads, TILE = Sh::tile;
    constexpr unsigned TILE_BYTES = TILE * sizeof(V);
    extern __shared__ __align__(1024) unsigned char pipe_smem_raw[];
    V *const buf0 = reinterpret_cast<V *>(pipe_smem_raw);
    V *const scratch = buf0 + 2 * TILE;
    unsigned long long *const bars = reinterpret_cast<unsigned long long *>(pipe_smem_raw + 3 * TILE_BYTES);
    const int tid = threadIdx.x;

    long long t = blockIdx.x;
    if (t >= ntiles) return;
    if (TMA && tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](long long tile_i, int b) {
        const long long tile = stage_order(tile_i, ntiles, rev);
        const long long o = tile / tiles_per_outer;
        const long long c0 = (tile - o * tiles_per_outer) * LINES;
        if constexpr (TMA) {
            if (tid == 0) {
                fence_async_shared();
                mbar_expect_tx(&bars[b], TILE_BYTES);
                constexpr int rows = Sh::box_rows;
                constexpr int per = (int)sizeof(V) / 8;
#pragma unroll
                for (int r0 = 0; r0 < N; r0 += rows)
                    tma_load_3d(buf0 + b * TILE + r0 * LINES, &tmap, (int)(c0 * per), r0, (int)o, &bars[b]);
            }
        } else {
            const V *src = in + o * (long long)N * W + c0;
            const int valid = (int)min((long long)LINES, W - c0);
            for (int e = tid; e < TILE; e += NT) {
                const int p = e >> LG, l = e & (LINES - 1);
                const bool ok = l < valid;
                cp_async_zfill<(int)sizeof(V)>(buf0 + b * TILE + e,
                                               ok ? (const void *)(src + (long long)p * W + l) : (const void *)src,
                                               ok);
            }
            cp_async_commit();
        }
    };

    // The load buffer is not released early here (unlike k_strided_pipe): the six passes of a
    // tile hide the next load already, and the in-place passes' extra barriers made the
    // 512-point operator slower.
    issue(t, 0);
    for (int i = 0;; ++i) {
        const int b = i & 1;
        if constexpr (TMA) {
            const bool ok = mbar_wait_bounded(&bars[b], (unsigned)((i >> 1) & 1));
            if (__syncthreads_or(!ok)) {
                if (tid == 0) atomicExch(err, 1u);
                return;
            }
        } else {
            cp_async_wait<0>();
            __syncthreads();
        }
        const long long tn = t + gridDim.x;
        if (tn < ntiles) issue(tn, b ^ 1);

        const long long tile = stage_order(t, ntiles, rev);
        const long long o = tile / tiles_per_outer;
        const long long c0 = (tile - o * tiles_per_outer) * LINES;
        const long long c = c0 + (tid & (LINES - 1));
        const int k1 = (int)(c / nhp), k2 = (int)(c - (long long)(c / nhp) * nhp);
        const bool keep = c < W && k2 < nh;
        V *X = buf0 + b * TILE;
        V *obase = out + o * (long long)N * W;
        bool done = false;
        if constexpr (std::is_same<V, double2>::value) {
            if (twdf) {
                // float-float: convert the tile into the scratch buffer, vote on range
                DfFlags f;
                dcx *Y = reinterpret_cast<dcx *>(scratch);
                for (int e = tid; e < TILE; e += NT) Y[e] = Conv<dcx, double2>::in(X[e], &f);
                if (df_tile_ok(f)) {
                    TileOut<V, dcx> g;
                    g.single = GlobalColFixedOut<V, dcx>{obase, W, c < W ? c : -1};
                    poisson_tile<Sh, N>(Y, reinterpret_cast<dcx *>(X), (const dcx *)twdf, g, n1, k1, k2, keep);
                    done = true;
                }
            }
        }
        if (!done) {
            TileOut<V> g;
            g.single = GlobalColFixedOut<V>{obase, W, c < W ? c : -1};
            if constexpr (sizeof(V) == 8) {
                const int lp = tid % (LINES / 2 > 0 ? LINES / 2 : 1);
                const long long a = c0 + 2 * lp;
                float2 *base = reinterpret_cast<float2 *>(obase);
                const bool vec = a + 1 < W && (a % 2) == 0 && (W % 2) == 0 &&
                                 (reinterpret_cast<unsigned long long>(base) & 15) == 0;
                g.pair = PairGlobalOut{base, W, a < W ? a : -1, a + 1 < W ? a + 1 : -1, vec};
            }
            poisson_tile<Sh, N>(X, scratch, tw, g, n1, k1, k2, keep);
        }
        __syncthreads();   // the next tile's load into this buffer waits for every read
        if (tn >= ntiles) break;
        t = tn;
    }
}

// The kernels of one family as untyped entry points for the host.
template <class F, typename V> KernelSet kernel_set(int n, int npass, const int *radix)
{
    KernelSet k{};
    k.n = n;
    k.npass = npass;
    for (int i = 0; i < npass && i < kMaxPasses; ++i) k.radix[i] = radix[i];
    k.fn[KS_STRIDED_FWD] = (const void *)k_strided<F, -1, V>;
    k.fn[KS_STRIDED_BWD] = (const void *)k_strided<F, +1, V>;
    k.fn[KS_CONTIG_FWD] = (const void *)k_contig<F, -1, V>;
    k.fn[KS_CONTIG_BWD] = (const void *)k_contig<F, +1, V>;
    k.fn[KS_R2C] = (const void *)k_r2c<F, V>;
    k.fn[KS_C2R] = (const void *)k_c2r<F, V>;
    k.max_threads = F::template threads<V>();
    k.generic = F::generic;
    if constexpr (F::generic) {
        k.four[0] = (const void *)k_fourstep<-1, V, F::split>;
        k.four[1] = (const void *)k_fourstep<+1, V, F::split>;
        k.poisson_mult = (const void *)k_poisson_mult<V>;
    }
    if constexpr (!F::generic) {
        // n = 1024 would need 64-byte tile rows to double-buffer; measured slower than the
        // single-buffered kernel with the same rows, so it keeps the non-pipelined kernel.
        if constexpr (F::plan::npass > 0 && F::plan::n <= 1024) {
            using P = typename F::plan;
            using Sh = PipeShape<P, V>;
            k.pipe[PIPE_FWD_TMA] = (const void *)k_strided_pipe<P, -1, V, true, F::split>;
            k.pipe[PIPE_FWD_CPASYNC] = (const void *)k_strided_pipe<P, -1, V, false, F::split>;
            k.pipe[PIPE_BWD_TMA] = (const void *)k_strided_pipe<P, +1, V, true, F::split>;
            k.pipe[PIPE_BWD_CPASYNC] = (const void *)k_strided_pipe<P, +1, V, false, F::split>;
            k.pipe_blk[0] = (const void *)k_strided_pipe<P, -1, V, true, F::split, true>;
            k.pipe_blk[1] = (const void *)k_strided_pipe<P, +1, V, true, F::split, true>;
            if constexpr (!F::split) {   // split plans run the Poisson multiply as its own kernel
                k.poisson[0] = (const void *)k_poisson_pipe<P, V, true>;
                k.poisson[1] = (const void *)k_poisson_pipe<P, V, false>;
            }
            k.pipe_lines = Sh::lines;
            k.pipe_threads = Sh::threads;
            k.pipe_smem = Sh::smem;
            if constexpr (Sh::rp_ok && !F::split) {
                k.pipe_rp[0] = (const void *)k_strided_pipe_rp<P, -1>;
                k.pipe_rp[1] = (const void *)k_strided_pipe_rp<P, +1>;
                if constexpr (P::npass >= 2) {
                    k.pipe_rp_early[0] = (const void *)k_strided_pipe_rp<P, -1, true>;
                    k.pipe_rp_early[1] = (const void *)k_strided_pipe_rp<P, +1, true>;
                }
                k.pipe_smem_rp = Sh::smem_rp;
            }
        }
    }
    return k;
}

}  // namespace afft
