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

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

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

// Waits for the given phase of the barrier for at most ~2 s.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0 && global_ns() - t0 > 2000000000ull) return false;
    }
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

__device__ __forceinline__ void fence_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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

// All passes with the tile already in shared memory: every pass but the
// last runs in place there; the last one writes to dst.
template <int S, int NT, bool First, int N, int Ns, int TwOff, typename V, class Map, class Sm, class Dst, int R,
          int... Rest>
__device__ __forceinline__ void run_passes_smem(Seq<R, Rest...>, const V *tw, int lines, const Map &map,
                                                const Sm &sm, const Dst &dst)
{
    constexpr bool Last = sizeof...(Rest) == 0;
    if (!First) __syncthreads();
    if constexpr (Last) radix_pass<R, S, false, NT>(N, Ns, tw + TwOff, lines, map, sm, dst);
    else radix_pass<R, S, true, NT>(N, Ns, tw + TwOff, lines, map, sm, sm);
    if constexpr (!Last) {
        constexpr int next = TwOff + (Ns > 1 ? Ns * (R - 1) : 0);
        run_passes_smem<S, NT, false, N, Ns * R, next>(Seq<Rest...>{}, tw, lines, map, sm, dst);
    }
}

// Compile-time shape of the pipelined strided kernel for line length N and
// complex type V: 128-byte rows, halved while two tile buffers exceed
// kPipeSmemCap; threads so that each carries at most 16 values per pass.
constexpr int kPipeSmemCap = 144 * 1024;

template <class P, typename V> struct PipeShape {
    static constexpr int row_lines = 128 / (int)sizeof(V);
    static constexpr int lines_for(int l)
    {
        return (l > 1 && 2 * P::n * l * (int)sizeof(V) > kPipeSmemCap) ? lines_for(l / 2) : l;
    }
    static constexpr int lines = lines_for(row_lines);
    static constexpr int lg = lines == 16 ? 4 : lines == 8 ? 3 : lines == 4 ? 2 : lines == 2 ? 1 : 0;
    template <int... Rs> static constexpr int threads_for(Seq<Rs...>)
    {
        int req = lines;
        for (int r : {Rs...}) {
            const int bf = lines * (P::n / r);
            const int per = bmax_for_radix(r);
            const int t = (bf + per - 1) / per;
            req = t > req ? t : req;
        }
        return (req + 31) / 32 * 32;
    }
    static constexpr int threads = threads_for(typename P::seq{});
    static_assert(threads % lines == 0, "each thread must own one column of the tile");
    static constexpr int tile = P::n * lines;                  // complex elements per tile
    static constexpr int smem = 2 * tile * (int)sizeof(V) + 16; // two buffers, then two mbarriers
    static constexpr int box_rows = tma_box_rows(P::n);
    static_assert((box_rows * lines * (int)sizeof(V)) % 128 == 0 || box_rows == P::n,
                  "TMA boxes must start 128-byte aligned in shared memory");
};

template <class P, int S, typename V, bool TMA>
__global__ void __launch_bounds__(PipeShape<P, V>::threads, 1)
    k_strided_pipe(const V *__restrict__ in, V *out, const __grid_constant__ CUtensorMap tmap,
                   const V *__restrict__ tw, long long W, long long tiles_per_outer, long long ntiles,
                   unsigned *err, long long Wout, int remap_in, int remap_out)
{
    using Sh = PipeShape<P, V>;
    constexpr int N = P::n, LINES = Sh::lines, LG = Sh::lg, NT = Sh::threads, TILE = Sh::tile;
    constexpr unsigned TILE_BYTES = TILE * sizeof(V);
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    V *const buf0 = reinterpret_cast<V *>(smem_raw);  // buffer b starts at buf0 + b * TILE
    unsigned long long *const bars = reinterpret_cast<unsigned long long *>(smem_raw + 2 * TILE_BYTES);
    const int tid = threadIdx.x;

    long long t = blockIdx.x;
    if (t >= ntiles) return;
    if (TMA && tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    auto issue = [&](long long tile, int b) {
        const long long o = tile / tiles_per_outer;
        const long long c0 = (tile - o * tiles_per_outer) * LINES;
        if constexpr (TMA) {
            if (tid == 0) {
                fence_async_shared();
                mbar_expect_tx(&bars[b], TILE_BYTES);
                constexpr int rows = Sh::box_rows;
                constexpr int per = (int)sizeof(V) / 8;  // 8-byte elements per complex value
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

    issue(t, 0);
    for (int i = 0;; ++i) {
        const int b = i & 1;
        const long long tn = t + gridDim.x;
        const bool more = tn < ntiles;
        if (more) issue(tn, b ^ 1);
        if constexpr (TMA) {
            const bool ok = mbar_wait_bounded(&bars[b], (unsigned)((i >> 1) & 1));
            if (__syncthreads_or(!ok)) {
                if (tid == 0) atomicExch(err, 1u);
                // let copies still in flight land before the CTA's shared memory goes away
                if (more) mbar_wait_bounded(&bars[b ^ 1], (unsigned)(((i + 1) >> 1) & 1));
                return;
            }
        } else {
            if (more) cp_async_wait<1>();
            else cp_async_wait<0>();
            __syncthreads();
        }
        const long long o = t / tiles_per_outer;
        const long long c0 = (t - o * tiles_per_outer) * LINES;
        // this thread's column (every pass maps it to the same column: NT is a multiple of LINES)
        const long long c = c0 + (tid & (LINES - 1));
        long long oc = c < W ? c : -1;
        if (remap_in > 0 && oc >= 0) {
            const long long q = c / remap_in, k = c - q * remap_in;
            oc = k < remap_out ? q * remap_out + k : -1;
        }
        const GlobalColRemapOut<V> dst{out + o * (long long)N * Wout, Wout, oc};
        const SmemRowsC<V, LG> tile{buf0 + b * TILE};
        run_passes_smem<S, NT, true, N, 1, 0>(typename P::seq{}, tw, LINES, MapLineFastC<LG>{}, tile, dst);
        __syncthreads();
        if (!more) break;
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
    if constexpr (!F::generic) {
        // n = 1024 would need 64-byte tile rows to double-buffer; measured slower than the
        // single-buffered kernel with the same rows, so it keeps the non-pipelined kernel.
        if constexpr (F::plan::npass > 0 && F::plan::n < 1024) {
            using P = typename F::plan;
            using Sh = PipeShape<P, V>;
            k.pipe[PIPE_FWD_TMA] = (const void *)k_strided_pipe<P, -1, V, true>;
            k.pipe[PIPE_FWD_CPASYNC] = (const void *)k_strided_pipe<P, -1, V, false>;
            k.pipe[PIPE_BWD_TMA] = (const void *)k_strided_pipe<P, +1, V, true>;
            k.pipe[PIPE_BWD_CPASYNC] = (const void *)k_strided_pipe<P, +1, V, false>;
            k.pipe_lines = Sh::lines;
            k.pipe_threads = Sh::threads;
            k.pipe_smem = Sh::smem;
        }
    }
    return k;
}

}  // namespace afft
