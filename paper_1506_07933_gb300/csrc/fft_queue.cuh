// fft_queue.cuh -- persistent executor of many r2c/c2r transforms of uneven sizes.
//
// AccFFT transforms a batch of arrays by repeating its stages for each one
// (Algorithm 2's bookkeeping over a batch) and picks its kernels per size with
// its planner (Section 3).  On one GPU a set of fields of different sizes can
// run as ONE persistent launch per direction: the host lists every tile of
// every stage of every field as a work item, in an order that respects the
// stages' dependencies, and each CTA walks its share of the list (item i goes
// to CTA i mod grid).  Dependencies are counted on the device:
//
//   forward   r2c tiles of plane p     -> signal plane counter (field, p)
//             N1 tiles of plane p      wait for that plane's r2c tiles, signal the field counter
//             N0 tiles of the field    wait for all of the field's N1 tiles
//   backward  N0 tiles of the field    (from the input spectrum) signal the field counter
//             N1 tiles of plane p      wait for all N0 tiles, signal plane counter (field, p)
//             c2r tiles of plane p     wait for that plane's N1 tiles
//
// A CTA publishes a finished item with a barrier, a device-scope fence and an
// atomic increment; a consumer polls the counter (relaxed loads), fences and
// then reads, and every load of data that another CTA wrote goes through L2
// (CG accessors).  An item only ever waits for items earlier in the list, and
// all CTAs are resident, so the smallest unfinished item can always run.  Every
// wait is bounded (about 2 s of %globaltimer): a CTA that gives up sets the
// error flag and an abort flag that makes every other CTA stop at its next
// item or poll.
//
// The tile bodies are those of the specialised stage kernels (compile-time
// radix sequences, complex64), instantiated for a fixed set of line lengths.
#pragma once

#include "fft_stage.cuh"

namespace afft {

// Work item operations.
enum : unsigned char { QOP_R2C = 0, QOP_Y_FWD, QOP_X_FWD, QOP_X_BWD, QOP_Y_BWD, QOP_C2R };
constexpr unsigned kQNone = 0xffffffffu;
constexpr int kQMaxGroups = 8;
constexpr int kQThreads = 512;
constexpr int kQPoints = 8192;               // complex points per tile (64 KB of complex64)

// Columns per strided tile for lines of n points: about kQPoints / n, a power of two from
// 16 (128-byte rows) to 64 (the same on host and device).
__host__ __device__ constexpr int q_lines_for(int n)
{
    int l = 16;
    while (l < 64 && 2 * l * n <= kQPoints) l *= 2;
    return l;
}
__host__ __device__ constexpr int q_log2(int v) { return v <= 1 ? 0 : 1 + q_log2(v / 2); }

struct QItem {
    unsigned char op, group;
    unsigned short fam;                      // index into the executor's family list for this op
    unsigned a;                              // outer line (N1/N0/r2c/c2r: plane or field of the group)
    unsigned b;                              // tile within it
    unsigned wait, need;                     // counter to wait for and its target (kQNone: none)
    unsigned signal;                         // counter to increment when done (kQNone: none)
};

// One batched r2c plan of the set: buffers of the current execution and its shapes.
struct QGroup {
    const void *in;                          // forward: real [B][n0][n1][n2]; backward: spectrum
    void *out;                               // forward: spectrum [B][n0][n1][nh]; backward: real
    float2 *work;                            // backward: the plan's workspace (N0/N1 results)
    const float2 *tw[3];                     // each axis' twiddle tables
    const float2 *post;                      // w_{n2}^k, k <= n2/2
    int n0, n1, M, nh;                       // M = n2 / 2
    int zlines;                              // lines per r2c / c2r tile (tiles never straddle planes)
    float scale;                             // backward: 1 / (n0 n1 n2)
};
struct QParams {
    QGroup g[kQMaxGroups];
};

// --------------------------------------------------------------- bodies ---

template <class P>
__device__ __noinline__ void q_r2c(const QGroup &g, unsigned plane, unsigned k, float2 *sm)
{
    constexpr int M = P::n;
    const long long b0 = (long long)plane * g.n1 + (long long)k * g.zlines;
    const int valid = min(g.zlines, g.n1 - (int)k * g.zlines);
    // the input is the caller's array, written before the launch: plain loads
    const GlobalLines<float2> src{reinterpret_cast<const float2 *>(g.in) + b0 * M, M, valid};
    const SmemLines<float2> tile{sm, M};
    run_plan<P, -1, true>(g.tw[2], g.zlines, MapButterflyFast{}, src, tile, tile);
    __syncthreads();
    float2 *o = reinterpret_cast<float2 *>(g.out) + b0 * (M + 1);
    if (!r2c_post_fixed_k<M, float2, float2>(tile, o, g.post, M + 1, valid))
        r2c_post<float2, float2>(tile, o, g.post, M, M + 1, valid);
}

template <class P, int S>
__device__ __noinline__ void q_strided(const float2 *in, float2 *out, const float2 *tw, long long W,
                                          long long o, unsigned tile, float2 *sm)
{
    constexpr int N = P::n, LINES = q_lines_for(P::n), LG = q_log2(LINES);
    const long long c0 = (long long)tile * LINES;
    const long long off = o * (long long)N * W + c0;
    const int valid = (int)min((long long)LINES, W - c0);
    const GlobalCols<float2, float2, true> src{in + off, W, valid};
    const GlobalColsOut<float2> dst{out + off, W, valid};
    run_plan<P, S, false>(tw, LINES, MapLineFast{LG}, src, SmemRows<float2>{sm, LG}, dst);
}

template <class P>
__device__ __noinline__ void q_c2r(const QGroup &g, unsigned plane, unsigned k, float2 *sm)
{
    constexpr int M = P::n;
    const long long b0 = (long long)plane * g.n1 + (long long)k * g.zlines;
    const int valid = min(g.zlines, g.n1 - (int)k * g.zlines);
    const float2 *xin = g.work + b0 * (M + 1);
    const GlobalLinesOut<float2> dst{reinterpret_cast<float2 *>(g.out) + b0 * M, M, valid, g.scale};
    if ((reinterpret_cast<unsigned long long>(xin) & 15) == 0) {
        // stage the tile's half spectra with 16-byte L2 copies (an odd tail through an L2 load),
        // then the first pass in place, as the c2r kernel does
        const int elems = valid * (M + 1);
        const char *s = reinterpret_cast<const char *>(xin);
        char *d = reinterpret_cast<char *>(sm);
        for (int c = threadIdx.x; c < elems / 2; c += blockDim.x) cp_async_zfill<16>(d + 16 * c, s + 16 * c, true);
        cp_async_commit();
        if ((elems & 1) && threadIdx.x == 0) sm[elems - 1] = __ldcg(xin + elems - 1);
        cp_async_wait<0>();
        __syncthreads();
        const C2RPre<float2> sx{sm, g.post, M, M + 1, valid};
        run_plan_staged<P, +1>(typename P::seq{}, g.tw[2], g.zlines, MapButterflyFast{}, sx,
                               SmemLines<float2>{sm, M}, dst);
    } else {
        const C2RPre<float2, float2, true> sx{xin, g.post, M, M + 1, valid};
        run_plan<P, +1, false>(g.tw[2], g.zlines, MapButterflyFast{}, sx, SmemLines<float2>{sm, M}, dst);
    }
}

// Calls f.template run<P>() for the fam-th plan of Ps.
template <class F> __device__ __forceinline__ void q_dispatch(int, const F &) {}
template <class F, class P0, class... Ps> __device__ __forceinline__ void q_dispatch(int fam, const F &f)
{
    if (fam == 0) f.template run<P0>();
    else q_dispatch<F, Ps...>(fam - 1, f);
}
template <class... Ps> struct QFams {};

struct QR2C {
    const QGroup &g; unsigned a, b; float2 *sm;
    template <class P> __device__ __forceinline__ void run() const { q_r2c<P>(g, a, b, sm); }
};
struct QC2R {
    const QGroup &g; unsigned a, b; float2 *sm;
    template <class P> __device__ __forceinline__ void run() const { q_c2r<P>(g, a, b, sm); }
};
template <int S> struct QStrided {
    const float2 *in; float2 *out; const float2 *tw; long long W, o; unsigned tile; float2 *sm;
    template <class P> __device__ __forceinline__ void run() const { q_strided<P, S>(in, out, tw, W, o, tile, sm); }
};

template <class... Ps> __device__ __forceinline__ void q_run_half(QFams<Ps...>, int op, int fam, const QGroup &g,
                                                                 unsigned a, unsigned b, float2 *sm)
{
    if (op == QOP_R2C) q_dispatch<QR2C, Ps...>(fam, QR2C{g, a, b, sm});
    else q_dispatch<QC2R, Ps...>(fam, QC2R{g, a, b, sm});
}

template <class... Ps> __device__ __forceinline__ void q_run_strided(QFams<Ps...>, int op, int fam, const QGroup &g,
                                                                    unsigned a, unsigned b, float2 *sm)
{
    const long long W1 = g.nh, W0 = (long long)g.n1 * g.nh;
    switch (op) {
    case QOP_Y_FWD: {   // in place on the forward output
        float2 *x = reinterpret_cast<float2 *>(g.out);
        q_dispatch<QStrided<-1>, Ps...>(fam, QStrided<-1>{x, x, g.tw[1], W1, a, b, sm});
        break;
    }
    case QOP_X_FWD: {
        float2 *x = reinterpret_cast<float2 *>(g.out);
        q_dispatch<QStrided<-1>, Ps...>(fam, QStrided<-1>{x, x, g.tw[0], W0, a, b, sm});
        break;
    }
    case QOP_X_BWD:     // input spectrum -> workspace (the input is never modified)
        q_dispatch<QStrided<+1>, Ps...>(fam, QStrided<+1>{reinterpret_cast<const float2 *>(g.in), g.work,
                                                          g.tw[0], W0, a, b, sm});
        break;
    default:            // QOP_Y_BWD, in place on the workspace
        q_dispatch<QStrided<+1>, Ps...>(fam, QStrided<+1>{g.work, g.work, g.tw[1], W1, a, b, sm});
        break;
    }
}

// Relaxed load of a counter (device scope).
__device__ __forceinline__ unsigned q_load(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long q_now()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The persistent executor: Half lists the r2c/c2r families (half lengths M),
// Full the strided families (n0, n1).  err: set on a wait that ran out;
// abort: tells every CTA to stop.
template <class Half, class Full>
__global__ void __launch_bounds__(kQThreads, 2)
    k_queue(const __grid_constant__ QParams prm, const QItem *__restrict__ items, unsigned nitems,
            unsigned *counters, unsigned *err, unsigned *abort_flag)
{
    extern __shared__ __align__(128) unsigned char q_smem_raw[];
    float2 *sm = reinterpret_cast<float2 *>(q_smem_raw);
    __shared__ int s_go;
    // thread 0 reads each item's counter one item ahead (relaxed), so that the round trip
    // overlaps the previous item's work; the fence before the item makes it an acquire
    unsigned pre = 0;
    if (threadIdx.x == 0 && blockIdx.x < nitems && items[blockIdx.x].wait != kQNone)
        pre = q_load(counters + items[blockIdx.x].wait);
    for (unsigned i = blockIdx.x; i < nitems; i += gridDim.x) {
        const QItem it = items[i];
        if (threadIdx.x == 0) {
            int go = q_load(abort_flag) == 0;
            if (go && it.wait != kQNone && pre < it.need) {
                const unsigned long long t0 = q_now();
                for (unsigned k = 1;; ++k) {
                    if (q_load(counters + it.wait) >= it.need) break;
                    if ((k & 63u) == 0) {
                        if (q_load(abort_flag) != 0) { go = 0; break; }
                        if (q_now() - t0 > 2000000000ull) {
                            atomicExch(err, 1u);
                            atomicExch(abort_flag, 1u);
                            go = 0;
                            break;
                        }
                    }
                }
            }
            __threadfence();   // acquire side: the counter reads above, then this CTA's data reads
            s_go = go;
        }
        __syncthreads();
        if (!s_go) return;
        if (threadIdx.x == 0 && i + gridDim.x < nitems) {
            const unsigned w = items[i + gridDim.x].wait;
            pre = w != kQNone ? q_load(counters + w) : 0;
        }
        const QGroup &g = prm.g[it.group];
        if (it.op == QOP_R2C || it.op == QOP_C2R) q_run_half(Half{}, it.op, it.fam, g, it.a, it.b, sm);
        else q_run_strided(Full{}, it.op, it.fam, g, it.a, it.b, sm);
        __syncthreads();   // every thread's stores are issued, every shared read is done
        if (threadIdx.x == 0 && it.signal != kQNone) {
            __threadfence();   // release side: the CTA's stores before the increment
            atomicAdd(counters + it.signal, 1u);
        }
    }
}

}  // namespace afft
