// afft_internal.h -- shared host/device declarations of the CUDA library.
//
// One 3-D transform is three "stages" (Algorithm 1 of AccFFT, with the
// process grid P0 = P1 = 1): batched 1-D FFTs along the contiguous axis N2,
// then along N1, then along N0 (reverse order for the backward transform).
// Each stage is one kernel launch.  A stage transforms every line of length n
// with a Stockham autosort FFT made of radix-R passes (R in 16, 8, 4, 2, 3, 5);
// StageDesc carries that factorisation and the offsets of each pass's twiddle
// table in the plan's device buffer.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

struct afft_plan;

namespace afft {

constexpr int kMaxPasses = 16;
constexpr int kMaxLine = 4096;     // longest line a single CTA transforms

struct StageDesc {
    int n;                         // line length in complex points
    int npass;                     // number of radix passes (0 when n == 1)
    int radix[kMaxPasses];         // radix of each pass
    int ns[kMaxPasses];            // product of the radices of the earlier passes
    int tw_off[kMaxPasses];        // first twiddle of each pass (complex entries)
    int ld;                        // r2c/c2r stage: stride between half-spectrum lines, in complex
                                   // elements; 0 means compact (M + 1 for a line of M points)
    // FP64 plans: the same twiddle tables as float-float values (hi, lo floats),
    // or null to compute in FP64 (specialised kernels then use float-float)
    const void *twdf;              // this axis' tables, same offsets as `tw`
    const void *post_df;           // the r2c/c2r table w_{2M}^k
    // split-precision plans: the tensor-core fragments of the 16-point DFT matrix
    // (both directions, see fft_split.cuh), else null
    const unsigned *mma;
    // contiguous c2c stage of a blocked plan: the lines of `in` (blk_in) or of `out` (blk_out)
    // lie in the layout [n1 / blk][planes][blk][n], line q = plane * n1 + j at line
    // ((j / blk) * planes + plane) * blk + j % blk; blk = 0: row-major on both sides
    int blk, blk_in, blk_out;
    long long blk_n1, blk_planes;
    unsigned *err;                 // set by a kernel whose bounded wait ran out (null: not reported)
    // 1: the CTAs take their line blocks (or tiles) in reverse order, last first, so that a stage
    // following one that wrote the same array front to back starts on the part still in L2
    int rev;
};

// Block (or tile) i of n in the order a stage walks them.
__host__ __device__ inline long long stage_order(long long i, long long n, int rev) { return rev ? n - 1 - i : i; }

// Line of the blocked layout holding row-major line q (see StageDesc::blk).
__host__ __device__ inline long long blocked_line(const StageDesc &d, long long q)
{
    const long long pl = q / d.blk_n1, j = q - pl * d.blk_n1;
    return ((j / d.blk) * d.blk_planes + pl) * d.blk + j % d.blk;
}

// Butterflies a thread carries per pass for radix R: at most 16 complex
// values in registers (15 for radix 3 and 5).  The host picks the thread
// count so that threads * bmax(R) covers every butterfly of every pass.
__host__ __device__ constexpr int bmax_for_radix(int r)
{
    return r >= 16 ? 1 : (r == 3 ? 5 : (r == 5 ? 3 : 16 / r));
}

// Rows per TMA box when a line of n rows is loaded in boxes of at most 256
// rows: the largest divisor of n not above 256, so the boxes tile the line
// exactly (used identically by the kernels and by the host's tensor maps).
__host__ __device__ constexpr int tma_box_rows(int n)
{
    int r = n < 256 ? n : 256;
    while (r > 1 && n % r != 0) --r;
    return r;
}

struct Launch {
    int lines;                     // lines (columns) per CTA
    int log2_lines;                // log2(lines) for the strided stage (lines is a power of 2)
    int threads;                   // threads per CTA
    size_t smem;                   // dynamic shared memory bytes
    long long blocks;              // grid size
    long long tiles_per_outer;     // strided stage: CTAs per outer slab
};

// Entry points of one kernel family (a specialised line length, or the
// generic kernels), indexed by KS_*.  Signatures, with V = float2 / double2
// and T its real type:
//   strided: (const V *in, V *out, StageDesc d, const V *tw, long long W,
//             long long tiles_per_outer, int log2_lines)
//   contig:  (const V *in, V *out, StageDesc d, const V *tw, long long nlines,
//             int lines, T scale)
//   r2c:     (const T *in, V *out, StageDesc d, const V *tw, const V *post_tw,
//             long long nlines, int lines)
//   c2r:     (const V *in, T *out, StageDesc d, const V *tw, const V *post_tw,
//             long long nlines, int lines, T scale)
enum { KS_STRIDED_FWD = 0, KS_STRIDED_BWD, KS_CONTIG_FWD, KS_CONTIG_BWD, KS_R2C, KS_C2R, KS_COUNT };

// Pipelined strided kernels (persistent CTAs, double-buffered tiles), indexed
// by PIPE_*.  Signature: (const V *in, V *out, CUtensorMap map, const V *tw,
// long long W, long long tiles_per_outer, long long ntiles, unsigned *err,
// const void *twdf, const unsigned *mma, int rev) (twdf: the float-float
// twiddles of an FP64 plan, or null; mma: the tensor-core DFT-16 table of a
// split-precision plan, or null; rev: walk the tiles last to first, see
// StageDesc::rev); the TMA variants read through `map`, a [outer][n][W] view,
// the cp.async ones through `in`; the blocked variants (pipe_blk, TMA) read a
// 4-D map [n / R][outer][R][W] with one box per tile (the blocked c2c
// workspace, or the rows of a [outer][n][W] array grouped by R).  The row-pair
// kernels (pipe_rp) take the same arguments.
enum { PIPE_FWD_TMA = 0, PIPE_FWD_CPASYNC, PIPE_BWD_TMA, PIPE_BWD_CPASYNC, PIPE_COUNT };

struct KernelSet {
    int n;                         // line length (0 for the generic family)
    int npass;
    int radix[kMaxPasses];         // the compile-time radix sequence of a specialised family
    const void *fn[KS_COUNT];
    int max_threads;               // largest CTA the kernels were compiled for
    bool generic;
    const void *pipe[PIPE_COUNT];  // null when the family has no pipelined strided kernel
    const void *pipe_blk[2];       // its blocked-row TMA variants ([0] forward, [1] backward)
    // generic family only: second half of a four-step line, (const V *in, V *out,
    // StageDesc d, const V *tw, const V *wn, long long W, long long tiles_per_outer,
    // int log2_lines, int nb, T scale); [0] forward, [1] backward
    const void *four[2];
    // generic family only: (V *x, long long planes, int n0, int n1, int nhp, int nh)
    const void *poisson_mult;
    // fused Poisson N0 stage (forward DFTs, 1/|k|^2, inverse DFTs) on pipelined tiles:
    // (const V *in, V *out, CUtensorMap map, const V *tw, long long W,
    // long long tiles_per_outer, long long ntiles, unsigned *err, const void *twdf,
    // int n1, int nhp, int nh, int rev); [0] TMA, [1] cp.async
    const void *poisson[2];
    int pipe_lines;                // columns per tile of the pipelined kernel
    int pipe_threads;              // its (compile-time) CTA size
    int pipe_smem;                 // its dynamic shared memory (two tile buffers)
    // complex64 families: the pipelined kernels for rows of odd width, read as row pairs
    // through TMA ([0] forward, [1] backward; the first ten arguments of pipe[], see
    // k_strided_pipe_rp) and their shared memory; null / 0 elsewhere
    const void *pipe_rp[2];
    const void *pipe_rp_early[2];  // the same with the load buffer released after the first pass
    int pipe_smem_rp;
};

// Specialised kernels for line length n, or nullptr.
const KernelSet *spec_kernels_f32(int n);
const KernelSet *spec_kernels_f64(int n);
// Generic kernels (any n whose radix plan the host builds).
const KernelSet *generic_kernels_f32();
const KernelSet *generic_kernels_f64();
// Generic complex64 kernels whose radix-16 passes run on the tensor cores
// (split-precision plans), and the device table of their DFT-16 fragments
// (kSplitTableBytes, written by split_fragments on `stream`).
// Failure-detection self-test (selftest.cu): one CTA waits at most limit_ns on
// an mbarrier that nothing completes, then sets *err.
cudaError_t launch_wait_probe(unsigned *err, unsigned long long limit_ns, cudaStream_t stream);
const KernelSet *generic_kernels_split();

// What the persistent multi-plan executor (queue.cu) reads from a plan.
struct PlanView {
    long long n[3], batch, nh;
    int kind, precision, axes;
    const void *tw;            // twiddle tables (complex of the plan's precision)
    int tw_base[3];            // first twiddle of each axis' tables
    int line_n[3];             // line length of each axis' stages (n0, n1, n2 or n2/2)
    bool specialised[3];       // the axis runs a specialised (compile-time radix) family
    int radix[3][kMaxPasses];  // that family's radix sequence (npass entries)
    int npass[3];
    bool four_step;            // some axis is split four-step
    int post_off;              // r2c: first entry of the w_{n2}^k table
    void *work;                // r2c workspace (n0 n1 nh complex per transform)
    int device;
};
bool plan_view(const afft_plan *p, PlanView *v);
const KernelSet *spec_kernels_split(int n);
// the mma.sync fragments (2 directions x 32 lanes x 32 words), then the tcgen05 operands
// F_hi, F_lo of both directions in the canonical shared-memory layout (2 x 2 x 2 KB)
constexpr size_t kSplitTableBytes = 2 * 32 * 32 * sizeof(unsigned) + 2 * 2 * 32 * 64;
cudaError_t split_fragments(unsigned *table, cudaStream_t stream);

}  // namespace afft
