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

namespace afft {

constexpr int kMaxPasses = 16;
constexpr int kMaxLine = 4096;     // longest line a single CTA transforms

struct StageDesc {
    int n;                         // line length in complex points
    int npass;                     // number of radix passes (0 when n == 1)
    int radix[kMaxPasses];         // radix of each pass
    int ns[kMaxPasses];            // product of the radices of the earlier passes
    int tw_off[kMaxPasses];        // first twiddle of each pass (complex entries)
};

// Butterflies a thread carries per pass for radix R: at most 16 complex
// values in registers (15 for radix 3 and 5).  The host picks the thread
// count so that threads * bmax(R) covers every butterfly of every pass.
__host__ __device__ constexpr int bmax_for_radix(int r)
{
    return r >= 16 ? 1 : (r == 3 ? 5 : (r == 5 ? 3 : 16 / r));
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

struct KernelSet {
    int n;                         // line length (0 for the generic family)
    int npass;
    int radix[kMaxPasses];         // the compile-time radix sequence of a specialised family
    const void *fn[KS_COUNT];
    int max_threads;               // largest CTA the kernels were compiled for
    bool generic;
};

// Specialised kernels for line length n, or nullptr.
const KernelSet *spec_kernels_f32(int n);
const KernelSet *spec_kernels_f64(int n);
// Generic kernels (any n whose radix plan the host builds).
const KernelSet *generic_kernels_f32();
const KernelSet *generic_kernels_f64();

}  // namespace afft
