// kernels_split.cu -- the complex64 kernel families of split-precision plans
// (radix-16 passes on the tensor cores, fft_split.cuh): one specialised family
// per length of AFFT_SPLIT_LINE_PLANS plus the generic family, and the table
// of DFT-16 fragments those passes load.
#include "kernel_tables.cuh"

namespace afft {

namespace {

// One thread per (direction, lane, word) of the table: direction 0 is the
// forward sign S = -1, direction 1 the backward sign S = +1.  The matrix
// entries are evaluated in FP64 from the exact angle (s r mod 16) pi / 8 and
// split into FP16 hi = rn(a), lo = rn(a - hi).
__global__ void k_mma_fragments(unsigned *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * 32 * 16) return;
    const int dir = i / (32 * 16), lane = (i / 16) % 32, w = i % 16;
    const double S = dir == 0 ? -1.0 : 1.0;
    const int g = lane >> 2, q = lane & 3;
    const int mt = w >> 3, ks = (w >> 2) & 1, reg = w & 3;
    const int s = g + 8 * (reg & 1), r = 8 * ks + q + 4 * (reg >> 1);
    double sn, cs;
    sincospi((double)((s * r) % 16) / 8.0, &sn, &cs);
    const double a0 = mt == 0 ? cs : S * sn;    // coefficient of Re x_r
    const double a1 = mt == 0 ? -S * sn : cs;   // coefficient of Im x_r
    const __half h0 = __double2half(a0), h1 = __double2half(a1);
    const __half l0 = __double2half(a0 - (double)__half2float(h0));
    const __half l1 = __double2half(a1 - (double)__half2float(h1));
    unsigned *base = out + (dir * 32 + lane) * kMmaWordsPerLane;
    base[w] = (unsigned)__half_as_ushort(h0) | ((unsigned)__half_as_ushort(h1) << 16);
    base[16 + w] = (unsigned)__half_as_ushort(l0) | ((unsigned)__half_as_ushort(l1) << 16);
}

// The tcgen05 operand F of both directions (fft_tc.cuh): F[n][k] for output row n (n < 16: real
// part of output s = n; n >= 16: imaginary part of s = n - 16) and input column k = 2 r + {re,
// im}, split into FP16 hi and lo, stored K-major in 8-row x 16-byte core matrices (row group
// n / 8 at 512 bytes, k group k / 8 at 128 bytes).  Layout of `out`: [direction][hi, lo][2 KB].
// One thread per (direction, n, k); entries from FP64 sincospi of the exact angle (s r mod 16) pi / 8.
__global__ void k_tc_matrix(unsigned char *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * 32 * 32) return;
    const int dir = i / 1024, n = (i / 32) % 32, k = i % 32;
    const double S = dir == 0 ? -1.0 : 1.0;
    const int s = n % 16, r = k / 2;
    double sn, cs;
    sincospi((double)((s * r) % 16) / 8.0, &sn, &cs);
    double v;
    if (n < 16) v = (k & 1) ? -S * sn : cs;   // Re y_s = sum_r Re x_r cos - Im x_r S sin
    else v = (k & 1) ? cs : S * sn;           // Im y_s = sum_r Re x_r S sin + Im x_r cos
    const __half h = __double2half(v);
    const __half l = __double2half(v - (double)__half2float(h));
    const int off = (n / 8) * 512 + (k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2;
    unsigned char *base = out + dir * kTcBBytes;
    *reinterpret_cast<__half *>(base + off) = h;
    *reinterpret_cast<__half *>(base + 2048 + off) = l;
}

}  // namespace

static_assert(kSplitTableBytes == kMmaTableWords * sizeof(unsigned) + kTcTableBytes, "fragment table size");

cudaError_t split_fragments(unsigned *table, cudaStream_t stream)
{
    k_mma_fragments<<<(2 * 32 * 16 + 255) / 256, 256, 0, stream>>>(table);
    k_tc_matrix<<<(2 * 32 * 32 + 255) / 256, 256, 0, stream>>>(reinterpret_cast<unsigned char *>(table) +
                                                                  kMmaTableWords * sizeof(unsigned));
    return cudaGetLastError();
}

#define AFFT_X(N, ...) AFFT_KERNEL_SET(float2, true, N, ##__VA_ARGS__)

const KernelSet *spec_kernels_split(int n)
{
    static const KernelSet table[] = {AFFT_SPLIT_LINE_PLANS(AFFT_X)};
    return find_set(table, n);
}

const KernelSet *generic_kernels_split()
{
    static const KernelSet g = kernel_set<GenericSplit, float2>(0, 0, nullptr);
    return &g;
}

}  // namespace afft
