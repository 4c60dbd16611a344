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

}  // namespace

static_assert(kSplitTableBytes == kMmaTableWords * sizeof(unsigned), "fragment table size");

cudaError_t split_fragments(unsigned *table, cudaStream_t stream)
{
    k_mma_fragments<<<(2 * 32 * 16 + 255) / 256, 256, 0, stream>>>(table);
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
