// kernels_f32.cu -- instantiates the stage kernels for float2: one specialised
// family per line length of AFFT_LINE_PLANS, plus the generic family.
#include "kernel_tables.cuh"

namespace afft {

#define AFFT_X(N, ...) AFFT_KERNEL_SET(float2, false, N, ##__VA_ARGS__)

const KernelSet *spec_kernels_f32(int n)
{
    static const KernelSet table[] = {AFFT_LINE_PLANS(AFFT_X)};
    return find_set(table, n);
}

const KernelSet *generic_kernels_f32()
{
    static const KernelSet g = kernel_set<Generic, float2>(0, 0, nullptr);
    return &g;
}

}  // namespace afft
