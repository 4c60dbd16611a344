// kernels_f64_d.cu -- the double2 specialised families of the line lengths in
// AFFT_LINE_PLANS_D (the complex128 instantiations are the slowest to compile,
// so they are split over five translation units).
#include "kernel_tables.cuh"

namespace afft {

#define AFFT_X(N, ...) AFFT_KERNEL_SET(double2, false, N, ##__VA_ARGS__)

const KernelSet *spec_kernels_f64_d(int n)
{
    static const KernelSet table[] = {AFFT_LINE_PLANS_D(AFFT_X)};
    return find_set(table, n);
}

}  // namespace afft
