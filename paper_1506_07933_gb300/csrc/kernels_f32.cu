// kernels_f32.cu -- instantiates the stage kernels for float2: one specialised
// family per line length of AFFT_LINE_PLANS, plus the generic family.  (One
// translation unit per precision, so the two compile in parallel.)
#include "fft_pipe.cuh"

namespace afft {

namespace {
template <class P> struct Radices;
template <int N, int... Rs> struct Radices<LinePlan<N, Rs...>> {
    static constexpr int value[] = {Rs..., 0};
};
}  // namespace

#define AFFT_SPEC_SET(N, ...)                                                                         \
    kernel_set<Spec<LinePlan<N, ##__VA_ARGS__>>, float2>(N, LinePlan<N, ##__VA_ARGS__>::npass,           \
                                                       Radices<LinePlan<N, ##__VA_ARGS__>>::value),

const KernelSet *spec_kernels_f32(int n)
{
    static const KernelSet table[] = {AFFT_LINE_PLANS(AFFT_SPEC_SET)};
    for (const KernelSet &k : table)
        if (k.n == n) return &k;
    return nullptr;
}

const KernelSet *generic_kernels_f32()
{
    static const KernelSet g = kernel_set<Generic, float2>(0, 0, nullptr);
    return &g;
}

}  // namespace afft
