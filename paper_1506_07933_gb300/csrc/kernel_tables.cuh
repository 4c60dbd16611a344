// kernel_tables.cuh -- lookup tables of specialised kernel families: each
// translation unit instantiates the families of some line lengths (an
// X-macro list of fft_stage.cuh) for one complex type, so the heavy
// instantiations compile in parallel.
#pragma once

#include "fft_pipe.cuh"

namespace afft {

template <class P> struct RadicesOf;
template <int N, int... Rs> struct RadicesOf<LinePlan<N, Rs...>> {
    static constexpr int value[] = {Rs..., 0};
};

template <size_t K> const KernelSet *find_set(const KernelSet (&table)[K], int n)
{
    for (const KernelSet &k : table)
        if (k.n == n) return &k;
    return nullptr;
}

}  // namespace afft

// One table entry: the specialised family of LinePlan<N, radices...> for complex type V.
#define AFFT_KERNEL_SET(V, SPLIT, N, ...)                                                            \
    afft::kernel_set<afft::Spec<afft::LinePlan<N, ##__VA_ARGS__>, SPLIT>, V>(                         \
        N, afft::LinePlan<N, ##__VA_ARGS__>::npass, afft::RadicesOf<afft::LinePlan<N, ##__VA_ARGS__>>::value),
