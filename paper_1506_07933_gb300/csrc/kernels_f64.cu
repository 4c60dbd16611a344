// kernels_f64.cu -- the double2 kernel families: the specialised ones (five
// translation units, kernels_f64_[a-e].cu) and the generic family.
#include "kernel_tables.cuh"

namespace afft {

const KernelSet *spec_kernels_f64_a(int n);
const KernelSet *spec_kernels_f64_b(int n);
const KernelSet *spec_kernels_f64_c(int n);
const KernelSet *spec_kernels_f64_d(int n);
const KernelSet *spec_kernels_f64_e(int n);

const KernelSet *spec_kernels_f64(int n)
{
    for (auto *f : {spec_kernels_f64_a, spec_kernels_f64_b, spec_kernels_f64_c, spec_kernels_f64_d,
                    spec_kernels_f64_e})
        if (const KernelSet *k = f(n)) return k;
    return nullptr;
}

const KernelSet *generic_kernels_f64()
{
    static const KernelSet g = kernel_set<Generic, double2>(0, 0, nullptr);
    return &g;
}

}  // namespace afft
