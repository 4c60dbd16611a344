// selftest.cu -- failure-detection self-test: a kernel whose bounded wait can
// only run out (an mbarrier that nothing arrives at), recording the timeout
// in a plan's flag the way the pipelined kernels do (afft_plan_wait_probe).
#include "fft_pipe.cuh"

namespace afft {

namespace {

__global__ void k_wait_probe(unsigned *err, unsigned long long limit_ns)
{
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);   // no arrival, no copy: never completes
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(err, 1u);
}

}  // namespace

cudaError_t launch_wait_probe(unsigned *err, unsigned long long limit_ns, cudaStream_t stream)
{
    k_wait_probe<<<1, 32, 0, stream>>>(err, limit_ns);
    return cudaGetLastError();
}

}  // namespace afft
