// noalloc.cu -- a c2r (backward) transform for callers that cannot allocate.
//
// Some callers cannot call cudaMalloc at all: a host framework that owns every
// byte of device memory through its own arena (a foreign cudaMalloc there is
// either refused by the arena's hard cap or breaks its accounting), or a
// latency-bound service loop that must never stall on the CUDA allocator once
// it is running.  afft_plan_create allocates a plan's twiddle tables and
// workspace, so those callers cannot use it.  afft_c2r_noalloc gives them the
// backward r2c-plan transform (half spectrum -> real field) without any
// allocation: the twiddle tables and the intermediate spectrum live in one
// file-scope __device__ array of fixed size, AFFT_NOALLOC_SCRATCH_BYTES, which
// every GPU that loads this library holds from load until process exit.  The
// caller still provides the input and the output buffers.
//
// Layout of the array: the first kTwiddleBytes hold the twiddle tables
// (rebuilt on the device by every call), the rest holds the n0*n1*(n2/2+1)
// complex intermediate.  Nothing in it has to start at zero: every call
// writes each entry it later reads.  All calls share the one array, so two
// calls whose work overlaps on the GPU (different streams, or different host
// threads) race on it and corrupt each other's results; calls on a single
// stream are ordered and safe.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so the first call on each device looks up the
// device address with cudaGetSymbolAddress, with that device current, and
// caches it.  That first call is the set-up: make it before any stream capture.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/afft.h"
#include "afft_internal.h"

using namespace afft;

namespace {

constexpr size_t kScratchBytes = AFFT_NOALLOC_SCRATCH_BYTES;
constexpr size_t kTwiddleBytes = 512 * 1024;
static_assert(kScratchBytes > kTwiddleBytes, "scratch too small");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices];

// Device address of g_scratch on `dev` (the current device), looked up once.
int scratch_address(int dev, unsigned char **addr)
{
    if (dev < 0 || dev >= kMaxDevices) return AFFT_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return AFFT_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *addr = (unsigned char *)g_scratch_addr[dev];
    return AFFT_OK;
}

bool smooth(int64_t n)
{
    if (n < 1) return false;
    for (int p : {2, 3, 5})
        while (n % p == 0) n /= p;
    return n == 1;
}

// Radix sequence for a length without specialised kernels (the generic
// kernels accept any sequence whose product is n): radix-16/8/4/2 passes of
// balanced size, then 3s, then 5s.
int radix_plan(int64_t n, int *r)
{
    int k = 0, a = 0;
    while (n % 2 == 0) { n /= 2; ++a; }
    if (a > 0) {
        const int passes = (a + 3) / 4;
        for (int i = 0; i < passes; ++i) r[k++] = 1 << (a / passes + (i < a % passes ? 1 : 0));
    }
    while (n % 3 == 0) { n /= 3; r[k++] = 3; }
    while (n % 5 == 0) { n /= 5; r[k++] = 5; }
    return k;
}

struct Axis {
    StageDesc d;
    const KernelSet *ks;
    int tw_base;
    int lines, log2_lines, threads;
    size_t smem;
    long long blocks, tpo;
};

int threads_for(const StageDesc &d, int lines)
{
    long long req = lines;
    for (int p = 0; p < d.npass; ++p) {
        const long long bf = (long long)lines * (d.n / d.radix[p]);
        const int per = bmax_for_radix(d.radix[p]);
        if ((bf + per - 1) / per > req) req = (bf + per - 1) / per;
    }
    req = (req + 31) / 32 * 32;
    return (int)(req < 32 ? 32 : req);
}

// Fills the descriptor (twiddle offsets relative to the axis) and counts its
// twiddle entries.
void describe(int64_t n, int precision, Axis &a, int &tw_count)
{
    std::memset(&a.d, 0, sizeof a.d);
    a.ks = precision == AFFT_F64 ? spec_kernels_f64((int)n) : spec_kernels_f32((int)n);
    if (!a.ks) a.ks = precision == AFFT_F64 ? generic_kernels_f64() : generic_kernels_f32();
    a.d.n = (int)n;
    int rad[kMaxPasses];
    int np;
    if (!a.ks->generic) {
        np = a.ks->npass;
        for (int i = 0; i < np; ++i) rad[i] = a.ks->radix[i];
    } else {
        np = radix_plan(n, rad);
    }
    a.d.npass = np;
    a.tw_base = tw_count;
    int ns = 1, off = 0;
    for (int p = 0; p < np; ++p) {
        a.d.radix[p] = rad[p];
        a.d.ns[p] = ns;
        a.d.tw_off[p] = off;
        if (ns > 1) off += ns * (rad[p] - 1);
        ns *= rad[p];
    }
    tw_count += off;
}

bool shape_strided(Axis &a, long long outer, long long W, size_t elem, size_t max_smem)
{
    int lines = (int)(128 / elem);
    while (lines > 1 && lines / 2 >= W) lines /= 2;
    for (;;) {
        const int thr = threads_for(a.d, lines);
        const size_t smem = (size_t)a.d.n * lines * elem;
        if (thr <= a.ks->max_threads && smem <= max_smem) {
            int lg = 0;
            while ((1 << (lg + 1)) <= lines) ++lg;
            a.lines = lines;
            a.log2_lines = lg;
            a.threads = thr;
            a.smem = smem;
            a.tpo = (W + lines - 1) / lines;
            a.blocks = outer * a.tpo;
            return a.blocks > 0 && a.blocks < (1LL << 31);
        }
        if (lines == 1) return false;
        lines /= 2;
    }
}

// even_lines: an even line count where possible, so that every CTA's run of complex64 lines
// of an odd bin count starts 16-byte aligned (the c2r kernel then stages it with 16-byte
// copies), as plans do.
bool shape_contig(Axis &a, long long nlines, size_t elem, size_t max_smem, bool even_lines)
{
    const int target = elem == 8 ? 4096 : 2048;
    int lines = target / (a.d.n > 0 ? a.d.n : 1);
    if (lines < 1) lines = 1;
    if (lines > nlines) lines = (int)(nlines > 0 ? nlines : 1);
    if (even_lines && lines > 1 && (lines & 1)) --lines;
    const int row = (int)(128 / elem);
    for (;;) {
        const int thr = threads_for(a.d, lines);
        const size_t smem = ((size_t)lines * a.d.n + row - 1) / row * row * elem;
        if (thr <= a.ks->max_threads && smem <= max_smem) {
            a.lines = lines;
            a.log2_lines = 0;
            a.threads = thr;
            a.smem = smem;
            a.tpo = 1;
            a.blocks = (nlines + lines - 1) / lines;
            return a.blocks > 0 && a.blocks < (1LL << 31);
        }
        if (lines == 1) return false;
        lines = (lines + 1) / 2;
    }
}

// Twiddle tables straight from the descriptors: for each pass with Ns > 1,
// entry k (R-1) + r-1 = exp(-2 pi i (r k mod R Ns) / (R Ns)); then the c2r
// table exp(-2 pi i k / n2), k = 0..n2/2.  FP64 sincospi, argument reduced.
struct TwJob {
    int nseg;
    int base[3 * kMaxPasses];
    int R[3 * kMaxPasses];
    int Ns[3 * kMaxPasses];
    int post_base;
    int n2;
    int total;
};

template <typename V>
__global__ void k_noalloc_twiddles(V *tw, const __grid_constant__ TwJob job)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= job.total) return;
    int m, L;
    if (i >= job.post_base) {
        m = i - job.post_base;
        L = job.n2;
    } else {
        int s = 0;
        while (s + 1 < job.nseg && i >= job.base[s + 1]) ++s;
        const int local = i - job.base[s];
        const int k = local / (job.R[s] - 1);
        const int r = local - k * (job.R[s] - 1) + 1;
        L = job.R[s] * job.Ns[s];
        m = (int)(((long long)r * k) % L);
    }
    if (2 * m > L) m -= L;
    double sn, cs;
    sincospi(2.0 * (double)m / (double)L, &sn, &cs);
    V v;
    v.x = (decltype(v.x))cs;
    v.y = (decltype(v.y))(-sn);
    tw[i] = v;
}

template <typename V>
int run(const int64_t n[3], int precision, const void *in, void *out, cudaStream_t s)
{
    using T = decltype(V().x);
    const size_t elem = sizeof(V);
    const long long n0 = n[0], n1 = n[1], M = n[2] / 2, nh = M + 1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return AFFT_ERR_CUDA;
    unsigned char *scratch = nullptr;
    int st = scratch_address(dev, &scratch);
    if (st != AFFT_OK) return st;

    Axis ax[3];  // 0: N0 (strided), 1: N1 (strided), 2: N2 c2r (contiguous, length M)
    int tw_count = 0;
    describe(n0, precision, ax[0], tw_count);
    describe(n1, precision, ax[1], tw_count);
    describe(M, precision, ax[2], tw_count);
    const int post_base = tw_count;
    tw_count += (int)nh;
    if ((size_t)tw_count * elem > kTwiddleBytes) return AFFT_ERR_SCRATCH;
    const size_t work_bytes = (size_t)n0 * n1 * nh * elem;
    if (work_bytes > kScratchBytes - kTwiddleBytes) return AFFT_ERR_SCRATCH;

    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (max_smem <= 0) max_smem = 48 * 1024;
    // the dynamic shared memory a kernel may take: the opt-in maximum less its static shared
    // memory (the c2r kernels hold an mbarrier there)
    const void *fns[3] = {ax[0].ks->fn[KS_STRIDED_BWD], ax[1].ks->fn[KS_STRIDED_BWD], ax[2].ks->fn[KS_C2R]};
    int dyn_max[3];
    for (int a = 0; a < 3; ++a) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, fns[a]) != cudaSuccess) return AFFT_ERR_CUDA;
        dyn_max[a] = max_smem - (int)fa.sharedSizeBytes;
    }
    auto budget = [&](int a) -> size_t {
        return ax[a].ks->generic ? (size_t)dyn_max[a] : (size_t)std::min(dyn_max[a], 112 * 1024);
    };
    if (!shape_strided(ax[0], 1, n1 * nh, elem, budget(0)) || !shape_strided(ax[1], n0, nh, elem, budget(1)) ||
        !shape_contig(ax[2], n0 * n1, elem, budget(2), elem == 8 && (nh & 1)))
        return AFFT_ERR_UNSUPPORTED;
    for (int a = 0; a < 3; ++a)
        if (cudaFuncSetAttribute(fns[a], cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max[a]) != cudaSuccess)
            return AFFT_ERR_CUDA;

    V *tw = (V *)scratch;
    V *work = (V *)(scratch + kTwiddleBytes);

    TwJob job;
    std::memset(&job, 0, sizeof job);
    for (int a = 0; a < 3; ++a)
        for (int p = 0; p < ax[a].d.npass; ++p) {
            if (ax[a].d.ns[p] <= 1) continue;
            job.base[job.nseg] = ax[a].tw_base + ax[a].d.tw_off[p];
            job.R[job.nseg] = ax[a].d.radix[p];
            job.Ns[job.nseg] = ax[a].d.ns[p];
            ++job.nseg;
        }
    job.post_base = post_base;
    job.n2 = (int)n[2];
    job.total = tw_count;
    k_noalloc_twiddles<V><<<(tw_count + 255) / 256, 256, 0, s>>>(tw, job);
    if (cudaGetLastError() != cudaSuccess) return AFFT_ERR_CUDA;

    const V *vin = (const V *)in;
    const V *post = tw + post_base;
    const double scale = 1.0 / ((double)n[0] * (double)n[1] * (double)n[2]);
    // N0 stage: in -> work
    {
        const Axis &a = ax[0];
        StageDesc d = a.d;
        const V *twa = tw + a.tw_base;
        long long W = n1 * nh, tpo = a.tpo;
        int lg = a.log2_lines;
        void *args[] = {(void *)&vin, (void *)&work, (void *)&d, (void *)&twa, (void *)&W, (void *)&tpo,
                        (void *)&lg};
        if (cudaLaunchKernel(a.ks->fn[KS_STRIDED_BWD], dim3((unsigned)a.blocks), dim3(a.threads), args, a.smem,
                             s) != cudaSuccess)
            return AFFT_ERR_CUDA;
    }
    // N1 stage: work -> work
    if (n1 > 1) {
        const Axis &a = ax[1];
        StageDesc d = a.d;
        const V *twa = tw + a.tw_base;
        const V *win = work;
        long long W = nh, tpo = a.tpo;
        int lg = a.log2_lines;
        void *args[] = {(void *)&win, (void *)&work, (void *)&d, (void *)&twa, (void *)&W, (void *)&tpo,
                        (void *)&lg};
        if (cudaLaunchKernel(a.ks->fn[KS_STRIDED_BWD], dim3((unsigned)a.blocks), dim3(a.threads), args, a.smem,
                             s) != cudaSuccess)
            return AFFT_ERR_CUDA;
    }
    // N2 c2r stage: work -> out (x 1/N)
    {
        const Axis &a = ax[2];
        StageDesc d = a.d;
        const V *twa = tw + a.tw_base;
        const V *win = work;
        T *o = (T *)out;
        long long nlines = n0 * n1;
        int lines = a.lines;
        T sc = (T)scale;
        void *args[] = {(void *)&win, (void *)&o, (void *)&d, (void *)&twa, (void *)&post, (void *)&nlines,
                        (void *)&lines, (void *)&sc};
        // specialised c2r kernels stage the tile's half spectra: complex128 behind the work tile,
        // complex64 in the work tile itself (lines * (M + 1) elements)
        const size_t staged = (size_t)a.lines * (a.d.n + 1) * sizeof(V);
        const size_t smem = a.ks->generic ? a.smem
                            : sizeof(V) == 16 ? a.smem + staged
                                              : (a.smem > (staged + 127) / 128 * 128 ? a.smem : (staged + 127) / 128 * 128);
        if (cudaLaunchKernel(a.ks->fn[KS_C2R], dim3((unsigned)a.blocks), dim3(a.threads), args, smem, s) !=
            cudaSuccess)
            return AFFT_ERR_CUDA;
    }
    return AFFT_OK;
}

}  // namespace

extern "C" int afft_c2r_noalloc(const int64_t n[3], int precision, const void *in, void *out,
                                void *cuda_stream)
{
    if (!n || !in || !out) return AFFT_ERR_NULL;
    if (precision != AFFT_F32 && precision != AFFT_F64 && precision != AFFT_F32_SPLIT)
        return AFFT_ERR_PRECISION;
    for (int i = 0; i < 3; ++i)
        if (!smooth(n[i])) return AFFT_ERR_SIZE;
    if (n[2] % 2 != 0) return AFFT_ERR_R2C_ODD;
    if (precision == AFFT_F32_SPLIT) return AFFT_ERR_UNSUPPORTED;
    if (n[0] > kMaxLine || n[1] > kMaxLine || n[2] / 2 > kMaxLine) return AFFT_ERR_UNSUPPORTED;
    const size_t c = precision == AFFT_F64 ? 16 : 8;
    const size_t in_bytes = (size_t)n[0] * n[1] * (n[2] / 2 + 1) * c;
    const size_t out_bytes = (size_t)n[0] * n[1] * n[2] * (c / 2);
    const char *a = (const char *)in, *b = (const char *)out;
    if (a < b + out_bytes && b < a + in_bytes) return AFFT_ERR_INPLACE;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    return precision == AFFT_F64 ? run<double2>(n, precision, in, out, s) : run<float2>(n, precision, in, out, s);
}
