// afft.cu -- plan creation, execution and the C ABI of the 3-D FFT library.
//
// A plan holds, for each of the three axes, the radix factorisation of its
// line length (the Cooley-Tukey reduction of AccFFT Section 2), the twiddle
// tables of every pass computed in FP64 on the device, and the launch shape
// of the stage kernel.  Executing runs the three stages of Algorithm 1
// (P0 = P1 = 1) on the caller's stream: forward N2, N1, N0; backward N0, N1,
// N2 with the 1/N of Section 2, footnote 2 folded into the last store.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/afft.h"
#include "afft_internal.h"

using namespace afft;

// An NVTX range around a host call (visible in Nsight timelines; inert without a tool attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

struct AxisPlan {
    StageDesc desc;
    Launch launch;
    const KernelSet *ks;   // kernels for this line length (specialised or generic)
    int tw_base;           // first twiddle of this axis in the plan's table; desc.tw_off is relative
    // pipelined strided kernel (persistent CTAs) when the family has one
    bool pipe_avail;       // the family has it and it fits this device
    bool pipe;             // in use (the autotuner may switch it off)
    int pipe_slots;        // CTAs resident at once (SMs x CTAs per SM): the persistent grid's cap
    int rp_slots;          // the same for the row-pair kernel of odd-width rows (0: none)
    bool rp_early;         // row-pair tiles release their load buffer after the first pass (tunable)
};

// Four-step split of one axis whose lines are longer than a CTA holds
// (n = n_a n_b): the axis plan ax[a] runs the length-n_b DFTs along j_b (stride
// n_a W), then `a` runs the twiddle + length-n_a DFT + transposed store.
struct FourStep {
    bool on;
    int na, nb;
    AxisPlan a;            // length n_a, generic family's k_fourstep
    int wn_base;           // offset of w_n^m, m < n, in the twiddle table
};

struct afft_plan {
    int64_t n[3];
    int64_t batch;         // transforms per execute, stored back to back
    int kind;
    int precision;
    int axes;              // bit a set: axis a is transformed (7: the full 3-D transform)
    double bscale;         // factor of the backward transform (default 1 / prod of transformed n_a)
    int64_t nh;            // last-axis length of the complex array: n2 (C2C) or n2/2+1 (R2C)
    AxisPlan ax[3];        // ax[2] transforms the contiguous axis (length n2, or n2/2 for R2C)
    int post_off;          // R2C: offset of the w_{n2}^k table (n2/2+1 entries)
    void *d_tw;            // twiddle tables (float2 or double2)
    void *d_twdf;          // FP64 plans: the same tables in float-float (16 bytes per entry)
    void *d_work;          // R2C workspace: n0*n1*nh complex (the c2r stages)
    size_t work_bytes;
    int device;
    // per-stage timing (afft_plan_timing_begin / _end)
    std::vector<cudaEvent_t> events;   // 4 per record
    int timing_cap;
    int timing_count;
    unsigned *d_err;       // set by a kernel whose bounded wait ran out
    // L2-resident fusion of the N2 and N1 stages: slabs of `chunk_planes` planes,
    // the N1 stage of slab c on a second stream while the N2 stage of slab c+1 runs
    FourStep four[3];      // per axis
    void *d_four;          // four-step intermediate: n0*n1*nh complex
    unsigned *d_mma;       // split-precision plans: DFT-16 tensor-core fragments
    int contig_target;     // points per CTA of the contiguous stage (0: default)
    size_t chunk_bytes;    // requested slab size (0: off)
    // stages walk their tiles in alternating order where the previous stage wrote the same array
    // in the same plane order (forward N1 last to first after N2; backward N2 last to first after
    // N1), so they start on the part of the array still in L2; measured on the 512^3 r2c step:
    // N1 forward 0.1988 -> 0.1967 ms, c2r 0.1848 -> 0.1820 ms, while reversing the backward N0
    // stage after the forward one (columns in the same order) measured 0.001 ms slower
    bool l2_order;
    int chunk_planes;      // planes per slab; 0 when the stages run unfused
    cudaStream_t aux;
    std::vector<cudaEvent_t> chunk_ev;  // [0]: fork, then two per slab
    // blocked layout of large c2c plans (see run_blocked): a workspace holding the array as
    // [n1 / kBlk][batch * n0][kBlk][n2] and the tensor maps of the N0 and N1 stages over it
    bool blk_eligible;     // the plan's shapes allow it
    bool blocked;          // in use (workspace allocated, maps encoded)
    void *d_blk;
    size_t blk_bytes;
    alignas(64) CUtensorMap blk_map0;   // N0 stage: [(n1 / kBlk) batch][n0][kBlk n2]
    alignas(64) CUtensorMap blk_map1;   // N1 stage: [(n1 / kBlk) batch n0][kBlk][n2] boxes of kBlk rows
};

namespace {
// Rows per block of the blocked c2c layout: an N0 column of the workspace has rows kBlk n2
// complex apart (256 KB for n2 = 1024 complex64), an N1 column is n1 / kBlk runs of kBlk rows.
constexpr int kBlk = 32;
}

namespace {

// ---------------------------------------------------------------- plans ----

bool factor_ok(int64_t n)
{
    if (n < 1) return false;
    for (int p : {2, 3, 5})
        while (n % p == 0) n /= p;
    return n == 1;
}

// Radix passes for a line of n points: the power-of-two part as evenly sized
// radix-16/8/4/2 passes, then one pass per factor 3 and 5.
std::vector<int> radix_plan(int64_t n)
{
    std::vector<int> r;
    int a = 0;
    while (n % 2 == 0) { n /= 2; ++a; }
    if (a > 0) {
        const int passes = (a + 3) / 4;
        for (int i = 0; i < passes; ++i) {
            const int bits = a / passes + (i < a % passes ? 1 : 0);
            r.push_back(1 << bits);
        }
    }
    while (n % 3 == 0) { n /= 3; r.push_back(3); }
    while (n % 5 == 0) { n /= 5; r.push_back(5); }
    return r;
}

// n = n_a n_b with both factors at most kMaxLine, n_a the largest such factor
// not above sqrt(n); false if no split exists.
bool four_step_split(int64_t n, int &na, int &nb)
{
    for (int64_t a = (int64_t)std::sqrt((double)n) + 1; a >= 1; --a) {
        if (a * a > n || n % a != 0) continue;
        const int64_t b = n / a;
        if (a <= kMaxLine && b <= kMaxLine) {
            na = (int)a;
            nb = (int)b;
            return true;
        }
        return false;  // the other factor only grows for smaller a
    }
    return false;
}

const KernelSet *lookup_kernels(int precision, int64_t n)
{
    if (precision == AFFT_F32_SPLIT) {
        // split-precision sequences where the length has radix-16 passes; the FP32 kernels
        // (which then compute the same) for the other specialised lengths
        if (const KernelSet *k = spec_kernels_split((int)n)) return k;
        if (const KernelSet *k = spec_kernels_f32((int)n)) return k;
        return generic_kernels_split();
    }
    const KernelSet *k = precision == AFFT_F64 ? spec_kernels_f64((int)n) : spec_kernels_f32((int)n);
    if (k) return k;
    return precision == AFFT_F64 ? generic_kernels_f64() : generic_kernels_f32();
}

// Fills desc for length n (with the radix sequence of the specialised kernel
// when there is one) and appends its twiddle entries (m, L), meaning
// exp(-2 pi i m / L), to the table lists.
void build_desc(int64_t n, const KernelSet *ks, StageDesc &d, std::vector<int> &tm,
                std::vector<int> &tl)
{
    std::memset(&d, 0, sizeof d);
    d.n = (int)n;
    const int base = (int)tm.size();
    std::vector<int> rad;
    if (!ks->generic) rad.assign(ks->radix, ks->radix + ks->npass);
    else rad = radix_plan(n);
    d.npass = (int)rad.size();
    int ns = 1;
    for (int p = 0; p < d.npass; ++p) {
        const int R = rad[p];
        d.radix[p] = R;
        d.ns[p] = ns;
        d.tw_off[p] = (int)tm.size() - base;
        if (ns > 1) {
            for (int k = 0; k < ns; ++k)
                for (int r = 1; r < R; ++r) {
                    tm.push_back((int)(((long long)r * k) % ((long long)R * ns)));
                    tl.push_back(R * ns);
                }
        }
        ns *= R;
    }
}

int required_threads(const StageDesc &d, int lines)
{
    long long req = lines;  // copy path (n == 1)
    for (int p = 0; p < d.npass; ++p) {
        const long long bf = (long long)lines * (d.n / d.radix[p]);
        const int per = bmax_for_radix(d.radix[p]);
        req = std::max(req, (bf + per - 1) / per);
    }
    return (int)std::max(32LL, (req + 31) / 32 * 32);
}

int ilog2(int v)
{
    int l = 0;
    while ((1 << (l + 1)) <= v) ++l;
    return l;
}

// Strided stage: `lines` adjacent columns per CTA, 128-byte rows when possible.
bool shape_strided(const StageDesc &d, long long outer, long long W, size_t elem, int max_threads,
                   size_t max_smem, Launch &L)
{
    int lines = (int)(128 / elem);
    while (lines > 1 && lines / 2 >= W) lines /= 2;  // narrow arrays: no idle columns
    for (;;) {
        const int thr = required_threads(d, lines);
        const size_t smem = (size_t)d.n * lines * elem;
        if (thr <= max_threads && smem <= max_smem) {
            L.lines = lines;
            L.log2_lines = ilog2(lines);
            L.threads = thr;
            L.smem = smem;
            L.tiles_per_outer = (W + lines - 1) / lines;
            L.blocks = outer * L.tiles_per_outer;
            return L.blocks > 0 && L.blocks < (1LL << 31);
        }
        if (lines == 1) return false;
        lines /= 2;
    }
}

// Contiguous stage: whole lines, about `target` complex points per CTA
// (0: 4096 for complex64, 2048 for complex128; the autotuner may pick others).
// even_lines: an even count where possible, so that every CTA's run of lines of
// an odd number of complex64 elements starts 16-byte aligned (the c2r kernel
// then stages it with 16-byte copies).
bool shape_contig(const StageDesc &d, long long nlines, size_t elem, int max_threads, size_t max_smem,
                  Launch &L, int target = 0, bool even_lines = false)
{
    if (target <= 0) target = elem == 8 ? 4096 : 2048;
    int lines = std::max(1, target / std::max(1, d.n));
    lines = (int)std::min<long long>(lines, std::max(1LL, nlines));
    if (even_lines && lines > 1 && (lines & 1)) --lines;
    const int row = (int)(128 / elem);
    for (;;) {
        const int thr = required_threads(d, lines);
        const size_t pts = ((size_t)lines * d.n + row - 1) / row * row;
        const size_t smem = pts * elem;
        if (thr <= max_threads && smem <= max_smem) {
            L.lines = lines;
            L.log2_lines = 0;
            L.threads = thr;
            L.smem = smem;
            L.tiles_per_outer = 1;
            L.blocks = (nlines + lines - 1) / lines;
            return L.blocks > 0 && L.blocks < (1LL << 31);
        }
        if (lines == 1) return false;
        lines = (lines + 1) / 2;
    }
}

// ------------------------------------------------------------- twiddles ----

// Entry i of the table is exp(-2 pi i m_i / L_i), evaluated in FP64 from the
// exact integer ratio (m reduced to (-L/2, L/2] so the argument of sincospi
// is at most 1 in magnitude), then rounded to the table's precision.
template <typename V>
__global__ void k_twiddles(const int *__restrict__ m, const int *__restrict__ L, V *out, int count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    int mm = m[i];
    const int ll = L[i];
    if (2 * mm > ll) mm -= ll;
    double s, c;
    sincospi(2.0 * (double)mm / (double)ll, &s, &c);
    V v;
    v.x = (decltype(v.x))c;
    v.y = (decltype(v.y))(-s);
    out[i] = v;
}

// Float-float copy of an FP64 twiddle table: hi = fl(w), lo = fl(w - hi)
// (plan-time FP64 arithmetic), stored as (re.hi, re.lo, im.hi, im.lo).
__global__ void k_twiddles_df(const double2 *__restrict__ w, float4 *out, int count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double2 v = w[i];
    const float rh = (float)v.x, ih = (float)v.y;
    out[i] = make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
}

// splitmix64 (Steele, Lea, Flood 2014) as a counter-based hash.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x)
{
    unsigned long long z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

template <typename T>
__global__ void k_fill_uniform(T *out, long long count, unsigned long long seed)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * count; i += stride) {
        // i = 2 * (complex index) + part
        const unsigned long long h = splitmix64(seed ^ (unsigned long long)i);
        out[i] = (T)((double)(h >> 40) * (1.0 / 16777216.0) * 2.0 - 1.0);
    }
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? AFFT_OK : AFFT_ERR_CUDA; }

size_t cplx_size(int precision) { return precision == AFFT_F64 ? 16 : 8; }
size_t real_size(int precision) { return precision == AFFT_F64 ? 8 : 4; }

template <typename V>
int upload_twiddles(afft_plan *p, const std::vector<int> &tm, const std::vector<int> &tl)
{
    const int count = (int)tm.size();
    if (count == 0) return AFFT_OK;
    int *d_m = nullptr;
    cudaError_t e = cudaMalloc(&p->d_tw, sizeof(V) * count);
    if (e != cudaSuccess) { p->d_tw = nullptr; return AFFT_ERR_NOMEM; }
    e = cudaMalloc(&d_m, sizeof(int) * 2 * count);
    if (e != cudaSuccess) return AFFT_ERR_NOMEM;
    std::vector<int> both(tm);
    both.insert(both.end(), tl.begin(), tl.end());
    e = cudaMemcpy(d_m, both.data(), sizeof(int) * 2 * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_twiddles<V><<<(count + 255) / 256, 256>>>(d_m, d_m + count, (V *)p->d_tw, count);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_m);
    return cuda_status(e);
}

// Lets `fn` use up to `bytes` of dynamic shared memory, capped at what the device's opt-in
// maximum leaves beside the kernel's static shared memory (the tensor-core split kernels
// hold a few KB of it).
cudaError_t allow_dynamic_smem(const void *fn, int bytes, int max_smem)
{
    cudaFuncAttributes attr;
    cudaError_t e = cudaFuncGetAttributes(&attr, fn);
    if (e != cudaSuccess) return e;
    const int cap = max_smem - (int)attr.sharedSizeBytes;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, std::min(bytes, cap));
}

// CTAs of `fn` resident on one SM, from its registers, shared memory and threads alone.  The
// runtime's occupancy query returns 1 for the kernels that allocate tensor memory, whatever
// their resources (measured on 256-point split stages: 79 registers, 105 KB of shared memory,
// two CTAs resident and 22% faster than one when the grid holds two per SM).  Tensor memory
// itself does not limit them: a CTA allocates 64 to 128 of the SM's 512 columns.
int resident_per_sm(const void *fn, int threads, int dyn_smem, int device)
{
    cudaFuncAttributes fa;
    int smem_sm = 0, reserved = 0, thr_sm = 0, blk_sm = 0, regs_sm = 0;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, device) != cudaSuccess)
        return 0;
    const int warps = (threads + 31) / 32;
    // registers go to warps in units of 256, and each of the four schedulers holds a quarter
    const int warp_regs = ((std::max(fa.numRegs, 1) * 32 + 255) / 256) * 256;
    const int by_regs = (regs_sm / 4 / warp_regs) * 4 / warps;
    const int by_smem = smem_sm / ((int)fa.sharedSizeBytes + dyn_smem + reserved);
    return std::min(std::min(by_regs, by_smem), std::min(thr_sm / (warps * 32), blk_sm));
}

template <typename V>
int plan_shapes(afft_plan *p)
{
    const size_t elem = sizeof(V);
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    if (max_smem <= 0) max_smem = 48 * 1024;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    const long long n0 = p->n[0], n1 = p->n[1], nh = p->nh, B = p->batch;
    // strided stages (and the first half of a four-step contiguous axis): persistent
    // double-buffered kernels where the family has them.  A 1024-point tile has 64-byte rows
    // (two buffers must fit).  Measured on 1024-point N0/N1 stages: rows 8 KB apart 3.04 ms
    // against 3.77 ms for the non-pipelined kernel (1024^3), 2 MB apart 1.20 against 1.35 ms
    // (1024 x 512^2), 8 MB apart 6.83 against 5.48 ms (1024^3): beyond 4 MB the many CTAs of
    // the non-pipelined kernel win.
    const long long row_bytes[3] = {n1 * nh * (long long)elem, nh * (long long)elem, (long long)elem};
    for (int a = 0; a < 3; ++a) {
        if (a == 2 && !p->four[2].on) continue;
        AxisPlan &ap = p->ax[a];
        ap.pipe = false;
        const KernelSet *ks = ap.ks;
        ap.pipe_avail = false;
        ap.pipe_slots = 0;
        if (ks->generic || !ks->pipe[PIPE_FWD_TMA] || ks->pipe_smem > max_smem) continue;
        for (int k = 0; k < PIPE_COUNT; ++k)
            if (cudaFuncSetAttribute(ks->pipe[k], cudaFuncAttributeMaxDynamicSharedMemorySize, ks->pipe_smem) !=
                cudaSuccess)
                return AFFT_ERR_CUDA;
        for (int k = 0; k < 2; ++k)
            if (ks->pipe_blk[k] && cudaFuncSetAttribute(ks->pipe_blk[k], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        ks->pipe_smem) != cudaSuccess)
                return AFFT_ERR_CUDA;
        for (int k = 0; k < 2; ++k)
            if (ks->poisson[k] && cudaFuncSetAttribute(ks->poisson[k], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       ks->pipe_smem) != cudaSuccess)
                return AFFT_ERR_CUDA;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ks->pipe[PIPE_FWD_TMA], ks->pipe_threads,
                                                          ks->pipe_smem) != cudaSuccess)
            continue;
        // the split kernels hold tensor memory; their CTAs never wait on one another, so a grid
        // above what is resident is still correct
        if (p->precision == AFFT_F32_SPLIT)
            per_sm = std::max(per_sm, resident_per_sm(ks->pipe[PIPE_FWD_TMA], ks->pipe_threads, ks->pipe_smem,
                                                      p->device));
        if (per_sm < 1) continue;
        ap.pipe_slots = sms * per_sm;   // also what the blocked c2c layout runs with
        // rows far apart: the many CTAs of the plain kernel win in the row-major layout
        const bool far = ks->n >= 1024 && row_bytes[a] > (1LL << 22);
        ap.pipe_avail = !far;
        ap.pipe = !far;
        ap.rp_slots = 0;
        ap.rp_early = false;
        if (ks->pipe_rp[0] && ks->pipe_smem_rp <= max_smem) {
            bool ok = true;
            for (int k = 0; k < 2 && ok; ++k)
                ok = cudaFuncSetAttribute(ks->pipe_rp[k], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          ks->pipe_smem_rp) == cudaSuccess &&
                     (!ks->pipe_rp_early[k] ||
                      cudaFuncSetAttribute(ks->pipe_rp_early[k], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           ks->pipe_smem_rp) == cudaSuccess);
            int rs = 0;
            if (ok && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rs, ks->pipe_rp[0], ks->pipe_threads,
                                                                    ks->pipe_smem_rp) == cudaSuccess && rs >= 1)
                ap.rp_slots = sms * rs;
            // early release by default when the first pass works on column pairs (radix <= 8):
            // measured on 512-point N1 stages 0.207 -> 0.201 ms, while a radix-16 first pass
            // (384 = 16 x 8 x 3) measured 0.100 -> 0.112 ms; the autotuner tries both
            ap.rp_early = ap.rp_slots > 0 && ks->pipe_rp_early[0] && ks->radix[0] <= 8;
            cudaGetLastError();
        }
    }
    // The half spectrum keeps its compact rows of nh bins in every stage.  An odd nh makes
    // complex64 rows 8 (mod 16) bytes long, which single-row TMA boxes cannot address; the N1
    // stage then reads row pairs (k_strided_pipe_rp), and the N0 stage sees each [n1][nh]
    // plane as one row of n1 nh columns, 16-byte aligned for even n1.  (A workspace padded to
    // nh + 1 columns was measured slower: the N0 stage that converts between the layouts
    // writes or reads misaligned sectors on one side, 0.243 ms against 0.19 ms on the 512^3
    // workload.)
    p->ax[2].desc.ld = 0;
    // Specialised kernels run two CTAs per SM: keep their tiles to half the SM.
    auto budget = [&](const AxisPlan &a) -> size_t {
        return a.ks->generic ? (size_t)max_smem : (size_t)std::min(max_smem, 112 * 1024);
    };
    AxisPlan &z = p->ax[2], &y = p->ax[1], &x = p->ax[0];
    // width of each axis' lines (W of its [outer][n][W] view); a four-step axis runs
    // its first half with W * n_a
    const long long outer[3] = {B, B * n0, B * n0 * n1};
    const long long width[3] = {n1 * nh, nh, 1};
    for (int a = 0; a < 3; ++a) {
        const FourStep &f = p->four[a];
        AxisPlan &ap = p->ax[a];
        bool ok;
        if (a == 2 && !f.on)
            ok = shape_contig(z.desc, B * n0 * n1, elem, z.ks->max_threads, budget(z), z.launch, 0,
                              p->kind == AFFT_R2C && (nh & 1));
        else ok = shape_strided(ap.desc, outer[a], width[a] * (f.on ? f.na : 1), elem, ap.ks->max_threads,
                                budget(ap), ap.launch);
        if (!ok) return AFFT_ERR_UNSUPPORTED;
        if (f.on) {
            AxisPlan &fa = p->four[a].a;
            if (!shape_strided(fa.desc, outer[a] * f.nb, width[a], elem, fa.ks->max_threads, (size_t)max_smem,
                               fa.launch))
                return AFFT_ERR_UNSUPPORTED;
            for (int k = 0; k < 2; ++k)
                if (allow_dynamic_smem(fa.ks->four[k], max_smem, max_smem) != cudaSuccess)
                    return AFFT_ERR_CUDA;
        }
    }
    (void)x;
    (void)y;
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < KS_COUNT; ++k) {
            const cudaError_t e = allow_dynamic_smem(p->ax[a].ks->fn[k], max_smem, max_smem);
            if (e != cudaSuccess) return AFFT_ERR_CUDA;
        }
    return AFFT_OK;
}

// --------------------------------------------------------------- execute ---

// Shared memory of the c2r kernel: the work tile, then (specialised complex128
// kernels) the tile's half spectra staged at M + 1 elements per line; specialised
// complex64 kernels stage them in the work tile itself, so it holds
// lines * (M + 1) elements.
size_t c2r_smem(const AxisPlan &a, size_t elem)
{
    if (a.ks->generic) return a.launch.smem;
    const size_t staged = (size_t)a.launch.lines * (a.desc.n + 1) * elem;
    if (elem == 16) return a.launch.smem + staged;
    if (a.desc.mma) return a.launch.smem;   // split precision: the first pass reads global memory
    return std::max(a.launch.smem, (staged + 127) / 128 * 128);
}

cudaError_t launch(const AxisPlan &a, int which, long long blocks, void **args, cudaStream_t s)
{
    const Launch &L = a.launch;
    if (blocks <= 0) return cudaSuccess;
    return cudaLaunchKernel(a.ks->fn[which], dim3((unsigned)blocks), dim3(L.threads), args, L.smem, s);
}

long long line_blocks(const AxisPlan &a, long long nlines)
{
    return (nlines + a.launch.lines - 1) / a.launch.lines;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = []() -> EncodeTiledFn {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return (EncodeTiledFn)f;
    }();
    return fn;
}

// TMA view of a [outer][n][W] complex64 array with W odd as row pairs: dims
// (2W, n/2, outer) 8-byte elements, box (lines + 2, n/2, 1) (k_strided_pipe_rp).
bool encode_rowpair_map(CUtensorMap *map, const void *base, long long outer, int n, long long W, int lines)
{
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    if ((W % 2) != 1 || (n % 2) != 0 || n / 2 > 256 || ((uintptr_t)base) % 16 != 0 || 2 * W < lines + 2) return false;
    cuuint64_t dims[3] = {(cuuint64_t)(2 * W), (cuuint64_t)(n / 2), (cuuint64_t)outer};
    cuuint64_t strides[2] = {(cuuint64_t)(2 * W * 8), (cuuint64_t)((long long)n * W * 8)};
    cuuint32_t box[3] = {(cuuint32_t)(lines + 2), (cuuint32_t)(n / 2), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// TMA view of a [outer][n][W] complex array as 8-byte elements: dims
// (W * C/8, n, outer), box (lines * C/8, min(n, 256), 1).
bool encode_strided_map(CUtensorMap *map, const void *base, long long outer, int n, long long W, size_t C,
                        int lines)
{
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const size_t per = C / 8;
    if ((W * C) % 16 != 0 || ((uintptr_t)base) % 16 != 0 || W < lines) return false;
    cuuint64_t dims[3] = {(cuuint64_t)(W * per), (cuuint64_t)n, (cuuint64_t)outer};
    cuuint64_t strides[2] = {(cuuint64_t)(W * C), (cuuint64_t)(n * W * C)};
    cuuint32_t box[3] = {(cuuint32_t)(lines * per), (cuuint32_t)tma_box_rows(n), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The N1-stage map of the blocked c2c layout: a [n / rows][planes][rows][W] array (W complex of C
// bytes) read in boxes of `lines` columns x all n rows of one plane (every block of it).
bool encode_blocked_map(CUtensorMap *map, const void *base, long long planes, int rows, int n, long long W,
                        size_t C, int lines)
{
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const size_t per = C / 8;
    if ((W * C) % 16 != 0 || ((uintptr_t)base) % 16 != 0 || W < lines || rows < 1 || rows > 256 || n % rows != 0 ||
        n / rows > 256)
        return false;
    // [n / rows blocks][planes][rows][W]: one box of every block of a plane, rows in natural order
    cuuint64_t dims[4] = {(cuuint64_t)(W * per), (cuuint64_t)rows, (cuuint64_t)planes, (cuuint64_t)(n / rows)};
    cuuint64_t strides[3] = {(cuuint64_t)(W * C), (cuuint64_t)(rows * W * C), (cuuint64_t)(planes * rows * W * C)};
    cuuint32_t box[4] = {(cuuint32_t)(lines * per), (cuuint32_t)rows, 1, (cuuint32_t)(n / rows)};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The same [outer][n][W] array for the blocked kernel variant: the n rows as n / R groups of R =
// tma_box_rows(n), dims (W * C/8, R, outer, n / R), so that one 4-D box (all groups of line o)
// holds a tile in natural row order.
bool encode_grouped_map(CUtensorMap *map, const void *base, long long outer, int n, long long W, size_t C, int lines)
{
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const size_t per = C / 8;
    const int R = tma_box_rows(n);
    if ((W * C) % 16 != 0 || ((uintptr_t)base) % 16 != 0 || W < lines || n / R > 256) return false;
    cuuint64_t dims[4] = {(cuuint64_t)(W * per), (cuuint64_t)R, (cuuint64_t)outer, (cuuint64_t)(n / R)};
    cuuint64_t strides[3] = {(cuuint64_t)(W * C), (cuuint64_t)(n * W * C), (cuuint64_t)(R * W * C)};
    cuuint32_t box[4] = {(cuuint32_t)(lines * per), (cuuint32_t)R, 1, (cuuint32_t)(n / R)};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The pipelined kernel over a [outer][n][W] stage whose tiles load through `map` (TMA) or
// from `in` (cp.async); grouped: the map is 4-D (encode_blocked_map, encode_grouped_map), one box
// per tile, read by the kernel's blocked variant.
template <typename V>
cudaError_t pipe_on_map(const AxisPlan &a, const CUtensorMap &map, bool tma, const V *in, V *out, const V *tw,
                        long long outer, long long W, int backward, unsigned *err, bool grouped, cudaStream_t s,
                        int rev = 0)
{
    const int which = backward ? (tma ? PIPE_BWD_TMA : PIPE_BWD_CPASYNC) : (tma ? PIPE_FWD_TMA : PIPE_FWD_CPASYNC);
    const void *fn = grouped ? a.ks->pipe_blk[backward ? 1 : 0] : a.ks->pipe[which];
    if (grouped && (!tma || !fn)) return cudaErrorInvalidValue;
    tw += a.tw_base;
    long long tpo = (W + a.ks->pipe_lines - 1) / a.ks->pipe_lines;
    long long nt = outer * tpo;
    const void *twdf = a.desc.twdf;
    const unsigned *mma = a.desc.mma;
    const unsigned grid = (unsigned)std::min<long long>(nt, a.pipe_slots);
    void *args[] = {(void *)&in,  (void *)&out, (void *)&map, (void *)&tw,   (void *)&W,
                    (void *)&tpo, (void *)&nt,  (void *)&err, (void *)&twdf, (void *)&mma, (void *)&rev};
    if (nt <= 0 || grid == 0) return nt <= 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
    return cudaLaunchKernel(fn, dim3(grid), dim3(a.ks->pipe_threads), args, (size_t)a.ks->pipe_smem, s);
}

template <typename V>
cudaError_t strided_pipe(const AxisPlan &a, const V *in, V *out, const V *tw, long long outer, long long W,
                         int backward, unsigned *err, cudaStream_t s, int rev)
{
    alignas(64) CUtensorMap map;
    std::memset(&map, 0, sizeof map);
    // odd-width complex64 rows: the row-pair kernel when the family has one
    if (sizeof(V) == 8 && (W % 2) == 1 && a.rp_slots > 0 &&
        encode_rowpair_map(&map, in, outer, a.desc.n, W, a.ks->pipe_lines)) {
        tw += a.tw_base;
        long long tpo = (W + a.ks->pipe_lines - 1) / a.ks->pipe_lines;
        long long nt = outer * tpo;
        const void *twdf = nullptr;
        const unsigned *mma = nullptr;
        const unsigned grid = (unsigned)std::min<long long>(nt, a.rp_slots);
        void *args[] = {(void *)&in,  (void *)&out, (void *)&map, (void *)&tw,   (void *)&W,
                        (void *)&tpo, (void *)&nt,  (void *)&err, (void *)&twdf, (void *)&mma, (void *)&rev};
        const void *fn = a.rp_early && a.ks->pipe_rp_early[0] ? a.ks->pipe_rp_early[backward ? 1 : 0]
                                                              : a.ks->pipe_rp[backward ? 1 : 0];
        return cudaLaunchKernel(fn, dim3(grid), dim3(a.ks->pipe_threads), args, (size_t)a.ks->pipe_smem_rp, s);
    }
    const bool tma = encode_strided_map(&map, in, outer, a.desc.n, W, sizeof(V), a.ks->pipe_lines);
    return pipe_on_map<V>(a, map, tma, in, out, tw, outer, W, backward, err, false, s, rev);
}

// A strided stage over a [outer][n][W] array (in place when in == out).
template <typename V>
cudaError_t strided(const AxisPlan &a, const V *in, V *out, const V *tw, long long outer, long long W,
                    int backward, cudaStream_t s, unsigned *err, int rev = 0)
{
    if (a.pipe) return strided_pipe<V>(a, in, out, tw, outer, W, backward, err, s, rev);
    StageDesc d = a.desc;
    d.rev = rev;
    tw += a.tw_base;
    long long tpo = (W + a.launch.lines - 1) / a.launch.lines;
    int lg = a.launch.log2_lines;
    void *args[] = {(void *)&in, (void *)&out, (void *)&d, (void *)&tw, (void *)&W, (void *)&tpo, (void *)&lg};
    return launch(a, backward ? KS_STRIDED_BWD : KS_STRIDED_FWD, outer * tpo, args, s);
}

// Second half of a four-step axis: twiddle, length-n_a DFTs, transposed store.
template <typename V>
cudaError_t fourstep(const FourStep &f, const V *in, V *out, const V *tw, long long outer, long long W,
                     int backward, double scale, cudaStream_t s)
{
    using T = decltype(V().x);
    const AxisPlan &a = f.a;
    StageDesc d = a.desc;
    const V *twa = tw + a.tw_base;
    const V *wn = tw + f.wn_base;
    long long tpo = (W + a.launch.lines - 1) / a.launch.lines;
    int lg = a.launch.log2_lines, nb = f.nb;
    T sc = (T)scale;
    void *args[] = {(void *)&in, (void *)&out, (void *)&d, (void *)&twa, (void *)&wn, (void *)&W, (void *)&tpo,
                    (void *)&lg, (void *)&nb, (void *)&sc};
    const long long blocks = outer * f.nb * tpo;
    if (blocks <= 0) return cudaSuccess;
    return cudaLaunchKernel(a.ks->four[backward ? 1 : 0], dim3((unsigned)blocks), dim3(a.launch.threads), args,
                            a.launch.smem, s);
}

template <typename V>
cudaError_t contig(const AxisPlan &a, const V *in, V *out, const V *tw, long long nlines, int backward,
                   double scale, cudaStream_t s, int rev = 0)
{
    using T = decltype(V().x);
    StageDesc d = a.desc;
    d.rev = rev;
    tw += a.tw_base;
    int lines = a.launch.lines;
    T sc = (T)scale;
    void *args[] = {(void *)&in, (void *)&out, (void *)&d, (void *)&tw, (void *)&nlines, (void *)&lines, (void *)&sc};
    return launch(a, backward ? KS_CONTIG_BWD : KS_CONTIG_FWD, line_blocks(a, nlines), args, s);
}

template <typename V, typename T>
cudaError_t r2c(const AxisPlan &a, const T *in, V *out, const V *tw, const V *post, long long nlines,
                cudaStream_t s, int rev = 0)
{
    StageDesc d = a.desc;
    d.rev = rev;
    tw += a.tw_base;
    int lines = a.launch.lines;
    void *args[] = {(void *)&in, (void *)&out, (void *)&d, (void *)&tw, (void *)&post, (void *)&nlines, (void *)&lines};
    return launch(a, KS_R2C, line_blocks(a, nlines), args, s);
}

template <typename V, typename T>
cudaError_t c2r(const AxisPlan &a, const V *in, T *out, const V *tw, const V *post, long long nlines,
                double scale, cudaStream_t s, int rev = 0)
{
    StageDesc d = a.desc;
    d.rev = rev;
    tw += a.tw_base;
    int lines = a.launch.lines;
    T sc = (T)scale;
    void *args[] = {(void *)&in, (void *)&out, (void *)&d, (void *)&tw, (void *)&post, (void *)&nlines,
                    (void *)&lines, (void *)&sc};
    const long long blocks = line_blocks(a, nlines);
    if (blocks <= 0) return cudaSuccess;
    return cudaLaunchKernel(a.ks->fn[KS_C2R], dim3((unsigned)blocks), dim3(a.launch.threads), args,
                            c2r_smem(a, sizeof(V)), s);
}

// Records the timing event `i` (0..3) of the current record, if timing is on.
void mark(afft_plan *p, int i, cudaStream_t s)
{
    if (p->timing_count < p->timing_cap) cudaEventRecord(p->events[4 * p->timing_count + i], s);
    if (i == 3 && p->timing_count < p->timing_cap) ++p->timing_count;
}

// One axis stage over a [outer][n][W] view from `in` to `out` (in place when
// equal): a strided stage, or the two halves of a four-step split through the
// plan's four-step buffer.  `scale` multiplies the result (four-step only;
// unsplit strided stages are never the scaled last stage).
template <typename V>
cudaError_t axis_stage(afft_plan *p, int a, const V *in, V *out, long long outer, long long W, int backward,
                       double scale, cudaStream_t s, int rev = 0)
{
    const V *tw = (const V *)p->d_tw;
    const FourStep &f = p->four[a];
    if (!f.on) return strided<V>(p->ax[a], in, out, tw, outer, W, backward, s, p->d_err, rev);
    V *tmp = (V *)p->d_four;
    cudaError_t e = strided<V>(p->ax[a], in, tmp, tw, outer, W * f.na, backward, s, p->d_err);
    if (e != cudaSuccess) return e;
    return fourstep<V>(f, tmp, out, tw, outer, W, backward, scale, s);
}

// ------------------------------------------------------ blocked c2c layout ---
// A c2c plan whose N0 rows lie more than 4 MB apart (1024^3 complex64: 8 MB) makes every
// 1024-row tile of the N0 stage touch 1024 different 2 MB pages; that stage then runs at
// about half the bandwidth of the others, bound by address translation.  Such plans run the
// three stages through a workspace holding the array as [n1 / kBlk][B n0][kBlk][n2]:
//   N2 stage   in -> workspace, each line to its blocked place (the CTA's lines stay
//              consecutive: its line count divides kBlk);
//   N0 stage   in place on the workspace, a [(n1 / kBlk) B][n0][kBlk n2] view: rows kBlk n2
//              complex apart, kBlk rows per 2 MB page for n2 = 1024 complex64;
//   N1 stage   workspace -> out, each column read as n1 / kBlk TMA boxes of kBlk rows
//              (block k of plane o at z = k B n0 + o), written row-major.
// The backward transform runs the same kernels in the same order, the N2 stage applying the
// 1/N.  DFTs along different axes commute, so the order changes only rounding.

// Whether the plan's shapes allow the blocked layout (not whether it is worth it).
bool blocked_eligible(const afft_plan *p)
{
    if (p->kind != AFFT_C2C || p->n[0] < 2 || p->axes != 7) return false;
    for (int a = 0; a < 3; ++a)
        if (p->four[a].on) return false;
    const AxisPlan &x = p->ax[0], &y = p->ax[1], &z = p->ax[2];
    if (x.pipe_slots <= 0 || y.pipe_slots <= 0 || !x.ks->pipe_blk[0] || !y.ks->pipe_blk[0] || p->n[1] % kBlk != 0)
        return false;
    if (z.launch.lines < 1 || kBlk % z.launch.lines != 0) return false;
    const size_t C = cplx_size(p->precision);
    return (p->n[2] * (long long)C) % 16 == 0 && p->n[2] >= y.ks->pipe_lines;
}

// Allocates the workspace and encodes the two maps (on), or frees them (off).
int set_blocked(afft_plan *p, bool on)
{
    if (!on) {
        if (p->d_blk) cudaFree(p->d_blk);
        p->d_blk = nullptr;
        p->work_bytes -= p->blk_bytes;
        p->blk_bytes = 0;
        p->blocked = false;
        return AFFT_OK;
    }
    if (p->blocked) return AFFT_OK;
    if (!blocked_eligible(p)) return AFFT_ERR_UNSUPPORTED;
    const size_t C = cplx_size(p->precision);
    const long long n0 = p->n[0], n1 = p->n[1], n2 = p->n[2], P0 = p->batch * n0;
    const size_t bytes = (size_t)P0 * n1 * n2 * C;
    if (cudaMalloc(&p->d_blk, bytes) != cudaSuccess) {
        p->d_blk = nullptr;
        cudaGetLastError();
        return AFFT_ERR_NOMEM;
    }
    std::memset(&p->blk_map0, 0, sizeof p->blk_map0);
    std::memset(&p->blk_map1, 0, sizeof p->blk_map1);
    const bool ok =
        encode_grouped_map(&p->blk_map0, p->d_blk, (n1 / kBlk) * p->batch, (int)n0, kBlk * n2, C,
                           p->ax[0].ks->pipe_lines) &&
        encode_blocked_map(&p->blk_map1, p->d_blk, P0, kBlk, (int)n1, n2, C, p->ax[1].ks->pipe_lines);
    if (!ok) {
        cudaFree(p->d_blk);
        p->d_blk = nullptr;
        return AFFT_ERR_UNSUPPORTED;
    }
    p->blk_bytes = bytes;
    p->work_bytes += bytes;
    p->blocked = true;
    return AFFT_OK;
}

// Forward or backward transform through the blocked layout (see above).
template <typename V>
int run_blocked(afft_plan *p, const void *in, void *out, int backward, cudaStream_t s)
{
    const V *tw = (const V *)p->d_tw;
    const long long n0 = p->n[0], n1 = p->n[1], n2 = p->n[2], P0 = p->batch * n0;
    V *ws = (V *)p->d_blk;
    AxisPlan z = p->ax[2];   // the N2 stage writes its lines to their blocked places
    z.desc.blk = kBlk;
    z.desc.blk_in = 0;
    z.desc.blk_out = 1;
    z.desc.blk_n1 = n1;
    z.desc.blk_planes = P0;
    const double scale = backward ? p->bscale : 1.0;
    mark(p, 0, s);
    if (contig<V>(z, (const V *)in, ws, tw, P0 * n1, backward, scale, s) != cudaSuccess) return AFFT_ERR_CUDA;
    mark(p, 1, s);
    if (pipe_on_map<V>(p->ax[0], p->blk_map0, true, ws, ws, tw, (n1 / kBlk) * p->batch, kBlk * n2, backward,
                       p->d_err, true, s) != cudaSuccess)
        return AFFT_ERR_CUDA;
    mark(p, 2, s);
    if (pipe_on_map<V>(p->ax[1], p->blk_map1, true, ws, (V *)out, tw, P0, n2, backward, p->d_err, true, s) !=
        cudaSuccess)
        return AFFT_ERR_CUDA;
    mark(p, 3, s);
    return AFFT_OK;
}

// The blocked layout runs when it is set up and the current shapes still allow it (the
// autotuner may pick a contiguous CTA size or an L2 slab schedule that do not).
bool use_blocked(const afft_plan *p)
{
    return p->blocked && p->chunk_planes == 0 && blocked_eligible(p);
}

// x *= scale over `count` complex values (the backward normalisation of plans whose last
// backward stage is a strided one, i.e. plans that leave the contiguous axis untransformed).
template <typename V>
__global__ void k_scale(V *x, long long count, double scale)
{
    using T = decltype(V().x);
    const T sc = (T)scale;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        V v = x[i];
        v.x *= sc;
        v.y *= sc;
        x[i] = v;
    }
}

// Forward transform of a plan over a subset of the axes (Algorithm 1's stages for the selected
// axes only, in its order N2, N1, N0): the first stage that runs reads `in`, every stage writes
// `out`; with no stage to run, `in` is copied to `out`.
template <typename V>
int run_forward_axes(afft_plan *p, const void *in, void *out, cudaStream_t s)
{
    using T = decltype(V().x);
    const V *tw = (const V *)p->d_tw;
    const long long n0 = p->n[0], n1 = p->n[1], nh = p->nh, B = p->batch, P0 = B * n0;
    const V *src = (const V *)in;
    V *w = (V *)out;
    mark(p, 0, s);
    if (p->axes & 4) {
        cudaError_t e;
        if (p->kind == AFFT_C2C && p->four[2].on) e = axis_stage<V>(p, 2, src, w, P0 * n1, 1, 0, 1.0, s);
        else if (p->kind == AFFT_C2C) e = contig<V>(p->ax[2], src, w, tw, P0 * n1, 0, 1.0, s);
        else e = r2c<V, T>(p->ax[2], (const T *)in, w, tw, tw + p->post_off, P0 * n1, s);
        if (e != cudaSuccess) return AFFT_ERR_CUDA;
        src = w;
    }
    mark(p, 1, s);
    if ((p->axes & 2) && n1 > 1) {
        if (axis_stage<V>(p, 1, src, w, P0, nh, 0, 1.0, s) != cudaSuccess) return AFFT_ERR_CUDA;
        src = w;
    }
    mark(p, 2, s);
    if ((p->axes & 1) && n0 > 1) {
        if (axis_stage<V>(p, 0, src, w, B, n1 * nh, 0, 1.0, s) != cudaSuccess) return AFFT_ERR_CUDA;
        src = w;
    }
    if (src != w && cudaMemcpyAsync(w, src, (size_t)P0 * n1 * nh * sizeof(V), cudaMemcpyDeviceToDevice, s) !=
                        cudaSuccess)
        return AFFT_ERR_CUDA;
    mark(p, 3, s);
    return AFFT_OK;
}

// Backward transform over a subset of the axes: N0, N1, N2 among the selected ones, then the
// plan's backward factor (folded into the contiguous stage, else a separate scaling pass when
// the factor is not 1).  r2c plans always include the contiguous axis (their c2r).
template <typename V>
int run_backward_axes(afft_plan *p, const void *in, void *out, cudaStream_t s)
{
    using T = decltype(V().x);
    const V *tw = (const V *)p->d_tw;
    const long long n0 = p->n[0], n1 = p->n[1], nh = p->nh, B = p->batch, P0 = B * n0;
    const long long count = P0 * n1 * nh;
    V *buf = p->kind == AFFT_C2C ? (V *)out : (V *)p->d_work;
    const V *src = (const V *)in;
    mark(p, 0, s);
    if ((p->axes & 1) && n0 > 1) {
        if (axis_stage<V>(p, 0, src, buf, B, n1 * nh, 1, 1.0, s) != cudaSuccess) return AFFT_ERR_CUDA;
        src = buf;
    }
    mark(p, 1, s);
    if ((p->axes & 2) && n1 > 1) {
        if (axis_stage<V>(p, 1, src, buf, P0, nh, 1, 1.0, s) != cudaSuccess) return AFFT_ERR_CUDA;
        src = buf;
    }
    mark(p, 2, s);
    if (p->axes & 4) {
        cudaError_t e;
        if (p->kind == AFFT_C2C && p->four[2].on) e = axis_stage<V>(p, 2, src, (V *)out, P0 * n1, 1, 1, p->bscale, s);
        else if (p->kind == AFFT_C2C) e = contig<V>(p->ax[2], src, (V *)out, tw, P0 * n1, 1, p->bscale, s);
        else e = c2r<V, T>(p->ax[2], src, (T *)out, tw, tw + p->post_off, P0 * n1, p->bscale, s);
        if (e != cudaSuccess) return AFFT_ERR_CUDA;
    } else {
        if (src != (const V *)out &&
            cudaMemcpyAsync(out, src, (size_t)count * sizeof(V), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return AFFT_ERR_CUDA;
        if (p->bscale != 1.0) {
            const unsigned blocks = (unsigned)std::max<long long>(1, std::min<long long>((count + 255) / 256, 152LL * 16));
            k_scale<V><<<blocks, 256, 0, s>>>((V *)out, count, p->bscale);
            if (cudaGetLastError() != cudaSuccess) return AFFT_ERR_CUDA;
        }
    }
    mark(p, 3, s);
    return AFFT_OK;
}

// Forward: N2 stage (c2c, or r2c), N1 stage, N0 stage, all writing `out`.
// With chunk_planes > 0 the N2 and N1 stages run slab by slab: N2 of slab c on
// the caller's stream, N1 of slab c on the plan's second stream right after, so
// the slab is still in L2 when N1 reads it; N2 of slab c+2 waits for N1 of slab c,
// which bounds the data in flight to about three slabs.
template <typename V>
int run_forward(afft_plan *p, const void *in, void *out, cudaStream_t s)
{
    if (use_blocked(p)) return run_blocked<V>(p, in, out, 0, s);
    if (p->axes != 7) return run_forward_axes<V>(p, in, out, s);
    using T = decltype(V().x);
    const V *tw = (const V *)p->d_tw;
    const long long n0 = p->n[0], n1 = p->n[1], n2 = p->n[2], nh = p->nh, B = p->batch;
    const long long P0 = B * n0;          // planes of all transforms of the batch
    V *w = (V *)out;                      // every forward stage writes `out` (the last ones in place)
    const long long plane_in = n1 * n2;   // elements of `in` per plane (reals for r2c)
    const long long plane_w = n1 * nh;    // complex elements of `out` per plane
    auto zstage = [&](long long p0, long long np, cudaStream_t st) -> cudaError_t {
        if (p->kind == AFFT_C2C && p->four[2].on)
            return axis_stage<V>(p, 2, (const V *)in + p0 * plane_in, w + p0 * plane_w, np * n1, 1, 0, 1.0, st);
        if (p->kind == AFFT_C2C)
            return contig<V>(p->ax[2], (const V *)in + p0 * plane_in, w + p0 * plane_w, tw, np * n1, 0, 1.0, st);
        return r2c<V, T>(p->ax[2], (const T *)in + p0 * plane_in, w + p0 * plane_w, tw, tw + p->post_off,
                         np * n1, st);
    };
    // alternating tile order (see afft_plan::l2_order), with the stages unfused
    const int alt = p->l2_order && p->chunk_planes == 0;
    auto ystage = [&](long long p0, long long np, cudaStream_t st) -> cudaError_t {
        if (n1 <= 1) return cudaSuccess;
        return axis_stage<V>(p, 1, w + p0 * plane_w, w + p0 * plane_w, np, nh, 0, 1.0, st, alt);
    };
    cudaError_t e = cudaSuccess;
    mark(p, 0, s);
    const int K = p->chunk_planes;
    if (K > 0) {
        const long long C = (P0 + K - 1) / K;
        cudaEvent_t *ev = p->chunk_ev.data();
        if ((e = cudaEventRecord(ev[0], s)) != cudaSuccess) return AFFT_ERR_CUDA;
        if ((e = cudaStreamWaitEvent(p->aux, ev[0], 0)) != cudaSuccess) return AFFT_ERR_CUDA;
        for (long long c = 0; c < C && e == cudaSuccess; ++c) {
            const long long p0 = c * K, np = std::min<long long>(K, P0 - p0);
            if (c >= 2) e = cudaStreamWaitEvent(s, ev[1 + 2 * (c - 2) + 1], 0);
            if (e == cudaSuccess) e = zstage(p0, np, s);
            if (e == cudaSuccess) e = cudaEventRecord(ev[1 + 2 * c], s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(p->aux, ev[1 + 2 * c], 0);
            if (e == cudaSuccess) e = ystage(p0, np, p->aux);
            if (e == cudaSuccess) e = cudaEventRecord(ev[1 + 2 * c + 1], p->aux);
        }
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[1 + 2 * (C - 1) + 1], 0);
        if (e != cudaSuccess) return AFFT_ERR_CUDA;
        mark(p, 1, s);
        mark(p, 2, s);
    } else {
        if (zstage(0, P0, s) != cudaSuccess) return AFFT_ERR_CUDA;
        mark(p, 1, s);
        if (ystage(0, P0, s) != cudaSuccess) return AFFT_ERR_CUDA;
        mark(p, 2, s);
    }
    if (n0 > 1 && axis_stage<V>(p, 0, w, w, B, n1 * nh, 0, 1.0, s) != cudaSuccess) return AFFT_ERR_CUDA;
    mark(p, 3, s);
    return AFFT_OK;
}

// Backward: N0 stage (into the workspace for r2c plans), N1 stage, N2 stage
// (c2c with x 1/N, or c2r), fused slab by slab through L2 like the forward.
template <typename V>
int run_backward(afft_plan *p, const void *in, void *out, cudaStream_t s)
{
    if (use_blocked(p)) return run_blocked<V>(p, in, out, 1, s);
    if (p->axes != 7) return run_backward_axes<V>(p, in, out, s);
    using T = decltype(V().x);
    const V *tw = (const V *)p->d_tw;
    const long long n0 = p->n[0], n1 = p->n[1], n2 = p->n[2], nh = p->nh, B = p->batch;
    const long long P0 = B * n0;
    const double scale = p->bscale;
    // C2C works in `out`; c2r works in the plan's workspace and writes real `out` last.
    V *buf = p->kind == AFFT_C2C ? (V *)out : (V *)p->d_work;
    const long long plane_w = n1 * nh, plane_out = n1 * n2;
    auto ystage = [&](long long p0, long long np, cudaStream_t st) -> cudaError_t {
        if (n1 <= 1) return cudaSuccess;
        return axis_stage<V>(p, 1, buf + p0 * plane_w, buf + p0 * plane_w, np, nh, 1, 1.0, st);
    };
    // alternating tile order (see afft_plan::l2_order), with the stages unfused
    const int alt = p->l2_order && p->chunk_planes == 0;
    auto zstage = [&](long long p0, long long np, cudaStream_t st) -> cudaError_t {
        if (p->kind == AFFT_C2C && p->four[2].on)
            return axis_stage<V>(p, 2, buf + p0 * plane_w, (V *)out + p0 * plane_out, np * n1, 1, 1, scale, st);
        if (p->kind == AFFT_C2C)
            return contig<V>(p->ax[2], buf + p0 * plane_w, (V *)out + p0 * plane_out, tw, np * n1, 1, scale, st,
                             alt);
        return c2r<V, T>(p->ax[2], buf + p0 * plane_w, (T *)out + p0 * plane_out, tw, tw + p->post_off, np * n1,
                         scale, st, alt);
    };
    mark(p, 0, s);
    // (n0 == 1: a copy of `in` into the buffer, which c2r then transforms without touching `in`)
    if (axis_stage<V>(p, 0, (const V *)in, buf, B, n1 * nh, 1, 1.0, s) != cudaSuccess) return AFFT_ERR_CUDA;
    mark(p, 1, s);
    const int K = p->chunk_planes;
    if (K > 0) {
        const long long C = (P0 + K - 1) / K;
        cudaEvent_t *ev = p->chunk_ev.data();
        cudaError_t e = cudaEventRecord(ev[0], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->aux, ev[0], 0);
        for (long long c = 0; c < C && e == cudaSuccess; ++c) {
            const long long p0 = c * K, np = std::min<long long>(K, P0 - p0);
            if (c >= 2) e = cudaStreamWaitEvent(s, ev[1 + 2 * (c - 2) + 1], 0);
            if (e == cudaSuccess) e = ystage(p0, np, s);
            if (e == cudaSuccess) e = cudaEventRecord(ev[1 + 2 * c], s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(p->aux, ev[1 + 2 * c], 0);
            if (e == cudaSuccess) e = zstage(p0, np, p->aux);
            if (e == cudaSuccess) e = cudaEventRecord(ev[1 + 2 * c + 1], p->aux);
        }
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[1 + 2 * (C - 1) + 1], 0);
        if (e != cudaSuccess) return AFFT_ERR_CUDA;
        mark(p, 2, s);
    } else {
        if (ystage(0, P0, s) != cudaSuccess) return AFFT_ERR_CUDA;
        mark(p, 2, s);
        if (zstage(0, P0, s) != cudaSuccess) return AFFT_ERR_CUDA;
    }
    mark(p, 3, s);
    return AFFT_OK;
}

// Chooses the slab size for L2-resident N2/N1 fusion and creates the second
// stream and the events it needs (host-side objects; no device memory).
int configure_chunks(afft_plan *p, size_t bytes)
{
    p->chunk_bytes = bytes;
    p->chunk_planes = 0;
    const long long n0 = p->batch * p->n[0], n1 = p->n[1];
    const size_t plane = (size_t)n1 * p->nh * cplx_size(p->precision);
    if (bytes == 0 || n1 <= 1 || n0 < 3 || plane == 0 || p->axes != 7) return AFFT_OK;
    long long K = (long long)(bytes / plane);
    if (K < 1) K = 1;
    if (K * 2 >= n0) return AFFT_OK;  // fewer than three slabs: nothing to gain
    const long long C = (n0 + K - 1) / K;
    if (!p->aux && cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking) != cudaSuccess) {
        p->aux = nullptr;
        return AFFT_ERR_CUDA;
    }
    const size_t need = (size_t)(1 + 2 * C);
    while (p->chunk_ev.size() < need) {
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return AFFT_ERR_CUDA;
        p->chunk_ev.push_back(ev);
    }
    p->chunk_planes = (int)K;
    return AFFT_OK;
}

// Spectral Poisson solve on an R2C plan: r2c N2 and N1 stages into the
// workspace, the fused N0 operator (or N0 forward, multiply, N0 backward),
// N1 backward, c2r N2 with x 1/N.
template <typename V>
int run_poisson(afft_plan *p, const void *in, void *out, cudaStream_t s)
{
    using T = decltype(V().x);
    const V *tw = (const V *)p->d_tw;
    const long long n0 = p->n[0], n1 = p->n[1], n2 = p->n[2], nh = p->nh, B = p->batch;
    const long long P0 = B * n0;
    const double scale = 1.0 / ((double)n0 * (double)n1 * (double)n2);
    V *w = (V *)p->d_work;
    mark(p, 0, s);
    const int alt = p->l2_order;   // alternating tile order, as in run_forward / run_backward
    if (r2c<V, T>(p->ax[2], (const T *)in, w, tw, tw + p->post_off, P0 * n1, s) != cudaSuccess) return AFFT_ERR_CUDA;
    if (n1 > 1 && axis_stage<V>(p, 1, w, w, P0, nh, 0, 1.0, s, alt) != cudaSuccess) return AFFT_ERR_CUDA;
    mark(p, 1, s);
    const AxisPlan &x = p->ax[0];
    const long long W = n1 * nh;
    if (n0 > 1 && x.pipe && !p->four[0].on && x.ks->poisson[0]) {
        alignas(64) CUtensorMap map;
        std::memset(&map, 0, sizeof map);
        const bool tma = encode_strided_map(&map, w, B, x.desc.n, W, sizeof(V), x.ks->pipe_lines);
        const V *twa = tw + x.tw_base;
        long long WW = W;
        long long tpo = (W + x.ks->pipe_lines - 1) / x.ks->pipe_lines, nt = B * tpo;
        const void *twdf = x.desc.twdf;
        unsigned *err = p->d_err;
        int in1 = (int)n1, ipitch = (int)nh, inh = (int)nh, rev = 0;
        const V *win = w;
        void *args[] = {(void *)&win, (void *)&w,    (void *)&map, (void *)&twa,    (void *)&WW,
                        (void *)&tpo, (void *)&nt,   (void *)&err, (void *)&twdf,   (void *)&in1,
                        (void *)&ipitch, (void *)&inh, (void *)&rev};
        const unsigned grid = (unsigned)std::min<long long>(nt, x.pipe_slots);
        if (cudaLaunchKernel(x.ks->poisson[tma ? 0 : 1], dim3(grid), dim3(x.ks->pipe_threads), args,
                             (size_t)x.ks->pipe_smem, s) != cudaSuccess)
            return AFFT_ERR_CUDA;
    } else {
        if (n0 > 1 && axis_stage<V>(p, 0, w, w, B, W, 0, 1.0, s) != cudaSuccess) return AFFT_ERR_CUDA;
        const KernelSet *g = p->precision == AFFT_F64 ? generic_kernels_f64() : generic_kernels_f32();
        long long planes = P0;
        int a0 = (int)n0, a1 = (int)n1, a2 = (int)nh, a3 = (int)nh;
        void *args[] = {(void *)&w, (void *)&planes, (void *)&a0, (void *)&a1, (void *)&a2, (void *)&a3};
        const long long total = P0 * n1 * nh;
        const unsigned blocks = (unsigned)std::min<long long>((total + 255) / 256, 152LL * 32);
        if (cudaLaunchKernel(g->poisson_mult, dim3(blocks), dim3(256), args, 0, s) != cudaSuccess) return AFFT_ERR_CUDA;
        if (n0 > 1 && axis_stage<V>(p, 0, w, w, B, W, 1, 1.0, s) != cudaSuccess) return AFFT_ERR_CUDA;
    }
    mark(p, 2, s);
    if (n1 > 1 && axis_stage<V>(p, 1, w, w, P0, nh, 1, 1.0, s) != cudaSuccess) return AFFT_ERR_CUDA;
    if (c2r<V, T>(p->ax[2], w, (T *)out, tw, tw + p->post_off, P0 * n1, scale, s, alt) != cudaSuccess)
        return AFFT_ERR_CUDA;
    mark(p, 3, s);
    return AFFT_OK;
}

size_t in_bytes(const afft_plan *p)
{
    const size_t N = (size_t)p->batch * p->n[0] * p->n[1] * p->n[2];
    return p->kind == AFFT_C2C ? N * cplx_size(p->precision) : N * real_size(p->precision);
}
size_t out_bytes(const afft_plan *p)
{
    return (size_t)p->batch * p->n[0] * p->n[1] * p->nh * cplx_size(p->precision);
}

bool overlaps(const void *a, size_t na, const void *b, size_t nb)
{
    const char *x = (const char *)a, *y = (const char *)b;
    return x < y + nb && y < x + na;
}

int check_exec(afft_plan *p, const void *in, void *out, int backward)
{
    if (!p || !in || !out) return AFFT_ERR_NULL;
    if (in == out) return AFFT_ERR_INPLACE;
    const size_t ni = backward ? out_bytes(p) : in_bytes(p);
    const size_t no = backward ? in_bytes(p) : out_bytes(p);
    if (overlaps(in, ni, out, no)) return AFFT_ERR_INPLACE;
    return AFFT_OK;
}

// Re-shapes the contiguous stage for `target` points per CTA.
template <typename V>
bool reshape_contig(afft_plan *p, int target)
{
    if (p->four[2].on) return false;
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    if (max_smem <= 0) max_smem = 48 * 1024;
    AxisPlan &z = p->ax[2];
    const size_t budget = z.ks->generic ? (size_t)max_smem : (size_t)std::min(max_smem, 112 * 1024);
    Launch L;
    const bool even = p->kind == AFFT_R2C && ((p->n[2] / 2 + 1) & 1);
    if (!shape_contig(z.desc, p->batch * p->n[0] * p->n[1], sizeof(V), z.ks->max_threads, budget, L, target, even))
        return false;
    z.launch = L;
    p->contig_target = target;
    return true;
}

}  // namespace

bool afft::plan_view(const afft_plan *p, PlanView *v)
{
    if (!p || !v) return false;
    for (int a = 0; a < 3; ++a) {
        v->n[a] = p->n[a];
        v->tw_base[a] = p->ax[a].tw_base;
        v->line_n[a] = p->ax[a].desc.n;
        v->specialised[a] = !p->ax[a].ks->generic;
        v->npass[a] = p->ax[a].desc.npass;
        for (int i = 0; i < kMaxPasses; ++i) v->radix[a][i] = p->ax[a].desc.radix[i];
    }
    v->batch = p->batch;
    v->nh = p->nh;
    v->kind = p->kind;
    v->precision = p->precision;
    v->axes = p->axes;
    v->tw = p->d_tw;
    v->four_step = p->four[0].on || p->four[1].on || p->four[2].on;
    v->post_off = p->post_off;
    v->work = p->d_work;
    v->device = p->device;
    return true;
}

// ================================================================== C ABI ===

extern "C" {

const char *afft_status_string(int status)
{
    switch (status) {
    case AFFT_OK: return "ok";
    case AFFT_ERR_NULL: return "null pointer argument";
    case AFFT_ERR_SIZE: return "size must be >= 1 with prime factors 2, 3, 5 only";
    case AFFT_ERR_R2C_ODD: return "r2c/c2r needs an even last dimension";
    case AFFT_ERR_KIND: return "unknown transform kind";
    case AFFT_ERR_PRECISION: return "unknown precision";
    case AFFT_ERR_NOMEM: return "out of memory";
    case AFFT_ERR_INPLACE: return "in-place or overlapping buffers are not supported";
    case AFFT_ERR_CUDA: return "CUDA error";
    case AFFT_ERR_UNSUPPORTED: return "not supported by this version";
    case AFFT_ERR_SCRATCH: return "transform exceeds the fixed no-allocation scratch array";
    case AFFT_ERR_TIMEOUT: return "a kernel's bounded wait ran out (asynchronous copy never completed)";
    case AFFT_ERR_AXES: return "axes must be a nonzero subset of {0, 1, 2}, including axis 2 for r2c";
    default: return "unknown status";
    }
}

int afft_plan_create(afft_plan **out, const int64_t n[3], int kind, int precision)
{
    return afft_plan_create_batched(out, n, 1, kind, precision);
}

int afft_plan_create_batched(afft_plan **out, const int64_t n[3], int64_t batch, int kind, int precision)
{
    return afft_plan_create_axes(out, n, batch, kind, precision, 7);
}

int afft_plan_create_axes(afft_plan **out, const int64_t n[3], int64_t batch, int kind, int precision, int axes)
{
    if (!out) return AFFT_ERR_NULL;
    *out = nullptr;
    if (!n) return AFFT_ERR_NULL;
    if (kind != AFFT_C2C && kind != AFFT_R2C) return AFFT_ERR_KIND;
    if (precision != AFFT_F32 && precision != AFFT_F64 && precision != AFFT_F32_SPLIT)
        return AFFT_ERR_PRECISION;
    if (axes < 1 || axes > 7) return AFFT_ERR_AXES;
    if (kind == AFFT_R2C && !(axes & 4)) return AFFT_ERR_AXES;   // r2c halves the contiguous axis
    // transformed axes need 2/3/5-smooth lengths; the others only a length
    for (int i = 0; i < 3; ++i)
        if (((axes >> i) & 1) ? !factor_ok(n[i]) : n[i] < 1) return AFFT_ERR_SIZE;
    if (kind == AFFT_R2C && n[2] % 2 != 0) return AFFT_ERR_R2C_ODD;
    if (batch < 1) return AFFT_ERR_SIZE;
    const int64_t zlen = kind == AFFT_R2C ? n[2] / 2 : n[2];
    // lines longer than one CTA holds are split four-step (n = n_a n_b, both <= kMaxLine);
    // the contiguous axis of an r2c plan is not split
    if (kind == AFFT_R2C && zlen > kMaxLine) return AFFT_ERR_UNSUPPORTED;
    int split_a[3] = {0, 0, 0}, split_b[3] = {0, 0, 0};
    {
        const int64_t len0[3] = {n[0], n[1], zlen};
        for (int a = 0; a < 3; ++a)
            if (((axes >> a) & 1) && len0[a] > kMaxLine && !four_step_split(len0[a], split_a[a], split_b[a]))
                return AFFT_ERR_UNSUPPORTED;
    }

    afft_plan *p = new (std::nothrow) afft_plan();
    if (!p) return AFFT_ERR_NOMEM;
    for (int i = 0; i < 3; ++i) p->n[i] = n[i];
    p->batch = batch;
    p->kind = kind;
    p->precision = precision;
    p->axes = axes;
    p->bscale = 1.0;
    p->l2_order = true;
    for (int i = 0; i < 3; ++i)
        if ((axes >> i) & 1) p->bscale /= (double)n[i];
    p->nh = kind == AFFT_R2C ? n[2] / 2 + 1 : n[2];
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return AFFT_ERR_CUDA;
    }

    std::vector<int> tm, tl;
    // an axis left untransformed gets the length-1 (copy) family, which its stage never launches
    const int64_t len[3] = {(axes & 1) ? n[0] : 1, (axes & 2) ? n[1] : 1, (axes & 4) ? zlen : 1};
    bool any_four = false;
    for (int a = 0; a < 3; ++a) {
        FourStep &f = p->four[a];
        f.on = split_a[a] > 0;
        const int64_t first = f.on ? split_b[a] : len[a];   // the first (or only) DFT length
        p->ax[a].ks = lookup_kernels(precision, first);
        p->ax[a].tw_base = (int)tm.size();
        build_desc(first, p->ax[a].ks, p->ax[a].desc, tm, tl);
        if (f.on) {
            any_four = true;
            f.na = split_a[a];
            f.nb = split_b[a];
            f.a.ks = precision == AFFT_F64 ? generic_kernels_f64()
                     : precision == AFFT_F32_SPLIT ? generic_kernels_split() : generic_kernels_f32();
            f.a.tw_base = (int)tm.size();
            build_desc(f.na, f.a.ks, f.a.desc, tm, tl);
            f.wn_base = (int)tm.size();
            for (int64_t m = 0; m < len[a]; ++m) {
                tm.push_back((int)m);
                tl.push_back((int)len[a]);
            }
        }
    }
    p->post_off = (int)tm.size();
    if (kind == AFFT_R2C) {
        for (int64_t k = 0; k <= n[2] / 2; ++k) {
            tm.push_back((int)k);
            tl.push_back((int)n[2]);
        }
    }

    int st = precision == AFFT_F64 ? plan_shapes<double2>(p) : plan_shapes<float2>(p);
    if (st == AFFT_OK)
        st = precision == AFFT_F64 ? upload_twiddles<double2>(p, tm, tl) : upload_twiddles<float2>(p, tm, tl);
    if (st == AFFT_OK) {
        if (cudaMalloc(&p->d_err, sizeof(unsigned)) != cudaSuccess) {
            p->d_err = nullptr;
            st = AFFT_ERR_NOMEM;
        } else if (cudaMemset(p->d_err, 0, sizeof(unsigned)) != cudaSuccess) {
            st = AFFT_ERR_CUDA;
        } else {
            for (int a = 0; a < 3; ++a) {
                p->ax[a].desc.err = p->d_err;
                p->four[a].a.desc.err = p->d_err;
            }
        }
    }
    if (st == AFFT_OK && precision == AFFT_F64 && p->d_tw) {
        // float-float tables for the FP64 kernels' fast path; every specialised axis uses them
        const int count = (int)tm.size();
        if (cudaMalloc(&p->d_twdf, (size_t)count * 16) != cudaSuccess) {
            p->d_twdf = nullptr;
            st = AFFT_ERR_NOMEM;
        } else {
            k_twiddles_df<<<(count + 255) / 256, 256>>>((const double2 *)p->d_tw, (float4 *)p->d_twdf, count);
            if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) st = AFFT_ERR_CUDA;
            const char *base = (const char *)p->d_twdf;
            for (int a = 0; a < 3; ++a) p->ax[a].desc.twdf = base + (size_t)p->ax[a].tw_base * 16;
            p->ax[2].desc.post_df = base + (size_t)p->post_off * 16;
        }
    }
    if (st == AFFT_OK && precision == AFFT_F32_SPLIT) {
        if (cudaMalloc(&p->d_mma, kSplitTableBytes) != cudaSuccess) {
            p->d_mma = nullptr;
            st = AFFT_ERR_NOMEM;
        } else if (split_fragments(p->d_mma, 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
            st = AFFT_ERR_CUDA;
        } else {
            for (int a = 0; a < 3; ++a) {
                p->ax[a].desc.mma = p->d_mma;
                p->four[a].a.desc.mma = p->d_mma;
            }
        }
    }
    if (st == AFFT_OK && any_four) {
        const size_t bytes = (size_t)batch * n[0] * n[1] * p->nh * cplx_size(precision);
        if (cudaMalloc(&p->d_four, bytes) != cudaSuccess) {
            p->d_four = nullptr;
            st = AFFT_ERR_NOMEM;
        }
    }
    if (st == AFFT_OK && kind == AFFT_R2C) {
        p->work_bytes = (size_t)batch * n[0] * n[1] * p->nh * cplx_size(precision);
        if (cudaMalloc(&p->d_work, p->work_bytes) != cudaSuccess) {
            p->d_work = nullptr;
            p->work_bytes = 0;
            st = AFFT_ERR_NOMEM;
        }
    }
    if (st == AFFT_OK && blocked_eligible(p) && p->ax[0].ks->n >= 1024 &&
        p->n[1] * p->n[2] * (long long)cplx_size(precision) > (1LL << 22)) {
        // N0 rows beyond 4 MB apart: the blocked layout, when its workspace fits (else row-major)
        if (set_blocked(p, true) != AFFT_OK) cudaGetLastError();
    }
    if (st != AFFT_OK) {
        cudaGetLastError();  // clear a sticky launch error from the failed step
        afft_plan_destroy(p);
        return st;
    }
    *out = p;
    return AFFT_OK;
}

int afft_execute_forward(afft_plan *p, const void *in, void *out, void *stream)
{
    const int st = check_exec(p, in, out, 0);
    if (st != AFFT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const NvtxRange range("afft_execute_forward");
    return p->precision == AFFT_F64 ? run_forward<double2>(p, in, out, s) : run_forward<float2>(p, in, out, s);
}

int afft_execute_backward(afft_plan *p, const void *in, void *out, void *stream)
{
    const int st = check_exec(p, in, out, 1);
    if (st != AFFT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const NvtxRange range("afft_execute_backward");
    return p->precision == AFFT_F64 ? run_backward<double2>(p, in, out, s)
                                    : run_backward<float2>(p, in, out, s);
}

int afft_execute_poisson(afft_plan *p, const void *in, void *out, void *stream)
{
    if (!p || !in || !out) return AFFT_ERR_NULL;
    if (p->kind != AFFT_R2C) return AFFT_ERR_KIND;
    if (p->axes != 7) return AFFT_ERR_AXES;
    if (in == out) return AFFT_ERR_INPLACE;
    const size_t nb = in_bytes(p);
    if (overlaps(in, nb, out, nb)) return AFFT_ERR_INPLACE;
    cudaStream_t s = (cudaStream_t)stream;
    const NvtxRange range("afft_execute_poisson");
    return p->precision == AFFT_F64 ? run_poisson<double2>(p, in, out, s) : run_poisson<float2>(p, in, out, s);
}

static int execute_host(afft_plan *p, const void *host_in, void *host_out, void *dev_in, void *dev_out,
                        void *stream, int backward)
{
    if (!p || !host_in || !host_out || !dev_in || !dev_out) return AFFT_ERR_NULL;
    const size_t ni = backward ? out_bytes(p) : in_bytes(p);
    const size_t no = backward ? in_bytes(p) : out_bytes(p);
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(dev_in, host_in, ni, cudaMemcpyHostToDevice, s) != cudaSuccess) return AFFT_ERR_CUDA;
    const int st = backward ? afft_execute_backward(p, dev_in, dev_out, stream)
                            : afft_execute_forward(p, dev_in, dev_out, stream);
    if (st != AFFT_OK) return st;
    if (cudaMemcpyAsync(host_out, dev_out, no, cudaMemcpyDeviceToHost, s) != cudaSuccess) return AFFT_ERR_CUDA;
    return AFFT_OK;
}

int afft_execute_forward_host(afft_plan *p, const void *host_in, void *host_out, void *dev_in,
                              void *dev_out, void *stream)
{
    return execute_host(p, host_in, host_out, dev_in, dev_out, stream, 0);
}

int afft_execute_backward_host(afft_plan *p, const void *host_in, void *host_out, void *dev_in,
                               void *dev_out, void *stream)
{
    return execute_host(p, host_in, host_out, dev_in, dev_out, stream, 1);
}

int afft_plan_destroy(afft_plan *p)
{
    if (!p) return AFFT_OK;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    int st = AFFT_OK;
    if (p->d_tw || p->d_work || p->d_err || p->d_four || p->d_twdf || p->d_mma || p->d_blk) {
        if (cudaDeviceSynchronize() != cudaSuccess) st = AFFT_ERR_CUDA;
        if (p->d_blk) cudaFree(p->d_blk);
        if (p->d_tw) cudaFree(p->d_tw);
        if (p->d_twdf) cudaFree(p->d_twdf);
        if (p->d_work) cudaFree(p->d_work);
        if (p->d_err) cudaFree(p->d_err);
        if (p->d_four) cudaFree(p->d_four);
        if (p->d_mma) cudaFree(p->d_mma);
    }
    for (cudaEvent_t ev : p->events) cudaEventDestroy(ev);
    for (cudaEvent_t ev : p->chunk_ev) cudaEventDestroy(ev);
    if (p->aux) cudaStreamDestroy(p->aux);
    if (cur >= 0 && cur != p->device) cudaSetDevice(cur);
    delete p;
    return st;
}

int afft_plan_timing_begin(afft_plan *p, int capacity)
{
    if (!p) return AFFT_ERR_NULL;
    if (capacity < 1) return AFFT_ERR_SIZE;
    for (cudaEvent_t ev : p->events) cudaEventDestroy(ev);
    p->events.clear();
    p->timing_cap = 0;
    p->timing_count = 0;
    p->events.resize((size_t)capacity * 4);
    for (size_t i = 0; i < p->events.size(); ++i) {
        if (cudaEventCreate(&p->events[i]) != cudaSuccess) {
            for (size_t j = 0; j < i; ++j) cudaEventDestroy(p->events[j]);
            p->events.clear();
            return AFFT_ERR_CUDA;
        }
    }
    p->timing_cap = capacity;
    return AFFT_OK;
}

int afft_plan_timing_end(afft_plan *p, float *ms, int *count)
{
    if (!p || !ms || !count) return AFFT_ERR_NULL;
    const int n = p->timing_count;
    int st = AFFT_OK;
    if (n > 0 && cudaEventSynchronize(p->events[4 * n - 1]) != cudaSuccess) st = AFFT_ERR_CUDA;
    for (int r = 0; r < n && st == AFFT_OK; ++r)
        for (int k = 0; k < 3; ++k) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, p->events[4 * r + k], p->events[4 * r + k + 1]) != cudaSuccess) {
                st = AFFT_ERR_CUDA;
                break;
            }
            ms[3 * r + k] = t;
        }
    *count = n;
    p->timing_cap = 0;  // stop recording; the events are kept for the next begin
    p->timing_count = 0;
    return st;
}

int afft_plan_wait_probe(afft_plan *p, int limit_us, void *stream)
{
    if (!p) return AFFT_ERR_NULL;
    if (limit_us < 1 || limit_us > 2000000) return AFFT_ERR_SIZE;
    if (!p->d_err) return AFFT_ERR_CUDA;
    return launch_wait_probe(p->d_err, (unsigned long long)limit_us * 1000ull, (cudaStream_t)stream) == cudaSuccess
               ? AFFT_OK
               : AFFT_ERR_CUDA;
}

int afft_plan_device_status(afft_plan *p)
{
    if (!p) return AFFT_ERR_NULL;
    if (!p->d_err) return AFFT_OK;
    unsigned flag = 0;
    if (cudaMemcpy(&flag, p->d_err, sizeof flag, cudaMemcpyDeviceToHost) != cudaSuccess) return AFFT_ERR_CUDA;
    if (flag == 0) return AFFT_OK;
    cudaMemset(p->d_err, 0, sizeof(unsigned));
    return AFFT_ERR_TIMEOUT;
}

// ----------------------------------------------------------------- tuner --

namespace {

// Mean milliseconds of forward + backward over `reps` runs on the tuning buffers.
float time_round_trip(afft_plan *p, void *in, void *spec, void *back, cudaStream_t s, int reps)
{
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1.f;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return -1.f;
    }
    float ms = -1.f;
    if (afft_execute_forward(p, in, spec, s) == AFFT_OK && afft_execute_backward(p, spec, back, s) == AFFT_OK &&
        cudaEventRecord(a, s) == cudaSuccess) {
        bool ok = true;
        for (int r = 0; r < reps && ok; ++r)
            ok = afft_execute_forward(p, in, spec, s) == AFFT_OK && afft_execute_backward(p, spec, back, s) == AFFT_OK;
        if (ok && cudaEventRecord(b, s) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
            cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
            ms /= (float)reps;
        else
            ms = -1.f;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

}  // namespace

int afft_plan_tune(afft_plan *p, void *stream)
{
    if (!p) return AFFT_ERR_NULL;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t ib = in_bytes(p), ob = out_bytes(p);
    void *in = nullptr, *spec = nullptr, *back = nullptr;
    if (cudaMalloc(&in, ib) != cudaSuccess || cudaMalloc(&spec, ob) != cudaSuccess ||
        cudaMalloc(&back, ib) != cudaSuccess) {
        cudaFree(in);
        cudaFree(spec);
        cudaFree(back);
        cudaGetLastError();
        return AFFT_ERR_NOMEM;
    }
    const int prec = p->precision == AFFT_F64 ? AFFT_F64 : AFFT_F32;
    const size_t c = cplx_size(p->precision);
    int st = afft_fill_uniform(in, (int64_t)(ib / c), 0x7453ull, prec, stream);
    const int reps = 3;
    auto measure = [&]() { return time_round_trip(p, in, spec, back, s, reps); };
    if (st == AFFT_OK) {
        // 1. points per CTA of the contiguous stage
        if (!p->four[2].on) {
            int best_t = p->contig_target;
            float best = measure();
            for (int t : {1024, 2048, 4096, 8192}) {
                const bool ok = p->precision == AFFT_F64 ? reshape_contig<double2>(p, t) : reshape_contig<float2>(p, t);
                if (!ok) continue;
                const float ms = measure();
                if (ms > 0 && (best < 0 || ms < best)) {
                    best = ms;
                    best_t = t;
                }
            }
            if (p->precision == AFFT_F64) reshape_contig<double2>(p, best_t);
            else reshape_contig<float2>(p, best_t);
        }
        // 2. pipelined or plain kernels for the strided stages
        for (int a = 1; a >= 0; --a) {
            AxisPlan &ap = p->ax[a];
            if (!ap.pipe_avail) continue;
            ap.pipe = true;
            const float with = measure();
            ap.pipe = false;
            const float without = measure();
            ap.pipe = !(without > 0 && (with < 0 || without < with));
        }
        // 2b. row-pair tiles (odd-width complex64 rows): early release of the load buffer or not
        for (int a = 1; a >= 0; --a) {
            AxisPlan &ap = p->ax[a];
            if (!ap.pipe || ap.rp_slots <= 0 || !ap.ks->pipe_rp_early[0]) continue;
            ap.rp_early = false;
            const float plain = measure();
            ap.rp_early = true;
            const float early = measure();
            ap.rp_early = early > 0 && (plain < 0 || early < plain);
        }
        // 3. L2 slab schedule for arrays well beyond L2
        const size_t array = (size_t)p->batch * p->n[0] * p->n[1] * p->nh * c;
        if (array > ((size_t)192 << 20)) {
            size_t best_b = 0;
            configure_chunks(p, 0);
            float best = measure();
            for (size_t mb : {32, 64}) {
                if (configure_chunks(p, mb << 20) != AFFT_OK) continue;
                const float ms = measure();
                if (ms > 0 && (best < 0 || ms < best)) {
                    best = ms;
                    best_b = mb << 20;
                }
            }
            configure_chunks(p, best_b);
        }
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) st = AFFT_ERR_CUDA;
    cudaFree(in);
    cudaFree(spec);
    cudaFree(back);
    return st;
}

int afft_plan_get_tuning(const afft_plan *p, int64_t cfg[6])
{
    if (!p || !cfg) return AFFT_ERR_NULL;
    cfg[0] = p->contig_target;
    cfg[1] = p->ax[0].pipe;
    cfg[2] = p->ax[1].pipe;
    cfg[3] = (int64_t)p->chunk_bytes;
    cfg[4] = p->ax[0].rp_early;
    cfg[5] = p->ax[1].rp_early;
    return AFFT_OK;
}

int afft_plan_set_tuning(afft_plan *p, const int64_t cfg[6])
{
    if (!p || !cfg) return AFFT_ERR_NULL;
    for (int a = 0; a < 2; ++a) {
        if (cfg[1 + a] && !p->ax[a].pipe_avail) return AFFT_ERR_UNSUPPORTED;
        if (cfg[4 + a] && (p->ax[a].rp_slots <= 0 || !p->ax[a].ks->pipe_rp_early[0])) return AFFT_ERR_UNSUPPORTED;
    }
    if (cfg[0] < 0 || cfg[3] < 0 || cfg[4] < 0 || cfg[5] < 0) return AFFT_ERR_SIZE;
    if (!p->four[2].on) {
        const bool ok = p->precision == AFFT_F64 ? reshape_contig<double2>(p, (int)cfg[0])
                                                 : reshape_contig<float2>(p, (int)cfg[0]);
        if (!ok) return AFFT_ERR_UNSUPPORTED;
    }
    for (int a = 0; a < 2; ++a) {
        p->ax[a].pipe = cfg[1 + a] != 0;
        p->ax[a].rp_early = cfg[4 + a] != 0;
    }
    return configure_chunks(p, (size_t)cfg[3]);
}

namespace {

// Name of the kernel a strided stage of axis a launches over rows of W complex values.
const char *strided_kernel_name(const afft_plan *p, int a, long long W)
{
    const AxisPlan &ap = p->ax[a];
    if (!ap.pipe) return "k_strided";
    if (cplx_size(p->precision) == 8 && (W % 2) == 1 && ap.rp_slots > 0 && ap.desc.n % 2 == 0 &&
        ap.desc.n / 2 <= 256 && 2 * W >= ap.ks->pipe_lines + 2)
        return "k_strided_pipe_rp";
    return "k_strided_pipe";
}

}  // namespace

int afft_plan_describe(const afft_plan *p, char *buf, size_t len)
{
    if (!p || !buf) return AFFT_ERR_NULL;
    char radix[3][64];
    for (int a = 0; a < 3; ++a) {
        const StageDesc &d = p->ax[a].desc;
        int o = 0;
        radix[a][0] = 0;
        for (int i = 0; i < d.npass && o < 56; ++i) o += snprintf(radix[a] + o, 64 - o, i ? "x%d" : "%d", d.radix[i]);
    }
    // kernels of the stages in launch order (forward N2, N1, N0; backward N0, N1, N2); a four-step
    // axis adds k_fourstep after its strided half
    const bool blk = use_blocked(p);
    const long long W1 = p->nh, W0 = p->n[1] * p->nh;
    const char *zf = p->four[2].on ? "k_strided+k_fourstep" : p->kind == AFFT_R2C ? "k_r2c" : "k_contig";
    const char *zb = p->four[2].on ? "k_strided+k_fourstep" : p->kind == AFFT_R2C ? "k_c2r" : "k_contig";
    const char *y = !(p->axes & 2) || p->n[1] < 2 ? "none"
                    : blk ? "k_strided_pipe" : p->four[1].on ? "k_strided+k_fourstep" : strided_kernel_name(p, 1, W1);
    const char *x = !(p->axes & 1) || p->n[0] < 2 ? "none"
                    : blk ? "k_strided_pipe" : p->four[0].on ? "k_strided+k_fourstep" : strided_kernel_name(p, 0, W0);
    if (!(p->axes & 4)) zf = zb = "none";
    const int need = snprintf(
        buf, len,
        "{\"n\": [%lld, %lld, %lld], \"batch\": %lld, \"kind\": \"%s\", \"precision\": \"%s\", "
        "\"radix\": [\"%s\", \"%s\", \"%s\"], \"specialised\": [%d, %d, %d], \"four_step\": [%d, %d, %d], "
        "\"pipelined\": [%d, %d], \"contig_lines\": %d, \"strided_lines\": [%d, %d], "
        "\"l2_slab_planes\": %d, \"blocked\": %d, \"axes\": %d, \"backward_scale\": %.17g, "
        "\"rp_early\": [%d, %d], \"pipe_ctas\": [%d, %d], \"l2_order\": %d, "
        "\"stage_kernels_forward\": [\"%s\", \"%s\", \"%s\"], \"stage_kernels_backward\": [\"%s\", \"%s\", \"%s\"]}",
        (long long)p->n[0], (long long)p->n[1], (long long)p->n[2], (long long)p->batch,
        p->kind == AFFT_C2C ? "c2c" : "r2c",
        p->precision == AFFT_F64 ? "f64" : p->precision == AFFT_F32_SPLIT ? "f32split" : "f32", radix[0], radix[1], radix[2],
        !p->ax[0].ks->generic, !p->ax[1].ks->generic, !p->ax[2].ks->generic, p->four[0].on, p->four[1].on,
        p->four[2].on, p->ax[0].pipe, p->ax[1].pipe, p->ax[2].launch.lines,
        p->ax[0].pipe ? p->ax[0].ks->pipe_lines : p->ax[0].launch.lines,
        p->ax[1].pipe ? p->ax[1].ks->pipe_lines : p->ax[1].launch.lines, p->chunk_planes, (int)blk, p->axes, p->bscale,
        (int)p->ax[0].rp_early, (int)p->ax[1].rp_early, p->ax[0].pipe_slots, p->ax[1].pipe_slots, (int)p->l2_order,
        blk ? "k_contig" : zf, y, x, x, y, blk ? "k_contig" : zb);
    if (need < 0) return AFFT_ERR_CUDA;
    return (size_t)need < len ? AFFT_OK : AFFT_ERR_SIZE;
}

size_t afft_plan_workspace_bytes(const afft_plan *p) { return p ? p->work_bytes : 0; }
size_t afft_plan_input_bytes(const afft_plan *p) { return p ? in_bytes(p) : 0; }
size_t afft_plan_output_bytes(const afft_plan *p) { return p ? out_bytes(p) : 0; }

int afft_plan_launches(const afft_plan *p, int backward)
{
    if (!p) return 0;
    if (p->axes != 7) {
        const int f0 = p->four[0].on, f1 = p->four[1].on, f2 = p->four[2].on && p->kind == AFFT_C2C;
        int k = 0;
        if ((p->axes & 1) && p->n[0] > 1) k += 1 + f0;
        if ((p->axes & 2) && p->n[1] > 1) k += 1 + f1;
        if (p->axes & 4) k += 1 + f2;
        // a stage-less execution is one copy (not a kernel); a strided-only backward with a factor
        // other than 1 adds the scaling kernel
        if (backward && !(p->axes & 4) && p->bscale != 1.0) k += 1;
        return k;
    }
    const long long planes = p->batch * p->n[0];
    const long long slabs = p->chunk_planes > 0 ? (planes + p->chunk_planes - 1) / p->chunk_planes : 1;
    const int f0 = p->four[0].on, f1 = p->four[1].on, f2 = p->four[2].on && p->kind == AFFT_C2C;
    const int y = p->n[1] > 1 ? 1 + f1 : 0;
    if (backward) return (int)(1 + f0 + slabs * (1 + f2 + y));
    const int x = p->n[0] > 1 ? 1 + f0 : 0;
    return (int)(slabs * (1 + f2 + y) + x);
}

int afft_plan_set_backward_scale(afft_plan *p, double scale)
{
    if (!p) return AFFT_ERR_NULL;
    if (!(scale == scale) || scale == 0.0) return AFFT_ERR_SIZE;   // NaN or zero
    p->bscale = scale;
    return AFFT_OK;
}

double afft_plan_backward_scale(const afft_plan *p) { return p ? p->bscale : 0.0; }

int afft_copy_2d(void *dst, size_t dpitch, const void *src, size_t spitch, size_t width, size_t rows,
                 void *stream)
{
    if (rows == 0 || width == 0) return AFFT_OK;
    if (!dst || !src) return AFFT_ERR_NULL;
    if (width > dpitch || width > spitch) return AFFT_ERR_SIZE;
    return cuda_status(cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, rows, cudaMemcpyDefault,
                                         (cudaStream_t)stream));
}

int afft_plan_set_l2_order(afft_plan *p, int on)
{
    if (!p) return AFFT_ERR_NULL;
    p->l2_order = on != 0;
    return AFFT_OK;
}

int afft_plan_l2_order(const afft_plan *p) { return p && p->l2_order ? 1 : 0; }

int afft_plan_set_blocked(afft_plan *p, int on)
{
    if (!p) return AFFT_ERR_NULL;
    return set_blocked(p, on != 0);
}

int afft_plan_set_l2_chunk(afft_plan *p, size_t bytes)
{
    if (!p) return AFFT_ERR_NULL;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    const int st = configure_chunks(p, bytes);
    if (cur >= 0 && cur != p->device) cudaSetDevice(cur);
    return st;
}

size_t afft_plan_l2_chunk(const afft_plan *p)
{
    if (!p || p->chunk_planes <= 0) return 0;
    return (size_t)p->chunk_planes * (size_t)p->n[1] * p->nh * cplx_size(p->precision);
}

int afft_fill_uniform(void *dev_out, int64_t count, uint64_t seed, int precision, void *stream)
{
    if (!dev_out) return AFFT_ERR_NULL;
    if (count < 0) return AFFT_ERR_SIZE;
    if (precision != AFFT_F32 && precision != AFFT_F64) return AFFT_ERR_PRECISION;
    if (count == 0) return AFFT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int threads = 256;
    const long long want = (2 * count + threads - 1) / threads;
    const unsigned blocks = (unsigned)std::min<long long>(want, 152LL * 64);
    if (precision == AFFT_F64)
        k_fill_uniform<double><<<blocks, threads, 0, s>>>((double *)dev_out, count, seed);
    else
        k_fill_uniform<float><<<blocks, threads, 0, s>>>((float *)dev_out, count, seed);
    return cuda_status(cudaGetLastError());
}

}  // extern "C"
