/*
 * afft.h -- C ABI of a single-GPU (GB300, sm_103a) 3-D FFT library.
 *
 * What it computes.  AccFFT (Gholami, Hill, Malhotra, Biros, arXiv 1506.07933)
 * describes a library that, given an N0 x N1 x N2 array, computes its Fourier
 * transform (Section 1, "Contributions"), R2C, C2C and C2R, in single and
 * double precision, by batched 1-D FFTs along one axis at a time with
 * transposes between them (Algorithm 1, pencil decomposition).  On one GPU the
 * process grid is P0 = P1 = 1 and the paper's all-to-all exchanges become data
 * movement inside the device; this library computes the same result:
 *
 *   forward   X[k0,k1,k2] = sum_j x[j0,j1,j2] exp(-2 pi i (j0k0/N0 + j1k1/N1 + j2k2/N2))
 *   backward  x[j]        = (1/N) sum_k X[k] exp(+2 pi i (...)),  N = N0 N1 N2
 *
 * The forward transform is unscaled and the backward one carries the full
 * 1/N normalisation (Section 2, footnote 2), so backward(forward(x)) = x.
 * The exponent sign is not printed in the paper; the one above is that of
 * the FFT libraries the paper builds on.
 *
 * Layout.  Row-major [n0][n1][n2], n[0] slowest and n[2] contiguous: the
 * paper's N0, N1, N2 (Section 2 notation).  The frequency-domain array keeps
 * the same axis order as the spatial one (Section 2: AccFFT keeps the xyz
 * layout in frequency space, no transposed-out option), bins in natural
 * order 0..n-1.  Complex values are interleaved {re, im}: float2 for
 * AFFT_F32, double2 for AFFT_F64.
 *   AFFT_C2C: in and out are n0*n1*n2 complex.
 *   AFFT_R2C: forward in = n0*n1*n2 real, out = n0*n1*(n2/2+1) complex (the
 *             halved axis is the contiguous one, transformed first as in
 *             Algorithm 1); backward (c2r) is the reverse.  n2 must be even.
 *             c2r reads only the real parts of bins k2 = 0 and k2 = n2/2.
 *
 * Ownership and execution.  The caller owns `in` and `out` (device pointers,
 * e.g. from torch tensors).  The plan owns its device twiddle tables and
 * workspace, allocated in afft_plan_create and freed in afft_plan_destroy;
 * execute allocates nothing.  `in` is never modified (c2r included).
 * Transforms are out-of-place: in == out returns AFFT_ERR_INPLACE, and the
 * two buffers must not overlap.  Execute enqueues kernels on the given
 * stream (a cudaStream_t, NULL = legacy default stream) and returns without
 * synchronising.  A plan may be used by one stream at a time; plans are
 * independent of each other.  A plan belongs to the device that was
 * current when it was created.
 *
 * Errors.  Every function returns an int status (AFFT_OK = 0).  Nothing
 * throws across this boundary and nothing aborts.  A CUDA launch error is
 * returned as AFFT_ERR_CUDA by the call that launched; an asynchronous fault
 * surfaces at the next CUDA call on that device.
 */
#ifndef AFFT_H
#define AFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct afft_plan afft_plan;

/* Transform kinds (AccFFT Section 1: R2C, C2C, C2R).  An R2C plan runs r2c
 * forward and c2r backward. */
enum { AFFT_C2C = 0, AFFT_R2C = 1 };

/* Precisions (AccFFT Section 1: single and double precision).
 * AFFT_F32_SPLIT: complex64/float32 data like AFFT_F32, with every radix-16
 * pass computed on the tensor cores as FP16 matrix products of hi + lo split
 * operands (a hi*hi + hi*lo + lo*hi, FP32 accumulation, each butterfly scaled
 * by a power of two into FP16 range); other radices run in FP32.  Relative L2
 * error <= 2e-5 against the exact transform.  The paper supports single and
 * double precision only and names mixed floating-point computation as missing
 * (the limitations at the end of Section 2); this mode is that extension. */
enum { AFFT_F32 = 0, AFFT_F64 = 1, AFFT_F32_SPLIT = 2 };

enum {
    AFFT_OK = 0,
    AFFT_ERR_NULL = 1,        /* a required pointer argument is NULL           */
    AFFT_ERR_SIZE = 2,        /* some n[i] < 1, or has a prime factor > 5      */
    AFFT_ERR_R2C_ODD = 3,     /* R2C plan with odd n[2]                        */
    AFFT_ERR_KIND = 4,        /* kind is not AFFT_C2C or AFFT_R2C              */
    AFFT_ERR_PRECISION = 5,   /* precision is not one of the enum values       */
    AFFT_ERR_NOMEM = 6,       /* device or host allocation failed in create    */
    AFFT_ERR_INPLACE = 7,     /* in == out                                     */
    AFFT_ERR_CUDA = 8,        /* a CUDA call or kernel launch failed           */
    AFFT_ERR_UNSUPPORTED = 9, /* valid request this version does not implement */
    AFFT_ERR_SCRATCH = 10,    /* afft_c2r_noalloc: the transform does not fit its fixed scratch */
    AFFT_ERR_TIMEOUT = 11,    /* a kernel gave up a bounded wait (see afft_plan_device_status) */
    AFFT_ERR_AXES = 12        /* axes mask empty or out of range, or r2c without axis 2  */
};

/*
 * Create a plan for an n[0] x n[1] x n[2] transform (AccFFT Section 1: the
 * library takes an N0 x N1 x N2 array).  Factors each axis into radix
 * 16/8/4/2/3/5 passes (the Cooley-Tukey reduction of Section 2), computes
 * the twiddle tables in FP64 on the current device, and allocates the
 * workspace.  Each n[i] must be >= 1 with prime factors in {2, 3, 5}.  A line
 * longer than 4096 points (the longest one CTA transforms) is split four-step,
 * n = n_a n_b with both factors at most 4096, through a plan-owned buffer of
 * the array's size; AFFT_ERR_UNSUPPORTED when no such split exists (n above
 * 4096^2), and for an r2c plan whose contiguous half length n[2]/2 exceeds 4096
 * (that axis is not split).
 *   out:       receives the plan (set to NULL on failure).
 *   n:         host array of 3 sizes, slowest first.
 *   kind:      AFFT_C2C or AFFT_R2C.
 *   precision: AFFT_F32, AFFT_F64 or AFFT_F32_SPLIT.
 * Synchronises the current device once (twiddle upload) before returning.
 */
int afft_plan_create(afft_plan **out, const int64_t n[3], int kind, int precision);

/*
 * A plan for `batch` independent transforms of the same size stored back to
 * back ([batch][n0][n1][n2], and [batch][n0][n1][n2/2+1] for r2c spectra).
 * The stages run over all of them at once (the batch simply adds lines to
 * every stage, as the paper's batched 1-D FFTs do within one rank).
 * afft_plan_create(out, n, kind, precision) is batch = 1.  batch < 1 returns
 * AFFT_ERR_SIZE; input/output byte counts below include the batch.
 */
int afft_plan_create_batched(afft_plan **out, const int64_t n[3], int64_t batch, int kind, int precision);

/*
 * A plan that transforms only some of the three axes: bit a of `axes` (1, 2, 4
 * for n[0], n[1], n[2]) selects axis a.  These are the building blocks of the
 * paper's distributed forms, where each process runs the 1-D FFT stages of the
 * axes it holds whole and exchanges data in between: the slab decomposition
 * (Algorithm 3) runs axes {1, 2} on its n0/P planes and, after the all-to-all,
 * axis {0} on its n1/P rows; the d-dimensional transform (Algorithm 2) runs a
 * batched 3-D plan on the trailing axes and a {0} plan on the leading one.
 * Layouts are those of afft_plan_create_batched; a transformed axis needs a
 * 2/3/5-smooth length, an untransformed one only n[a] >= 1.  An R2C plan must
 * include axis 2 (the halved axis, AFFT_ERR_AXES otherwise).  The forward
 * transform runs the selected stages in Algorithm 1's order (N2, N1, N0) and
 * the backward one in reverse, multiplied by 1 / (product of the transformed
 * n[a]) unless afft_plan_set_backward_scale says otherwise.  With axis 2
 * untransformed the factor costs a separate pass over the output when it is
 * not 1.  axes = 7 is afft_plan_create_batched.  The L2 slab schedule, the
 * blocked layout and the Poisson solve need axes = 7 (AFFT_ERR_AXES from
 * afft_execute_poisson otherwise).
 */
int afft_plan_create_axes(afft_plan **out, const int64_t n[3], int64_t batch, int kind, int precision, int axes);

/*
 * The factor the backward transform multiplies its result by (default 1 / N of
 * the transformed axes, the normalisation of Section 2, footnote 2).  A
 * distributed transform sets 1 / N_global on the plan that runs last and 1 on
 * the others, so that the whole backward transform carries 1/N exactly once.
 * AFFT_ERR_SIZE for 0 or NaN.  Not while the plan is in use on a stream.
 */
int afft_plan_set_backward_scale(afft_plan *p, double scale);
double afft_plan_backward_scale(const afft_plan *p);   /* 0 for NULL */

/*
 * rows x width bytes from src (row pitch spitch bytes) to dst (pitch dpitch),
 * asynchronous on the stream (cudaMemcpy2DAsync, any memory kind).  The pack
 * and unpack of the slab decomposition's all-to-all (Algorithm 3; the paper's
 * pack/unpack kernels of Section 2) are such copies: the n0/P x n1/P x n2h
 * block bound for each process is n0/P rows of n1/P * n2h elements, n1 * n2h
 * elements apart.  AFFT_ERR_SIZE if width exceeds a pitch; nothing to do for
 * zero rows or width.
 */
int afft_copy_2d(void *dst, size_t dpitch, const void *src, size_t spitch, size_t width, size_t rows,
                 void *cuda_stream);

/*
 * Forward transform (Algorithm 1, left column): 1-D FFTs along N2, then N1,
 * then N0, unscaled.  C2C: in, out complex [n0][n1][n2].  R2C: in real
 * [n0][n1][n2], out complex [n0][n1][n2/2+1].  Device pointers; stream is a
 * cudaStream_t (may be NULL).  Asynchronous.
 */
int afft_execute_forward(afft_plan *p, const void *in, void *out, void *cuda_stream);

/*
 * Backward transform (Algorithm 1, right column): inverse 1-D FFTs along
 * N0, then N1, then N2, and x 1/N folded into the last store (Section 2,
 * footnote 2).  C2C: complex -> complex.  R2C plan: complex [n0][n1][n2/2+1]
 * -> real [n0][n1][n2] (c2r; the half spectrum is treated as Hermitian
 * along k2).  `in` is not modified.  Asynchronous.
 */
int afft_execute_backward(afft_plan *p, const void *in, void *out, void *cuda_stream);

/*
 * Spectral Poisson solve (AccFFT Section 1 lists fast spectral operators as a
 * feature without describing them; this is the one the serving workload
 * uses): for an AFFT_R2C plan, u = -Laplacian^{-1} f on the periodic box
 * [0, 2 pi)^3 with grid x_j = 2 pi j / n, i.e. u_hat(k) = f_hat(k) / |k|^2 with
 * integer wavenumbers k_i = m (m <= n_i/2) or m - n_i, and u_hat(0) = 0 (the
 * zero-mean solution).  in = f, out = u, both real [batch][n0][n1][n2] device
 * arrays, out-of-place; the plan's workspace holds the spectrum.  The N0
 * stage runs forward DFT, division and inverse DFT in one kernel when the
 * plan's N0 stage is pipelined.  AFFT_ERR_KIND for C2C plans.  Asynchronous.
 */
int afft_execute_poisson(afft_plan *p, const void *in, void *out, void *cuda_stream);

/*
 * The same transforms with the data in host memory: copies host_in into the
 * caller's device buffer dev_in, runs the transform into dev_out, and copies
 * dev_out back to host_out, all enqueued on the stream (pinned host memory
 * makes the copies asynchronous; pageable memory makes them synchronous).
 * The caller owns all four buffers; sizes are those of the device variant.
 * dev_in and dev_out must not overlap.  Returns before the copy back completes
 * when host_out is pinned: synchronise the stream before reading it.
 */
int afft_execute_forward_host(afft_plan *p, const void *host_in, void *host_out,
                              void *dev_in, void *dev_out, void *cuda_stream);
int afft_execute_backward_host(afft_plan *p, const void *host_in, void *host_out,
                               void *dev_in, void *dev_out, void *cuda_stream);

/* Destroy a plan and free its device memory.  NULL is a no-op (AFFT_OK).
 * Synchronises the plan's device before freeing. */
int afft_plan_destroy(afft_plan *p);

/*
 * Failure detection.  Kernels that wait for asynchronous tile copies bound the
 * wait (about 2 s); a CTA that gives up records it in a flag the plan owns and
 * returns early, leaving that tile's output unwritten.  This call
 * synchronises with the device, returns AFFT_ERR_TIMEOUT if any execution since
 * the last call recorded such a timeout (and clears the flag), else AFFT_OK.
 */
int afft_plan_device_status(afft_plan *p);

/*
 * Failure-detection self-test: launches on `cuda_stream` one CTA whose bounded
 * wait cannot be satisfied (an mbarrier that nothing arrives at), for at most
 * limit_us microseconds (1 ... 2,000,000); it then records the timeout in the
 * plan's flag exactly as the pipelined kernels do and exits, so the next
 * afft_plan_device_status returns AFFT_ERR_TIMEOUT (once).  No memory is
 * touched besides the flag and no fault is raised: the device stays usable.
 * AFFT_ERR_SIZE for limit_us out of range.  Asynchronous.
 */
int afft_plan_wait_probe(afft_plan *p, int limit_us, void *cuda_stream);

/* Bytes of device workspace the plan holds (0 for a NULL plan). */
size_t afft_plan_workspace_bytes(const afft_plan *p);

/* Bytes of the input / output buffer of the forward transform (0 for NULL).
 * The backward transform swaps them. */
size_t afft_plan_input_bytes(const afft_plan *p);
size_t afft_plan_output_bytes(const afft_plan *p);

/*
 * Blocked layout of c2c plans.  A c2c plan whose N0 rows lie more than 4 MB apart
 * (1024^3 complex64) would make every tile of the N0 stage touch as many 2 MB pages
 * as it has rows.  Such a plan instead runs its stages through a workspace that
 * holds the array as [n1/32][batch*n0][32][n2]: the contiguous N2 stage writes
 * its lines there, the N0 stage runs on rows 32*n2 complex apart, and the N1
 * stage reads each column as n1/32 runs of 32 rows and writes `out` row-major
 * (the paper's stage order, Algorithm 1, with the N0 and N1 stages swapped: the
 * DFTs along different axes commute).  The backward transform runs the same
 * stages in the same order and applies the 1/N in its first stage.
 * afft_plan_create turns this on where it applies and the workspace fits;
 * afft_plan_set_blocked(p, 1) turns it on for any plan whose shapes allow it
 * (c2c, n0 >= 2, n1 a multiple of 32, no four-step axis, pipelined kernels for
 * the n0 and n1 line lengths, a contiguous-stage CTA size dividing 32;
 * AFFT_ERR_UNSUPPORTED otherwise, AFFT_ERR_NOMEM if the workspace cannot be
 * allocated) and allocates the workspace (batch*n0*n1*n2 complex, counted by
 * afft_plan_workspace_bytes); (p, 0) frees it and returns to row-major stages.
 * Results differ only by rounding.  Not while the plan is in use on a stream.
 */
int afft_plan_set_blocked(afft_plan *p, int on);

/*
 * L2-resident stage fusion.  The N2 and N1 stages can run slab by slab (a slab
 * is a range of N0 planes): the N2 stage of slab c, then the N1 stage of slab c
 * on a second stream the plan owns, while the N2 stage of slab c+1 runs, so the
 * N1 stage reads its slab from L2 instead of HBM (AccFFT's stage order, Algorithm
 * 1, is unchanged; only the schedule is).  `bytes` is the slab size to aim for;
 * 0 runs the stages unfused (the default).  Plans whose array is under three
 * slabs are not fused.  Creates the
 * second stream and its events (no device memory).  Execute still returns
 * asynchronously and joins the second stream back into the caller's stream.
 */
int afft_plan_set_l2_chunk(afft_plan *p, size_t bytes);

/* Slab size in use (0 when the stages run unfused). */
size_t afft_plan_l2_chunk(const afft_plan *p);

/*
 * Alternating stage order.  Each stage of Algorithm 1 walks its tiles (or line
 * blocks) in one order; a stage that starts where the previous stage finished
 * finds that part of the array still in L2 (129 MB on GB300) instead of HBM.
 * With this on (the default), the unfused stages that follow a stage walking the
 * same planes run last to first: the forward N1 stage after the N2 stage, and the
 * backward N2 stage after the N1 stage (also in afft_execute_poisson).  Only the
 * order of independent tiles changes, so
 * results are bit-for-bit the same either way.  (p, 0) walks every stage first to
 * last.  Allocates nothing.  Not while the plan is in use on a stream.
 */
int afft_plan_set_l2_order(afft_plan *p, int on);

/* 1 when the plan's stages alternate their tile order (see above), else 0. */
int afft_plan_l2_order(const afft_plan *p);

/*
 * Autotuner (the counterpart of the MEASURE planner flag AccFFT passes to FFTW
 * and cuFFT, Section 3 "Implementation Details").  Times forward + backward
 * round trips of this plan on temporary buffers (allocated and freed here,
 * filled by afft_fill_uniform) for: the points per CTA of the contiguous
 * stage (1024 .. 8192), pipelined or plain kernels for each strided stage,
 * early release of the load buffer for row-pair tiles (odd-width complex64
 * rows), and, for arrays beyond 192 MB, the L2 slab size (0, 32, 64 MB); keeps
 * the fastest choice of each, in that order.  Results do not depend on the choice
 * beyond rounding.  Synchronises the stream.  AFFT_ERR_NOMEM if the temporary
 * buffers do not fit.
 */
int afft_plan_tune(afft_plan *p, void *cuda_stream);

/*
 * The autotuner's choices, to store and apply again (the Python binding keeps
 * them in a cache file keyed by shape, kind, precision, batch and GPU):
 * cfg[0] points per CTA of the contiguous stage (0: the default), cfg[1] and
 * cfg[2] pipelined (1) or plain (0) kernels for the N0 and N1 stages, cfg[3]
 * the L2 slab size in bytes (0: unfused), cfg[4] and cfg[5] whether the N0 and
 * N1 stages' row-pair tiles (odd-width complex64 rows) release their load
 * buffer after the first pass.  set returns AFFT_ERR_UNSUPPORTED for a choice
 * this plan cannot use, AFFT_ERR_SIZE for a negative value; it allocates
 * nothing on the device.  Not while the plan is in use on a stream.
 */
int afft_plan_get_tuning(const afft_plan *p, int64_t cfg[6]);
int afft_plan_set_tuning(afft_plan *p, const int64_t cfg[6]);

/*
 * Writes a one-line JSON description of the plan's configuration (radix
 * sequences per axis, kernel families, four-step splits, pipelined stages,
 * lines per CTA, padded row pitch, L2 slab) into buf (NUL-terminated).
 * AFFT_ERR_SIZE if len is too small.
 */
int afft_plan_describe(const afft_plan *p, char *buf, size_t len);

/*
 * Multi-plan executor: several plans (for example one batched plan per
 * distinct size of a set of uneven transforms) run as one CUDA graph.  The
 * first execute with a given direction and set of buffers captures, on a
 * private stream, one branch per plan (forked from a common event, so the
 * groups overlap on the GPU) and instantiates the graph; later executes with
 * the same buffers replay it with one cudaGraphLaunch on `cuda_stream`.  Up to
 * 8 captured graphs are kept (least recently used evicted).  The plans stay
 * owned by the caller and must outlive the executor; while captured graphs
 * exist, plans must not be reconfigured (tune, L2 slab, timing).  in[i] and
 * out[i] are device buffers for plans[i] (forward: its spatial input and
 * spectral output; backward: the reverse).
 */
typedef struct afft_multi afft_multi;
int afft_multi_create(afft_multi **out, int nplans, afft_plan *const *plans);
int afft_multi_execute(afft_multi *m, int backward, const void *const *in, void *const *out, void *cuda_stream);
int afft_multi_destroy(afft_multi *m);

/*
 * Persistent executor: several FP32 r2c plans (typically one batched plan per
 * distinct size of a set of uneven fields) run as ONE kernel launch per
 * direction.  This is the GPU form of the paper's batch bookkeeping (Algorithm
 * 2 repeats the stages per array; Section 3's planner picks kernels per size):
 * creation lists every tile of every stage (r2c, N1, N0 forward; N0, N1, c2r
 * backward) of every field as a work item, ordered so that each item comes
 * after the items it depends on; during the launch each CTA walks its share of
 * the list and waits, on device counters, for the r2c tiles of a plane before
 * its N1 tiles and for all N1 tiles of a field before its N0 tiles (backward:
 * N0 before N1, a plane's N1 before its c2r).  A field's stages thus run close
 * together in time and its intermediate spectrum is often still in L2.
 * Supported: r2c, AFFT_F32, all three axes, no four-step axis, line lengths
 * n0, n1 in {48, 64, 96, 120, 128, 160, 256} and n2/2 in {24, 32, 48, 60, 64,
 * 80, 128}, at most 8 plans, all on the current device (AFFT_ERR_UNSUPPORTED
 * otherwise).  Creation allocates the item lists (about 24 bytes per tile) and
 * the counters and synchronises; the plans stay owned by the caller and must
 * outlive the executor.  Execution: in[i], out[i] as for afft_execute_forward /
 * _backward on plans[i] (forward: real in, spectrum out; backward: spectrum in,
 * not modified, real out, x 1/N), asynchronous on the stream, allocates
 * nothing; the plans' workspaces are used, so a plan must not run elsewhere
 * meanwhile, and two executions of one executor must not overlap.  Every wait
 * on a counter is bounded (about 2 s): a CTA that gives up records it and makes
 * the others stop early; afft_queue_status (synchronising) then returns
 * AFFT_ERR_TIMEOUT once, and that execution's outputs are incomplete.
 */
typedef struct afft_queue afft_queue;
int afft_queue_create(afft_queue **out, int nplans, afft_plan *const *plans);
int afft_queue_execute(afft_queue *q, int backward, const void *const *in, void *const *out, void *cuda_stream);
int afft_queue_status(afft_queue *q);
int afft_queue_items(const afft_queue *q, int backward);   /* work items of one direction (0 for NULL) */
int afft_queue_destroy(afft_queue *q);                    /* NULL is a no-op */

/* Number of kernel launches one execute_forward / execute_backward makes. */
int afft_plan_launches(const afft_plan *p, int backward);

/*
 * Per-stage timing (the tracing facility; not part of the transform).
 * afft_plan_timing_begin makes the next `capacity` executions of this plan
 * (forward or backward, device or host variant) record a CUDA event before
 * the first stage and after each stage, on the execution's stream.  Events
 * are host-side objects created here; execute still allocates no memory.
 * Returns AFFT_ERR_SIZE for capacity < 1, AFFT_ERR_CUDA if event creation
 * fails.  Calling it again discards earlier records.
 */
int afft_plan_timing_begin(afft_plan *p, int capacity);

/*
 * Waits for the recorded events, writes the elapsed milliseconds of each
 * stage to ms[3 * r + s] (record r in execution order; stage s in launch
 * order: forward N2, N1, N0 -- backward N0, N1, N2; a stage skipped for a
 * length-1 axis reads 0; when the N2 and N1 stages run fused through L2, the
 * first of the two slots holds their combined time and the second reads 0),
 * stores the number of records in *count (at most
 * the capacity), and stops recording.  ms must hold 3 * capacity floats.
 */
int afft_plan_timing_end(afft_plan *p, float *ms, int *count);

/* Static description of a status code. */
const char *afft_status_string(int status);

/*
 * Synthetic input generator (not part of the transform): fills `count`
 * interleaved complex values at dev_out with U[-1, 1) numbers from the
 * counter-based splitmix64 generator (Steele, Lea, Flood 2014):
 *   value(i, part) = (splitmix64(seed ^ (2 i + part)) >> 40) * 2^-24 * 2 - 1,
 * part 0 = re, 1 = im, complex index i = 0..count-1.  precision AFFT_F32
 * writes float2, AFFT_F64 writes double2 (same values, exact in both).
 * Asynchronous on the stream.
 */
int afft_fill_uniform(void *dev_out, int64_t count, uint64_t seed, int precision,
                      void *cuda_stream);

/*
 * Size of the fixed device array used by afft_c2r_noalloc: 64 MiB, held on
 * every GPU that loads this library until the process exits.  The first
 * 512 KiB hold twiddle tables, the rest the intermediate spectrum.
 */
#define AFFT_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)

/*
 * Backward transform of an r2c plan (c2r: complex [n0][n1][n2/2+1] -> real
 * [n0][n1][n2], x 1/N) that allocates nothing.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- a host
 * framework that owns all device memory through its own arena and refuses
 * (or cannot account for) foreign allocations, or a latency-bound loop that
 * must not stall on the allocator once running -- and therefore cannot create
 * a plan.  Its twiddle tables and intermediate live in one file-scope
 * __device__ array of AFFT_NOALLOC_SCRATCH_BYTES; the caller passes `in`
 * (device, not modified) and `out` (device), laid out as for
 * afft_execute_backward on an AFFT_R2C plan of the same n and precision, and
 * gets the same result.
 *   n:         host array of 3 sizes (n[2] even), as afft_plan_create.
 *   precision: AFFT_F32 or AFFT_F64.
 *   stream:    a cudaStream_t (NULL = legacy default stream); asynchronous.
 * Errors as afft_plan_create / afft_execute_backward, plus AFFT_ERR_SCRATCH when
 * n0*n1*(n2/2+1) complex values exceed the array's 63.5 MiB workspace part
 * (e.g. 256^3 float32 does not fit; 128^3 float64 does), and
 * AFFT_ERR_UNSUPPORTED when n[0], n[1] or n[2]/2 exceeds 4096 (such lines need
 * the four-step split's buffer, which this entry point does not have; e.g.
 * (1, 1, 16384) is refused although it fits the array) or for AFFT_F32_SPLIT.
 * The first call on each device looks up the array's device address (with
 * that device current) and caches it: make that first call before any
 * stream capture.  All calls share the array and leave their data in it:
 * calls whose work overlaps on the GPU (other streams or host threads) race
 * and corrupt each other's results; calls on one stream are safe.
 */
int afft_c2r_noalloc(const int64_t n[3], int precision, const void *in, void *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* AFFT_H */
