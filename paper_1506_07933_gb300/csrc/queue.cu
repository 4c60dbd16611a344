// queue.cu -- one persistent launch per direction for a set of uneven-size r2c transforms.
//
// The caller hands over batched FP32 r2c plans (one per size, as for afft_multi);
// creation lists every tile of every stage of every field as a work item (see
// fft_queue.cuh for the device side and the dependency rules) and uploads the
// lists; an execution zeroes the completion counters and launches k_queue once.
//
// Item order.  CTA k runs items k, k + G, k + 2G, ... (G = resident CTAs), so an
// item that waits for items within the last G positions would often find them
// still running.  The order is built greedily: a stage-2 or stage-3 item (N1,
// N0 / c2r) is emitted as soon as every item it depends on was emitted at least
// 2G positions earlier, the later stage first (finishing a field frees its share
// of L2); otherwise the next first-stage item is emitted, unless the data of
// fields begun but not finished already exceeds an L2 budget, in which case the
// earliest waiting item whose dependencies are all emitted goes first.  Items of
// one field that stay close in the list find their data still in L2.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/afft.h"
#include "fft_queue.cuh"

using namespace afft;

namespace {

// Families compiled into the executor: r2c/c2r half lengths and strided line lengths (the
// radix sequences of the specialised kernels with the same length).
using QHalf = QFams<LinePlan<24, 8, 3>, LinePlan<32, 8, 4>, LinePlan<48, 16, 3>, LinePlan<60, 4, 3, 5>,
                    LinePlan<64, 8, 8>, LinePlan<80, 16, 5>, LinePlan<128, 16, 8>>;
using QFull = QFams<LinePlan<48, 16, 3>, LinePlan<64, 8, 8>, LinePlan<96, 8, 4, 3>, LinePlan<120, 8, 3, 5>,
                    LinePlan<128, 16, 8>, LinePlan<160, 8, 4, 5>, LinePlan<256, 16, 16>>;
constexpr int kHalfN[] = {24, 32, 48, 60, 64, 80, 128};
constexpr int kFullN[] = {48, 64, 96, 120, 128, 160, 256};
const int kHalfR[][4] = {{8, 3}, {8, 4}, {16, 3}, {4, 3, 5}, {8, 8}, {16, 5}, {16, 8}};
const int kFullR[][4] = {{16, 3}, {8, 8}, {8, 4, 3}, {8, 3, 5}, {16, 8}, {8, 4, 5}, {16, 16}};

const void *queue_kernel() { return (const void *)k_queue<QHalf, QFull>; }

constexpr size_t kQSmem = 72 * 1024;   // the largest tile: 8192 complex64 points, or c2r staging

int family(const int *ns, const int (*rad)[4], int count, const PlanView &v, int axis)
{
    for (int f = 0; f < count; ++f) {
        if (ns[f] != v.line_n[axis]) continue;
        if (!v.specialised[axis]) return -1;
        for (int i = 0; i < v.npass[axis]; ++i)
            if (i >= 4 || rad[f][i] != v.radix[axis][i]) return -1;
        return f;
    }
    return -1;
}

// Butterflies a thread carries per radix-R pass (as the stage kernels assume).
int per_thread(int r) { return bmax_for_radix(r); }

// Largest even line count <= want whose passes fit kQThreads threads and kQPoints points.
int tile_lines(const PlanView &v, int want)
{
    int lines = std::max(1, std::min(want, kQPoints / v.line_n[2]));
    for (; lines > 1; --lines) {
        if ((lines & 1) && lines > 1) continue;
        bool ok = true;
        for (int i = 0; i < v.npass[2] && ok; ++i) {
            const int r = v.radix[2][i];
            const long long bf = (long long)lines * (v.line_n[2] / r);
            ok = (bf + per_thread(r) - 1) / per_thread(r) <= kQThreads;
        }
        if (ok) break;
    }
    return lines;
}

struct Group {
    PlanView v;
    afft_plan *plan;
    int fam_half, fam_y, fam_x;
    int zl;                 // lines per r2c/c2r tile
    int tz, ty, tx;         // tiles per plane (r2c/c2r), per plane (N1), per field (N0)
    unsigned pbase, fbase;  // first plane / field counter
    double field_bytes;     // the field's spectrum
};

struct Pending {
    std::vector<QItem> items;
    size_t next = 0;
    bool empty() const { return next >= items.size(); }
    const QItem &front() const { return items[next]; }
};

// Builds the ordered item list of one direction.
std::vector<QItem> order_items(std::vector<Group> &gs, bool backward, unsigned ncounters, int G,
                               double l2_budget)
{
    Pending st[3];   // stage 1, 2, 3 in execution order
    std::vector<unsigned> total(ncounters, 0);
    std::vector<int> field_of_counter(ncounters, -1);
    std::vector<double> field_bytes;
    int fidx = 0;
    for (size_t gi = 0; gi < gs.size(); ++gi) {
        Group &g = gs[gi];
        const unsigned n0 = (unsigned)g.v.n[0];
        for (unsigned f = 0; f < (unsigned)g.v.batch; ++f, ++fidx) {
            field_bytes.push_back(g.field_bytes);
            const unsigned fc = g.fbase + f;
            field_of_counter[fc] = fidx;
            auto item = [&](unsigned char op, int fam, unsigned a, unsigned b, unsigned wait, unsigned need,
                            unsigned signal) {
                QItem it;
                it.op = op;
                it.group = (unsigned char)gi;
                it.fam = (unsigned short)fam;
                it.a = a;
                it.b = b;
                it.wait = wait;
                it.need = need;
                it.signal = signal;
                return it;
            };
            if (!backward) {
                for (unsigned p = 0; p < n0; ++p) {
                    const unsigned pc = g.pbase + f * n0 + p;
                    field_of_counter[pc] = fidx;
                    for (int k = 0; k < g.tz; ++k)
                        st[0].items.push_back(item(QOP_R2C, g.fam_half, f * n0 + p, k, kQNone, 0, pc));
                    total[pc] += g.tz;
                    for (int k = 0; k < g.ty; ++k)
                        st[1].items.push_back(item(QOP_Y_FWD, g.fam_y, f * n0 + p, k, pc, g.tz, fc));
                    total[fc] += g.ty;
                }
                for (int k = 0; k < g.tx; ++k)
                    st[2].items.push_back(item(QOP_X_FWD, g.fam_x, f, k, fc, n0 * g.ty, kQNone));
            } else {
                for (int k = 0; k < g.tx; ++k) st[0].items.push_back(item(QOP_X_BWD, g.fam_x, f, k, kQNone, 0, fc));
                total[fc] += g.tx;
                for (unsigned p = 0; p < n0; ++p) {
                    const unsigned pc = g.pbase + f * n0 + p;
                    field_of_counter[pc] = fidx;
                    for (int k = 0; k < g.ty; ++k)
                        st[1].items.push_back(item(QOP_Y_BWD, g.fam_y, f * n0 + p, k, fc, g.tx, pc));
                    total[pc] += g.ty;
                    for (int k = 0; k < g.tz; ++k)
                        st[2].items.push_back(item(QOP_C2R, g.fam_half, f * n0 + p, k, pc, g.ty, kQNone));
                }
            }
        }
    }
    std::vector<unsigned> emitted(ncounters, 0);
    std::vector<long long> last_pos(ncounters, -1);
    std::vector<unsigned char> started(field_bytes.size(), 0);
    std::vector<size_t> third_left(field_bytes.size(), 0);
    for (const QItem &it : st[2].items) {
        const unsigned c = it.wait;
        ++third_left[field_of_counter[c]];
    }
    double live = 0;
    std::vector<QItem> out;
    out.reserve(st[0].items.size() + st[1].items.size() + st[2].items.size());
    auto ready = [&](const QItem &it) { return emitted[it.wait] == total[it.wait]; };
    auto emit = [&](Pending &s, int stage) {
        const QItem it = s.front();
        ++s.next;
        const long long pos = (long long)out.size();
        if (it.signal != kQNone) {
            ++emitted[it.signal];
            last_pos[it.signal] = pos;
        }
        const int fld = field_of_counter[it.signal != kQNone ? it.signal : it.wait];
        if (stage == 0 && !started[fld]) {
            started[fld] = 1;
            live += field_bytes[fld];
        }
        if (stage == 2 && --third_left[fld] == 0) live -= field_bytes[fld];
        out.push_back(it);
    };
    while (!(st[0].empty() && st[1].empty() && st[2].empty())) {
        const long long pos = (long long)out.size();
        bool done = false;
        for (int s = 2; s >= 1 && !done; --s)
            if (!st[s].empty() && ready(st[s].front()) && last_pos[st[s].front().wait] + G <= pos) {
                emit(st[s], s);
                done = true;
            }
        if (done) continue;
        if (!st[0].empty() && (live < l2_budget || (st[1].empty() && st[2].empty()))) {
            emit(st[0], 0);
            continue;
        }
        // over budget (or no first-stage item left): the next later-stage item whose dependencies
        // are all emitted, even if they were emitted recently
        for (int s = 2; s >= 1 && !done; --s)
            if (!st[s].empty() && ready(st[s].front())) {
                emit(st[s], s);
                done = true;
            }
        if (!done) emit(st[0], 0);   // later stages still wait for first-stage items
    }
    return out;
}

}  // namespace

struct afft_queue {
    std::vector<Group> groups;
    QItem *d_items[2] = {nullptr, nullptr};
    unsigned nitems[2] = {0, 0};
    unsigned *d_counters = nullptr;   // counters, then the error flag, then the abort flag
    unsigned ncounters = 0;
    int grid = 0;
    int device = 0;
};

extern "C" {

int afft_queue_create(afft_queue **out, int nplans, afft_plan *const *plans)
{
    if (!out) return AFFT_ERR_NULL;
    *out = nullptr;
    if (!plans || nplans < 1) return AFFT_ERR_NULL;
    if (nplans > kQMaxGroups) return AFFT_ERR_UNSUPPORTED;
    afft_queue *q = new (std::nothrow) afft_queue();
    if (!q) return AFFT_ERR_NOMEM;
    cudaGetDevice(&q->device);
    unsigned nc = 0;
    for (int i = 0; i < nplans; ++i) {
        Group g;
        std::memset(&g, 0, sizeof g);
        g.plan = plans[i];
        if (!plans[i] || !plan_view(plans[i], &g.v)) {
            delete q;
            return AFFT_ERR_NULL;
        }
        const PlanView &v = g.v;
        g.fam_half = family(kHalfN, kHalfR, 7, v, 2);
        g.fam_y = family(kFullN, kFullR, 7, v, 1);
        g.fam_x = family(kFullN, kFullR, 7, v, 0);
        if (v.kind != AFFT_R2C || v.precision != AFFT_F32 || v.axes != 7 || v.four_step || g.fam_half < 0 ||
            g.fam_y < 0 || g.fam_x < 0 || v.device != q->device) {
            delete q;
            return AFFT_ERR_UNSUPPORTED;
        }
        const long long n0 = v.n[0], n1 = v.n[1], nh = v.nh;
        g.zl = tile_lines(v, (int)n1);
        g.tz = (int)((n1 + g.zl - 1) / g.zl);
        g.ty = (int)((nh + q_lines_for((int)n1) - 1) / q_lines_for((int)n1));
        g.tx = (int)((n1 * nh + q_lines_for((int)n0) - 1) / q_lines_for((int)n0));
        g.pbase = nc;
        nc += (unsigned)(v.batch * n0);
        g.fbase = nc;
        nc += (unsigned)v.batch;
        g.field_bytes = (double)n0 * n1 * nh * 8.0;
        q->groups.push_back(g);
    }
    q->ncounters = nc;
    int per_sm = 0, sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, q->device);
    int st = AFFT_OK;
    if (cudaFuncSetAttribute(queue_kernel(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kQSmem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, queue_kernel(), kQThreads, kQSmem) != cudaSuccess ||
        per_sm < 1)
        st = AFFT_ERR_CUDA;
    q->grid = sms * per_sm;
    for (int dir = 0; dir < 2 && st == AFFT_OK; ++dir) {
        // a dependency emitted two rounds of the grid earlier has usually finished; fields begun
        // but not finished are kept to 96 MB (of the 126 MB L2).  Measured on the 200-field
        // workload, forward: one round and 48 MB 8.1 ms, two rounds and 96 MB 6.6 ms
        const std::vector<QItem> items = order_items(q->groups, dir == 1, nc, 2 * q->grid, 96.0 * (1 << 20));
        q->nitems[dir] = (unsigned)items.size();
        if (cudaMalloc(&q->d_items[dir], items.size() * sizeof(QItem)) != cudaSuccess) {
            q->d_items[dir] = nullptr;
            st = AFFT_ERR_NOMEM;
        } else if (cudaMemcpy(q->d_items[dir], items.data(), items.size() * sizeof(QItem), cudaMemcpyHostToDevice) !=
                   cudaSuccess) {
            st = AFFT_ERR_CUDA;
        }
    }
    if (st == AFFT_OK) {
        if (cudaMalloc(&q->d_counters, (nc + 2) * sizeof(unsigned)) != cudaSuccess) {
            q->d_counters = nullptr;
            st = AFFT_ERR_NOMEM;
        } else if (cudaMemset(q->d_counters, 0, (nc + 2) * sizeof(unsigned)) != cudaSuccess) {
            st = AFFT_ERR_CUDA;
        }
    }
    if (st != AFFT_OK) {
        cudaGetLastError();
        afft_queue_destroy(q);
        return st;
    }
    *out = q;
    return AFFT_OK;
}

int afft_queue_execute(afft_queue *q, int backward, const void *const *in, void *const *out, void *stream)
{
    if (!q || !in || !out) return AFFT_ERR_NULL;
    const int dir = backward ? 1 : 0;
    QParams prm;
    std::memset(&prm, 0, sizeof prm);
    for (size_t i = 0; i < q->groups.size(); ++i) {
        const Group &g = q->groups[i];
        if (!in[i] || !out[i]) return AFFT_ERR_NULL;
        if (in[i] == out[i]) return AFFT_ERR_INPLACE;
        QGroup &d = prm.g[i];
        d.in = in[i];
        d.out = out[i];
        d.work = (float2 *)g.v.work;
        const float2 *tw = (const float2 *)g.v.tw;
        for (int a = 0; a < 3; ++a) d.tw[a] = tw + g.v.tw_base[a];
        d.post = tw + g.v.post_off;
        d.n0 = (int)g.v.n[0];
        d.n1 = (int)g.v.n[1];
        d.M = g.v.line_n[2];
        d.nh = (int)g.v.nh;
        d.zlines = g.zl;
        d.scale = (float)(1.0 / ((double)g.v.n[0] * (double)g.v.n[1] * (double)g.v.n[2]));
    }
    cudaStream_t s = (cudaStream_t)stream;
    // counters restart from zero; the error flag is kept until afft_queue_status reads it
    if (cudaMemsetAsync(q->d_counters, 0, q->ncounters * sizeof(unsigned), s) != cudaSuccess ||
        cudaMemsetAsync(q->d_counters + q->ncounters + 1, 0, sizeof(unsigned), s) != cudaSuccess)
        return AFFT_ERR_CUDA;
    const QItem *items = q->d_items[dir];
    unsigned n = q->nitems[dir];
    unsigned *counters = q->d_counters, *err = q->d_counters + q->ncounters, *abort_flag = err + 1;
    void *args[] = {(void *)&prm, (void *)&items, (void *)&n, (void *)&counters, (void *)&err, (void *)&abort_flag};
    const unsigned grid = (unsigned)std::min<long long>(q->grid, n);
    if (grid == 0) return AFFT_OK;
    return cudaLaunchKernel(queue_kernel(), dim3(grid), dim3(kQThreads), args, kQSmem, s) == cudaSuccess
               ? AFFT_OK
               : AFFT_ERR_CUDA;
}

int afft_queue_status(afft_queue *q)
{
    if (!q) return AFFT_ERR_NULL;
    unsigned flag = 0;
    if (cudaMemcpy(&flag, q->d_counters + q->ncounters, sizeof flag, cudaMemcpyDeviceToHost) != cudaSuccess)
        return AFFT_ERR_CUDA;
    if (!flag) return AFFT_OK;
    cudaMemset(q->d_counters + q->ncounters, 0, sizeof(unsigned));
    return AFFT_ERR_TIMEOUT;
}

int afft_queue_items(const afft_queue *q, int backward)
{
    return q ? (int)q->nitems[backward ? 1 : 0] : 0;
}

int afft_queue_destroy(afft_queue *q)
{
    if (!q) return AFFT_OK;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != q->device) cudaSetDevice(q->device);
    int st = AFFT_OK;
    if (q->d_items[0] || q->d_items[1] || q->d_counters) {
        if (cudaDeviceSynchronize() != cudaSuccess) st = AFFT_ERR_CUDA;
        cudaFree(q->d_items[0]);
        cudaFree(q->d_items[1]);
        cudaFree(q->d_counters);
    }
    if (cur >= 0 && cur != q->device) cudaSetDevice(cur);
    delete q;
    return st;
}

}  // extern "C"
