// multi.cu -- several plans executed as one CUDA graph.
//
// Transforms of uneven sizes (for example many fields whose cubic sizes are
// drawn from a small set) are grouped into one batched plan per size; a
// multi-plan executor runs every group's stages as one CUDA graph: the first
// call with a given set of buffers captures, on a private stream, one branch
// per plan forked from a common event (so small groups overlap on the GPU),
// joins them, and instantiates the graph; later calls with the same buffers
// replay it with a single cudaGraphLaunch on the caller's stream.
#include <cstring>
#include <new>
#include <vector>

#include "../../include/afft.h"

struct afft_multi {
    std::vector<afft_plan *> plans;
    std::vector<cudaStream_t> branch;   // one capture branch per plan
    std::vector<cudaEvent_t> joined;    // branch end events
    cudaStream_t capture = nullptr;
    cudaEvent_t fork = nullptr;
    struct Graph {
        int backward;
        std::vector<const void *> in;
        std::vector<void *> out;
        cudaGraphExec_t exec;
        unsigned long long last_use;
    };
    std::vector<Graph> graphs;          // small cache keyed by direction and buffers
    unsigned long long tick = 0;
    int device = 0;
};

namespace {
constexpr size_t kMaxGraphs = 8;

void release(afft_multi *m)
{
    for (auto &g : m->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    m->graphs.clear();
    for (cudaStream_t s : m->branch) cudaStreamDestroy(s);
    for (cudaEvent_t e : m->joined) cudaEventDestroy(e);
    if (m->capture) cudaStreamDestroy(m->capture);
    if (m->fork) cudaEventDestroy(m->fork);
}

int capture_graph(afft_multi *m, int backward, const void *const *in, void *const *out, cudaGraphExec_t *exec)
{
    if (cudaStreamBeginCapture(m->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return AFFT_ERR_CUDA;
    int st = AFFT_OK;
    if (cudaEventRecord(m->fork, m->capture) != cudaSuccess) st = AFFT_ERR_CUDA;
    for (size_t i = 0; i < m->plans.size() && st == AFFT_OK; ++i) {
        if (cudaStreamWaitEvent(m->branch[i], m->fork, 0) != cudaSuccess) {
            st = AFFT_ERR_CUDA;
            break;
        }
        st = backward ? afft_execute_backward(m->plans[i], in[i], out[i], m->branch[i])
                      : afft_execute_forward(m->plans[i], in[i], out[i], m->branch[i]);
        if (st != AFFT_OK) break;
        if (cudaEventRecord(m->joined[i], m->branch[i]) != cudaSuccess ||
            cudaStreamWaitEvent(m->capture, m->joined[i], 0) != cudaSuccess)
            st = AFFT_ERR_CUDA;
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t end = cudaStreamEndCapture(m->capture, &graph);
    if (st == AFFT_OK && (end != cudaSuccess || !graph)) st = AFFT_ERR_CUDA;
    if (st == AFFT_OK && cudaGraphInstantiate(exec, graph, 0) != cudaSuccess) st = AFFT_ERR_CUDA;
    if (graph) cudaGraphDestroy(graph);
    if (st != AFFT_OK) cudaGetLastError();
    return st;
}
}  // namespace

extern "C" {

int afft_multi_create(afft_multi **out, int nplans, afft_plan *const *plans)
{
    if (!out) return AFFT_ERR_NULL;
    *out = nullptr;
    if (!plans || nplans < 1) return nplans < 1 ? AFFT_ERR_SIZE : AFFT_ERR_NULL;
    for (int i = 0; i < nplans; ++i)
        if (!plans[i]) return AFFT_ERR_NULL;
    afft_multi *m = new (std::nothrow) afft_multi();
    if (!m) return AFFT_ERR_NOMEM;
    cudaGetDevice(&m->device);
    m->plans.assign(plans, plans + nplans);
    int st = AFFT_OK;
    if (cudaStreamCreateWithFlags(&m->capture, cudaStreamNonBlocking) != cudaSuccess) st = AFFT_ERR_CUDA;
    if (st == AFFT_OK && cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming) != cudaSuccess) st = AFFT_ERR_CUDA;
    for (int i = 0; i < nplans && st == AFFT_OK; ++i) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            st = AFFT_ERR_CUDA;
            break;
        }
        m->branch.push_back(s);
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            st = AFFT_ERR_CUDA;
            break;
        }
        m->joined.push_back(e);
    }
    if (st != AFFT_OK) {
        release(m);
        delete m;
        return st;
    }
    *out = m;
    return AFFT_OK;
}

int afft_multi_execute(afft_multi *m, int backward, const void *const *in, void *const *out, void *stream)
{
    if (!m || !in || !out) return AFFT_ERR_NULL;
    const size_t n = m->plans.size();
    for (size_t i = 0; i < n; ++i)
        if (!in[i] || !out[i]) return AFFT_ERR_NULL;
    backward = backward ? 1 : 0;
    afft_multi::Graph *hit = nullptr;
    for (auto &g : m->graphs) {
        if (g.backward != backward) continue;
        bool same = true;
        for (size_t i = 0; i < n && same; ++i) same = g.in[i] == in[i] && g.out[i] == out[i];
        if (same) {
            hit = &g;
            break;
        }
    }
    if (!hit) {
        cudaGraphExec_t exec = nullptr;
        const int st = capture_graph(m, backward, in, out, &exec);
        if (st != AFFT_OK) return st;
        if (m->graphs.size() >= kMaxGraphs) {
            size_t oldest = 0;
            for (size_t i = 1; i < m->graphs.size(); ++i)
                if (m->graphs[i].last_use < m->graphs[oldest].last_use) oldest = i;
            cudaGraphExecDestroy(m->graphs[oldest].exec);
            m->graphs.erase(m->graphs.begin() + (long)oldest);
        }
        afft_multi::Graph g;
        g.backward = backward;
        g.in.assign(in, in + n);
        g.out.assign(out, out + n);
        g.exec = exec;
        g.last_use = 0;
        m->graphs.push_back(g);
        hit = &m->graphs.back();
    }
    hit->last_use = ++m->tick;
    return cudaGraphLaunch(hit->exec, (cudaStream_t)stream) == cudaSuccess ? AFFT_OK : AFFT_ERR_CUDA;
}

int afft_multi_destroy(afft_multi *m)
{
    if (!m) return AFFT_OK;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != m->device) cudaSetDevice(m->device);
    const int st = cudaDeviceSynchronize() == cudaSuccess ? AFFT_OK : AFFT_ERR_CUDA;
    release(m);
    if (cur >= 0 && cur != m->device) cudaSetDevice(cur);
    delete m;
    return st;
}

}  // extern "C"
