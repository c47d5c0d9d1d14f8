// batch.cu -- many cells in one launch: the H^V, rho and force/stress calls of
// every cell of a batch are captured once into a CUDA graph and the graph is
// then launched as one unit on the caller's stream.  The cells are dealt to
// kBranches independent branches of the graph (capture forks onto internal
// streams), so the kernels of small cells overlap.  A later call with
// different buffers re-captures.
#include <algorithm>
#include <cstring>
#include <vector>

#include "gint_impl.cuh"

constexpr int kBranches = 4;

struct gint_batch {
    int n = 0;
    int device = 0;
    std::vector<gint_handle*> h;
    std::vector<const void*> key;  // buffers of the captured graph
    cudaStream_t cap = nullptr;    // capture origin, also branch 0
    cudaStream_t br[kBranches] = {};
    cudaEvent_t ev_join[kBranches] = {};
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace gint {
gint_status tc_prepare(gint_handle* h);  // allocations the tensor-core calls make on first use
}

using namespace gint;

static void batch_free_graph(gint_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->key.clear();
}

extern "C" {

gint_status gint_batch_create(int n, gint_handle* const* handles, gint_batch** out) {
    set_error("");
    if (!out || n < 1 || !handles) { set_error("gint_batch_create: need n >= 1 handles and an output"); return GINT_ERR_INVALID_ARG; }
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (!handles[i]) { set_error("gint_batch_create: handle %d is NULL", i); return GINT_ERR_INVALID_ARG; }
    const int dev = handles[0]->device;
    for (int i = 1; i < n; ++i)
        if (handles[i]->device != dev) { set_error("gint_batch_create: handles on different devices"); return GINT_ERR_INVALID_ARG; }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(dev);
    gint_batch* b = new gint_batch();
    b->n = n;
    b->device = dev;
    b->h.assign(handles, handles + n);
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    b->br[0] = b->cap;
    for (int k = 1; k < kBranches && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&b->br[k], cudaStreamNonBlocking);
    for (int k = 0; k < kBranches && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming);
    gint_status s = GINT_OK;
    if (e != cudaSuccess) { set_error("gint_batch_create: %s", cudaGetErrorString(e)); s = GINT_ERR_CUDA; }
    for (int i = 0; i < n && s == GINT_OK; ++i) s = tc_prepare(b->h[i]);
    if (prev >= 0) cudaSetDevice(prev);
    if (s != GINT_OK) {
        gint_batch_destroy(b);
        return s;
    }
    *out = b;
    return GINT_OK;
}

void gint_batch_destroy(gint_batch* b) {
    if (!b) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    batch_free_graph(b);
    for (int k = 1; k < kBranches; ++k)
        if (b->br[k]) cudaStreamDestroy(b->br[k]);
    for (int k = 0; k < kBranches; ++k)
        if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (prev >= 0) cudaSetDevice(prev);
    delete b;
}

gint_status gint_batch_run(gint_batch* b, const double* const* V, const double* const* D, double* const* H,
                           double* const* rho, double* const* F, double* const* sigma, double* const* E,
                           gint_stream stream) {
    set_error("");
    if (!b || !V || !D) { set_error("gint_batch_run: NULL argument"); return GINT_ERR_INVALID_ARG; }
    const int n = b->n;
    std::vector<const void*> key;
    key.reserve((size_t)7 * n);
    for (int i = 0; i < n; ++i) {
        if (!V[i] || !D[i]) { set_error("gint_batch_run: cell %d has no V or D", i); return GINT_ERR_INVALID_ARG; }
        key.push_back(V[i]);
        key.push_back(D[i]);
        key.push_back(H ? H[i] : nullptr);
        key.push_back(rho ? rho[i] : nullptr);
        key.push_back(F ? F[i] : nullptr);
        key.push_back(sigma ? sigma[i] : nullptr);
        key.push_back(E ? E[i] : nullptr);
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    gint_status s = GINT_OK;
    cudaError_t e = cudaSuccess;
    if (!b->exec || key != b->key) {
        batch_free_graph(b);
        // capture every cell's calls: fork onto the branches, deal the cells round robin, join
        e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) {
            set_error("cudaStreamBeginCapture: %s", cudaGetErrorString(e));
            if (prev >= 0) cudaSetDevice(prev);
            return GINT_ERR_CUDA;
        }
        const int nbr = std::min(kBranches, n);
        int forked = 1;
        e = cudaEventRecord(b->ev_fork, b->cap);
        for (int k = 1; k < nbr && e == cudaSuccess; ++k, ++forked) e = cudaStreamWaitEvent(b->br[k], b->ev_fork, 0);
        if (e != cudaSuccess) { set_error("gint_batch_run: fork: %s", cudaGetErrorString(e)); s = GINT_ERR_CUDA; }
        for (int i = 0; i < n && s == GINT_OK; ++i) {
            gint_stream cs = (gint_stream)b->br[i % nbr];
            if (H && H[i]) s = gint_vlocal(b->h[i], V[i], H[i], 0, cs);
            if (s == GINT_OK && rho && rho[i]) s = gint_rho(b->h[i], D[i], rho[i], cs);
            if (s == GINT_OK && ((F && F[i]) || (sigma && sigma[i]) || (E && E[i])))
                s = gint_force_stress(b->h[i], V[i], D[i], F ? F[i] : nullptr, sigma ? sigma[i] : nullptr, nullptr,
                                      E ? E[i] : nullptr, cs);
        }
        // join every forked branch (also after an error, so that the capture can end)
        for (int k = 1; k < forked; ++k) {
            cudaError_t ej = cudaEventRecord(b->ev_join[k], b->br[k]);
            if (ej == cudaSuccess) ej = cudaStreamWaitEvent(b->cap, b->ev_join[k], 0);
            if (ej != cudaSuccess && s == GINT_OK) { set_error("gint_batch_run: join: %s", cudaGetErrorString(ej)); s = GINT_ERR_CUDA; }
        }
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
        if (s == GINT_OK && e2 != cudaSuccess) { set_error("cudaStreamEndCapture: %s", cudaGetErrorString(e2)); s = GINT_ERR_CUDA; }
        if (s == GINT_OK) {
            e = cudaGraphInstantiate(&b->exec, g, 0);
            if (e != cudaSuccess) { set_error("cudaGraphInstantiate: %s", cudaGetErrorString(e)); s = GINT_ERR_CUDA; }
            b->graph = g;
            b->key = key;
        } else if (g) {
            cudaGraphDestroy(g);
        }
    }
    if (s == GINT_OK) {
        // order the graph after the caller's stream and the caller's stream after the graph
        cudaStream_t us = (cudaStream_t)stream;
        e = cudaEventRecord(b->ev_in, us);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->ev_in, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->cap);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_out, b->cap);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(us, b->ev_out, 0);
        if (e != cudaSuccess) { set_error("gint_batch_run: %s", cudaGetErrorString(e)); s = GINT_ERR_CUDA; }
    }
    if (prev >= 0) cudaSetDevice(prev);
    return s;
}

}  // extern "C"
