// batch.cu -- many cells in one launch (the uneven multi-cell workload).
//
// Tensor-core forms: every cell's bricks form one (cell, brick) work queue, and
// each of H^V, rho and force is ONE persistent launch over that queue (the
// kernels' multi-cell mode: a CTA takes the next item, loads the cell's tables
// when the cell changes and reads its buffers from a device table of CellJob).
// The small per-cell kernels around them (D formatting, H normalisation and
// mirror, empty-brick rho, force finalisation) run on four graph branches.
// SIMT forms (FP64, FP32): the cells' calls are dealt to the four branches.
// Either way the whole sequence is captured once into a CUDA graph and
// launched as one unit on the caller's stream; new buffers re-capture.
#include <algorithm>
#include <cstring>
#include <vector>

#include "gint_impl.cuh"
#include "nvtx.cuh"

constexpr int kBranches = 4;

struct gint_batch {
    int n = 0;
    int device = 0;
    int form = -1;  // tensor-core form shared by every cell (queue path), -1: per-cell calls
    std::vector<gint_handle*> h;
    std::vector<int> gen;            // each handle's generation when the batch was made
    std::vector<int> item0;          // first queue item of each cell
    int n_items = 0;
    gint::CellJob* d_jobs = nullptr;  // device table of the cells' jobs
    int* d_item_cell = nullptr;       // queue item -> cell
    int* d_counter = nullptr;         // work counter of the persistent launches
    std::vector<const void*> key;     // buffers of the captured graph
    cudaStream_t cap = nullptr;       // capture origin, also branch 0
    cudaStream_t br[kBranches] = {};
    cudaEvent_t ev_fork[8] = {}, ev_join[8][kBranches] = {};
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace gint {
gint_status tc_prepare(gint_handle* h);
int tc_form_of(const gint_handle* h);
gint_status tc_vlocal_check(const gint_handle* h, int form);
gint_status tc_rhoforce_check(const gint_handle* h);
gint_status tc_format_d(gint_handle* h, int form, const double* D, cudaStream_t st);
CellJob tc_cell_job(gint_handle* h, const double* V, double* H, double* rho, double* facc, double* acc_e);
gint_status tc_vlocal_multi(int form, const MultiArgs& M, int* counter, int sm_count, cudaStream_t st);
gint_status tc_rhoforce_multi(int form, bool force, const MultiArgs& M, int* counter, int sm_count, cudaStream_t st);
gint_status launch_norm_h(gint_handle* h, double* H, cudaStream_t st);
gint_status launch_mirror(gint_handle* h, double* H, cudaStream_t st);
gint_status launch_rho_empty(gint_handle* h, double* rho, cudaStream_t st);
gint_status launch_force_finalize(gint_handle* h, double* F, double* sigma, double* virial, double* E,
                                  cudaStream_t st);
}  // namespace gint

using namespace gint;

static void batch_free_graph(gint_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->key.clear();
}

// Run fn(cell, stream) for every cell, dealt round robin to the branches; fork k
// uses its own events.  Returns the first error; always joins the branches.
template <typename Fn>
static gint_status for_cells(gint_batch* b, int k, Fn&& fn) {
    const int nbr = std::min(kBranches, b->n);
    gint_status s = GINT_OK;
    cudaError_t e = cudaEventRecord(b->ev_fork[k], b->cap);
    int forked = 1;
    for (int j = 1; j < nbr && e == cudaSuccess; ++j, ++forked) e = cudaStreamWaitEvent(b->br[j], b->ev_fork[k], 0);
    if (e != cudaSuccess) { set_error("gint_batch_run: fork: %s", cudaGetErrorString(e)); s = GINT_ERR_CUDA; }
    for (int i = 0; i < b->n && s == GINT_OK; ++i) s = fn(i, b->br[i % nbr]);
    for (int j = 1; j < forked; ++j) {
        cudaError_t ej = cudaEventRecord(b->ev_join[k][j], b->br[j]);
        if (ej == cudaSuccess) ej = cudaStreamWaitEvent(b->cap, b->ev_join[k][j], 0);
        if (ej != cudaSuccess && s == GINT_OK) { set_error("gint_batch_run: join: %s", cudaGetErrorString(ej)); s = GINT_ERR_CUDA; }
    }
    return s;
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
    for (int i = 0; i < n; ++i) b->gen.push_back(handles[i]->generation);
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    b->br[0] = b->cap;
    for (int k = 1; k < kBranches && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&b->br[k], cudaStreamNonBlocking);
    for (int f = 0; f < 8 && e == cudaSuccess; ++f) {
        e = cudaEventCreateWithFlags(&b->ev_fork[f], cudaEventDisableTiming);
        for (int k = 0; k < kBranches && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&b->ev_join[f][k], cudaEventDisableTiming);
    }
    gint_status s = GINT_OK;
    if (e != cudaSuccess) { set_error("gint_batch_create: %s", cudaGetErrorString(e)); s = GINT_ERR_CUDA; }
    for (int i = 0; i < n && s == GINT_OK; ++i) s = tc_prepare(b->h[i]);
    // one work queue over every cell's bricks when all cells share a tensor-core form that accepts them
    if (s == GINT_OK) {
        int form = tc_form_of(b->h[0]);
        for (int i = 1; i < n; ++i)
            if (tc_form_of(b->h[i]) != form) form = -1;
        for (int i = 0; i < n && form >= 0; ++i)
            if (tc_vlocal_check(b->h[i], form) != GINT_OK || tc_rhoforce_check(b->h[i]) != GINT_OK) form = -1;
        set_error("");
        b->form = form;
        if (form >= 0) {
            std::vector<int> item_cell;
            b->item0.resize(n);
            for (int i = 0; i < n; ++i) {
                b->item0[i] = (int)item_cell.size();
                item_cell.insert(item_cell.end(), (size_t)b->h[i]->n_work, i);
            }
            b->n_items = (int)item_cell.size();
            e = dev_malloc(&b->d_item_cell, sizeof(int) * std::max<size_t>(1, item_cell.size()));
            if (e == cudaSuccess && !item_cell.empty())
                e = cudaMemcpy(b->d_item_cell, item_cell.data(), sizeof(int) * item_cell.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = dev_malloc(&b->d_jobs, sizeof(CellJob) * n);
            if (e == cudaSuccess) e = dev_malloc(&b->d_counter, sizeof(int));
            if (e != cudaSuccess) { set_error("gint_batch_create: %s", cudaGetErrorString(e)); s = GINT_ERR_CUDA; }
        }
    }
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
    for (int f = 0; f < 8; ++f) {
        if (b->ev_fork[f]) cudaEventDestroy(b->ev_fork[f]);
        for (int k = 0; k < kBranches; ++k)
            if (b->ev_join[f][k]) cudaEventDestroy(b->ev_join[f][k]);
    }
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->d_jobs) cudaFree(b->d_jobs);
    if (b->d_item_cell) cudaFree(b->d_item_cell);
    if (b->d_counter) cudaFree(b->d_counter);
    if (prev >= 0) cudaSetDevice(prev);
    delete b;
}

gint_status gint_batch_run(gint_batch* b, const double* const* V, const double* const* D, double* const* H,
                           double* const* rho, double* const* F, double* const* sigma, double* const* E,
                           gint_stream stream) {
    gint::NvtxRange nvtx_range_("gint_batch_run");
    set_error("");
    if (!b || !V || !D) { set_error("gint_batch_run: NULL argument"); return GINT_ERR_INVALID_ARG; }
    const int n = b->n;
    for (int i = 0; i < n; ++i)
        if (b->h[i]->generation != b->gen[i]) {
            set_error("gint_batch_run: cell %d's handle changed (gint_update_positions or gint_select_bricks) after "
                      "gint_batch_create; create the batch again", i);
            return GINT_ERR_INVALID_ARG;
        }
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
    auto want_h = [&](int i) { return H && H[i]; };
    auto want_rho = [&](int i) { return rho && rho[i]; };
    auto want_f = [&](int i) { return (F && F[i]) || (sigma && sigma[i]) || (E && E[i]); };
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    gint_status s = GINT_OK;
    cudaError_t e = cudaSuccess;
    if (!b->exec || key != b->key) {
        batch_free_graph(b);
        bool any_h = false, any_rho = false, any_f = false, all_h = true, all_rho = true, all_f = true;
        for (int i = 0; i < n; ++i) {
            any_h |= want_h(i); any_rho |= want_rho(i); any_f |= want_f(i);
            all_h &= want_h(i); all_rho &= want_rho(i); all_f &= want_f(i);
        }
        // the queue runs every cell's bricks: it needs every cell to ask for the same outputs
        const bool queue = b->form >= 0 && any_h == all_h && any_rho == all_rho && any_f == all_f;
        MultiArgs M{b->d_jobs, b->d_item_cell, b->n_items};
        if (queue) {
            // the cells' job table (uploaded before the capture; the graph reads it on every launch)
            std::vector<CellJob> jobs(n);
            for (int i = 0; i < n; ++i) {
                jobs[i] = tc_cell_job(b->h[i], V[i], want_h(i) ? H[i] : nullptr, want_rho(i) ? rho[i] : nullptr,
                                      b->h[i]->d_facc, b->h[i]->d_red);
                jobs[i].item0 = b->item0[i];
            }
            e = cudaMemcpy(b->d_jobs, jobs.data(), sizeof(CellJob) * n, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                set_error("gint_batch_run: %s", cudaGetErrorString(e));
                if (prev >= 0) cudaSetDevice(prev);
                return GINT_ERR_CUDA;
            }
        }
        e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) {
            set_error("cudaStreamBeginCapture: %s", cudaGetErrorString(e));
            if (prev >= 0) cudaSetDevice(prev);
            return GINT_ERR_CUDA;
        }
        if (queue) {
            const int form = b->form;
            const int sms = b->h[0]->sm_count;
            // per cell: zero H, format D (once for rho and force), clear the force accumulators
            s = for_cells(b, 0, [&](int i, cudaStream_t cs) -> gint_status {
                gint_handle* h = b->h[i];
                if (want_h(i) && h->n_values > 0) GINT_CUDA_TRY(cudaMemsetAsync(H[i], 0, sizeof(double) * h->n_values, cs));
                if (want_rho(i) || want_f(i)) {
                    gint_status r = tc_format_d(h, form, D[i], cs);
                    if (r != GINT_OK) return r;
                }
                if (want_f(i)) {
                    GINT_CUDA_TRY(cudaMemsetAsync(h->d_facc, 0, sizeof(double) * 12 * h->n_atoms, cs));
                    GINT_CUDA_TRY(cudaMemsetAsync(h->d_red, 0, sizeof(double), cs));
                }
                return GINT_OK;
            });
            if (s == GINT_OK && any_h) s = tc_vlocal_multi(form, M, b->d_counter, sms, b->cap);
            if (s == GINT_OK && any_h)
                s = for_cells(b, 1, [&](int i, cudaStream_t cs) -> gint_status {
                    if (!want_h(i)) return GINT_OK;
                    gint_status r = form == 2 ? launch_norm_h(b->h[i], H[i], cs) : GINT_OK;
                    return r == GINT_OK ? launch_mirror(b->h[i], H[i], cs) : r;
                });
            if (s == GINT_OK && any_rho) s = tc_rhoforce_multi(form, false, M, b->d_counter, sms, b->cap);
            if (s == GINT_OK && any_rho)
                s = for_cells(b, 2, [&](int i, cudaStream_t cs) -> gint_status {
                    return want_rho(i) ? launch_rho_empty(b->h[i], rho[i], cs) : GINT_OK;
                });
            if (s == GINT_OK && any_f) s = tc_rhoforce_multi(form, true, M, b->d_counter, sms, b->cap);
            if (s == GINT_OK && any_f)
                s = for_cells(b, 3, [&](int i, cudaStream_t cs) -> gint_status {
                    if (!want_f(i)) return GINT_OK;
                    return launch_force_finalize(b->h[i], F ? F[i] : nullptr, sigma ? sigma[i] : nullptr, nullptr,
                                                 E ? E[i] : nullptr, cs);
                });
        } else {
            s = for_cells(b, 0, [&](int i, cudaStream_t cs) -> gint_status {
                gint_stream gs = (gint_stream)cs;
                gint_status r = GINT_OK;
                if (want_h(i)) r = gint_vlocal(b->h[i], V[i], H[i], 0, gs);
                if (r == GINT_OK && want_rho(i)) r = gint_rho(b->h[i], D[i], rho[i], gs);
                if (r == GINT_OK && want_f(i))
                    r = gint_force_stress(b->h[i], V[i], D[i], F ? F[i] : nullptr, sigma ? sigma[i] : nullptr, nullptr,
                                          E ? E[i] : nullptr, gs);
                return r;
            });
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
