// Batched stepping of many independent problems: fork/join over worker
// streams, captured into a CUDA graph and replayed.
#include <vector>

#include "kfac_internal.cuh"

struct kfac_pinn_batch {
    std::vector<kfac_handle_t> handles;
    std::vector<cudaStream_t> streams;
    cudaEvent_t fork;
    std::vector<cudaEvent_t> join;
    int device;
    int calls;
    cudaGraphExec_t exec;
    std::vector<const void*> key_ptr;     // pointers and counts the graph was captured with
    std::vector<int> key_n;
    std::vector<long long> graph_launches;   // kernels each handle has in the graph
    cudaStream_t cap;                        // capture / replay stream (the caller's may be the legacy one)
    cudaEvent_t ev_in, ev_out;
};

namespace {

void batch_free(kfac_pinn_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

// Queue every handle's step on the worker streams between a fork and a join
// on `s` (recorded into a graph when `s` is capturing).
kfac_status_t enqueue(kfac_pinn_batch* b, cudaStream_t s, double* const* theta, const double* const* X_int,
                      const int* N_int, const double* const* f, const double* const* X_bdy, const int* N_bdy,
                      const double* const* g, double* const* loss) {
    KFAC_CUDA_TRY(cudaEventRecord(b->fork, s));
    for (cudaStream_t w : b->streams) KFAC_CUDA_TRY(cudaStreamWaitEvent(w, b->fork, 0));
    const int ns = (int)b->streams.size();
    for (size_t i = 0; i < b->handles.size(); i++) {
        kfac_status_t st = kfac_pinn_step(b->handles[i], b->streams[i % ns], theta[i], X_int[i], N_int[i], f[i],
                                          X_bdy[i], N_bdy[i], g[i], loss ? loss[i] : nullptr);
        if (st) return st;
    }
    for (int w = 0; w < ns; w++) {
        KFAC_CUDA_TRY(cudaEventRecord(b->join[w], b->streams[w]));
        KFAC_CUDA_TRY(cudaStreamWaitEvent(s, b->join[w], 0));
    }
    return KFAC_OK;
}

}  // namespace

extern "C" {

kfac_status_t kfac_pinn_batch_create(const kfac_handle_t* handles, int count, int n_streams, kfac_batch_t* out) {
    if (!out) return KFAC_BAD_ARG;
    *out = nullptr;
    if (!handles || count < 1 || n_streams < 1 || n_streams > 64) return KFAC_BAD_ARG;
    int dev = 0;
    KFAC_CUDA_TRY(cudaGetDevice(&dev));
    for (int i = 0; i < count; i++)
        if (!handles[i] || handles[i]->device != dev) return KFAC_BAD_ARG;
    kfac_pinn_batch* b = new kfac_pinn_batch();
    b->handles.assign(handles, handles + count);
    b->device = dev;
    b->calls = 0;
    b->exec = nullptr;
    b->fork = nullptr;
    b->cap = nullptr;
    b->ev_in = b->ev_out = nullptr;
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
        batch_free(b);
        return KFAC_CUDA_ERROR;
    }
    for (int w = 0; w < n_streams; w++) {
        cudaStream_t st;
        cudaEvent_t ev;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { batch_free(b); return KFAC_CUDA_ERROR; }
        b->streams.push_back(st);
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) { batch_free(b); return KFAC_CUDA_ERROR; }
        b->join.push_back(ev);
    }
    *out = b;
    return KFAC_OK;
}

kfac_status_t kfac_pinn_batch_destroy(kfac_batch_t b) {
    if (!b) return KFAC_BAD_ARG;
    for (cudaStream_t s : b->streams) cudaStreamSynchronize(s);
    if (b->cap) cudaStreamSynchronize(b->cap);
    batch_free(b);
    return KFAC_OK;
}

kfac_status_t kfac_pinn_batch_step(kfac_batch_t b, void* stream, double* const* theta, const double* const* X_int,
                                   const int* N_int, const double* const* f, const double* const* X_bdy,
                                   const int* N_bdy, const double* const* g, double* const* loss, int use_graph) {
    if (!b || !theta || !X_int || !N_int || !f || !X_bdy || !N_bdy || !g) return KFAC_BAD_ARG;
    const int count = (int)b->handles.size();
    for (int i = 0; i < count; i++) {
        kfac_handle_t h = b->handles[i];
        if (!theta[i] || !X_int[i] || !f[i] || !X_bdy[i] || !g[i]) return KFAC_BAD_ARG;
        if (N_int[i] < 1 || N_int[i] > h->cfg.max_n_int || N_bdy[i] < 1 || N_bdy[i] > h->cfg.max_n_bdy)
            return KFAC_BAD_ARG;
        if (h->timing) use_graph = 0;
    }
    cudaStream_t s = (cudaStream_t)stream;
    b->calls++;
    if (!use_graph || b->calls == 1) return enqueue(b, s, theta, X_int, N_int, f, X_bdy, N_bdy, g, loss);

    std::vector<const void*> kp;
    std::vector<int> kn;
    for (int i = 0; i < count; i++) {
        kp.insert(kp.end(), {theta[i], X_int[i], f[i], X_bdy[i], g[i], loss ? loss[i] : nullptr});
        kn.push_back(N_int[i]);
        kn.push_back(N_bdy[i]);
    }
    // Graphs are captured and replayed on the batch's own stream, ordered after
    // the work already queued on the caller's stream and before what follows it.
    KFAC_CUDA_TRY(cudaEventRecord(b->ev_in, s));
    KFAC_CUDA_TRY(cudaStreamWaitEvent(b->cap, b->ev_in, 0));
    if (!b->exec || kp != b->key_ptr || kn != b->key_n) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        std::vector<long long> before;
        for (kfac_handle_t h : b->handles) before.push_back(h->launches);
        // the host-side step counters advance during capture exactly as in an eager step
        KFAC_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        kfac_status_t st = enqueue(b, b->cap, theta, X_int, N_int, f, X_bdy, N_bdy, g, loss);
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamEndCapture(b->cap, &graph);
        if (st) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (ce != cudaSuccess) {
            kfac_record_cuda_error(ce);
            return KFAC_CUDA_ERROR;
        }
        ce = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            kfac_record_cuda_error(ce);
            b->exec = nullptr;
            return KFAC_CUDA_ERROR;
        }
        b->key_ptr = kp;
        b->key_n = kn;
        b->graph_launches.clear();
        for (int i = 0; i < count; i++) b->graph_launches.push_back(b->handles[i]->launches - before[i]);
    } else {
        // a replay runs no host code: advance the handles' counters here
        for (int i = 0; i < count; i++) {
            b->handles[i]->t++;
            b->handles[i]->launches += b->graph_launches[i];
        }
    }
    KFAC_CUDA_TRY(cudaGraphLaunch(b->exec, b->cap));
    KFAC_CUDA_TRY(cudaEventRecord(b->ev_out, b->cap));
    KFAC_CUDA_TRY(cudaStreamWaitEvent(s, b->ev_out, 0));
    return KFAC_OK;
}

}  // extern "C"

// Graph mode of a single handle: the handle owns a batch of itself, created at
// the first graph step.  The nested kfac_pinn_step calls of the batch run
// eagerly (in_graph), so the step is captured once and then replayed.
kfac_status_t handle_graph_step(kfac_pinn_handle* h, cudaStream_t s, double* theta, const double* X_int, int N_int,
                                const double* f, const double* X_bdy, int N_bdy, const double* g, double* loss) {
    if (!h->gbatch) {
        kfac_batch_t b = nullptr;
        kfac_handle_t hh = h;
        kfac_status_t st = kfac_pinn_batch_create(&hh, 1, 1, &b);
        if (st) return st;
        h->gbatch = b;
    }
    h->in_graph = 1;
    kfac_status_t st = kfac_pinn_batch_step(h->gbatch, s, &theta, &X_int, &N_int, &f, &X_bdy, &N_bdy, &g,
                                            &loss, 1);
    h->in_graph = 0;
    return st;
}

void handle_graph_free(kfac_pinn_handle* h) {
    if (h->gbatch) kfac_pinn_batch_destroy(h->gbatch);
    h->gbatch = nullptr;
}
