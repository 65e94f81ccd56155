// Batched stepping of many independent problems, captured into a CUDA graph
// and replayed, in one of two forms:
//   streams  every handle's own step queued on worker streams (fork / join);
//   grouped  every handle's step recorded launch by launch (group.cuh), the
//            launches of the same kernel merged across handles into one
//            grouped launch over a member table, and the eigensolves of all
//            handles run as one batched eigensolve: the launches of a batch
//            step do not grow with the number of problems.
#include <map>
#include <vector>

#include "kfac_internal.cuh"
#include "group.cuh"

// ---------------------------------------------------------------------------
// Recording (group.cuh)
// ---------------------------------------------------------------------------
GroupRecorder*& group_recorder() {
    static thread_local GroupRecorder* r = nullptr;
    return r;
}

void group_record_marker() {
    LaunchRec rec;
    rec.key = nullptr;
    rec.launch = nullptr;
    rec.grid = make_uint3(0, 0, 0);
    rec.smem = 0;
    rec.align = 1;
    rec.marker = 1;
    group_recorder()->list->push_back(std::move(rec));
}

namespace {
struct k_copy_words {
    static constexpr int THREADS = 256;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, unsigned long long* dst, const unsigned long long* src,
                               long long n) {
        for (long long i = (long long)vb.x * THREADS + threadIdx.x; i < n; i += (long long)vg.x * THREADS)
            dst[i] = src[i];
    }
};

}  // namespace

kfac_status_t group_copy(kfac_pinn_handle* h, cudaStream_t s, void* dst, const void* src, size_t bytes) {
    if (group_recording()) {
        const long long n = (long long)(bytes / 8);
        return KL<k_copy_words>(h, s, ceil_div_u(n, 256), 0, (unsigned long long*)dst,
                                (const unsigned long long*)src, n);
    }
    KFAC_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s));
    return KFAC_OK;
}

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
    // grouped form (kfac_pinn_batch_set_grouped)
    int grouped;
    void* eigb;                              // the batched eigensolve of every handle's factor pairs
    unsigned char* gtab;                     // device member tables of the captured grouped launches
    long long step_launches;                 // kernels of one replayed batch step (-1: no graph yet)
};

namespace {

void batch_free(kfac_pinn_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->gtab) cudaFree(b->gtab);
    eig_batch_free(b->eigb);
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

// One launch of a grouped batch step: a kernel over its members, or the
// batched eigensolve.
struct GroupedLaunch {
    const LaunchRec* first;                  // kernel, launcher and argument layout
    std::vector<const LaunchRec*> members;
    bool eig;
};

// Merge the handles' recorded launch lists into one sequence of grouped
// launches that keeps every list's order: repeatedly take the kernel that
// heads the most lists (ties: the one heading the earliest list) and launch
// it for every list it heads; the eigensolve markers are taken once every
// list has reached its own.
std::vector<GroupedLaunch> merge_lists(const std::vector<std::vector<LaunchRec>>& lists) {
    std::vector<GroupedLaunch> out;
    std::vector<size_t> pos(lists.size(), 0);
    for (;;) {
        std::map<const void*, int> count;
        const void* best = nullptr;
        int best_n = 0, active = 0, markers = 0;
        for (size_t i = 0; i < lists.size(); i++) {
            if (pos[i] >= lists[i].size()) continue;
            active++;
            const LaunchRec& r = lists[i][pos[i]];
            if (r.marker) {
                markers++;
                continue;
            }
            const int n = ++count[r.key];
            if (n > best_n) {
                best_n = n;
                best = r.key;
            }
        }
        if (active == 0) break;
        GroupedLaunch g;
        g.first = nullptr;
        g.eig = (markers == active);
        for (size_t i = 0; i < lists.size(); i++) {
            if (pos[i] >= lists[i].size()) continue;
            const LaunchRec& r = lists[i][pos[i]];
            if (g.eig ? r.marker != 0 : (!r.marker && r.key == best)) {
                if (!g.first) g.first = &r;
                g.members.push_back(&r);
                pos[i]++;
            }
        }
        out.push_back(std::move(g));
    }
    return out;
}

// Records every handle's step (on b->cap, outside capture), merges the
// launches, uploads the member tables and captures the grouped step into
// b->exec.
kfac_status_t capture_grouped(kfac_pinn_batch* b, double* const* theta, const double* const* X_int,
                              const int* N_int, const double* const* f, const double* const* X_bdy,
                              const int* N_bdy, const double* const* g, double* const* loss) {
    const int count = (int)b->handles.size();
    std::vector<std::vector<LaunchRec>> lists(count);
    kfac_status_t st = KFAC_OK;
    for (int i = 0; i < count && st == KFAC_OK; i++) {
        kfac_pinn_handle* h = b->handles[i];
        const long long before = h->launches;
        GroupRecorder rec{&lists[i]};
        group_recorder() = &rec;
        const int in_graph = h->in_graph;
        h->in_graph = 1;          // the handle's own graph mode does not apply inside the batch
        st = kfac_pinn_step(h, b->cap, theta[i], X_int[i], N_int[i], f[i], X_bdy[i], N_bdy[i], g[i],
                            loss ? loss[i] : nullptr);
        h->in_graph = in_graph;
        group_recorder() = nullptr;
        // every launch of a recorded step goes through the recorder
        if (st == KFAC_OK && h->launches != before) st = KFAC_BAD_ARG;
    }
    if (st) return st;
    const std::vector<GroupedLaunch> seq = merge_lists(lists);

    // member tables: per launch the argument packs, then the start blocks and grids
    struct Tab {
        size_t packs, start, grid;
        int stride;
        unsigned blocks;
    };
    std::vector<Tab> tabs(seq.size());
    size_t bytes = 0;
    auto take = [&](size_t n, size_t align) {
        bytes = (bytes + align - 1) / align * align;
        const size_t at = bytes;
        bytes += n;
        return at;
    };
    for (size_t k = 0; k < seq.size(); k++) {
        if (seq[k].eig) continue;
        const LaunchRec& r0 = *seq[k].first;
        const size_t al = (size_t)std::max(r0.align, 16);
        Tab& t = tabs[k];
        t.stride = (int)((r0.args.size() + al - 1) / al * al);
        t.packs = take((size_t)t.stride * seq[k].members.size(), std::max<size_t>(al, 256));
        t.start = take(sizeof(unsigned) * seq[k].members.size(), 16);
        t.grid = take(sizeof(uint3) * seq[k].members.size(), 16);
    }
    std::vector<unsigned char> host(std::max<size_t>(bytes, 1), 0);
    for (size_t k = 0; k < seq.size(); k++) {
        if (seq[k].eig) continue;
        Tab& t = tabs[k];
        unsigned long long blocks = 0;
        for (size_t m = 0; m < seq[k].members.size(); m++) {
            const LaunchRec& r = *seq[k].members[m];
            memcpy(host.data() + t.packs + (size_t)m * t.stride, r.args.data(), r.args.size());
            const unsigned st0 = (unsigned)blocks;
            memcpy(host.data() + t.start + m * sizeof(unsigned), &st0, sizeof(unsigned));
            memcpy(host.data() + t.grid + m * sizeof(uint3), &r.grid, sizeof(uint3));
            blocks += (unsigned long long)r.grid.x * r.grid.y * r.grid.z;
        }
        if (blocks >= (1ull << 31)) return KFAC_BAD_ARG;
        t.blocks = (unsigned)blocks;
    }
    if (b->gtab) {
        KFAC_CUDA_TRY(cudaStreamSynchronize(b->cap));    // a replay of the previous graph may still read it
        cudaFree(b->gtab);
        b->gtab = nullptr;
    }
    void* dev = nullptr;
    if ((st = kfac_device_alloc(&dev, host.size()))) return st;
    b->gtab = (unsigned char*)dev;
    KFAC_CUDA_TRY(cudaMemcpy(b->gtab, host.data(), host.size(), cudaMemcpyHostToDevice));
    if (!b->eigb) {
        std::vector<kfac_pinn_handle*> hs(b->handles.begin(), b->handles.end());
        if ((st = eig_batch_alloc(hs.data(), count, &b->eigb))) {
            eig_batch_free(b->eigb);
            b->eigb = nullptr;
            return st;
        }
    }

    kfac_pinn_handle* h0 = b->handles[0];
    long long launches = 0;
    KFAC_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    for (size_t k = 0; k < seq.size() && st == KFAC_OK; k++) {
        if (seq[k].eig) {
            const long long l0 = h0->launches;
            st = eig_batch_run(h0, b->eigb, b->cap);
            launches += h0->launches - l0;
            continue;
        }
        const Tab& t = tabs[k];
        GroupTab gt;
        gt.packs = b->gtab + t.packs;
        gt.start = (const unsigned*)(b->gtab + t.start);
        gt.grid = (const uint3*)(b->gtab + t.grid);
        gt.n = (int)seq[k].members.size();
        gt.stride = t.stride;
        size_t smem = 0;
        for (const LaunchRec* r : seq[k].members) smem = std::max(smem, r->smem);
        const cudaError_t e = seq[k].first->launch(gt, t.blocks, smem, b->cap);
        if (e != cudaSuccess) {
            kfac_record_cuda_error(e);
            st = KFAC_CUDA_ERROR;
        }
        launches++;
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(b->cap, &graph);
    if (st == KFAC_OK && ce != cudaSuccess) {
        kfac_record_cuda_error(ce);
        st = KFAC_CUDA_ERROR;
    }
    if (st == KFAC_OK) {
        const cudaError_t ie = cudaGraphInstantiate(&b->exec, graph, 0);
        if (ie != cudaSuccess) {
            kfac_record_cuda_error(ie);
            b->exec = nullptr;
            st = KFAC_CUDA_ERROR;
        }
    }
    if (graph) cudaGraphDestroy(graph);
    if (st == KFAC_OK) b->step_launches = launches;
    return st;
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
    b->grouped = 0;
    b->eigb = nullptr;
    b->gtab = nullptr;
    b->step_launches = -1;
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
        if (b->grouped) {
            // the host-side step counters advance while recording exactly as in an eager step
            kfac_status_t st = capture_grouped(b, theta, X_int, N_int, f, X_bdy, N_bdy, g, loss);
            if (st) return st;
            b->key_ptr = kp;
            b->key_n = kn;
            b->graph_launches.assign(count, 0);
            KFAC_CUDA_TRY(cudaGraphLaunch(b->exec, b->cap));
            KFAC_CUDA_TRY(cudaEventRecord(b->ev_out, b->cap));
            KFAC_CUDA_TRY(cudaStreamWaitEvent(s, b->ev_out, 0));
            return KFAC_OK;
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
        b->step_launches = 0;
        for (int i = 0; i < count; i++) {
            b->graph_launches.push_back(b->handles[i]->launches - before[i]);
            b->step_launches += b->graph_launches.back();
        }
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

kfac_status_t kfac_pinn_batch_set_grouped(kfac_batch_t b, int enable) {
    if (!b) return KFAC_BAD_ARG;
    if (enable) {
        for (kfac_handle_t h : b->handles)
            if (!is_mixed(h)) return KFAC_BAD_ARG;
    }
    enable = enable ? 1 : 0;
    if (enable != b->grouped && b->exec) {
        KFAC_CUDA_TRY(cudaStreamSynchronize(b->cap));
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
        b->step_launches = -1;
    }
    b->grouped = enable;
    return KFAC_OK;
}

kfac_status_t kfac_pinn_batch_launches(kfac_batch_t b, long long* per_step) {
    if (!b || !per_step) return KFAC_BAD_ARG;
    if (!b->exec || b->step_launches < 0) return KFAC_NOT_READY;
    *per_step = b->step_launches;
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
