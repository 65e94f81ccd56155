// Allocation-free forward Laplacian (FP64).
//
// Some callers cannot allocate device memory while they run: code executing
// inside a memory pool or a fixed device-memory budget that another runtime
// owns, or a process that must not grow its footprint after start-up.  For
// them kfac_pinn_forward_laplacian_noalloc computes the same u, grad u and
// Laplacian as kfac_pinn_forward_laplacian on an FP64 handle, without a
// handle and without any allocation: the per-layer Taylor matrices live in
// one fixed scratch array in device memory, compiled into this library.
//
// The scratch array is file-scope (`static __device__`), so every GPU that
// loads the library holds it for the life of the process, and every call
// shares it: calls that overlap on the GPU (different streams, or different
// host threads) race on it and must be serialised by the caller.  Each call
// writes every scratch element it reads before reading it, so nothing has to
// be cleared between calls.
#include <string.h>

#include <atomic>

#include "kfac_internal.cuh"

namespace {

// 32 MiB of FP64 scratch: room for the Z and T matrices of all layers,
// sum over layers of 2 * (d + 2) * N * h_l doubles.
constexpr size_t NOALLOC_SCRATCH_DOUBLES = (size_t)4 << 20;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

constexpr int MAX_DEVICES = 64;
std::atomic<double*> g_scratch_addr[MAX_DEVICES];   // static storage: all null

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, not a device address).
// Concurrent first calls may both look it up; they store the same address.
kfac_status_t scratch_address(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return KFAC_CUDA_ERROR;
    double* a = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!a) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return KFAC_CUDA_ERROR;
        a = (double*)p;
        g_scratch_addr[dev].store(a, std::memory_order_release);
    }
    *out = a;
    return KFAC_OK;
}

// Channel weights of the second-order column: 1 for a Laplacian coordinate,
// 0 for time under the heat operator.
__global__ void k_noalloc_weights(double* w, int d, int heat) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < d) w[i] = (heat && i == 0) ? 0.0 : 1.0;
}

}  // namespace

extern "C" {

kfac_status_t kfac_pinn_forward_laplacian_noalloc(const kfac_config_t* cfg, void* stream, const double* theta,
                                                  const double* X, int N, double* u, double* grad, double* lap) {
    if (!cfg || !theta || !X || !u || N < 1) return KFAC_BAD_ARG;
    // the network limits of kfac_pinn_create; the general operator (which
    // needs the coefficient matrix's eigenvectors set up on a handle) is not
    // available here
    if (!kfac_valid_network(cfg) || cfg->op == KFAC_OP_GENERAL) return KFAC_BAD_ARG;

    // A handle on the host stack describes the network for the FP64 kernels;
    // its buffers point into the static scratch array.
    kfac_pinn_handle h;
    memset(&h, 0, sizeof(h));
    h.cfg = *cfg;
    h.cfg.precision = KFAC_FP64;
    h.dims[0] = cfg->d;
    for (int l = 0; l < cfg->L; l++) h.dims[l + 1] = cfg->widths[l];
    h.woff[0] = 0;
    for (int l = 1; l <= cfg->L; l++) h.woff[l] = h.woff[l - 1] + (int64_t)h.dims[l] * (h.dims[l - 1] + 1);
    h.D = h.woff[cfg->L];
    h.S = cfg->d + 2;

    size_t need = (size_t)cfg->d;    // channel weights
    for (int l = 1; l <= cfg->L; l++) need += (size_t)(l < cfg->L ? 2 : 1) * h.S * (size_t)N * h.dims[l];
    if (need > NOALLOC_SCRATCH_DOUBLES) return KFAC_BAD_ARG;   // beyond the fixed scratch capacity

    double* base = nullptr;
    kfac_status_t st = scratch_address(&base);
    if (st != KFAC_OK) return st;
    PassBuffers pb;
    memset(&pb, 0, sizeof(pb));
    pb.N = N;
    pb.S = h.S;
    double* cur = base;
    h.chw64 = cur;
    cur += cfg->d;
    for (int l = 1; l <= cfg->L; l++) {
        const size_t e = (size_t)h.S * N * h.dims[l];
        pb.Z[l - 1] = cur;
        cur += e;
        if (l < cfg->L) {
            pb.T[l - 1] = cur;
            cur += e;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    k_noalloc_weights<<<(cfg->d + 255) / 256, 256, 0, s>>>(h.chw64, cfg->d, cfg->op == KFAC_OP_HEAT);
    if (cudaGetLastError() != cudaSuccess) return KFAC_CUDA_ERROR;
    if ((st = simt_forward(&h, s, theta, X, N, pb, h.S))) return st;
    return simt_extract_outputs(&h, s, pb, N, h.S, u, grad, lap);
}

}  // extern "C"
