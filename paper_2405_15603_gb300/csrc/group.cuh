// Grouped launches: one launch of a kernel over the argument sets of many
// independent problems ("members"), each member with the grid of its own
// launch.  Used by the grouped batch step (batch.cu), which records every
// launch of every handle's step and merges launches of the same kernel.
//
// A groupable kernel is a struct K with
//     static constexpr int THREADS;                       // block size
//     __device__ __noinline__ static void run(uint3 vb, uint3 vg, P... args);
// where vb / vg stand for blockIdx / gridDim of the member's own launch (not
// inlined, so that the solo and the grouped kernel call one compiled body and
// round alike).
// KL<K>(h, s, grid, smem, args...) launches it as an ordinary kernel
// (k_solo: vb = blockIdx, vg = gridDim), or, while a recorder is active on
// this host thread, appends the launch (kernel, grid, shared memory and the
// arguments converted to P...) to the recorder's list instead.  A grouped
// launch (k_group) runs the blocks of all members as one flat grid: block b
// belongs to the member m with start[m] <= b < start[m + 1], whose arguments
// it reads from the member table in global memory.  The body is the same
// code in both kernels, so a member computes exactly what its own launch
// would.
#pragma once
#include <string.h>
#include <type_traits>
#include <utility>
#include <vector>

#include "kfac_internal.cuh"

// ---------------------------------------------------------------------------
// Argument packs: the arguments of one launch, in order, as one plain struct
// ---------------------------------------------------------------------------
template <class... T>
struct KPack;
template <>
struct KPack<> {};
template <class H, class... T>
struct KPack<H, T...> {
    H head;
    KPack<T...> tail;
};

template <size_t I, class H, class... T>
__host__ __device__ __forceinline__ const auto& kpack_get(const KPack<H, T...>& p) {
    if constexpr (I == 0)
        return p.head;
    else
        return kpack_get<I - 1>(p.tail);
}

__host__ __device__ inline KPack<> kpack_make() { return {}; }
template <class H, class... T>
__host__ __device__ KPack<H, T...> kpack_make(H h, T... t) {
    return {h, kpack_make(t...)};
}

// Member table of a grouped launch (device memory).
struct GroupTab {
    const unsigned char* packs;   // member m's arguments at packs + m * stride
    const unsigned* start;        // first flat block of member m (n entries, increasing)
    const uint3* grid;            // member m's grid
    int n;
    int stride;
};

template <class K, class... P, size_t... I>
__device__ __forceinline__ void kgroup_apply(uint3 vb, uint3 vg, const KPack<P...>& p, std::index_sequence<I...>) {
    K::run(vb, vg, kpack_get<I>(p)...);
}

template <class K, class... P>
__global__ void __launch_bounds__(K::THREADS) k_solo(const __grid_constant__ P... p) {
    K::run(blockIdx, make_uint3(gridDim.x, gridDim.y, gridDim.z), p...);
}

// The member of flat block b: the last m with start[m] <= b.
__device__ __forceinline__ int group_member(const GroupTab& t, unsigned b) {
    int lo = 0, hi = t.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (t.start[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Block index of flat block b within its member's grid g (x fastest, like a
// launch's own linear block order).
__device__ __forceinline__ uint3 group_block(unsigned local, uint3 g) {
    return make_uint3(local % g.x, (local / g.x) % g.y, local / (g.x * g.y));
}

template <class K, class... P>
__global__ void __launch_bounds__(K::THREADS) k_group(const __grid_constant__ GroupTab t) {
    const int m = group_member(t, blockIdx.x);
    const uint3 g = t.grid[m];
    const uint3 vb = group_block(blockIdx.x - t.start[m], g);
    const KPack<P...>& pk = *reinterpret_cast<const KPack<P...>*>(t.packs + (size_t)m * t.stride);
    kgroup_apply<K>(vb, g, pk, std::index_sequence_for<P...>{});
}

// ---------------------------------------------------------------------------
// Recording (host)
// ---------------------------------------------------------------------------
// Launches the grouped kernel of a record's type over a member table.
typedef cudaError_t (*GroupLaunchFn)(const GroupTab& t, unsigned blocks, size_t smem, cudaStream_t s);

struct LaunchRec {
    const void* key;                 // the grouped kernel (one per body and argument types)
    GroupLaunchFn launch;
    uint3 grid;
    size_t smem;
    int align;
    std::vector<unsigned char> args; // the KPack of the arguments
    int marker;                      // 1: the step's eigensolve (run once for all members)
};

struct GroupRecorder {
    std::vector<LaunchRec>* list;
};

// The recorder of this host thread (nullptr: launches run).
GroupRecorder*& group_recorder();
inline bool group_recording() { return group_recorder() != nullptr; }
// Appends the eigensolve marker of the step being recorded.
void group_record_marker();

template <class F>
struct KSig;

template <class... P>
struct KSig<void (*)(uint3, uint3, P...)> {
    template <class K>
    static cudaError_t launch_group(const GroupTab& t, unsigned blocks, size_t smem, cudaStream_t s) {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute((const void*)&k_group<K, std::decay_t<P>...>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k_group<K, std::decay_t<P>...><<<blocks, K::THREADS, smem, s>>>(t);
        return cudaGetLastError();
    }

    template <class K, class... A>
    static kfac_status_t go(kfac_pinn_handle* h, cudaStream_t s, dim3 grid, size_t smem, A&&... a) {
        if (grid.x == 0 || grid.y == 0 || grid.z == 0) return KFAC_OK;
        if (GroupRecorder* r = group_recorder()) {
            using Pk = KPack<std::decay_t<P>...>;
            Pk pk = kpack_make<std::decay_t<P>...>(std::decay_t<P>(std::forward<A>(a))...);
            LaunchRec rec;
            rec.key = (const void*)&k_group<K, std::decay_t<P>...>;
            rec.launch = &launch_group<K>;
            rec.grid = make_uint3(grid.x, grid.y, grid.z);
            rec.smem = smem;
            rec.align = (int)alignof(Pk);
            rec.args.resize(sizeof(Pk));
            memcpy(rec.args.data(), &pk, sizeof(Pk));
            rec.marker = 0;
            r->list->push_back(std::move(rec));
            return KFAC_OK;
        }
        if (smem > 48 * 1024)
            KFAC_CUDA_TRY(cudaFuncSetAttribute((const void*)&k_solo<K, std::decay_t<P>...>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_solo<K, std::decay_t<P>...><<<grid, K::THREADS, smem, s>>>(std::decay_t<P>(std::forward<A>(a))...);
        KFAC_LAUNCH_CHECK(h);
        return KFAC_OK;
    }
};

// Launch (or record) the groupable kernel K over `grid` with `smem` bytes of
// dynamic shared memory; the arguments are converted to K::run's parameter
// types.
template <class K, class... A>
kfac_status_t KL(kfac_pinn_handle* h, cudaStream_t s, dim3 grid, size_t smem, A&&... a) {
    return KSig<decltype(&K::run)>::template go<K>(h, s, grid, smem, std::forward<A>(a)...);
}

// Device-to-device copy of `bytes` (a multiple of 8) as a groupable kernel
// while recording, cudaMemcpyAsync otherwise.
kfac_status_t group_copy(kfac_pinn_handle* h, cudaStream_t s, void* dst, const void* src, size_t bytes);
