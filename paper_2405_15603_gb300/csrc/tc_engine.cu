// The kernels of the tcgen05 engine (tc_kernels.cuh), instantiated in a
// translation unit of their own that is compiled without floating-point
// contraction (build.py): the ordinary kernel and the grouped kernel inline
// the same engine body, and with every FMA written out as fmaf both copies
// round alike, so a member of a grouped launch computes exactly what its own
// launch computes.  The rest of the tensor-core path keeps contraction.
#include "tc_kernels.cuh"
#include "tc_engine.cuh"

namespace {

template <int MODE, bool SPLIT>
cudaError_t launch_solo(const tck::Args& a, dim3 grid, cudaStream_t s) {
    using C = tck::Cfg<MODE, SPLIT>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tck::tc_engine<MODE, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             C::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    tck::tc_engine<MODE, SPLIT><<<grid, tck::NUM_THREADS, C::SMEM, s>>>(a);
    return cudaGetLastError();
}

template <int MODE, bool SPLIT>
cudaError_t launch_solo_pair(const tck::Args& a, dim3 grid, cudaStream_t s) {
    using C = tck::Cfg<MODE, SPLIT, true>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tck::tc_engine_pair<MODE, SPLIT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    tck::tc_engine_pair<MODE, SPLIT><<<grid, tck::NUM_THREADS, C::SMEM, s>>>(a);
    return cudaGetLastError();
}

template <int MODE, bool SPLIT>
cudaError_t launch_group_pair(const GroupTab& t, unsigned blocks, size_t, cudaStream_t s) {
    using C = tck::Cfg<MODE, SPLIT, true>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tck::tc_engine_group_pair<MODE, SPLIT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    tck::tc_engine_group_pair<MODE, SPLIT><<<blocks, tck::NUM_THREADS, C::SMEM, s>>>(t);
    return cudaGetLastError();
}

template <int MODE, bool SPLIT>
cudaError_t launch_group(const GroupTab& t, unsigned blocks, size_t, cudaStream_t s) {
    using C = tck::Cfg<MODE, SPLIT>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tck::tc_engine_group<MODE, SPLIT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    tck::tc_engine_group<MODE, SPLIT><<<blocks, tck::NUM_THREADS, C::SMEM, s>>>(t);
    return cudaGetLastError();
}

// f(integral_constant<MODE>, integral_constant<SPLIT>) for the built modes.
template <class F>
auto with_mode(int mode, bool split, F&& f) {
    using tck::Mode;
    auto sp = [&](auto m) {
        return split ? f(m, std::integral_constant<bool, true>{}) : f(m, std::integral_constant<bool, false>{});
    };
    switch (mode) {
        case tck::FWD_VALUE: return sp(std::integral_constant<int, tck::FWD_VALUE>{});
        case tck::FWD_TANLAP: return sp(std::integral_constant<int, tck::FWD_TANLAP>{});
        case tck::BWD_LAP: return sp(std::integral_constant<int, tck::BWD_LAP>{});
        case tck::BWD_TAN: return sp(std::integral_constant<int, tck::BWD_TAN>{});
        case tck::BWD_VALUE: return sp(std::integral_constant<int, tck::BWD_VALUE>{});
        case tck::GRAM: return sp(std::integral_constant<int, tck::GRAM>{});
        default: return sp(std::integral_constant<int, tck::JDOT>{});
    }
}

// The same for the modes built on CTA pairs (the forward modes).
template <class F>
auto with_pair_mode(int mode, bool split, F&& f) {
    auto sp = [&](auto m) {
        return split ? f(m, std::integral_constant<bool, true>{}) : f(m, std::integral_constant<bool, false>{});
    };
    if (mode == tck::FWD_VALUE) return sp(std::integral_constant<int, tck::FWD_VALUE>{});
    return sp(std::integral_constant<int, tck::FWD_TANLAP>{});
}

}  // namespace

namespace tck {

bool engine_has_pair(int mode) { return mode == FWD_VALUE || mode == FWD_TANLAP; }

cudaError_t engine_launch(int mode, bool split, bool pair, const Args& a, dim3 grid, cudaStream_t s) {
    if (pair) {
        if (!engine_has_pair(mode) || grid.x % 2 != 0) return cudaErrorInvalidValue;
        return with_pair_mode(mode, split, [&](auto m, auto sp) {
            return launch_solo_pair<decltype(m)::value, decltype(sp)::value>(a, grid, s);
        });
    }
    return with_mode(mode, split, [&](auto m, auto sp) {
        return launch_solo<decltype(m)::value, decltype(sp)::value>(a, grid, s);
    });
}

const void* engine_group_key(int mode, bool split, bool pair) {
    if (pair)
        return with_pair_mode(mode, split, [&](auto m, auto sp) {
            return (const void*)&tc_engine_group_pair<decltype(m)::value, decltype(sp)::value>;
        });
    return with_mode(mode, split, [&](auto m, auto sp) {
        return (const void*)&tc_engine_group<decltype(m)::value, decltype(sp)::value>;
    });
}

GroupLaunchFn engine_group_launcher(int mode, bool split, bool pair) {
    if (pair)
        return with_pair_mode(mode, split, [&](auto m, auto sp) {
            return (GroupLaunchFn)&launch_group_pair<decltype(m)::value, decltype(sp)::value>;
        });
    return with_mode(mode, split, [&](auto m, auto sp) {
        return (GroupLaunchFn)&launch_group<decltype(m)::value, decltype(sp)::value>;
    });
}

}  // namespace tck
