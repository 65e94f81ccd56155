// Launchers of the tcgen05 engine's kernels (tc_engine.cu, compiled without
// floating-point contraction); mode is a tck::Mode.
#pragma once
#include "tc_kernels.cuh"

namespace tck {
// The ordinary kernel over `grid` with the arguments in kernel parameters.
cudaError_t engine_launch(int mode, bool split, const Args& a, dim3 grid, cudaStream_t s);
// The grouped kernel's identity (the key under which recorded launches merge)
// and its launcher over a member table of Args (group.cuh).
const void* engine_group_key(int mode, bool split);
GroupLaunchFn engine_group_launcher(int mode, bool split);
}  // namespace tck
