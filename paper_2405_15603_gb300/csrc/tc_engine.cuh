// Launchers of the tcgen05 engine's kernels (tc_engine.cu, compiled without
// floating-point contraction); mode is a tck::Mode.
#pragma once
#include "tc_kernels.cuh"

namespace tck {
// Whether the mode is built on CTA pairs as well (tc_engine_pair).
bool engine_has_pair(int mode);
// The ordinary kernel over `grid` with the arguments in kernel parameters;
// pair: the CTA-pair kernel (grid.x = 2 x feature tiles, grid.y = pairs of
// point blocks; the weight maps b0 / b1 with 64-row boxes).
cudaError_t engine_launch(int mode, bool split, bool pair, const Args& a, dim3 grid, cudaStream_t s);
// The grouped kernel's identity (the key under which recorded launches merge)
// and its launcher over a member table of Args (group.cuh).
const void* engine_group_key(int mode, bool split, bool pair = false);
GroupLaunchFn engine_group_launcher(int mode, bool split, bool pair = false);
}  // namespace tck
