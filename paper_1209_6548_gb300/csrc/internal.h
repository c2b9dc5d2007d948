// Launch helpers of liblesbgk's single-domain kernels that the batched solver
// reuses for its per-instance initialisation, moments and population export.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "setup.h"

namespace lesbgk_internal {

// An NVTX range around one library call (named after the entry point), so
// that a profiler's timeline (nsys, ncu --nvtx) shows which call issued which
// kernels; without a tool attached a push or pop is a no-op call.
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range &) = delete;
  Range &operator=(const Range &) = delete;
};

using lesbgk_setup::KArgs;

constexpr int kMomentPartials = 1024;  // FP64 partial sums per quantity (block count)

// The 2D sets and D3Q64 in FP32, FP16 or BF16 storage (storage: LESBGK_F32,
// _F16, _BF16; dim 2 or 3; f: populations of that type in the grouped layout;
// A: the solve's tables).

// f = rho S(T,u), then the wall rule (fields: device double[4][ny][nx] or NULL).
cudaError_t launch_init(const KArgs &A, int nr, int order, int storage, int dim, const double *fields, void *f,
                        int sm_count, cudaStream_t s);

// Nine moment fields (out may be NULL) and the four FP64 totals into sums
// (device double[4]); partial: device double[4 * kMomentPartials].
cudaError_t launch_moments(const KArgs &A, int nr, int order, int storage, int dim, const void *f, float *out,
                           double *partial, double *sums, cudaStream_t s);

// Grouped layout -> public [a][j][i] layout (FP32 deviations).
cudaError_t launch_ungroup(const KArgs &A, int nr, int order, int storage, int dim, const void *f, float *out,
                           long long cells, int sm_count, cudaStream_t s);

}  // namespace lesbgk_internal
