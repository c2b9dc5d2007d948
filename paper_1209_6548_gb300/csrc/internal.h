// Launch helpers of liblesbgk's single-domain kernels that the batched solver
// reuses for its per-instance initialisation, moments and population export.
#pragma once

#include <cuda_runtime.h>

#include "setup.h"

namespace lesbgk_internal {

using lesbgk_setup::KArgs;

constexpr int kMomentPartials = 1024;  // FP64 partial sums per quantity (block count)

// f = rho S(T,u), then the wall rule (fields: device double[4][ny][nx] or NULL).
cudaError_t launch_init(const KArgs &A, int nr, int order, const double *fields, float *f, int sm_count,
                        cudaStream_t s);

// Nine moment fields (out may be NULL) and the four FP64 totals into sums
// (device double[4]); partial: device double[4 * kMomentPartials].
cudaError_t launch_moments(const KArgs &A, int nr, const float *f, float *out, double *partial, double *sums,
                           cudaStream_t s);

// Grouped layout -> public [a][j][i] layout.
cudaError_t launch_ungroup(int nr, const float *f, float *out, long long cells, int sm_count, cudaStream_t s);

}  // namespace lesbgk_internal
