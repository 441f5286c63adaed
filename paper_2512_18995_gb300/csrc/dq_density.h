// Density-matrix expectations (internal; see k_density.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dq {

struct DevTerm;
template <typename R>
cudaError_t density_expect(const void *rho, int n, const DevTerm *d_terms, const int32_t *d_obs_ptr, int nobs,
                           int batch, double *out, cudaStream_t s, int64_t *launches);

}  // namespace dq
