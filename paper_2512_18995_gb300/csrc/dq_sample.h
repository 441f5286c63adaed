// Shot sampling from |psi|^2 (internal; see k_sample.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace dq {

// Chunks of 2^c amplitudes, groups of 2^g chunks, ngroups groups per row.
struct SampleGeom {
    int n, batch, c, g;
    int64_t ngroups;
};

SampleGeom sample_geom(int n, int batch);
size_t sample_workspace_bytes(int n, int batch);
// out[row * shots + s] for every row and shot; uniforms may be NULL (then the
// splitmix64 stream of `seed` supplies them); ws holds
// sample_workspace_bytes(n, batch) bytes.
template <typename R>
cudaError_t sample_run(const void *state, int n, int batch, int64_t shots, const double *uniforms, uint64_t seed,
                       uint64_t wmask, int64_t *out, void *ws, int nsm, cudaStream_t s, int64_t *launches);

}  // namespace dq
