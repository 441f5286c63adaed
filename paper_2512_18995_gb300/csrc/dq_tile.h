// Fused k-qubit tiles staged in shared memory by TMA (internal interface).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <unordered_map>
#include <vector>

#include "dq_plan.h"

namespace dq {

// Autotuned configuration for one circuit structure.
struct TileTune {
    int k = 0;          // tile qubits (0 = default)
    int low = 0;        // always-resident low bits
};

// Host-side cache of fused-pass schedules and the driver entry point used to
// encode TMA descriptors.
struct TileCache {
    void *encode_fn = nullptr;
    std::unordered_map<uint64_t, void *> schedules;
    void release();
};

bool tile_supported(int n, int amp_bytes);
size_t tile_workspace_bytes(const Plan &p, int batch, int amp_bytes);
size_t tile_adjoint_part_bytes(const Plan &p, int batch);
size_t tile_expect_part_bytes(int n, int nterms, int batch);

template <typename R>
cudaError_t tile_apply(TileCache &tc, std::unordered_map<uint64_t, TileTune> &tuned, const Plan &p,
                       const void *coef, void *state, int batch, void *tws, int nsm, cudaStream_t s,
                       int64_t *launches);
template <typename R>
cudaError_t tile_expect(TileCache &tc, int n, const std::vector<DevTerm> &bits, const DevTerm *d_bits,
                        const int32_t *d_ptr, int nobs, const void *state, int batch, double *part,
                        double *out, void *tws, int nsm, cudaStream_t s, int64_t *launches);
template <typename R>
cudaError_t tile_adjoint(TileCache &tc, std::unordered_map<uint64_t, TileTune> &tuned, const Plan &p,
                         const void *coef, const std::vector<DevTerm> &bits, int nobs, const double *rw,
                         void *psi, void *lam, int batch, double *part, double *gp, double *gd, void *tws,
                         int nsm, cudaStream_t s, int64_t *launches);
template <typename R>
cudaError_t tile_autotune(TileCache &tc, std::unordered_map<uint64_t, TileTune> &tuned, const Plan &p,
                          const void *coef, void *state, int batch, void *tws, int nsm, cudaStream_t s,
                          int64_t *launches);

}  // namespace dq
