// Fused k-qubit tiles staged in shared memory by TMA.
#include "dq_tile.h"

namespace dq {

void TileCache::release() { schedules.clear(); }

bool tile_supported(int, int) { return false; }
size_t tile_workspace_bytes(const Plan &, int, int) { return 0; }
size_t tile_adjoint_part_bytes(const Plan &, int) { return 0; }
size_t tile_expect_part_bytes(int, int, int) { return 0; }

template <typename R>
cudaError_t tile_apply(TileCache &, std::unordered_map<uint64_t, TileTune> &, const Plan &, const void *, void *,
                       int, void *, int, cudaStream_t, int64_t *) {
    return cudaErrorNotSupported;
}
template <typename R>
cudaError_t tile_expect(TileCache &, int, const std::vector<DevTerm> &, const DevTerm *, const int32_t *, int,
                        const void *, int, double *, double *, void *, int, cudaStream_t, int64_t *) {
    return cudaErrorNotSupported;
}
template <typename R>
cudaError_t tile_adjoint(TileCache &, std::unordered_map<uint64_t, TileTune> &, const Plan &, const void *,
                         const std::vector<DevTerm> &, int, const double *, void *, void *, int, double *,
                         double *, double *, void *, int, cudaStream_t, int64_t *) {
    return cudaErrorNotSupported;
}
template <typename R>
cudaError_t tile_autotune(TileCache &, std::unordered_map<uint64_t, TileTune> &, const Plan &, const void *,
                          void *, int, void *, int, cudaStream_t, int64_t *) {
    return cudaSuccess;
}

#define DQ_INST(R)                                                                                            \
    template cudaError_t tile_apply<R>(TileCache &, std::unordered_map<uint64_t, TileTune> &, const Plan &,   \
                                       const void *, void *, int, void *, int, cudaStream_t, int64_t *);     \
    template cudaError_t tile_expect<R>(TileCache &, int, const std::vector<DevTerm> &, const DevTerm *,      \
                                        const int32_t *, int, const void *, int, double *, double *, void *,  \
                                        int, cudaStream_t, int64_t *);                                        \
    template cudaError_t tile_adjoint<R>(TileCache &, std::unordered_map<uint64_t, TileTune> &, const Plan &, \
                                         const void *, const std::vector<DevTerm> &, int, const double *,     \
                                         void *, void *, int, double *, double *, double *, void *, int,      \
                                         cudaStream_t, int64_t *);                                            \
    template cudaError_t tile_autotune<R>(TileCache &, std::unordered_map<uint64_t, TileTune> &, const Plan &, \
                                          const void *, void *, int, void *, int, cudaStream_t, int64_t *);
DQ_INST(float)
DQ_INST(double)
#undef DQ_INST

}  // namespace dq
