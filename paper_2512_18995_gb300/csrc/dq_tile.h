// Fused k-qubit tiles staged in shared memory by TMA (internal interface).
//
// A pass loads, for every value of the amplitude-index bits outside a set T
// of k bit positions (the tile), the 2^k amplitudes that differ only in T,
// applies every scheduled gate whose non-diagonal bits lie in T (diagonal
// factors and controls may sit anywhere), and stores the tile back: one HBM
// read and write of the state for many gates.  T always contains the lowest
// bits, so every TMA box row is a contiguous run of memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <unordered_map>
#include <vector>

#include "dq_engine.cuh"
#include "dq_plan.h"

namespace dq {

constexpr int kTileMaxK = 14;
constexpr int kTileLaneBits = 5;      // local bits 0..4 live across the 32 lanes of a warp
constexpr int kTileMaxOps = 384;      // operations per pass (bounds the shared-memory program)

// Tile programs use the engine's operation and layout records.
using TOp = EOp;
using TSeg = ESeg;

struct TPass {
    std::vector<int> T;     // tile bits, ascending (amplitude bits)
    int seg0 = 0, nseg = 0; // into the schedule's segment array
    int op0 = 0, nops = 0;  // into the schedule's op array
};

struct TileSchedule {
    int n = 0, k = 0, low = 0, M = 0;
    std::vector<TPass> passes;
    std::vector<TOp> ops;
    std::vector<TSeg> segs;
    TOp *d_ops = nullptr;
    TSeg *d_segs = nullptr;
    void release();
};

// Autotuned configuration for one circuit structure.
struct TileTune {
    int k = 0;          // tile qubits (0 = default)
    int low = 0;        // always-resident low bits
    int M = 0;          // register bits per thread
};

// Host-side cache of schedules and the driver entry point used to encode
// TMA descriptors.
struct TileCache {
    void *encode_fn = nullptr;
    int *errflag = nullptr;             // device error flag of the owning context
    std::unordered_map<uint64_t, TileSchedule *> schedules;
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

// Host planner (exposed for tests of the schedule logic).
bool tile_build_schedule(const Plan &p, int k, int low, int M, int amp_bytes, TileSchedule &out);

}  // namespace dq
