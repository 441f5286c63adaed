// Fused k-qubit tiles staged in shared memory by TMA (internal interface).
//
// A pass loads, for every value of the amplitude-index bits outside a set T
// of k bit positions (the tile), the 2^k amplitudes that differ only in T,
// applies every scheduled gate whose non-diagonal bits lie in T (diagonal
// factors and controls may sit anywhere), and stores the tile back: one HBM
// read and write of the state for many gates.  T always contains the lowest
// bits, so every TMA box row is a contiguous run of memory.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <unordered_map>
#include <vector>

#include "dq_engine.cuh"
#include "dq_plan.h"

namespace dq {

constexpr int kTileMaxK = 14;
constexpr int kTileLaneBits = 5;      // local bits 0..4 live across the 32 lanes of a warp
constexpr int kTileMaxOps = 384;      // operations per pass (bounds the shared-memory program)
// States up to this size (all rows) take the persistent multi-pass forward
// kernel: they stay in L2 from one pass to the next.
constexpr int64_t kMultiMaxStateBytes = int64_t(32) << 20;

// Tile programs use the engine's operation and layout records.
using TOp = EOp;
using TSeg = ESeg;

struct TPass {
    std::vector<int> T;       // tile bits, ascending (amplitude bits)
    int seg0 = 0, nseg = 0;   // into the schedule's segment array
    int op0 = 0, nops = 0;    // into the schedule's op array
    int rseg0 = 0, nrseg = 0; // reverse-sweep layouts (adjoint schedules)
    int slot0 = 0, nslot = 0; // gradient slots of the pass (adjoint schedules)
    bool pdiag = false;       // holds parity-diagonal ops
    // Host inspection: the plan gate of every executed op in forward order,
    // with flags (bit 0: one gate of a parity-diagonal triple, listed as its
    // three gates; bit 1: one of the three CNOTs a SWAP runs as).
    std::vector<int> gates;
    std::vector<char> flags;
};

// Passes of fused gates.  Adjoint schedules also carry, per pass, the ops
// decoded for reverse-sweep layouts (rops[i] pairs with ops[i]; reverse
// segments name their highest op in op0 and run downwards) and the global
// gradient slots of the pass (rops carry local slot indices).
struct TileSchedule {
    int n = 0, k = 0, low = 0, M = 0;
    bool adjoint = false;
    std::vector<TPass> passes;
    std::vector<TOp> ops, rops;
    std::vector<TSeg> segs, rsegs;
    std::vector<int32_t> slots;
    TOp *d_ops = nullptr, *d_rops = nullptr;
    TSeg *d_segs = nullptr, *d_rsegs = nullptr;
    int32_t *d_slots = nullptr;
    // Launch data of the forward passes for the last state buffer seen (TMA
    // descriptors, shared memory, grid), so repeated calls on one buffer do
    // no host-side encoding or occupancy queries.
    struct Launch {
        CUtensorMap map;
        size_t smem;
        int grid;
    };
    std::vector<Launch> fwd_launch;
    const void *fwd_state = nullptr;
    int fwd_batch = -1;
    // the same for the reverse passes (psi and lambda descriptors)
    std::vector<CUtensorMap> adj_psi, adj_lam;
    const void *adj_p = nullptr, *adj_l = nullptr;
    int adj_batch = -1;
    // run-time specialised passes (null: not compiled; jit_failed: compiling
    // failed once, the interpreter stays in use)
    struct JitModule *jit = nullptr;
    bool jit_failed = false;
    // launch data of the persistent multi-pass kernel (chunks of passes) for
    // the last state buffer seen
    void *multi = nullptr;
    const void *multi_state = nullptr;
    int multi_batch = -1;
    int multi_nte = -1;
    void release();
};

// Autotuned configuration for one circuit structure.
struct TileTune {
    int k = 0;          // tile qubits (0 = default)
    int low = 0;        // always-resident low bits
    int M = 0;          // register bits per thread
    int dense = 0;      // 1: runs of gates on the six lowest-order bits go to tensor-core dense blocks
    int jit = 0;        // 1: forward passes run as run-time specialised kernels
    int rows_jit = 0;   // 1: the whole-row kernel runs as the program's specialised kernel
};

// Host-side cache of schedules and the driver entry point used to encode
// TMA descriptors.
struct TileCache {
    void *encode_fn = nullptr;
    int *errflag = nullptr;             // device error flag of the owning context
    unsigned int *gridbar = nullptr;    // arrival counter of the multi-pass kernel's grid barrier (device)
    bool multi_on = true;               // run all forward passes of an L2-resident state in one launch
    int jit_mode = 2;                   // DQ_OPT_JIT: 0 never, 1 always, 2 when the autotuner measured it faster
    int device = 0;                     // the owning context's device
    std::string jit_err;                // why the last run-time compile failed (empty: none)
    std::unordered_map<uint64_t, TileSchedule *> schedules;
    std::unordered_map<uint64_t, void *> obs;   // observable-pass schedules
    std::unordered_map<const void *, size_t> smem_set;   // dynamic shared memory limit set per kernel
    void release();
};

void tile_release_obs(TileCache &tc);

bool tile_supported(int n, int amp_bytes);
size_t tile_workspace_bytes(const Plan &p, int batch, int amp_bytes);
size_t tile_adjoint_part_bytes(const Plan &p, int batch, int nsm);
size_t tile_expect_part_bytes(int n, int nterms, int batch, int nsm);

template <typename R>
cudaError_t tile_apply(TileCache &tc, std::unordered_map<uint64_t, TileTune> &tuned, const Plan &p,
                       const void *coef, void *state, int batch, void *tws, int nsm, cudaStream_t s,
                       int64_t *launches);
// Observable passes: expectations (when out != null) and, when lam != null,
// lambda = sum_o w_o O_o psi for the adjoint sweep.  part: expectation
// partials [term][row][cta].
template <typename R>
cudaError_t tile_observe(TileCache &tc, int n, const std::vector<DevTerm> &bits, const DevTerm *d_bits,
                         const int32_t *d_ptr, int nobs, const double *rw, const void *psi, void *lam, int batch,
                         double *part, double *out, int nsm, cudaStream_t s, int64_t *launches);
// Reverse sweep on (psi, lam) with gradients.  part: [slot][row][cta].
template <typename R>
cudaError_t tile_adjoint(TileCache &tc, std::unordered_map<uint64_t, TileTune> &tuned, const Plan &p,
                         const void *coef, void *psi, void *lam, int batch, double *part, double *gp, double *gd,
                         int nsm, cudaStream_t s, int64_t *launches);
// Forward passes with the diagonal observables (Z strings only) measured on
// the last pass's tiles, then the FP64 finalisation into out[row][obs].
// part: [term][row][cta] workspace of tile_expect_part_bytes.  Returns
// cudaErrorNotSupported when a term is not diagonal.
template <typename R>
cudaError_t tile_apply_expect(TileCache &tc, std::unordered_map<uint64_t, TileTune> &tuned, const Plan &p,
                              const void *coef, void *state, int batch, const std::vector<DevTerm> &bits,
                              const DevTerm *d_bits, const int32_t *d_ptr, int nobs, double *part, double *out,
                              int nsm, cudaStream_t s, int64_t *launches, bool part_zeroed = false);
template <typename R>
// graphs: time the specialised candidates as CUDA-graph replays (the way a
// context with graphs on runs repeated calls), else as stream launches.
cudaError_t tile_autotune(TileCache &tc, std::unordered_map<uint64_t, TileTune> &tuned, const Plan &p,
                          const void *coef, void *state, int batch, void *tws, int nsm, cudaStream_t s,
                          int64_t *launches, bool graphs = false);

// g0: first gate of the circuit to schedule (adjoint sweeps that stop early).
TileSchedule *get_schedule(TileCache &tc, const Plan &p, int k, int low, int M, int amp, bool adjoint, int g0 = 0);

// Host planner.
bool tile_build_schedule(const Plan &p, int k, int low, int M, int amp_bytes, TileSchedule &out,
                         bool adjoint = false, int g0 = 0);

}  // namespace dq
