// Dense fused blocks on the tensor cores (internal interface).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dq_tile.h"

namespace dq {

// Block width of the tensor-core kernel: a dense unitary on the 6 lowest-order
// qubits (64 x 64 complex, 128 x 128 in real form).  Narrower blocks are
// embedded as I (x) U.
constexpr int kDenseBits = 6;

// Bytes of the operand images (hi and lo TF32 parts of the real form).
constexpr size_t dense_image_bytes() { return 2u * 128u * 128u * 4u; }

bool dense_supported(int n, int batch);

// Real form of the caller's unitary U (complex128, row-major 2^nw x 2^nw on
// the nw lowest-order qubits), embedded into 6 qubits, split into TF32 hi/lo
// parts and laid out as the kernel's shared-memory operand image.
cudaError_t dense_prepare(const void *unitary, int nw, void *image, cudaStream_t s, int64_t *launches);

// The product of a run of gates on bits 0..5 (device DevGate records, their
// blocks in the bound coefficient table of precision R) as a row-major 64 x
// 64 complex128 unitary, ready for dense_prepare with nw = 6.
struct DevGate;
template <typename R>
cudaError_t dense_compose(const DevGate *d_gates, int ngates, const void *coef, void *unitary, cudaStream_t s,
                          int64_t *launches);
// Shortest run of gates on the six lowest-order bits that the planner turns
// into a dense block.
constexpr int kDenseMinRun = 8;

// Apply the prepared block to every row of a complex64 state, in place.
cudaError_t dense_apply(TileCache &tc, const void *image, void *state, int n, int batch, int nsm,
                        cudaStream_t s, int64_t *launches);

}  // namespace dq
