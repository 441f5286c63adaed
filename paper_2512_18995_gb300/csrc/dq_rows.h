// Whole-row in-register kernel (internal interface).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "dq_engine.cuh"
#include "dq_plan.h"

namespace dq {

struct JitModule;

// Engine program for whole rows of one circuit: ops in an execution order
// that keeps every pair of non-commuting ops in gate order (SWAP as three
// CNOTs), register layouts for the forward and the reverse sweep.
// Reverse segments list their first (highest) op in op0 and run downwards.
struct RowProgram {
    int n = 0, M = 0;
    int nacc_shared = 0, nacc_row = 0;
    bool pdiag = false;            // holds parity-diagonal ops
    std::vector<EOp> fops, rops;   // op i decoded for its forward / reverse layout
    std::vector<int> gates;        // host inspection: plan gate per executed op (see record_order)
    std::vector<char> flags;
    std::vector<ESeg> fsegs, rsegs;
    EOp *d_fops = nullptr, *d_rops = nullptr;
    ESeg *d_fsegs = nullptr, *d_rsegs = nullptr;
    JitModule *jit[2] = {nullptr, nullptr};   // the program compiled into a kernel, for 1 and 2 rows per CTA
    bool jit_failed[2] = {false, false};
    void release();
};

// rows_launch with jit set runs rp.jit[rpc - 1]'s kernel (built by
// jit_rows_build for that many rows per CTA) instead of the interpreting one;
// same arguments, same results.

// Register bits the whole-row kernel uses for an n-qubit row (0: the row
// does not fit the kernel).
int rows_pick_M(int n, int amp_bytes);
bool rows_build_program(const Plan &p, int M, RowProgram &out);
size_t rows_smem_bytes(const RowProgram &rp, int amp, bool grad, int nobs, int threads, int rpc = 1);
// Rows per CTA for a call (1 or 2; want: 0 automatic, 1, 2 -- a choice that
// does not fit falls back to 1).  Two rows per CTA share one instruction
// stream (the halves of the CTA run the same program).
int rows_pick_rpc(const RowProgram &rp, int amp, bool grad, int nobs, int batch, int nsm, size_t smem_optin,
                  int want);
size_t rows_part_bytes(const Plan &p, int nsm);

template <typename R>
cudaError_t rows_launch(const RowProgram &rp, const Plan &p, const void *coef, const void *state_in, int forward,
                        const DevTerm *d_wterms, int nterms, int nobs, const double *row_weights, int batch,
                        void *state_out, double *expect_out, double *grad_params, double *grad_data, double *part,
                        int nsm, size_t smem_optin, cudaStream_t s, int64_t *launches, bool jit = false,
                        int rpc = 1);

}  // namespace dq
