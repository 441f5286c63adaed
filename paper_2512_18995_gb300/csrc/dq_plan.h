// Host-side plan structures and kernel launcher declarations (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dq.h"
#include "dq_devterm.h"

namespace dq {

template <typename R> struct Mat2;

// Gate as the kernels see it (bit positions, not wires).  32 bytes.
struct DevGate {
    int32_t kind;       // dq_gate_kind
    int32_t cls;        // GateClass
    int32_t t;          // target bit (SWAP: lower bit)
    int32_t c;          // control bit, or -1 (SWAP: upper bit)
    int32_t coef;       // index of this gate's Mat2 in the bound table (row 0)
    int32_t rowstep;    // row stride of its Mat2 (0: one shared angle)
    int32_t gout;       // gradient output: -1 none; >= 0 see grad_kind
    int32_t gkind;      // 0 none, 1 shared param, 2 per-row param, 3 per-row data
};

// Gate angle source for the bind kernel.  32 bytes.
struct BindGate {
    int32_t kind;
    int32_t pidx;       // parameter index (already offset for uneven batches)
    int32_t didx;       // data feature index
    int32_t coef;       // output slot (row 0)
    int32_t rowstep;    // row stride of the output slot (0: shared angle)
    int32_t aux;        // bit 0: store the complex conjugate of the block;
                        // bits 1..: 1 + index of a fixed block in the plan's table (0: none)
    double angle;
};

// Internal kernel-level kinds (never in the public enum): a fixed 2x2 block
// from the plan's table, uncontrolled or controlled (c = control bit).
constexpr int kKindFixed = 64;
constexpr int kKindCFixed = 65;

// Compiled circuit (cached by structure).
struct Plan {
    uint64_t key = 0;
    int n = 0;
    int ngates = 0;
    int nparams = 0;
    int nfeat = 0;
    int ppr = 0;                       // per-row params
    std::vector<DevGate> gates;        // host copy
    std::vector<BindGate> bind;        // host copy
    int ncoef_shared = 0;              // Mat2 slots with rowstep 0
    int ncoef_rows = 0;                // gates with rowstep 1
    DevGate *d_gates = nullptr;
    BindGate *d_bind = nullptr;
    Mat2<double> *d_fixed = nullptr;   // fixed (possibly non-unitary) blocks, referenced by BindGate.aux
    // Gradient slots: one per gate with a trainable/encoded angle.
    int nslots = 0;
    std::vector<int> slot_of_gate;     // -1 or slot id
    // CSR: output index -> slots (params then data features)
    int32_t *d_pslot_ptr = nullptr, *d_pslots = nullptr;
    int32_t *d_dslot_ptr = nullptr, *d_dslots = nullptr;
    void release();
    // Whether gradient slot `slot` feeds a requested output (parameters when
    // want_params, encoded data when want_data).
    bool slot_needed(int slot, bool want_params, bool want_data) const {
        if (slot < 0) return false;
        return slot_is_data[slot] ? want_data : want_params;
    }
    // First gate (in circuit order) whose gradient is requested; ngates when
    // none.  The reverse sweep never needs to go below it.
    int first_grad_gate(bool want_params, bool want_data) const {
        for (int i = 0; i < ngates; ++i)
            if (slot_needed(slot_of_gate[i], want_params, want_data)) return i;
        return ngates;
    }
    std::vector<char> slot_is_data;    // per slot: encoded-data gradient
};

// Workspace bump allocator over the context's device buffer.
struct Arena {
    char *base = nullptr;
    size_t cap = 0, used = 0;
    bool measuring = false;            // only count bytes
    void *take(size_t bytes) {
        used = (used + 255) & ~size_t(255);
        void *p = measuring ? nullptr : (void *)(base + used);
        used += bytes;
        return p;
    }
};

// Per-launch accounting.  Every kernel launch of the library is wrapped in a
// LaunchScope: it bumps the context's launch counter and, when tracing is on,
// records a CUDA event pair around the launch on its stream so per-kernel
// device time can be read back (dq_ctx_trace_get).
struct Tracer {
    bool on = false;
    std::vector<std::string> names;
    struct Rec { int name; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    // launches and milliseconds per name accumulated from replayed CUDA graphs
    std::vector<std::pair<int64_t, double>> acc;
    cudaEvent_t get_event();
    int name_id(const char *n);
    void release();
};
extern thread_local Tracer *g_tracer;

struct LaunchScope {
    LaunchScope(cudaStream_t s, const char *name, int64_t *counter);
    ~LaunchScope();
    cudaStream_t s;
    int64_t *counter;
    int rec = -1;
};

// ---- plain per-gate path -------------------------------------------------
template <typename R>
cudaError_t plain_bind(const Plan &p, const double *params, const double *data, int batch,
                       void *coef, cudaStream_t s, int64_t *launches);
template <typename R>
cudaError_t plain_init_zero(void *state, int n, int batch, cudaStream_t s, int64_t *launches);
// plain_bind, the clearing of nzero doubles at `zero` (may be NULL) and
// plain_init_zero of `state` (p.n qubits), in one launch
template <typename R>
cudaError_t plain_bind_init(const Plan &p, const double *params, const double *data, int batch, void *coef,
                            void *state, double *zero, int64_t nzero, cudaStream_t s, int64_t *launches);
template <typename R>
cudaError_t plain_apply(const Plan &p, const void *coef, void *state, int batch, int dagger,
                        cudaStream_t s, int64_t *launches);
template <typename R>
cudaError_t plain_expect(int n, const std::vector<DevTerm> &terms, int nobs, const void *state,
                         int batch, double *part, double *out, cudaStream_t s, int64_t *launches);
size_t plain_expect_part_bytes(int n, int nterms, int batch);
cudaError_t plain_expect_finalize(const double *part, const DevTerm *d_terms, const int32_t *d_obs_ptr,
                                  int nobs, int n, int batch, double *out, cudaStream_t s,
                                  int64_t *launches);
template <typename R>
cudaError_t plain_lambda(int n, const std::vector<DevTerm> &terms, int nobs, const double *w,
                         const void *psi, void *lam, int batch, cudaStream_t s, int64_t *launches);
template <typename R>
cudaError_t plain_adjoint(const Plan &p, const void *coef, const std::vector<DevTerm> &terms,
                          int nobs, const double *row_weights, void *psi, void *lam, int batch,
                          double *part, double *grad_params, double *grad_data,
                          cudaStream_t s, int64_t *launches);
size_t plain_adjoint_part_bytes(const Plan &p, int batch);
// grad[...] from partials laid out [slot][row][blk] (nblk blocks per row).
cudaError_t grad_reduce(const Plan &p, const double *part, int batch, int nblk, double *grad_params,
                        double *grad_data, cudaStream_t s, int64_t *launches);
// out[row, o] from expectation partials laid out [term][row][blk].
cudaError_t expect_finalize_nblk(const double *part, const DevTerm *d_terms, const int32_t *d_obs_ptr, int nobs,
                                 int batch, int nblk, double *out, cudaStream_t s, int64_t *launches);

// ---- squared norms with FP64 accumulation; bounded-wait self-test ----------
int norm_blocks_per_row(int n, int batch);
size_t norm_part_bytes(int n, int batch);
template <typename R>
cudaError_t state_norm(const void *state, int n, int batch, double *part, double *out, cudaStream_t s,
                       int64_t *launches);
cudaError_t selftest_wait_expiry(int *errflag, cudaStream_t s, int64_t *launches);
// bounds-checking build: one failing check (cudaErrorNotSupported otherwise)
cudaError_t selftest_bounds(cudaStream_t s, int64_t *launches);

// ---- whole state in shared memory (small n) --------------------------------
size_t wsv_smem_bytes(int n, int dtype_bytes, bool grad, int ngrad_acc);
bool wsv_supported(int n, int amp_bytes, bool grad, size_t smem_optin, int ndouble);
// doubles the whole-state kernel keeps next to the vectors
inline int wsv_doubles(const Plan &p, int nobs) {
    return (p.ppr ? 0 : p.nparams) + p.nfeat + (p.ppr ? p.nparams : 0) + nobs;
}
template <typename R>
cudaError_t wsv_launch(const Plan &p, const void *coef, const void *state_in, int forward,
                       const DevTerm *d_wterms, int nterms, int nobs,
                       const double *row_weights, int batch, void *state_out, double *expect_out,
                       double *grad_params, double *grad_data, double *part, int nsm, cudaStream_t s,
                       int64_t *launches);
size_t wsv_part_bytes(const Plan &p, int nsm);

// ---- uneven batch, one persistent launch ----------------------------------
struct BatchCirc {
    int32_t n;
    int32_t gate0;       // first gate in the concatenated table
    int32_t ngates;
    int32_t param0;      // first parameter (global index)
    int32_t nparams;
    int32_t pad[3];
};
// Launch choices of the persistent uneven-batch kernel (autotuned per batch
// signature by dq_batch_autotune, else batch_default_tune).
struct BatchTune {
    int nsmem = 0;       // circuits with at most this many qubits run in shared memory, larger ones in L2 scratch
    int threads = 0;     // threads per circuit (power of two, 64 .. 512)
    int per_sm = 0;      // CTAs per SM at most (1 .. kBatchMaxPerSm)
    int l2_mb = 0;       // scratch of the circuits in global memory in flight at once, MiB (0: every CTA)
};
constexpr int kBatchMaxPerSm = 8;   // L2 scratch slices per SM (circuits of up to 16 qubits; 4 above)
inline int batch_max_per_sm(int nmax) { return nmax <= 16 ? kBatchMaxPerSm : 4; }
BatchTune batch_default_tune(int amp_bytes);
template <typename R>
cudaError_t batch_run(const BatchCirc *d_circ, int ncirc, const int32_t *d_order,
                      const DevGate *d_gates, const void *coef, const DevTerm *d_terms, int nterms,
                      int nobs, int nmax, int maxparams, double *expect_out, double *grad_params,
                      void *scratch, int *d_counter, int nsm, size_t smem_optin, const BatchTune &tune,
                      cudaStream_t s, int64_t *launches);
size_t batch_scratch_bytes(int nmax, int amp_bytes, int nsm, size_t smem_optin);

}  // namespace dq
