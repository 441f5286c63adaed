/*
 * dq.h -- C ABI of libdq, a batched state-vector simulator for parameterised
 * qubit circuits on NVIDIA GB300 (sm_103a).
 *
 * The library computes, on the GPU, what the qubit-circuit backend of
 * DeepQuantum (arXiv 2512.18995) computes: the evolution of a batch of pure
 * states |psi_n> = U_n ... U_1 |psi_0> (Sec. "Quantum Computing with Qubits",
 * Background), expectation values of observables given as (weighted sums of)
 * Pauli strings (same section, API Overview: observable()/expectation()), and
 * gradients of those expectations with respect to trainable parameters and
 * encoded inputs by adjoint differentiation (Sec. "Distributed Simulations":
 * a custom autograd function using the adjoint method).
 *
 * Conventions
 *   - Wire q of an n-qubit register is bit (n-1-q) of the amplitude index:
 *     wire 0 is the most significant bit.
 *   - Rotations are R_P(t) = exp(-i t P / 2) for P in {X, Y, Z}; RZ(t) =
 *     diag(e^{-it/2}, e^{it/2}).  CP(t) = diag(1, 1, 1, e^{it}) (the
 *     controlled phase of Sec. "Distributed Quantum Fourier Transform").
 *     Controlled rotations apply R_P(t) to the target when the control is |1>.
 *   - A state batch is `batch` contiguous rows of 2^n amplitudes.  DQ_C64
 *     amplitudes are interleaved float pairs (re, im), 8 bytes; DQ_C128 are
 *     interleaved double pairs, 16 bytes.  Row r starts at element r * 2^n.
 *     State pointers must be 16-byte aligned.
 *   - Angles: gate g uses params[g.param_idx] (or params[row * nparams +
 *     g.param_idx] when params_per_row != 0) when param_idx >= 0, else
 *     data[row * nfeatures + g.data_idx] when data_idx >= 0 (an encoded input
 *     feature), else the fixed g.angle.  params and data are FP64.
 *
 * Ownership and streams
 *   - All device buffers (states, params, data, outputs) are allocated and
 *     freed by the caller; the library never frees caller memory.  Host
 *     arrays (gate lists, Pauli terms, offsets) are only read during the call.
 *   - Scratch memory comes from the context's workspace: attach one with
 *     dq_ctx_set_workspace (size from dq_workspace_bytes); otherwise the
 *     context grows its own device workspace with cudaMalloc on first need.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Every compute call is asynchronous on that stream.
 *
 * Errors
 *   Every call returns a dq_status.  Arguments are validated on the host
 *   before any launch (DQ_ERR_INVALID_ARG, nothing launched); CUDA failures
 *   return DQ_ERR_CUDA.  Device-side bounded waits that give up record
 *   DQ_ERR_TIMEOUT in the context, reported by dq_ctx_check.  A
 *   human-readable message for the last failure is in dq_last_error.  The
 *   library never aborts the process and throws nothing across the ABI.
 */
#ifndef DQ_H_INCLUDED
#define DQ_H_INCLUDED

#ifndef __CUDACC_RTC__   /* run-time compiled kernels bring their own integer types */
#include <stddef.h>
#include <stdint.h>
#endif

#if defined(__GNUC__)
#define DQ_API __attribute__((visibility("default")))
#else
#define DQ_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dq_status {
    DQ_OK = 0,
    DQ_ERR_INVALID_ARG = 1,
    DQ_ERR_UNSUPPORTED = 2,
    DQ_ERR_OOM = 3,
    DQ_ERR_CUDA = 4,
    DQ_ERR_TIMEOUT = 5
} dq_status;

typedef enum dq_dtype { DQ_C64 = 0, DQ_C128 = 1 } dq_dtype;

/* Gate kinds.
 *   One-qubit kinds (H X Y Z S RX RY RZ P U3) act on wires[0].
 *   Controlled kinds (CNOT CZ CP CRX CRY CRZ) take wires[0] as the control and
 *   wires[1] as the target.
 *   SWAP, RXX, RYY and RZZ act on wires[0] and wires[1] (symmetric).
 *   CCX (Toffoli, the two-control X) takes wires[0] and wires[1] as controls
 *   and wires[2] as the target.
 * Wires of a gate must be distinct; unused entries of `wires` are ignored.
 *
 * Parametric kinds: RX RY RZ CP CRX CRY CRZ P RXX RYY RZZ (one angle t) and U3
 * (three angles).  Definitions beyond the rotations of the conventions above:
 *   P(t)     = diag(1, e^{it}), the phase shift.
 *   R_PP(t)  = exp(-i t P(x)P / 2) for PP in {XX, YY, ZZ} (the two-qubit
 *              rotations of the paper's QCNN and Trotterised-TFIM examples,
 *              Sec. "Quantum Machine Learning" and "Simulation of Large
 *              Quantum Systems with MPS").
 *   U3(theta, phi, lam) = [[cos(theta/2), -e^{i lam} sin(theta/2)],
 *                          [e^{i phi} sin(theta/2), e^{i(phi+lam)} cos(theta/2)]]
 *              (the general one-qubit gate of the paper's QNN example, whose
 *              action on |0> is the Bloch form of Sec. "Quantum Computing with
 *              Qubits").  Its three angles are params[param_idx + 0, 1, 2]
 *              (theta, phi, lam), or data[row, data_idx + 0, 1, 2]; a U3 with
 *              neither index set is rejected (DQ_ERR_INVALID_ARG).
 * The library lowers RXX, RYY, RZZ, U3 and CCX to exact products of the other
 * kinds before planning (gradients of their angles are exact as well).
 *
 * Noise channels (the "single-qubit noise channels" of the API Overview) act
 * on wires[0] with the probability p in `angle` (fixed; param_idx and
 * data_idx must be -1), and are accepted only by dq_density_forward:
 *   DQ_BITFLIP       rho -> (1-p) rho + p X rho X
 *   DQ_PHASEFLIP     rho -> (1-p) rho + p Z rho Z
 *   DQ_DEPOLARIZING  rho -> (1-p) rho + p/3 (X rho X + Y rho Y + Z rho Z), p <= 3/4
 *   DQ_AMPDAMP       Kraus operators [[1, 0], [0, sqrt(1-p)]], [[0, sqrt(p)], [0, 0]]
 *                    (amplitude damping with decay probability p). */
typedef enum dq_gate_kind {
    DQ_H = 0, DQ_X, DQ_Y, DQ_Z, DQ_S,
    DQ_RX, DQ_RY, DQ_RZ,
    DQ_CNOT, DQ_CZ, DQ_CP, DQ_SWAP,
    DQ_CRX, DQ_CRY, DQ_CRZ,
    DQ_P, DQ_U3, DQ_RXX, DQ_RYY, DQ_RZZ, DQ_CCX,
    DQ_BITFLIP, DQ_PHASEFLIP, DQ_DEPOLARIZING, DQ_AMPDAMP,
    DQ_NUM_GATE_KINDS
} dq_gate_kind;

/* Which implementation runs the circuit.
 *   DQ_PATH_PLAIN: one kernel launch per gate (and per adjoint step), each a
 *                  full sweep over the batch -- the paper's gate-by-gate
 *                  evolution, kept as the baseline.  Its expectation and
 *                  adjoint kernels take one grid row per batch row, so they
 *                  accept at most 65535 rows per call (more return
 *                  DQ_ERR_CUDA, invalid configuration).
 *   DQ_PATH_FUSED: whole states in shared memory for small n, otherwise
 *                  k-qubit tiles staged in shared memory by TMA with many
 *                  gates applied per HBM pass.
 *   DQ_PATH_AUTO:  fused where supported (default). */
typedef enum dq_path { DQ_PATH_AUTO = 0, DQ_PATH_PLAIN = 1, DQ_PATH_FUSED = 2 } dq_path;

typedef struct dq_gate {
    int32_t kind;        /* dq_gate_kind */
    int32_t wires[3];    /* see dq_gate_kind */
    int32_t param_idx;   /* >= 0: trainable parameter index, else -1 */
    int32_t data_idx;    /* >= 0: encoded feature index, else -1 */
    double angle;        /* fixed angle when param_idx < 0 and data_idx < 0 */
} dq_gate;              /* 32 bytes */

typedef struct dq_circuit {
    int32_t nqubits;       /* 1 .. 34 */
    int32_t ngates;        /* >= 0 */
    const dq_gate *gates;  /* host array of ngates */
    int32_t nparams;       /* number of trainable parameters (per row if per-row) */
    int32_t nfeatures;     /* encoded features per row (0 if none) */
} dq_circuit;

/* One Pauli string with a real weight.  Bit q of xmask / zmask refers to wire
 * q: X only -> X, Z only -> Z, both -> Y. */
typedef struct dq_pauli_term {
    double coeff;
    uint64_t xmask;
    uint64_t zmask;
} dq_pauli_term;

/* nobs observables; observable o is sum_{k in [term_offsets[o],
 * term_offsets[o+1])} terms[k].coeff * P_k.  Host arrays. */
typedef struct dq_observables {
    int32_t nobs;
    const int32_t *term_offsets;   /* nobs + 1 entries, non-decreasing, [0] = 0 */
    const dq_pauli_term *terms;
} dq_observables;

typedef struct dq_ctx dq_ctx;

/* ---- context ----------------------------------------------------------- */

/* Create a context on CUDA device `device` (made current for the calls of
 * this context).  *out receives the handle.  Holds plan caches and the
 * workspace; not thread-safe: use one context per host thread. */
DQ_API dq_status dq_ctx_create(dq_ctx **out, int device);

/* Destroy a context, freeing its own allocations (never caller memory).
 * Synchronises the device first. */
DQ_API dq_status dq_ctx_destroy(dq_ctx *ctx);

/* Message of the last failure on this context ("" if none).  Valid until the
 * next call on the context. */
DQ_API const char *dq_last_error(const dq_ctx *ctx);

/* Select the implementation (dq_path) used by later calls. */
DQ_API dq_status dq_ctx_set_path(dq_ctx *ctx, int path);

/* Context options (dq_ctx_set_option).
 *
 * DQ_OPT_MULTIPASS (default 1): on the fused path, run every forward tile
 *   pass of a state whose rows together hold at most 32 MiB (it stays in L2
 *   between passes) in one persistent launch, the passes separated by a grid
 *   barrier whose wait is bounded like every other device-side wait; 0 runs
 *   one launch per pass.  Results are identical either way.
 * DQ_OPT_WAIT_LIMIT_US (default 2000000): the limit, in microseconds (1 ..
 *   60000000), of every device-side bounded wait of the context's kernels (a
 *   TMA copy's or a tensor-core product's completion barrier, the multi-pass
 *   grid barrier).  A wait that runs out sets the context's device error
 *   flag; the kernel then waits (with the same limit) for its own copies in
 *   flight, frees what it holds and returns, and the next dq_ctx_check
 *   returns DQ_ERR_TIMEOUT.  Setting it synchronises the device.
 * DQ_OPT_DENSE_BLOCKS (default 2): on forward-only calls of the fused path
 *   (dq_apply_circuit, dq_forward_grad without gradients) for complex64
 *   states of more than 6 qubits, runs of at least 8 consecutive gates on the
 *   six lowest-order qubits (wires nqubits-6 .. nqubits-1, angles shared by
 *   all rows) are multiplied into one 64 x 64 unitary on the device (FP64
 *   products of the bound gate blocks) and applied by the tensor-core kernel
 *   of dq_apply_dense; gates on the other wires that commute with a run
 *   (disjoint wires) move past it, the rest run as tile passes.  0: never;
 *   1: whenever the circuit has such a run; 2: when dq_plan_autotune measured
 *   the blocks faster for this circuit.  Gradient calls always run gate by
 *   gate (the adjoint sweep needs every gate's generator).
 * DQ_OPT_JIT (default 2): tile passes (forward and reverse sweep) and the
 *   whole-row kernel as run-time specialised kernels -- each pass's (or the
 *   row program's) ops compiled (NVRTC, loaded with the runtime's library
 *   API) into direct calls of the same handlers the interpreting kernel
 *   dispatches to, with every register position, control mask and layout a
 *   literal; same arithmetic per element.  0: never; 1: always (compiled on
 *   first use, which takes seconds); 2: when dq_plan_autotune measured them
 *   faster for this circuit and precision (tile passes and the whole-row
 *   kernel are measured separately).  Without NVRTC, or if a compile fails,
 *   the interpreting kernel runs.
 * DQ_OPT_ROWS_PER_CTA (default 0): complex64 rows of up to 16 qubits held
 *   on chip run one (1) or two (2) rows per CTA; 0 chooses two for rows of at
 *   most 128 threads when the batch gives every SM at least four rows and two
 *   rows' buffers fit in shared memory.  The two halves of a CTA run the same
 *   program in step (one instruction stream for both rows).  Expectations,
 *   states and per-row gradients are identical either way, shared-parameter
 *   gradients up to the order of their FP64 sums; complex128 rows and a
 *   choice that does not fit run one row per CTA. */
enum dq_option {
    DQ_OPT_MULTIPASS = 1,
    DQ_OPT_WAIT_LIMIT_US = 2,
    DQ_OPT_DENSE_BLOCKS = 3,
    DQ_OPT_JIT = 4,
    DQ_OPT_ROWS_PER_CTA = 5
};

/* Set a context option; DQ_ERR_INVALID_ARG for an unknown option or value.
 * Captured graphs of the context are dropped (the next calls capture anew). */
DQ_API dq_status dq_ctx_set_option(dq_ctx *ctx, int option, int64_t value);

/* Attach caller-owned device memory of `bytes` bytes (16-byte aligned) as the
 * workspace; ptr == NULL detaches it.  The memory must stay valid while calls
 * that use it are in flight. */
DQ_API dq_status dq_ctx_set_workspace(dq_ctx *ctx, void *ptr, size_t bytes);

/* Bytes of workspace that dq_apply_circuit / dq_expect / dq_adjoint_grad /
 * dq_forward_grad need for this circuit, observable set (may be NULL), batch
 * and dtype under the context's current path, written to *out. */
DQ_API dq_status dq_workspace_bytes(dq_ctx *ctx, const dq_circuit *circuit,
                             const dq_observables *obs, int batch, int dtype,
                             size_t *out);

/* Bytes of workspace that dq_batch_forward_grad needs for these circuits
 * and dtype under the context's current path (observables of up to 256
 * terms), written to *out. */
DQ_API dq_status dq_batch_workspace_bytes(dq_ctx *ctx, int ncirc, const dq_circuit *circuits,
                                          int dtype, size_t *out);

/* Synchronise `stream` and report device-side failures recorded by earlier
 * calls (DQ_ERR_TIMEOUT for a bounded wait that gave up; in the
 * bounds-checking build, DQ_ERR_CUDA for indices outside their buffer, the
 * message naming the first one and its source site), then clear them. */
DQ_API dq_status dq_ctx_check(dq_ctx *ctx, void *stream);

/* The bounds-checking build: libdq_debug.so, compiled with DQ_DEBUG_BOUNDS
 * (build.build(debug=True); the Python binding loads it when the environment
 * variable DQ_DEBUG_BOUNDS is 1).  The per-gate sweep kernels, the engine's
 * register-layout loads and stores (tile passes, whole-row kernels), the
 * observable passes' partner reads, the reverse passes' result stores and
 * the whole-row kernels' global state and partner accesses check every index
 * against its buffer (2^n amplitudes per row, 2^k per tile); an index outside
 * skips its access and is counted for dq_ctx_check.  Run-time specialisation
 * (DQ_OPT_JIT) is off in that build.  dq_selftest_bounds launches one check
 * that fails without touching memory (the next dq_ctx_check reports it);
 * DQ_ERR_UNSUPPORTED in the normal build. */
DQ_API dq_status dq_selftest_bounds(dq_ctx *ctx, void *stream);

/* Failure-detection self-test (no counterpart in the paper): launches on
 * `stream` one kernel whose bounded wait runs out on purpose -- it waits on
 * an mbarrier that nothing arrives on and that no copy targets, so nothing
 * is in flight -- and records the timeout in the context's device error
 * flag the way a kernel whose copy never landed would.  After it, with the
 * wait limit lowered by DQ_OPT_WAIT_LIMIT_US to keep the test short,
 * dq_ctx_check returns DQ_ERR_TIMEOUT and clears the flag; the context stays
 * usable. */
DQ_API dq_status dq_selftest_wait_expiry(dq_ctx *ctx, void *stream);

/* Number of kernels this context has launched since creation (for launch
 * accounting by callers). */
DQ_API int64_t dq_ctx_launch_count(const dq_ctx *ctx);

/* CUDA-graph replay.  With replay on, the second dq_forward_grad or
 * dq_apply_circuit call with the same circuit structure, observables, batch,
 * dtype, path and buffer pointers (parameters, data, weights, outputs,
 * workspace) is captured into a CUDA graph on a stream owned by the context,
 * and that call and later identical ones launch the graph on the caller's
 * stream instead of issuing the kernels one by one.  Values behind the
 * pointers (parameters, data) are read when the graph runs, so they may change
 * between calls; pointers and shapes may not.  With tracing on, calls use
 * their own traced graphs (see dq_ctx_set_tracing).  Off by default. */
DQ_API dq_status dq_ctx_set_graphs(dq_ctx *ctx, int on);

/* Tracing (the library's profiling hook).  With tracing on, every kernel the
 * context launches is bracketed by a CUDA event pair on its stream and the
 * device time is aggregated per kernel name.  With graph replay on, the
 * event pairs are captured into the graph as event-record nodes, and every
 * replay of a traced graph synchronises the caller's stream and adds the
 * graph's per-kernel times (device time inside the graph, no host launch
 * gaps).  Turning tracing on or off clears the records and the captured
 * graphs.  dq_ctx_trace_count synchronises the device, then
 * returns the number of distinct kernel names recorded (or -1 on error);
 * dq_ctx_trace_get copies entry i's name (NUL-terminated, truncated to
 * name_len) and writes its launch count and total device milliseconds. */
DQ_API dq_status dq_ctx_set_tracing(dq_ctx *ctx, int on);
DQ_API int dq_ctx_trace_count(dq_ctx *ctx);
DQ_API dq_status dq_ctx_trace_get(dq_ctx *ctx, int i, char *name, size_t name_len,
                                  int64_t *launches, double *total_ms);

/* ---- hot path ----------------------------------------------------------- */

/* State preparation |psi_0> = |0...0> for every row (the initial state of
 * the evolution in Sec. "Quantum Computing with Qubits", Background).
 * state: device, batch * 2^nqubits amplitudes of `dtype`, overwritten. */
DQ_API dq_status dq_state_init(dq_ctx *ctx, int nqubits, int batch, int dtype,
                        void *state, void *stream);

/* In-place evolution |psi> <- U_G ... U_1 |psi> of every row (Sec. "Quantum
 * Computing with Qubits": discrete time evolution of a pure state; API
 * Overview: forward execution).  params: device FP64, nparams values (shared)
 * or batch * nparams (params_per_row != 0); may be NULL if no gate uses a
 * parameter.  data: device FP64 batch * nfeatures, or NULL. */
DQ_API dq_status dq_apply_circuit(dq_ctx *ctx, const dq_circuit *circuit,
                           const double *params, int params_per_row,
                           const double *data, void *state, int batch,
                           int dtype, void *stream);

/* Expectations out[row * nobs + o] = sum_k c_k Re <psi_row| P_k |psi_row>
 * (API Overview: expectation() of predefined observables; weighted sums as
 * in the TFIM Hamiltonian of Sec. "Simulation of Large Quantum Systems with
 * MPS").  Products are formed in the state precision and summed in FP64.
 * state: device, read only.  out: device FP64, batch * nobs. */
DQ_API dq_status dq_expect(dq_ctx *ctx, int nqubits, const dq_observables *obs,
                    const void *state, int batch, int dtype, double *out,
                    void *stream);

/* Squared norm <psi|psi> of every row of `state` (batch rows of 2^nqubits
 * amplitudes, device) into out[batch] (device, FP64): |psi_i|^2 in the
 * state's precision, summed in runs of eight in that precision and in FP64
 * above that, the per-block partials of a row added in a fixed order.  With
 * a normalised initial state this is the drift of the norm that rounding in
 * the state's precision accumulated over the gates (the paper's evolution is
 * unitary: Sec. "Quantum Computing with Qubits", Background).  Uses the
 * context workspace; asynchronous on `stream`. */
DQ_API dq_status dq_state_norm(dq_ctx *ctx, int nqubits, const void *state, int batch, int dtype,
                               double *out, void *stream);

/* Adjoint differentiation (Sec. "Distributed Simulations", adjoint method)
 * of L = sum_row sum_o w[row, o] <psi_row| O_o |psi_row>, where state holds
 * the final states psi_row produced by dq_apply_circuit with the same
 * circuit, params and data.  row_weights: device FP64 batch * nobs, or NULL
 * for all ones.  Outputs (device FP64, overwritten; either may be NULL):
 *   grad_params: nparams values summed over rows (shared params) or
 *                batch * nparams (params_per_row != 0);
 *   grad_data:   batch * nfeatures.
 * flags: DQ_ADJ_CLOBBER_STATE lets the call use `state` as the reverse-sweep
 * vector (its contents are unspecified afterwards: the sweep stops at the
 * earliest gate whose gradient is requested); without it the state is
 * preserved and one extra state-sized buffer of workspace is used. */
#define DQ_ADJ_CLOBBER_STATE 1
DQ_API dq_status dq_adjoint_grad(dq_ctx *ctx, const dq_circuit *circuit,
                          const double *params, int params_per_row,
                          const double *data, const dq_observables *obs,
                          const double *row_weights, void *state, int batch,
                          int dtype, int flags, double *grad_params,
                          double *grad_data, void *stream);

/* One call for the whole batched hot path: state preparation, evolution,
 * expectations and adjoint gradients.  expect_out: device FP64 batch * nobs
 * (may be NULL).  grad_params / grad_data as in dq_adjoint_grad (either may
 * be NULL; both NULL = forward only).  state_out: device buffer for the final
 * states (batch * 2^n), or NULL when the states are not needed -- the small-n
 * fused path then keeps them on chip only. */
DQ_API dq_status dq_forward_grad(dq_ctx *ctx, const dq_circuit *circuit,
                          const double *params, int params_per_row,
                          const double *data, const dq_observables *obs,
                          const double *row_weights, int batch, int dtype,
                          double *expect_out, double *grad_params,
                          double *grad_data, void *state_out, void *stream);

/* The forward path with host buffers, for callers that hold their inputs
 * and want their results in host memory (Sec. "Quantum Computing with
 * Qubits", API Overview: a parameterised circuit run to expectation values).
 *   params:     host FP64, the circuit's nparams shared parameters (NULL
 *               when nparams == 0); read during the call.
 *   expect_out: host FP64, batch * nobs expectations, written before the
 *               call returns (may be NULL when batch == 0).
 * The call copies params to the device, prepares |0...0> for every row,
 * runs the circuit and the expectations as dq_forward_grad does, copies the
 * expectations back and synchronises `stream`.  With graphs on
 * (dq_ctx_set_graphs) and both buffers in pinned host memory (cudaHostAlloc
 * or cudaHostRegister), the two copies and the kernels of a repeated call
 * are one CUDA graph replay; pageable buffers work, with the copies issued
 * one by one.  Circuits with encoded data (data_idx gates) return
 * DQ_ERR_UNSUPPORTED: use dq_forward_grad.  The device copies live in a
 * context-owned buffer (grown with cudaMalloc when a call needs more,
 * DQ_ERR_OOM if that fails); the rest uses the context workspace. */
DQ_API dq_status dq_forward_host(dq_ctx *ctx, const dq_circuit *circuit, const double *params,
                                 const dq_observables *obs, int batch, int dtype, double *expect_out,
                                 void *stream);

/* Uneven batch: ncirc independent circuits (own qubit count, depth and
 * parameters) run to expectations and per-circuit adjoint gradients in one
 * persistent launch.  circuits: host array.  params: device FP64, circuit c's
 * parameters at params[param_offsets[c] ...]; param_offsets: host, ncirc + 1
 * entries.  expect_out: device FP64 ncirc * nobs.  grad_params: device FP64
 * laid out like params (may be NULL for forward only).  The observable must
 * act on wires below every circuit's qubit count.  Under DQ_PATH_PLAIN the
 * circuits run one after another on the per-gate path (the baseline of the
 * persistent kernel). */
DQ_API dq_status dq_batch_forward_grad(dq_ctx *ctx, int ncirc, const dq_circuit *circuits,
                                const double *params, const int64_t *param_offsets,
                                const dq_observables *obs, int dtype,
                                double *expect_out, double *grad_params,
                                void *stream);

/* Autotuner of the uneven-batch launch (batches of circuits of uneven qubit
 * counts and depths; the API Overview batches encode=True circuits).  Runs
 * dq_batch_forward_grad with every candidate launch configuration -- the
 * largest qubit count kept in shared memory (10, 11, 12; larger circuits
 * work in per-CTA scratch in global memory), threads per circuit (128, 256,
 * 512), CTAs per SM (2, 4, 8), and the scratch in flight at once (0, 64, 96,
 * 128, 160 MiB: only as many CTAs take the larger circuits as keep their
 * scratch within it, so it stays in L2; 0: every CTA) -- on the caller's own inputs,
 * keeps the fastest for this batch structure and dtype (later
 * dq_batch_forward_grad calls of the same structure use it), and leaves the
 * outputs as that configuration computes them.  choice (host, 4 ints, may be
 * NULL) receives {qubits in shared memory, threads, CTAs per SM, scratch
 * MiB}.  Synchronises the stream; arguments as dq_batch_forward_grad. */
DQ_API dq_status dq_batch_autotune(dq_ctx *ctx, int ncirc, const dq_circuit *circuits,
                                   const double *params, const int64_t *param_offsets,
                                   const dq_observables *obs, int dtype, double *expect_out,
                                   double *grad_params, int *choice, void *stream);

/* Allocation-free variant of dq_forward_grad, for callers that must not
 * allocate device memory at call time -- for example a serving loop that
 * reserves all its memory at start-up because cudaMalloc/cudaFree can stall
 * the whole device, or a host application whose own allocator owns the GPU's
 * memory budget.  It takes no context and calls no cudaMalloc, cudaFree or
 * other allocating routine.  The paper has no counterpart to this entry
 * point.
 *
 * It runs the on-chip path (every row's state and adjoint vector held in one
 * CTA's shared memory), so it accepts only circuits for which that path
 * applies (about 13 qubits for complex64, 12 for complex128) and returns
 * DQ_ERR_UNSUPPORTED otherwise.  Its scratch (gate tables, bound gate
 * coefficients, Pauli terms and per-CTA gradient partials) is a fixed
 * static device array of DQ_NOALLOC_SCRATCH_BYTES bytes that every GPU that
 * loads the library's device code holds until the process exits; a call
 * needing more returns DQ_ERR_UNSUPPORTED with the required size in `err`.
 *
 * The first call on each device looks up that array's device address (with
 * that device current).  Under CUDA's lazy module loading (the default) that
 * lookup is also what loads the device code and reserves the array on the
 * device, so make the first call at start-up, before the caller's own
 * allocator takes the rest of the memory and before any stream capture.
 * The call uploads its gate and term tables from host buffers of its own on
 * `stream`; on a stream that is capturing it returns DQ_ERR_UNSUPPORTED
 * before doing anything.
 * All calls on a device share the one array and it keeps the last call's
 * contents, so two calls whose work overlaps on the GPU (different streams,
 * or host threads) race: serialise them, e.g. on one stream.
 *
 * Arguments are those of dq_forward_grad (expect_out, grad_params and
 * grad_data may each be NULL), without a context and without state_out; the
 * current CUDA device is used.  err (may be NULL) receives a message of up to
 * err_len bytes on failure. */
#define DQ_NOALLOC_SCRATCH_BYTES (8u << 20)
DQ_API dq_status dq_forward_grad_noalloc(const dq_circuit *circuit, const double *params,
                                         int params_per_row, const double *data,
                                         const dq_observables *obs, const double *row_weights,
                                         int batch, int dtype, double *expect_out,
                                         double *grad_params, double *grad_data, void *stream,
                                         char *err, size_t err_len);

/* Dense fused block on the tensor cores.  Applies a dense 2^nw x 2^nw
 * unitary U to the nw lowest-order qubits (wires nqubits-nw .. nqubits-1)
 * of every row of a complex64 state, in place: amplitude index h*2^nw + j of
 * a row becomes sum_j U[i][j] psi[h*2^nw + j] at h*2^nw + i.  This is the
 * pure-state evolution of Sec. "Quantum Computing with Qubits" (Background)
 * with a run of consecutive gates multiplied into one matrix; the paper
 * itself applies gates one at a time and has no such fusion.
 *
 * unitary: device, complex128 row-major (interleaved re, im), 2^nw x 2^nw;
 * index bit b of i and j is wire nqubits-1-b.  Unitarity is not checked.
 * 1 <= nw <= 6 and nqubits >= 6; the block is applied as I (x) U on the six
 * lowest-order qubits.  The products run on the tensor cores as three TF32
 * passes (hi/lo splits of U and of the state) accumulated in FP32, which
 * keeps FP32-level accuracy.  state: device, 16-byte aligned, batch rows of
 * 2^nqubits complex64; batch * 2^(nqubits-6) < 2^31.  dtype must be DQ_C64
 * (DQ_C128 returns DQ_ERR_UNSUPPORTED: the FP64 tensor rate of this GPU gives
 * no fast path).  Asynchronous on `stream`; the workspace holds a 128 KiB
 * operand image until the kernel has read it. */
DQ_API dq_status dq_apply_dense(dq_ctx *ctx, int nqubits, int nw, const double *unitary, void *state,
                                int batch, int dtype, void *stream);

/* Mixed-state evolution (Sec. "Quantum Computing with Qubits", Background:
 * rho_n = U_n ... U_1 rho_0 U_1^dagger ... U_n^dagger, with the noise channels
 * of dq_gate_kind applied as Kraus maps) from rho_0 = |0...0><0...0| for
 * every row, then out[row * nobs + o] = sum_k c_k Re Tr(P_k rho_row).
 * rho is kept vectorised row-major -- entry (i, j) of row r at
 * r * 4^n + i * 2^n + j -- so that it is a 2n-qubit "state" whose first n
 * wires carry i and last n wires carry j: a gate U on wire q becomes U on wire
 * q and conj(U) on wire q + n, and a channel on wire q a non-unitary map on
 * the pair (q, q + n) (lowered to two-qubit products of kernel gates and one
 * non-unitary one-qubit matrix).  The fused and plain paths then run it like
 * a 2n-qubit circuit.  nqubits <= 17.  params/data as in dq_apply_circuit
 * (shared parameters only).  expect_out: device FP64 batch * nobs, or NULL.
 * rho_out: device, batch * 4^n amplitudes of `dtype` (16-byte aligned), or
 * NULL (then context-owned device memory holds rho).  No gradients. */
/* Workspace bytes dq_density_forward needs for this circuit, batch and
 * dtype under the context's current path (the vectorised matrices
 * themselves are rho_out or context-owned). */
DQ_API dq_status dq_density_workspace_bytes(dq_ctx *ctx, const dq_circuit *circuit, int batch, int dtype,
                                            size_t *out);
DQ_API dq_status dq_density_forward(dq_ctx *ctx, const dq_circuit *circuit, const double *params,
                                    const double *data, const dq_observables *obs, int batch, int dtype,
                                    double *expect_out, void *rho_out, void *stream);

/* Gradient of L = sum_row sum_o w[row, o] Re Tr(O_o rho_row) for a density
 * circuit (gates and noise channels, as in dq_density_forward) with respect
 * to the shared trainable parameters.  The adjoint sweep of the pure-state
 * path does not apply (channels have no inverse), so every angle occurrence
 * is differentiated by exact shift rules on the expectation itself: the
 * expectation is a trigonometric polynomial in each gate angle whatever the
 * channels around the gate, with the frequencies of the pure case (two-term
 * rule for eigenvalue gap 1, four-term rule for the controlled rotations).
 * All shifted points times the data rows run as one batch of per-row
 * parameters through the density path, chunked so that their vectorised
 * matrices fit in max_bytes (0: a quarter of the free device memory).
 *   expect_out: device FP64 batch * nobs (the unshifted expectations) or NULL.
 *   grad_params: device FP64 nparams or NULL.  row_weights as in
 *   dq_adjoint_grad.  Encoded inputs are held fixed.  Scratch lives in
 *   context-owned device memory. */
DQ_API dq_status dq_density_grad(dq_ctx *ctx, const dq_circuit *circuit, const double *params,
                                 const double *data, const dq_observables *obs, const double *row_weights,
                                 int batch, int dtype, size_t max_bytes, double *expect_out,
                                 double *grad_params, void *stream);

/* Hessian of L = sum_row sum_o w[row, o] <psi_row| O_o |psi_row> with respect
 * to the shared trainable parameters (the second derivatives of the paper's
 * gradient-and-Hessian benchmark, Sec. "Benchmarks").  Every angle slot of a
 * gate with a trainable parameter is an occurrence; row v of the occurrence
 * Hessian comes from adjoint gradients at shifted angles -- the two-term rule
 * [g(t + pi/2) - g(t - pi/2)] / 2 for generators with eigenvalue gap 1 (RX RY
 * RZ P CP RXX RYY RZZ and the three angles of U3) and the four-term rule for
 * the controlled rotations CRX CRY CRZ -- and parameters used by several
 * gates sum their occurrences.  Both rules are exact, so the result equals
 * the analytic Hessian up to rounding.  All shifted points (times the data
 * rows) run as one batch through the fused forward + adjoint path with
 * per-row parameters, in chunks of occurrences whose shifted rows' states
 * (psi and lambda per row on the tiled path) fit in max_bytes (0: a quarter
 * of the free device memory); a chunk holds at least one occurrence.
 *   params: device FP64, nparams (shared).  data: device FP64 batch *
 *   nfeatures or NULL (encoded inputs are held fixed).  row_weights: device
 *   FP64 batch * nobs or NULL (ones).  batch >= 1 (1 without data).
 *   hess: device FP64 nparams x nparams, row p = d/dtheta_p of the gradient
 *   (symmetric up to rounding), overwritten.  grad: device FP64 nparams (the
 *   gradient at params) or NULL.
 * The row tables and per-row gradients live in context-owned device memory
 * (freed by dq_ctx_destroy); the fused path's scratch is the workspace. */
DQ_API dq_status dq_hessian(dq_ctx *ctx, const dq_circuit *circuit, const double *params,
                            const double *data, const dq_observables *obs, const double *row_weights,
                            int batch, int dtype, size_t max_bytes, double *hess, double *grad,
                            void *stream);

/* Shot sampling (API Overview: measure(shots, wires) -- outcomes drawn with
 * the Born probabilities |psi_i|^2 of the current state).  For row r and shot
 * s, with u = the uniform of that shot in [0, 1), the outcome is the smallest
 * basis index i with u * Z < p_0 + ... + p_i, p_i = |psi_r[i]|^2 and Z the
 * row's total probability (inversion of the cumulative distribution; Z
 * absorbs the rounding of the norm).  Outcomes of zero probability are never
 * drawn.  A target within rounding of a cumulative boundary may select either
 * neighbour; both are valid outcomes for it.
 *   state:     device, batch rows of 2^nqubits amplitudes of `dtype`, read only.
 *   uniforms:  device FP64, batch * shots values in [0, 1), row-major; or
 *              NULL, in which case shot k = r * shots + s uses output k of the
 *              splitmix64 stream seeded with `seed` (Steele, Lea & Flood,
 *              OOPSLA 2014), mapped to [0, 1) by its top 53 bits.
 *   wire_mask: 0 for the full basis index; otherwise bit q selects wire q and
 *              the outcome packs the selected wires' bits, the lowest selected
 *              wire in the most significant position (the marginal outcome of
 *              those wires).  Bits at or above nqubits are invalid.
 *   out:       device int64, batch * shots outcomes.
 * Uses sample_workspace_bytes of workspace (dq_sample_workspace_bytes); the
 * state is streamed once, then each shot reads 2^5 amplitudes and a few
 * partial sums.  A row of zeros returns 2^nqubits - 1.  For complex64 states
 * a uniform below 2^-126 (or negative) acts as 0 and one of 1 or more (or
 * NaN) as 1. */
DQ_API dq_status dq_sample_workspace_bytes(dq_ctx *ctx, int nqubits, int batch, size_t *out);
DQ_API dq_status dq_sample(dq_ctx *ctx, int nqubits, const void *state, int batch, int dtype,
                           int64_t shots, const double *uniforms, uint64_t seed,
                           uint64_t wire_mask, int64_t *out, void *stream);

/* Time the fused-path variants (fusion width k and tile schedule; the
 * interpreting against the specialised tile passes; for rows of up to 16
 * qubits, the interpreting against the specialised whole-row kernel; dense
 * blocks against tile passes) for this circuit shape on `state` (device,
 * batch rows, contents destroyed) and cache the fastest for later calls with
 * the same circuit structure.  With graphs on (dq_ctx_set_graphs) the
 * specialised tile passes are timed as CUDA-graph replays, the way the
 * context then runs repeated calls; call dq_ctx_set_graphs first.  They are
 * timed from a cleared L2 (a temporary 256 MiB buffer is filled before each
 * timed forward).
 * Synchronises `stream`. */
DQ_API dq_status dq_plan_autotune(dq_ctx *ctx, const dq_circuit *circuit, int batch,
                           int dtype, void *state, void *stream);

/* The fused forward configuration dq_plan_autotune chose for this circuit
 * structure and dtype: tile qubits *k, always-resident low bits *low and
 * register bits per thread *M (all 0 when the circuit was not tuned and the
 * size-based default applies). */
DQ_API dq_status dq_plan_tuned(dq_ctx *ctx, const dq_circuit *circuit, int dtype, int *k, int *low, int *M);

/* Pin the fused forward configuration of this circuit structure and dtype
 * without timing anything (a shape measured before, on this or another run):
 * tile qubits k, always-resident low bits low, register bits per thread M
 * (the ranges dq_tile_schedule takes; 2^(k - M) threads at most 512, 256
 * for wide register sets), and jit 1 for run-time specialised passes under
 * DQ_OPT_JIT = 2 (0: interpreted).  Later forward calls use it as they use a
 * dq_plan_autotune result; the whole-row and dense-block choices of the plan
 * are kept.  DQ_ERR_INVALID_ARG for values out of range; DQ_ERR_UNSUPPORTED
 * when no tile schedule of that shape exists for the circuit.  Captured
 * graphs of the context are dropped. */
DQ_API dq_status dq_plan_set_tile(dq_ctx *ctx, const dq_circuit *circuit, int dtype, int k, int low, int M,
                                  int jit);

/* ---- host-side plan inspection (no context, no GPU) ----------------------
 * These calls run only the host code that the compute calls run before any
 * launch -- argument validation, lowering to kernel-level gates, the tile
 * planner and the shift-rule tables -- and touch no device, so a caller can
 * see what a circuit becomes without a GPU.  They take no context: failures
 * return a status only (no message). */

/* One kernel-level operation of a lowered circuit.
 *   kind:  a kernel-level dq_gate_kind (H X Y Z S RX RY RZ P CNOT CZ CP SWAP
 *          CRX CRY CRZ), or DQ_LOWERED_BLOCK / DQ_LOWERED_CBLOCK for the
 *          fixed 2x2 matrix `block` (not unitary in the channels of density
 *          circuits), uncontrolled or applied to wires[1] when wires[0] is |1>.
 *   wires: one-wire ops use wires[0] (wires[1] = -1); controlled ops are
 *          (control, target); SWAP is the pair.  Density circuits number the
 *          2n wires of the vectorised rho (wire q + n carries column bit q).
 *   param_idx, data_idx, angle: the angle source as in dq_gate; U3's three
 *          angles become the ops P(lam), RY(theta), P(phi), applied in that
 *          order, with param_idx (or data_idx) + 2, + 0, + 1.
 *   conj:  1 when the op's matrix is replaced by its complex conjugate (the
 *          column-wire copy of a gate in a density circuit).
 *   block: DQ_LOWERED_BLOCK / CBLOCK only: row-major 2x2 as (re, im) pairs. */
#define DQ_LOWERED_BLOCK 64
#define DQ_LOWERED_CBLOCK 65
typedef struct dq_lowered_op {
    int32_t kind;
    int32_t wires[2];
    int32_t param_idx;
    int32_t data_idx;
    int32_t conj;
    double angle;
    double block[8];
} dq_lowered_op;      /* 96 bytes */

/* Validate `circuit` exactly as the compute calls do and lower it: pure
 * circuits (density = 0) to the ops that dq_apply_circuit runs, density
 * circuits (density = 1, noise channels allowed, nqubits <= 17) to the ops
 * that dq_density_forward runs on the 2n-qubit vectorised rho.  The composite
 * gates become exact products (the product of the ops, first op applied
 * first, equals the circuit's operator; for a density circuit it equals the
 * superoperator on row-major vec(rho)).  *count receives the number of ops.
 * ops may be NULL (count only); otherwise it holds `capacity` entries and a
 * capacity below *count returns DQ_ERR_INVALID_ARG with nothing written. */
DQ_API dq_status dq_lower_circuit(const dq_circuit *circuit, int density, dq_lowered_op *ops, int capacity,
                                  int *count);

/* The fused-path tile schedule of the pure circuit's lowered ops (numbered as
 * by dq_lower_circuit) for tile qubits k, always-resident low bits `low` and
 * register bits per thread M: forward passes (adjoint = 0) or the passes of
 * the adjoint sweep (adjoint = 1).  Pass p acts on tiles of the amplitude
 * bits set in tile_bits[p] (bit b = wire nqubits-1-b) and runs the entries
 * order[pass_start[p] .. pass_start[p+1]) in its execution order (the
 * planner regroups commuting ops to save register-layout changes); the
 * adjoint sweep un-applies the passes and their entries last to first.
 * Entry i names a lowered op, with op_flags[i] (may be NULL): bit 0 when the
 * op is one of a CNOT-diagonal-CNOT triple run as one parity-diagonal op
 * (listed as its three ops; it needs no tile bit); bit 1 when the entry is
 * one of the three CNOTs that a SWAP of wires a < b runs as -- the first and
 * third with control b and target a, the second with control a and target
 * b.  So there are at most three entries per op.  Every array holds
 * `capacity` entries (pass_start one more); too few return
 * DQ_ERR_INVALID_ARG.  Returns DQ_ERR_UNSUPPORTED when no schedule exists
 * for these values (for instance k > nqubits), the number of passes in
 * *npasses otherwise. */
DQ_API dq_status dq_tile_schedule(const dq_circuit *circuit, int dtype, int k, int low, int M, int adjoint,
                                  int capacity, int32_t *order, int32_t *pass_start, uint64_t *tile_bits,
                                  int32_t *op_flags, int *npasses);

/* Host-only (no context, no device): the source of a run-time specialised
 * program (DQ_OPT_JIT).  kind 0: the forward passes, kind 1: the reverse-sweep
 * passes of the tile schedule (k, low, M) that dq_tile_schedule describes --
 * one op runner and one kernel per pass; kind 2: the whole-row kernel of the
 * program dq_row_program describes for M register bits (0: the kernel's own
 * choice; k and low are ignored) -- one kernel.  buf (may be NULL) receives
 * the NUL-terminated text when cap exceeds its length; *len receives the
 * length.  DQ_ERR_INVALID_ARG for another kind; DQ_ERR_UNSUPPORTED when no
 * schedule or row program exists for the shape.  No counterpart in the paper
 * (an implementation choice of this library). */
DQ_API dq_status dq_jit_source(const dq_circuit *circuit, int dtype, int k, int low, int M, int kind,
                               char *buf, size_t cap, size_t *len);

/* Host-only: compile that source with NVRTC for compute capability cc (103
 * for sm_103a) without loading it.  DQ_OK when it compiles; DQ_ERR_CUDA with
 * the compiler log in `log` (cap bytes) when it does not;
 * DQ_ERR_UNSUPPORTED when NVRTC cannot be opened. */
DQ_API dq_status dq_jit_compile_check(const dq_circuit *circuit, int dtype, int k, int low, int M,
                                      int kind, int cc, char *log, size_t cap);

/* The program of the whole-row kernel (the fused path for rows of up to 16
 * qubits held on chip) for the pure circuit's lowered ops: M register bits
 * per thread (0: the kernel's own choice for this size and dtype, written to
 * *M_used).  The entries order[0 .. *count) and op_flags are as in
 * dq_tile_schedule for a single pass: the forward sweep runs them first to
 * last, the adjoint sweep last to first.  Returns DQ_ERR_UNSUPPORTED when the
 * rows do not fit the kernel. */
DQ_API dq_status dq_row_program(const dq_circuit *circuit, int dtype, int M, int capacity, int32_t *order,
                                int32_t *op_flags, int *count, int *M_used);

/* The shift rules that dq_hessian and dq_density_grad apply.  Occurrence v
 * (each angle of each gate with a trainable parameter, in gate order; U3
 * gives three, theta phi lam) belongs to parameter occ_param[v], and
 * d f / d t_v = sum_{j in [row0[v], row0[v+1])} weight[j] f(t_v + shift[j])
 * for every f trigonometric in that angle (two rows for eigenvalue gap 1,
 * four for CRX CRY CRZ).  occ_param and row0 hold cap_occ entries (row0 one
 * more), shift and weight cap_rows; *nocc and *nrows receive the counts, and
 * too small a capacity returns DQ_ERR_INVALID_ARG with nothing written (NULL
 * arrays: counts only). */
DQ_API dq_status dq_shift_rules(const dq_circuit *circuit, int cap_occ, int cap_rows, int32_t *occ_param,
                                int32_t *row0, double *shift, double *weight, int *nocc, int *nrows);

#ifdef __cplusplus
}
#endif

#endif /* DQ_H_INCLUDED */
