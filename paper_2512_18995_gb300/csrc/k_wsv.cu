// Fused small-state path: a whole row (state and adjoint vector) lives in
// on-chip memory for the entire circuit.
//
// One CTA takes one row at a time and runs, without touching HBM except for
// inputs and outputs: state preparation |0...0>, every gate of the circuit
// (Sec. "Quantum Computing with Qubits", evolution U_n ... U_1 |psi_0>), the
// Pauli-sum expectations (API Overview: expectation()), and the adjoint
// reverse sweep (Sec. "Distributed Simulations": adjoint differentiation),
// which accumulates 2 Im <lambda| G_j |psi> for every parametric gate j while
// un-applying U_j^dagger from both vectors.
//
// k_wsv: a uniform batch (one circuit, many rows: encoded inputs, shared or
// per-row parameters).  Shared-parameter gradients are summed per CTA in
// FP64 and written to a [grid][nparams] scratch array, then reduced in a
// second, deterministic kernel.
//
// k_batch: an uneven batch of independent circuits in one persistent launch.
// CTAs take circuits from an atomic ticket counter in longest-first order;
// circuits whose two vectors fit in the CTA's shared memory run there, larger
// ones run on a per-CTA scratch slice of global memory, taken only by as many
// CTAs as keep the scratch in flight within a budget that fits in L2.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "dq_common.cuh"
#include "dq_plan.h"

namespace dq {

namespace {

constexpr int kMaxThreads = 512;

// Wire-space mask -> bit-space mask for an n-qubit row (wire q -> bit n-1-q).
__device__ __forceinline__ uint64_t wires_to_bits(uint64_t m, int n) {
    return m ? (__brevll(m) >> (64 - n)) : 0;
}

// Apply gate (or its inverse) to vector v of 2^n amplitudes (shared or global).
template <typename R>
__device__ __forceinline__ void vec_gate(cx<R> *v, int n, const DevGate &g, const Mat2<R> &u) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if (g.cls == CLS_SWAP) {
        const int64_t items = int64_t(1) << (n - 2);
        const uint64_t ba = uint64_t(1) << g.t, bb = uint64_t(1) << g.c;
        for (int64_t j = tid; j < items; j += nt) {
            const uint64_t i = insert0x2((uint64_t)j, g.t, g.c) | ba;
            const uint64_t k = i ^ ba ^ bb;
            const cx<R> x = v[i];
            v[i] = v[k];
            v[k] = x;
        }
        return;
    }
    const uint64_t tb = uint64_t(1) << g.t;
    if (g.c >= 0) {
        const int lo = min(g.t, g.c), hi = max(g.t, g.c);
        const uint64_t cb = uint64_t(1) << g.c;
        const int64_t items = int64_t(1) << (n - 2);
        for (int64_t j = tid; j < items; j += nt) {
            const uint64_t i0 = insert0x2((uint64_t)j, lo, hi) | cb;
            cx<R> a0 = v[i0], a1 = v[i0 | tb];
            apply2_rt<R>(g.cls, u, a0, a1);
            v[i0] = a0;
            v[i0 | tb] = a1;
        }
    } else {
        const int64_t items = int64_t(1) << (n - 1);
        for (int64_t j = tid; j < items; j += nt) {
            const uint64_t i0 = insert0((uint64_t)j, g.t);
            cx<R> a0 = v[i0], a1 = v[i0 | tb];
            apply2_rt<R>(g.cls, u, a0, a1);
            v[i0] = a0;
            v[i0 | tb] = a1;
        }
    }
}

// Reverse step on (psi, lam): returns this thread's FP32 partial of
// 2 Im <lam|G|psi> (0 when !grad), then un-applies U^dagger on both.
template <typename R>
__device__ __forceinline__ R vec_adj(cx<R> *psi, cx<R> *lam, int n, const DevGate &g, const Mat2<R> &ud,
                                     bool grad) {
    const int tid = threadIdx.x, nt = blockDim.x;
    R acc = R(0);
    if (g.cls == CLS_SWAP) {
        const int64_t items = int64_t(1) << (n - 2);
        const uint64_t ba = uint64_t(1) << g.t, bb = uint64_t(1) << g.c;
        for (int64_t j = tid; j < items; j += nt) {
            const uint64_t i = insert0x2((uint64_t)j, g.t, g.c) | ba;
            const uint64_t k = i ^ ba ^ bb;
            cx<R> x = psi[i]; psi[i] = psi[k]; psi[k] = x;
            x = lam[i]; lam[i] = lam[k]; lam[k] = x;
        }
        return acc;
    }
    const uint64_t tb = uint64_t(1) << g.t;
    const bool ctl = g.c >= 0;
    const int lo = ctl ? min(g.t, g.c) : g.t, hi = ctl ? max(g.t, g.c) : 0;
    const uint64_t cb = ctl ? (uint64_t(1) << g.c) : 0;
    const int64_t items = int64_t(1) << (n - (ctl ? 2 : 1));
    for (int64_t j = tid; j < items; j += nt) {
        const uint64_t i0 = (ctl ? insert0x2((uint64_t)j, lo, hi) : insert0((uint64_t)j, lo)) | cb;
        cx<R> p0 = psi[i0], p1 = psi[i0 | tb], l0 = lam[i0], l1 = lam[i0 | tb];
        if (grad) acc += grad_pair<R>(g.kind, l0, l1, p0, p1);
        apply2_rt<R>(g.cls, ud, p0, p1);
        apply2_rt<R>(g.cls, ud, l0, l1);
        psi[i0] = p0; psi[i0 | tb] = p1;
        lam[i0] = l0; lam[i0 | tb] = l1;
    }
    return acc;
}

// Thread-partial of <psi|P|psi> for one term (wire-space masks converted).
template <typename R>
__device__ __forceinline__ R vec_term(const cx<R> *psi, int n, uint64_t f, uint64_t s, int nY) {
    const int tid = threadIdx.x, nt = blockDim.x;
    R acc = R(0);
    if (f == 0) {
        const int64_t items = int64_t(1) << n;
        for (int64_t b = tid; b < items; b += nt) {
            const cx<R> x = psi[b];
            const R p = x.x * x.x + x.y * x.y;
            acc += parity64((uint64_t)b & s) ? -p : p;
        }
    } else {
        const int lf = __ffsll((long long)f) - 1;
        const int64_t items = int64_t(1) << (n - 1);
        for (int64_t j = tid; j < items; j += nt) {
            const uint64_t b = insert0((uint64_t)j, lf);
            const cx<R> x = psi[b], y = psi[b ^ f];
            const R re = re_conj_mul(y, x), im = im_conj_mul(y, x);
            const int ph = (nY + 2 * parity64(b & s)) & 3;
            const R v = (ph == 0) ? re : (ph == 1 ? -im : (ph == 2 ? -re : im));
            acc += R(2) * v;
        }
    }
    return acc;
}

// Block reduction helper with double-buffered slots: every thread calls it
// with its partial; after the following __syncthreads thread 0 may read
// red[buf][0..nwarps).
__device__ __forceinline__ void warp_partial(double v, double *red, int buf) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[buf * 32 + (threadIdx.x >> 5)] = v;
}
__device__ __forceinline__ double sum_partials(const double *red, int buf) {
    double s = 0.0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) s += red[buf * 32 + i];
    return s;
}

struct RowIO {
    const double *w;        // row weights (nobs) or null
    double *exp_out;        // nobs or null
    void *state_out;        // 2^n amplitudes or null
    const void *state_in;   // initial state (2^n amplitudes) or null for |0...0>
    bool forward;           // apply the gates
};

// Full hot path for one row on vectors psi/lam (shared or global memory).
// acc: gradient accumulators indexed by DevGate::gout + (gkind offsets).
template <typename R>
__device__ void run_row(cx<R> *psi, cx<R> *lam, int n, const DevGate *__restrict__ gates, int ngates,
                        const Mat2<R> *__restrict__ coef, int row, bool grad,
                        const DevTerm *__restrict__ terms, int nterms, int nobs, RowIO io,
                        double *acc_shared, double *acc_row, int nfeat, double *red, double *exp_acc) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t dim = int64_t(1) << n;
    // initial state: given, or |0...0>
    if (io.state_in) {
        const cx<R> *si = (const cx<R> *)io.state_in;
        for (int64_t i = tid; i < dim; i += nt) psi[i] = si[i];
    } else {
        for (int64_t i = tid; i < dim; i += nt) psi[i] = mk<R>(i == 0 ? R(1) : R(0), R(0));
    }
    if (tid < nobs) exp_acc[tid] = 0.0;
    __syncthreads();
    // forward
    for (int gi = 0; io.forward && gi < ngates; ++gi) {
        const DevGate g = gates[gi];
        const Mat2<R> u = coef[g.coef + row * g.rowstep];
        vec_gate<R>(psi, n, g, u);
        __syncthreads();
    }
    if (io.state_out) {
        cx<R> *so = (cx<R> *)io.state_out;
        __syncthreads();   // state_out may alias state_in
        for (int64_t i = tid; i < dim; i += nt) so[i] = psi[i];
    }
    // expectations
    for (int k = 0; k < nterms; ++k) {
        const DevTerm t = terms[k];
        const R v = vec_term<R>(psi, n, wires_to_bits(t.f, n), wires_to_bits(t.s, n), t.nY);
        warp_partial((double)v, red, k & 1);
        __syncthreads();
        if (tid == 0) exp_acc[t.obs] += t.coeff * sum_partials(red, k & 1);
    }
    __syncthreads();
    if (io.exp_out && tid < nobs) io.exp_out[tid] = exp_acc[tid];
    if (!grad) {
        __syncthreads();
        return;
    }
    // lambda = sum_o w_o O_o psi
    for (int64_t b = tid; b < dim; b += nt) {
        R lx = R(0), ly = R(0);
        for (int k = 0; k < nterms; ++k) {
            const DevTerm t = terms[k];
            const uint64_t f = wires_to_bits(t.f, n), s = wires_to_bits(t.s, n);
            const uint64_t src = (uint64_t)b ^ f;
            float pr, pi;
            pauli_phase(src, s, t.nY, pr, pi);
            const R wt = (R)((io.w ? io.w[t.obs] : 1.0) * t.coeff);
            const cx<R> x = psi[src];
            lx += wt * ((R)pr * x.x - (R)pi * x.y);
            ly += wt * ((R)pr * x.y + (R)pi * x.x);
        }
        lam[b] = mk<R>(lx, ly);
    }
    __syncthreads();
    // reverse sweep
    for (int gi = ngates - 1; gi >= 0; --gi) {
        const DevGate g = gates[gi];
        const Mat2<R> ud = dagger(coef[g.coef + row * g.rowstep]);
        const bool gg = g.gkind != 0;
        const R part = vec_adj<R>(psi, lam, n, g, ud, gg);
        if (gg) warp_partial((double)part, red, gi & 1);
        __syncthreads();
        if (gg && tid == 0) {
            const double s = sum_partials(red, gi & 1);
            if (g.gkind == 1) acc_shared[g.gout] += s;
            else if (g.gkind == 2) acc_row[nfeat + g.gout] += s;
            else acc_row[g.gout] += s;
        }
    }
    __syncthreads();
}

struct WsvArgs {
    const void *state_in;   // null: start from |0...0>
    int forward;
    const DevGate *gates;
    int ngates;
    int n;
    const void *coef;
    const DevTerm *terms;   // wire-space masks
    int nterms;
    int nobs;
    const double *row_weights;
    int batch;
    void *state_out;
    double *expect_out;
    double *grad_params;
    double *grad_data;
    double *part;           // [gridDim.x][nparams] shared-param partials
    int nparams;
    int nfeat;
    int ppr;
    int grad;
};

template <typename R>
__global__ void __launch_bounds__(kMaxThreads) k_wsv(WsvArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int64_t dim = int64_t(1) << a.n;
    cx<R> *psi = reinterpret_cast<cx<R> *>(smem);
    cx<R> *lam = psi + dim;
    double *dbl = reinterpret_cast<double *>(psi + (a.grad ? 2 : 1) * dim);
    const int nshared = a.ppr ? 0 : a.nparams;
    const int nrow = a.nfeat + (a.ppr ? a.nparams : 0);
    double *acc_shared = dbl;
    double *acc_row = acc_shared + nshared;
    double *exp_acc = acc_row + nrow;
    double *red = exp_acc + a.nobs;           // 2 x 32
    const int tid = threadIdx.x;
    for (int i = tid; i < nshared + nrow; i += blockDim.x) dbl[i] = 0.0;
    __syncthreads();
    const Mat2<R> *coef = (const Mat2<R> *)a.coef;
    for (int row = blockIdx.x; row < a.batch; row += gridDim.x) {
        RowIO io;
        io.w = a.row_weights ? a.row_weights + (int64_t)row * a.nobs : nullptr;
        io.exp_out = a.expect_out ? a.expect_out + (int64_t)row * a.nobs : nullptr;
        io.state_out = a.state_out ? (void *)((cx<R> *)a.state_out + row * dim) : nullptr;
        io.state_in = a.state_in ? (const void *)((const cx<R> *)a.state_in + row * dim) : nullptr;
        io.forward = a.forward != 0;
        run_row<R>(psi, lam, a.n, a.gates, a.ngates, coef, row, a.grad != 0, a.terms, a.nterms, a.nobs,
                   io, acc_shared, acc_row, a.nfeat, red, exp_acc);
        if (a.grad && nrow) {
            for (int i = tid; i < nrow; i += blockDim.x) {
                if (i < a.nfeat) {
                    if (a.grad_data) a.grad_data[(int64_t)row * a.nfeat + i] = acc_row[i];
                } else if (a.grad_params) {
                    a.grad_params[(int64_t)row * a.nparams + (i - a.nfeat)] = acc_row[i];
                }
                acc_row[i] = 0.0;
            }
            __syncthreads();
        }
    }
    if (a.grad && nshared && a.part)
        for (int i = tid; i < nshared; i += blockDim.x) a.part[(int64_t)blockIdx.x * nshared + i] = acc_shared[i];
}

// out[p] = sum_b part[b][p] in a fixed order.
__global__ void k_part_reduce(const double *__restrict__ part, int nblk, int np, double *__restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * np + p];
    out[p] = s;
}

// --------------------------------------------------------------------------
// uneven batch
// --------------------------------------------------------------------------
struct BatchArgs {
    const BatchCirc *circ;
    int ncirc;
    const int32_t *order;
    const DevGate *gates;
    const void *coef;
    const DevTerm *terms;   // wire-space
    int nterms;
    int nobs;
    int nsmem;              // circuits with n <= nsmem run in shared memory
    int nmax;
    int maxparams;
    double *expect_out;
    double *grad_params;
    void *scratch;          // [lcap][2 * 2^nmax] amplitudes
    int lcap;               // CTAs that take circuits larger than nsmem (their scratch fits in L2)
    int *counter;           // [2]: tickets of the scratch queue and of the shared-memory queue
};

template <typename R>
__global__ void __launch_bounds__(kMaxThreads) k_batch(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int64_t sdim = int64_t(1) << a.nsmem;
    cx<R> *spsi = reinterpret_cast<cx<R> *>(smem);
    cx<R> *slam = spsi + sdim;
    double *acc = reinterpret_cast<double *>(slam + sdim);
    double *exp_acc = acc + a.maxparams;
    double *red = exp_acc + a.nobs;
    int *ticket = reinterpret_cast<int *>(red + 64);
    const int tid = threadIdx.x;
    const int64_t gdim = int64_t(1) << a.nmax;
    cx<R> *gpsi = (cx<R> *)a.scratch + (int64_t)blockIdx.x * 2 * gdim;
    cx<R> *glam = gpsi + gdim;
    const Mat2<R> *coef = (const Mat2<R> *)a.coef;
    // Two queues over the same longest-first order: circuits larger than
    // nsmem (scratch in global memory) go only to the first lcap CTAs, so that
    // the scratch in use stays L2-resident; those CTAs then join the others on
    // the shared-memory circuits.  A queue's ticket that lands on the other
    // kind of circuit is skipped, so every circuit runs once.
    int queue = blockIdx.x < a.lcap ? 0 : 1;   // thread 0's
    for (;;) {
        if (tid == 0) {
            int c = -1;
            for (;;) {
                const int idx = atomicAdd(&a.counter[queue], 1);
                if (idx >= a.ncirc) {
                    if (queue == 0) {
                        queue = 1;
                        continue;
                    }
                    break;
                }
                const int cand = a.order[idx];
                if ((a.circ[cand].n > a.nsmem) == (queue == 0)) {
                    c = cand;
                    break;
                }
            }
            *ticket = c;
        }
        __syncthreads();
        const int c = *ticket;
        __syncthreads();
        if (c < 0) break;
        const BatchCirc bc = a.circ[c];
        for (int i = tid; i < bc.nparams; i += blockDim.x) acc[i] = 0.0;
        __syncthreads();
        const bool on_chip = bc.n <= a.nsmem;
        RowIO io;
        io.w = nullptr;
        io.exp_out = a.expect_out ? a.expect_out + (int64_t)c * a.nobs : nullptr;
        io.state_out = nullptr;
        io.state_in = nullptr;
        io.forward = true;
        const bool grad = a.grad_params != nullptr;
        run_row<R>(on_chip ? spsi : gpsi, on_chip ? slam : glam, bc.n, a.gates + bc.gate0, bc.ngates, coef,
                   0, grad, a.terms, a.nterms, a.nobs, io, acc, acc, 0, red, exp_acc);
        if (grad)
            for (int i = tid; i < bc.nparams; i += blockDim.x) a.grad_params[bc.param0 + i] = acc[i];
        __syncthreads();
    }
}

inline int threads_for(int n) {
    int t = 1 << std::max(0, n - 2);
    return std::min(kMaxThreads, std::max(64, t));
}

}  // namespace

size_t wsv_smem_bytes(int n, int amp_bytes, bool grad, int ndouble) {
    return (size_t)(grad ? 2 : 1) * ((size_t)amp_bytes << n) + (size_t)(ndouble + 64) * sizeof(double);
}

bool wsv_supported(int n, int amp_bytes, bool grad, size_t smem_optin, int ndouble) {
    if (n < 1 || n > 16) return false;
    return wsv_smem_bytes(n, amp_bytes, grad, ndouble) <= smem_optin;
}

static int wsv_grid(const void *kernel, int threads, size_t smem, int batch, int nsm) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return std::max(1, std::min(batch, per_sm * nsm));
}

size_t wsv_part_bytes(const Plan &p, int nsm) {
    return (size_t)std::max(1, p.ppr ? 0 : p.nparams) * (size_t)nsm * 8 * sizeof(double);
}

// Real entry (terms already on the device).
template <typename R>
cudaError_t wsv_launch(const Plan &p, const void *coef, const void *state_in, int forward,
                       const DevTerm *d_wterms, int nterms, int nobs,
                       const double *row_weights, int batch, void *state_out, double *expect_out,
                       double *grad_params, double *grad_data, double *part, int nsm, cudaStream_t s,
                       int64_t *launches) {
    const bool grad = grad_params || grad_data;
    WsvArgs a;
    a.state_in = state_in;
    a.forward = forward;
    a.gates = p.d_gates;
    a.ngates = p.ngates;
    a.n = p.n;
    a.coef = coef;
    a.terms = d_wterms;
    a.nterms = nterms;
    a.nobs = nobs;
    a.row_weights = row_weights;
    a.batch = batch;
    a.state_out = state_out;
    a.expect_out = expect_out;
    a.grad_params = grad_params;
    a.grad_data = grad_data;
    a.part = part;
    a.nparams = p.nparams;
    a.nfeat = p.nfeat;
    a.ppr = p.ppr;
    a.grad = grad ? 1 : 0;
    const int nd = (p.ppr ? 0 : p.nparams) + p.nfeat + (p.ppr ? p.nparams : 0) + nobs;
    const size_t smem = wsv_smem_bytes(p.n, (int)sizeof(cx<R>), grad, nd);
    const int threads = threads_for(p.n);
    cudaError_t e = cudaFuncSetAttribute(k_wsv<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int cap = (int)std::min<int64_t>((int64_t)nsm * 8, (int64_t)batch);
    int grid = wsv_grid((const void *)k_wsv<R>, threads, smem, batch, nsm);
    grid = std::min(grid, cap);
    {
        LaunchScope ls(s, "k_wsv", launches);
        k_wsv<R><<<grid, threads, smem, s>>>(a);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (grad && grad_params && !p.ppr && p.nparams > 0) {
        LaunchScope ls(s, "k_part_reduce", launches);
        k_part_reduce<<<(p.nparams + 127) / 128, 128, 0, s>>>(part, grid, p.nparams, grad_params);
        e = cudaGetLastError();
    }
    return e;
}

size_t batch_scratch_bytes(int nmax, int amp_bytes, int nsm, size_t smem_optin) {
    (void)smem_optin;
    return (size_t)nsm * batch_max_per_sm(nmax) * 2 * ((size_t)amp_bytes << nmax);
}

// Defaults of the persistent uneven-batch launch: circuits up to 12 qubits
// (complex64; 11 for complex128) in shared memory, 512 threads per circuit,
// at most four CTAs per SM, 128 MiB of scratch in flight for the larger
// circuits (measured on the 1024-circuit 8..16-qubit batch with these
// defaults: 0 (every CTA) 3.20 ms, 32 MiB 7.08, 64 MiB 3.75, 96 MiB 2.79,
// 128 MiB 2.52, 160 MiB 2.77).
BatchTune batch_default_tune(int amp_bytes) {
    BatchTune t;
    t.nsmem = amp_bytes == 8 ? 12 : 11;
    t.threads = kMaxThreads;
    t.per_sm = 4;
    t.l2_mb = 128;
    return t;
}

template <typename R>
cudaError_t batch_run(const BatchCirc *d_circ, int ncirc, const int32_t *d_order,
                      const DevGate *d_gates, const void *coef, const DevTerm *d_terms, int nterms,
                      int nobs, int nmax, int maxparams, double *expect_out, double *grad_params,
                      void *scratch, int *d_counter, int nsm, size_t smem_optin, const BatchTune &tune,
                      cudaStream_t s, int64_t *launches) {
    if (tune.threads < 64 || tune.threads > kMaxThreads || (tune.threads & (tune.threads - 1)) ||
        tune.per_sm < 1 || tune.per_sm > batch_max_per_sm(nmax) || tune.nsmem < 2 || tune.l2_mb < 0)
        return cudaErrorInvalidValue;
    BatchArgs a;
    a.circ = d_circ;
    a.ncirc = ncirc;
    a.order = d_order;
    a.gates = d_gates;
    a.coef = coef;
    a.terms = d_terms;
    a.nterms = nterms;
    a.nobs = nobs;
    a.nmax = nmax;
    a.maxparams = std::max(1, maxparams);
    a.expect_out = expect_out;
    a.grad_params = grad_params;
    a.scratch = scratch;
    a.counter = d_counter;
    // Shared memory for on-chip circuits: two vectors of 2^nsmem amplitudes.
    int nsmem = std::min(nmax, tune.nsmem);
    while (nsmem > 2 && wsv_smem_bytes(nsmem, (int)sizeof(cx<R>), true, a.maxparams + nobs + 8) > smem_optin) --nsmem;
    a.nsmem = nsmem;
    const size_t smem = wsv_smem_bytes(nsmem, (int)sizeof(cx<R>), true, a.maxparams + nobs + 8);
    const int threads = tune.threads;
    cudaError_t e = cudaFuncSetAttribute(k_batch<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<R>, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    per_sm = std::min(per_sm, tune.per_sm);   // scratch holds kBatchMaxPerSm slices per SM
    const int grid = std::max(1, std::min(ncirc, per_sm * nsm));
    // CTAs allowed on scratch circuits: the budget of tune.l2_mb MiB of
    // scratch (two vectors of 2^nmax amplitudes each), all CTAs when 0
    const size_t slice = 2 * ((size_t)sizeof(cx<R>) << nmax);
    a.lcap = tune.l2_mb > 0 ? (int)std::max<size_t>(1, std::min<size_t>(grid, ((size_t)tune.l2_mb << 20) / slice))
                            : grid;
    e = cudaMemsetAsync(d_counter, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    LaunchScope ls(s, "k_batch", launches);
    k_batch<R><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

#define DQ_INST(R)                                                                                          \
    template cudaError_t wsv_launch<R>(const Plan &, const void *, const void *, int, const DevTerm *, int, int, \
                                       const double *,                                                      \
                                       int, void *, double *, double *, double *, double *, int,             \
                                       cudaStream_t, int64_t *);                                            \
    template cudaError_t batch_run<R>(const BatchCirc *, int, const int32_t *, const DevGate *, const void *, \
                                      const DevTerm *, int, int, int, int, double *, double *, void *, int *, \
                                      int, size_t, const BatchTune &, cudaStream_t, int64_t *);
DQ_INST(float)
DQ_INST(double)
#undef DQ_INST

}  // namespace dq
