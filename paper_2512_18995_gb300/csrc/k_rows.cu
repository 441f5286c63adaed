// Fused small-state path on the in-register engine: one CTA holds a whole
// row (state, and adjoint vector when gradients are requested) in registers.
//
// Per row: state preparation |0...0> (or a given state), every gate of the
// circuit (Sec. "Quantum Computing with Qubits": U_n ... U_1 |psi_0>), the
// Pauli-sum expectations (API Overview: expectation()), lambda = sum_o w_o
// O_o psi, and the adjoint reverse sweep (Sec. "Distributed Simulations":
// adjoint differentiation) accumulating 2 Im <lambda|G_j|psi> per parametric
// gate while un-applying U_j^dagger from both register sets.  Shared memory
// is used only to change register layouts and to read partner amplitudes of
// Pauli terms.  Gradient partials are summed per warp in FP32 (32 lanes x a
// few pairs) and accumulated per warp in FP64; shared-parameter sums are
// written per CTA to a [grid][nparams] array and reduced by a second kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <cstdlib>
#include <vector>

#include "dq_common.cuh"
#include "dq_engine.cuh"
#include "dq_jit.h"
#include "dq_plan.h"
#include "dq_rows.h"
#include "dq_rows_body.cuh"

namespace dq {

void RowProgram::release() {
    for (JitModule *&m : jit) {
        if (!m) continue;
        m->release();
        delete m;
        m = nullptr;
    }
    cudaFree(d_fops);
    cudaFree(d_rops);
    cudaFree(d_fsegs);
    cudaFree(d_rsegs);
    d_fops = d_rops = nullptr;
    d_fsegs = nullptr;
    d_rsegs = nullptr;
}

namespace {

// Greedy register layouts over ops visited in `order`; every op is decoded
// against the layout of the segment it falls in (into dec[op index]).
void build_segments(const std::vector<GOp> &ops, const std::vector<int> &order, int M, int k,
                    std::vector<ESeg> &segs, std::vector<EOp> &dec) {
    dec.assign(ops.size(), EOp{});
    std::vector<int> B;
    int first = order.empty() ? 0 : order[0];
    int count = 0;
    size_t start = 0;
    auto close = [&](size_t end) {
        ESeg sg{};
        sg.op0 = first;
        sg.nops = count;
        std::vector<int> full = B;
        for (int j = kLaneBits; j < k && (int)full.size() < M; ++j)
            if (std::find(full.begin(), full.end(), j) == full.end()) full.push_back(j);
        for (int i = 0; i < 8; ++i) sg.B[i] = i < M ? (int8_t)full[i] : (int8_t)-1;
        for (size_t x = start; x < end; ++x) dec[order[x]] = decode_op(ops[order[x]], sg.B, M);
        segs.push_back(sg);
    };
    for (size_t idx = 0; idx < order.size(); ++idx) {
        const GOp &o = ops[order[idx]];
        const int need = (!cls_diagonal(o.cls) && o.tl >= kLaneBits) ? o.tl : -1;
        if (need >= 0 && std::find(B.begin(), B.end(), need) == B.end()) {
            if ((int)B.size() < M) {
                B.push_back(need);
            } else {
                close(idx);
                B.assign(1, need);
                first = order[idx];
                count = 0;
                start = idx;
            }
        }
        ++count;
    }
    close(order.size());
}

}  // namespace

// Register bits per thread for an n-qubit row.  The widest set that fits
// (4 for complex64, 3 for complex128) with 256 threads, or 3 / 2 with 512
// threads; rows whose set would exceed 512 threads use another path.  The
// environment variable DQ_ROWS_M overrides the choice (tuning experiments).
int rows_pick_M(int n, int amp_bytes) {
    const int mwide = amp_bytes == 8 ? 4 : 3;
    int m = std::min(mwide, n - kLaneBits);
    if (n - m > 8) m = mwide - 1;                 // narrower set, up to 512 threads
    if (const char *env = getenv("DQ_ROWS_M")) {
        const int v = atoi(env);
        if (v >= 2 && v <= mwide) m = v;
    }
    m = std::min(m, n - kLaneBits);
    if (m < 2) return 0;
    const int maxt = ((1 << m) * amp_bytes <= 64) ? 512 : 256;
    if ((1 << (n - m)) > maxt) return 0;
    return m;
}

bool rows_build_program(const Plan &p, int M, RowProgram &out) {
    const int n = p.n;
    if (M < 2 || n < kLaneBits + M || n > 16) return false;
    out = RowProgram();
    out.n = n;
    out.M = M;
    out.nacc_shared = p.ppr ? 0 : p.nparams;
    out.nacc_row = p.nfeat + (p.ppr ? p.nparams : 0);
    auto acc_of = [&](const DevGate &g) -> int {
        if (g.gkind == 1) return g.gout;
        if (g.gkind == 3) return out.nacc_shared + g.gout;
        if (g.gkind == 2) return out.nacc_shared + p.nfeat + g.gout;
        return -1;
    };
    std::vector<GOp> ops;
    for (int gi = 0; gi < p.ngates; ++gi) {
        const DevGate &g = p.gates[gi];
        if (gi + 2 < p.ngates && parity_triple(g, p.gates[gi + 1], p.gates[gi + 2])) {
            // CNOT, diagonal, CNOT: one parity-diagonal op with the diagonal's slot
            const DevGate &d = p.gates[gi + 1];
            GOp o{};
            o.gi = gi;
            o.cls = CLS_PDIAG;
            o.tl = o.tg = g.t;
            o.cl = o.cg = g.c;
            o.kind = d.kind;
            o.coef = d.coef;
            o.rowstep = d.rowstep;
            o.slot = acc_of(d);
            ops.push_back(o);
            out.pdiag = true;
            gi += 2;
            continue;
        }
        auto push = [&](int cls, int t, int c, int slot) {
            GOp o{};
            o.gi = gi;
            o.cls = cls;
            o.tl = t;
            o.tg = t;
            o.cl = c;
            o.cg = c;
            o.kind = g.kind;
            o.coef = g.coef;
            o.rowstep = g.rowstep;
            o.slot = slot;
            ops.push_back(o);
        };
        if (g.cls == CLS_SWAP) {
            push(CLS_ANTI, g.c, g.t, -1);
            push(CLS_ANTI, g.t, g.c, -1);
            push(CLS_ANTI, g.c, g.t, -1);
        } else {
            push(g.cls, g.t, g.c, acc_of(g));
        }
    }
    schedule_for_layouts(ops, M, kLaneBits);
    const std::vector<char> head = pair_real_diag(ops);
    record_order(ops, p.gates, out.gates, out.flags);
    std::vector<int> fwd(ops.size()), rev(ops.size());
    for (size_t i = 0; i < ops.size(); ++i) {
        fwd[i] = (int)i;
        rev[i] = (int)(ops.size() - 1 - i);
    }
    build_segments(ops, fwd, M, n, out.fsegs, out.fops);
    build_segments(ops, rev, M, n, out.rsegs, out.rops);
    // rotation pairs whose two ops share a reverse layout run as one op there
    // (forward, the folded product costs as much as the two ops)
    std::vector<int> rseg(ops.size(), -1);
    for (size_t s = 0; s < out.rsegs.size(); ++s)
        for (int i = out.rsegs[s].op0; i > out.rsegs[s].op0 - out.rsegs[s].nops; --i) rseg[i] = (int)s;
    for (size_t i = 0; i + 1 < ops.size(); ++i) {
        if (!head[i]) continue;
        if (rseg[i] == rseg[i + 1] && pair_handlers_match(out.rops[i], out.rops[i + 1])) out.rops[i + 1].pad[1] = 1;
    }
    return true;
}

namespace {

template <typename R, int M, bool PD, int RPC>
__global__ void __launch_bounds__(rows_max_threads<R, M>() * RPC, (sizeof(R) == 4 && RPC == 1) ? 2 : 1)
k_rows(RowArgs a) {
    rows_body<R, M, PD, InterpRows, RPC>(a);
}

__global__ void k_rows_part_reduce(const double *__restrict__ part, int nblk, int np, double *__restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * np + p];
    out[p] = s;
}

}  // namespace

size_t rows_smem_bytes(const RowProgram &rp, int amp, bool grad, int nobs, int threads, int rpc) {
    const int nw = threads / 32;
    const size_t matb = amp == 8 ? sizeof(Mat2<float>) : sizeof(Mat2<double>);
    return (size_t)rpc * (grad ? 2 : 1) * ((size_t)amp << rp.n) + 2 * rp.fops.size() * sizeof(EOp) +
           (rp.fsegs.size() + rp.rsegs.size()) * sizeof(ESeg) + (size_t)rpc * rp.fops.size() * matb +
           (size_t)(rp.nacc_shared + rp.nacc_row + nw * nobs) * sizeof(double) +
           (size_t)nw * (rp.nacc_shared + rp.nacc_row) * (amp == 8 ? sizeof(float) : sizeof(double)) + 64;
}

int rows_pick_rpc(const RowProgram &rp, int amp, bool grad, int nobs, int batch, int nsm, size_t smem_optin,
                  int want) {
    const int threads = 1 << (rp.n - rp.M);
    const int maxt = ((1 << rp.M) * amp <= 64) ? 512 : 256;
    const bool two_fit = 2 * threads <= 2 * maxt && 2 * threads <= 1024 &&
                         rows_smem_bytes(rp, amp, grad, nobs, 2 * threads, 2) <= smem_optin;
    if (want == 1 || !two_fit || amp != 8) return 1;   // complex64 only: two complex128 rows spill
    if (want == 2) return 2;
    // automatic: two rows per CTA for rows of at most 128 threads when the
    // batch still gives every SM four rows -- measured on 4096-row batches:
    // 10 qubits (64 threads a row) 1.19 -> 0.87 ms specialised, 1.23 -> 1.03 ms
    // interpreted; 12 qubits (256 threads) 2.70 -> 2.81 ms specialised
    return (batch >= 4 * nsm && threads <= 128) ? 2 : 1;
}

size_t rows_part_bytes(const Plan &p, int nsm) {
    return (size_t)std::max(1, p.ppr ? 0 : p.nparams) * (size_t)nsm * 4 * sizeof(double);
}

template <typename R>
cudaError_t rows_launch(const RowProgram &rp, const Plan &p, const void *coef, const void *state_in, int forward,
                        const DevTerm *d_wterms, int nterms, int nobs, const double *row_weights, int batch,
                        void *state_out, double *expect_out, double *grad_params, double *grad_data, double *part,
                        int nsm, size_t smem_optin, cudaStream_t s, int64_t *launches, bool jit, int rpc) {
    const bool grad = grad_params || grad_data;
    if (rpc != 1 && rpc != 2) return cudaErrorInvalidValue;
    JitModule *jm = rp.jit[rpc - 1];
    jit = jit && jm && !jm->kernels.empty();
    const int threads = rpc << (rp.n - rp.M);
    const size_t smem = rows_smem_bytes(rp, (int)sizeof(cx<R>), grad, nobs, threads, rpc);
    if (smem > smem_optin) return cudaErrorInvalidValue;
    RowArgs a;
    a.fops = rp.d_fops;
    a.rops = rp.d_rops;
    a.fsegs = rp.d_fsegs;
    a.rsegs = rp.d_rsegs;
    a.nops = (int)rp.fops.size();
    a.nfseg = (int)rp.fsegs.size();
    a.nrseg = (int)rp.rsegs.size();
    a.coef = coef;
    a.n = rp.n;
    a.batch = batch;
    a.state_in = state_in;
    a.state_out = state_out;
    a.forward = forward;
    a.terms = d_wterms;
    a.nterms = nterms;
    a.nobs = std::max(1, nobs);
    a.row_weights = row_weights;
    a.expect_out = expect_out;
    a.grad = grad ? 1 : 0;
    a.nacc_shared = rp.nacc_shared;
    a.nacc_row = rp.nacc_row;
    a.nfeat = p.nfeat;
    a.nparams = p.nparams;
    a.ppr = p.ppr;
    a.grad_params = grad_params;
    a.grad_data = grad_data;
    a.part = part;
    // reverse segments run from the last op down; stop after the one holding
    // the first op whose gradient is requested
    a.nrseg_run = 0;
    if (grad) {
        int first = (int)rp.fops.size();
        for (int i = 0; i < (int)rp.fops.size(); ++i) {
            const int acc = rp.fops[i].slot;
            if (acc < 0) continue;
            const bool data = acc >= rp.nacc_shared && acc < rp.nacc_shared + p.nfeat;
            const bool params = !data;
            if ((data && grad_data) || (params && grad_params)) {
                first = i;
                break;
            }
        }
        for (int sg = 0; sg < (int)rp.rsegs.size(); ++sg) {
            a.nrseg_run = sg + 1;
            if (rp.rsegs[sg].op0 - rp.rsegs[sg].nops + 1 <= first) break;
        }
    }
    constexpr int Mmax = sizeof(R) == 4 ? 4 : 3;
    const bool pd = rp.pdiag;
    auto pick = [&](auto rpc_tag) -> const void * {
        constexpr int C = decltype(rpc_tag)::value;
        switch (rp.M) {
        case 2: return pd ? (const void *)k_rows<R, 2, true, C> : (const void *)k_rows<R, 2, false, C>;
        case 3: return pd ? (const void *)k_rows<R, 3, true, C> : (const void *)k_rows<R, 3, false, C>;
        default: return pd ? (const void *)k_rows<R, Mmax, true, C> : (const void *)k_rows<R, Mmax, false, C>;
        }
    };
    // two rows per CTA for complex64 only (complex128 rows would not keep their registers)
    const void *kfn = pick(std::integral_constant<int, 1>());
    if constexpr (sizeof(R) == 4) {
        if (rpc == 2) kfn = pick(std::integral_constant<int, 2>());
    } else {
        if (rpc == 2) return cudaErrorInvalidValue;
    }
    if (jit) kfn = (const void *)jm->kernels[0];
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int grid = std::max(1, std::min((batch + rpc - 1) / rpc, std::min(per_sm, 4) * nsm));
    if (jit) {
        LaunchScope ls(s, "k_rows_jit", launches);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3((unsigned)threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        void *args[] = {(void *)&a};
        e = cudaLaunchKernelExC(&cfg, kfn, args);
        if (e != cudaSuccess) return e;
    } else {
        LaunchScope ls(s, "k_rows", launches);
        void *args[] = {(void *)&a};
        e = cudaLaunchKernel(kfn, dim3((unsigned)grid), dim3((unsigned)threads), args, smem, s);
        if (e != cudaSuccess) return e;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (grad && grad_params && !p.ppr && p.nparams > 0) {
        LaunchScope ls(s, "k_rows_part_reduce", launches);
        k_rows_part_reduce<<<(p.nparams + 127) / 128, 128, 0, s>>>(part, grid, p.nparams, grad_params);
        e = cudaGetLastError();
    }
    return e;
}

#define DQ_INST(R)                                                                                          \
    template cudaError_t rows_launch<R>(const RowProgram &, const Plan &, const void *, const void *, int,  \
                                        const DevTerm *, int, int, const double *, int, void *, double *,   \
                                        double *, double *, double *, int, size_t, cudaStream_t, int64_t *, bool, \
                                        int);
DQ_INST(float)
DQ_INST(double)
#undef DQ_INST

}  // namespace dq
