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
#include <cstdlib>
#include <vector>

#include "dq_common.cuh"
#include "dq_engine.cuh"
#include "dq_plan.h"
#include "dq_rows.h"

namespace dq {

void RowProgram::release() {
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

struct RowArgs {
    const EOp *fops;
    const EOp *rops;
    const ESeg *fsegs;
    const ESeg *rsegs;
    int nops, nfseg, nrseg;
    const void *coef;
    int n;
    int batch;
    int nrseg_run;          // reverse segments to run (later ones only un-apply gradient-free gates)
    const void *state_in;
    void *state_out;
    int forward;
    const DevTerm *terms;   // wire-space masks
    int nterms, nobs;
    const double *row_weights;
    double *expect_out;
    int grad;
    int nacc_shared, nacc_row, nfeat, nparams, ppr;
    double *grad_params, *grad_data, *part;
};

__device__ __forceinline__ uint64_t wire_bits(uint64_t m, int n) { return m ? (__brevll(m) >> (64 - n)) : 0; }

// Threads per CTA are 2^(n - M): narrow register sets (at most 64 bytes of
// amplitudes per vector and thread) may use 512 threads.
template <typename R, int M>
constexpr int rows_max_threads() { return ((1 << M) * (int)sizeof(cx<R>) <= 64) ? 512 : 256; }

template <typename R, int M, bool PD>
__global__ void __launch_bounds__(rows_max_threads<R, M>(), sizeof(R) == 4 ? 2 : 1) k_rows(RowArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int n = a.n;
    const int64_t dim = int64_t(1) << n;
    cx<R> *bufP = reinterpret_cast<cx<R> *>(smem);
    cx<R> *bufL = bufP + dim;
    unsigned char *q = smem + (a.grad ? 2 : 1) * dim * sizeof(cx<R>);
    EOp *sops = reinterpret_cast<EOp *>(q);          // forward decodings
    EOp *srops = sops + a.nops;                        // reverse decodings
    ESeg *sf = reinterpret_cast<ESeg *>(srops + a.nops);
    ESeg *sr = sf + a.nfseg;
    Mat2<R> *scoef = reinterpret_cast<Mat2<R> *>(sr + a.nrseg);
    const int nacc = a.nacc_shared + a.nacc_row;
    double *acc = reinterpret_cast<double *>(scoef + a.nops);     // [nacc] FP64 per CTA
    double *expw = acc + nacc;                                     // [nw][nobs]
    R *accw = reinterpret_cast<R *>(expw + (size_t)nw * a.nobs);   // [nw][nacc] per-row partials (state precision)
    const Mat2<R> *gcoef = reinterpret_cast<const Mat2<R> *>(a.coef);
    for (int i = tid; i < a.nops; i += blockDim.x) {
        sops[i] = a.fops[i];
        srops[i] = a.rops[i];
        scoef[i] = gcoef[sops[i].coef];
    }
    for (int i = tid; i < a.nfseg; i += blockDim.x) sf[i] = a.fsegs[i];
    for (int i = tid; i < a.nrseg; i += blockDim.x) sr[i] = a.rsegs[i];
    for (int i = tid; i < nacc + nw * a.nobs; i += blockDim.x) acc[i] = 0.0;
    for (int i = tid; i < nw * nacc; i += blockDim.x) accw[i] = R(0);
    __syncthreads();

    cx<R> ps[1 << M], ls[1 << M];
    // ops whose coefficients depend on the row (per-row parameters, encoded
    // features) have their block refreshed in the shared table for every row,
    // so every op reads its coefficients from shared memory
    bool any_row = false;
    for (int i = 0; i < a.nops; ++i) any_row |= sops[i].rowstep != 0;
    for (int row = blockIdx.x; row < a.batch; row += gridDim.x) {
        if (any_row) {
            for (int i = tid; i < a.nops; i += blockDim.x)
                if (sops[i].rowstep) scoef[i] = gcoef[sops[i].coef + (int64_t)row * sops[i].rowstep];
            __syncthreads();
        }
        // ---- state preparation ------------------------------------------------
        Layout L = make_layout(sf[0], M, n, lane, warp);
        if (a.state_in) {
            const cx<R> *gi = reinterpret_cast<const cx<R> *>(a.state_in) + row * dim;
#pragma unroll
            for (int e = 0; e < (1 << M); ++e) ps[e] = gi[L.tb | reg_off<M>(L, e)];
        } else {
#pragma unroll
            for (int e = 0; e < (1 << M); ++e)
                ps[e] = mk<R>((L.tb | reg_off<M>(L, e)) == 0 ? R(1) : R(0), R(0));
        }
        // ---- forward ----------------------------------------------------------
        if (a.forward) {
            for (int s = 0; s < a.nfseg; ++s) {
                const ESeg sg = sf[s];
                if (s > 0) {
                    eng_store<R, M>(ps, bufP, L);
                    __syncthreads();
                    L = make_layout(sg, M, n, lane, warp);
                    eng_load<R, M>(ps, bufP, L);
                }
                for (int oi = sg.op0; oi < sg.op0 + sg.nops; ++oi) {
                    const EOp o = sops[oi];
                    const Mat2<R> u = scoef[oi];
                    eng_apply<R, M, PD>(ps, o, u, 0, L, lane);
                }
            }
        }
        __syncthreads();   // every thread has finished reading this row's input
        if (a.state_out) {
            cx<R> *go = reinterpret_cast<cx<R> *>(a.state_out) + row * dim;
#pragma unroll
            for (int e = 0; e < (1 << M); ++e) go[L.tb | reg_off<M>(L, e)] = ps[e];
        }
        const bool need_smem_state = a.nterms > 0 || a.grad;
        if (need_smem_state) {
            eng_store<R, M>(ps, bufP, L);
            __syncthreads();
            // expectations: thread partial in the state precision, FP32 warp
            // sum, FP64 per warp
            for (int k = 0; k < a.nterms; ++k) {
                const DevTerm t = a.terms[k];
                const uint64_t f = wire_bits(t.f, n), sm = wire_bits(t.s, n);
                R v = R(0);
                if (f == 0) {
                    for (int64_t b = tid; b < dim; b += blockDim.x) {
                        const cx<R> x = bufP[b];
                        const R pr = x.x * x.x + x.y * x.y;
                        v += parity64((uint64_t)b & sm) ? -pr : pr;
                    }
                } else {
                    for (int64_t b = tid; b < dim; b += blockDim.x) {
                        const cx<R> x = bufP[b], y = bufP[b ^ f];
                        const R re = re_conj_mul(y, x), im = im_conj_mul(y, x);
                        const int ph = (t.nY + 2 * parity64((uint64_t)b & sm)) & 3;
                        v += (ph == 0) ? re : (ph == 1 ? -im : (ph == 2 ? -re : im));
                    }
                }
                v = warp_sum_t(v);
                if (lane == 0) expw[warp * a.nobs + t.obs] += t.coeff * (double)v;
            }
            __syncthreads();
            if (tid < a.nobs) {
                double s = 0.0;
                for (int w = 0; w < nw; ++w) {
                    s += expw[w * a.nobs + tid];
                    expw[w * a.nobs + tid] = 0.0;
                }
                if (a.expect_out) a.expect_out[(int64_t)row * a.nobs + tid] = s;
            }
        }
        if (!a.grad) {
            __syncthreads();
            continue;
        }
        // ---- lambda = sum_o w_o O_o psi in the first reverse layout ------------
        L = make_layout(sr[0], M, n, lane, warp);
        eng_load<R, M>(ps, bufP, L);
        const double *w = a.row_weights ? a.row_weights + (int64_t)row * a.nobs : nullptr;
#pragma unroll
        for (int e = 0; e < (1 << M); ++e) {
            const uint64_t l = L.tb | reg_off<M>(L, e);
            R lx = R(0), ly = R(0);
            for (int k = 0; k < a.nterms; ++k) {
                const DevTerm t = a.terms[k];
                const uint64_t f = wire_bits(t.f, n), sm = wire_bits(t.s, n);
                const uint64_t src = l ^ f;
                float pr, pi;
                pauli_phase(src, sm, t.nY, pr, pi);
                const R wt = (R)((w ? w[t.obs] : 1.0) * t.coeff);
                const cx<R> x = bufP[src];
                lx += wt * ((R)pr * x.x - (R)pi * x.y);
                ly += wt * ((R)pr * x.y + (R)pi * x.x);
            }
            ls[e] = mk<R>(lx, ly);
        }
        __syncthreads();   // bufP is rewritten by the first layout change
        // ---- reverse sweep -----------------------------------------------------
        for (int s = 0; s < a.nrseg_run; ++s) {
            const ESeg sg = sr[s];
            if (s > 0) {
                eng_store<R, M>(ps, bufP, L);
                eng_store<R, M>(ls, bufL, L);
                __syncthreads();
                L = make_layout(sg, M, n, lane, warp);
                eng_load<R, M>(ps, bufP, L);
                eng_load<R, M>(ls, bufL, L);
            }
            // segment ops run from sg.op0 downwards
            for (int c = 0; c < sg.nops; ++c) {
                const int oi = sg.op0 - c;
                const EOp o = srops[oi];
                const Mat2<R> u = scoef[oi];
                if (o.pad[1]) {   // rotation pair: this DIAG op, then the REAL op before it
                    const EOp o2 = srops[oi - 1];
                    const Mat2<R> u2 = scoef[oi - 1];
                    R gd, gr;
                    eng_adjoint_pair<R, M>(ps, ls, o, dagger(u), o2, dagger(u2), lane, gd, gr);
                    if (o.slot >= 0) {
                        const R gs = warp_sum_t(gd);
                        if (lane == 0) accw[warp * nacc + o.slot] += gs;
                    }
                    if (o2.slot >= 0) {
                        const R gs = warp_sum_t(gr);
                        if (lane == 0) accw[warp * nacc + o2.slot] += gs;
                    }
                    ++c;
                    continue;
                }
                const R g = eng_adjoint<R, M, PD>(ps, ls, o, dagger(u), 0, L, lane);
                if (o.slot >= 0) {
                    // this row's partial over the warp's amplitude pairs
                    const R gs = warp_sum_t(g);
                    if (lane == 0) accw[warp * nacc + o.slot] += gs;
                }
            }
        }
        __syncthreads();
        // fold this row's warp partials into FP64: shared parameters
        // accumulate over the CTA's rows, per-row outputs are written out
        for (int i = tid; i < a.nacc_shared; i += blockDim.x) {
            double s = 0.0;
            for (int ww = 0; ww < nw; ++ww) {
                s += (double)accw[ww * nacc + i];
                accw[ww * nacc + i] = R(0);
            }
            acc[i] += s;
        }
        for (int i = tid; i < a.nacc_row; i += blockDim.x) {
            double s = 0.0;
            for (int ww = 0; ww < nw; ++ww) {
                s += (double)accw[ww * nacc + a.nacc_shared + i];
                accw[ww * nacc + a.nacc_shared + i] = R(0);
            }
            if (i < a.nfeat) {
                if (a.grad_data) a.grad_data[(int64_t)row * a.nfeat + i] = s;
            } else if (a.grad_params) {
                a.grad_params[(int64_t)row * a.nparams + (i - a.nfeat)] = s;
            }
        }
        __syncthreads();
    }
    if (a.grad && a.nacc_shared && a.part)
        for (int i = tid; i < a.nacc_shared; i += blockDim.x) a.part[(int64_t)blockIdx.x * a.nacc_shared + i] = acc[i];
}

__global__ void k_rows_part_reduce(const double *__restrict__ part, int nblk, int np, double *__restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * np + p];
    out[p] = s;
}

}  // namespace

size_t rows_smem_bytes(const RowProgram &rp, int amp, bool grad, int nobs, int threads) {
    const int nw = threads / 32;
    const size_t matb = amp == 8 ? sizeof(Mat2<float>) : sizeof(Mat2<double>);
    return (size_t)(grad ? 2 : 1) * ((size_t)amp << rp.n) + 2 * rp.fops.size() * sizeof(EOp) +
           (rp.fsegs.size() + rp.rsegs.size()) * sizeof(ESeg) + rp.fops.size() * matb +
           (size_t)(rp.nacc_shared + rp.nacc_row + nw * nobs) * sizeof(double) +
           (size_t)nw * (rp.nacc_shared + rp.nacc_row) * (amp == 8 ? sizeof(float) : sizeof(double)) + 64;
}

size_t rows_part_bytes(const Plan &p, int nsm) {
    return (size_t)std::max(1, p.ppr ? 0 : p.nparams) * (size_t)nsm * 4 * sizeof(double);
}

template <typename R>
cudaError_t rows_launch(const RowProgram &rp, const Plan &p, const void *coef, const void *state_in, int forward,
                        const DevTerm *d_wterms, int nterms, int nobs, const double *row_weights, int batch,
                        void *state_out, double *expect_out, double *grad_params, double *grad_data, double *part,
                        int nsm, size_t smem_optin, cudaStream_t s, int64_t *launches) {
    const bool grad = grad_params || grad_data;
    const int threads = 1 << (rp.n - rp.M);
    const size_t smem = rows_smem_bytes(rp, (int)sizeof(cx<R>), grad, nobs, threads);
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
    const void *kfn = nullptr;
    const bool pd = rp.pdiag;
    switch (rp.M) {
    case 2: kfn = pd ? (const void *)k_rows<R, 2, true> : (const void *)k_rows<R, 2, false>; break;
    case 3: kfn = pd ? (const void *)k_rows<R, 3, true> : (const void *)k_rows<R, 3, false>; break;
    default: kfn = pd ? (const void *)k_rows<R, Mmax, true> : (const void *)k_rows<R, Mmax, false>; break;
    }
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int grid = std::max(1, std::min(batch, std::min(per_sm, 4) * nsm));
    {
        LaunchScope ls(s, "k_rows", launches);
        switch (rp.M * 2 + (pd ? 1 : 0)) {
        case 4: k_rows<R, 2, false><<<grid, threads, smem, s>>>(a); break;
        case 5: k_rows<R, 2, true><<<grid, threads, smem, s>>>(a); break;
        case 6: k_rows<R, 3, false><<<grid, threads, smem, s>>>(a); break;
        case 7: k_rows<R, 3, true><<<grid, threads, smem, s>>>(a); break;
        default:
            if (pd) k_rows<R, Mmax, true><<<grid, threads, smem, s>>>(a);
            else k_rows<R, Mmax, false><<<grid, threads, smem, s>>>(a);
            break;
        }
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
                                        double *, double *, double *, int, size_t, cudaStream_t, int64_t *);
DQ_INST(float)
DQ_INST(double)
#undef DQ_INST

}  // namespace dq
