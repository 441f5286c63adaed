// Whole-row kernel body (internal): one CTA holds a whole row in registers;
// state preparation, forward ops, Pauli-sum expectations, lambda and the
// reverse sweep with gradient partials.  Shared by the library's kernel,
// which interprets the row program from shared memory, and the run-time
// specialised kernels, which have the program's ops compiled in.
#pragma once

#include "dq_devterm.h"
#include "dq_engine.cuh"

namespace dq {
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

// The interpreter: forward and reverse segments dispatched from the staged
// program.  L is the current register layout (updated at layout changes).
struct InterpRows {
    template <typename R, int M, bool PD>
    __device__ __forceinline__ static void fwd(cx<R> (&ps)[1 << M], cx<R> *bufP, Layout &L, const ESeg *sf,
                                               const EOp *sops, const Mat2<R> *scoef, int nfseg, int n, int lane,
                                               int warp) {
            for (int s = 0; s < nfseg; ++s) {
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
    template <typename R, int M, bool PD>
    __device__ __forceinline__ static void rev(cx<R> (&ps)[1 << M], cx<R> (&ls)[1 << M], cx<R> *bufP, cx<R> *bufL,
                                               Layout &L, const ESeg *sr, const EOp *srops, const Mat2<R> *scoef,
                                               R *accw, int nacc, int nrun, int n, int lane, int warp) {
        for (int s = 0; s < nrun; ++s) {
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
    }
};

// RPC rows per CTA: the CTA's warps split into RPC halves, half h holding
// row rbase + h with its own state buffers and coefficient table.  Every half
// runs the same instructions (the same program, the same barriers), so the
// SM's schedulers fetch one instruction stream for RPC rows; a half without a
// row (the batch's ragged end) computes on zeros and writes nothing.
template <typename R, int M, bool PD, typename Runner, int RPC = 1>
__device__ __forceinline__ void rows_body(const RowArgs &a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int hthreads = blockDim.x / RPC, nwh = nw / RPC;
    const int half = RPC == 1 ? 0 : warp / nwh;
    const int hwarp = RPC == 1 ? warp : warp % nwh;
    const int htid = RPC == 1 ? tid : tid % hthreads;
    const int n = a.n;
    const int64_t dim = int64_t(1) << n;
    const int nbuf = a.grad ? 2 : 1;
    cx<R> *bufP = reinterpret_cast<cx<R> *>(smem) + (int64_t)half * nbuf * dim;
    cx<R> *bufL = bufP + dim;
    unsigned char *q = smem + (size_t)RPC * nbuf * dim * sizeof(cx<R>);
    EOp *sops = reinterpret_cast<EOp *>(q);          // forward decodings
    EOp *srops = sops + a.nops;                        // reverse decodings
    ESeg *sf = reinterpret_cast<ESeg *>(srops + a.nops);
    ESeg *sr = sf + a.nfseg;
    Mat2<R> *scoef_all = reinterpret_cast<Mat2<R> *>(sr + a.nrseg);   // [RPC][nops]
    Mat2<R> *scoef = scoef_all + (size_t)half * a.nops;
    const int nacc = a.nacc_shared + a.nacc_row;
    double *acc = reinterpret_cast<double *>(scoef_all + (size_t)RPC * a.nops);   // [nacc] FP64 per CTA
    double *expw = acc + nacc;                                     // [nw][nobs]
    R *accw = reinterpret_cast<R *>(expw + (size_t)nw * a.nobs);   // [nw][nacc] per-row partials (state precision)
    R *accwh = accw + (size_t)half * nwh * nacc;                   // this half's warps
    const Mat2<R> *gcoef = reinterpret_cast<const Mat2<R> *>(a.coef);
    for (int i = tid; i < a.nops; i += blockDim.x) {
        sops[i] = a.fops[i];
        srops[i] = a.rops[i];
        for (int h = 0; h < RPC; ++h) scoef_all[(size_t)h * a.nops + i] = gcoef[a.fops[i].coef];
    }
    for (int i = tid; i < a.nfseg; i += blockDim.x) sf[i] = a.fsegs[i];
    for (int i = tid; i < a.nrseg; i += blockDim.x) sr[i] = a.rsegs[i];
    for (int i = tid; i < nacc + nw * a.nobs; i += blockDim.x) acc[i] = 0.0;
    for (int i = tid; i < nw * nacc; i += blockDim.x) accw[i] = R(0);
    __syncthreads();

    cx<R> ps[1 << M], ls[1 << M];
    // ops whose coefficients depend on the row (per-row parameters, encoded
    // features) have their block refreshed in the half's table for every row,
    // so every op reads its coefficients from shared memory
    bool any_row = false;
    for (int i = 0; i < a.nops; ++i) any_row |= sops[i].rowstep != 0;
    for (int64_t rbase = (int64_t)blockIdx.x * RPC; rbase < a.batch; rbase += (int64_t)gridDim.x * RPC) {
        const int64_t row = rbase + half;
        const bool valid = row < a.batch;
        const int64_t crow = valid ? row : rbase;   // a row that exists, for the half without one
        if (any_row) {
            for (int i = htid; i < a.nops; i += hthreads)
                if (sops[i].rowstep) scoef[i] = gcoef[sops[i].coef + crow * sops[i].rowstep];
            __syncthreads();
        }
        // ---- state preparation ------------------------------------------------
        Layout L = make_layout(sf[0], M, n, lane, hwarp);
        if (a.state_in) {
            const cx<R> *gi = reinterpret_cast<const cx<R> *>(a.state_in) + crow * dim;
#pragma unroll
            for (int e = 0; e < (1 << M); ++e) {
                const uint32_t i = L.tb | reg_off<M>(L, e);
                ps[e] = (valid && DQ_INB(i, dim)) ? gi[i] : mk<R>(R(0), R(0));
            }
        } else {
#pragma unroll
            for (int e = 0; e < (1 << M); ++e)
                ps[e] = mk<R>((L.tb | reg_off<M>(L, e)) == 0 ? R(1) : R(0), R(0));
        }
        // ---- forward ----------------------------------------------------------
        if (a.forward) Runner::template fwd<R, M, PD>(ps, bufP, L, sf, sops, scoef, a.nfseg, n, lane, hwarp);
        __syncthreads();   // every thread has finished reading this row's input
        if (a.state_out && valid) {
            cx<R> *go = reinterpret_cast<cx<R> *>(a.state_out) + row * dim;
#pragma unroll
            for (int e = 0; e < (1 << M); ++e) {
                const uint32_t i = L.tb | reg_off<M>(L, e);
                if (DQ_INB(i, dim)) go[i] = ps[e];
            }
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
                    for (int64_t b = htid; b < dim; b += hthreads) {
                        const cx<R> x = bufP[b];
                        const R pr = x.x * x.x + x.y * x.y;
                        v += parity64((uint64_t)b & sm) ? -pr : pr;
                    }
                } else {
                    for (int64_t b = htid; b < dim; b += hthreads) {
                        if (!DQ_INB(b ^ f, dim)) continue;
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
            if (htid < a.nobs) {
                double s = 0.0;
                for (int w = half * nwh; w < (half + 1) * nwh; ++w) {
                    s += expw[w * a.nobs + htid];
                    expw[w * a.nobs + htid] = 0.0;
                }
                if (a.expect_out && valid) a.expect_out[row * a.nobs + htid] = s;
            }
        }
        if (!a.grad) {
            __syncthreads();
            continue;
        }
        // ---- lambda = sum_o w_o O_o psi in the first reverse layout ------------
        L = make_layout(sr[0], M, n, lane, hwarp);
        eng_load<R, M>(ps, bufP, L);
        const double *w = a.row_weights ? a.row_weights + crow * a.nobs : nullptr;
#pragma unroll
        for (int e = 0; e < (1 << M); ++e) {
            const uint64_t l = L.tb | reg_off<M>(L, e);
            R lx = R(0), ly = R(0);
            for (int k = 0; k < a.nterms; ++k) {
                const DevTerm t = a.terms[k];
                const uint64_t f = wire_bits(t.f, n), sm = wire_bits(t.s, n);
                const uint64_t src = l ^ f;
                if (!DQ_INB(src, dim)) continue;
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
        Runner::template rev<R, M, PD>(ps, ls, bufP, bufL, L, sr, srops, scoef, accwh, nacc, a.nrseg_run, n, lane,
                                       hwarp);
        __syncthreads();
        // fold the rows' warp partials into FP64: shared parameters
        // accumulate over the CTA's rows (halves with a row), per-row outputs
        // are written out
        for (int i = tid; i < a.nacc_shared; i += blockDim.x) {
            double s = 0.0;
            for (int ww = 0; ww < nw; ++ww) {
                if (rbase + ww / nwh < a.batch) s += (double)accw[ww * nacc + i];
                accw[ww * nacc + i] = R(0);
            }
            acc[i] += s;
        }
        for (int i = htid; i < a.nacc_row; i += hthreads) {
            double s = 0.0;
            for (int ww = 0; ww < nwh; ++ww) {
                s += (double)accwh[ww * nacc + a.nacc_shared + i];
                accwh[ww * nacc + a.nacc_shared + i] = R(0);
            }
            if (!valid) continue;
            if (i < a.nfeat) {
                if (a.grad_data) a.grad_data[row * a.nfeat + i] = s;
            } else if (a.grad_params) {
                a.grad_params[row * a.nparams + (i - a.nfeat)] = s;
            }
        }
        __syncthreads();
    }
    if (a.grad && a.nacc_shared && a.part)
        for (int i = tid; i < a.nacc_shared; i += blockDim.x) a.part[(int64_t)blockIdx.x * a.nacc_shared + i] = acc[i];
}

}  // namespace
}  // namespace dq
