// Forward tile pass: the kernel body shared by the library's kernel, which
// interprets each pass's op program from shared memory, and the run-time
// specialised kernels, which have each pass's ops compiled in (internal).
//
// A pass streams tiles of 2^k amplitudes in and out with TMA (two shared
// buffers, mbarrier completion, bounded waits); inside a tile the amplitudes
// live in registers (dq_engine.cuh) and the pass's ops run segment by
// segment, one register layout per segment.  The diagonal observables of a
// circuit's last pass are measured on the finished tiles beside the store.
#pragma once

#include "dq_devterm.h"
#include "dq_engine.cuh"
#include "dq_tma.cuh"

namespace dq {
namespace {

// Diagonal observables measured on the last pass's tiles (Z strings): the
// pass's tile bits map each term's sign mask to tile-local and block parts.
struct TileEpi {
    const DevTerm *terms;   // device, all terms diagonal
    int nterms;
    double *part;           // [term][row][cta]
    int batch;
    int8_t T[16];           // tile bit -> amplitude bit
};

struct TileKArgs {
    const EOp *ops;
    const ESeg *segs;
    int op0, nops, seg0, nseg;
    const void *coef;
    TileGeom g;
    int *errflag;
    int any_row;            // some op's coefficients depend on the batch row
    TileEpi epi;            // epi.nterms == 0: none
};

struct ETerm {
    uint32_t sloc;
    uint32_t pad;
    uint64_t sout;
};

// Threads per CTA are 2^(k - M); wide register sets (256 bytes of amplitudes
// per thread) are limited to 256 threads so that they keep their registers.
template <typename R, int M>
constexpr int tile_max_threads() { return ((1 << M) * (int)sizeof(cx<R>) >= 256) ? 256 : 512; }
// Narrow register sets (<= 64 bytes of amplitudes per thread) are held to 64
// registers, so that four 256-thread tiles fit on an SM.
template <typename R, int M>
constexpr int tile_min_blocks() { return ((1 << M) * (int)sizeof(cx<R>) <= 64) ? 2 : 1; }

// The scheduled ops of one pass on one tile held in shared memory: per
// layout segment, load the register set, run the segment's ops, store back.
template <typename R, int M, bool PD>
__device__ __forceinline__ void tile_run_ops(cx<R> (&r)[1 << M], cx<R> *cur, const EOp *sops, const ESeg *ssegs,
                                             const Mat2<R> *scoef, int nseg, int op0, int k, uint64_t base,
                                             int lane, int warp) {
    for (int si = 0; si < nseg; ++si) {
        const ESeg sg = ssegs[si];
        const Layout L = make_layout(sg, M, k, lane, warp);
        eng_load<R, M>(r, cur, L);
        for (int oi = sg.op0 - op0; oi < sg.op0 - op0 + sg.nops; ++oi) {
            const EOp o = sops[oi];
            if (o.h == H_FAN) {
                oi += eng_fan<R, M>(r, sops + oi, scoef + oi, base, L) - 1;
                continue;
            }
            eng_apply<R, M, PD>(r, o, scoef[oi], base, L, lane);
        }
        // each thread writes back exactly the addresses it read in this
        // layout; the barrier orders them before the next layout's reads
        eng_store<R, M>(r, cur, L);
        __syncthreads();
    }
}

// Diagonal (Z-string) observables of one finished tile: per-warp FP32 sums
// of signed probabilities, folded into the CTA's FP64 accumulators.  The
// CTA has 2^(k-M) threads and thread t reads tile amplitudes t + i 2^(k-M),
// i < 2^M, so the sign of amplitude i under a term with tile-local mask s is
// (-1)^(parity(t & s) + parity(i & (s >> (k-M)))): the thread's signed sum is
// +-W[s >> (k-M)], W the Walsh-Hadamard transform of its 2^M probabilities
// (w_h = sum_i (-1)^popc(i & h) p_i).  The amplitudes are read and squared
// once per tile, however many terms there are.
template <typename R, int M>
__device__ __forceinline__ void tile_epi_accum(const cx<R> *cur, const ETerm *sterm, int nte, double *eacc,
                                               R *eaccw, int k, uint64_t base, int tid, int lane, int warp,
                                               int nw) {
    constexpr int P = 1 << M;
    const int lb = k - M;
    R w[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
        const cx<R> x = cur[tid + (i << lb)];
        w[i] = x.x * x.x + x.y * x.y;
    }
#pragma unroll
    for (int st = 1; st < P; st <<= 1) {
#pragma unroll
        for (int i = 0; i < P; ++i) {
            if (!(i & st)) {
                const R a0 = w[i], a1 = w[i | st];
                w[i] = a0 + a1;
                w[i | st] = a0 - a1;
            }
        }
    }
    for (int j = 0; j < nte; ++j) {
        const ETerm et = sterm[j];
        const int h = (int)(et.sloc >> lb) & (P - 1);
        // w[h] by halving on the bits of h (selects, no indexed registers)
        R v[P];
#pragma unroll
        for (int i = 0; i < P; ++i) v[i] = w[i];
#pragma unroll
        for (int half = P >> 1; half >= 1; half >>= 1) {
#pragma unroll
            for (int i = 0; i < half; ++i) v[i] = (h & half) ? v[i + half] : v[i];
        }
        const int neg = (__popcll(base & et.sout) + __popc((uint32_t)tid & et.sloc)) & 1;
        R e = neg ? -v[0] : v[0];
        e = warp_sum_t(e);
        if (lane == 0) eaccw[warp * nte + j] += e;
    }
    __syncthreads();
    for (int j = tid; j < nte; j += blockDim.x) {
        double sum = 0.0;
        for (int ww = 0; ww < nw; ++ww) {
            sum += (double)eaccw[ww * nte + j];
            eaccw[ww * nte + j] = R(0);
        }
        eacc[j] += sum;
    }
}

// Stage ETerm records of the diagonal observables for a pass whose tile bits
// are T (tile-local sign bits and the sign bits outside the tile).
__device__ __forceinline__ void tile_epi_setup(const TileEpi &epi, int k, ETerm *sterm, double *eacc, int tid) {
    for (int j = tid; j < epi.nterms; j += blockDim.x) {
        const uint64_t sm = epi.terms[j].s;
        ETerm e{};
        uint64_t in = 0;
        for (int i = 0; i < k; ++i)
            if ((sm >> epi.T[i]) & 1) {
                e.sloc |= 1u << i;
                in |= uint64_t(1) << epi.T[i];
            }
        e.sout = sm & ~in;
        sterm[j] = e;
        eacc[j] = 0.0;
    }
}

// The interpreter: every op dispatched from the staged program.
struct InterpOps {
    template <typename R, int M, bool PD>
    __device__ __forceinline__ static void run(cx<R> (&r)[1 << M], cx<R> *cur, const EOp *sops, const ESeg *ssegs,
                                               const Mat2<R> *scoef, int nseg, int op0, int k, uint64_t base,
                                               int lane, int warp) {
        tile_run_ops<R, M, PD>(r, cur, sops, ssegs, scoef, nseg, op0, k, base, lane, warp);
    }
};

// One forward pass (see the file comment).  Ops::run applies the pass's ops
// to one tile in shared memory.
template <typename R, int M, bool PD, typename Ops>
__device__ __forceinline__ void tile_fwd_body(const CUtensorMap &tmap, const TileKArgs &a) {
    extern __shared__ __align__(128) unsigned char smem[];
    if (!DQ_SMEM_ALIGNED(smem)) return;   // bounds-checking build: no copy into a misaligned buffer
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t tbytes = sizeof(cx<R>) << a.g.k;
    const unsigned long long wlim = wait_limit_ns(a.errflag);
    cx<R> *buf0 = reinterpret_cast<cx<R> *>(smem);
    cx<R> *buf1 = reinterpret_cast<cx<R> *>(smem + tbytes);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * tbytes);
    EOp *sops = reinterpret_cast<EOp *>(smem + 2 * tbytes + 64);
    ESeg *ssegs = reinterpret_cast<ESeg *>(sops + a.nops);
    Mat2<R> *scoef = reinterpret_cast<Mat2<R> *>(ssegs + a.nseg);
    const int nte = a.epi.nterms, nw = blockDim.x >> 5;
    ETerm *sterm = reinterpret_cast<ETerm *>(scoef + a.nops);     // [nte]
    double *eacc = reinterpret_cast<double *>(sterm + nte);         // [nte]
    R *eaccw = reinterpret_cast<R *>(eacc + nte);                   // [nw][nte]
    const Mat2<R> *gcoef = reinterpret_cast<const Mat2<R> *>(a.coef);
    const int64_t per = (a.g.ntiles + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * per;
    const int64_t t1 = min(a.g.ntiles, t0 + per);
    int c[5];
    uint64_t base;
    int64_t row;
    // The pass's program (uploaded at planning time) is staged before waiting
    // for the previous kernel of the stream (programmatic dependent launch:
    // this prologue overlaps that kernel's tail); the state and the bound
    // coefficients are read only after the wait.
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_async_smem();
    }
    for (int i = tid; i < a.nops; i += blockDim.x) sops[i] = a.ops[a.op0 + i];
    for (int i = tid; i < a.nseg; i += blockDim.x) ssegs[i] = a.segs[a.seg0 + i];
    grid_dep_wait();
    if (tid == 0 && t0 < t1) {
        geom_coords(a.g, t0, c, base, row);
        mbar_expect_tx(&bar[0], (uint32_t)tbytes);
        tma_load5(buf0, &tmap, c, &bar[0]);
    }
    for (int i = tid; i < a.nops; i += blockDim.x) scoef[i] = gcoef[sops[i].coef];
    tile_epi_setup(a.epi, a.g.k, sterm, eacc, tid);
    for (int i = tid; i < nw * nte; i += blockDim.x) eaccw[i] = R(0);
    __syncthreads();
    if (t0 >= t1) return;
    int64_t erow = -1;
    auto eflush = [&](int64_t rr) {
        for (int j = tid; j < nte; j += blockDim.x) {
            a.epi.part[((int64_t)j * a.epi.batch + rr) * gridDim.x + blockIdx.x] = eacc[j];
            eacc[j] = 0.0;
        }
    };
    uint32_t phase0 = 0, phase1 = 0;
    int64_t crow = 0;   // the table holds row 0's coefficient blocks
    cx<R> r[1 << M];
    bool failed = false;
    for (int64_t t = t0, i = 0; t < t1; ++t, ++i) {
        const int b = (int)(i & 1);
        cx<R> *cur = b ? buf1 : buf0;
        if (tid == 0 && t + 1 < t1) {
            int cn[5];
            uint64_t bn;
            int64_t rn;
            geom_coords(a.g, t + 1, cn, bn, rn);
            bulk_wait_read0();   // the other buffer's previous store has read its data
            uint64_t *nb = b ? &bar[0] : &bar[1];
            mbar_expect_tx(nb, (uint32_t)tbytes);
            tma_load5(b ? buf0 : buf1, &tmap, cn, nb);
        }
        const bool ok = mbar_wait_bounded(b ? &bar[1] : &bar[0], b ? phase1 : phase0, wlim);
        if (b) phase1 ^= 1; else phase0 ^= 1;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        geom_coords(a.g, t, c, base, row);
        if (a.any_row && row != crow) {
            // row-dependent coefficient blocks of this tile's row into the table
            for (int i = tid; i < a.nops; i += blockDim.x)
                if (sops[i].rowstep) scoef[i] = gcoef[sops[i].coef + row * sops[i].rowstep];
            __syncthreads();
            crow = row;
        }
        Ops::template run<R, M, PD>(r, cur, sops, ssegs, scoef, a.nseg, a.op0, a.g.k, base, lane, warp);
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tma_store5(&tmap, c, cur);
            bulk_commit();
        }
        if (nte) {
            // diagonal observables of the final tile (read-only, beside the store)
            if (row != erow) {
                if (erow >= 0) eflush(erow);
                erow = row;
            }
            tile_epi_accum<R, M>(cur, sterm, nte, eacc, eaccw, a.g.k, base, tid, lane, warp, nw);
        }
    }
    grid_dep_launch();   // the next kernel of the stream may start its prologue
    if (nte && !failed && erow >= 0) {
        __syncthreads();
        eflush(erow);
    }
    if (failed && tid == 0) {
        atomicCAS(a.errflag, 0, DEVERR_TIMEOUT);
        // let any load still in flight land before the CTA exits (bounded)
        mbar_wait_bounded(&bar[0], phase0, wlim);
        mbar_wait_bounded(&bar[1], phase1, wlim);
    }
    if (tid == 0) bulk_wait0();
}

}  // namespace
}  // namespace dq
