// Reverse tile pass: the kernel body shared by the library's kernel, which
// interprets each pass's reverse program from shared memory, and the run-time
// specialised kernels, which have each pass's ops compiled in (internal).
//
// A pass streams psi and lambda tiles in with TMA; inside a tile each op's
// gradient partial 2 Im <lambda|G|psi> is formed (after its gate) and the
// gate is un-applied on both vectors, segment by segment; per-warp FP32
// partials are folded into the CTA's FP64 accumulators per tile.  Once the
// last segment's register layout has been read from shared memory, the next
// tile's copies are issued into the same buffers, and the results go from
// registers straight to global memory (a warp's 32 lanes hold 32 consecutive
// amplitudes: the low tile bits are the low amplitude bits), so the copy-in
// of tile t + 1 overlaps the last segment of tile t and nothing waits for a
// copy-out.
#pragma once

#include "dq_engine.cuh"
#include "dq_tma.cuh"

namespace dq {
namespace {

struct AdjArgs {
    TileGeom g;
    const EOp *ops;      // the pass's reverse decodings (op0 .. op0 + nops)
    const ESeg *segs;    // the pass's reverse segments
    int op0, nops, nseg;
    const int32_t *slots;   // global slot of each local slot
    int nslot;
    const void *coef;
    double *part;        // [slot][row][cta]
    int batch;
    int *errflag;
    int any_row;       // some op's coefficients depend on the batch row
    void *psi, *lam;   // the vectors the tensor maps describe (direct stores)
    // amplitude bit of tile bit i (ascending; the low ones are 0, 1, ...):
    // byte i of tbit[0] for i < 8, byte i - 8 of tbit[1] otherwise
    uint64_t tbit[2];
};

// Tile copy-in of the next tile and copy-out of the current one (see the
// file comment).  Runners call prefetch() once every thread holds the last
// segment's registers (all reads of the tile buffers done) and store() with
// that segment's layout instead of writing the buffers back.
// The per-tile values the copies need live in shared memory next to the
// copy barrier (written by thread 0 before the tile's first barrier), so
// nothing of them stays in registers through the tile's ops.
struct AdjTileSlot {
    uint64_t bar;       // copy barrier
    uint64_t gbase;     // row * 2^n + base of the current tile (amplitudes)
    int next_c[5];      // TMA coordinates of the next tile
    int has_next;
};
static_assert(sizeof(AdjTileSlot) <= 64, "tile slot fits the reserved 64 bytes");

template <typename R>
struct AdjIo {
    const AdjArgs *a;                 // the kernel's (grid-constant) arguments
    const CUtensorMap *mp, *ml;
    AdjTileSlot *slot;
    cx<R> *bufP, *bufL;

    __device__ __forceinline__ void prefetch() const {
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0 && slot->has_next) {
            const uint32_t tbytes = (uint32_t)(sizeof(cx<R>) << a->g.k);
            mbar_expect_tx(&slot->bar, 2 * tbytes);
            tma_load5(bufP, mp, slot->next_c, &slot->bar);
            tma_load5(bufL, ml, slot->next_c, &slot->bar);
        }
    }
    // amplitude bit of tile bit i
    __device__ __forceinline__ int tbit(int i) const { return (int)((a->tbit[i >> 3] >> (8 * (i & 7))) & 63); }
    // amplitude offset of local index l within the row's state (the lane
    // bits are the low amplitude bits)
    __device__ __forceinline__ uint64_t scatter(uint32_t l) const {
        uint64_t r = l & ((1u << kLaneBits) - 1);
#pragma unroll
        for (int i = kLaneBits; i < 16; ++i)
            if (i < a->g.k && ((l >> i) & 1)) r |= uint64_t(1) << tbit(i);
        return r;
    }
    template <int M>
    __device__ __forceinline__ void store(const cx<R> (&ps)[1 << M], const cx<R> (&ls)[1 << M],
                                          const Layout &L) const {
        const uint64_t t0 = slot->gbase | scatter(L.tb);
        cx<R> *gp = reinterpret_cast<cx<R> *>(a->psi) + t0;
        const int64_t dl = reinterpret_cast<cx<R> *>(a->lam) - reinterpret_cast<cx<R> *>(a->psi);
        uint64_t so[M];   // register bit i: one tile bit (L.off[i]) at its amplitude bit
#pragma unroll
        for (int i = 0; i < M; ++i) so[i] = uint64_t(1) << tbit(__ffs((int)L.off[i]) - 1);
#ifdef DQ_BOUNDS_BUILD
        {   // the largest index has every register bit set
            uint64_t top = t0;
            for (int i = 0; i < M; ++i) top |= so[i];
            if (!DQ_INB(top, (uint64_t)a->batch << a->g.n)) return;
        }
#endif
#pragma unroll
        for (int e = 0; e < (1 << M); ++e) {
            uint64_t o = 0;
#pragma unroll
            for (int i = 0; i < M; ++i)
                if ((e >> i) & 1) o |= so[i];
            gp[o] = ps[e];
            gp[o + dl] = ls[e];
        }
    }
};

template <typename R, int M>
constexpr int adj_max_threads() { return ((1 << M) * (int)sizeof(cx<R>) <= 64) ? 512 : 256; }
// Two CTAs of 256 threads per SM for complex64 (the large-state shape: 12-qubit
// tiles, four register bits): 128 registers a thread.
template <typename R, int M>
constexpr int adj_min_blocks() { return (sizeof(R) == 4 && M == 4) ? 2 : 1; }

// The interpreter: every op dispatched from the staged reverse program.
struct InterpRev {
    template <typename R, int M>
    __device__ __forceinline__ static void run(cx<R> (&ps)[1 << M], cx<R> (&ls)[1 << M], cx<R> *bufP, cx<R> *bufL,
                                               const EOp *sops, const ESeg *ssegs, const Mat2<R> *scoef, R *accw,
                                               int nslot, int nseg, int op0, int k, uint64_t base, int lane,
                                               int warp, const AdjIo<R> &io) {
        if (nseg == 0) io.prefetch();   // nothing changes in this tile: no copy-out
        for (int si = 0; si < nseg; ++si) {
            const ESeg sg = ssegs[si];
            const Layout L = make_layout(sg, M, k, lane, warp);
            eng_load<R, M>(ps, bufP, L);
            eng_load<R, M>(ls, bufL, L);
            const bool last = si == nseg - 1;
            if (last) io.prefetch();
            for (int cc = 0; cc < sg.nops; ++cc) {
                const int oi = sg.op0 - op0 - cc;
                const EOp o = sops[oi];
                const Mat2<R> u = scoef[oi];
                if (o.pad[1]) {   // rotation pair: this DIAG op, then the REAL op before it
                    const EOp o2 = sops[oi - 1];
                    const Mat2<R> u2 = scoef[oi - 1];
                    R gd, gr;
                    eng_adjoint_pair<R, M>(ps, ls, o, dagger(u), o2, dagger(u2), lane, gd, gr);
                    if (o.slot >= 0) {
                        const R gs = warp_sum_t(gd);
                        if (lane == 0) accw[warp * nslot + o.slot] += gs;
                    }
                    if (o2.slot >= 0) {
                        const R gs = warp_sum_t(gr);
                        if (lane == 0) accw[warp * nslot + o2.slot] += gs;
                    }
                    ++cc;
                    continue;
                }
                const R gv = eng_adjoint<R, M, false>(ps, ls, o, dagger(u), base, L, lane);
                if (o.slot >= 0) {
                    const R gs = warp_sum_t(gv);
                    if (lane == 0) accw[warp * nslot + o.slot] += gs;
                }
            }
            if (last) {
                io.template store<M>(ps, ls, L);
            } else {
                eng_store<R, M>(ps, bufP, L);
                eng_store<R, M>(ls, bufL, L);
                __syncthreads();
            }
        }
    }
};

// One reverse pass (see the file comment).  Runner::run un-applies the
// pass's ops on one tile pair in shared memory and accumulates gradients.
template <typename R, int M, typename Runner>
__device__ __forceinline__ void tile_adj_body(const CUtensorMap &mp, const CUtensorMap &ml, const AdjArgs &a) {
    extern __shared__ __align__(128) unsigned char smem[];
    if (!DQ_SMEM_ALIGNED(smem)) return;   // bounds-checking build: no copy into a misaligned buffer
    const unsigned long long wlim = wait_limit_ns(a.errflag);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const size_t tbytes = sizeof(cx<R>) << a.g.k;
    cx<R> *bufP = reinterpret_cast<cx<R> *>(smem);
    cx<R> *bufL = reinterpret_cast<cx<R> *>(smem + tbytes);
    AdjTileSlot *slot = reinterpret_cast<AdjTileSlot *>(smem + 2 * tbytes);
    uint64_t *bar = &slot->bar;
    EOp *sops = reinterpret_cast<EOp *>(smem + 2 * tbytes + 64);
    ESeg *ssegs = reinterpret_cast<ESeg *>(sops + a.nops);
    Mat2<R> *scoef = reinterpret_cast<Mat2<R> *>(ssegs + a.nseg);
    double *acc = reinterpret_cast<double *>(scoef + a.nops);       // [nslot]
    R *accw = reinterpret_cast<R *>(acc + a.nslot);                  // [nw][nslot]
    const Mat2<R> *gcoef = reinterpret_cast<const Mat2<R> *>(a.coef);
    const int64_t per = (a.g.ntiles + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * per;
    const int64_t t1 = min(a.g.ntiles, t0 + per);
    // the first tile's copies overlap the staging of the pass's ops
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        fence_async_smem();
        if (t0 < t1) {
            int c[5];
            uint64_t base;
            int64_t row;
            geom_coords(a.g, t0, c, base, row);
            mbar_expect_tx(&bar[0], (uint32_t)(2 * tbytes));
            tma_load5(bufP, &mp, c, &bar[0]);
            tma_load5(bufL, &ml, c, &bar[0]);
        }
    }
    for (int i = tid; i < a.nops; i += blockDim.x) {
        const EOp o = a.ops[i];
        sops[i] = o;
        scoef[i] = gcoef[o.coef];
    }
    for (int i = tid; i < a.nseg; i += blockDim.x) ssegs[i] = a.segs[i];
    for (int i = tid; i < a.nslot; i += blockDim.x) acc[i] = 0.0;
    for (int i = tid; i < nw * a.nslot; i += blockDim.x) accw[i] = R(0);
    __syncthreads();
    uint32_t phase = 0;
    int64_t cur_row = -1;
    bool failed = false;
    auto flush = [&](int64_t row) {
        for (int j = tid; j < a.nslot; j += blockDim.x) {
            a.part[((int64_t)a.slots[j] * a.batch + row) * gridDim.x + blockIdx.x] = acc[j];
            acc[j] = 0.0;
        }
    };
    cx<R> ps[1 << M], ls[1 << M];
    AdjIo<R> io;
    io.a = &a;
    io.mp = &mp;
    io.ml = &ml;
    io.slot = slot;
    io.bufP = bufP;
    io.bufL = bufL;
    int64_t crow = 0;   // the table holds row 0's coefficient blocks
    for (int64_t t = t0; t < t1; ++t) {
        int c[5];
        uint64_t base;
        int64_t row;
        geom_coords(a.g, t, c, base, row);
        if (row != cur_row) {
            if (cur_row >= 0) flush(cur_row);
            cur_row = row;
        }
        if (a.any_row && row != crow) {
            // row-dependent coefficient blocks of this tile's row into the table
            __syncthreads();
            for (int i = tid; i < a.nops; i += blockDim.x)
                if (sops[i].rowstep) scoef[i] = gcoef[sops[i].coef + row * sops[i].rowstep];
            __syncthreads();
            crow = row;
        }
        if (tid == 0) {
            slot->gbase = ((uint64_t)row << a.g.n) | base;
            slot->has_next = t + 1 < t1;
            if (t + 1 < t1) {
                uint64_t nb;
                int64_t nr;
                geom_coords(a.g, t + 1, slot->next_c, nb, nr);
            }
        }
        // this tile's copies were issued by the prologue or by the previous
        // tile's prefetch
        const bool ok = mbar_wait_bounded(&bar[0], phase, wlim);
        phase ^= 1;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        Runner::template run<R, M>(ps, ls, bufP, bufL, sops, ssegs, scoef, accw, a.nslot, a.nseg, a.op0, a.g.k,
                                   base, lane, warp, io);
        __syncthreads();   // every warp's partials are in accw
        for (int j = tid; j < a.nslot; j += blockDim.x) {
            double sum = 0.0;
            for (int ww = 0; ww < nw; ++ww) {
                sum += (double)accw[ww * a.nslot + j];
                accw[ww * a.nslot + j] = R(0);
            }
            acc[j] += sum;
        }
    }
    if (!failed && cur_row >= 0) {
        __syncthreads();
        flush(cur_row);
    }
    if (failed && tid == 0) {
        atomicCAS(a.errflag, 0, DEVERR_TIMEOUT);
        mbar_wait_bounded(&bar[0], phase, wlim);
    }
}

}  // namespace
}  // namespace dq
