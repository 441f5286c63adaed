// Fused k-qubit tiles staged in shared memory by TMA, with an in-register
// gate engine.
//
// Planner (host): gates are packed into passes.  A pass owns a tile bit set T
// (the lowest `low` bits plus the non-diagonal bits of its gates, at most k
// bits, at most five TMA box dimensions).  A gate may join the current pass
// when its non-diagonal bits fit in T and it commutes with every gate that
// was deferred to a later pass (on each shared bit both act diagonally);
// otherwise it is deferred and blocks its bits.  SWAP becomes three CNOTs.
//
// Kernel (device): one launch per pass, persistent CTAs over contiguous tile
// ranges.  Thread 0 streams tiles in and out with cp.async.bulk.tensor (two
// shared-memory buffers, mbarrier completion, bounded waits).  Inside a tile
// the 2^k amplitudes live in registers: lanes carry local bits 0..4, each
// thread holds 2^M amplitudes over M "register bits" B, warps carry the rest.
// Gates on register bits are register arithmetic, gates on lane bits use warp
// shuffles, diagonal gates on any bit are per-element phases, and controls
// anywhere are predicates.  Shared memory is touched only to change B.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "dq_common.cuh"
#include "dq_engine.cuh"
#include "dq_tile.h"
#include "dq_tma.cuh"
#include "dq_tile_fwd.cuh"
#include "dq_jit.h"

namespace dq {

static void release_multi(void *p);

void TileSchedule::release() {
    if (jit) {
        jit->release();
        delete jit;
        jit = nullptr;
    }
    release_multi(multi);
    multi = nullptr;
    multi_state = nullptr;
    cudaFree(d_ops);
    cudaFree(d_segs);
    cudaFree(d_rops);
    cudaFree(d_rsegs);
    cudaFree(d_slots);
    d_ops = d_rops = nullptr;
    d_segs = d_rsegs = nullptr;
    d_slots = nullptr;
}

void TileCache::release() {
    tile_release_obs(*this);
    for (auto &kv : schedules) {
        kv.second->release();
        delete kv.second;
    }
    schedules.clear();
}

namespace {

template <typename R> struct TileCfg;
template <> struct TileCfg<float> { static constexpr int wb = 0; static constexpr int Mmax = 5; };
template <> struct TileCfg<double> { static constexpr int wb = 1; static constexpr int Mmax = 4; };

inline int popc64(uint64_t x) { return __builtin_popcountll(x); }

// Number of TMA box dimensions the bit set needs (runs of consecutive word
// bits, each at most 8 bits wide because a box side is at most 256).
int dims_needed(uint64_t T, int wb) {
    uint64_t w = (T << wb) | ((uint64_t(1) << wb) - 1);
    int dims = 0;
    int b = 0;
    while (w >> b) {
        if (!((w >> b) & 1)) { ++b; continue; }
        int len = 0;
        while ((w >> (b + len)) & 1) ++len;
        dims += (len + 7) / 8;
        b += len;
    }
    return dims;
}

struct GateBits {
    uint64_t N;   // bits acted on non-diagonally
    uint64_t D;   // bits acted on diagonally (controls, diagonal targets)
};

// A schedulable item: one gate, or a CNOT-diagonal-CNOT triple run as one
// parity-diagonal op (acts diagonally on both of its bits).
struct Item {
    int g, len;
};

GateBits gate_bits(const DevGate &g) {
    GateBits gb{0, 0};
    if (g.cls == CLS_SWAP) {
        gb.N = (uint64_t(1) << g.t) | (uint64_t(1) << g.c);
    } else if (g.cls == CLS_DIAG) {
        gb.D = uint64_t(1) << g.t;
        if (g.c >= 0) gb.D |= uint64_t(1) << g.c;
    } else {
        gb.N = uint64_t(1) << g.t;
        if (g.c >= 0) gb.D = uint64_t(1) << g.c;
    }
    return gb;
}

}  // namespace

bool tile_build_schedule(const Plan &p, int k, int low, int M, int amp_bytes, TileSchedule &out, bool adjoint,
                         int g0) {
    const int n = p.n;
    const int wb = amp_bytes == 16 ? 1 : 0;
    // a SWAP of two high bits needs two free tile bits
    if (k > n || k < kTileLaneBits + M || low < kTileLaneBits || low > k - 2) return false;
    out = TileSchedule();
    out.n = n;
    out.k = k;
    out.low = low;
    out.M = M;
    out.adjoint = adjoint;
    const uint64_t lowmask = (uint64_t(1) << low) - 1;
    // gates [0, g0) are left out (an adjoint sweep that stops before them);
    // on forward passes parity triples become single items (the reverse
    // kernel keeps them as three ops, which keeps its code smaller)
    std::vector<Item> items;
    for (int i = std::max(0, g0); i < p.ngates;) {
        if (!adjoint && i + 2 < p.ngates && parity_triple(p.gates[i], p.gates[i + 1], p.gates[i + 2])) {
            items.push_back({i, 3});
            i += 3;
        } else {
            items.push_back({i, 1});
            ++i;
        }
    }
    auto item_bits = [&](const Item &it) {
        if (it.len == 3) {
            const DevGate &c = p.gates[it.g];
            return GateBits{0, (uint64_t(1) << c.t) | (uint64_t(1) << c.c)};
        }
        return gate_bits(p.gates[it.g]);
    };
    std::vector<int> remaining;
    for (int i = 0; i < (int)items.size(); ++i) remaining.push_back(i);
    int guard = 0;
    while (!remaining.empty()) {
        if (++guard > p.ngates + 2) return false;
        uint64_t T = lowmask, bnd = 0, bany = 0;
        std::vector<int> sched, deferred;
        int nops = 0;
        for (int ii : remaining) {
            const DevGate &g = p.gates[items[ii].g];
            const GateBits gb = item_bits(items[ii]);
            const int cost = (items[ii].len == 1 && g.cls == CLS_SWAP) ? 3 : 1;
            bool ok = !(gb.N & bany) && !(gb.D & bnd) && nops + cost <= kTileMaxOps;
            if (ok) {
                const uint64_t nt = T | gb.N;
                if (popc64(nt) <= k && dims_needed(nt, wb) <= 5) {
                    T = nt;
                    sched.push_back(ii);
                    nops += cost;
                    continue;
                }
            }
            deferred.push_back(ii);
            bnd |= gb.N;
            bany |= gb.N | gb.D;
        }
        if (sched.empty()) return false;
        // pad T to exactly k bits without exceeding five box dimensions
        for (int b = 0; b < n && popc64(T) < k; ++b) {
            if ((T >> b) & 1) continue;
            const uint64_t nt = T | (uint64_t(1) << b);
            if (dims_needed(nt, wb) <= 5) T = nt;
        }
        if (popc64(T) != k) return false;
        TPass pass;
        int loc[64];
        for (int b = 0, j = 0; b < n; ++b) {
            loc[b] = -1;
            if ((T >> b) & 1) {
                pass.T.push_back(b);
                loc[b] = j++;
            }
        }
        pass.op0 = (int)out.ops.size();
        std::vector<GOp> gops;
        auto push_op = [&](int cls, int tb, int cb, const DevGate &g, int slot, int gi) {
            GOp o{};
            o.gi = gi;
            o.cls = cls;
            o.tl = loc[tb];
            o.tg = tb;
            o.cl = cb >= 0 ? loc[cb] : -1;
            o.cg = cb;
            o.kind = g.kind;
            o.coef = g.coef;
            o.rowstep = g.rowstep;
            o.slot = slot;
            gops.push_back(o);
        };
        for (int ii : sched) {
            const Item &it = items[ii];
            if (it.len == 3) {
                const DevGate &c = p.gates[it.g], &d = p.gates[it.g + 1];
                const int slot = it.g + 1 < (int)p.slot_of_gate.size() ? p.slot_of_gate[it.g + 1] : -1;
                push_op(CLS_PDIAG, c.t, c.c, d, slot, it.g);
                pass.pdiag = true;
                continue;
            }
            const int gi = it.g;
            const DevGate &g = p.gates[gi];
            const int slot = gi < (int)p.slot_of_gate.size() ? p.slot_of_gate[gi] : -1;
            if (g.cls == CLS_SWAP) {
                push_op(CLS_ANTI, g.c, g.t, g, -1, gi);
                push_op(CLS_ANTI, g.t, g.c, g, -1, gi);
                push_op(CLS_ANTI, g.c, g.t, g, -1, gi);
            } else {
                push_op(g.cls, g.t, g.c, g, slot, gi);
            }
        }
        pass.nops = (int)gops.size();
        schedule_for_layouts(gops, M, kTileLaneBits);
        const std::vector<char> head = pair_real_diag(gops);
        record_order(gops, p.gates, pass.gates, pass.flags);
        // register layouts, then decode every op against its layout
        pass.seg0 = (int)out.segs.size();
        std::vector<int> B;
        int sop0 = 0;
        auto close_seg = [&](int end) {
            TSeg sg{};
            sg.op0 = pass.op0 + sop0;
            sg.nops = end - sop0;
            std::vector<int> full = B;
            for (int j = kTileLaneBits; j < k && (int)full.size() < M; ++j)
                if (std::find(full.begin(), full.end(), j) == full.end()) full.push_back(j);
            for (int i = 0; i < 8; ++i) sg.B[i] = i < M ? (int8_t)full[i] : (int8_t)-1;
            decode_with_fans(gops, sop0, end, sg.B, M, out.ops);
            out.segs.push_back(sg);
        };
        for (int i = 0; i < pass.nops; ++i) {
            const GOp &o = gops[i];
            const int need = (!cls_diagonal(o.cls) && o.tl >= kTileLaneBits) ? o.tl : -1;
            if (need < 0 || std::find(B.begin(), B.end(), need) != B.end()) continue;
            if ((int)B.size() < M) {
                B.push_back(need);
                continue;
            }
            close_seg(i);
            sop0 = i;
            B.assign(1, need);
        }
        close_seg(pass.nops);
        pass.nseg = (int)out.segs.size() - pass.seg0;

        if (adjoint) {
            // local gradient slots of the pass
            pass.slot0 = (int)out.slots.size();
            for (GOp &o : gops) {
                if (o.slot < 0) continue;
                int loc_slot = -1;
                for (int i = pass.slot0; i < (int)out.slots.size(); ++i)
                    if (out.slots[i] == o.slot) loc_slot = i - pass.slot0;
                if (loc_slot < 0) {
                    loc_slot = (int)out.slots.size() - pass.slot0;
                    out.slots.push_back(o.slot);
                }
                o.slot = loc_slot;
            }
            pass.nslot = (int)out.slots.size() - pass.slot0;
            // reverse-sweep layouts over the pass's ops, last op first
            out.rops.resize(out.ops.size());
            pass.rseg0 = (int)out.rsegs.size();
            std::vector<int> RB;
            int first = pass.nops - 1, count = 0, start = pass.nops - 1;
            auto close_r = [&](int stop) {   // ops start .. stop+1 (descending)
                TSeg sg{};
                sg.op0 = pass.op0 + first;
                sg.nops = count;
                std::vector<int> full = RB;
                for (int j = kTileLaneBits; j < k && (int)full.size() < M; ++j)
                    if (std::find(full.begin(), full.end(), j) == full.end()) full.push_back(j);
                for (int i = 0; i < 8; ++i) sg.B[i] = i < M ? (int8_t)full[i] : (int8_t)-1;
                for (int i = start; i > stop; --i) out.rops[pass.op0 + i] = decode_op(gops[i], sg.B, M);
                out.rsegs.push_back(sg);
            };
            for (int i = pass.nops - 1; i >= 0; --i) {
                const GOp &o = gops[i];
                const int need = (!cls_diagonal(o.cls) && o.tl >= kTileLaneBits) ? o.tl : -1;
                if (need >= 0 && std::find(RB.begin(), RB.end(), need) == RB.end()) {
                    if ((int)RB.size() < M) {
                        RB.push_back(need);
                    } else {
                        close_r(i);
                        RB.assign(1, need);
                        first = i;
                        count = 0;
                        start = i;
                    }
                }
                ++count;
            }
            close_r(-1);
            pass.nrseg = (int)out.rsegs.size() - pass.rseg0;
            std::vector<int> rseg(gops.size(), -1);
            for (int sgi = pass.rseg0; sgi < pass.rseg0 + pass.nrseg; ++sgi)
                for (int i = out.rsegs[sgi].op0; i > out.rsegs[sgi].op0 - out.rsegs[sgi].nops; --i)
                    rseg[i - pass.op0] = sgi;
            for (int i = 0; i + 1 < pass.nops; ++i)
                if (head[i] && rseg[i] == rseg[i + 1] &&
                    pair_handlers_match(out.rops[pass.op0 + i], out.rops[pass.op0 + i + 1]))
                    out.rops[pass.op0 + i + 1].pad[1] = 1;
        }
        out.passes.push_back(pass);
        remaining.swap(deferred);
    }
    return true;
}

namespace {

template <typename R, int M, bool PD>
__global__ void __launch_bounds__(tile_max_threads<R, M>(), tile_min_blocks<R, M>())
k_tile_fwd(const __grid_constant__ CUtensorMap tmap, TileKArgs a) {
    tile_fwd_body<R, M, PD, InterpOps>(tmap, a);
}

// ---------------------------------------------------------------------------
// Persistent multi-pass forward kernel for states that stay in L2.
//
// All passes of a schedule (up to kMultiMaxPasses per launch) run in one
// launch: each CTA streams its share of the tiles of pass p exactly as
// k_tile_fwd does, waits until its bulk stores have completed, and then the
// grid meets at a barrier before pass p + 1 reads the state in its new tile
// layout.  Every CTA of the grid must be resident at once (the grid is sized
// by the occupancy calculator, one wave); the barrier wait is bounded, and a
// CTA that gives up sets the context's error flag, which the others see in
// their own wait and leave too.
// ---------------------------------------------------------------------------
constexpr int kMultiMaxPasses = 20;

struct MultiPass {
    int op0, nops, seg0, nseg;
    int any_row;
    TileGeom g;
};

// Tensor maps travel as kernel parameters (so no device copy is needed and
// the launch can be captured into a graph); __grid_constant__ keeps them in
// parameter space, where TMA may read them.
struct MultiArgs {
    CUtensorMap map[kMultiMaxPasses];
    MultiPass pass[kMultiMaxPasses];
    int npass;
    const TOp *ops;
    const TSeg *segs;
    const void *coef;
    int *errflag;
    unsigned int *bar;      // arrival counter, zero at launch
    TileEpi epi;            // diagonal observables of the last pass (nterms == 0: none)
};

// Launch data of one chunk of passes for the last state buffer seen.
struct MultiLaunch {
    MultiArgs args;
    size_t smem;
    int grid;
    bool pd;
};

}  // namespace

static void release_multi(void *p) { delete reinterpret_cast<std::vector<MultiLaunch> *>(p); }

namespace {

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void red_add_release_gpu(unsigned int *p, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0 of every CTA: arrive (after this CTA's completed bulk stores) and
// wait until `target` arrivals have been counted.  False when the wait ran
// out (the error flag is then set) or another CTA has set the error flag.
__device__ __forceinline__ bool grid_arrive_wait(unsigned int *bar, unsigned int target, int *errflag,
                                                 unsigned long long limit_ns) {
    fence_proxy_async_global();
    red_add_release_gpu(bar, 1u);
    if (ld_acquire_gpu(bar) < target) {
        const uint64_t t0 = global_ns();
        for (;;) {
            __nanosleep(64);
            if (ld_acquire_gpu(bar) >= target) break;
            if (*reinterpret_cast<volatile int *>(errflag) != 0) return false;
            if (global_ns() - t0 > limit_ns) {
                atomicCAS(errflag, 0, DEVERR_TIMEOUT);
                return false;
            }
        }
    }
    // the other CTAs' stores (made by the async proxy) before this CTA's
    // next tensor loads
    fence_proxy_async_global();
    return true;
}

template <typename R, int M, bool PD>
__global__ void __launch_bounds__(tile_max_threads<R, M>(), tile_min_blocks<R, M>())
k_tile_multi(const __grid_constant__ MultiArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_stop;
    if (!DQ_SMEM_ALIGNED(smem)) return;   // bounds-checking build (every CTA alike): no misaligned copy
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned long long wlim = wait_limit_ns(a.errflag);
    const int k = a.pass[0].g.k;
    const size_t tbytes = sizeof(cx<R>) << k;
    cx<R> *buf0 = reinterpret_cast<cx<R> *>(smem);
    cx<R> *buf1 = reinterpret_cast<cx<R> *>(smem + tbytes);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * tbytes);
    int maxops = 0, maxseg = 0;
    for (int p = 0; p < a.npass; ++p) {
        maxops = max(maxops, a.pass[p].nops);
        maxseg = max(maxseg, a.pass[p].nseg);
    }
    TOp *sops = reinterpret_cast<TOp *>(smem + 2 * tbytes + 64);
    TSeg *ssegs = reinterpret_cast<TSeg *>(sops + maxops);
    Mat2<R> *scoef = reinterpret_cast<Mat2<R> *>(ssegs + maxseg);
    const int nte = a.epi.nterms, nw = blockDim.x >> 5;
    ETerm *sterm = reinterpret_cast<ETerm *>(scoef + maxops);     // [nte]
    double *eacc = reinterpret_cast<double *>(sterm + nte);         // [nte]
    R *eaccw = reinterpret_cast<R *>(eacc + nte);                   // [nw][nte]
    const Mat2<R> *gcoef = reinterpret_cast<const Mat2<R> *>(a.coef);
    const int64_t ntiles = a.pass[0].g.ntiles;
    const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * per;
    const int64_t t1 = min(ntiles, t0 + per);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_async_smem();
        s_stop = 0;
    }
    for (int i = tid; i < nw * nte; i += blockDim.x) eaccw[i] = R(0);
    grid_dep_wait();
    uint32_t phase0 = 0, phase1 = 0;
    bool failed = false;
    int64_t erow = -1;
    cx<R> r[1 << M];
    for (int p = 0; p < a.npass && !failed; ++p) {
        const MultiPass &P = a.pass[p];
        const CUtensorMap *map = &a.map[p];
        const bool last = p + 1 == a.npass;
        int c[5];
        uint64_t base;
        int64_t row;
        if (tid == 0 && t0 < t1) {
            geom_coords(P.g, t0, c, base, row);
            mbar_expect_tx(&bar[0], (uint32_t)tbytes);
            tma_load5(buf0, map, c, &bar[0]);
        }
        // this pass's program and row-0 coefficient blocks
        for (int i = tid; i < P.nops; i += blockDim.x) {
            const TOp o = a.ops[P.op0 + i];
            sops[i] = o;
            scoef[i] = gcoef[o.coef];
        }
        for (int i = tid; i < P.nseg; i += blockDim.x) ssegs[i] = a.segs[P.seg0 + i];
        if (last && nte) tile_epi_setup(a.epi, k, sterm, eacc, tid);
        __syncthreads();
        int64_t crow = 0;
        for (int64_t t = t0, i = 0; t < t1; ++t, ++i) {
            const int b = (int)(i & 1);
            cx<R> *cur = b ? buf1 : buf0;
            if (tid == 0 && t + 1 < t1) {
                int cn[5];
                uint64_t bn;
                int64_t rn;
                geom_coords(P.g, t + 1, cn, bn, rn);
                bulk_wait_read0();
                uint64_t *nb = b ? &bar[0] : &bar[1];
                mbar_expect_tx(nb, (uint32_t)tbytes);
                tma_load5(b ? buf0 : buf1, map, cn, nb);
            }
            const bool ok = mbar_wait_bounded(b ? &bar[1] : &bar[0], b ? phase1 : phase0, wlim);
            if (b) phase1 ^= 1; else phase0 ^= 1;
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            geom_coords(P.g, t, c, base, row);
            if (P.any_row && row != crow) {
                for (int i2 = tid; i2 < P.nops; i2 += blockDim.x)
                    if (sops[i2].rowstep) scoef[i2] = gcoef[sops[i2].coef + row * sops[i2].rowstep];
                __syncthreads();
                crow = row;
            }
            tile_run_ops<R, M, PD>(r, cur, sops, ssegs, scoef, P.nseg, P.op0, k, base, lane, warp);
            fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tma_store5(map, c, cur);
                bulk_commit();
            }
            if (last && nte) {
                if (row != erow) {
                    if (erow >= 0)
                        for (int j = tid; j < nte; j += blockDim.x) {
                            a.epi.part[((int64_t)j * a.epi.batch + erow) * gridDim.x + blockIdx.x] = eacc[j];
                            eacc[j] = 0.0;
                        }
                    erow = row;
                }
                tile_epi_accum<R, M>(cur, sterm, nte, eacc, eaccw, k, base, tid, lane, warp, nw);
            }
        }
        if (failed) break;
        if (!last) {
            // every store of this pass has landed before any CTA reads the
            // next layout
            if (tid == 0) {
                bulk_wait0();
                if (!grid_arrive_wait(a.bar, (unsigned int)(p + 1) * gridDim.x, a.errflag, wlim)) s_stop = 1;
            }
            __syncthreads();
            if (s_stop) return;   // no copies in flight: the stores were waited for, no load was issued
        }
    }
    grid_dep_launch();
    if (nte && !failed && erow >= 0) {
        __syncthreads();
        for (int j = tid; j < nte; j += blockDim.x)
            a.epi.part[((int64_t)j * a.epi.batch + erow) * gridDim.x + blockIdx.x] = eacc[j];
    }
    if (failed && tid == 0) {
        atomicCAS(a.errflag, 0, DEVERR_TIMEOUT);
        mbar_wait_bounded(&bar[0], phase0, wlim);
        mbar_wait_bounded(&bar[1], phase1, wlim);
    }
    if (tid == 0) bulk_wait0();
}

size_t tile_smem_bytes(int k, int amp, int nops, int nseg, int nterms = 0, int threads = 0) {
    return 2 * ((size_t)amp << k) + 64 + (size_t)nops * sizeof(TOp) + (size_t)nseg * sizeof(TSeg) +
           (size_t)nops * (amp == 8 ? sizeof(Mat2<float>) : sizeof(Mat2<double>)) +
           (size_t)nterms * (sizeof(ETerm) + sizeof(double) + (size_t)(threads / 32) * (amp == 8 ? 4 : 8)) + 64;
}

uint64_t sched_key(const Plan &p, int k, int low, int amp, int M, bool adjoint = false, int g0 = 0) {
    uint64_t h = p.key ^ (adjoint ? 0x51ED270B27A4C3F1ull : 0x9E3779B97F4A7C15ull);
    h = (h ^ (uint64_t)(uint32_t)g0) * 1099511628211ull;
    h = (h ^ (uint64_t)M) * 1099511628211ull;
    h = (h ^ (uint64_t)k) * 1099511628211ull;
    h = (h ^ (uint64_t)low) * 1099511628211ull;
    h = (h ^ (uint64_t)amp) * 1099511628211ull;
    return h;
}

template <typename R>
void default_tile(int n, int &k, int &low, int &M, bool jit) {
    if (n >= 25 && sizeof(R) == 4 && jit) {
        // large complex64 states, passes compiled per circuit: 12-qubit tiles
        // of 256 threads, four register bits, lane bits resident (fewer
        // passes now that the ops cost no dispatch) -- measured on the
        // 30-qubit QFT + ansatz circuit, forward passes: 45 in 190 ms against
        // 66 in 245 ms for the one-warp 10-qubit tiles below (11 / 5 / 4: 54
        // in 211 ms; 13 / 5 / 4: 39 in 215 ms)
        k = 12;
        M = 4;
        low = kTileLaneBits;
        return;
    }
    if (n >= 25 && sizeof(R) == 4) {
        // large complex64 states: one-warp CTAs of 32 amplitudes per thread
        // (no inter-warp barriers at layout changes) on 10-qubit tiles with
        // the five lane bits always resident -- measured on the 30-qubit QFT +
        // ansatz circuit: 396 ms against 438 ms for 12-qubit tiles, 4
        // register bits and 7 resident bits
        k = 10;
        M = 5;
        low = kTileLaneBits;
        return;
    }
    if (n >= 20 && sizeof(R) == 4) {
        // 20..24 qubits (often many rows: Hessian and density-gradient
        // batches): 11-qubit tiles, four register bits, lane bits resident --
        // measured on the 22-qubit Hessian batch (176 rows): 114 ms against
        // 175 ms for three register bits and seven resident bits
        k = std::min(11, n - 1);
        M = 4;
        low = kTileLaneBits;
        return;
    }
    if (n >= 25) {
        M = 4;
        k = 12;
    } else {
        M = 3;
        k = std::max(kTileLaneBits + M, std::min(11, n - 9));
    }
    k = std::min(k, n - 1);
    M = std::min(M, k - kTileLaneBits);
    low = std::max(kTileLaneBits, std::min(7, k - 3));   // keep >= 2 free tile bits (SWAP)
}

template <typename R>
const void *tile_kernel(int M, bool pd) {
    switch (M) {
    case 2: return pd ? (const void *)k_tile_fwd<R, 2, true> : (const void *)k_tile_fwd<R, 2, false>;
    case 3: return pd ? (const void *)k_tile_fwd<R, 3, true> : (const void *)k_tile_fwd<R, 3, false>;
    case 4: return pd ? (const void *)k_tile_fwd<R, 4, true> : (const void *)k_tile_fwd<R, 4, false>;
    default:
        return pd ? (const void *)k_tile_fwd<R, (TileCfg<R>::Mmax), true>
                  : (const void *)k_tile_fwd<R, (TileCfg<R>::Mmax), false>;
    }
}

template <typename T>
bool upload_vec(T **dst, const std::vector<T> &v) {
    if (cudaMalloc((void **)dst, sizeof(T) * std::max<size_t>(1, v.size())) != cudaSuccess) {
        cudaGetLastError();
        *dst = nullptr;
        return false;
    }
    if (!v.empty() && cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return false;
    return true;
}

}  // namespace

TileSchedule *get_schedule(TileCache &tc, const Plan &p, int k, int low, int M, int amp, bool adjoint, int g0) {
    const uint64_t key = sched_key(p, k, low, amp, M, adjoint, g0);
    auto it = tc.schedules.find(key);
    if (it != tc.schedules.end()) return it->second;
    TileSchedule *s = new TileSchedule();
    if (!tile_build_schedule(p, k, low, M, amp, *s, adjoint, g0)) {
        delete s;
        return nullptr;
    }
    bool ok = upload_vec(&s->d_ops, s->ops) && upload_vec(&s->d_segs, s->segs);
    if (ok && adjoint)
        ok = upload_vec(&s->d_rops, s->rops) && upload_vec(&s->d_rsegs, s->rsegs) && upload_vec(&s->d_slots, s->slots);
    if (!ok) {
        s->release();
        delete s;
        return nullptr;
    }
    tc.schedules[key] = s;
    return s;
}

namespace {

template <typename R>
const void *multi_kernel(int M, bool pd) {
    switch (M) {
    case 2: return pd ? (const void *)k_tile_multi<R, 2, true> : (const void *)k_tile_multi<R, 2, false>;
    case 3: return pd ? (const void *)k_tile_multi<R, 3, true> : (const void *)k_tile_multi<R, 3, false>;
    case 4: return pd ? (const void *)k_tile_multi<R, 4, true> : (const void *)k_tile_multi<R, 4, false>;
    default:
        return pd ? (const void *)k_tile_multi<R, (TileCfg<R>::Mmax), true>
                  : (const void *)k_tile_multi<R, (TileCfg<R>::Mmax), false>;
    }
}

// The persistent multi-pass kernel serves states that stay in L2 between
// passes, with at least two passes to merge.
bool multi_applies(const TileCache &tc, const TileSchedule &sc, int n, int64_t batch, int amp) {
#ifdef DQ_BOUNDS_BUILD
    return false;   // the bounds-checking build runs one launch per pass
#endif
    return tc.multi_on && tc.gridbar && sc.passes.size() >= 2 && ((batch << n) * (int64_t)amp) <= kMultiMaxStateBytes;
}

template <typename R>
cudaError_t run_forward_multi(TileCache &tc, const Plan &p, TileSchedule &sc, const void *coef, void *state,
                              int batch, int nsm, cudaStream_t s, int64_t *launches, const TileEpi *epi,
                              int *epi_grid) {
    const int M = sc.M;
    constexpr int wb = TileCfg<R>::wb;
    const int amp = (int)sizeof(cx<R>);
    const int threads = 1 << (sc.k - M);
    const int npass = (int)sc.passes.size();
    const int nchunk = (npass + kMultiMaxPasses - 1) / kMultiMaxPasses;
    const int nte = epi ? epi->nterms : 0;
    auto *cache = reinterpret_cast<std::vector<MultiLaunch> *>(sc.multi);
    if (!cache) {
        cache = new std::vector<MultiLaunch>();
        sc.multi = cache;
    }
    if (sc.multi_state != state || sc.multi_batch != batch || sc.multi_nte != nte || (int)cache->size() != nchunk) {
        cache->assign(nchunk, MultiLaunch{});
        sc.multi_state = nullptr;
        for (int ch = 0; ch < nchunk; ++ch) {
            MultiLaunch &L = (*cache)[ch];
            MultiArgs &a = L.args;
            std::memset(&a, 0, sizeof(a));
            const int p0 = ch * kMultiMaxPasses, p1 = std::min(npass, p0 + kMultiMaxPasses);
            const bool last_chunk = ch + 1 == nchunk;
            a.npass = p1 - p0;
            int maxops = 0, maxseg = 0;
            bool pd = false;
            for (int pi = p0; pi < p1; ++pi) {
                const TPass &ps = sc.passes[pi];
                TileDims d;
                if (!make_dims(ps.T, p.n, wb, d)) return cudaErrorInvalidValue;
                if (!encode_map(tc.encode_fn, &a.map[pi - p0], d, state, batch, wb)) return cudaErrorInvalidValue;
                MultiPass &mp = a.pass[pi - p0];
                mp.op0 = ps.op0;
                mp.nops = ps.nops;
                mp.seg0 = ps.seg0;
                mp.nseg = ps.nseg;
                mp.any_row = 0;
                for (int j = ps.op0; j < ps.op0 + ps.nops; ++j) mp.any_row |= sc.ops[j].rowstep != 0;
                mp.g = make_geom(d, p.n, sc.k, wb, batch);
                maxops = std::max(maxops, ps.nops);
                maxseg = std::max(maxseg, ps.nseg);
                pd |= ps.pdiag;
            }
            L.pd = pd;
            L.smem = tile_smem_bytes(sc.k, amp, maxops, maxseg, last_chunk ? nte : 0, threads);
            const void *kfn = multi_kernel<R>(M, pd);
            if (tc.smem_set[kfn] < L.smem) {
                cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
                if (e != cudaSuccess) return e;
                tc.smem_set[kfn] = L.smem;
            }
            int per_sm = 0;
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, threads, L.smem);
            if (e != cudaSuccess) return e;
            if (per_sm < 1) return cudaErrorInvalidConfiguration;
            const int64_t ntiles = (int64_t)batch << (p.n - sc.k);
            // one wave: every CTA resident at once (the grid barrier needs it)
            int64_t grid = std::min<int64_t>(ntiles, (int64_t)per_sm * nsm);
            if (last_chunk && nte) grid = std::min<int64_t>(grid, 4 * (int64_t)nsm);   // epilogue partials
            L.grid = (int)grid;
        }
        sc.multi_state = state;
        sc.multi_batch = batch;
        sc.multi_nte = nte;
    }
    for (int ch = 0; ch < nchunk; ++ch) {
        MultiLaunch &L = (*cache)[ch];
        MultiArgs &a = L.args;
        const bool last_chunk = ch + 1 == nchunk;
        a.ops = sc.d_ops;
        a.segs = sc.d_segs;
        a.coef = coef;
        a.errflag = tc.errflag;
        a.bar = tc.gridbar;
        a.epi = TileEpi{};
        if (last_chunk && epi) {
            a.epi = *epi;
            const TPass &ps = sc.passes[npass - 1];
            for (int j = 0; j < 16; ++j) a.epi.T[j] = (int8_t)(j < (int)ps.T.size() ? ps.T[j] : 0);
            if (epi_grid) *epi_grid = L.grid;
        }
        cudaError_t e = cudaMemsetAsync(tc.gridbar, 0, sizeof(unsigned int), s);
        if (e != cudaSuccess) return e;
        LaunchScope ls(s, "k_tile_multi", launches);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        cfg.gridDim = dim3((unsigned)L.grid);
        cfg.blockDim = dim3((unsigned)threads);
        cfg.dynamicSmemBytes = L.smem;
        cfg.stream = s;
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        switch (M * 2 + (L.pd ? 1 : 0)) {
        case 4: e = cudaLaunchKernelEx(&cfg, k_tile_multi<R, 2, false>, a); break;
        case 5: e = cudaLaunchKernelEx(&cfg, k_tile_multi<R, 2, true>, a); break;
        case 6: e = cudaLaunchKernelEx(&cfg, k_tile_multi<R, 3, false>, a); break;
        case 7: e = cudaLaunchKernelEx(&cfg, k_tile_multi<R, 3, true>, a); break;
        case 8: e = cudaLaunchKernelEx(&cfg, k_tile_multi<R, 4, false>, a); break;
        case 9: e = cudaLaunchKernelEx(&cfg, k_tile_multi<R, 4, true>, a); break;
        default:
            e = L.pd ? cudaLaunchKernelEx(&cfg, k_tile_multi<R, (TileCfg<R>::Mmax), true>, a)
                     : cudaLaunchKernelEx(&cfg, k_tile_multi<R, (TileCfg<R>::Mmax), false>, a);
            break;
        }
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename R>
cudaError_t run_forward(TileCache &tc, const Plan &p, TileSchedule &sc, const void *coef, void *state,
                        int batch, int nsm, cudaStream_t s, int64_t *launches, const TileEpi *epi = nullptr,
                        int *epi_grid = nullptr, bool use_jit = false) {
    const int M = sc.M;
    const bool jit = use_jit && sc.jit != nullptr;
    if (!jit && multi_applies(tc, sc, p.n, batch, (int)sizeof(cx<R>)))
        return run_forward_multi<R>(tc, p, sc, coef, state, batch, nsm, s, launches, epi, epi_grid);
    constexpr int wb = TileCfg<R>::wb;
    const int amp = (int)sizeof(cx<R>);
    const int threads = 1 << (sc.k - M);
    if (sc.fwd_state != state || sc.fwd_batch != batch || sc.fwd_launch.size() != sc.passes.size()) {
        // encode every pass once for this buffer
        sc.fwd_launch.assign(sc.passes.size(), TileSchedule::Launch{});
        sc.fwd_state = nullptr;
        for (size_t i = 0; i < sc.passes.size(); ++i) {
            const TPass &ps = sc.passes[i];
            TileDims d;
            if (!make_dims(ps.T, p.n, wb, d)) return cudaErrorInvalidValue;
            TileSchedule::Launch &L = sc.fwd_launch[i];
            if (!encode_map(tc.encode_fn, &L.map, d, state, batch, wb)) return cudaErrorInvalidValue;
            L.smem = tile_smem_bytes(sc.k, amp, ps.nops, ps.nseg);
            const void *kfn = tile_kernel<R>(M, ps.pdiag);
            if (tc.smem_set[kfn] < L.smem) {
                cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
                if (e != cudaSuccess) return e;
                tc.smem_set[kfn] = L.smem;
            }
        }
        for (size_t i = 0; i < sc.passes.size(); ++i) {
            TileSchedule::Launch &L = sc.fwd_launch[i];
            const void *kfn = tile_kernel<R>(M, sc.passes[i].pdiag);
            int per_sm = 1;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, threads, L.smem);
            per_sm = std::max(1, per_sm);
            const int64_t ntiles = (int64_t)batch << (p.n - sc.k);
            L.grid = (int)std::min<int64_t>(ntiles, (int64_t)per_sm * nsm);
        }
        sc.fwd_state = state;
        sc.fwd_batch = batch;
        if (sc.jit) sc.jit->grid.assign(sc.passes.size(), 0);
    }
    for (size_t i = 0; i < sc.passes.size(); ++i) {
        const TPass &ps = sc.passes[i];
        const TileSchedule::Launch &L = sc.fwd_launch[i];
        TileDims d;
        if (!make_dims(ps.T, p.n, wb, d)) return cudaErrorInvalidValue;
        TileKArgs a;
        a.epi = TileEpi{};
        size_t smem = L.smem;
        int grid = L.grid;
        const void *kfn = jit ? (const void *)sc.jit->kernels[i] : tile_kernel<R>(M, ps.pdiag);
        if (jit) {
            // the specialised kernel has its own register count: its own grid
            if (sc.jit->smem_set[i] < smem) {
                cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
                sc.jit->smem_set[i] = smem;
            }
            if (!sc.jit->grid[i]) {
                int per_sm = 1;
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, threads, smem);
                per_sm = std::max(1, per_sm);
                sc.jit->grid[i] = (int)std::min<int64_t>((int64_t)batch << (p.n - sc.k), (int64_t)per_sm * nsm);
            }
            grid = sc.jit->grid[i];
        }
        if (epi && i + 1 == sc.passes.size()) {
            // the last pass also measures the diagonal observables
            a.epi = *epi;
            for (int j = 0; j < 16; ++j) a.epi.T[j] = (int8_t)(j < (int)ps.T.size() ? ps.T[j] : 0);
            smem = tile_smem_bytes(sc.k, amp, ps.nops, ps.nseg, epi->nterms, threads);
            size_t &opened = jit ? sc.jit->smem_set[i] : tc.smem_set[kfn];
            if (opened < smem) {
                cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
                opened = smem;
            }
            grid = std::min(grid, 4 * nsm);   // the partials hold at most 4 CTAs per SM
            if (epi_grid) *epi_grid = grid;
        }
        a.ops = sc.d_ops;
        a.segs = sc.d_segs;
        a.op0 = ps.op0;
        a.nops = ps.nops;
        a.seg0 = ps.seg0;
        a.nseg = ps.nseg;
        a.coef = coef;
        a.g = make_geom(d, p.n, sc.k, wb, batch);
        a.errflag = tc.errflag;
        a.any_row = 0;
        for (int j = ps.op0; j < ps.op0 + ps.nops; ++j) a.any_row |= sc.ops[j].rowstep != 0;
        LaunchScope ls(s, jit ? "k_tile_fwd_jit" : "k_tile_fwd", launches);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3((unsigned)threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t e;
        const bool pd = ps.pdiag;
        if (jit) {
            void *args[] = {(void *)&L.map, (void *)&a};
            e = cudaLaunchKernelExC(&cfg, kfn, args);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            continue;
        }
        switch (M * 2 + (pd ? 1 : 0)) {
        case 4: e = cudaLaunchKernelEx(&cfg, k_tile_fwd<R, 2, false>, L.map, a); break;
        case 5: e = cudaLaunchKernelEx(&cfg, k_tile_fwd<R, 2, true>, L.map, a); break;
        case 6: e = cudaLaunchKernelEx(&cfg, k_tile_fwd<R, 3, false>, L.map, a); break;
        case 7: e = cudaLaunchKernelEx(&cfg, k_tile_fwd<R, 3, true>, L.map, a); break;
        case 8: e = cudaLaunchKernelEx(&cfg, k_tile_fwd<R, 4, false>, L.map, a); break;
        case 9: e = cudaLaunchKernelEx(&cfg, k_tile_fwd<R, 4, true>, L.map, a); break;
        default:
            e = pd ? cudaLaunchKernelEx(&cfg, k_tile_fwd<R, (TileCfg<R>::Mmax), true>, L.map, a)
                   : cudaLaunchKernelEx(&cfg, k_tile_fwd<R, (TileCfg<R>::Mmax), false>, L.map, a);
            break;
        }
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

bool tile_supported(int n, int amp_bytes) {
    (void)amp_bytes;
    return n >= kTileLaneBits + 3 + 1 && n <= 34;
}

size_t tile_workspace_bytes(const Plan &, int, int) { return 0; }

template <typename R>
cudaError_t tile_apply(TileCache &tc, std::unordered_map<uint64_t, TileTune> &tuned, const Plan &p,
                       const void *coef, void *state, int batch, void *tws, int nsm, cudaStream_t s,
                       int64_t *launches) {
    (void)tws;
    if (!ensure_encode_fn(tc)) return cudaErrorNotSupported;
    int k, low, M;
    // untuned plans take specialised passes only when DQ_OPT_JIT is 1
    default_tile<R>(p.n, k, low, M, tc.jit_mode == 1 && jit_available());
    auto it = tuned.find(p.key ^ (sizeof(R) == 8 ? 1ull : 0ull));
    if (it != tuned.end() && it->second.k) {
        k = it->second.k;
        low = it->second.low;
        M = it->second.M;
    }
    TileSchedule *sc = get_schedule(tc, p, k, low, M, (int)sizeof(cx<R>), false);
    if (!sc) return cudaErrorNotSupported;
    const bool jit = jit_want(tc, tuned, p, (int)sizeof(cx<R>), *sc);
    return run_forward<R>(tc, p, *sc, coef, state, batch, nsm, s, launches, nullptr, nullptr, jit);
}

template <typename R>
cudaError_t tile_apply_expect(TileCache &tc, std::unordered_map<uint64_t, TileTune> &tuned, const Plan &p,
                              const void *coef, void *state, int batch, const std::vector<DevTerm> &bits,
                              const DevTerm *d_bits, const int32_t *d_ptr, int nobs, double *part, double *out,
                              int nsm, cudaStream_t s, int64_t *launches, bool part_zeroed) {
    if (!ensure_encode_fn(tc)) return cudaErrorNotSupported;
    for (const DevTerm &t : bits)
        if (t.f != 0 || t.nY != 0) return cudaErrorNotSupported;   // diagonal terms only
    if (bits.empty() || bits.size() > 64) return cudaErrorNotSupported;
    int k, low, M;
    // untuned plans take specialised passes only when DQ_OPT_JIT is 1
    default_tile<R>(p.n, k, low, M, tc.jit_mode == 1 && jit_available());
    auto it = tuned.find(p.key ^ (sizeof(R) == 8 ? 1ull : 0ull));
    if (it != tuned.end() && it->second.k) {
        k = it->second.k;
        low = it->second.low;
        M = it->second.M;
    }
    TileSchedule *sc = get_schedule(tc, p, k, low, M, (int)sizeof(cx<R>), false);
    if (!sc || sc->passes.empty()) return cudaErrorNotSupported;
    const int nsm4 = 4 * nsm;
    cudaError_t e = cudaSuccess;
    if (!part_zeroed) {   // CTAs without a tile of a row leave its partial slots alone
        e = cudaMemsetAsync(part, 0, sizeof(double) * bits.size() * (size_t)batch * nsm4, s);
        if (e != cudaSuccess) return e;
    }
    TileEpi epi{};
    epi.terms = d_bits;
    epi.nterms = (int)bits.size();
    epi.part = part;
    epi.batch = batch;
    int grid = 0;
    const bool jit = jit_want(tc, tuned, p, (int)sizeof(cx<R>), *sc);
    e = run_forward<R>(tc, p, *sc, coef, state, batch, nsm, s, launches, &epi, &grid, jit);
    if (e != cudaSuccess) return e;
    if (grid < 1 || grid > nsm4) return cudaErrorInvalidValue;
    return expect_finalize_nblk(part, d_bits, d_ptr, nobs, batch, grid, out, s, launches);
}

template <typename R>
cudaError_t tile_autotune(TileCache &tc, std::unordered_map<uint64_t, TileTune> &tuned, const Plan &p,
                          const void *coef, void *state, int batch, void *tws, int nsm, cudaStream_t s,
                          int64_t *launches, bool graphs) {
    (void)tws;
    if (!ensure_encode_fn(tc)) return cudaErrorNotSupported;
    struct Cand {
        float ms;
        int k, low, M;
    };
    std::vector<Cand> cands;
    TileTune bt;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    Tracer *saved = g_tracer;
    g_tracer = nullptr;
    // time three forwards after a warm-up one (j: specialised passes)
    auto timed = [&](TileSchedule &sc, bool j, float &ms) {
        cudaError_t err = run_forward<R>(tc, p, sc, coef, state, batch, nsm, s, launches, nullptr, nullptr, j);
        cudaEventRecord(e0, s);
        for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep)
            err = run_forward<R>(tc, p, sc, coef, state, batch, nsm, s, launches, nullptr, nullptr, j);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (err != cudaSuccess) cudaGetLastError();
        return err == cudaSuccess;
    };
    for (int M = 2; M <= TileCfg<R>::Mmax; ++M)
    for (int k = kTileLaneBits + M; k <= std::min(p.n - 1, sizeof(R) == 4 ? 13 : 12); ++k) {
        const int maxt = ((1 << M) * (int)sizeof(cx<R>) >= 256) ? 256 : 512;
        if ((1 << (k - M)) > maxt) continue;
        for (int low : {5, 7}) {
            if (low > k - 2) continue;
            TileSchedule *sc = get_schedule(tc, p, k, low, M, (int)sizeof(cx<R>), false);
            float ms = 0.f;
            if (sc && timed(*sc, false, ms)) cands.push_back({ms, k, low, M});
        }
    }
    std::sort(cands.begin(), cands.end(), [](const Cand &a, const Cand &b) { return a.ms < b.ms; });
    float best = 1e30f;
    if (!cands.empty()) {
        best = cands[0].ms;
        bt.k = cands[0].k;
        bt.low = cands[0].low;
        bt.M = cands[0].M;
    }
    // the three fastest shapes' passes as run-time specialised kernels: a
    // pass without dispatch may favour another shape (DQ_OPT_JIT = 2 uses
    // the fastest of all).  Their times can lie within a few percent of one
    // another, so short forwards (under 10 ms) are timed in seven rounds, the
    // shapes taken in turn, and each keeps its fastest round.
    if (tc.jit_mode != 0 && jit_available()) {
        // Also up to three of the next five shapes whose schedules have no
        // more passes than the fewest of the first three: the interpreter's
        // per-op dispatch can rank a wider tile (fewer, longer passes), or
        // another register split of it, below shapes that its specialised
        // passes beat.
        std::vector<std::pair<TileSchedule *, Cand>> js;
        size_t fewest = SIZE_MAX;
        int extra = 0;
        for (size_t ci = 0; ci < cands.size() && ci < 8; ++ci) {
            const Cand &cd = cands[ci];
            TileSchedule *sc = get_schedule(tc, p, cd.k, cd.low, cd.M, (int)sizeof(cx<R>), false);
            if (!sc || sc->jit_failed) continue;
            if (ci >= 3) {
                if (extra >= 3 || sc->passes.size() > fewest) continue;
                ++extra;
            }
            std::string err;
            if (!sc->jit && !jit_build(*sc, (int)sizeof(cx<R>), tc.device, &err)) {
                sc->jit_failed = true;
                tc.jit_err = err;
                continue;
            }
            if (ci < 3) fewest = std::min(fewest, sc->passes.size());
            js.push_back({sc, cd});
        }
        // with graphs on, each candidate's forward is captured once (after a
        // stream run that loads its module) and replayed
        std::vector<cudaGraphExec_t> gx(js.size(), nullptr);
        cudaStream_t cs = nullptr;
        if (graphs && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            cs = nullptr;
        }
        for (size_t q = 0; q < js.size() && cs; ++q) {
            if (run_forward<R>(tc, p, *js[q].first, coef, state, batch, nsm, s, launches, nullptr, nullptr, true) !=
                    cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            int64_t captured = 0;   // captured launches run only when replayed
            const cudaError_t re =
                run_forward<R>(tc, p, *js[q].first, coef, state, batch, nsm, cs, &captured, nullptr, nullptr, true);
            const cudaError_t ce = cudaStreamEndCapture(cs, &g);
            if (re != cudaSuccess || ce != cudaSuccess || !g || cudaGraphInstantiate(&gx[q], g, 0) != cudaSuccess)
                gx[q] = nullptr;
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
        }
        // Each timed forward starts from a cleared L2 (a 256 MiB fill), as a
        // call between other work finds it: back-to-back runs of one circuit
        // keep its kernels' code and tables cached and favour schedules with
        // more, smaller passes, which a cold start makes slower.
        const size_t flush_bytes = size_t(256) << 20;
        void *flush = nullptr;
        if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
            cudaGetLastError();
            flush = nullptr;
        }
        auto timed_one = [&](size_t q, int round, float &ms) {
            if (flush) cudaMemsetAsync(flush, (int)(q + round) & 0xff, flush_bytes, s);
            cudaEventRecord(e0, s);
            cudaError_t err = gx[q] ? cudaGraphLaunch(gx[q], s)
                                    : run_forward<R>(tc, p, *js[q].first, coef, state, batch, nsm, s, launches,
                                                     nullptr, nullptr, true);
            if (gx[q] && err == cudaSuccess && launches) *launches += (int64_t)js[q].first->passes.size();
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
            if (err != cudaSuccess) cudaGetLastError();
            return err == cudaSuccess;
        };
        std::vector<float> fastest(js.size(), 1e30f);
        for (size_t q = 0; q < js.size(); ++q) {   // warm-up: modules loaded, graphs uploaded
            float ms = 0.f;
            timed_one(q, 0, ms);
        }
        int rounds = 1;
        for (int round = 0; round < rounds; ++round) {
            for (size_t q = 0; q < js.size(); ++q) {
                float ms = 0.f;
                if (!timed_one(q, round + 1, ms)) continue;
                fastest[q] = std::min(fastest[q], ms);
                if (round == 0 && ms < 10.f) rounds = 7;
            }
        }
        if (flush) cudaFree(flush);
        for (cudaGraphExec_t x : gx)
            if (x) cudaGraphExecDestroy(x);
        if (cs) cudaStreamDestroy(cs);
        // within 3 % of the fastest, the fewest passes: fewer launches and
        // less kernel code to fetch when the caches are cold, which the
        // back-to-back replays above do not see
        float fmin = 1e30f;
        for (float f : fastest) fmin = std::min(fmin, f);
        int pick = -1;
        for (size_t q = 0; q < js.size(); ++q) {
            if (fastest[q] > 1.03f * fmin) continue;
            if (pick < 0 || js[q].first->passes.size() < js[pick].first->passes.size() ||
                (js[q].first->passes.size() == js[pick].first->passes.size() && fastest[q] < fastest[pick]))
                pick = (int)q;
        }
        if (pick >= 0 && fastest[pick] < best) {
            best = fastest[pick];
            bt.k = js[pick].second.k;
            bt.low = js[pick].second.low;
            bt.M = js[pick].second.M;
            bt.jit = 1;
        }
    }
    g_tracer = saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (bt.k) {
        // keep what other tuners recorded for the plan (whole-row kernel, dense blocks)
        TileTune &t = tuned[p.key ^ (sizeof(R) == 8 ? 1ull : 0ull)];
        bt.rows_jit = t.rows_jit;
        bt.dense = t.dense;
        t = bt;
    }
    return cudaSuccess;
}

#define DQ_INST(R)                                                                                            \
    template cudaError_t tile_apply<R>(TileCache &, std::unordered_map<uint64_t, TileTune> &, const Plan &,   \
                                       const void *, void *, int, void *, int, cudaStream_t, int64_t *);     \
    template cudaError_t tile_autotune<R>(TileCache &, std::unordered_map<uint64_t, TileTune> &, const Plan &, \
                                          const void *, void *, int, void *, int, cudaStream_t, int64_t *, bool); \
    template cudaError_t tile_apply_expect<R>(TileCache &, std::unordered_map<uint64_t, TileTune> &,             \
                                              const Plan &, const void *, void *, int,                         \
                                              const std::vector<DevTerm> &, const DevTerm *, const int32_t *,  \
                                              int, double *, double *, int, cudaStream_t, int64_t *, bool);
DQ_INST(float)
DQ_INST(double)
#undef DQ_INST

}  // namespace dq
