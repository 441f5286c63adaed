// In-register gate engine shared by the tile kernels and the whole-row kernel.
//
// A block of 2^k amplitudes (a tile, or a whole row) is spread over the
// threads of a CTA: local index bits 0..4 select the lane, M "register bits"
// B[0..M-1] select one of the 2^M amplitudes a thread holds, the remaining
// bits select the warp.  A gate whose non-diagonal bit is a register bit is
// register arithmetic; on a lane bit it exchanges amplitudes with warp
// shuffles; diagonal gates (and controls) on any bit become per-element
// factors (predicates).  Changing the set of register bits is the only
// operation that goes through shared memory.
//
// Operations are decoded on the host against the register layout they run
// in (handler id, ready-made control mask), so the device dispatches with a
// single switch into straight-line code.
#pragma once

#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <unordered_map>
#include <vector>
#endif

#include "dq_common.cuh"

namespace dq {

constexpr int kLaneBits = 5;

// Handlers: pair updates on register position P (uncontrolled REAL and DIAG
// take straight-line paths; controlled ones and GEN/ANTI take branch-free
// selects on the control mask), lane-bit updates, and a diagonal factor that
// is uniform for the thread.
enum Handler : int16_t {
    H_REAL = 0,     // + P, uncontrolled
    H_GEN = 5,      // + P
    H_ANTI = 10,    // + P
    H_DIAG = 15,    // + P, uncontrolled
    H_CREAL = 20,   // + P, controlled
    H_CDIAG = 25,   // + P, controlled
    H_LREAL = 30,
    H_LGEN = 31,
    H_LANTI = 32,
    H_DUNI = 33,
    H_FAN = 34,     // first op of a controlled-phase fan (see decode_fans)
    H_FANM = 35,    // further members of a fan (consumed by its first op)
    H_PDIAG = 36,   // parity-diagonal op (see parity_triple)
};

// Parity-diagonal ops.  CNOT(c -> t), a diagonal D = diag(d0, d1) on t,
// CNOT(c -> t) is the diagonal op that multiplies an amplitude by d0 when
// its bits t and c are equal and by d1 when they differ (the CNOT maps bit t
// to t xor c for D and back), with D's generator and gradient slot.  The
// fused planners replace such triples (RZZ, the inner part of RXX and RYY,
// phase-flip superoperators of density circuits) by one op that needs no
// tile or register bit; GOp carries t in (tl, tg) and c in (cl, cg).
template <typename G>
inline bool parity_triple(const G &a, const G &b, const G &c) {
    return a.kind == DQ_CNOT && c.kind == DQ_CNOT && a.t == c.t && a.c == c.c && a.c >= 0 && b.cls == CLS_DIAG &&
           b.c < 0 && b.t == a.t;
}

// One operation decoded for one register layout.  32 bytes.
struct EOp {
    int16_t h;       // Handler
    int16_t kind;    // dq_gate_kind (gradient generator)
    uint32_t cmc;    // control element mask (register-bit control), ~0 when uncontrolled
    int8_t cmode;    // 0: use cmc; 1: control = local bit carg of the thread; 2: global bit carg of the block base
    int8_t carg;
    int8_t tmode;    // H_DUNI target: 1: local bit targ of the thread; 2: global bit targ of the block base
    int8_t targ;     // lane bit (lane handlers) or the H_DUNI target bit
    int32_t coef;    // Mat2 index (row 0)
    int32_t rowstep; // Mat2 row stride
    int32_t slot;    // gradient accumulator or -1
    int32_t pad[2];
};

// Undecoded gate operation (bit positions in the block).
struct GOp {
    int cls;         // GateClass (never CLS_SWAP)
    int tl;          // target local bit or -1 (outside the block, diagonal only)
    int tg;          // target global bit
    int cl;          // control local bit or -1
    int cg;          // control global bit or -1 (none)
    int kind, coef, rowstep, slot;
    int gi;          // plan gate it comes from (a parity triple: its first CNOT; host inspection)
};

// A run of operations executed with one register layout.
struct ESeg {
    int32_t op0, nops;
    int8_t B[8];
};

#ifndef __CUDACC_RTC__   // host-side decoding (not part of run-time compiled kernels)
// Host decode of a gate against a layout with register bits B[0..M-1].
inline EOp decode_op(const GOp &g, const int8_t *B, int M) {
    auto pos = [&](int j) {
        for (int i = 0; i < M; ++i)
            if (B[i] == j) return i;
        return -1;
    };
    static const uint32_t regmask_h[5] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u, 0xFFFF0000u};
    EOp o{};
    o.kind = (int16_t)g.kind;
    o.coef = g.coef;
    o.rowstep = g.rowstep;
    o.slot = g.slot;
    o.cmc = ~0u;
    o.cmode = 0;
    if (g.cg >= 0) {
        if (g.cl >= 0) {
            const int pc = pos(g.cl);
            if (pc >= 0) {
                o.cmc = regmask_h[pc];
            } else {
                o.cmode = 1;
                o.carg = (int8_t)g.cl;
            }
        } else {
            o.cmode = 2;
            o.carg = (int8_t)g.cg;
        }
    }
    if (g.cls == CLS_PDIAG) {
        // a non-register bit's location: thread-local (mode 1) or block (mode 2)
        auto where = [&](int lbit, int gbit, int8_t &mode, int8_t &arg) {
            if (lbit >= 0) {
                mode = 1;
                arg = (int8_t)lbit;
            } else {
                mode = 2;
                arg = (int8_t)gbit;
            }
        };
        const int pt = g.tl >= 0 ? pos(g.tl) : -1, pc = g.cl >= 0 ? pos(g.cl) : -1;
        // cmc: element mask of the register part of the parity (used in reverse)
        o.cmc = (pt >= 0 ? regmask_h[pt] : 0u) ^ (pc >= 0 ? regmask_h[pc] : 0u);
        o.h = H_PDIAG;
        if (pt < 0) where(g.tl, g.tg, o.tmode, o.targ);
        if (pc < 0) where(g.cl, g.cg, o.cmode, o.carg);
        return o;
    }
    const bool ctrl = g.cg >= 0;
    if (g.cls == CLS_DIAG) {
        const int pt = g.tl >= 0 ? pos(g.tl) : -1;
        if (pt >= 0) {
            o.h = (int16_t)((ctrl ? H_CDIAG : H_DIAG) + pt);
        } else {
            o.h = H_DUNI;
            if (g.tl >= 0) {
                o.tmode = 1;
                o.targ = (int8_t)g.tl;
            } else {
                o.tmode = 2;
                o.targ = (int8_t)g.tg;
            }
        }
        return o;
    }
    if (g.tl < kLaneBits) {
        o.h = g.cls == CLS_ANTI ? H_LANTI : (g.cls == CLS_REAL ? H_LREAL : H_LGEN);
        o.targ = (int8_t)g.tl;
        return o;
    }
    const int p = pos(g.tl);   // the planners guarantee p >= 0
    const int base = g.cls == CLS_ANTI ? H_ANTI : (g.cls == CLS_REAL ? (ctrl ? H_CREAL : H_REAL) : H_GEN);
    o.h = (int16_t)(base + (p < 0 ? 0 : p));
    return o;
}

// Controlled-phase fans.  Consecutive CP gates (no gradient, shared angle)
// that all touch one common qubit q commute and multiply to
//     diag: amplitude * prod_j e^{i phi_j b_j}  when b_q = 1,
// so a run of them is decoded as one fan: its first op (H_FAN) carries the
// location of q in (cmode, carg) (0: register position, 1: thread-local bit,
// 2: block bit), the register positions of members in cmc, and the member
// count in pad[0]; every op of the run (H_FAN then H_FANM) carries its member
// qubit's location in (tmode, targ) and its own coefficient (the CP block,
// whose m[3] is e^{i phi}).  Members on register bits come first, in position
// order.  The run keeps its length, so op indices do not move.
inline int fan_loc(int lbit, int gbit, const int8_t *B, int M, int8_t &mode, int8_t &arg) {
    if (lbit >= 0)
        for (int i = 0; i < M; ++i)
            if (B[i] == lbit) {
                mode = 0;
                arg = (int8_t)i;
                return i;
            }
    if (lbit >= 0) {
        mode = 1;
        arg = (int8_t)lbit;
    } else {
        mode = 2;
        arg = (int8_t)gbit;
    }
    return -1;
}

inline bool fan_member(const GOp &g) { return g.cls == CLS_DIAG && g.kind == DQ_CP && g.slot < 0 && g.rowstep == 0; }

// Decode ops [i0, i1) of `g` against register layout B, fusing CP runs of at
// least kMinFan gates into fans; appends exactly i1 - i0 ops to `out`.
constexpr int kMinFan = 3;
inline void decode_with_fans(const std::vector<GOp> &g, int i0, int i1, const int8_t *B, int M,
                             std::vector<EOp> &out) {
    int i = i0;
    while (i < i1) {
        int end = i;
        int q = -1;
        if (fan_member(g[i])) {
            // longest run from i sharing one qubit
            for (int cand : {g[i].tg, g[i].cg}) {
                int e = i;
                while (e < i1 && fan_member(g[e]) && (g[e].tg == cand || g[e].cg == cand)) ++e;
                if (e - i > end - i) {
                    end = e;
                    q = cand;
                }
            }
        }
        if (end - i < kMinFan) {
            out.push_back(decode_op(g[i], B, M));
            ++i;
            continue;
        }
        // members: the other qubit of each CP, register members first
        struct Mem { int pos, lbit, gbit, idx; };
        std::vector<Mem> mem;
        int qlbit = -1;
        for (int j = i; j < end; ++j) {
            const bool qt = g[j].tg == q;
            const int ol = qt ? g[j].cl : g[j].tl, og = qt ? g[j].cg : g[j].tg;
            if (qlbit < 0) qlbit = qt ? g[j].tl : g[j].cl;
            int8_t md, ar;
            const int pos = fan_loc(ol, og, B, M, md, ar);
            mem.push_back({pos, ol, og, j});
        }
        std::stable_sort(mem.begin(), mem.end(), [](const Mem &a, const Mem &b) {
            const int ka = a.pos >= 0 ? a.pos : 64, kb = b.pos >= 0 ? b.pos : 64;
            return ka < kb;
        });
        uint32_t rmask = 0;
        for (const Mem &x : mem)
            if (x.pos >= 0) rmask |= 1u << x.pos;
        for (size_t j = 0; j < mem.size(); ++j) {
            const GOp &src = g[mem[j].idx];
            EOp o{};
            o.h = (int16_t)(j == 0 ? H_FAN : H_FANM);
            o.kind = (int16_t)src.kind;
            o.coef = src.coef;
            o.rowstep = 0;
            o.slot = -1;
            fan_loc(mem[j].lbit, mem[j].gbit, B, M, o.tmode, o.targ);
            if (j == 0) {
                fan_loc(qlbit, q, B, M, o.cmode, o.carg);
                o.cmc = rmask;
                o.pad[0] = (int32_t)mem.size();
            }
            out.push_back(o);
        }
        i = end;
    }
}

// Reorders ops into another valid order that changes the register layout
// less often.  Two ops must keep their order when they share a qubit on which
// at least one of them is not diagonal (a control acts diagonally on its
// qubit; DIAG ops on every qubit they touch).  List scheduling: among the
// ops whose predecessors are done, run those that need no new register bit
// (diagonal, lane-bit or already-resident targets) first, in circuit order;
// otherwise take the earliest ready op, adding its bit while fewer than M
// are held, else starting a new layout with it.
inline void schedule_for_layouts(std::vector<GOp> &ops, int M, int lane_bits) {
    const int n = (int)ops.size();
    if (n < 3 || M < 1) return;
    std::vector<std::vector<int>> succ(n);
    std::vector<int> indeg(n, 0);
    std::unordered_map<int, int> last_nd;                 // qubit -> last op not diagonal on it
    std::unordered_map<int, std::vector<int>> diag_since; // qubit -> diagonal ops since then
    auto edge = [&](int a, int b) {
        succ[a].push_back(b);
        ++indeg[b];
    };
    for (int j = 0; j < n; ++j) {
        const GOp &o = ops[j];
        int qs[2] = {o.tg, o.cg};
        bool nd[2] = {!cls_diagonal(o.cls), false};
        for (int t = 0; t < 2; ++t) {
            const int q = qs[t];
            if (q < 0) continue;
            auto it = last_nd.find(q);
            if (it != last_nd.end()) edge(it->second, j);
            if (nd[t]) {
                for (int d : diag_since[q]) edge(d, j);
                diag_since[q].clear();
                last_nd[q] = j;
            } else {
                diag_since[q].push_back(j);
            }
        }
    }
    auto need = [&](const GOp &o) { return (!cls_diagonal(o.cls) && o.tl >= lane_bits) ? o.tl : -1; };
    std::vector<int> ready, order;
    for (int j = 0; j < n; ++j)
        if (!indeg[j]) ready.push_back(j);
    std::vector<int> B;
    order.reserve(n);
    while (!ready.empty()) {
        std::sort(ready.begin(), ready.end());
        int pick = -1;
        for (int j : ready) {
            const int b = need(ops[j]);
            if (b < 0 || std::find(B.begin(), B.end(), b) != B.end()) {
                pick = j;
                break;
            }
        }
        if (pick < 0) {
            // a new bit: the one most ready ops need (earliest on ties); a full
            // set starts over with the most needed bits
            std::vector<std::pair<int, int>> cnt;   // (bit, count) in first-need order
            for (int j : ready) {
                const int b = need(ops[j]);
                auto it = std::find_if(cnt.begin(), cnt.end(), [&](const std::pair<int, int> &x) { return x.first == b; });
                if (it == cnt.end()) cnt.push_back({b, 1});
                else ++it->second;
            }
            std::stable_sort(cnt.begin(), cnt.end(),
                             [](const std::pair<int, int> &a, const std::pair<int, int> &b) { return a.second > b.second; });
            if ((int)B.size() >= M) {
                B.clear();
                for (size_t i = 0; i < cnt.size() && (int)B.size() < M; ++i) B.push_back(cnt[i].first);
            } else {
                B.push_back(cnt[0].first);
            }
            for (int j : ready)
                if (need(ops[j]) == cnt[0].first) {
                    pick = j;
                    break;
                }
        }
        ready.erase(std::find(ready.begin(), ready.end(), pick));
        order.push_back(pick);
        for (int k : succ[pick])
            if (--indeg[k] == 0) ready.push_back(k);
    }
    if ((int)order.size() != n) return;   // (cannot happen: the graph follows circuit order)
    std::vector<GOp> out(n);
    for (int i = 0; i < n; ++i) out[i] = ops[order[i]];
    ops.swap(out);
}

// Rotation pairs.  An uncontrolled REAL op (RY, H) whose next op on the same
// target is an uncontrolled DIAG op (RZ, Z, S) commutes that op up to itself
// (the ops in between act on other qubits).  In the reverse sweep the two run
// as one register sweep that un-applies both and forms both gradients.
// pair_real_diag reorders `ops` so that every such partner directly follows
// its head and returns the head flags; the reverse decoders then mark the
// DIAG op (pad[1] = 1; it runs first there) when both ops share a register
// layout and decode to matching handlers.
inline std::vector<char> pair_real_diag(std::vector<GOp> &ops, int i0 = 0, int i1 = -1) {
    if (i1 < 0) i1 = (int)ops.size();
    std::vector<char> head(ops.size(), 0);
    for (int i = i0; i < i1; ++i) {
        const GOp a = ops[i];
        if (a.cls != CLS_REAL || a.cg >= 0 || a.tl < 0) continue;
        for (int j = i + 1; j < i1; ++j) {
            const GOp &b = ops[j];
            if (b.tg != a.tg && b.cg != a.tg) continue;
            if (b.cls == CLS_DIAG && b.cg < 0 && b.tg == a.tg) {
                const GOp moved = b;
                for (int k = j; k > i + 1; --k) ops[k] = ops[k - 1];
                ops[i + 1] = moved;
                head[i] = 1;
            }
            break;
        }
    }
    return head;
}

// Host inspection: the plan gate of every op in `ops` order, flagged (bit 0:
// one gate of a parity-diagonal triple, which is listed as its three gates;
// bit 1: one of the three CNOTs a SWAP runs as).  `gates` holds the plan's
// gates (their class tells SWAPs apart).
template <typename Gates>
inline void record_order(const std::vector<GOp> &ops, const Gates &gates, std::vector<int> &order,
                         std::vector<char> &flags) {
    for (const GOp &o : ops) {
        if (o.cls == CLS_PDIAG) {
            for (int j = 0; j < 3; ++j) {
                order.push_back(o.gi + j);
                flags.push_back(1);
            }
            continue;
        }
        order.push_back(o.gi);
        flags.push_back(gates[o.gi].cls == CLS_SWAP ? 2 : 0);
    }
}

inline bool pair_handlers_match(const EOp &real, const EOp &diag) {
    if (real.h >= H_REAL && real.h < H_REAL + 5) return diag.h == H_DIAG + (real.h - H_REAL);
    if (real.h == H_LREAL) return diag.h == H_DUNI && diag.tmode == 1 && diag.targ == real.targ && diag.cmode == 0 &&
                                  diag.cmc == ~0u;
    return false;
}

#endif  // __CUDACC_RTC__

struct Layout {
    uint32_t tb;     // this thread's local index with register bits zero
    uint32_t off[8]; // local offset of register bit i
#ifdef DQ_BOUNDS_BUILD
    uint32_t lim;    // 2^k: the buffer's amplitudes (bounds-checking build)
#endif
};

__device__ __forceinline__ Layout make_layout(const ESeg &sg, int M, int k, int lane, int warp) {
    Layout L;
    uint32_t inB = 0;
    for (int i = 0; i < M; ++i) {
        const int b = sg.B[i];
        L.off[i] = 1u << b;
        inB |= 1u << b;
    }
    uint32_t tb = (uint32_t)lane;
    int wi = 0;
    for (int b = kLaneBits; b < k; ++b) {
        if ((inB >> b) & 1) continue;
        tb |= (uint32_t)((warp >> wi) & 1) << b;
        ++wi;
    }
    L.tb = tb;
#ifdef DQ_BOUNDS_BUILD
    L.lim = 1u << k;
#endif
    return L;
}

template <int M>
__device__ __forceinline__ uint32_t reg_off(const Layout &L, int e) {
    uint32_t o = 0;
#pragma unroll
    for (int i = 0; i < M; ++i)
        if ((e >> i) & 1) o |= L.off[i];
    return o;
}

// Every index of a layout is tb with a subset of the register offsets set,
// so none exceeds tb | (all offsets): the bounds-checking build checks that
// one index per load or store.
template <int M>
__device__ __forceinline__ bool eng_layout_in_bounds(const Layout &L) {
#ifdef DQ_BOUNDS_BUILD
    return DQ_INB(L.tb | reg_off<M>(L, (1 << M) - 1), L.lim);
#else
    (void)L;
    return true;
#endif
}

template <typename R, int M>
__device__ __forceinline__ void eng_load(cx<R> (&a)[1 << M], const cx<R> *buf, const Layout &L) {
    if (!eng_layout_in_bounds<M>(L)) return;
#pragma unroll
    for (int e = 0; e < (1 << M); ++e) a[e] = buf[L.tb | reg_off<M>(L, e)];
}

template <typename R, int M>
__device__ __forceinline__ void eng_store(const cx<R> (&a)[1 << M], cx<R> *buf, const Layout &L) {
    if (!eng_layout_in_bounds<M>(L)) return;
#pragma unroll
    for (int e = 0; e < (1 << M); ++e) buf[L.tb | reg_off<M>(L, e)] = a[e];
}

template <typename T> __device__ __forceinline__ T shfl_xor_cx(T v, int m);
template <> __device__ __forceinline__ float2 shfl_xor_cx<float2>(float2 v, int m) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
template <> __device__ __forceinline__ double2 shfl_xor_cx<double2>(double2 v, int m) {
    return make_double2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

__device__ __forceinline__ uint32_t op_cmask(const EOp &o, const Layout &L, uint64_t base) {
    if (o.cmode == 0) return o.cmc;
    if (o.cmode == 1) return ((L.tb >> o.carg) & 1) ? ~0u : 0u;
    return ((base >> o.carg) & 1) ? ~0u : 0u;
}

// ---------------------------------------------------------------------------
// forward application
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T sel(bool c, T x, T y) { return c ? x : y; }

// Uncontrolled pair update on register position P.
template <typename R, int M, int P, int CLS>
__device__ __forceinline__ void pairs_at(cx<R> (&a)[1 << M], const Mat2<R> &u) {
#pragma unroll
    for (int e0 = 0; e0 < (1 << M); ++e0) {
        if (e0 & (1 << P)) continue;
        apply2<R, CLS>(u, a[e0], a[e0 | (1 << P)]);
    }
}

// Pair update on the elements whose control bit (mask cm) is set: both
// results are formed and selected, so lanes never diverge.
template <typename R, int M, int P, int CLS>
__device__ __forceinline__ void pairs_sel(cx<R> (&a)[1 << M], const Mat2<R> &u, uint32_t cm) {
#pragma unroll
    for (int e0 = 0; e0 < (1 << M); ++e0) {
        if (e0 & (1 << P)) continue;
        const int e1 = e0 | (1 << P);
        const bool c = (cm >> e0) & 1;
        cx<R> b0 = a[e0], b1 = a[e1];
        apply2<R, CLS>(u, b0, b1);
        a[e0] = sel(c, b0, a[e0]);
        a[e1] = sel(c, b1, a[e1]);
    }
}

template <typename R, int M, int P>
__device__ __forceinline__ void diag_at(cx<R> (&a)[1 << M], const Mat2<R> &u) {
#pragma unroll
    for (int e = 0; e < (1 << M); ++e) a[e] = cmul(((e >> P) & 1) ? u.m[3] : u.m[0], a[e]);
}

template <typename R, int M, int P>
__device__ __forceinline__ void diag_sel(cx<R> (&a)[1 << M], const Mat2<R> &u, uint32_t cm) {
#pragma unroll
    for (int e = 0; e < (1 << M); ++e) a[e] = sel((cm >> e) & 1, cmul(((e >> P) & 1) ? u.m[3] : u.m[0], a[e]), a[e]);
}

template <typename R, int M, int CLS>
__device__ __forceinline__ void lane_at(cx<R> (&a)[1 << M], const Mat2<R> &u, int j, int lane, uint32_t cm) {
    const bool hi = (lane >> j) & 1;
    const cx<R> cs = hi ? u.m[3] : u.m[0];
    const cx<R> cp = hi ? u.m[2] : u.m[1];
    const int m = 1 << j;
#pragma unroll
    for (int e = 0; e < (1 << M); ++e) {
        const cx<R> p = shfl_xor_cx(a[e], m);
        cx<R> r;
        if (CLS == CLS_ANTI) r = p;
        else if (CLS == CLS_REAL) r = mk<R>(cs.x * a[e].x + cp.x * p.x, cs.x * a[e].y + cp.x * p.y);
        else r = cadd(cmul(cs, a[e]), cmul(cp, p));
        a[e] = sel((cm >> e) & 1, r, a[e]);
    }
}

template <typename R, int M>
__device__ __forceinline__ void diag_uni(cx<R> (&a)[1 << M], const Mat2<R> &u, const EOp &o, const Layout &L,
                                         uint64_t base, uint32_t cm) {
    const int t = o.tmode == 1 ? (int)((L.tb >> o.targ) & 1) : (int)((base >> o.targ) & 1);
    const cx<R> f = t ? u.m[3] : u.m[0];
#pragma unroll
    for (int e = 0; e < (1 << M); ++e) a[e] = sel((cm >> e) & 1, cmul(f, a[e]), a[e]);
}

// Parity-diagonal ops (see parity_triple).  uni_bit reads a thread-uniform
// bit (mode 1: thread-local index bit, mode 2: block base bit).
__device__ __forceinline__ int uni_bit(int mode, int arg, const Layout &L, uint64_t base) {
    return mode == 1 ? (int)((L.tb >> arg) & 1) : (int)((base >> arg) & 1);
}

// Forward parity-diagonal op: the element mask cmc holds the register part
// of the parity (set at decode), (tmode, targ) and (cmode, carg) the bits
// that are thread-uniform (mode 0: none).  One compact body for every
// placement of the two bits (code size matters more than the selects).
template <typename R, int M>
__device__ __forceinline__ void eng_pdiag(cx<R> (&a)[1 << M], const EOp &o, const Mat2<R> &u, uint64_t base,
                                          const Layout &L) {
    const int upar = (o.tmode ? uni_bit(o.tmode, o.targ, L, base) : 0) ^ (o.cmode ? uni_bit(o.cmode, o.carg, L, base) : 0);
    const cx<R> fe = upar ? u.m[3] : u.m[0], fo = upar ? u.m[0] : u.m[3];
#pragma unroll
    for (int e = 0; e < (1 << M); ++e) a[e] = cmul(((o.cmc >> e) & 1) ? fo : fe, a[e]);
}

#define DQ_ENG_P(MACRO) MACRO(0) MACRO(1) MACRO(2) MACRO(3) MACRO(4)

// Apply one op (u already daggered by the caller when un-applying).
// Uncontrolled REAL and DIAG ops run straight-line code; the others take the
// control mask as selects, so every lane runs the same instructions and the
// lane handlers' full-mask shuffles stay convergent, and a warp whose
// controls are all off skips the op (a warp-uniform vote).
// PD: the kernel's programs may hold parity-diagonal ops (kernels are
// compiled with and without them, to keep the common code small).
template <typename R, int M, bool PD = false>
__device__ __forceinline__ void eng_apply(cx<R> (&a)[1 << M], const EOp &o, const Mat2<R> &u, uint64_t base,
                                          const Layout &L, int lane) {
    if (o.h < H_GEN) {
        switch (o.h) {
#define DQ_CASE(P) \
        case H_REAL + P: if (P < M) pairs_at<R, M, (P < M ? P : 0), CLS_REAL>(a, u); break;
        DQ_ENG_P(DQ_CASE)
#undef DQ_CASE
        }
        return;
    }
    if (o.h >= H_DIAG && o.h < H_CREAL) {
        switch (o.h) {
#define DQ_CASE(P) \
        case H_DIAG + P: if (P < M) diag_at<R, M, (P < M ? P : 0)>(a, u); break;
        DQ_ENG_P(DQ_CASE)
#undef DQ_CASE
        }
        return;
    }
    if (PD && o.h == H_PDIAG) {
        eng_pdiag<R, M>(a, o, u, base, L);
        return;
    }
    if (o.h >= H_FAN) return;   // fans are run by eng_fan from their first op
    const uint32_t cm = op_cmask(o, L, base);
    if (__all_sync(0xffffffffu, cm == 0)) return;
    switch (o.h) {
#define DQ_CASE(P)                                                                                  \
    case H_GEN + P: if (P < M) pairs_sel<R, M, (P < M ? P : 0), CLS_GENERAL>(a, u, cm); break;      \
    case H_ANTI + P: if (P < M) pairs_sel<R, M, (P < M ? P : 0), CLS_ANTI>(a, u, cm); break;        \
    case H_CREAL + P: if (P < M) pairs_sel<R, M, (P < M ? P : 0), CLS_REAL>(a, u, cm); break;       \
    case H_CDIAG + P: if (P < M) diag_sel<R, M, (P < M ? P : 0)>(a, u, cm); break;
        DQ_ENG_P(DQ_CASE)
#undef DQ_CASE
    case H_LREAL: lane_at<R, M, CLS_REAL>(a, u, o.targ, lane, cm); break;
    case H_LGEN: lane_at<R, M, CLS_GENERAL>(a, u, o.targ, lane, cm); break;
    case H_LANTI: lane_at<R, M, CLS_ANTI>(a, u, o.targ, lane, cm); break;
    default: diag_uni<R, M>(a, u, o, L, base, cm); break;
    }
}

// A controlled-phase fan (ops[0] is its H_FAN op, cf the coefficients of
// its ops): every amplitude with b_q = 1 is multiplied by F * prod of the
// register members' phases whose bits are set in it, F being the product of
// the phases of members on thread or block bits that are set.  Thread-
// uniform branches only (no shuffles), so lanes may diverge.
template <typename R, int M, int QP>
__device__ __forceinline__ void fan_elems(cx<R> (&a)[1 << M], const cx<R> &F, const cx<R> (&wp)[M]) {
#pragma unroll
    for (int e = 0; e < (1 << M); ++e) {
        if (QP >= 0 && !((e >> QP) & 1)) continue;
        cx<R> f = F;
#pragma unroll
        for (int p = 0; p < M; ++p)
            if (p != QP && ((e >> p) & 1)) f = cmul(f, wp[p]);
        a[e] = cmul(f, a[e]);
    }
}

template <typename R, int M>
__device__ __forceinline__ int eng_fan(cx<R> (&a)[1 << M], const EOp *ops, const Mat2<R> *cf, uint64_t base,
                                       const Layout &L) {
    const EOp h = ops[0];
    const int m = h.pad[0];
    if (h.cmode != 0) {
        const int qb = h.cmode == 1 ? (int)((L.tb >> h.carg) & 1) : (int)((base >> h.carg) & 1);
        if (!qb) return m;
    }
    cx<R> wp[M];
    int j = 0;
#pragma unroll
    for (int p = 0; p < M; ++p) {
        if ((h.cmc >> p) & 1) {
            wp[p] = cf[j].m[3];
            ++j;
        } else {
            wp[p] = mk<R>(R(1), R(0));
        }
    }
    cx<R> F = mk<R>(R(1), R(0));
    for (; j < m; ++j) {
        const EOp e = ops[j];
        const int bit = e.tmode == 1 ? (int)((L.tb >> e.targ) & 1) : (int)((base >> e.targ) & 1);
        if (bit) F = cmul(F, cf[j].m[3]);
    }
    switch (h.cmode == 0 ? (int)h.carg : -1) {
    case 0: fan_elems<R, M, 0>(a, F, wp); break;
    case 1: if (M > 1) fan_elems<R, M, (M > 1 ? 1 : 0)>(a, F, wp); break;
    case 2: if (M > 2) fan_elems<R, M, (M > 2 ? 2 : 0)>(a, F, wp); break;
    case 3: if (M > 3) fan_elems<R, M, (M > 3 ? 3 : 0)>(a, F, wp); break;
    case 4: if (M > 4) fan_elems<R, M, (M > 4 ? 4 : 0)>(a, F, wp); break;
    default: fan_elems<R, M, -1>(a, F, wp); break;
    }
    return m;
}

// ---------------------------------------------------------------------------
// adjoint step: gradient partial 2 Im <lam|G|psi> (after the gate), then
// un-apply U^dagger on both register sets.  Returns this thread's partial.
// ---------------------------------------------------------------------------
// 2 Im <l|G|p> on one amplitude pair for the parametric kinds of a class:
// REAL: RY/CRY (G = Y/2), GENERAL: RX/CRX (G = X/2).
template <typename R, int CLS>
__device__ __forceinline__ R grad_cls(cx<R> l0, cx<R> l1, cx<R> p0, cx<R> p1) {
    if (CLS == CLS_REAL) return re_conj_mul(l1, p0) - re_conj_mul(l0, p1);
    if (CLS == CLS_GENERAL) return im_conj_mul(l0, p1) + im_conj_mul(l1, p0);
    return R(0);
}

// Uncontrolled pair update with optional gradient (GRAD compile-time).
template <typename R, int M, int P, int CLS, bool GRAD>
__device__ __forceinline__ R adj_pairs_at(cx<R> (&ps)[1 << M], cx<R> (&ls)[1 << M], const Mat2<R> &ud) {
    R g = R(0);
#pragma unroll
    for (int e0 = 0; e0 < (1 << M); ++e0) {
        if (e0 & (1 << P)) continue;
        const int e1 = e0 | (1 << P);
        if (GRAD) g += grad_cls<R, CLS>(ls[e0], ls[e1], ps[e0], ps[e1]);
        apply2<R, CLS>(ud, ps[e0], ps[e1]);
        apply2<R, CLS>(ud, ls[e0], ls[e1]);
    }
    return g;
}

// Controlled (or GEN/ANTI) pair update: selects on the control mask.
template <typename R, int M, int P, int CLS, bool GRAD>
__device__ __forceinline__ R adj_pairs_sel(cx<R> (&ps)[1 << M], cx<R> (&ls)[1 << M], const Mat2<R> &ud,
                                           uint32_t cm) {
    R g = R(0);
#pragma unroll
    for (int e0 = 0; e0 < (1 << M); ++e0) {
        if (e0 & (1 << P)) continue;
        const int e1 = e0 | (1 << P);
        const bool c = (cm >> e0) & 1;
        if (GRAD) g += c ? grad_cls<R, CLS>(ls[e0], ls[e1], ps[e0], ps[e1]) : R(0);
        cx<R> p0 = ps[e0], p1 = ps[e1], l0 = ls[e0], l1 = ls[e1];
        apply2<R, CLS>(ud, p0, p1);
        apply2<R, CLS>(ud, l0, l1);
        ps[e0] = sel(c, p0, ps[e0]);
        ps[e1] = sel(c, p1, ps[e1]);
        ls[e0] = sel(c, l0, ls[e0]);
        ls[e1] = sel(c, l1, ls[e1]);
    }
    return g;
}

// Diagonal generator weights: RZ/CRZ +1 on target 0, -1 on target 1; CP and P 0 / -2.
template <typename R>
__device__ __forceinline__ void diag_weights(int kind, R &w0, R &w1) {
    const bool ph = kind == DQ_CP || kind == DQ_P;
    w0 = ph ? R(0) : R(1);
    w1 = ph ? R(-2) : R(-1);
}

template <typename R, int M, int P, bool GRAD>
__device__ __forceinline__ R adj_diag_at(cx<R> (&ps)[1 << M], cx<R> (&ls)[1 << M], const Mat2<R> &ud, int kind) {
    R g = R(0), w0, w1;
    diag_weights<R>(kind, w0, w1);
#pragma unroll
    for (int e = 0; e < (1 << M); ++e) {
        const bool t = (e >> P) & 1;
        if (GRAD) g += (t ? w1 : w0) * im_conj_mul(ls[e], ps[e]);
        const cx<R> f = t ? ud.m[3] : ud.m[0];
        ps[e] = cmul(f, ps[e]);
        ls[e] = cmul(f, ls[e]);
    }
    return g;
}

template <typename R, int M, int P, bool GRAD>
__device__ __forceinline__ R adj_diag_sel(cx<R> (&ps)[1 << M], cx<R> (&ls)[1 << M], const Mat2<R> &ud, int kind,
                                          uint32_t cm) {
    R g = R(0), w0, w1;
    diag_weights<R>(kind, w0, w1);
#pragma unroll
    for (int e = 0; e < (1 << M); ++e) {
        const bool c = (cm >> e) & 1;
        const bool t = (e >> P) & 1;
        if (GRAD) g += c ? (t ? w1 : w0) * im_conj_mul(ls[e], ps[e]) : R(0);
        const cx<R> f = t ? ud.m[3] : ud.m[0];
        ps[e] = sel(c, cmul(f, ps[e]), ps[e]);
        ls[e] = sel(c, cmul(f, ls[e]), ls[e]);
    }
    return g;
}

template <typename R, int M, bool GRAD>
__device__ __forceinline__ R adj_diag_uni(cx<R> (&ps)[1 << M], cx<R> (&ls)[1 << M], const Mat2<R> &ud, const EOp &o,
                                          const Layout &L, uint64_t base, uint32_t cm) {
    R g = R(0), w0, w1;
    diag_weights<R>(o.kind, w0, w1);
    const int t = o.tmode == 1 ? (int)((L.tb >> o.targ) & 1) : (int)((base >> o.targ) & 1);
    const cx<R> f = t ? ud.m[3] : ud.m[0];
    const R w = t ? w1 : w0;
#pragma unroll
    for (int e = 0; e < (1 << M); ++e) {
        const bool c = (cm >> e) & 1;
        if (GRAD) g += c ? w * im_conj_mul(ls[e], ps[e]) : R(0);
        ps[e] = sel(c, cmul(f, ps[e]), ps[e]);
        ls[e] = sel(c, cmul(f, ls[e]), ls[e]);
    }
    return g;
}

template <typename R, int M, int CLS, bool GRAD>
__device__ __forceinline__ R adj_lane_at(cx<R> (&ps)[1 << M], cx<R> (&ls)[1 << M], const Mat2<R> &ud, int j, int lane,
                                         uint32_t cm) {
    R g = R(0);
    const int m = 1 << j;
    const bool hi = (lane >> j) & 1;
    const cx<R> cs = hi ? ud.m[3] : ud.m[0];
    const cx<R> cp = hi ? ud.m[2] : ud.m[1];
#pragma unroll
    for (int e = 0; e < (1 << M); ++e) {
        const cx<R> pp = shfl_xor_cx(ps[e], m);
        const cx<R> lp = shfl_xor_cx(ls[e], m);
        const bool c = (cm >> e) & 1;
        if (GRAD) g += (c && !hi) ? grad_cls<R, CLS>(ls[e], lp, ps[e], pp) : R(0);
        cx<R> rp, rl;
        if (CLS == CLS_ANTI) {
            rp = pp;
            rl = lp;
        } else if (CLS == CLS_REAL) {
            rp = mk<R>(cs.x * ps[e].x + cp.x * pp.x, cs.x * ps[e].y + cp.x * pp.y);
            rl = mk<R>(cs.x * ls[e].x + cp.x * lp.x, cs.x * ls[e].y + cp.x * lp.y);
        } else {
            rp = cadd(cmul(cs, ps[e]), cmul(cp, pp));
            rl = cadd(cmul(cs, ls[e]), cmul(cp, lp));
        }
        ps[e] = sel(c, rp, ps[e]);
        ls[e] = sel(c, rl, ls[e]);
    }
    return g;
}

// Reverse parity-diagonal op: gradient partial with the generator's weight
// for the amplitude's parity (taken after the gate), then un-apply.  The
// register part of the parity is the element mask cmc (set at decode), the
// thread-uniform part comes from the (tmode, targ) and (cmode, carg) bits
// that are not register bits (mode 0: none).
template <typename R, int M, bool GRAD>
__device__ __forceinline__ R adj_pdiag(cx<R> (&ps)[1 << M], cx<R> (&ls)[1 << M], const EOp &o, const Mat2<R> &ud,
                                       uint64_t base, const Layout &L) {
    const int upar = (o.tmode ? uni_bit(o.tmode, o.targ, L, base) : 0) ^ (o.cmode ? uni_bit(o.cmode, o.carg, L, base) : 0);
    R g = R(0), w0, w1;
    diag_weights<R>(o.kind, w0, w1);
    const cx<R> fe = upar ? ud.m[3] : ud.m[0], fo = upar ? ud.m[0] : ud.m[3];
    const R we = upar ? w1 : w0, wo = upar ? w0 : w1;
#pragma unroll
    for (int e = 0; e < (1 << M); ++e) {
        const bool odd = (o.cmc >> e) & 1;
        if (GRAD) g += (odd ? wo : we) * im_conj_mul(ls[e], ps[e]);
        const cx<R> f = odd ? fo : fe;
        ps[e] = cmul(f, ps[e]);
        ls[e] = cmul(f, ls[e]);
    }
    return g;
}

template <typename R, int M, bool GRAD, bool PD>
__device__ __forceinline__ R eng_adjoint_g(cx<R> (&ps)[1 << M], cx<R> (&ls)[1 << M], const EOp &o, const Mat2<R> &ud,
                                           uint64_t base, const Layout &L, int lane) {
    if (o.h < H_GEN) {
        switch (o.h) {
#define DQ_CASE(P) \
        case H_REAL + P: return P < M ? adj_pairs_at<R, M, (P < M ? P : 0), CLS_REAL, GRAD>(ps, ls, ud) : R(0);
        DQ_ENG_P(DQ_CASE)
#undef DQ_CASE
        }
        return R(0);
    }
    if (o.h >= H_DIAG && o.h < H_CREAL) {
        switch (o.h) {
#define DQ_CASE(P) \
        case H_DIAG + P: return P < M ? adj_diag_at<R, M, (P < M ? P : 0), GRAD>(ps, ls, ud, o.kind) : R(0);
        DQ_ENG_P(DQ_CASE)
#undef DQ_CASE
        }
        return R(0);
    }
    if (PD && o.h == H_PDIAG) return adj_pdiag<R, M, GRAD>(ps, ls, o, ud, base, L);
    const uint32_t cm = op_cmask(o, L, base);
    if (__all_sync(0xffffffffu, cm == 0)) return R(0);   // warp-uniform skip (see eng_apply)
    switch (o.h) {
#define DQ_CASE(P)                                                                                              \
    case H_GEN + P:                                                                                             \
        return P < M ? adj_pairs_sel<R, M, (P < M ? P : 0), CLS_GENERAL, GRAD>(ps, ls, ud, cm) : R(0);          \
    case H_ANTI + P:                                                                                            \
        return P < M ? adj_pairs_sel<R, M, (P < M ? P : 0), CLS_ANTI, false>(ps, ls, ud, cm) : R(0);            \
    case H_CREAL + P:                                                                                           \
        return P < M ? adj_pairs_sel<R, M, (P < M ? P : 0), CLS_REAL, GRAD>(ps, ls, ud, cm) : R(0);             \
    case H_CDIAG + P:                                                                                           \
        return P < M ? adj_diag_sel<R, M, (P < M ? P : 0), GRAD>(ps, ls, ud, o.kind, cm) : R(0);
        DQ_ENG_P(DQ_CASE)
#undef DQ_CASE
    case H_LREAL: return adj_lane_at<R, M, CLS_REAL, GRAD>(ps, ls, ud, o.targ, lane, cm);
    case H_LGEN: return adj_lane_at<R, M, CLS_GENERAL, GRAD>(ps, ls, ud, o.targ, lane, cm);
    case H_LANTI: return adj_lane_at<R, M, CLS_ANTI, false>(ps, ls, ud, o.targ, lane, cm);
    default: return adj_diag_uni<R, M, GRAD>(ps, ls, ud, o, L, base, cm);
    }
}

// One reverse step; the gradient partial is formed only for ops with a slot.
// PD: the kernel's reverse programs may hold parity-diagonal ops (compiled in
// only where they can occur, to keep the other kernels' code small).
template <typename R, int M, bool PD>
__device__ __forceinline__ R eng_adjoint(cx<R> (&ps)[1 << M], cx<R> (&ls)[1 << M], const EOp &o, const Mat2<R> &ud,
                                         uint64_t base, const Layout &L, int lane) {
    return o.slot >= 0 ? eng_adjoint_g<R, M, true, PD>(ps, ls, o, ud, base, L, lane)
                       : eng_adjoint_g<R, M, false, PD>(ps, ls, o, ud, base, L, lane);
}

// ---------------------------------------------------------------------------
// rotation pairs in the reverse sweep (see pair_real_diag)
// ---------------------------------------------------------------------------
// Reverse: un-apply the DIAG op d (daggered matrix dd, generator by kind) and
// then the REAL op r (daggered rr) on one pair sweep; gd / gr receive the
// gradient partials 2 Im <lambda|G|psi> of each (taken after its own gate).
template <typename R, int M, int P, bool GRAD>
__device__ __forceinline__ void adj_pair_reg(cx<R> (&ps)[1 << M], cx<R> (&ls)[1 << M], const Mat2<R> &dd,
                                             const Mat2<R> &rr, int dkind, R &gd, R &gr) {
    R w0, w1;
    diag_weights<R>(dkind, w0, w1);
#pragma unroll
    for (int e0 = 0; e0 < (1 << M); ++e0) {
        if (e0 & (1 << P)) continue;
        const int e1 = e0 | (1 << P);
        cx<R> p0 = ps[e0], p1 = ps[e1], l0 = ls[e0], l1 = ls[e1];
        if (GRAD) gd += w0 * im_conj_mul(l0, p0) + w1 * im_conj_mul(l1, p1);
        p0 = cmul(dd.m[0], p0);
        p1 = cmul(dd.m[3], p1);
        l0 = cmul(dd.m[0], l0);
        l1 = cmul(dd.m[3], l1);
        if (GRAD) gr += grad_cls<R, CLS_REAL>(l0, l1, p0, p1);
        apply2<R, CLS_REAL>(rr, p0, p1);
        apply2<R, CLS_REAL>(rr, l0, l1);
        ps[e0] = p0;
        ps[e1] = p1;
        ls[e0] = l0;
        ls[e1] = l1;
    }
}

template <typename R, int M, bool GRAD>
__device__ __forceinline__ void adj_pair_lane(cx<R> (&ps)[1 << M], cx<R> (&ls)[1 << M], const Mat2<R> &dd,
                                              const Mat2<R> &rr, int dkind, int j, int lane, R &gd, R &gr) {
    R w0, w1;
    diag_weights<R>(dkind, w0, w1);
    const int m = 1 << j;
    const bool hi = (lane >> j) & 1;
    const cx<R> f = hi ? dd.m[3] : dd.m[0];
    const R w = hi ? w1 : w0;
    const R cs = hi ? rr.m[3].x : rr.m[0].x;
    const R cp = hi ? rr.m[2].x : rr.m[1].x;
#pragma unroll
    for (int e = 0; e < (1 << M); ++e) {
        cx<R> p = ps[e], l = ls[e];
        if (GRAD) gd += w * im_conj_mul(l, p);
        p = cmul(f, p);
        l = cmul(f, l);
        const cx<R> pp = shfl_xor_cx(p, m);
        const cx<R> lp = shfl_xor_cx(l, m);
        if (GRAD && !hi) gr += grad_cls<R, CLS_REAL>(l, lp, p, pp);
        ps[e] = mk<R>(cs * p.x + cp * pp.x, cs * p.y + cp * pp.y);
        ls[e] = mk<R>(cs * l.x + cp * lp.x, cs * l.y + cp * lp.y);
    }
}

template <typename R, int M>
__device__ __forceinline__ void eng_adjoint_pair(cx<R> (&ps)[1 << M], cx<R> (&ls)[1 << M], const EOp &d,
                                                 const Mat2<R> &dd, const EOp &r, const Mat2<R> &rr, int lane,
                                                 R &gd, R &gr) {
    gd = R(0);
    gr = R(0);
    const bool grad = d.slot >= 0 || r.slot >= 0;
    if (r.h == H_LREAL) {
        if (grad) adj_pair_lane<R, M, true>(ps, ls, dd, rr, d.kind, r.targ, lane, gd, gr);
        else adj_pair_lane<R, M, false>(ps, ls, dd, rr, d.kind, r.targ, lane, gd, gr);
        return;
    }
    switch (r.h - H_REAL) {
#define DQ_CASE(P)                                                                                      \
    case P:                                                                                             \
        if (P < M) {                                                                                    \
            if (grad) adj_pair_reg<R, M, (P < M ? P : 0), true>(ps, ls, dd, rr, d.kind, gd, gr);        \
            else adj_pair_reg<R, M, (P < M ? P : 0), false>(ps, ls, dd, rr, d.kind, gd, gr);            \
        }                                                                                               \
        break;
        DQ_ENG_P(DQ_CASE)
#undef DQ_CASE
    default: break;
    }
}

// FP32 (or FP64) warp sum.
template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace dq
