// In-register gate engine shared by the tile kernels and the whole-row kernel.
//
// A block of 2^k amplitudes (a tile, or a whole row) is spread over the
// threads of a CTA: local index bits 0..4 select the lane, M "register bits"
// B[0..M-1] select one of the 2^M amplitudes a thread holds, the remaining
// bits select the warp.  A gate whose non-diagonal bit is a register bit is
// register arithmetic; on a lane bit it exchanges amplitudes with warp
// shuffles; diagonal gates (and controls) on any bit become per-element
// factors (predicates) computed from element bit masks.  Changing the set of
// register bits is the only operation that goes through shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dq_common.cuh"

namespace dq {

constexpr int kLaneBits = 5;

// One operation of an engine program.  32 bytes.
struct EOp {
    int8_t cls;      // GateClass (never CLS_SWAP: lowered to three CNOTs)
    int8_t tl;       // target local bit (-1: outside the block; diagonal only)
    int8_t cl;       // control local bit (-1: none or outside the block)
    int8_t hasc;     // 1 when controlled
    int16_t kind;    // dq_gate_kind (gradient generator)
    int16_t pad;
    int32_t tg;      // target global amplitude bit
    int32_t cg;      // control global amplitude bit (-1: none)
    int32_t coef;    // Mat2 index (row 0)
    int32_t rowstep; // Mat2 row stride
    int32_t slot;    // gradient accumulator or -1
    int32_t pad2;
};

// A run of operations executed with one register layout.
struct ESeg {
    int32_t op0, nops;
    int8_t B[8];
};

struct Layout {
    uint32_t tb;     // this thread's local index with register bits zero
    uint64_t posB;   // 4 bits per local bit: register position, 15 = not a register bit
    uint32_t off[8]; // local offset of register bit i
};

__device__ __forceinline__ Layout make_layout(const ESeg &sg, int M, int k, int lane, int warp) {
    Layout L;
    L.posB = ~0ull;
    uint32_t inB = 0;
    for (int i = 0; i < M; ++i) {
        const int b = sg.B[i];
        L.off[i] = 1u << b;
        inB |= 1u << b;
        L.posB &= ~(uint64_t(15) << (4 * b));
        L.posB |= uint64_t(i) << (4 * b);
    }
    uint32_t tb = (uint32_t)lane;
    int wi = 0;
    for (int b = kLaneBits; b < k; ++b) {
        if ((inB >> b) & 1) continue;
        tb |= (uint32_t)((warp >> wi) & 1) << b;
        ++wi;
    }
    L.tb = tb;
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

// Elements e (< 32) whose register bit p is set.
__device__ __forceinline__ uint32_t regmask(int p) {
    return p == 0 ? 0xAAAAAAAAu : p == 1 ? 0xCCCCCCCCu : p == 2 ? 0xF0F0F0F0u : p == 3 ? 0xFF00FF00u : 0xFFFF0000u;
}

__device__ __forceinline__ int pos_in_B(const Layout &L, int j) { return (int)((L.posB >> (4 * j)) & 15); }

// Element mask of "bit is 1" for a local bit j (or, when j < 0, the global
// bit g of the block base).
__device__ __forceinline__ uint32_t bit_mask(int j, int g, uint64_t base, const Layout &L) {
    if (j < 0) return ((base >> g) & 1) ? ~0u : 0u;
    const int pb = pos_in_B(L, j);
    if (pb < 15) return regmask(pb);
    return ((L.tb >> j) & 1) ? ~0u : 0u;
}

template <typename R, int M>
__device__ __forceinline__ void eng_load(cx<R> (&a)[1 << M], const cx<R> *buf, const Layout &L) {
#pragma unroll
    for (int e = 0; e < (1 << M); ++e) a[e] = buf[L.tb | reg_off<M>(L, e)];
}

template <typename R, int M>
__device__ __forceinline__ void eng_store(const cx<R> (&a)[1 << M], cx<R> *buf, const Layout &L) {
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

// ---------------------------------------------------------------------------
// forward application
// ---------------------------------------------------------------------------
template <typename R, int M, int P, bool ANTI>
__device__ __forceinline__ void pairs_at(cx<R> (&a)[1 << M], const Mat2<R> &u, uint32_t cm) {
#pragma unroll
    for (int e0 = 0; e0 < (1 << M); ++e0) {
        if (e0 & (1 << P)) continue;
        if (!((cm >> e0) & 1)) continue;
        const int e1 = e0 | (1 << P);
        if (ANTI) {
            const cx<R> t = a[e0];
            a[e0] = a[e1];
            a[e1] = t;
        } else {
            apply2<R, CLS_GENERAL>(u, a[e0], a[e1]);
        }
    }
}

template <typename R, int M, bool ANTI>
__device__ __forceinline__ void pairs_dispatch(int p, cx<R> (&a)[1 << M], const Mat2<R> &u, uint32_t cm) {
    if (p == 0) pairs_at<R, M, 0, ANTI>(a, u, cm);
    else if (p == 1) pairs_at<R, M, (M > 1 ? 1 : 0), ANTI>(a, u, cm);
    else if (p == 2) pairs_at<R, M, (M > 2 ? 2 : 0), ANTI>(a, u, cm);
    else if (p == 3) pairs_at<R, M, (M > 3 ? 3 : 0), ANTI>(a, u, cm);
    else pairs_at<R, M, (M > 4 ? 4 : 0), ANTI>(a, u, cm);
}

// Gate on lane bit j (partner amplitude in lane ^ (1 << j)).
template <typename R, int M>
__device__ __forceinline__ void lane_apply(cx<R> (&a)[1 << M], const Mat2<R> &u, int j, int lane, uint32_t cm,
                                           bool anti) {
    const bool hi = (lane >> j) & 1;
    const cx<R> cs = hi ? u.m[3] : u.m[0];
    const cx<R> cp = hi ? u.m[2] : u.m[1];
    const int m = 1 << j;
#pragma unroll
    for (int e = 0; e < (1 << M); ++e) {
        const cx<R> p = shfl_xor_cx(a[e], m);
        if (!((cm >> e) & 1)) continue;
        a[e] = anti ? p : cadd(cmul(cs, a[e]), cmul(cp, p));
    }
}

// Apply one op (u already daggered by the caller when un-applying).
template <typename R, int M>
__device__ __forceinline__ void eng_apply(cx<R> (&a)[1 << M], const EOp &o, const Mat2<R> &u, uint64_t base,
                                          const Layout &L, int lane) {
    const uint32_t cm = o.hasc ? bit_mask(o.cl, o.cg, base, L) : ~0u;
    // cm can differ between lanes (control on a lane bit): leave only when the
    // whole warp has nothing to do, so lane operations below keep every lane
    // in their full-mask shuffles.
    if (__all_sync(0xffffffffu, cm == 0)) return;
    if (o.cls == CLS_DIAG) {
        const uint32_t tm = bit_mask(o.tl, o.tg, base, L);
#pragma unroll
        for (int e = 0; e < (1 << M); ++e)
            if ((cm >> e) & 1) a[e] = cmul(((tm >> e) & 1) ? u.m[3] : u.m[0], a[e]);
        return;
    }
    const bool anti = o.cls == CLS_ANTI;
    if (o.tl < kLaneBits) {
        lane_apply<R, M>(a, u, o.tl, lane, cm, anti);
        return;
    }
    const int p = pos_in_B(L, o.tl);
    if (anti) pairs_dispatch<R, M, true>(p, a, u, cm);
    else pairs_dispatch<R, M, false>(p, a, u, cm);
}

// ---------------------------------------------------------------------------
// adjoint step: gradient partial 2 Im <lam|G|psi> (after the gate), then
// un-apply U^dagger on both register sets.  Returns this thread's partial.
// ---------------------------------------------------------------------------
template <typename R, int M, int P>
__device__ __forceinline__ R adj_pairs_at(cx<R> (&ps)[1 << M], cx<R> (&ls)[1 << M], const Mat2<R> &ud, uint32_t cm,
                                          int kind, bool grad, bool anti) {
    R g = R(0);
#pragma unroll
    for (int e0 = 0; e0 < (1 << M); ++e0) {
        if (e0 & (1 << P)) continue;
        if (!((cm >> e0) & 1)) continue;
        const int e1 = e0 | (1 << P);
        if (grad) g += grad_pair<R>(kind, ls[e0], ls[e1], ps[e0], ps[e1]);
        if (anti) {
            cx<R> t = ps[e0]; ps[e0] = ps[e1]; ps[e1] = t;
            t = ls[e0]; ls[e0] = ls[e1]; ls[e1] = t;
        } else {
            apply2<R, CLS_GENERAL>(ud, ps[e0], ps[e1]);
            apply2<R, CLS_GENERAL>(ud, ls[e0], ls[e1]);
        }
    }
    return g;
}

template <typename R, int M>
__device__ __forceinline__ R eng_adjoint(cx<R> (&ps)[1 << M], cx<R> (&ls)[1 << M], const EOp &o, const Mat2<R> &ud,
                                         uint64_t base, const Layout &L, int lane) {
    const bool grad = o.slot >= 0;
    const uint32_t cm = o.hasc ? bit_mask(o.cl, o.cg, base, L) : ~0u;
    R g = R(0);
    if (__all_sync(0xffffffffu, cm == 0)) return g;   // warp-uniform exit (see eng_apply)
    if (o.cls == CLS_DIAG) {
        const uint32_t tm = bit_mask(o.tl, o.tg, base, L);
        // generator weights: RZ/CRZ: +1 on target 0, -1 on target 1; CP: -2 on target 1
        const R w0 = (o.kind == DQ_CP) ? R(0) : R(1);
        const R w1 = (o.kind == DQ_CP) ? R(-2) : R(-1);
#pragma unroll
        for (int e = 0; e < (1 << M); ++e) {
            if (!((cm >> e) & 1)) continue;
            const bool t = (tm >> e) & 1;
            if (grad) g += (t ? w1 : w0) * (ls[e].x * ps[e].y - ls[e].y * ps[e].x);
            const cx<R> f = t ? ud.m[3] : ud.m[0];
            ps[e] = cmul(f, ps[e]);
            ls[e] = cmul(f, ls[e]);
        }
        return g;
    }
    const bool anti = o.cls == CLS_ANTI;
    if (o.tl < kLaneBits) {
        const int j = o.tl, m = 1 << j;
        const bool hi = (lane >> j) & 1;
        const cx<R> cs = hi ? ud.m[3] : ud.m[0];
        const cx<R> cp = hi ? ud.m[2] : ud.m[1];
#pragma unroll
        for (int e = 0; e < (1 << M); ++e) {
            const cx<R> pp = shfl_xor_cx(ps[e], m);
            const cx<R> lp = shfl_xor_cx(ls[e], m);
            if (!((cm >> e) & 1)) continue;
            if (grad && !hi) g += grad_pair<R>(o.kind, ls[e], lp, ps[e], pp);
            if (anti) {
                ps[e] = pp;
                ls[e] = lp;
            } else {
                ps[e] = cadd(cmul(cs, ps[e]), cmul(cp, pp));
                ls[e] = cadd(cmul(cs, ls[e]), cmul(cp, lp));
            }
        }
        return g;
    }
    const int p = pos_in_B(L, o.tl);
    if (p == 0) g = adj_pairs_at<R, M, 0>(ps, ls, ud, cm, o.kind, grad, anti);
    else if (p == 1) g = adj_pairs_at<R, M, (M > 1 ? 1 : 0)>(ps, ls, ud, cm, o.kind, grad, anti);
    else if (p == 2) g = adj_pairs_at<R, M, (M > 2 ? 2 : 0)>(ps, ls, ud, cm, o.kind, grad, anti);
    else if (p == 3) g = adj_pairs_at<R, M, (M > 3 ? 3 : 0)>(ps, ls, ud, cm, o.kind, grad, anti);
    else g = adj_pairs_at<R, M, (M > 4 ? 4 : 0)>(ps, ls, ud, cm, o.kind, grad, anti);
    return g;
}

// FP32 (or FP64) warp sum.
template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace dq
