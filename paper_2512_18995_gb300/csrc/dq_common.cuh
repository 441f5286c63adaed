// Shared device/host definitions of libdq (internal).
//
// Conventions: wire q of an n-qubit row is bit p = n-1-q of the amplitude
// index.  Inside the library every gate is stored by bit position.  A
// complex amplitude is float2 (DQ_C64) or double2 (DQ_C128).
#pragma once

#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#include <stdint.h>
#endif

#include "dq.h"

namespace dq {

// ---------------------------------------------------------------------------
// complex arithmetic on float2 / double2
// ---------------------------------------------------------------------------
template <typename R> struct CT;
template <> struct CT<float> { using type = float2; using unit = float4; };
template <> struct CT<double> { using type = double2; };

template <typename R> using cx = typename CT<R>::type;

template <typename R> __host__ __device__ __forceinline__ cx<R> mk(R x, R y) { cx<R> c; c.x = x; c.y = y; return c; }
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) { a.x *= s; a.y *= s; return a; }

// Re(conj(l) p) and Im(conj(l) p) with each product rounded on its own (no
// FMA contraction).  Sums of the form a*b - c*d then vanish exactly whenever
// the two products are equal: the imaginary part of conj(p) p, or the
// per-term cancellation of a generator's expectation when lambda is a real
// multiple of psi element by element (a diagonal observable).  A contracted
// fma(a, b, -(c*d)) would leave one product's rounding error behind in every
// such term, which a gradient or expectation that is exactly zero does not
// survive in single precision.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
template <typename C> __device__ __forceinline__ auto re_conj_mul(C l, C p) -> decltype(l.x) {
    return mul_rn(l.x, p.x) + mul_rn(l.y, p.y);
}
template <typename C> __device__ __forceinline__ auto im_conj_mul(C l, C p) -> decltype(l.x) {
    return mul_rn(l.x, p.y) - mul_rn(l.y, p.x);
}

// 2x2 block acting on the target qubit (applied on control = |1> for
// controlled kinds).  m[0] m[1] / m[2] m[3] row-major.
template <typename R> struct Mat2 { cx<R> m[4]; };

// Gate classes used to specialise the sweeps.
enum GateClass : int {
    CLS_GENERAL = 0,   // full complex 2x2
    CLS_REAL = 1,      // real 2x2 (H, RY, CRY)
    CLS_DIAG = 2,      // diagonal (Z, S, RZ, CZ, CP, CRZ)
    CLS_ANTI = 3,      // X / CNOT: exchange
    CLS_SWAP = 4,      // SWAP of two qubits
    CLS_PDIAG = 5      // diagonal in the parity of two bits (fused CNOT, diagonal, CNOT; fused engines only)
};

// Classes that act diagonally on every bit they touch.
__host__ __device__ inline bool cls_diagonal(int cls) { return cls == CLS_DIAG || cls == CLS_PDIAG; }

__host__ __device__ inline int gate_class(int kind) {
    switch (kind) {
    case DQ_H: case DQ_RY: case DQ_CRY: return CLS_REAL;
    case DQ_Z: case DQ_S: case DQ_RZ: case DQ_CZ: case DQ_CP: case DQ_CRZ: case DQ_P: return CLS_DIAG;
    case DQ_X: case DQ_CNOT: return CLS_ANTI;
    case DQ_SWAP: return CLS_SWAP;
    default: return CLS_GENERAL;   // Y, RX, CRX
    }
}

__host__ __device__ inline bool kind_controlled(int k) {
    return k == DQ_CNOT || k == DQ_CZ || k == DQ_CP || k == DQ_CRX || k == DQ_CRY || k == DQ_CRZ;
}
__host__ __device__ inline bool kind_parametric(int k) {
    return k == DQ_RX || k == DQ_RY || k == DQ_RZ || k == DQ_CP || k == DQ_CRX || k == DQ_CRY || k == DQ_CRZ ||
           k == DQ_P;
}

// Target block of `kind` at angle t, evaluated in double and rounded to R.
// R_P(t) = cos(t/2) I - i sin(t/2) P;  CP(t) and P(t): diag(1, e^{i t}).
// Only the kinds that reach the kernels (everything but the composite kinds
// U3, RXX, RYY, RZZ and CCX, which are lowered first).
template <typename R>
__host__ __device__ inline Mat2<R> gate_matrix(int kind, double t) {
    double c = 1.0, s = 0.0;
    if (kind_parametric(kind)) {
        const double h = (kind == DQ_CP || kind == DQ_P) ? t : 0.5 * t;
#ifdef __CUDA_ARCH__
        sincos(h, &s, &c);
#else
        s = ::sin(h); c = ::cos(h);
#endif
    }
    const double r2 = 0.70710678118654752440;
    double a[8] = {1, 0, 0, 0, 0, 0, 1, 0};   // identity, (re, im) x 4
    switch (kind) {
    case DQ_H: a[0] = r2; a[2] = r2; a[4] = r2; a[6] = -r2; break;
    case DQ_X: case DQ_CNOT: a[0] = 0; a[2] = 1; a[4] = 1; a[6] = 0; break;
    case DQ_Y: a[0] = 0; a[3] = -1; a[5] = 1; a[6] = 0; break;
    case DQ_Z: case DQ_CZ: a[6] = -1; break;
    case DQ_S: a[6] = 0; a[7] = 1; break;
    case DQ_RX: case DQ_CRX: a[0] = c; a[3] = -s; a[5] = -s; a[6] = c; break;
    case DQ_RY: case DQ_CRY: a[0] = c; a[2] = -s; a[4] = s; a[6] = c; break;
    case DQ_RZ: case DQ_CRZ: a[0] = c; a[1] = -s; a[6] = c; a[7] = s; break;
    case DQ_CP: case DQ_P: a[6] = c; a[7] = s; break;
    default: break;
    }
    Mat2<R> m;
    for (int i = 0; i < 4; ++i) m.m[i] = mk<R>((R)a[2 * i], (R)a[2 * i + 1]);
    return m;
}

template <typename R>
__host__ __device__ __forceinline__ Mat2<R> dagger(const Mat2<R>& u) {
    Mat2<R> d;
    d.m[0] = cconj(u.m[0]); d.m[1] = cconj(u.m[2]);
    d.m[2] = cconj(u.m[1]); d.m[3] = cconj(u.m[3]);
    return d;
}

// (a0, a1) <- M (a0, a1), specialised by class.
template <typename R, int CLS>
__device__ __forceinline__ void apply2(const Mat2<R>& u, cx<R>& a0, cx<R>& a1) {
    if (CLS == CLS_ANTI) {
        cx<R> t = a0; a0 = a1; a1 = t;
    } else if (CLS == CLS_DIAG) {
        a0 = cmul(u.m[0], a0);
        a1 = cmul(u.m[3], a1);
    } else if (CLS == CLS_REAL) {
        const R u0 = u.m[0].x, u1 = u.m[1].x, u2 = u.m[2].x, u3 = u.m[3].x;
        cx<R> b0, b1;
        b0.x = u0 * a0.x + u1 * a1.x; b0.y = u0 * a0.y + u1 * a1.y;
        b1.x = u2 * a0.x + u3 * a1.x; b1.y = u2 * a0.y + u3 * a1.y;
        a0 = b0; a1 = b1;
    } else {
        cx<R> b0 = cadd(cmul(u.m[0], a0), cmul(u.m[1], a1));
        cx<R> b1 = cadd(cmul(u.m[2], a0), cmul(u.m[3], a1));
        a0 = b0; a1 = b1;
    }
}

// Runtime-class variant (used where the class is data, e.g. fused programs).
template <typename R>
__device__ __forceinline__ void apply2_rt(int cls, const Mat2<R>& u, cx<R>& a0, cx<R>& a1) {
    switch (cls) {
    case CLS_ANTI: apply2<R, CLS_ANTI>(u, a0, a1); break;
    case CLS_DIAG: apply2<R, CLS_DIAG>(u, a0, a1); break;
    case CLS_REAL: apply2<R, CLS_REAL>(u, a0, a1); break;
    default: apply2<R, CLS_GENERAL>(u, a0, a1); break;
    }
}

// Contribution of one target pair to dL/dt = 2 Im <lambda| G |psi>, where
// U(t) = exp(-i t G) and (l0, l1), (p0, p1) are the pair's amplitudes after
// the gate.  G is P/2 for R_P (restricted to control = |1>), -|11><11| for
// CP and -|1><1| for P; the factor 2 is folded in.
template <typename R>
__device__ __forceinline__ R grad_pair(int kind, cx<R> l0, cx<R> l1, cx<R> p0, cx<R> p1) {
    switch (kind) {
    case DQ_RX: case DQ_CRX:   // Im(conj(l0) p1 + conj(l1) p0)
        return im_conj_mul(l0, p1) + im_conj_mul(l1, p0);
    case DQ_RY: case DQ_CRY:   // Im(-i conj(l0) p1 + i conj(l1) p0) = -Re(conj(l0) p1) + Re(conj(l1) p0)
        return re_conj_mul(l1, p0) - re_conj_mul(l0, p1);
    case DQ_RZ: case DQ_CRZ:   // Im(conj(l0) p0 - conj(l1) p1)
        return im_conj_mul(l0, p0) - im_conj_mul(l1, p1);
    case DQ_CP: case DQ_P:     // 2 Im(conj(l1) (-p1))
        return (R)(-2) * im_conj_mul(l1, p1);
    default:
        return (R)0;
    }
}

// ---------------------------------------------------------------------------
// bit helpers
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t insert0(uint64_t x, int p) {
    const uint64_t lo = x & ((uint64_t(1) << p) - 1);
    return ((x >> p) << (p + 1)) | lo;
}
// Insert zeros at bit positions a < b (positions in the result).
__host__ __device__ __forceinline__ uint64_t insert0x2(uint64_t x, int a, int b) {
    return insert0(insert0(x, a), b);
}

__device__ __forceinline__ int parity64(uint64_t x) { return __popcll(x) & 1; }

// ---------------------------------------------------------------------------
// Pauli phase: P|b> = ph(b) |b ^ f>, ph(b) = i^{nY} (-1)^{popc(b & s)}.
// Returns ph as (re, im) in {+-1, +-i}.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pauli_phase(uint64_t b, uint64_t s, int nY, float& pr, float& pi) {
    const int k = (nY + 2 * parity64(b & s)) & 3;   // i^k
    pr = (k == 0) ? 1.f : (k == 2 ? -1.f : 0.f);
    pi = (k == 1) ? 1.f : (k == 3 ? -1.f : 0.f);
}

// ---------------------------------------------------------------------------
// reductions: FP64 warp sum
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Device-side error flag codes (written with atomicCAS so the first wins).
enum DevErr : int { DEVERR_NONE = 0, DEVERR_TIMEOUT = 1, DEVERR_BOUNDS = 2 };

// Bounds-checking build (DQ_DEBUG_BOUNDS, libdq_debug.so): DQ_INB(i, lim)
// is false when index i is not below lim; the access it guards is skipped
// and the failure is counted in g_dq_bounds (count, first index, its limit,
// source site), which dq_ctx_check reports.  Every translation unit has its
// own record and registers a reader for it with the library (no relocatable
// device code: the build differs from the normal one only by the checks).
// DQ_SMEM_ALIGNED(p) checks, in that build, that dynamic shared memory has
// the 128-byte alignment the TMA copies need before any copy is issued.  In
// the normal build both are the constant true and guard nothing.
#if defined(DQ_DEBUG_BOUNDS) && !defined(__CUDACC_RTC__)
#define DQ_BOUNDS_BUILD 1
void dq_bounds_register(bool (*read)(unsigned long long *rec), void (*clear)());   // capi.cu
namespace {
__device__ unsigned long long g_dq_bounds[4];
bool dq_bounds_read_tu(unsigned long long *rec) {
    return cudaMemcpyFromSymbol(rec, g_dq_bounds, sizeof(unsigned long long) * 4) == cudaSuccess;
}
void dq_bounds_clear_tu() {
    const unsigned long long zero[4] = {0, 0, 0, 0};
    cudaMemcpyToSymbol(g_dq_bounds, zero, sizeof(zero));
}
struct DqBoundsRegistration {
    DqBoundsRegistration() { dq_bounds_register(&dq_bounds_read_tu, &dq_bounds_clear_tu); }
};
const DqBoundsRegistration dq_bounds_registration;
}  // namespace
constexpr unsigned dq_site_hash(const char *f, unsigned h = 2166136261u) {
    return *f ? dq_site_hash(f + 1, (h ^ (unsigned char)*f) * 16777619u) : h;
}
__device__ __forceinline__ bool dq_in_bounds(uint64_t i, uint64_t lim, unsigned long long site) {
    if (i < lim) return true;
    if (atomicAdd(&g_dq_bounds[0], 1ull) == 0) {
        g_dq_bounds[1] = i;
        g_dq_bounds[2] = lim;
        g_dq_bounds[3] = site;
    }
    return false;
}
#ifdef __FILE_NAME__
#define DQ_SITE_FILE __FILE_NAME__
#else
#define DQ_SITE_FILE __FILE__
#endif
#define DQ_SITE ((unsigned long long)::dq::dq_site_hash(DQ_SITE_FILE) << 32 | (unsigned long long)__LINE__)
#define DQ_INB(i, lim) ::dq::dq_in_bounds((uint64_t)(i), (uint64_t)(lim), DQ_SITE)
#define DQ_SMEM_ALIGNED(p) ::dq::dq_in_bounds((uint64_t)(__cvta_generic_to_shared(p) & 127u), 1, DQ_SITE)
#else
#define DQ_INB(i, lim) true
#define DQ_SMEM_ALIGNED(p) true
#endif

// The context's 256-byte flag block: the error flag at byte 0, the limit of
// every device-side bounded wait (nanoseconds, uint64) at byte 64, the
// multi-pass grid barrier's arrival counter at byte 128.
constexpr int kFlagWaitLimitOffset = 64;
constexpr int kFlagGridBarOffset = 128;
constexpr unsigned long long kDefaultWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long wait_limit_ns(const int *errflag) {
    if (!errflag) return kDefaultWaitNs;
    const unsigned long long v = *reinterpret_cast<const volatile unsigned long long *>(
        reinterpret_cast<const char *>(errflag) + kFlagWaitLimitOffset);
    return v ? v : kDefaultWaitNs;
}

}  // namespace dq
