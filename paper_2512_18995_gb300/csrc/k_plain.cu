// Plain per-gate path: one launch per gate, each a full sweep over the batch.
//
// This is the gate-by-gate evolution |psi_n> = U_n ... U_1 |psi_0> (Sec.
// "Quantum Computing with Qubits", Background) executed literally on the GPU,
// with coalesced 16-byte accesses.  It is the baseline the fused paths are
// measured against, and the general fallback for any shape.
//
// Work decomposition of a one-qubit gate on bit t (optionally controlled on
// bit c): the row is viewed as "units" of two amplitudes that differ only in
// bit 0 (one float4 for complex64, two double2 for complex128).  If t >= 1 a
// work item is a pair of units (u0, u0 | 2^(t-1)) and updates two amplitude
// pairs; if t == 0 the pair lives inside one unit.  A control on bit c >= 1
// restricts the items to units with that bit set (only the touched half of
// the state is read); a control on bit 0 restricts the update to the odd
// element of each unit.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "dq_common.cuh"
#include "dq_plan.h"

namespace dq {

namespace {

constexpr int kThreads = 256;

template <typename R> struct Unit { cx<R> a, b; };

__device__ __forceinline__ Unit<float> ldu(const float2 *p) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    Unit<float> u; u.a = make_float2(v.x, v.y); u.b = make_float2(v.z, v.w); return u;
}
__device__ __forceinline__ void stu(float2 *p, const Unit<float> &u) {
    *reinterpret_cast<float4 *>(p) = make_float4(u.a.x, u.a.y, u.b.x, u.b.y);
}
__device__ __forceinline__ Unit<double> ldu(const double2 *p) {
    Unit<double> u; u.a = p[0]; u.b = p[1]; return u;
}
__device__ __forceinline__ void stu(double2 *p, const Unit<double> &u) { p[0] = u.a; p[1] = u.b; }

// Unit-space description of a one-qubit (optionally controlled) gate.
struct UnitMap {
    int zb0, zb1;        // zero-insert positions in unit space (ascending), -1 = none
    uint64_t setm;       // bits forced to 1 (control in unit space)
    uint64_t pbit;       // partner offset in unit space (0: pair inside a unit)
    int only1;           // control on bit 0: update element b only
    int ib;              // log2(items per row)
};

__host__ UnitMap make_unitmap(int n, int t, int c) {
    UnitMap m{-1, -1, 0, 0, 0, 0};
    std::vector<int> z;
    int ib = n - 1;                 // units per row = 2^(n-1)
    if (t >= 1) { z.push_back(t - 1); m.pbit = uint64_t(1) << (t - 1); --ib; }
    if (c >= 1) { z.push_back(c - 1); m.setm = uint64_t(1) << (c - 1); --ib; }
    if (c == 0) m.only1 = 1;
    std::sort(z.begin(), z.end());
    if (z.size() > 0) m.zb0 = z[0];
    if (z.size() > 1) m.zb1 = z[1];
    m.ib = ib;
    return m;
}

__device__ __forceinline__ uint64_t unit_of(const UnitMap &m, uint64_t j) {
    uint64_t u = j;
    if (m.zb0 >= 0) u = insert0(u, m.zb0);
    if (m.zb1 >= 0) u = insert0(u, m.zb1);
    return u | m.setm;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// The 2x2 block of gate record bg for row r.
template <typename R>
__device__ __forceinline__ void bind_one(const BindGate &bg, int r, const double *__restrict__ params, int nparams,
                                         int ppr, const double *__restrict__ data, int nfeat,
                                         const Mat2<double> *__restrict__ fixed, Mat2<R> *__restrict__ coef) {
    Mat2<R> m;
    if (bg.aux >> 1) {   // a fixed block from the plan's table
        const Mat2<double> &f = fixed[(bg.aux >> 1) - 1];
        for (int i = 0; i < 4; ++i) m.m[i] = mk<R>((R)f.m[i].x, (R)f.m[i].y);
    } else {
        double t = bg.angle;
        if (bg.pidx >= 0) t = ppr ? params[(int64_t)r * nparams + bg.pidx] : params[bg.pidx];
        else if (bg.didx >= 0) t = data[(int64_t)r * nfeat + bg.didx];
        m = gate_matrix<R>(bg.kind, t);
    }
    if (bg.aux & 1)
        for (int i = 0; i < 4; ++i) m.m[i] = cconj(m.m[i]);
    coef[bg.coef + (int64_t)r * bg.rowstep] = m;
}

template <typename R>
__global__ void k_bind(const BindGate *__restrict__ g, int ngates, const double *__restrict__ params,
                       int nparams, int ppr, const double *__restrict__ data, int nfeat,
                       int batch, const Mat2<double> *__restrict__ fixed, Mat2<R> *__restrict__ coef) {
    for (int gi = blockIdx.y; gi < ngates; gi += gridDim.y) {
        const BindGate bg = g[gi];
        const int rows = bg.rowstep ? batch : 1;
        for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x)
            bind_one<R>(bg, r, params, nparams, ppr, data, nfeat, fixed, coef);
    }
}

// k_bind and the preparation of |0...0> in one launch, for calls that run
// them back to back: the first `bind_blocks` blocks bind (item i = gate
// i / rows, row i % rows, rows = the batch when some gate's block depends on
// the row, else 1), the next `zero_blocks` clear `nzero` doubles (partial
// sums that later kernels accumulate into), the others write the state as
// k_init_zero does.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_bind_init(const BindGate *__restrict__ g, int ngates, const double *__restrict__ params, int nparams, int ppr,
            const double *__restrict__ data, int nfeat, int batch, int rows, const Mat2<double> *__restrict__ fixed,
            Mat2<R> *__restrict__ coef, int bind_blocks, double *__restrict__ zero, int64_t nzero, int zero_blocks,
            cx<R> *__restrict__ st, int n, int64_t units) {
    if ((int)blockIdx.x < bind_blocks) {
        const int64_t items = (int64_t)ngates * rows;
        for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < items; i += (int64_t)bind_blocks * kThreads) {
            const int gi = (int)(i / rows), r = (int)(i - (int64_t)gi * rows);
            const BindGate bg = g[gi];
            if (r < (bg.rowstep ? batch : 1)) bind_one<R>(bg, r, params, nparams, ppr, data, nfeat, fixed, coef);
        }
        return;
    }
    if ((int)blockIdx.x < bind_blocks + zero_blocks) {
        const int64_t i = (int64_t)(blockIdx.x - bind_blocks) * kThreads + threadIdx.x;
        if (i < nzero) zero[i] = 0.0;
        return;
    }
    const int64_t i = (int64_t)(blockIdx.x - bind_blocks - zero_blocks) * kThreads + threadIdx.x;
    if (i >= units) return;
    Unit<R> u;
    u.a = mk<R>(((i << 1) & ((int64_t(1) << n) - 1)) == 0 ? R(1) : R(0), R(0));
    u.b = mk<R>(R(0), R(0));
    stu(st + 2 * i, u);
}

template <typename R>
__global__ void k_init_zero(cx<R> *__restrict__ st, int n, int64_t total) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    using C = cx<R>;
    Unit<R> u;
    u.a = mk<R>(((i << 1) & ((int64_t(1) << n) - 1)) == 0 ? R(1) : R(0), R(0));
    u.b = mk<R>(R(0), R(0));
    stu(reinterpret_cast<C *>(st) + 2 * i, u);
}

// One-qubit (optionally controlled) gate sweep, two items per thread.
template <typename R, int CLS>
__global__ void __launch_bounds__(kThreads)
k_sweep(cx<R> *__restrict__ st, int n, UnitMap m, int64_t total, const Mat2<R> *__restrict__ coef,
        int rowstep, int dag) {
    constexpr int UN = 2;
    const int64_t base = (int64_t)blockIdx.x * (kThreads * UN) + threadIdx.x;
    Unit<R> A[UN], B[UN];
    cx<R> *pa[UN], *pb[UN];
    Mat2<R> u[UN];
    bool ok[UN];
#pragma unroll
    for (int k = 0; k < UN; ++k) {
        const int64_t w = base + k * kThreads;
        ok[k] = w < total;
        if (!ok[k]) continue;
        const int64_t row = w >> m.ib;
        const uint64_t un = unit_of(m, (uint64_t)w & ((uint64_t(1) << m.ib) - 1));
        ok[k] = DQ_INB(2 * un + 1, uint64_t(1) << n) && (!m.pbit || DQ_INB(2 * (un | m.pbit) + 1, uint64_t(1) << n));
        if (!ok[k]) continue;
        cx<R> *rp = st + (row << n);
        pa[k] = rp + 2 * un;
        A[k] = ldu(pa[k]);
        if (m.pbit) { pb[k] = rp + 2 * (un | m.pbit); B[k] = ldu(pb[k]); }
        u[k] = coef[row * rowstep];
    }
#pragma unroll
    for (int k = 0; k < UN; ++k) {
        if (!ok[k]) continue;
        Mat2<R> mm = dag ? dagger(u[k]) : u[k];
        if (m.pbit) {
            if (!m.only1) apply2<R, CLS>(mm, A[k].a, B[k].a);
            apply2<R, CLS>(mm, A[k].b, B[k].b);
            stu(pa[k], A[k]);
            stu(pb[k], B[k]);
        } else {
            apply2<R, CLS>(mm, A[k].a, A[k].b);
            stu(pa[k], A[k]);
        }
    }
}

// SWAP of index bits a < b on one or two vectors.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_swap(cx<R> *__restrict__ v0, cx<R> *__restrict__ v1, int n, int a, int b, int ib, int64_t total) {
    const int64_t w = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (w >= total) return;
    const int64_t row = w >> ib;
    const uint64_t j = (uint64_t)w & ((uint64_t(1) << ib) - 1);
    for (int v = 0; v < 2; ++v) {
        cx<R> *st = v == 0 ? v0 : v1;
        if (!st) continue;
        cx<R> *rp = st + (row << n);
        if (a >= 1) {
            const uint64_t u0 = insert0x2(j, a - 1, b - 1) | (uint64_t(1) << (a - 1));
            const uint64_t u1 = u0 ^ (uint64_t(1) << (a - 1)) ^ (uint64_t(1) << (b - 1));
            if (!DQ_INB(2 * u0 + 1, uint64_t(1) << n) || !DQ_INB(2 * u1 + 1, uint64_t(1) << n)) continue;
            Unit<R> A = ldu(rp + 2 * u0), B = ldu(rp + 2 * u1);
            stu(rp + 2 * u0, B);
            stu(rp + 2 * u1, A);
        } else {
            const uint64_t u0 = insert0(j, b - 1);
            const uint64_t u1 = u0 | (uint64_t(1) << (b - 1));
            if (!DQ_INB(2 * u1 + 1, uint64_t(1) << n)) continue;
            Unit<R> A = ldu(rp + 2 * u0), B = ldu(rp + 2 * u1);
            const cx<R> t = A.b; A.b = B.a; B.a = t;
            stu(rp + 2 * u0, A);
            stu(rp + 2 * u1, B);
        }
    }
}

// Block-wide FP64 sum of one value per thread; result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NT / 32; ++i) s += red[i];
    }
    __syncthreads();
    return s;
}

constexpr int kMaxT = 8;    // terms per expectation launch
struct TermPack {
    uint64_t s[kMaxT];
    int nY[kMaxT];
    int nt;
};

// Partial sums of <psi| P_k |psi> for terms sharing flip mask f.  grid = (nblk, batch).
// Each thread forms products in the state precision, sums runs of up to 32
// items in that precision, and carries FP64 beyond.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_expect(const cx<R> *__restrict__ st, int n, uint64_t f, int lf, TermPack tp, int64_t per_blk,
         double *__restrict__ part, int slot0, int nbatch) {
    __shared__ double red[kThreads / 32];
    const int row = blockIdx.y;
    const int64_t items = f ? (int64_t(1) << (n - 1)) : (int64_t(1) << n);
    const int64_t i0 = (int64_t)blockIdx.x * per_blk;
    const int64_t i1 = min(items, i0 + per_blk);
    const cx<R> *rp = st + ((int64_t)row << n);
    double accd[kMaxT];
    R accf[kMaxT];
#pragma unroll
    for (int k = 0; k < kMaxT; ++k) { accd[k] = 0.0; accf[k] = R(0); }
    int run = 0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kThreads) {
        uint64_t b = (uint64_t)i;
        R re, im;
        if (f) {
            b = insert0(b, lf);
            if (!DQ_INB(b, uint64_t(1) << n) || !DQ_INB(b ^ f, uint64_t(1) << n)) continue;
            const cx<R> x = rp[b], y = rp[b ^ f];     // z = conj(psi_{b^f}) psi_b
            re = re_conj_mul(y, x);
            im = im_conj_mul(y, x);
        } else {
            const cx<R> x = rp[b];
            re = x.x * x.x + x.y * x.y;
            im = R(0);
        }
#pragma unroll
        for (int k = 0; k < kMaxT; ++k) {
            if (k >= tp.nt) break;
            // term value: 2 Re(i^{nY} (-1)^{popc(b&s)} z) for pairs, p for diagonal
            const int ph = (tp.nY[k] + 2 * parity64(b & tp.s[k])) & 3;
            R v = (ph == 0) ? re : (ph == 1 ? -im : (ph == 2 ? -re : im));
            accf[k] += f ? R(2) * v : v;
        }
        if (++run == 32) {
            run = 0;
#pragma unroll
            for (int k = 0; k < kMaxT; ++k) { accd[k] += (double)accf[k]; accf[k] = R(0); }
        }
    }
#pragma unroll
    for (int k = 0; k < kMaxT; ++k) {
        if (k >= tp.nt) break;
        const double s = block_sum<kThreads>(accd[k] + (double)accf[k], red);
        if (threadIdx.x == 0)
            part[((int64_t)(slot0 + k) * nbatch + row) * gridDim.x + blockIdx.x] = s;
    }
}

// out[row, o] = sum_{k in o} coeff_k * sum_blk part[k][row][blk].  One block per (row, o).
__global__ void k_expect_finalize(const double *__restrict__ part, const DevTerm *__restrict__ terms,
                                  const int32_t *__restrict__ obs_ptr, int nobs, int nbatch, int nblk,
                                  double *__restrict__ out) {
    // launched as a programmatic dependent of the kernel that writes `part`
    // (a no-op otherwise): wait for it to complete before reading
    asm volatile("griddepcontrol.wait;" ::: "memory");
    __shared__ double red[kThreads / 32];
    const int row = blockIdx.x / nobs, o = blockIdx.x % nobs;
    const int k0 = obs_ptr[o], k1 = obs_ptr[o + 1];
    // (term, block) items, four independent loads in flight per thread
    const int cnt = (k1 - k0) * nblk;
    auto item = [&](int i) {
        const int k = k0 + i / nblk, blk = i - (k - k0) * nblk;
        return terms[k].coeff * part[((int64_t)k * nbatch + row) * nblk + blk];
    };
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int i = threadIdx.x;
    for (; i + 3 * kThreads < cnt; i += 4 * kThreads) {
        a0 += item(i);
        a1 += item(i + kThreads);
        a2 += item(i + 2 * kThreads);
        a3 += item(i + 3 * kThreads);
    }
    for (; i < cnt; i += kThreads) a0 += item(i);
    const double acc = (a0 + a1) + (a2 + a3);
    const double s = block_sum<kThreads>(acc, red);
    if (threadIdx.x == 0) out[(int64_t)row * nobs + o] = s;
}

// lambda_b += w * coeff * ph(b^f) * psi_{b^f}  for one term, every row.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_lambda_term(const cx<R> *__restrict__ psi, cx<R> *__restrict__ lam, int n, DevTerm t,
              const double *__restrict__ w, int nobs, int64_t total) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= total) return;
    const int64_t row = i >> n;
    const uint64_t b = (uint64_t)i & ((uint64_t(1) << n) - 1);
    const uint64_t src = b ^ t.f;
    if (!DQ_INB(src, uint64_t(1) << n)) return;
    float pr, pim;
    pauli_phase(src, t.s, t.nY, pr, pim);
    const R wt = (R)((w ? w[row * nobs + t.obs] : 1.0) * t.coeff);
    const cx<R> x = psi[(row << n) + src];
    cx<R> l = lam[(row << n) + b];
    l.x += wt * ((R)pr * x.x - (R)pim * x.y);
    l.y += wt * ((R)pr * x.y + (R)pim * x.x);
    lam[(row << n) + b] = l;
}

// One reverse-sweep step of the adjoint method on (psi, lambda):
// optionally accumulate 2 Im <lambda|G|psi> (both after the gate), then
// un-apply U^dagger on both.  grid = (nblk, batch).
template <typename R, int CLS, bool GRAD>
__global__ void __launch_bounds__(kThreads)
k_adj(cx<R> *__restrict__ psi, cx<R> *__restrict__ lam, int n, UnitMap m, int kind,
      const Mat2<R> *__restrict__ coef, int rowstep, int64_t per_blk, double *__restrict__ part,
      int slot, int nbatch) {
    __shared__ double red[kThreads / 32];
    const int row = blockIdx.y;
    const int64_t items = int64_t(1) << m.ib;
    const int64_t i0 = (int64_t)blockIdx.x * per_blk;
    const int64_t i1 = min(items, i0 + per_blk);
    const Mat2<R> ud = dagger(coef[row * rowstep]);
    cx<R> *pp = psi + ((int64_t)row << n);
    cx<R> *lp = lam + ((int64_t)row << n);
    double accd = 0.0;
    R accf = R(0);
    int run = 0;
    for (int64_t j = i0 + threadIdx.x; j < i1; j += kThreads) {
        const uint64_t un = unit_of(m, (uint64_t)j);
        if (!DQ_INB(2 * un + 1, uint64_t(1) << n) || (m.pbit && !DQ_INB(2 * (un | m.pbit) + 1, uint64_t(1) << n)))
            continue;
        Unit<R> PA = ldu(pp + 2 * un), LA = ldu(lp + 2 * un);
        if (m.pbit) {
            const uint64_t un1 = un | m.pbit;
            Unit<R> PB = ldu(pp + 2 * un1), LB = ldu(lp + 2 * un1);
            if (GRAD) {
                if (!m.only1) accf += grad_pair<R>(kind, LA.a, LB.a, PA.a, PB.a);
                accf += grad_pair<R>(kind, LA.b, LB.b, PA.b, PB.b);
            }
            if (!m.only1) { apply2<R, CLS>(ud, PA.a, PB.a); apply2<R, CLS>(ud, LA.a, LB.a); }
            apply2<R, CLS>(ud, PA.b, PB.b);
            apply2<R, CLS>(ud, LA.b, LB.b);
            stu(pp + 2 * un1, PB);
            stu(lp + 2 * un1, LB);
        } else {
            if (GRAD) accf += grad_pair<R>(kind, LA.a, LA.b, PA.a, PA.b);
            apply2<R, CLS>(ud, PA.a, PA.b);
            apply2<R, CLS>(ud, LA.a, LA.b);
        }
        stu(pp + 2 * un, PA);
        stu(lp + 2 * un, LA);
        if (GRAD && ++run == 32) { run = 0; accd += (double)accf; accf = R(0); }
    }
    if (GRAD) {
        const double s = block_sum<kThreads>(accd + (double)accf, red);
        if (threadIdx.x == 0) part[((int64_t)slot * nbatch + row) * gridDim.x + blockIdx.x] = s;
    }
}

// grad[out] = sum over the output's slots (and rows when shared) of the partials.
// mode 0: shared params -> out[p];  mode 1: per-row -> out[row * nout + p].
__global__ void k_grad_reduce(const double *__restrict__ part, const int32_t *__restrict__ ptr,
                              const int32_t *__restrict__ slots, int nout, int nbatch, int nblk,
                              int per_row, double *__restrict__ out) {
    __shared__ double red[kThreads / 32];
    const int p = blockIdx.x % nout;
    const int row = per_row ? blockIdx.x / nout : 0;
    const int s0 = ptr[p], s1 = ptr[p + 1];
    double acc = 0.0;
    if (per_row) {
        const int64_t cnt = (int64_t)(s1 - s0) * nblk;
        for (int64_t i = threadIdx.x; i < cnt; i += kThreads) {
            const int s = slots[s0 + (int)(i / nblk)], blk = (int)(i % nblk);
            acc += part[((int64_t)s * nbatch + row) * nblk + blk];
        }
    } else {
        const int64_t per = (int64_t)nbatch * nblk;
        const int64_t cnt = (int64_t)(s1 - s0) * per;
        for (int64_t i = threadIdx.x; i < cnt; i += kThreads) {
            const int s = slots[s0 + (int)(i / per)];
            acc += part[(int64_t)s * per + (i % per)];
        }
    }
    const double sum = block_sum<kThreads>(acc, red);
    if (threadIdx.x == 0) out[per_row ? (int64_t)row * nout + p : p] = sum;
}

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Blocks per row for the (nblk, batch) grids: aim for ~4096 blocks in total.
inline int blocks_per_row(int n, int batch) {
    const int64_t max_useful = std::max<int64_t>(1, (int64_t(1) << std::max(0, n - 3)) / kThreads);
    const int64_t want = std::max<int64_t>(1, cdiv(4096, batch));
    return (int)std::min(max_useful, want);
}

template <typename R>
cudaError_t launch_sweep(const DevGate &g, int n, cx<R> *st, int batch, const Mat2<R> *coef, int dag,
                         cudaStream_t s, int64_t *launches) {
    if (g.cls == CLS_SWAP) {
        LaunchScope ls(s, "k_swap", launches);
        const int a = g.t, b = g.c;
        const int ib = (a >= 1) ? n - 3 : n - 2;
        const int64_t total = (int64_t)batch << ib;
        k_swap<R><<<(unsigned)cdiv(total, kThreads), kThreads, 0, s>>>(st, nullptr, n, a, b, ib, total);
        return cudaGetLastError();
    }
    const UnitMap m = make_unitmap(n, g.t, g.c);
    const int64_t total = (int64_t)batch << m.ib;
    const unsigned grid = (unsigned)cdiv(total, kThreads * 2);
    const Mat2<R> *cf = coef + g.coef;
    LaunchScope ls(s, "k_sweep", launches);
    switch (g.cls) {
    case CLS_ANTI: k_sweep<R, CLS_ANTI><<<grid, kThreads, 0, s>>>(st, n, m, total, cf, g.rowstep, dag); break;
    case CLS_DIAG: k_sweep<R, CLS_DIAG><<<grid, kThreads, 0, s>>>(st, n, m, total, cf, g.rowstep, dag); break;
    case CLS_REAL: k_sweep<R, CLS_REAL><<<grid, kThreads, 0, s>>>(st, n, m, total, cf, g.rowstep, dag); break;
    default: k_sweep<R, CLS_GENERAL><<<grid, kThreads, 0, s>>>(st, n, m, total, cf, g.rowstep, dag); break;
    }
    return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename R>
cudaError_t plain_bind(const Plan &p, const double *params, const double *data, int batch,
                       void *coef, cudaStream_t s, int64_t *launches) {
    if (p.ngates == 0) return cudaSuccess;
    const int rows = p.ncoef_rows ? batch : 1;
    dim3 grid((unsigned)std::min<int64_t>(cdiv(rows, 128), 64), (unsigned)std::min(p.ngates, 65535));
    LaunchScope ls(s, "k_bind", launches);
    k_bind<R><<<grid, 128, 0, s>>>(p.d_bind, p.ngates, params, p.nparams, p.ppr, data, p.nfeat, batch, p.d_fixed,
                                   (Mat2<R> *)coef);
    return cudaGetLastError();
}

template <typename R>
cudaError_t plain_bind_init(const Plan &p, const double *params, const double *data, int batch, void *coef,
                            void *state, double *zero, int64_t nzero, cudaStream_t s, int64_t *launches) {
    if (p.n == 0) return cudaErrorInvalidValue;
    const int rows = p.ncoef_rows ? batch : 1;
    const int64_t items = (int64_t)p.ngates * rows;
    const int bind_blocks = (int)std::min<int64_t>(cdiv(items, kThreads), 4096);
    const int64_t zb = zero ? cdiv(nzero, kThreads) : 0;
    const int64_t units = (int64_t)batch << (p.n - 1);
    const int64_t blocks = bind_blocks + zb + cdiv(units, kThreads);
    if (blocks > INT32_MAX) {   // more than one launch's blocks: separate kernels
        cudaError_t e = plain_bind<R>(p, params, data, batch, coef, s, launches);
        if (e == cudaSuccess && zero && nzero) e = cudaMemsetAsync(zero, 0, (size_t)nzero * sizeof(double), s);
        return e != cudaSuccess ? e : plain_init_zero<R>(state, p.n, batch, s, launches);
    }
    LaunchScope ls(s, "k_bind_init", launches);
    k_bind_init<R><<<(unsigned)blocks, kThreads, 0, s>>>(p.d_bind, p.ngates, params, p.nparams, p.ppr, data, p.nfeat,
                                                         batch, rows, p.d_fixed, (Mat2<R> *)coef, bind_blocks, zero,
                                                         nzero, (int)zb, (cx<R> *)state, p.n, units);
    return cudaGetLastError();
}

template <typename R>
cudaError_t plain_init_zero(void *state, int n, int batch, cudaStream_t s, int64_t *launches) {
    const int64_t units = (int64_t)batch << (n - 1);
    if (n == 0) return cudaErrorInvalidValue;
    LaunchScope ls(s, "k_init_zero", launches);
    k_init_zero<R><<<(unsigned)cdiv(units, kThreads), kThreads, 0, s>>>((cx<R> *)state, n, units);
    return cudaGetLastError();
}

template <typename R>
cudaError_t plain_apply(const Plan &p, const void *coef, void *state, int batch, int dagger,
                        cudaStream_t s, int64_t *launches) {
    const Mat2<R> *cf = (const Mat2<R> *)coef;
    for (int i = 0; i < p.ngates; ++i) {
        const DevGate &g = p.gates[dagger ? p.ngates - 1 - i : i];
        cudaError_t e = launch_sweep<R>(g, p.n, (cx<R> *)state, batch, cf, dagger, s, launches);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

size_t plain_expect_part_bytes(int n, int nterms, int batch) {
    return (size_t)std::max(nterms, 1) * batch * blocks_per_row(n, batch) * sizeof(double);
}

template <typename R>
cudaError_t plain_expect(int n, const std::vector<DevTerm> &terms, int nobs, const void *state,
                         int batch, double *part, double *out, cudaStream_t s, int64_t *launches) {
    (void)nobs;
    const int nblk = blocks_per_row(n, batch);
    // Group consecutive terms with the same flip mask, up to kMaxT per launch.
    size_t k = 0;
    while (k < terms.size()) {
        TermPack tp{};
        const uint64_t f = terms[k].f;
        size_t e = k;
        while (e < terms.size() && terms[e].f == f && (int)(e - k) < kMaxT) {
            tp.s[e - k] = terms[e].s;
            tp.nY[e - k] = terms[e].nY;
            ++e;
        }
        tp.nt = (int)(e - k);
        const int lf = f ? __builtin_ctzll(f) : 0;
        const int64_t items = f ? (int64_t(1) << (n - 1)) : (int64_t(1) << n);
        const int64_t per_blk = cdiv(items, nblk);
        {
            LaunchScope ls(s, "k_expect", launches);
            k_expect<R><<<dim3(nblk, batch), kThreads, 0, s>>>((const cx<R> *)state, n, f, lf, tp, per_blk,
                                                               part, (int)k, batch);
        }
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
        k = e;
    }
    return cudaSuccess;
}

// Finalize uses device copies of the terms and observable offsets; they are
// passed by the caller through these two entry points.
cudaError_t plain_expect_finalize(const double *part, const DevTerm *d_terms, const int32_t *d_obs_ptr,
                                  int nobs, int n, int batch, double *out, cudaStream_t s,
                                  int64_t *launches) {
    const int nblk = blocks_per_row(n, batch);
    LaunchScope ls(s, "k_expect_finalize", launches);
    k_expect_finalize<<<(unsigned)((int64_t)batch * nobs), kThreads, 0, s>>>(part, d_terms, d_obs_ptr,
                                                                            nobs, batch, nblk, out);
    return cudaGetLastError();
}

size_t plain_adjoint_part_bytes(const Plan &p, int batch) {
    return (size_t)std::max(p.nslots, 1) * batch * blocks_per_row(p.n, batch) * sizeof(double);
}

template <typename R>
cudaError_t plain_lambda(int n, const std::vector<DevTerm> &terms, int nobs, const double *w,
                         const void *psi, void *lam, int batch, cudaStream_t s, int64_t *launches) {
    const int64_t total = (int64_t)batch << n;
    cudaError_t e = cudaMemsetAsync(lam, 0, (size_t)total * sizeof(cx<R>), s);
    if (e != cudaSuccess) return e;
    for (const DevTerm &t : terms) {
        {
            LaunchScope ls(s, "k_lambda_term", launches);
            k_lambda_term<R><<<(unsigned)cdiv(total, kThreads), kThreads, 0, s>>>(
                (const cx<R> *)psi, (cx<R> *)lam, n, t, w, nobs, total);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename R>
cudaError_t plain_adjoint(const Plan &p, const void *coef, const std::vector<DevTerm> &terms,
                          int nobs, const double *row_weights, void *psi, void *lam, int batch,
                          double *part, double *grad_params, double *grad_data,
                          cudaStream_t s, int64_t *launches) {
    const int n = p.n;
    cudaError_t e = plain_lambda<R>(n, terms, nobs, row_weights, psi, lam, batch, s, launches);
    if (e != cudaSuccess) return e;
    const int nblk = blocks_per_row(n, batch);
    const Mat2<R> *cf = (const Mat2<R> *)coef;
    cx<R> *ps = (cx<R> *)psi, *ls = (cx<R> *)lam;
    // gates before the first requested gradient are never un-applied
    const int gstop = p.first_grad_gate(grad_params != nullptr, grad_data != nullptr);
    for (int gi = p.ngates - 1; gi >= gstop; --gi) {
        const DevGate &g = p.gates[gi];
        if (g.cls == CLS_SWAP) {
            const int ib = (g.t >= 1) ? n - 3 : n - 2;
            const int64_t total = (int64_t)batch << ib;
            LaunchScope sc(s, "k_swap", launches);
            k_swap<R><<<(unsigned)cdiv(total, kThreads), kThreads, 0, s>>>(ps, ls, n, g.t, g.c, ib, total);
        } else {
            LaunchScope sc(s, "k_adj", launches);
            const UnitMap m = make_unitmap(n, g.t, g.c);
            const int64_t per_blk = cdiv(int64_t(1) << m.ib, nblk);
            const int slot = p.slot_of_gate[gi];
            const dim3 grid(nblk, batch);
            const Mat2<R> *gc = cf + g.coef;
#define DQ_ADJ_LAUNCH(CLS)                                                                            \
    if (slot >= 0)                                                                                    \
        k_adj<R, CLS, true><<<grid, kThreads, 0, s>>>(ps, ls, n, m, g.kind, gc, g.rowstep, per_blk,  \
                                                      part, slot, batch);                            \
    else                                                                                              \
        k_adj<R, CLS, false><<<grid, kThreads, 0, s>>>(ps, ls, n, m, g.kind, gc, g.rowstep, per_blk, \
                                                       part, 0, batch);
            switch (g.cls) {
            case CLS_ANTI: DQ_ADJ_LAUNCH(CLS_ANTI) break;
            case CLS_DIAG: DQ_ADJ_LAUNCH(CLS_DIAG) break;
            case CLS_REAL: DQ_ADJ_LAUNCH(CLS_REAL) break;
            default: DQ_ADJ_LAUNCH(CLS_GENERAL) break;
            }
#undef DQ_ADJ_LAUNCH
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return grad_reduce(p, part, batch, nblk, grad_params, grad_data, s, launches);
}

cudaError_t grad_reduce(const Plan &p, const double *part, int batch, int nblk, double *grad_params,
                        double *grad_data, cudaStream_t s, int64_t *launches) {
    if (grad_params && p.nparams > 0) {
        const int per_row = p.ppr;
        const int64_t nb = per_row ? (int64_t)batch * p.nparams : p.nparams;
        LaunchScope sc(s, "k_grad_reduce", launches);
        k_grad_reduce<<<(unsigned)nb, kThreads, 0, s>>>(part, p.d_pslot_ptr, p.d_pslots, p.nparams, batch,
                                                        nblk, per_row, grad_params);
    }
    if (grad_data && p.nfeat > 0) {
        LaunchScope sc(s, "k_grad_reduce", launches);
        k_grad_reduce<<<(unsigned)((int64_t)batch * p.nfeat), kThreads, 0, s>>>(
            part, p.d_dslot_ptr, p.d_dslots, p.nfeat, batch, nblk, 1, grad_data);
    }
    return cudaGetLastError();
}

cudaError_t expect_finalize_nblk(const double *part, const DevTerm *d_terms, const int32_t *d_obs_ptr, int nobs,
                                 int batch, int nblk, double *out, cudaStream_t s, int64_t *launches) {
    // a programmatic dependent launch: its launch overlaps the tail of the
    // forward pass that writes the partials (the kernel waits for it first)
    LaunchScope ls(s, "k_expect_finalize", launches);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)((int64_t)batch * nobs));
    cfg.blockDim = dim3(kThreads);
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_expect_finalize, part, d_terms, d_obs_ptr, nobs, batch, nblk, out);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// explicit instantiations
#define DQ_INST(R)                                                                                       \
    template cudaError_t plain_bind<R>(const Plan &, const double *, const double *, int, void *,        \
                                       cudaStream_t, int64_t *);                                        \
    template cudaError_t plain_init_zero<R>(void *, int, int, cudaStream_t, int64_t *);                 \
    template cudaError_t plain_bind_init<R>(const Plan &, const double *, const double *, int, void *, void *, \
                                            double *, int64_t, cudaStream_t, int64_t *);                 \
    template cudaError_t plain_apply<R>(const Plan &, const void *, void *, int, int, cudaStream_t,      \
                                        int64_t *);                                                     \
    template cudaError_t plain_expect<R>(int, const std::vector<DevTerm> &, int, const void *, int,     \
                                         double *, double *, cudaStream_t, int64_t *);                  \
    template cudaError_t plain_lambda<R>(int, const std::vector<DevTerm> &, int, const double *,        \
                                         const void *, void *, int, cudaStream_t, int64_t *);           \
    template cudaError_t plain_adjoint<R>(const Plan &, const void *, const std::vector<DevTerm> &, int, \
                                          const double *, void *, void *, int, double *, double *,       \
                                          double *, cudaStream_t, int64_t *);
DQ_INST(float)
DQ_INST(double)
#undef DQ_INST

}  // namespace dq
