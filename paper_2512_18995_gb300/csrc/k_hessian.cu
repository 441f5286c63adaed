// Hessian of expectations by shift rules on adjoint gradients.
//
// The paper benchmarks gradients and Hessians of circuit expectations
// (Sec. "Benchmarks", gradient and Hessian).  Here every trainable angle
// occurrence v (one angle slot of one gate) gets its own "virtual" parameter
// t_v, so the loss is L(theta) = L~(A theta) with A the 0/1 map from
// parameters to occurrences and
//     H = A^T H~ A,   H~[v][u] = d/dt_v (dL~/dt_u).
// Row v of H~ comes from adjoint gradients at shifted points: the loss is a
// trigonometric polynomial in t_v whose frequencies are set by the
// generator's spectrum, and so is every gradient component dL~/dt_u.
//   * generator eigenvalue gap 1 (RX RY RZ RXX RYY RZZ P CP, U3's angles):
//     f'(t) = [f(t + pi/2) - f(t - pi/2)] / 2          (two-term rule);
//   * generator |1><1| (x) P/2 of the controlled rotations (gaps 1/2, 1):
//     f'(t) = c1 [f(t + pi/2) - f(t - pi/2)] - c2 [f(t + 3pi/2) - f(t - 3pi/2)]
//     with c1 = (sqrt2 + 1) / (4 sqrt2), c2 = (sqrt2 - 1) / (4 sqrt2)
//     (the four-term rule for two frequencies; both are exact, see Wierichs
//     et al., "General parameter-shift rules for quantum gradients",
//     Quantum 6, 677 (2022)).
// All shifted points of a chunk of occurrences, times every data row, run as
// ONE batch through the fused forward + adjoint path with per-row
// parameters; the kernels below build the row tables and fold the
// per-row gradients into H~ and then H (fixed summation order, no atomics).
#include <cuda_runtime.h>
#include <stdint.h>

#include "dq_plan.h"

namespace dq {

namespace {

constexpr int kThreads = 256;

// Row j * batch + r (shift row j, data row r): virtual parameters
// theta[occ[u]] (+ shift[j] on u == shift_v[j]), data row r, weights row r.
__global__ void __launch_bounds__(kThreads)
k_hess_rows(const double *__restrict__ params, const int32_t *__restrict__ occ, int V,
            const int32_t *__restrict__ shift_v, const double *__restrict__ shift, int J, int batch,
            const double *__restrict__ data, int nfeat, const double *__restrict__ rw, int nobs,
            double *__restrict__ prow, double *__restrict__ drow, double *__restrict__ wrow) {
    const int64_t R = (int64_t)J * batch;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = t0; i < R * V; i += stride) {
        const int64_t row = i / V;
        const int u = (int)(i - row * V);
        const int j = (int)(row / batch);
        prow[i] = params[occ[u]] + (u == shift_v[j] ? shift[j] : 0.0);
    }
    if (data)
        for (int64_t i = t0; i < R * nfeat; i += stride) {
            const int64_t row = i / nfeat;
            const int f = (int)(i - row * nfeat);
            drow[i] = data[(row % batch) * nfeat + f];
        }
    if (rw)
        for (int64_t i = t0; i < R * nobs; i += stride) {
            const int64_t row = i / nobs;
            const int o = (int)(i - row * nobs);
            wrow[i] = rw[(row % batch) * nobs + o];
        }
}

// H~[v0 + vl][u] = sum_s coef[j_s] sum_r G[((j_s - j0) * batch + r) * V + u]
// over the shift rows j_s = vrow0[vl] + s, s < nshift[vl], of local
// occurrence vl (G holds the chunk's rows, starting at shift row j0).
__global__ void __launch_bounds__(kThreads)
k_hess_combine(const double *__restrict__ G, const int32_t *__restrict__ vrow0, const int32_t *__restrict__ nshift,
               const double *__restrict__ coef, int j0, int nv, int v0, int batch, int V, double *__restrict__ Ht) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nv * V) return;
    const int vl = (int)(i / V), u = (int)(i - (int64_t)vl * V);
    double acc = 0.0;
    for (int s = 0; s < nshift[vl]; ++s) {
        const int j = vrow0[vl] + s;
        double col = 0.0;
        for (int r = 0; r < batch; ++r) col += G[((int64_t)(j - j0) * batch + r) * V + u];
        acc += coef[j] * col;
    }
    Ht[(int64_t)(v0 + vl) * V + u] = acc;
}

// H[p][q] = sum over occurrences v of p and u of q of H~[v][u].
__global__ void __launch_bounds__(kThreads)
k_hess_fold(const double *__restrict__ Ht, const int32_t *__restrict__ optr, const int32_t *__restrict__ oidx, int P,
            int V, double *__restrict__ H) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)P * P) return;
    const int p = (int)(i / P), q = (int)(i - (int64_t)p * P);
    double acc = 0.0;
    for (int a = optr[p]; a < optr[p + 1]; ++a)
        for (int b = optr[q]; b < optr[q + 1]; ++b) acc += Ht[(int64_t)oidx[a] * V + oidx[b]];
    H[i] = acc;
}

// Expectation-level shift rules: one thread per local occurrence (the rows
// and observables are summed in a fixed order).
__global__ void __launch_bounds__(kThreads)
k_shift_combine(const double *__restrict__ E, const double *__restrict__ w, const int32_t *__restrict__ vrow0,
                const int32_t *__restrict__ nshift, const double *__restrict__ coef, int j0, int nv, int v0, int batch,
                int nobs, double *__restrict__ g) {
    const int vl = blockIdx.x * blockDim.x + threadIdx.x;
    if (vl >= nv) return;
    double acc = 0.0;
    for (int s = 0; s < nshift[vl]; ++s) {
        const int j = vrow0[vl] + s;
        double sum = 0.0;
        for (int r = 0; r < batch; ++r)
            for (int o = 0; o < nobs; ++o)
                sum += (w ? w[(int64_t)r * nobs + o] : 1.0) * E[((int64_t)(j - j0) * batch + r) * nobs + o];
        acc += coef[j] * sum;
    }
    g[v0 + vl] = acc;
}

__global__ void __launch_bounds__(kThreads)
k_shift_fold(const double *__restrict__ g, const int32_t *__restrict__ optr, const int32_t *__restrict__ oidx, int P,
             double *__restrict__ grad) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    double acc = 0.0;
    for (int a = optr[p]; a < optr[p + 1]; ++a) acc += g[oidx[a]];
    grad[p] = acc;
}

unsigned blocks_for(int64_t work, int nsm) {
    const int64_t b = (work + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)nsm * 32;
    return (unsigned)(b < 1 ? 1 : (b < cap ? b : cap));
}

}  // namespace

cudaError_t hess_rows(const double *params, const int32_t *occ, int V, const int32_t *shift_v, const double *shift,
                      int J, int batch, const double *data, int nfeat, const double *rw, int nobs, double *prow,
                      double *drow, double *wrow, int nsm, cudaStream_t s, int64_t *launches) {
    const int64_t R = (int64_t)J * batch;
    const int64_t work = R * (int64_t)(V > nfeat ? (V > nobs ? V : nobs) : (nfeat > nobs ? nfeat : nobs));
    LaunchScope ls(s, "k_hess_rows", launches);
    k_hess_rows<<<blocks_for(work, nsm), kThreads, 0, s>>>(params, occ, V, shift_v, shift, J, batch, data, nfeat,
                                                           rw, nobs, prow, drow, wrow);
    return cudaGetLastError();
}

cudaError_t hess_combine(const double *G, const int32_t *vrow0, const int32_t *nshift, const double *coef, int j0,
                         int nv, int v0, int batch, int V, double *Ht, cudaStream_t s, int64_t *launches) {
    const int64_t work = (int64_t)nv * V;
    LaunchScope ls(s, "k_hess_combine", launches);
    k_hess_combine<<<(unsigned)((work + kThreads - 1) / kThreads), kThreads, 0, s>>>(G, vrow0, nshift, coef, j0, nv,
                                                                                     v0, batch, V, Ht);
    return cudaGetLastError();
}

cudaError_t hess_fold(const double *Ht, const int32_t *optr, const int32_t *oidx, int P, int V, double *H,
                      cudaStream_t s, int64_t *launches) {
    const int64_t work = (int64_t)P * P;
    LaunchScope ls(s, "k_hess_fold", launches);
    k_hess_fold<<<(unsigned)((work + kThreads - 1) / kThreads), kThreads, 0, s>>>(Ht, optr, oidx, P, V, H);
    return cudaGetLastError();
}

cudaError_t shift_combine(const double *E, const double *w, const int32_t *vrow0, const int32_t *nshift,
                          const double *coef, int j0, int nv, int v0, int batch, int nobs, double *g, cudaStream_t s,
                          int64_t *launches) {
    LaunchScope ls(s, "k_shift_combine", launches);
    k_shift_combine<<<(unsigned)((nv + kThreads - 1) / kThreads), kThreads, 0, s>>>(E, w, vrow0, nshift, coef, j0, nv,
                                                                                   v0, batch, nobs, g);
    return cudaGetLastError();
}

cudaError_t shift_fold(const double *g, const int32_t *optr, const int32_t *oidx, int P, double *grad, cudaStream_t s,
                       int64_t *launches) {
    LaunchScope ls(s, "k_shift_fold", launches);
    k_shift_fold<<<(unsigned)((P + kThreads - 1) / kThreads), kThreads, 0, s>>>(g, optr, oidx, P, grad);
    return cudaGetLastError();
}

}  // namespace dq
