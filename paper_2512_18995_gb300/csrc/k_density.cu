// Expectation values of Pauli sums in a vectorised density matrix.
//
// Tr(P rho) for a Pauli string P with flip mask f and phase P|k> = ph(k)
// |k ^ f> is sum_k <k ^ f| P |k> rho[k][k ^ f] = sum_k ph(k) rho[k][k ^ f]
// (Sec. "Quantum Computing with Qubits": expectations of observables, here
// for mixed states).  rho is stored row-major per batch row, entry (i, j) at
// i * 2^n + j.  The sum touches 2^n of the 4^n entries (one per row of rho),
// so it is a strided gather, not a stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dq_common.cuh"
#include "dq_density.h"
#include "dq_plan.h"

namespace dq {

namespace {

constexpr int kThreads = 256;

// One CTA per (row, observable): out[row * nobs + o] = sum over the
// observable's terms of coeff * Re sum_k ph(k) rho[k][k ^ f].
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_density_expect(const cx<R> *__restrict__ rho, int n, const DevTerm *__restrict__ terms,
                 const int32_t *__restrict__ obs_ptr, int nobs, double *__restrict__ out) {
    __shared__ double part[kThreads / 32];
    const int row = blockIdx.x / nobs, o = blockIdx.x - row * nobs;
    const uint64_t dim = uint64_t(1) << n;
    const cx<R> *r = rho + (uint64_t)row * dim * dim;
    double acc = 0.0;
    for (int t = obs_ptr[o]; t < obs_ptr[o + 1]; ++t) {
        const DevTerm T = terms[t];
        double s = 0.0;
        for (uint64_t k = threadIdx.x; k < dim; k += blockDim.x) {
            float pr, pi;
            pauli_phase(k, T.s, T.nY, pr, pi);
            const cx<R> v = r[k * dim + (k ^ T.f)];
            s += (double)((R)pr * v.x - (R)pi * v.y);
        }
        acc += T.coeff * s;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) tot += part[w];
        out[(int64_t)row * nobs + o] = tot;
    }
}

}  // namespace

template <typename R>
cudaError_t density_expect(const void *rho, int n, const DevTerm *d_terms, const int32_t *d_obs_ptr, int nobs,
                           int batch, double *out, cudaStream_t s, int64_t *launches) {
    LaunchScope ls(s, "k_density_expect", launches);
    k_density_expect<R><<<(unsigned)((int64_t)batch * nobs), kThreads, 0, s>>>((const cx<R> *)rho, n, d_terms,
                                                                                 d_obs_ptr, nobs, out);
    return cudaGetLastError();
}

template cudaError_t density_expect<float>(const void *, int, const DevTerm *, const int32_t *, int, int, double *,
                                           cudaStream_t, int64_t *);
template cudaError_t density_expect<double>(const void *, int, const DevTerm *, const int32_t *, int, int, double *,
                                            cudaStream_t, int64_t *);

}  // namespace dq
