// Squared norm of every row with FP64 accumulation, and the self-test of the
// bounded-wait failure path.
//
// Norm: <psi|psi> = sum_i |psi_i|^2 over the 2^n amplitudes of a row.  Each
// thread forms |psi_i|^2 in the state's precision and sums a short run of
// them (eight) in that precision; everything above runs in FP64 -- the
// thread's running sum, the warp and block reductions, and the fixed-order
// sum of the per-block partials of a row (so the result does not depend on
// scheduling).  For complex64 states this keeps FP64 off the per-amplitude
// path (GB300's FP64 rate is a small fraction of its FP32 rate) while the
// 2^n-term reduction carries FP64 error.
#include <cuda_runtime.h>

#include <algorithm>

#include "dq_common.cuh"
#include "dq_plan.h"
#include "dq_tma.cuh"

namespace dq {

namespace {

constexpr int kNormThreads = 256;
constexpr int kNormRun = 8;   // amplitudes summed in the state's precision before FP64

template <typename R>
__global__ void __launch_bounds__(kNormThreads)
k_norm_part(const cx<R> *__restrict__ st, int n, int bpr, double *__restrict__ part) {
    __shared__ double wsum[kNormThreads / 32];
    const int64_t dim = int64_t(1) << n;
    const int64_t row = blockIdx.x / bpr;
    const int64_t blk = blockIdx.x - row * bpr;
    const int64_t per = dim / bpr;     // dim and bpr are powers of two, bpr <= dim
    const cx<R> *p = st + row * dim + blk * per;
    double acc = 0.0;
    for (int64_t i0 = threadIdx.x; i0 < per; i0 += (int64_t)kNormThreads * kNormRun) {
        R s = R(0);
#pragma unroll
        for (int j = 0; j < kNormRun; ++j) {
            const int64_t i = i0 + (int64_t)j * kNormThreads;
            if (i < per) {
                const cx<R> x = p[i];
                s += x.x * x.x + x.y * x.y;
            }
        }
        acc += (double)s;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kNormThreads / 32; ++w) t += wsum[w];
        part[blockIdx.x] = t;
    }
}

__global__ void k_norm_finalize(const double *__restrict__ part, int bpr, int batch, double *__restrict__ out) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= batch) return;
    double t = 0.0;
    for (int b = 0; b < bpr; ++b) t += part[(int64_t)row * bpr + b];
    out[row] = t;
}

// One thread waits on an mbarrier that nothing arrives on and that no copy
// targets, with the context's wait limit; when the wait runs out it records
// the timeout in the error flag, exactly as a kernel whose copy never landed
// would.  Nothing is in flight, so the kernel simply returns.
__global__ void k_wait_expiry(int *errflag) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    if (!mbar_wait_bounded(&bar, 0u, wait_limit_ns(errflag))) atomicCAS(errflag, 0, DEVERR_TIMEOUT);
}

#ifdef DQ_BOUNDS_BUILD
// One check that fails (index 1 against a limit of 0) and guards nothing:
// the bounds-checking build records it as it would a bad index of a kernel.
__global__ void k_bounds_selftest() {
    if (threadIdx.x == 0 && !DQ_INB(1, 0)) return;
}
#endif

}  // namespace

int norm_blocks_per_row(int n, int batch) {
    // about four blocks per SM in total, each over at least 2048 amplitudes
    int bpr = 1;
    while (bpr < 1024 && ((int64_t)batch * bpr * 2) <= 1024 && (int64_t(1) << n) / (bpr * 2) >= 2048) bpr *= 2;
    return bpr;
}

size_t norm_part_bytes(int n, int batch) { return (size_t)batch * norm_blocks_per_row(n, batch) * sizeof(double); }

template <typename R>
cudaError_t state_norm(const void *state, int n, int batch, double *part, double *out, cudaStream_t s,
                       int64_t *launches) {
    const int bpr = norm_blocks_per_row(n, batch);
    {
        LaunchScope ls(s, "k_norm_part", launches);
        k_norm_part<R><<<(unsigned)((int64_t)batch * bpr), kNormThreads, 0, s>>>((const cx<R> *)state, n, bpr, part);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    LaunchScope ls(s, "k_norm_finalize", launches);
    k_norm_finalize<<<(unsigned)((batch + 127) / 128), 128, 0, s>>>(part, bpr, batch, out);
    return cudaGetLastError();
}

cudaError_t selftest_wait_expiry(int *errflag, cudaStream_t s, int64_t *launches) {
    LaunchScope ls(s, "k_wait_expiry", launches);
    k_wait_expiry<<<1, 32, 0, s>>>(errflag);
    return cudaGetLastError();
}

cudaError_t selftest_bounds(cudaStream_t s, int64_t *launches) {
#ifdef DQ_BOUNDS_BUILD
    LaunchScope ls(s, "k_bounds_selftest", launches);
    k_bounds_selftest<<<1, 32, 0, s>>>();
    return cudaGetLastError();
#else
    (void)s;
    (void)launches;
    return cudaErrorNotSupported;
#endif
}

template cudaError_t state_norm<float>(const void *, int, int, double *, double *, cudaStream_t, int64_t *);
template cudaError_t state_norm<double>(const void *, int, int, double *, double *, cudaStream_t, int64_t *);

}  // namespace dq
