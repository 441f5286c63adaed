// Shot sampling: basis-state outcomes drawn from |psi_row|^2 by inversion.
//
// The measurement of the paper's qubit API (Sec. "Quantum Computing with
// Qubits", API Overview: measure(shots, wires)) samples outcomes with the
// Born probabilities p_i = |psi_i|^2.  Shot s of row r takes a uniform
// u in [0, 1) and returns the smallest index i with u * Z < C(i), where
// C(i) = p_0 + ... + p_i and Z = C(2^n - 1) (dividing by Z absorbs the
// rounding of the state's norm).
//
// Layout of the cumulative sums: a row of 2^n amplitudes is cut into chunks
// of 2^c amplitudes (c = min(8, n)) and the chunks into groups of 2^g chunks
// (g = min(10, n - c)).  k_chunk_sums streams the state once (one CTA per
// group, a warp per chunk) and writes every chunk's probability and every
// group's total, each summed in a fixed order; k_group_scan forms each row's
// exclusive prefix over its groups and the row total Z.  k_draw then gives
// each shot one warp: a 32-way search over the group prefixes, a scan of the
// group's chunk sums, and a scan of the chunk's amplitudes -- 2^c amplitudes
// and 2^g chunk sums per shot, the latter usually from L2.
//
// Scans inside k_draw add in a different order than k_chunk_sums did, so a
// target within rounding of a group or chunk boundary can run past the last
// element of the chosen group or chunk; the draw then takes the last element
// with non-zero probability there, which is a valid outcome for that target.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dq_common.cuh"
#include "dq_plan.h"
#include "dq_sample.h"

namespace dq {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

template <typename R>
__device__ __forceinline__ double born(cx<R> a) {
    return (double)a.x * (double)a.x + (double)a.y * (double)a.y;
}

// One CTA per group: warp w sums chunks w, w + 8, ... of the group (lanes
// stride over the chunk's amplitudes), then the CTA adds the warps' partial
// totals in warp order.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_chunk_sums(const cx<R> *__restrict__ st, SampleGeom G,
                                                         double *__restrict__ chunk, double *__restrict__ group) {
    __shared__ double wsum[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t grp = blockIdx.x;                     // row * ngroups + group
    const int L = 1 << G.c, K = 1 << G.g;
    const int64_t ch0 = grp << G.g;
    double acc = 0.0;
    for (int k = warp; k < K; k += kWarps) {
        const cx<R> *p = st + ((ch0 + k) << G.c);
        double s = 0.0;
#pragma unroll 8
        for (int i = lane; i < L; i += 32) s += born<R>(p[i]);
        s = warp_sum(s);
        if (lane == 0) chunk[ch0 + k] = s;
        acc += s;
    }
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kWarps; ++w) t += wsum[w];
        group[grp] = t;
    }
}

// One CTA per row: exclusive prefix of the row's group totals, then the row
// total at index ngroups.  pre has ngroups + 1 entries per row.
__global__ void __launch_bounds__(1024) k_group_scan(const double *__restrict__ group, int64_t ngroups,
                                                     double *__restrict__ pre) {
    __shared__ double part[32];
    const int64_t row = blockIdx.x;
    const double *in = group + row * ngroups;
    double *out = pre + row * (ngroups + 1);
    const int T = blockDim.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t per = (ngroups + T - 1) / T;
    const int64_t b = min(ngroups, (int64_t)t * per), e = min(ngroups, b + per);
    double loc = 0.0;
    for (int64_t k = b; k < e; ++k) loc += in[k];
    // exclusive scan of loc over the block
    double incl = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) part[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = T >> 5;
        double v = lane < nw ? part[lane] : 0.0;
        double x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane < nw) part[lane] = x - v;            // exclusive warp offsets
        if (lane == nw - 1) out[ngroups] = x;         // row total Z
    }
    __syncthreads();
    double run = part[warp] + incl - loc;
    for (int64_t k = b; k < e; ++k) {
        out[k] = run;
        run += in[k];
    }
}

// splitmix64 (Steele, Lea & Flood, OOPSLA 2014): output k of the stream
// seeded with `seed`, as a double in [0, 1) from its top 53 bits.
__device__ __forceinline__ double splitmix_uniform(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// Warp search for the first element whose running sum exceeds `target`:
// values are read 32 at a time (value j * 32 + lane in round j), scanned
// across the warp and added to the running base.  Returns the element index,
// or -1 when the sum of all `count` values does not exceed target; `last_nz`
// receives the last element with a positive value (or -1).  `before`
// receives the running sum in front of the returned element.
template <typename F>
__device__ __forceinline__ int warp_find(F value, int count, double target, int lane, int &last_nz,
                                         double &before) {
    double base = 0.0;
    last_nz = -1;
    for (int j0 = 0; j0 < count; j0 += 32) {
        const int i = j0 + lane;
        const double v = i < count ? value(i) : 0.0;
        double incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t hit = __ballot_sync(0xffffffffu, i < count && base + incl > target);
        const uint32_t nz = __ballot_sync(0xffffffffu, v > 0.0);
        if (nz) last_nz = j0 + 31 - __clz(nz);
        if (hit) {
            const int l = __ffs(hit) - 1;
            before = base + __shfl_sync(0xffffffffu, incl - v, l);
            return j0 + l;
        }
        base += __shfl_sync(0xffffffffu, incl, 31);
    }
    before = base;
    return -1;
}

// Packed outcome of the wires in `wmask` (bit q = wire q), the lowest
// selected wire first (most significant); wmask == 0: the full index.
__device__ __forceinline__ int64_t pack_outcome(uint64_t idx, int n, uint64_t wmask) {
    if (!wmask) return (int64_t)idx;
    uint64_t r = 0;
    for (int q = 0; q < n; ++q)
        if ((wmask >> q) & 1) r = (r << 1) | ((idx >> (n - 1 - q)) & 1);
    return (int64_t)r;
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_draw(const cx<R> *__restrict__ st, SampleGeom G,
                                                   const double *__restrict__ chunk, const double *__restrict__ pre,
                                                   int64_t shots, const double *__restrict__ uniforms, uint64_t seed,
                                                   uint64_t wmask, int64_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = (int64_t)G.batch * shots;
    const int64_t ngroups = G.ngroups;
    const int K = 1 << G.g, L = 1 << G.c;
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < total; k += nwarps) {
        const int64_t row = k / shots;
        const double u = uniforms ? uniforms[k] : splitmix_uniform(seed, (uint64_t)k);
        const double *gp = pre + row * (ngroups + 1);
        const double target = u * gp[ngroups];
        // group: largest index with prefix <= target (32-way search)
        int64_t lo = 0, hi = ngroups;                  // answer in [lo, hi)
        while (hi - lo > 1) {
            const int64_t step = (hi - lo + 31) / 32;
            const int64_t probe = lo + (int64_t)lane * step;
            const bool le = probe < hi && gp[probe] <= target;
            const uint32_t m = __ballot_sync(0xffffffffu, le);
            const int l = 31 - __clz(m | 1u);          // last lane with prefix <= target (lane 0 always)
            lo = lo + (int64_t)l * step;
            hi = min(hi, lo + step);
        }
        const int64_t grp = row * ngroups + lo;
        const double gtarget = target - gp[lo];
        const double *cs = chunk + (grp << G.g);
        int cnz;
        double cbefore;
        int ci = warp_find([&](int i) { return cs[i]; }, K, gtarget, lane, cnz, cbefore);
        if (ci < 0) {
            ci = cnz >= 0 ? cnz : K - 1;
            cbefore = 0.0;
            for (int i = 0; i < ci; ++i) cbefore += cs[i];
        }
        const int64_t c0 = ((grp << G.g) + ci) << G.c;
        const cx<R> *amp = st + c0;
        int anz;
        double abefore;
        int ai = warp_find([&](int i) { return born<R>(amp[i]); }, L, gtarget - cbefore, lane, anz, abefore);
        if (ai < 0) ai = anz >= 0 ? anz : L - 1;
        if (lane == 0) out[k] = pack_outcome((uint64_t)(c0 - (row << G.n)) + (uint64_t)ai, G.n, wmask);
    }
}

}  // namespace

SampleGeom sample_geom(int n, int batch) {
    SampleGeom G;
    G.n = n;
    G.batch = batch;
    G.c = n < 8 ? n : 8;
    G.g = (n - G.c) < 10 ? (n - G.c) : 10;
    G.ngroups = (int64_t)1 << (n - G.c - G.g);
    return G;
}

size_t sample_workspace_bytes(int n, int batch) {
    const SampleGeom G = sample_geom(n, batch);
    const size_t nch = (size_t)batch << (n - G.c);
    const size_t ng = (size_t)batch * (size_t)G.ngroups;
    const size_t pre = (size_t)batch * (size_t)(G.ngroups + 1);
    return (nch + ng + pre) * sizeof(double) + 3 * 256;
}

template <typename R>
cudaError_t sample_run(const void *state, int n, int batch, int64_t shots, const double *uniforms, uint64_t seed,
                       uint64_t wmask, int64_t *out, void *ws, int nsm, cudaStream_t s, int64_t *launches) {
    const SampleGeom G = sample_geom(n, batch);
    char *w = (char *)ws;
    auto take = [&](size_t bytes) {
        void *p = w;
        w += (bytes + 255) & ~size_t(255);
        return p;
    };
    double *chunk = (double *)take(((size_t)batch << (n - G.c)) * sizeof(double));
    double *group = (double *)take((size_t)batch * (size_t)G.ngroups * sizeof(double));
    double *pre = (double *)take((size_t)batch * (size_t)(G.ngroups + 1) * sizeof(double));
    const cx<R> *st = (const cx<R> *)state;
    {
        LaunchScope ls(s, "k_chunk_sums", launches);
        k_chunk_sums<R><<<(unsigned)((int64_t)batch * G.ngroups), kThreads, 0, s>>>(st, G, chunk, group);
    }
    {
        LaunchScope ls(s, "k_group_scan", launches);
        const int t = G.ngroups >= 1024 ? 1024 : (G.ngroups >= 256 ? 256 : 32);
        k_group_scan<<<batch, t, 0, s>>>(group, G.ngroups, pre);
    }
    const int64_t total = (int64_t)batch * shots;
    const int64_t want = (total + kWarps - 1) / kWarps;
    const int64_t cap = (int64_t)nsm * 16;
    {
        LaunchScope ls(s, "k_draw", launches);
        k_draw<R><<<(unsigned)(want < cap ? want : cap), kThreads, 0, s>>>(st, G, chunk, pre, shots, uniforms,
                                                                           seed, wmask, out);
    }
    return cudaGetLastError();
}

template cudaError_t sample_run<float>(const void *, int, int, int64_t, const double *, uint64_t, uint64_t,
                                       int64_t *, void *, int, cudaStream_t, int64_t *);
template cudaError_t sample_run<double>(const void *, int, int, int64_t, const double *, uint64_t, uint64_t,
                                        int64_t *, void *, int, cudaStream_t, int64_t *);

}  // namespace dq
