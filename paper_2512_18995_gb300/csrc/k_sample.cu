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
// (g chosen so that a row has min(1024, 2^(n-c)) or more groups, g <= 10).
// k_chunk_sums streams the state once (one CTA per group, a warp per chunk)
// and writes, per group, the inclusive prefix sums of its chunks'
// probabilities and the group total, each added in a fixed order;
// k_group_scan forms each row's inclusive prefix over its groups (the last
// entry is the row total Z).  k_draw then gives each shot one warp: a 32-way
// search over the group prefixes, another over the group's chunk prefixes,
// and a scan of the chunk's 2^c amplitudes (eight per lane, one round of
// loads) -- a handful of dependent memory rounds per shot.
//
// Precision: GB300's FP64 rate is a small fraction of its FP32 rate, and
// per-amplitude (or per-shot, per-comparison) FP64 instructions would cost
// more than the memory traffic.  For complex64 states every probability,
// partial sum, prefix and comparison is therefore an unevaluated float pair
// hi + lo built with error-free transformations (TwoSum and the FMA residual
// of a product: Dekker 1971; Knuth, TAOCP vol. 2, 4.2.2), about 44 bits of
// precision; a shot converts only its uniform from FP64.  Probabilities
// below the smallest FP32 subnormal count as zero.  Complex128 states use
// FP64 throughout.
//
// The prefixes of different levels are added separately, so a target within
// rounding of a boundary can run past the end of the chosen group or chunk;
// the search then takes the first group (chunk) at which the prefix reaches
// the total, and the amplitude scan the last amplitude with non-zero
// probability of the chunk: a valid outcome for that target either way.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dq_common.cuh"
#include "dq_plan.h"
#include "dq_sample.h"

namespace dq {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// Unevaluated float pair hi + lo, normalised (hi = fl(hi + lo)), so that
// pairs compare lexicographically.
struct FF {
    float hi, lo;
};

// s + e = a + b exactly (TwoSum; the _rn intrinsics keep the compiler from
// contracting or reassociating the steps).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

__device__ __forceinline__ FF ff_norm(float s, float e) {
    const float h = __fadd_rn(s, e);
    return FF{h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return ff_norm(s, e);
}

// Probability accumulator and prefix type: float pairs for complex64
// amplitudes, double for complex128.
template <typename R> struct Acc;
template <> struct Acc<float> {
    using T = FF;
    static __device__ __forceinline__ T zero() { return FF{0.f, 0.f}; }
    // |a|^2 = x^2 + y^2: each square split exactly into float + FMA residual
    static __device__ __forceinline__ T prob(float2 a) {
        const float h1 = __fmul_rn(a.x, a.x), l1 = __fmaf_rn(a.x, a.x, -h1);
        const float h2 = __fmul_rn(a.y, a.y), l2 = __fmaf_rn(a.y, a.y, -h2);
        float s, e;
        two_sum(h1, h2, s, e);
        return ff_norm(s, __fadd_rn(e, __fadd_rn(l1, l2)));
    }
    static __device__ __forceinline__ T add(T a, T b) { return ff_add(a, b); }
    static __device__ __forceinline__ T sub(T a, T b) { return ff_add(a, FF{-b.hi, -b.lo}); }
    static __device__ __forceinline__ bool gt(T a, T b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
    static __device__ __forceinline__ bool ge(T a, T b) { return a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo); }
    static __device__ __forceinline__ bool positive(T a) { return a.hi > 0.f; }
    // u (FP64, in [0, 1)) times z, as a pair: u split into two floats, then
    // the products with the FMA residual of the leading one
    static __device__ __forceinline__ T scale(double u, T z) {
        const float uh = __double2float_rn(u);
        const float ul = __double2float_rn(u - (double)uh);
        const float p = __fmul_rn(uh, z.hi);
        float e = __fmaf_rn(uh, z.hi, -p);
        e = __fadd_rn(e, __fadd_rn(__fmul_rn(uh, z.lo), __fmul_rn(ul, z.hi)));
        return ff_norm(p, e);
    }
    static __device__ __forceinline__ T shfl_up(T a, int o) {
        return FF{__shfl_up_sync(0xffffffffu, a.hi, o), __shfl_up_sync(0xffffffffu, a.lo, o)};
    }
    static __device__ __forceinline__ T shfl_xor(T a, int o) {
        return FF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
    }
    static __device__ __forceinline__ T shfl(T a, int l) {
        return FF{__shfl_sync(0xffffffffu, a.hi, l), __shfl_sync(0xffffffffu, a.lo, l)};
    }
};
template <> struct Acc<double> {
    using T = double;
    static __device__ __forceinline__ T zero() { return 0.0; }
    static __device__ __forceinline__ T prob(double2 a) { return a.x * a.x + a.y * a.y; }
    static __device__ __forceinline__ T add(T a, T b) { return a + b; }
    static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
    static __device__ __forceinline__ bool gt(T a, T b) { return a > b; }
    static __device__ __forceinline__ bool ge(T a, T b) { return a >= b; }
    static __device__ __forceinline__ bool positive(T a) { return a > 0.0; }
    static __device__ __forceinline__ T scale(double u, T z) { return u * z; }
    static __device__ __forceinline__ T shfl_up(T a, int o) { return __shfl_up_sync(0xffffffffu, a, o); }
    static __device__ __forceinline__ T shfl_xor(T a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
    static __device__ __forceinline__ T shfl(T a, int l) { return __shfl_sync(0xffffffffu, a, l); }
};

// Exclusive prefix of `loc` over the block (threads in order; lanes are
// scanned within a warp, warps' totals added in warp order); part holds one
// entry per warp.
template <typename A>
__device__ __forceinline__ typename A::T block_excl(typename A::T loc, typename A::T *part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    typename A::T incl = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const typename A::T y = A::shfl_up(incl, o);
        if (lane >= o) incl = A::add(y, incl);
    }
    if (lane == 31) part[warp] = incl;
    __syncthreads();
    typename A::T off = A::zero();
    for (int w = 0; w < warp; ++w) off = A::add(off, part[w]);
    typename A::T before = A::shfl_up(incl, 1);
    if (lane == 0) before = A::zero();
    return A::add(off, before);
}

// One CTA per group: warp w sums chunks w, w + 8, ... of the group (lanes
// stride over the chunk's amplitudes) into shared memory; the CTA then forms
// the inclusive prefix over the group's chunks (thread t adds its run of
// consecutive chunks in order, then the runs are scanned) and the total.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_chunk_sums(const cx<R> *__restrict__ st, SampleGeom G,
                                                         typename Acc<R>::T *__restrict__ cpre,
                                                         typename Acc<R>::T *__restrict__ group) {
    using A = Acc<R>;
    using T = typename A::T;
    __shared__ T sums[1024];
    __shared__ T part[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t grp = blockIdx.x;                     // row * ngroups + group
    const int L = 1 << G.c, K = 1 << G.g;
    const int64_t ch0 = grp << G.g;
    for (int k = warp; k < K; k += kWarps) {
        const cx<R> *p = st + ((ch0 + k) << G.c);
        T s = A::zero();
#pragma unroll 8
        for (int i = lane; i < L; i += 32) s = A::add(s, A::prob(p[i]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = A::add(s, A::shfl_xor(s, o));
        if (lane == 0) sums[k] = s;
    }
    __syncthreads();
    // run of consecutive chunks per thread (K <= 1024, 256 threads)
    const int per = (K + kThreads - 1) / kThreads;
    const int b = min(K, (int)threadIdx.x * per), e = min(K, b + per);
    T loc = A::zero();
    for (int k = b; k < e; ++k) loc = A::add(loc, sums[k]);
    T run = block_excl<A>(loc, part);
    for (int k = b; k < e; ++k) {
        run = A::add(run, sums[k]);
        cpre[ch0 + k] = run;
    }
    if (e == K && b < e) group[grp] = run;
}

// One CTA per row: inclusive prefix of the row's group totals (the last
// entry is the row total Z).
template <typename R>
__global__ void __launch_bounds__(1024) k_group_scan(const typename Acc<R>::T *__restrict__ group, int64_t ngroups,
                                                     typename Acc<R>::T *__restrict__ gpre) {
    using A = Acc<R>;
    using T = typename A::T;
    __shared__ T part[32];
    const int64_t row = blockIdx.x;
    const T *in = group + row * ngroups;
    T *out = gpre + row * ngroups;
    const int nt = blockDim.x;
    const int64_t per = (ngroups + nt - 1) / nt;
    const int64_t b = min(ngroups, (int64_t)threadIdx.x * per), e = min(ngroups, b + per);
    T loc = A::zero();
    for (int64_t k = b; k < e; ++k) loc = A::add(loc, in[k]);
    T run = block_excl<A>(loc, part);
    for (int64_t k = b; k < e; ++k) {
        run = A::add(run, in[k]);
        out[k] = run;
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

// First index i in [0, count) with pre[i] > x (strict) or >= x (!strict),
// for non-decreasing pre; count when there is none.  32-way search by the
// whole warp: every round probes 32 evenly spaced positions.
template <typename A>
__device__ __forceinline__ int64_t warp_first(const typename A::T *__restrict__ pre, int64_t count,
                                              typename A::T x, bool strict, int lane) {
    int64_t lo = 0, hi = count;    // answer in [lo, hi]; hi == count: none found yet
    while (lo < hi) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t probe = lo + (int64_t)lane * step;
        bool t = false;
        if (probe < hi) {
            const typename A::T v = pre[probe];
            t = strict ? A::gt(v, x) : A::ge(v, x);
        }
        const uint32_t m = __ballot_sync(0xffffffffu, t);
        const uint32_t valid = __ballot_sync(0xffffffffu, probe < hi);
        if (m) {
            const int f = __ffs(m) - 1;
            hi = lo + (int64_t)f * step;
            lo = f > 0 ? lo + (int64_t)(f - 1) * step + 1 : lo;
        } else {
            const int last = 31 - __clz(valid);
            lo = lo + (int64_t)last * step + 1;
        }
    }
    return lo;
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

constexpr int kAmpPerLane = 8;   // 2^8 amplitudes per chunk over 32 lanes

template <typename R>
__global__ void __launch_bounds__(kThreads) k_draw(const cx<R> *__restrict__ st, SampleGeom G,
                                                   const typename Acc<R>::T *__restrict__ cpre,
                                                   const typename Acc<R>::T *__restrict__ gpre, int64_t shots,
                                                   const double *__restrict__ uniforms, uint64_t seed, uint64_t wmask,
                                                   int64_t *__restrict__ out) {
    using A = Acc<R>;
    using T = typename A::T;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = (int64_t)G.batch * shots;
    const int64_t ngroups = G.ngroups;
    const int K = 1 << G.g, L = 1 << G.c;
    const int per = L >= 32 * kAmpPerLane ? kAmpPerLane : (L + 31) / 32;   // amplitudes per lane (L <= 256)
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < total; k += nwarps) {
        const int64_t row = G.batch == 1 ? 0 : k / shots;
        const double u = uniforms ? uniforms[k] : splitmix_uniform(seed, (uint64_t)k);
        const T *gp = gpre + row * ngroups;
        const T z = gp[ngroups - 1];
        if (!A::positive(z)) {   // a row without probability: the last index, as documented
            if (lane == 0) out[k] = pack_outcome((uint64_t(1) << G.n) - 1, G.n, wmask);
            continue;
        }
        const T target = A::scale(u, z);
        // group: first inclusive prefix above the target, else the first at the total
        int64_t g = warp_first<A>(gp, ngroups, target, true, lane);
        if (g == ngroups) g = warp_first<A>(gp, ngroups, z, false, lane);
        if (g == ngroups) g = ngroups - 1;
        const T tg = g > 0 ? A::sub(target, gp[g - 1]) : target;
        const int64_t grp = row * ngroups + g;
        const T *cp = cpre + (grp << G.g);
        int64_t ch = warp_first<A>(cp, K, tg, true, lane);
        if (ch == K) ch = warp_first<A>(cp, K, cp[K - 1], false, lane);
        if (ch == K) ch = K - 1;
        const T ta = ch > 0 ? A::sub(tg, cp[ch - 1]) : tg;
        // amplitudes: lane l holds [l * per, l * per + per) of the chunk
        const int64_t c0 = ((grp << G.g) + ch) << G.c;
        const cx<R> *amp = st + c0;
        T pr[kAmpPerLane];
        T mine = A::zero();
#pragma unroll
        for (int j = 0; j < kAmpPerLane; ++j) {
            const int i = lane * per + j;
            pr[j] = (j < per && i < L) ? A::prob(amp[i]) : A::zero();
            mine = A::add(mine, pr[j]);
        }
        // inclusive scan of the lanes' sums (lane order = index order)
        T incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = A::shfl_up(incl, o);
            if (lane >= o) incl = A::add(y, incl);
        }
        T before = A::shfl_up(incl, 1);
        if (lane == 0) before = A::zero();
        const uint32_t hit = __ballot_sync(0xffffffffu, A::gt(incl, ta));
        const uint32_t nz = __ballot_sync(0xffffffffu, A::positive(mine));
        int a;
        if (hit) {
            const int l = __ffs(hit) - 1;
            // walk lane l's run in order, starting from the sum of the lanes before it
            T run = A::shfl(before, l);
            int pick = -1, lastnz = -1;
#pragma unroll
            for (int j = 0; j < kAmpPerLane; ++j) {
                if (lane == l && j < per) {
                    run = A::add(run, pr[j]);
                    if (A::positive(pr[j])) lastnz = j;
                    if (pick < 0 && A::gt(run, ta)) pick = j;
                }
            }
            pick = __shfl_sync(0xffffffffu, pick >= 0 ? pick : lastnz, l);
            a = l * per + (pick >= 0 ? pick : per - 1);
        } else {
            // rounding ran past the chunk: its last amplitude with non-zero probability
            const int l = nz ? 31 - __clz(nz) : 31;
            int lastnz = -1;
#pragma unroll
            for (int j = 0; j < kAmpPerLane; ++j)
                if (lane == l && j < per && A::positive(pr[j])) lastnz = j;
            lastnz = __shfl_sync(0xffffffffu, lastnz, l);
            a = l * per + (lastnz >= 0 ? lastnz : per - 1);
        }
        if (a >= L) a = L - 1;
        if (lane == 0) out[k] = pack_outcome((uint64_t)(c0 - (row << G.n)) + (uint64_t)a, G.n, wmask);
    }
}

}  // namespace

SampleGeom sample_geom(int n, int batch) {
    SampleGeom G;
    G.n = n;
    G.batch = batch;
    G.c = n < 8 ? n : 8;
    const int rest = n - G.c;                 // chunk-index bits of a row
    G.g = rest <= 10 ? 0 : (rest - 10 < 10 ? rest - 10 : 10);
    G.ngroups = (int64_t)1 << (rest - G.g);
    return G;
}

size_t sample_workspace_bytes(int n, int batch) {
    const SampleGeom G = sample_geom(n, batch);
    const size_t nch = (size_t)batch << (n - G.c);
    const size_t ng = (size_t)batch * (size_t)G.ngroups;
    return (nch + 2 * ng) * 8 + 3 * 256;      // 8-byte prefixes (float pair or double)
}

template <typename R>
cudaError_t sample_run(const void *state, int n, int batch, int64_t shots, const double *uniforms, uint64_t seed,
                       uint64_t wmask, int64_t *out, void *ws, int nsm, cudaStream_t s, int64_t *launches) {
    using T = typename Acc<R>::T;
    static_assert(sizeof(T) == 8, "prefix entries are 8 bytes");
    const SampleGeom G = sample_geom(n, batch);
    char *w = (char *)ws;
    auto take = [&](size_t bytes) {
        void *p = w;
        w += (bytes + 255) & ~size_t(255);
        return p;
    };
    T *cpre = (T *)take(((size_t)batch << (n - G.c)) * sizeof(T));
    T *group = (T *)take((size_t)batch * (size_t)G.ngroups * sizeof(T));
    T *gpre = (T *)take((size_t)batch * (size_t)G.ngroups * sizeof(T));
    const cx<R> *st = (const cx<R> *)state;
    {
        LaunchScope ls(s, "k_chunk_sums", launches);
        k_chunk_sums<R><<<(unsigned)((int64_t)batch * G.ngroups), kThreads, 0, s>>>(st, G, cpre, group);
    }
    {
        LaunchScope ls(s, "k_group_scan", launches);
        const int t = G.ngroups >= 1024 ? 1024 : (G.ngroups >= 256 ? 256 : 32);
        k_group_scan<R><<<batch, t, 0, s>>>(group, G.ngroups, gpre);
    }
    const int64_t total = (int64_t)batch * shots;
    const int64_t want = (total + kWarps - 1) / kWarps;
    const int64_t cap = (int64_t)nsm * 32;
    {
        LaunchScope ls(s, "k_draw", launches);
        k_draw<R><<<(unsigned)(want < cap ? want : cap), kThreads, 0, s>>>(st, G, cpre, gpre, shots, uniforms,
                                                                           seed, wmask, out);
    }
    return cudaGetLastError();
}

template cudaError_t sample_run<float>(const void *, int, int, int64_t, const double *, uint64_t, uint64_t,
                                       int64_t *, void *, int, cudaStream_t, int64_t *);
template cudaError_t sample_run<double>(const void *, int, int, int64_t, const double *, uint64_t, uint64_t,
                                        int64_t *, void *, int, cudaStream_t, int64_t *);

}  // namespace dq
