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
// of 2^c amplitudes (c = min(5, n): one amplitude per lane of a warp) and the
// chunks into groups of 2^g chunks (g chosen so that a row has
// min(1024, 2^(n-c)) or more groups, g <= 10).  k_chunk_sums streams the
// state once (one CTA per group; a warp reads eight chunks at a time,
// coalesced, and sums them with a butterfly that exchanges half of its
// partial sums at each step) and writes, per group, the inclusive prefix
// sums of its chunks' probabilities and the group total, each added in a
// fixed order; k_group_scan forms each row's inclusive prefix over its groups
// (the last entry is the row total Z).  k_draw then gives each shot one
// thread: a binary search over the group prefixes, another over the group's
// chunk prefixes, and an in-order scan of the chunk's 2^c amplitudes (256
// contiguous bytes).  A warp per shot (32-way searches, a lane scan) spent
// about 600 warp instructions per shot and was bound by instruction issue; a
// thread per shot trades them for chains of dependent loads that the many
// resident threads overlap.  The chunk prefixes take 8 bytes per 32
// amplitudes, 1/32 of a complex64 state.
//
// Precision: GB300's FP64 rate is a small fraction of its FP32 rate, and
// per-amplitude (or per-shot, per-comparison) FP64 instructions would cost
// more than the memory traffic.  For complex64 states every probability,
// partial sum, prefix and comparison is therefore an unevaluated float pair
// hi + lo built with error-free transformations (TwoSum and the FMA residual
// of a product: Dekker 1971; Knuth, TAOCP vol. 2, 4.2.2), about 44 bits of
// precision; a shot splits its uniform into such a pair from the fields of
// its double with integer operations (no FP64 instruction).  Probabilities
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
    // u times z as a pair, for u = uh + ul (|ul| <= 2^-23 uh): the
    // product of the leading parts with its FMA residual, plus the cross terms
    static __device__ __forceinline__ T scale(float uh, float ul, T z) {
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
    if (L == 32 && K >= 8) {
        // eight 32-amplitude chunks per warp step: load j is amplitude `lane`
        // of chunk j.  Lane bits 4, 3 and 2 each halve the chunks a lane
        // keeps (it sends the other half to its partner and adds what it
        // receives), leaving chunk lane >> 2 summed over eight lanes; bits 0
        // and 1 then complete the sum over the warp.
        const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
        for (int kb = warp * 8; kb < K; kb += kWarps * 8) {
            const cx<R> *p = st + ((ch0 + kb) << 5) + lane;
            T v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = A::prob(p[j << 5]);
            T w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                w[j] = A::add(b4 ? v[j + 4] : v[j], A::shfl_xor(b4 ? v[j] : v[j + 4], 16));
            T x[2];
#pragma unroll
            for (int j = 0; j < 2; ++j)
                x[j] = A::add(b3 ? w[j + 2] : w[j], A::shfl_xor(b3 ? w[j] : w[j + 2], 8));
            T y = A::add(b2 ? x[1] : x[0], A::shfl_xor(b2 ? x[0] : x[1], 4));
            y = A::add(y, A::shfl_xor(y, 1));
            y = A::add(y, A::shfl_xor(y, 2));
            if ((lane & 3) == 0) sums[kb + (lane >> 2)] = y;
        }
    } else {
        // chunks under 32 amplitudes (n < 5) or groups under eight chunks: a warp per chunk
        for (int k = warp; k < K; k += kWarps) {
            const cx<R> *p = st + ((ch0 + k) << G.c);
            T s = lane < L ? A::prob(p[lane]) : A::zero();
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s = A::add(s, A::shfl_xor(s, o));
            if (lane == 0) sums[k] = s;
        }
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
// entry is the row total Z).  The row is taken in tiles of 8 entries per
// thread (thread t reads entries 8t .. 8t + 7 of the tile, consecutive); a
// tile's prefix is the carry of the tiles before it, the block's exclusive
// prefix of the threads' sums, then the thread's entries in order.
template <typename R>
__global__ void __launch_bounds__(1024) k_group_scan(const typename Acc<R>::T *__restrict__ group, int64_t ngroups,
                                                     typename Acc<R>::T *__restrict__ gpre) {
    using A = Acc<R>;
    using T = typename A::T;
    constexpr int P = 8;
    __shared__ T part[32];
    __shared__ T carry_s;
    const int64_t row = blockIdx.x;
    const T *in = group + row * ngroups;
    T *out = gpre + row * ngroups;
    const int nt = blockDim.x;
    T carry = A::zero();
    for (int64_t base = 0; base < ngroups; base += (int64_t)nt * P) {
        const int64_t b = base + (int64_t)threadIdx.x * P;
        T v[P];
        T loc = A::zero();
#pragma unroll
        for (int j = 0; j < P; ++j) {
            v[j] = b + j < ngroups ? in[b + j] : A::zero();
            loc = A::add(loc, v[j]);
        }
        T run = A::add(carry, block_excl<A>(loc, part));
#pragma unroll
        for (int j = 0; j < P; ++j) {
            run = A::add(run, v[j]);
            if (b + j < ngroups) out[b + j] = run;
        }
        __syncthreads();                      // part[] is read before the next tile writes it
        if (threadIdx.x == nt - 1) carry_s = run;
        __syncthreads();
        carry = carry_s;
    }
}

// splitmix64 (Steele, Lea & Flood, OOPSLA 2014): output k of the stream
// seeded with `seed`; its top 53 bits m give the uniform m * 2^-53 in [0, 1).
__device__ __forceinline__ uint64_t splitmix_bits53(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z >> 11;
}

__device__ __forceinline__ double splitmix_uniform(uint64_t seed, uint64_t k) {
    return (double)splitmix_bits53(seed, k) * (1.0 / 9007199254740992.0);
}

// A uniform u = m * 2^(E - 1075), m in [2^52, 2^53) (the fields of the
// double u), as two floats u = uh + ul without FP64 arithmetic (GB300's FP64
// pipe is narrow, and every lane of a shot's warp needs the target):
// uh = (m >> 29) * 2^(E - 1046) exactly, ul = (m mod 2^29) * 2^(E - 1075)
// rounded to float.  u below 2^-126 counts as 0, u of 1 or more as 1.
__device__ __forceinline__ void split_uniform(int E, uint64_t m, float &uh, float &ul) {
    if (E < 897) {
        uh = 0.f;
        ul = 0.f;
        return;
    }
    if (E >= 1023) {
        uh = 1.f;
        ul = 0.f;
        return;
    }
    const uint32_t mh = (uint32_t)(m >> 29), ml = (uint32_t)m & 0x1FFFFFFFu;
    uh = __int_as_float(((E - 896) << 23) | (int)(mh & 0x7FFFFFu));
    ul = __fmul_rn(__fmul_rn(__uint2float_rn(ml), 0x1p-64f), __int_as_float((E - 884) << 23));
}

// The fields of a given FP64 uniform (negative values and -0 count as 0,
// NaN as 1).
__device__ __forceinline__ void split_given(double u, float &uh, float &ul) {
    const uint64_t b = (uint64_t)__double_as_longlong(u);
    if (b >> 63) {
        uh = 0.f;
        ul = 0.f;
        return;
    }
    const int E = (int)(b >> 52);
    split_uniform(E, (b & 0xFFFFFFFFFFFFFull) | (1ull << 52), uh, ul);
}

// The same fields for the stream's m * 2^-53: m normalised to [2^52, 2^53).
__device__ __forceinline__ void split_stream(uint64_t m, float &uh, float &ul) {
    if (m == 0) {
        uh = 0.f;
        ul = 0.f;
        return;
    }
    const int lz = __clzll((long long)m) - 11;    // leading zeros within 53 bits
    split_uniform(1022 - lz, m << lz, uh, ul);
}

// First index i in [0, count) with pre[i] > x (strict) or >= x (!strict),
// for non-decreasing pre; count when there is none.  Binary search by one
// thread.  (Rounds of three, seven or fifteen independent probes shorten the
// chain of dependent loads but measured slower: the draw is bound by the
// memory system's requests, not by the chain.)
template <typename A>
__device__ __forceinline__ int first_above(const typename A::T *__restrict__ pre, int count, typename A::T x,
                                           bool strict) {
    int lo = 0, hi = count;
    while (lo < hi) {
        const int mid = (int)(((unsigned)lo + (unsigned)hi) >> 1);
        const typename A::T v = pre[mid];
        if (strict ? A::gt(v, x) : A::ge(v, x))
            hi = mid;
        else
            lo = mid + 1;
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

// One thread per shot: the group (first inclusive prefix above the target,
// else the first at the total), the chunk within it (the same rule on the
// group's chunk prefixes and the remainder), then the chunk's amplitudes in
// order: the first whose running sum passes the remainder.  The running sum
// grows only at amplitudes with probability, so a zero-probability outcome
// is never chosen; when rounding runs past the chunk, its last amplitude with
// probability.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_draw(const cx<R> *__restrict__ st, SampleGeom G,
                                                   const typename Acc<R>::T *__restrict__ cpre,
                                                   const typename Acc<R>::T *__restrict__ gpre, int64_t shots,
                                                   const double *__restrict__ uniforms, uint64_t seed, uint64_t wmask,
                                                   int64_t *__restrict__ out) {
    using A = Acc<R>;
    using T = typename A::T;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t total = (int64_t)G.batch * shots;
    const int ngroups = (int)G.ngroups;
    const int K = 1 << G.g, L = 1 << G.c;   // L <= 32
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += nthreads) {
        const int64_t row = G.batch == 1 ? 0 : k / shots;
        const T *gp = gpre + row * ngroups;
        const T z = gp[ngroups - 1];
        if (!A::positive(z)) {   // a row without probability: the last index, as documented
            out[k] = pack_outcome((uint64_t(1) << G.n) - 1, G.n, wmask);
            continue;
        }
        T target;
        if constexpr (sizeof(R) == 4) {
            float uh, ul;
            if (uniforms)
                split_given(uniforms[k], uh, ul);
            else
                split_stream(splitmix_bits53(seed, (uint64_t)k), uh, ul);
            target = A::scale(uh, ul, z);
        } else {
            target = A::scale(uniforms ? uniforms[k] : splitmix_uniform(seed, (uint64_t)k), z);
        }
        int g = first_above<A>(gp, ngroups, target, true);
        if (g == ngroups) g = first_above<A>(gp, ngroups, z, false);
        if (g == ngroups) g = ngroups - 1;
        const T tg = g > 0 ? A::sub(target, gp[g - 1]) : target;
        const int64_t grp = row * ngroups + g;
        const T *cp = cpre + (grp << G.g);
        int ch = first_above<A>(cp, K, tg, true);
        if (ch == K) ch = first_above<A>(cp, K, cp[K - 1], false);
        if (ch == K) ch = K - 1;
        const T ta = ch > 0 ? A::sub(tg, cp[ch - 1]) : tg;
        const int64_t c0 = ((grp << G.g) + ch) << G.c;
        const cx<R> *amp = st + c0;
        T run = A::zero();
        int a = -1, lastnz = -1;
#pragma unroll 8
        for (int i = 0; i < L; ++i) {   // 8-byte loads (16-byte pairs measured slower)
            const T p = A::prob(amp[i]);
            if (A::positive(p)) {
                lastnz = i;
                run = A::add(run, p);
                if (a < 0 && A::gt(run, ta)) a = i;
            }
        }
        if (a < 0) a = lastnz >= 0 ? lastnz : L - 1;
        out[k] = pack_outcome((uint64_t)(c0 - (row << G.n)) + (uint64_t)a, G.n, wmask);
    }
}

}  // namespace

SampleGeom sample_geom(int n, int batch) {
    SampleGeom G;
    G.n = n;
    G.batch = batch;
    G.c = n < 5 ? n : 5;                      // 32-amplitude chunks: one amplitude per lane
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
        const int64_t want = (G.ngroups + 7) / 8;     // threads of 8 entries each, whole warps, <= 1024
        const int t = want >= 1024 ? 1024 : (int)((want + 31) / 32 * 32);
        k_group_scan<R><<<batch, t, 0, s>>>(group, G.ngroups, gpre);
    }
    const int64_t total = (int64_t)batch * shots;
    const int64_t want = (total + kThreads - 1) / kThreads;   // a thread per shot
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
