// Large-state observables and adjoint sweep on TMA-staged tiles.
//
// Observable passes (k_tile_obs): Pauli terms are grouped so that every
// term's flip bits lie inside the pass's tile.  For each tile the pass adds
// sum_l conj(psi[l ^ f]) ph(l) psi[l] to the term's expectation partial
// (API Overview: expectation of Pauli-string observables) and, for the
// adjoint method, lambda[l] += w c ph(l ^ f) psi[l ^ f] (lambda = sum_o w_o O_o
// psi), writing lambda back.  Products are formed in the state precision,
// warp sums too, and everything above a tile's warp sum is FP64.
//
// Reverse sweep (k_tile_adj): the passes of an adjoint schedule are visited
// last to first; each loads a psi tile and a lambda tile, runs the pass's gates
// in reverse on the in-register engine (gradient partial 2 Im <lambda|G|psi>
// of every parametric gate, then U^dagger on both vectors; Sec. "Distributed
// Simulations", adjoint differentiation) and stores both tiles.  Gradient
// partials are kept per CTA in FP64 and written per batch row to a
// [slot][row][cta] array that the deterministic slot reduction sums.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "dq_common.cuh"
#include "dq_engine.cuh"
#include "dq_plan.h"
#include "dq_tile.h"
#include "dq_tma.cuh"
#include "dq_tile_adj.cuh"
#include "dq_jit.h"

namespace dq {

namespace {

// One Pauli term of an observable pass, in the pass's tile coordinates.
struct OTerm {
    uint32_t floc;   // flip mask (local tile bits)
    uint32_t sloc;   // sign mask (local tile bits)
    uint64_t sout;   // sign mask outside the tile (amplitude bits)
    int32_t nY;
    int32_t term;    // global term index
    int32_t obs;
    int32_t pad;
    double coeff;
    double pad2;
};

struct OPass {
    std::vector<int> T;
    int t0 = 0, nt = 0;
};

struct ObsSchedule {
    int n = 0, k = 0, low = 0;
    std::vector<OPass> passes;
    std::vector<OTerm> terms;
    OTerm *d_terms = nullptr;
};

int dims_needed_obs(uint64_t T, int wb) {
    uint64_t w = (T << wb) | ((uint64_t(1) << wb) - 1);
    int dims = 0, b = 0;
    while (w >> b) {
        if (!((w >> b) & 1)) {
            ++b;
            continue;
        }
        int len = 0;
        while ((w >> (b + len)) & 1) ++len;
        dims += (len + 7) / 8;
        b += len;
    }
    return dims;
}

bool build_obs_schedule(const std::vector<DevTerm> &bits, int n, int k, int low, int wb, ObsSchedule &out) {
    out = ObsSchedule();
    out.n = n;
    out.k = k;
    out.low = low;
    const uint64_t lowmask = (uint64_t(1) << low) - 1;
    std::vector<int> remaining(bits.size());
    for (size_t i = 0; i < bits.size(); ++i) remaining[i] = (int)i;
    int guard = 0;
    while (!remaining.empty()) {
        if (++guard > (int)bits.size() + 2) return false;
        uint64_t T = lowmask;
        std::vector<int> take, rest;
        for (int i : remaining) {
            const uint64_t nt = T | bits[i].f;
            if (__builtin_popcountll(nt) <= k && dims_needed_obs(nt, wb) <= 5) {
                T = nt;
                take.push_back(i);
            } else {
                rest.push_back(i);
            }
        }
        if (take.empty()) return false;
        for (int b = 0; b < n && __builtin_popcountll(T) < k; ++b) {
            if ((T >> b) & 1) continue;
            const uint64_t nt = T | (uint64_t(1) << b);
            if (dims_needed_obs(nt, wb) <= 5) T = nt;
        }
        if (__builtin_popcountll(T) != k) return false;
        OPass ps;
        int loc[64];
        for (int b = 0, j = 0; b < n; ++b) {
            loc[b] = -1;
            if ((T >> b) & 1) {
                ps.T.push_back(b);
                loc[b] = j++;
            }
        }
        auto compress = [&](uint64_t m) {
            uint32_t r = 0;
            for (int b = 0; b < n; ++b)
                if (((m >> b) & 1) && loc[b] >= 0) r |= 1u << loc[b];
            return r;
        };
        ps.t0 = (int)out.terms.size();
        for (int i : take) {
            const DevTerm &d = bits[i];
            OTerm o{};
            o.floc = compress(d.f);
            o.sloc = compress(d.s & T);
            o.sout = d.s & ~T;
            o.nY = d.nY;
            o.term = i;
            o.obs = d.obs;
            o.coeff = d.coeff;
            out.terms.push_back(o);
        }
        ps.nt = (int)out.terms.size() - ps.t0;
        out.passes.push_back(ps);
        remaining.swap(rest);
    }
    return true;
}

template <typename R> struct AdjCfg;
template <> struct AdjCfg<float> { static constexpr int wb = 0; };
template <> struct AdjCfg<double> { static constexpr int wb = 1; };

// Tile width for observable and adjoint passes: two vectors are resident.
template <typename R>
void adjoint_tile(int n, int &k, int &low, int &M) {
    if (n >= 25) {
        M = sizeof(R) == 4 ? 4 : 3;
        k = sizeof(R) == 4 ? 12 : 11;
    } else {
        M = 3;
        k = std::max(kLaneBits + M, std::min(11, n - 9));
    }
    k = std::min(k, n - 1);
    M = std::min(M, k - kLaneBits);
    low = std::max(kLaneBits, std::min(7, k - 3));
    // complex64 states of 20 qubits or more: 12-qubit tiles, four register
    // bits and only the lane bits always resident, which leaves more tile
    // bits to the passes (measured on the 30-qubit QFT + ansatz reverse sweep:
    // 40 passes / 655 ms against 54 / 739 ms; on the 22-qubit Hessian batch
    // together with the forward default: 114 ms against 175 ms)
    if (n >= 20 && sizeof(R) == 4) {
        k = std::min(12, n - 1);
        M = 4;
        low = kLaneBits;
    }
}

// Persistent grid: two CTAs per SM, one when the two tiles of a CTA (psi and
// lambda, 2^k amplitudes each) take more than half of shared memory.
int adjoint_grid(int64_t ntiles, int nsm, int k, int amp) {
    const int per_sm = ((size_t)2 * amp << k) > 100 * 1024 ? 1 : 2;
    return (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)per_sm * nsm));
}

// ---------------------------------------------------------------------------
// observable pass
// ---------------------------------------------------------------------------
struct ObsArgs {
    TileGeom g;
    const OTerm *terms;
    int nt;
    const double *rw;
    int nobs;
    int lam_mode;     // 0: no lambda, 1: lambda = contributions, 2: lambda += contributions
    double *part;     // [term][row][cta] or null
    int batch;
    int *errflag;
    void *lam;        // lambda in global memory (results are stored from registers)
    uint64_t tbit[2]; // amplitude bit of each tile bit, one byte each (as AdjArgs::tbit)
};

// Amplitudes each thread owns in an observable pass (threads = 2^k / kObsJ).
constexpr int kObsJ = 8;

template <typename R>
constexpr int obs_max_threads() { return sizeof(R) == 4 ? 1024 : 512; }

// Every tile: psi (and, after the first pass, lambda) arrive by TMA; each
// thread reads its amplitudes and their partners from shared memory; once
// every read is done the next tile's copies are issued into the same
// buffers (overlapping the partial sums and the stores), and lambda leaves
// the registers by coalesced stores (consecutive threads hold consecutive
// amplitudes, and the low tile bits are the low amplitude bits).
template <typename R>
__global__ void __launch_bounds__(obs_max_threads<R>()) k_tile_obs(const __grid_constant__ CUtensorMap mp,
                                                   const __grid_constant__ CUtensorMap ml,
                                                   const __grid_constant__ ObsArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    if (!DQ_SMEM_ALIGNED(smem)) return;   // bounds-checking build: no copy into a misaligned buffer
    const unsigned long long wlim = wait_limit_ns(a.errflag);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int64_t dim = int64_t(1) << a.g.k;
    const size_t tbytes = sizeof(cx<R>) * (size_t)dim;
    const uint32_t load_bytes = (uint32_t)(a.lam_mode == 2 ? 2 * tbytes : tbytes);
    cx<R> *bufP = reinterpret_cast<cx<R> *>(smem);
    cx<R> *bufL = reinterpret_cast<cx<R> *>(smem + tbytes);
    AdjTileSlot *slot = reinterpret_cast<AdjTileSlot *>(smem + 2 * tbytes);
    uint64_t *bar = &slot->bar;
    OTerm *st = reinterpret_cast<OTerm *>(smem + 2 * tbytes + 64);
    double *acc = reinterpret_cast<double *>(st + a.nt);            // [nt]
    R *accw = reinterpret_cast<R *>(acc + a.nt);                     // [nw][nt]
    R *wzs = reinterpret_cast<R *>(((uintptr_t)(accw + nw * a.nt) + 15) & ~uintptr_t(15));   // [kObsJ][threads]
    const int64_t per = (a.g.ntiles + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * per;
    const int64_t t1 = min(a.g.ntiles, t0 + per);
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_async_smem();
        if (t0 < t1) {
            int c[5];
            uint64_t base;
            int64_t row;
            geom_coords(a.g, t0, c, base, row);
            mbar_expect_tx(bar, load_bytes);
            tma_load5(bufP, &mp, c, bar);
            if (a.lam_mode == 2) tma_load5(bufL, &ml, c, bar);
        }
    }
    for (int i = tid; i < a.nt; i += blockDim.x) {
        st[i] = a.terms[i];
        acc[i] = 0.0;
    }
    for (int i = tid; i < nw * a.nt; i += blockDim.x) accw[i] = R(0);
    __syncthreads();
    // scattered offset of this thread's amplitudes l_i = tid + i * blockDim:
    // the bits of tid and those of i * blockDim are disjoint
    auto scatter = [&](uint32_t l) {
        uint64_t r = l & ((1u << kLaneBits) - 1);
        for (int i = kLaneBits; i < a.g.k; ++i)
            if ((l >> i) & 1) r |= uint64_t(1) << ((a.tbit[i >> 3] >> (8 * (i & 7))) & 63);
        return r;
    };
    const uint64_t s_tid = scatter((uint32_t)tid);
    // l_i = tid + i * blockDim: i sits on the top three tile bits (blockDim = 2^k / 8)
    uint64_t s_hi[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const int i = a.g.k - 3 + b;
        s_hi[b] = uint64_t(1) << ((a.tbit[i >> 3] >> (8 * (i & 7))) & 63);
    }
    uint32_t phase = 0;
    int64_t cur_row = -1;
    bool failed = false;
    auto flush = [&](int64_t row) {
        if (a.part)
            for (int j = tid; j < a.nt; j += blockDim.x) {
                a.part[((int64_t)st[j].term * a.batch + row) * gridDim.x + blockIdx.x] = acc[j];
                acc[j] = 0.0;
            }
    };
    for (int64_t t = t0; t < t1; ++t) {
        int c[5];
        uint64_t base;
        int64_t row;
        geom_coords(a.g, t, c, base, row);
        if (row != cur_row) {
            if (cur_row >= 0) flush(cur_row);
            cur_row = row;
        }
        // this tile's copies were issued by the prologue or by the previous tile
        const bool ok = mbar_wait_bounded(bar, phase, wlim);
        phase ^= 1;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        // this thread's amplitudes l_i = tid + i * blockDim and their lambda
        cx<R> x[kObsJ], lv[kObsJ];
#pragma unroll
        for (int i = 0; i < kObsJ; ++i) {
            const int l = tid + i * (int)blockDim.x;
            x[i] = bufP[l];
            lv[i] = a.lam_mode == 2 ? bufL[l] : mk<R>(R(0), R(0));
        }
        const double *w = a.rw ? a.rw + row * a.nobs : nullptr;
        // Z strings: amplitude i of this thread sits at l = tid + i 2^lb
        // (lb = k - 3), so the sign of its probability under a term with mask
        // s is (-1)^(parity(tid & s) + parity(i & (s >> lb))) times that of the
        // tile base: a term's expectation is +-wz[s >> lb], wz the
        // Walsh-Hadamard transform of the thread's probabilities, kept in its
        // shared-memory column.
        const int lb = a.g.k - 3;
        {
            R *col = wzs + tid;
            const int ld = (int)blockDim.x;
#pragma unroll
            for (int i = 0; i < kObsJ; ++i) col[i * ld] = x[i].x * x[i].x + x[i].y * x[i].y;
#pragma unroll 1
            for (int st = 1; st < kObsJ; st <<= 1) {
                for (int i = 0; i < kObsJ; ++i) {
                    if (!(i & st)) {
                        const R a0 = col[i * ld], a1 = col[(i | st) * ld];
                        col[i * ld] = a0 + a1;
                        col[(i | st) * ld] = a0 - a1;
                    }
                }
            }
        }
        for (int j = 0; j < a.nt; ++j) {
            const OTerm o = st[j];
            const int bpar = __popcll(base & o.sout) & 1;
            const R wc = (R)((w ? w[o.obs] : 1.0) * o.coeff);
            R e = R(0);
            if (o.floc == 0) {
                const bool tneg = (__popc((uint32_t)tid & o.sloc) ^ bpar) & 1;
                const R v = wzs[((o.sloc >> lb) & (kObsJ - 1)) * blockDim.x + tid];
                e = tneg ? -v : v;
                // lambda[l] += wc (-1)^(parity(l & s) + bpar) psi[l]
#pragma unroll
                for (int i = 0; i < kObsJ; ++i) {
                    const bool neg = tneg ^ (__popc((uint32_t)i & (o.sloc >> lb)) & 1);
                    const R f = neg ? -wc : wc;
                    lv[i].x += f * x[i].x;
                    lv[i].y += f * x[i].y;
                }
            } else if (o.sloc == 0 && o.sout == 0 && o.nY == 0) {
                // X string: <x|X|x> terms Re(conj(y) x), lambda += wc y
#pragma unroll
                for (int i = 0; i < kObsJ; ++i) {
                    const int l = tid + i * (int)blockDim.x;
                    const uint32_t src = (uint32_t)l ^ o.floc;
                    const cx<R> y = DQ_INB(src, 1u << a.g.k) ? bufP[src] : mk<R>(R(0), R(0));
                    e += y.x * x[i].x + y.y * x[i].y;
                    lv[i].x += wc * y.x;
                    lv[i].y += wc * y.y;
                }
            } else {
#pragma unroll
                for (int i = 0; i < kObsJ; ++i) {
                    const int l = tid + i * (int)blockDim.x;
                    const uint32_t src = (uint32_t)l ^ o.floc;
                    const cx<R> y = DQ_INB(src, 1u << a.g.k) ? bufP[src] : mk<R>(R(0), R(0));
                    const int k4 = (o.nY + 2 * ((__popc((uint32_t)l & o.sloc) & 1) ^ bpar)) & 3;
                    const R re = re_conj_mul(y, x[i]), im = im_conj_mul(y, x[i]);
                    e += (k4 == 0) ? re : (k4 == 1 ? -im : (k4 == 2 ? -re : im));
                    const int k5 = (o.nY + 2 * ((__popc(src & o.sloc) & 1) ^ bpar)) & 3;
                    // lambda[l] += wc * i^k5 * y
                    const R yr = (k5 & 1) ? -y.y : y.x, yi = (k5 & 1) ? y.x : y.y;
                    const R sg = (k5 & 2) ? -wc : wc;
                    lv[i].x += sg * yr;
                    lv[i].y += sg * yi;
                }
            }
            e = warp_sum_t(e);
            if (lane == 0) accw[warp * a.nt + j] += e;
        }
        fence_async_smem();
        __syncthreads();   // every read of this tile's buffers is done; every warp's partials are in accw
        if (tid == 0 && t + 1 < t1) {
            int cn[5];
            uint64_t bn;
            int64_t rn;
            geom_coords(a.g, t + 1, cn, bn, rn);
            mbar_expect_tx(bar, load_bytes);
            tma_load5(bufP, &mp, cn, bar);
            if (a.lam_mode == 2) tma_load5(bufL, &ml, cn, bar);
        }
        for (int j = tid; j < a.nt; j += blockDim.x) {
            double sum = 0.0;
            for (int ww = 0; ww < nw; ++ww) {
                sum += (double)accw[ww * a.nt + j];
                accw[ww * a.nt + j] = R(0);
            }
            acc[j] += sum;
        }
        if (a.lam_mode) {
            const uint64_t t0 = ((uint64_t)row << a.g.n) | base | s_tid;
            cx<R> *gl = reinterpret_cast<cx<R> *>(a.lam) + t0;
            // the largest index has the three high bits set
            if (DQ_INB(t0 | s_hi[0] | s_hi[1] | s_hi[2], (uint64_t)a.batch << a.g.n)) {
#pragma unroll
                for (int i = 0; i < kObsJ; ++i) {
                    const uint64_t o = ((i & 1) ? s_hi[0] : 0) | ((i & 2) ? s_hi[1] : 0) | ((i & 4) ? s_hi[2] : 0);
                    gl[o] = lv[i];
                }
            }
        }
    }
    if (!failed && cur_row >= 0) {
        __syncthreads();
        flush(cur_row);
    }
    if (failed && tid == 0) {
        atomicCAS(a.errflag, 0, DEVERR_TIMEOUT);
        mbar_wait_bounded(bar, phase, wlim);
    }
}

template <typename R, int M>
__global__ void __launch_bounds__(adj_max_threads<R, M>(), adj_min_blocks<R, M>()) k_tile_adj(const __grid_constant__ CUtensorMap mp,
                                                                       const __grid_constant__ CUtensorMap ml,
                                                                       const __grid_constant__ AdjArgs a) {
    tile_adj_body<R, M, InterpRev>(mp, ml, a);
}

uint64_t obs_key(const std::vector<DevTerm> &bits, int n, int k, int low, int amp) {
    uint64_t h = 1469598103934665603ull ^ (uint64_t)(n * 131 + k * 7 + low + amp * 1000);
    for (const DevTerm &t : bits) {
        const unsigned char *b = (const unsigned char *)&t;
        for (size_t i = 0; i < sizeof(DevTerm); ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
    }
    return h;
}

}  // namespace

size_t tile_adjoint_part_bytes(const Plan &p, int batch, int nsm) {
    return (size_t)std::max(1, p.nslots) * (size_t)std::max(1, batch) * (size_t)(2 * nsm) * sizeof(double);
}

size_t tile_expect_part_bytes(int n, int nterms, int batch, int nsm) {
    (void)n;
    // [term][row][cta]: observable passes use up to 2 CTAs per SM, the forward
    // epilogue (diagonal observables) up to 4
    return (size_t)std::max(1, nterms) * (size_t)std::max(1, batch) * (size_t)(4 * nsm) * sizeof(double);
}

template <typename R>
cudaError_t tile_observe(TileCache &tc, int n, const std::vector<DevTerm> &bits, const DevTerm *d_bits,
                         const int32_t *d_ptr, int nobs, const double *rw, const void *psi, void *lam, int batch,
                         double *part, double *out, int nsm, cudaStream_t s, int64_t *launches) {
    constexpr int wb = AdjCfg<R>::wb;
    if (!ensure_encode_fn(tc)) return cudaErrorNotSupported;
    const size_t sbytes = ((size_t)batch << n) * sizeof(cx<R>);
    if (bits.empty()) {
        if (lam) {
            cudaError_t e = cudaMemsetAsync(lam, 0, sbytes, s);
            if (e != cudaSuccess) return e;
        }
        if (out) return cudaMemsetAsync(out, 0, sizeof(double) * (size_t)batch * nobs, s);
        return cudaSuccess;
    }
    int k, low, M;
    adjoint_tile<R>(n, k, low, M);
    low = kLaneBits;   // observable passes want as many free tile bits as possible
    const uint64_t key = obs_key(bits, n, k, low, (int)sizeof(cx<R>));
    ObsSchedule *os = nullptr;
    auto it = tc.obs.find(key);
    if (it != tc.obs.end()) {
        os = reinterpret_cast<ObsSchedule *>(it->second);
    } else {
        ObsSchedule *ns = new ObsSchedule();
        if (!build_obs_schedule(bits, n, k, low, wb, *ns)) {
            delete ns;
            return cudaErrorNotSupported;
        }
        if (cudaMalloc((void **)&ns->d_terms, sizeof(OTerm) * ns->terms.size()) != cudaSuccess) {
            cudaGetLastError();
            delete ns;
            return cudaErrorMemoryAllocation;
        }
        cudaMemcpy(ns->d_terms, ns->terms.data(), sizeof(OTerm) * ns->terms.size(), cudaMemcpyHostToDevice);
        os = ns;
        tc.obs[key] = ns;   // owned by the cache, released by tile_release_obs
    }
    const int64_t ntiles = (int64_t)batch << (n - k);
    const int grid = adjoint_grid(ntiles, nsm, k, (int)sizeof(cx<R>));
    if (k < 8 || (1 << k) / kObsJ > obs_max_threads<R>()) return cudaErrorNotSupported;
    const int threads = (1 << k) / kObsJ;
    const int nw = threads / 32;
    if (out) {
        cudaError_t e = cudaMemsetAsync(part, 0, sizeof(double) * bits.size() * (size_t)batch * grid, s);
        if (e != cudaSuccess) return e;
    }
    for (size_t pi = 0; pi < os->passes.size(); ++pi) {
        const OPass &ps = os->passes[pi];
        TileDims d;
        if (!make_dims(ps.T, n, wb, d)) return cudaErrorInvalidValue;
        CUtensorMap mp, ml;
        if (!encode_map(tc.encode_fn, &mp, d, const_cast<void *>(psi), batch, wb)) return cudaErrorInvalidValue;
        if (lam && !encode_map(tc.encode_fn, &ml, d, lam, batch, wb)) return cudaErrorInvalidValue;
        if (!lam) ml = mp;
        ObsArgs a;
        a.g = make_geom(d, n, k, wb, batch);
        a.terms = os->d_terms + ps.t0;
        a.nt = ps.nt;
        a.rw = rw;
        a.nobs = nobs;
        a.lam_mode = lam ? (pi == 0 ? 1 : 2) : 0;
        a.part = out ? part : nullptr;
        a.batch = batch;
        a.errflag = tc.errflag;
        a.lam = lam;
        // lambda leaves the registers as 32 consecutive amplitudes per warp
        // store: the lane bits must be the lowest amplitude bits
        if ((int)ps.T.size() != k || k > 16) return cudaErrorInvalidValue;
        a.tbit[0] = a.tbit[1] = 0;
        for (int i = 0; i < k; ++i) {
            if (i < kLaneBits && ps.T[i] != i) return cudaErrorInvalidValue;
            a.tbit[i >> 3] |= (uint64_t)ps.T[i] << (8 * (i & 7));
        }
        const size_t smem = 2 * (sizeof(cx<R>) << k) + 64 + ps.nt * sizeof(OTerm) + ps.nt * sizeof(double) +
                            (size_t)nw * ps.nt * sizeof(R) + 16 + (size_t)kObsJ * threads * sizeof(R) + 64;
        const void *ofn = (const void *)k_tile_obs<R>;
        if (tc.smem_set[ofn] < smem) {
            cudaError_t e = cudaFuncSetAttribute(ofn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            tc.smem_set[ofn] = smem;
        }
        LaunchScope ls(s, "k_tile_obs", launches);
        k_tile_obs<R><<<grid, threads, smem, s>>>(mp, ml, a);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (out) return expect_finalize_nblk(part, d_bits, d_ptr, nobs, batch, grid, out, s, launches);
    return cudaSuccess;
}

template <typename R>
cudaError_t tile_adjoint(TileCache &tc, std::unordered_map<uint64_t, TileTune> &tuned, const Plan &p,
                         const void *coef, void *psi, void *lam, int batch, double *part, double *gp, double *gd,
                         int nsm, cudaStream_t s, int64_t *launches) {
    constexpr int wb = AdjCfg<R>::wb;
    if (!ensure_encode_fn(tc)) return cudaErrorNotSupported;
    int k, low, M;
    adjoint_tile<R>(p.n, k, low, M);
    // the sweep stops at the first gate whose gradient is requested: schedule
    // only the gates from there on
    const int g0 = p.first_grad_gate(gp != nullptr, gd != nullptr);
    TileSchedule *sc = get_schedule(tc, p, k, low, M, (int)sizeof(cx<R>), true, g0);
    if (!sc) return cudaErrorNotSupported;
    const int64_t ntiles = (int64_t)batch << (p.n - k);
    const int grid = adjoint_grid(ntiles, nsm, k, (int)sizeof(cx<R>));
    const int threads = 1 << (k - M);
    const int nw = threads / 32;
    cudaError_t e = cudaMemsetAsync(part, 0, sizeof(double) * (size_t)std::max(1, p.nslots) * batch * grid, s);
    if (e != cudaSuccess) return e;
    // passes below the first one holding a requested gradient are never
    // un-applied (passes are in application order)
    int pstop = (int)sc->passes.size();
    for (int pi = 0; pi < (int)sc->passes.size() && pstop == (int)sc->passes.size(); ++pi)
        for (int j = 0; j < sc->passes[pi].nslot; ++j)
            if (p.slot_needed(sc->slots[sc->passes[pi].slot0 + j], gp != nullptr, gd != nullptr)) {
                pstop = pi;
                break;
            }
    if (sc->adj_p != psi || sc->adj_l != lam || sc->adj_batch != batch ||
        sc->adj_psi.size() != sc->passes.size()) {
        // encode every pass once for these buffers
        sc->adj_psi.assign(sc->passes.size(), CUtensorMap{});
        sc->adj_lam.assign(sc->passes.size(), CUtensorMap{});
        sc->adj_p = nullptr;
        for (size_t pi = 0; pi < sc->passes.size(); ++pi) {
            TileDims d;
            if (!make_dims(sc->passes[pi].T, p.n, wb, d)) return cudaErrorInvalidValue;
            if (!encode_map(tc.encode_fn, &sc->adj_psi[pi], d, psi, batch, wb) ||
                !encode_map(tc.encode_fn, &sc->adj_lam[pi], d, lam, batch, wb))
                return cudaErrorInvalidValue;
        }
        sc->adj_p = psi;
        sc->adj_l = lam;
        sc->adj_batch = batch;
    }
    const bool jit = jit_want(tc, tuned, p, (int)sizeof(cx<R>), *sc);
    const void *ikfn = M == 3 ? (const void *)k_tile_adj<R, 3>
                              : (M == 2 ? (const void *)k_tile_adj<R, 2> : (const void *)k_tile_adj<R, 4>);
    for (int pi = (int)sc->passes.size() - 1; pi >= pstop; --pi) {
        const void *kfn = jit ? (const void *)sc->jit->kernels[pi] : ikfn;
        const TPass &ps = sc->passes[pi];
        TileDims d;
        if (!make_dims(ps.T, p.n, wb, d)) return cudaErrorInvalidValue;
        const CUtensorMap &mp = sc->adj_psi[pi], &ml = sc->adj_lam[pi];
        AdjArgs a;
        a.g = make_geom(d, p.n, k, wb, batch);
        a.ops = sc->d_rops + ps.op0;
        a.segs = sc->d_rsegs + ps.rseg0;
        a.op0 = ps.op0;
        a.nops = ps.nops;
        a.nseg = ps.nrseg;
        a.slots = sc->d_slots + ps.slot0;
        a.nslot = ps.nslot;
        a.coef = coef;
        a.part = part;
        a.batch = batch;
        a.errflag = tc.errflag;
        a.any_row = 0;
        for (int j = ps.op0; j < ps.op0 + ps.nops; ++j) a.any_row |= sc->rops[j].rowstep != 0;
        a.psi = psi;
        a.lam = lam;
        // results leave the registers as 32 consecutive amplitudes per warp
        // store: the lane bits must be the lowest amplitude bits
        if ((int)ps.T.size() != k || k > 16) return cudaErrorInvalidValue;
        a.tbit[0] = a.tbit[1] = 0;
        for (int i = 0; i < k; ++i) {
            if (i < kLaneBits && ps.T[i] != i) return cudaErrorInvalidValue;
            a.tbit[i >> 3] |= (uint64_t)ps.T[i] << (8 * (i & 7));
        }
        const size_t smem = 2 * (sizeof(cx<R>) << k) + 64 + (size_t)ps.nops * sizeof(EOp) +
                            (size_t)ps.nrseg * sizeof(ESeg) + (size_t)ps.nops * sizeof(Mat2<R>) +
                            (size_t)ps.nslot * sizeof(double) + (size_t)nw * ps.nslot * sizeof(R) + 64;
        size_t &opened = jit ? sc->jit->smem_set[pi] : tc.smem_set[kfn];
        if (opened < smem) {
            e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            opened = smem;
        }
        LaunchScope ls(s, jit ? "k_tile_adj_jit" : "k_tile_adj", launches);
        if (jit) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)grid);
            cfg.blockDim = dim3((unsigned)threads);
            cfg.dynamicSmemBytes = smem;
            cfg.stream = s;
            void *args[] = {(void *)&mp, (void *)&ml, (void *)&a};
            e = cudaLaunchKernelExC(&cfg, kfn, args);
        } else if (M == 3) {
            k_tile_adj<R, 3><<<grid, threads, smem, s>>>(mp, ml, a);
        } else if (M == 2) {
            k_tile_adj<R, 2><<<grid, threads, smem, s>>>(mp, ml, a);
        } else {
            k_tile_adj<R, 4><<<grid, threads, smem, s>>>(mp, ml, a);
        }
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return grad_reduce(p, part, batch, grid, gp, gd, s, launches);
}

#define DQ_INST(R)                                                                                               \
    template cudaError_t tile_observe<R>(TileCache &, int, const std::vector<DevTerm> &, const DevTerm *,        \
                                         const int32_t *, int, const double *, const void *, void *, int,        \
                                         double *, double *, int, cudaStream_t, int64_t *);                      \
    template cudaError_t tile_adjoint<R>(TileCache &, std::unordered_map<uint64_t, TileTune> &, const Plan &,    \
                                         const void *, void *, void *, int, double *, double *, double *, int,   \
                                         cudaStream_t, int64_t *);
DQ_INST(float)
DQ_INST(double)
#undef DQ_INST

void tile_release_obs(TileCache &tc) {
    for (auto &kv : tc.obs) {
        ObsSchedule *os = reinterpret_cast<ObsSchedule *>(kv.second);
        cudaFree(os->d_terms);
        delete os;
    }
    tc.obs.clear();
}

}  // namespace dq
