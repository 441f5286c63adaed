// Dense fused block on the 5th-generation tensor cores.
//
// A group of consecutive gates acting on the lowest-order qubits is one
// unitary U (Sec. "Quantum Computing with Qubits": the evolution U_n ... U_1
// |psi_0>, with a run of the U_j multiplied together).  On the 6 lowest-order
// qubits every row of the state is a matrix S with 2^(n-6) rows of 64
// amplitudes (128 interleaved floats), and the update is S <- S U^T: a dense
// contraction.  In real form
//
//     D[l][r] = sum_p W[l][p] S[r][p],   W[2i+a][2j+b] = [[Re, -Im], [Im, Re]]_ab (U_ij)
//
// with M = 128 (output floats l), K = 128 (input floats p) and N = 64 state
// rows per tile.  W and each S tile are split into TF32 parts x ~ hi + lo
// (hi the nearest TF32 value, lo the nearest TF32 value of the remainder,
// ties away from zero, so |x - hi - lo| <= 2^-22 |x|) and D = W_hi S_hi + W_lo S_hi + W_hi S_lo is
// accumulated in FP32 in tensor memory: FP32-level accuracy from TF32
// tensor-core products (the three-pass TF32 scheme; the dropped W_lo S_lo
// term is below 2^-22 of each product).
//
// Layout: W_hi and W_lo live in tensor memory for the whole kernel (lane l =
// row l, column p = element p), so each tcgen05.mma reads only its 2 KB S
// slice from shared memory; two FP32 accumulators of 64 columns follow them.
// Shared memory holds a ring of five TMA landing buffers (S tiles in the
// 128-byte-swizzled K-major layout, split to hi in place) and two buffers of
// lo parts.
//
// Pipeline per CTA (one per SM, persistent over tiles), warp-specialised: a
// TMA warp keeps the landing ring full, four splitter warps split each landed
// tile and later drain its accumulator with tcgen05.ld into coalesced
// 128-byte warp stores, and an MMA warp issues 48 tcgen05.mma per tile (16
// K-steps x 3 products) into one of two TMEM accumulators.  The roles meet
// only at mbarriers, so loads, splits, products and stores of neighbouring
// tiles overlap.  Every wait is bounded.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "dq_common.cuh"
#include "dq_dense.h"
#include "dq_plan.h"
#include "dq_tile.h"
#include "dq_tma.cuh"

namespace dq {
namespace {

constexpr int DKR = 128;                       // real dimension of the block (2 * 64)
constexpr int DN = 64;                         // state rows per tile (MMA N)
constexpr int DLAND = 5;                       // TMA landing buffers (S tiles in flight + 1)
constexpr int kSplitters = 128;                // warps 0-3: one per TMEM lane quadrant
constexpr int DTHREADS = kSplitters + 64;      // + one TMA warp + one MMA warp
constexpr uint32_t S_BYTES = DN * DKR * 4;     // 32 KB per tile and TF32 part
constexpr uint32_t TMEM_COLS = 512;            // W_hi | W_lo | two accumulators
constexpr uint32_t COL_WHI = 0, COL_WLO = DKR, COL_ACC = 2 * DKR;
constexpr size_t DENSE_SMEM = 1024 + (size_t)(DLAND + 2) * S_BYTES + 256;

// ---------------------------------------------------------------------------
// tcgen05 / TMA wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D (+)= A * B^T with A (M x K) in tensor memory (lane = row, one 32-bit
// column per element) and B (N x K) K-major in shared memory.
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// 32 consecutive 32-bit columns of this thread's TMEM lane from registers.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
        "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
        "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]),
        "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]),
        "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}

// Arrive once on `bar` when every tcgen05.mma issued so far by this thread
// has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tma_load2(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | (uint64_t(1) << 16) | (uint64_t(1024 >> 4) << 32) |
           (uint64_t(1) << 46) | (uint64_t(2) << 61);
}

// Instruction descriptor: FP32 accumulator, TF32 A and B, both K-major,
// N = DN, M = 128 (bits 4-5 accumulator type, 7-9 / 10-12 A / B type,
// 17-22 N >> 3, 24-28 M >> 4).
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(DN >> 3) << 17) | ((128u >> 4) << 24);

// Nearest TF32 value of x (10 explicit mantissa bits; ties away from zero):
// exactly representable, so the tensor cores read it without further rounding.
__device__ __forceinline__ float tf32_round(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

struct DenseArgs {
    const float4 *image;  // W hi then lo, row-major 128 x 128 each
    float *state;         // complex64 amplitudes as interleaved floats
    int64_t rows;         // batch * 2^(n-6) rows of 128 floats
    int *errflag;
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Warp roles: warps 0-3 split landed tiles and drain accumulators (warp w
// owns TMEM lanes 32w..32w+31), warp 4 issues the TMA loads, warp 5 issues
// the tensor-core products.  They meet only at mbarriers:
//   full[s]      TMA -> splitters        (landing buffer s holds tile t)
//   split[b]     splitters -> MMA warp   (tile t split into landing + lo[b], b = t & 1)
//   mmad[b]      MMA -> splitters        (accumulator b holds tile t)
//   accfree[b]   splitters -> MMA warp   (accumulator b drained)
//   landfree[s]  MMA -> TMA warp         (landing buffer s read by the products)
// A role that gives up on a wait (2 s) sets the error flag and leaves its
// loop; the others then give up on theirs, and one thread waits (bounded) for
// copies and products still in flight before TMEM is freed.
__global__ void __launch_bounds__(DTHREADS, 1) k_dense(const __grid_constant__ CUtensorMap tmap, DenseArgs a) {
    extern __shared__ unsigned char dsm_raw[];
    const unsigned long long wlim = wait_limit_ns(a.errflag);
    const uint32_t raw = smem_u32(dsm_raw);
    unsigned char *sm = dsm_raw + (((raw + 1023u) & ~1023u) - raw);   // 1024-byte aligned operand area
    unsigned char *land = sm;                                         // DLAND tiles (hi after the split)
    unsigned char *lob = sm + DLAND * S_BYTES;                        // 2 tiles of lo parts
    uint64_t *full = reinterpret_cast<uint64_t *>(lob + 2 * S_BYTES);
    uint64_t *landfree = full + DLAND;
    uint64_t *split = landfree + DLAND;
    uint64_t *mmad = split + 2;
    uint64_t *accfree = mmad + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(accfree + 2);
    int64_t *cnt = reinterpret_cast<int64_t *>(tslot + 2);   // [0] loads issued, [1] tiles split, [2] last commit
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const int64_t ntiles = (a.rows + DN - 1) / DN;
    const int64_t T = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (tid == 0) {
        for (int s = 0; s < DLAND; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&landfree[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&split[b], kSplitters);
            mbar_init(&mmad[b], 1);
            mbar_init(&accfree[b], kSplitters);
        }
        cnt[0] = 0;
        cnt[1] = 0;
        cnt[2] = -1;
    }
    if (warp == 0) {
        tmem_alloc(tslot, TMEM_COLS);
        tmem_relinquish();
    }
    fence_async_smem();   // barrier inits visible to the async proxy
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    auto tile_row = [&](int64_t i) -> int64_t { return ((int64_t)blockIdx.x + i * (int64_t)gridDim.x) * DN; };
    bool failed = false;

    if (warp < 4) {
        const uint32_t my_lanes = (uint32_t)(warp * 32) << 16;
        // W (hi, lo) into tensor memory: this thread writes row 32 warp + lane
        {
            const int l = warp * 32 + lane;
#pragma unroll 1
            for (int part = 0; part < 2; ++part) {
#pragma unroll 1
                for (int c = 0; c < DKR / 32; ++c) {
                    uint32_t v[32];
                    const float4 *src = a.image + ((size_t)part * DKR * DKR + (size_t)l * DKR + c * 32) / 4;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float4 x = src[q];
                        v[4 * q] = __float_as_uint(x.x);
                        v[4 * q + 1] = __float_as_uint(x.y);
                        v[4 * q + 2] = __float_as_uint(x.z);
                        v[4 * q + 3] = __float_as_uint(x.w);
                    }
                    tmem_st32(tmem + my_lanes + (part ? COL_WLO : COL_WHI) + (uint32_t)(c * 32), v);
                }
            }
            tmem_wait_st();
            tc_fence_before();
        }
        auto drain = [&](int64_t i) -> bool {
            const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&mmad[i & 1], (uint32_t)((i >> 1) & 1), wlim));
            tc_fence_after();
            const int64_t row0 = tile_row(i);
            float *out = a.state + row0 * DKR + warp * 32 + lane;
#pragma unroll
            for (int h = 0; h < DN / 32; ++h) {
                uint32_t v[32];
                tmem_ld32(tmem + my_lanes + COL_ACC + (uint32_t)((i & 1) * DN + h * 32), v);
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (row0 + h * 32 + j < a.rows) out[(int64_t)(h * 32 + j) * DKR] = __uint_as_float(v[j]);
            }
            tc_fence_before();
            mbar_arrive(&accfree[i & 1]);
            return ok;
        };
        int64_t t = 0;
        for (; t < T; ++t) {
            const int s = (int)(t % DLAND);
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[s], (uint32_t)((t / DLAND) & 1), wlim))) {
                failed = true;
                break;
            }
            // lo[t & 1] was last read by the products of tile t - 2, drained in
            // the previous iteration (program order)
            float4 *hi = reinterpret_cast<float4 *>(land + s * S_BYTES);
            float4 *lo = reinterpret_cast<float4 *>(lob + (t & 1) * S_BYTES);
#pragma unroll 4
            for (int i = tid; i < (int)(S_BYTES / 16); i += kSplitters) {
                const float4 x = hi[i];
                const float4 h = make_float4(tf32_round(x.x), tf32_round(x.y), tf32_round(x.z), tf32_round(x.w));
                hi[i] = h;
                lo[i] = make_float4(tf32_round(x.x - h.x), tf32_round(x.y - h.y), tf32_round(x.z - h.z),
                                    tf32_round(x.w - h.w));
            }
            fence_async_smem();
            mbar_arrive(&split[t & 1]);
            if (t >= 1 && !drain(t - 1)) {
                failed = true;
                break;
            }
        }
        if (!failed && T > 0 && !drain(T - 1)) failed = true;
        if (tid == 0) cnt[1] = t;
    } else if (warp == 4) {
        if (lane == 0) {
            int64_t i = 0;
            for (; i < T; ++i) {
                const int s = (int)(i % DLAND);
                if (i >= DLAND && !mbar_wait_bounded(&landfree[s], (uint32_t)(((i - DLAND) / DLAND) & 1), wlim)) {
                    failed = true;
                    break;
                }
                const int y = (int)tile_row(i);
                mbar_expect_tx(&full[s], S_BYTES);
#pragma unroll
                for (int c = 0; c < DKR / 32; ++c)
                    tma_load2(land + s * S_BYTES + c * (DN * 128), &tmap, 32 * c, y, &full[s]);
            }
            cnt[0] = i;
        }
    } else {
        if (lane == 0) {
            const uint64_t dland0 = sdesc(smem_u32(land)), dlo0 = sdesc(smem_u32(lob));
            for (int64_t t = 0; t < T; ++t) {
                if (!mbar_wait_bounded(&split[t & 1], (uint32_t)((t >> 1) & 1), wlim) ||
                    (t >= 2 && !mbar_wait_bounded(&accfree[t & 1], (uint32_t)(((t - 2) >> 1) & 1), wlim))) {
                    failed = true;
                    break;
                }
                tc_fence_after();
                const int s = (int)(t % DLAND);
                const uint32_t d = tmem + COL_ACC + (uint32_t)((t & 1) * DN);
                const uint64_t bh0 = dland0 + (uint64_t)((s * S_BYTES) >> 4);
                const uint64_t bl0 = dlo0 + (uint64_t)(((t & 1) * S_BYTES) >> 4);
#pragma unroll
                for (int ks = 0; ks < DKR / 8; ++ks) {
                    const uint64_t o = (uint64_t)((((ks >> 2) * (DN * 128)) + (ks & 3) * 32) >> 4);
                    const uint32_t ah = tmem + COL_WHI + (uint32_t)(ks * 8), al = tmem + COL_WLO + (uint32_t)(ks * 8);
                    mma_tf32_ts(d, ah, bh0 + o, kIdesc, ks > 0 ? 1u : 0u);
                    mma_tf32_ts(d, al, bh0 + o, kIdesc, 1u);
                    mma_tf32_ts(d, ah, bl0 + o, kIdesc, 1u);
                }
                mma_commit(&mmad[t & 1]);
                mma_commit(&landfree[s]);
                cnt[2] = t;
            }
        }
    }
    if (failed) atomicCAS(a.errflag, 0, DEVERR_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        // copies and products still in flight after a failure (bounded waits)
        for (int64_t i = cnt[1]; i < cnt[0]; ++i) mbar_wait_bounded(&full[i % DLAND], (uint32_t)((i / DLAND) & 1), wlim);
        const int64_t c = cnt[2];
        if (c >= 0) mbar_wait_bounded(&mmad[c & 1], (uint32_t)((c >> 1) & 1), wlim);
    }
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// Real form of U embedded as I (x) U on 6 qubits, split into TF32 hi and lo
// parts, row-major (row l = output float, column p = input float).
__global__ void k_dense_prepare(const double2 *__restrict__ U, int nw, float *__restrict__ img) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= DKR * DKR) return;
    const int l = idx >> 7, p = idx & 127;
    const int i = l >> 1, ri = l & 1, j = p >> 1, rj = p & 1;
    const int mask = (1 << nw) - 1;
    double v = 0.0;
    if ((i >> nw) == (j >> nw)) {
        const double2 u = U[(size_t)(i & mask) * (size_t)(1 << nw) + (size_t)(j & mask)];
        v = ri == 0 ? (rj == 0 ? u.x : -u.y) : (rj == 0 ? u.y : u.x);
    }
    const float h = tf32_round((float)v);
    img[idx] = h;
    img[DKR * DKR + idx] = tf32_round((float)(v - (double)h));
}

// The product U = G_m ... G_1 of a run of gates on bits 0..5 (row-major 64 x
// 64 complex128): block j forms column j by applying the run's gates, in
// order, to the basis vector e_j in FP64, each gate's 2x2 block read from the
// call's bound coefficient table (controlled blocks act where the control bit
// is 1, a SWAP exchanges its two bits).
template <typename R>
__global__ void __launch_bounds__(64) k_dense_compose(const DevGate *__restrict__ g, int ngates,
                                                      const Mat2<R> *__restrict__ coef, double2 *__restrict__ U) {
    __shared__ double2 v[64];
    const int j = blockIdx.x, i = threadIdx.x;
    v[i] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    __syncthreads();
    for (int k = 0; k < ngates; ++k) {
        const DevGate G = g[k];
        double2 r = v[i];
        if (G.cls == CLS_SWAP) {
            if (((i >> G.t) & 1) != ((i >> G.c) & 1)) r = v[i ^ ((1 << G.t) | (1 << G.c))];
        } else if (G.c < 0 || ((i >> G.c) & 1)) {
            const Mat2<R> m = coef[G.coef];
            const int tb = (i >> G.t) & 1;
            const double2 a0 = v[i & ~(1 << G.t)], a1 = v[i | (1 << G.t)];
            const double u0x = (double)m.m[2 * tb].x, u0y = (double)m.m[2 * tb].y;
            const double u1x = (double)m.m[2 * tb + 1].x, u1y = (double)m.m[2 * tb + 1].y;
            r.x = u0x * a0.x - u0y * a0.y + u1x * a1.x - u1y * a1.y;
            r.y = u0x * a0.y + u0y * a0.x + u1x * a1.y + u1y * a1.x;
        }
        __syncthreads();
        v[i] = r;
        __syncthreads();
    }
    U[(size_t)i * 64 + j] = v[i];
}

}  // namespace

template <typename R>
cudaError_t dense_compose(const DevGate *d_gates, int ngates, const void *coef, void *unitary, cudaStream_t s,
                          int64_t *launches) {
    LaunchScope ls(s, "k_dense_compose", launches);
    k_dense_compose<R><<<64, 64, 0, s>>>(d_gates, ngates, (const Mat2<R> *)coef, (double2 *)unitary);
    return cudaGetLastError();
}
template cudaError_t dense_compose<float>(const DevGate *, int, const void *, void *, cudaStream_t, int64_t *);
template cudaError_t dense_compose<double>(const DevGate *, int, const void *, void *, cudaStream_t, int64_t *);

bool dense_supported(int n, int batch) {
    if (n < kDenseBits || batch < 1) return false;
    const int64_t rows = (int64_t)batch << (n - kDenseBits);
    return rows + DN < (int64_t(1) << 31);
}

cudaError_t dense_prepare(const void *unitary, int nw, void *image, cudaStream_t s, int64_t *launches) {
    if (nw < 1 || nw > kDenseBits) return cudaErrorInvalidValue;
    LaunchScope ls(s, "k_dense_prepare", launches);
    k_dense_prepare<<<DKR * DKR / 256, 256, 0, s>>>(reinterpret_cast<const double2 *>(unitary), nw,
                                                    reinterpret_cast<float *>(image));
    return cudaGetLastError();
}

cudaError_t dense_apply(TileCache &tc, const void *image, void *state, int n, int batch, int nsm, cudaStream_t s,
                        int64_t *launches) {
    if (!dense_supported(n, batch)) return cudaErrorNotSupported;
    if (!ensure_encode_fn(tc)) return cudaErrorNotSupported;
    const int64_t rows = (int64_t)batch << (n - kDenseBits);
    CUtensorMap map;
    cuuint64_t dims[2] = {(cuuint64_t)DKR, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)DKR * 4};
    cuuint32_t box[2] = {32, (cuuint32_t)DN};
    cuuint32_t estr[2] = {1, 1};
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tc.encode_fn);
    if (encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, state, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_dense, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DENSE_SMEM);
    if (e != cudaSuccess) return e;
    DenseArgs a;
    a.image = reinterpret_cast<const float4 *>(image);
    a.state = reinterpret_cast<float *>(state);
    a.rows = rows;
    a.errflag = tc.errflag;
    const int64_t ntiles = (rows + DN - 1) / DN;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, nsm));
    LaunchScope ls(s, "k_dense", launches);
    k_dense<<<grid, DTHREADS, DENSE_SMEM, s>>>(map, a);
    return cudaGetLastError();
}

}  // namespace dq
