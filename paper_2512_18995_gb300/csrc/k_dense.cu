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
// with M = 128 (output floats l), K = 128 (input floats p) and N = 32 state
// rows per tile.  W and each S tile are split into TF32 parts x ~ hi + lo
// (hi the nearest TF32 value, lo the nearest TF32 value of the remainder, so
// |x - hi - lo| <= 2^-22 |x|) and D = W_hi S_hi + W_lo S_hi + W_hi S_lo is
// accumulated in FP32 in tensor memory: FP32-level accuracy from TF32
// tensor-core products (the three-pass TF32 scheme; the dropped W_lo S_lo
// term is below 2^-22 of each product).
//
// Pipeline per CTA (one per SM, persistent over tiles): TMA loads S tiles
// (128-byte swizzle, the tensor cores' canonical K-major layout) three tiles
// ahead; all threads split the landed tile into hi/lo in place; one thread
// issues 48 tcgen05.mma (16 K-steps x 3 products) into one of two TMEM
// accumulators and commits them to an mbarrier; while they run, the warps
// drain the previous tile's accumulator with tcgen05.ld and store it to
// global memory with coalesced 128-byte warp stores.  Every wait is bounded.
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
constexpr int DN = 32;                         // state rows per tile (MMA N)
constexpr int DSTAGE = 3;                      // S tiles in flight
constexpr int DTHREADS = 128;                  // 4 warps: one per TMEM lane quadrant
constexpr uint32_t W_BYTES = DKR * DKR * 4;    // 64 KB per TF32 part
constexpr uint32_t S_BYTES = DN * DKR * 4;     // 16 KB per TF32 part
constexpr uint32_t TMEM_COLS = 2 * DN;         // two FP32 accumulators of N columns
constexpr size_t DENSE_SMEM = 1024 + 2 * (size_t)W_BYTES + 2 * (size_t)DSTAGE * S_BYTES + 256;

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

// D (+)= A * B^T, A: M x K and B: N x K, both K-major in shared memory.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
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
// N = DN, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(DN >> 3) << 17) | ((128u >> 4) << 24);

// Nearest TF32 value of x (10 explicit mantissa bits; ties away from zero):
// exactly representable, so the tensor cores read it without further rounding.
__device__ __forceinline__ float tf32_round(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

struct DenseArgs {
    const uint4 *image;   // W hi then lo, already in the swizzled shared-memory layout
    float *state;         // complex64 amplitudes as interleaved floats
    int64_t rows;         // batch * 2^(n-6) rows of 128 floats
    int *errflag;
};

__global__ void __launch_bounds__(DTHREADS, 1) k_dense(const __grid_constant__ CUtensorMap tmap, DenseArgs a) {
    extern __shared__ unsigned char dsm_raw[];
    const uint32_t raw = smem_u32(dsm_raw);
    unsigned char *sm = dsm_raw + (((raw + 1023u) & ~1023u) - raw);   // 1024-byte aligned operand area
    unsigned char *w_hi = sm;
    unsigned char *w_lo = sm + W_BYTES;
    unsigned char *s_hi = sm + 2 * W_BYTES;              // DSTAGE tiles
    unsigned char *s_lo = s_hi + DSTAGE * S_BYTES;       // DSTAGE tiles
    uint64_t *full = reinterpret_cast<uint64_t *>(s_lo + DSTAGE * S_BYTES);
    uint64_t *mmab = full + DSTAGE;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mmab + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const int64_t ntiles = (a.rows + DN - 1) / DN;
    const int64_t T = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    // operand image of W (hi, lo): plain copy, the image is pre-swizzled
    {
        uint4 *dst = reinterpret_cast<uint4 *>(w_hi);
        for (int i = tid; i < (int)(2 * W_BYTES / 16); i += DTHREADS) dst[i] = a.image[i];
    }
    if (tid == 0) {
        for (int s = 0; s < DSTAGE; ++s) mbar_init(&full[s], 1);
        mbar_init(&mmab[0], 1);
        mbar_init(&mmab[1], 1);
    }
    if (warp == 0) {
        tmem_alloc(tslot, TMEM_COLS);
        tmem_relinquish();
    }
    fence_async_smem();   // W image and barrier inits visible to the async proxy
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    auto tile_row = [&](int64_t i) -> int64_t { return ((int64_t)blockIdx.x + i * (int64_t)gridDim.x) * DN; };
    auto issue_load = [&](int64_t i) {
        const int s = (int)(i % DSTAGE);
        const int y = (int)tile_row(i);
        mbar_expect_tx(&full[s], S_BYTES);
#pragma unroll
        for (int c = 0; c < DKR / 32; ++c) tma_load2(s_hi + s * S_BYTES + c * (DN * 128), &tmap, 32 * c, y, &full[s]);
    };
    int64_t issued = 0;
    if (tid == 0)
        for (; issued < DSTAGE && issued < T; ++issued) issue_load(issued);

    auto epilogue = [&](int64_t i) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((i & 1) * DN), v);
        const int64_t row0 = tile_row(i);
        float *out = a.state + row0 * DKR + warp * 32 + lane;
#pragma unroll
        for (int j = 0; j < DN; ++j)
            if (row0 + j < a.rows) out[(int64_t)j * DKR] = __uint_as_float(v[j]);
    };

    bool ok = true, failed = false;
    int64_t committed = -1;
    for (int64_t t = 0; t < T; ++t) {
        const int s = (int)(t % DSTAGE);
        ok = mbar_wait_bounded(&full[s], (uint32_t)((t / DSTAGE) & 1)) && ok;
        {
            float4 *hi = reinterpret_cast<float4 *>(s_hi + s * S_BYTES);
            float4 *lo = reinterpret_cast<float4 *>(s_lo + s * S_BYTES);
#pragma unroll 4
            for (int i = tid; i < (int)(S_BYTES / 16); i += DTHREADS) {
                const float4 x = hi[i];
                const float4 h = make_float4(tf32_round(x.x), tf32_round(x.y), tf32_round(x.z), tf32_round(x.w));
                hi[i] = h;
                lo[i] = make_float4(tf32_round(x.x - h.x), tf32_round(x.y - h.y), tf32_round(x.z - h.z),
                                    tf32_round(x.w - h.w));
            }
        }
        fence_async_smem();
        tc_fence_before();
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (tid == 0) {
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)((t & 1) * DN);
            const uint32_t wh = smem_u32(w_hi), wl = smem_u32(w_lo);
            const uint32_t sh = smem_u32(s_hi + s * S_BYTES), sl = smem_u32(s_lo + s * S_BYTES);
#pragma unroll
            for (int ks = 0; ks < DKR / 8; ++ks) {
                const uint32_t c = (uint32_t)(ks >> 2), o = (uint32_t)((ks & 3) * 32);
                const uint64_t ah = sdesc(wh + c * (128 * 128) + o), al = sdesc(wl + c * (128 * 128) + o);
                const uint64_t bh = sdesc(sh + c * (DN * 128) + o), bl = sdesc(sl + c * (DN * 128) + o);
                mma_tf32(d, ah, bh, kIdesc, ks > 0 ? 1u : 0u);
                mma_tf32(d, al, bh, kIdesc, 1u);
                mma_tf32(d, ah, bl, kIdesc, 1u);
            }
            mma_commit(&mmab[t & 1]);
        }
        committed = t;
        if (t >= 1) {
            ok = mbar_wait_bounded(&mmab[(t - 1) & 1], (uint32_t)(((t - 1) >> 1) & 1)) && ok;
            // tile t-1's operands are no longer read: refill its stage
            if (tid == 0 && ok && issued < T && issued == t - 1 + DSTAGE) issue_load(issued++);
            tc_fence_after();
            epilogue(t - 1);
            tc_fence_before();
        }
    }
    if (!failed && T > 0) {
        ok = mbar_wait_bounded(&mmab[(T - 1) & 1], (uint32_t)(((T - 1) >> 1) & 1)) && ok;
        tc_fence_after();
        epilogue(T - 1);
        tc_fence_before();
        if (__syncthreads_or(!ok)) failed = true;
    }
    if (failed && tid == 0) {
        atomicCAS(a.errflag, 0, DEVERR_TIMEOUT);
        // let loads and products still in flight land before the CTA exits (bounded)
        for (int64_t i = committed + 1; i < issued; ++i) mbar_wait_bounded(&full[i % DSTAGE], (uint32_t)((i / DSTAGE) & 1));
        if (committed >= 0) mbar_wait_bounded(&mmab[committed & 1], (uint32_t)((committed >> 1) & 1));
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// Real form of U embedded as I (x) U on 6 qubits, TF32 hi/lo split, written in
// the K-major 128-byte-swizzled layout: chunk c of 32 input floats, row l at
// 128 bytes, 16-byte piece j of the row at piece j ^ (l mod 8).
__global__ void k_dense_prepare(const double2 *__restrict__ U, int nw, uint32_t *__restrict__ img) {
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
    const float lo = tf32_round((float)(v - (double)h));
    const int c = p >> 5, q = p & 31;
    const uint32_t off = (uint32_t)(c * (128 * 32) + l * 32 + ((((q >> 2) ^ (l & 7)) << 2) | (q & 3)));
    img[off] = __float_as_uint(h);
    img[DKR * DKR + off] = __float_as_uint(lo);
}

}  // namespace

bool dense_supported(int n, int batch) {
    if (n < kDenseBits || batch < 1) return false;
    const int64_t rows = (int64_t)batch << (n - kDenseBits);
    return rows + DN < (int64_t(1) << 31);
}

cudaError_t dense_prepare(const void *unitary, int nw, void *image, cudaStream_t s, int64_t *launches) {
    if (nw < 1 || nw > kDenseBits) return cudaErrorInvalidValue;
    LaunchScope ls(s, "k_dense_prepare", launches);
    k_dense_prepare<<<DKR * DKR / 256, 256, 0, s>>>(reinterpret_cast<const double2 *>(unitary), nw,
                                                    reinterpret_cast<uint32_t *>(image));
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
    a.image = reinterpret_cast<const uint4 *>(image);
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
