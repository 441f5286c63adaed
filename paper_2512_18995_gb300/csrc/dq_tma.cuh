// TMA (cp.async.bulk.tensor) and mbarrier helpers shared by the tile kernels
// (internal).
#pragma once

#ifndef __CUDACC_RTC__
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "dq_common.cuh"
#include "dq_tile.h"
#else
#include "dq_common.cuh"
// Run-time compiled kernels receive tensor maps by value; the layout is the
// driver's opaque 128-byte, 128-byte-aligned descriptor.
typedef struct alignas(128) CUtensorMap_st { unsigned long long opaque[16]; } CUtensorMap;
#endif

namespace dq {
namespace {

#ifndef __CUDACC_RTC__   // host-side descriptor encoding

// ---------------------------------------------------------------------------
// TMA descriptor for one pass
// ---------------------------------------------------------------------------
struct TileDims {
    int rank = 0;
    int rlen[5] = {0, 0, 0, 0, 0};   // log2 box side (word bits)
    int glen[5] = {0, 0, 0, 0, 0};   // gap bits after the run (tile-index bits of this dim)
    int s[5] = {0, 0, 0, 0, 0};      // first word bit of the dim
};

inline bool make_dims(const std::vector<int> &T, int n, int wb, TileDims &d) {
    std::vector<int> w;
    for (int i = 0; i < wb; ++i) w.push_back(i);
    for (int t : T) w.push_back(t + wb);
    const int W = n + wb;
    // runs split into chunks of at most 8 bits
    std::vector<std::pair<int, int>> runs;   // (start, len)
    size_t i = 0;
    while (i < w.size()) {
        size_t j = i;
        while (j + 1 < w.size() && w[j + 1] == w[j] + 1) ++j;
        int st = w[i], len = (int)(j - i + 1);
        while (len > 0) {
            const int l = std::min(8, len);
            runs.push_back({st, l});
            st += l;
            len -= l;
        }
        i = j + 1;
    }
    if (runs.empty() || runs.size() > 5 || runs[0].first != 0) return false;
    d.rank = (int)runs.size();
    for (int r = 0; r < d.rank; ++r) {
        d.s[r] = runs[r].first;
        d.rlen[r] = runs[r].second;
        const int next = (r + 1 < d.rank) ? runs[r + 1].first : W;
        d.glen[r] = next - runs[r].first - runs[r].second;
    }
    return true;
}

inline bool encode_map(void *fn, CUtensorMap *map, const TileDims &d, void *base, int64_t batch, int wb) {
    cuuint64_t dims[5];
    cuuint64_t strides[4];
    cuuint32_t box[5], estr[5] = {1, 1, 1, 1, 1};
    uint64_t stride = 8;   // bytes of one 8-byte word
    for (int r = 0; r < 5; ++r) {
        if (r < d.rank) {
            const int width = d.rlen[r] + d.glen[r];
            uint64_t size = uint64_t(1) << width;
            if (r == d.rank - 1) size *= (uint64_t)batch;
            dims[r] = size;
            box[r] = 1u << d.rlen[r];
            if (r > 0) strides[r - 1] = stride;
            stride <<= width;
        } else {
            dims[r] = 1;
            box[r] = 1;
            strides[r - 1] = stride;
        }
    }
    (void)wb;
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    CUresult res = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, base, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return res == CUDA_SUCCESS;
}

#endif  // __CUDACC_RTC__

// ---------------------------------------------------------------------------
// device helpers: mbarrier and TMA
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of the barrier for at most `limit_ns` of wall time
// (the context's wait limit, 2 s unless set otherwise).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  unsigned long long limit_ns = kDefaultWaitNs) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void tma_load5(void *dst, const CUtensorMap *map, const int c[5], uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]),
        "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_store5(const CUtensorMap *map, const int c[5], const void *src) {
    asm volatile(
        "cp.async.bulk.tensor.5d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(smem_u32(src))
        : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Programmatic dependent launch: wait until the preceding kernels of the
// stream have completed and their writes are visible (a no-op for launches
// without the attribute), and allow the next kernel to start its prologue.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }


// Tile index -> TMA coordinates, block base (amplitude bits outside the tile)
// and batch row.  Geometry of one pass.
struct TileGeom {
    int n, k, wb;
    int64_t ntiles;
    int rank;
    int rlen[5], glen[5], s[5];
};

#ifndef __CUDACC_RTC__
inline TileGeom make_geom(const TileDims &d, int n, int k, int wb, int64_t batch) {
    TileGeom g;
    g.n = n;
    g.k = k;
    g.wb = wb;
    g.ntiles = batch << (n - k);
    g.rank = d.rank;
    for (int r = 0; r < 5; ++r) {
        g.rlen[r] = d.rlen[r];
        g.glen[r] = d.glen[r];
        g.s[r] = d.s[r];
    }
    return g;
}

#endif  // __CUDACC_RTC__

__device__ __forceinline__ void geom_coords(const TileGeom &a, int64_t t, int c[5], uint64_t &base, int64_t &row) {
    uint64_t rem = (uint64_t)t;
    uint64_t word = 0;
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        c[r] = 0;
        if (r < a.rank) {
            uint64_t v;
            if (r < a.rank - 1) {
                v = rem & ((uint64_t(1) << a.glen[r]) - 1);
                rem >>= a.glen[r];
            } else {
                v = rem;
            }
            const uint64_t coord = v << a.rlen[r];
            c[r] = (int)coord;
            word |= coord << a.s[r];
        }
    }
    const uint64_t amp = word >> a.wb;
    row = (int64_t)(amp >> a.n);
    base = amp & ((uint64_t(1) << a.n) - 1);
}

#ifndef __CUDACC_RTC__
inline bool ensure_encode_fn(TileCache &tc) {
    if (tc.encode_fn) return true;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return false;
    }
    tc.encode_fn = fn;
    return true;
}

#endif  // __CUDACC_RTC__

}  // namespace
}  // namespace dq
