// Small device helpers: shared-memory addresses, mbarriers with bounded
// waits, 1-D bulk async copies, streaming loads and deterministic block sums.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace act {

// Default limit of a bounded wait (a grid can lower it, act_set_wait_limit);
// the drain waits that let copies already in flight land before a CTA exits
// always take this full limit.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Whether the phase with the given parity has completed, without waiting.
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity to complete, for at most
// limit_ns of wall time; limit 0 polls once without suspending (a copy or
// a consumer that is not already done makes it give up).  Returns false when
// it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned long long limit_ns) {
    if (limit_ns == 0) return mbar_test_wait(bar, parity);
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer_ns() - t0 >= limit_ns) return false;
    }
    return true;
}

// The wait of an exit path: lets a copy already issued land, with the full
// default limit whatever the grid's setting.
__device__ __forceinline__ bool mbar_drain(uint64_t *bar, uint32_t parity) {
    return mbar_wait(bar, parity, kWaitLimitNs);
}

// 1-D bulk copy global -> shared (TMA engine), completing on `bar`.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *smem_dst, const void *gsrc, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(smem_dst)),
        "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// 128-bit load that bypasses L1 (the dictionary is streamed once per order).
__device__ __forceinline__ float4 ldg_stream(const float4 *p) {
    float4 v;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p));
    return v;
}

// FP32 score of one dictionary row against a residual, both padded to
// nv * 128 floats: lane l takes float4 l + 32 j, accumulating x/z and y/w in
// two chains, then a butterfly sum.  The GEMV uses the same order, so every
// kernel gets the same bits for the same (atom, residual).
__device__ __forceinline__ float row_score(const float4 *__restrict__ row, const float4 *__restrict__ res, int nv,
                                           int lane) {
    float x0 = 0.f, x1 = 0.f;
    for (int j = 0; j < nv; ++j) {
        const float4 a = row[lane + 32 * j];
        const float4 r = res[lane + 32 * j];
        x0 = fmaf(a.x, r.x, x0);
        x1 = fmaf(a.y, r.y, x1);
        x0 = fmaf(a.z, r.z, x0);
        x1 = fmaf(a.w, r.w, x1);
    }
    float s = x0 + x1;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    return s;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Sum over the block in a fixed order (same result on every run).
// `sh` must hold 32 elements; every thread receives the total.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        T t = lane < nw ? sh[lane] : T(0);
        t = warp_sum(t);
        if (lane == 0) sh[0] = t;
    }
    __syncthreads();
    T r = sh[0];
    __syncthreads();
    return r;
}

}  // namespace act
