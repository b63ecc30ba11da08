// FP32 search of the projection P = D X^T (Sec. IV-A) with the selection
// i* = argmax_i |<g_i, r>| (Sec. III-A) fused: an HBM-bound GEMV over the
// stored FP32 dictionary.
#include <cuda_runtime.h>
#include <stdint.h>

#include "act_device.cuh"
#include "act_internal.cuh"

namespace act {

// ---------------------------------------------------------------------------
// FP32 GEMV over the stored dictionary with the selection fused.
// ---------------------------------------------------------------------------
// Each warp owns rows gw, gw + nw, gw + 2 nw, ... (nw = warps in the grid)
// and streams two rows at a time with 128-bit loads: lane l reads float4
// l + 32 j of a row, j = 0..NV-1.  The NB residuals of a channel group are
// brought into shared memory by the TMA bulk-copy engine and then held in
// registers.  A warp-shuffle reduction gives every lane the row's score;
// the warp keeps its best |score| (lowest row on ties, rows are visited in
// increasing order), the block combines its warps and issues one 64-bit
// atomicMax of the packed key per channel.
// With WRITE_SCORES the raw scores are stored instead (projection only).
template <int NV, int NB, bool WRITE_SCORES>
__global__ void __launch_bounds__(kGemvThreads) k_gemv(const float *__restrict__ D, int64_t K, int Lp,
                                                       const float *__restrict__ R, int B,
                                                       const int *__restrict__ chlist,
                                                       const int *__restrict__ count_dev,
                                                       unsigned long long *__restrict__ keys,
                                                       float *__restrict__ scores, int *status,
                                                       unsigned long long wait_ns) {
    extern __shared__ __align__(128) float smem_r[];  // NB * Lp floats
    __shared__ __align__(8) uint64_t bar;
    __shared__ float red_s[kGemvThreads / 32][NB];
    __shared__ uint32_t red_i[kGemvThreads / 32][NB];

    // launched as a programmatic dependent of the kernel before it (the
    // residual update, or the queue that count_dev counts): every block waits
    // for it before reading the residuals, the count or the keys, then lets
    // the next kernel launch
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int kWarps = kGemvThreads / 32;
    const int64_t gw = (int64_t)blockIdx.x * kWarps + wid;
    const int64_t nw = (int64_t)gridDim.x * kWarps;
    const int count = count_dev ? *count_dev : B;
    const int Lp4 = Lp >> 2;
    const float4 *D4 = reinterpret_cast<const float4 *>(D);

    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t parity = 0;

    for (int g0 = 0; g0 < count; g0 += NB) {
        const int ng = min(NB, count - g0);
        if (threadIdx.x == 0) {
            mbar_expect_tx(&bar, (uint32_t)(ng * Lp * 4));
            for (int c = 0; c < ng; ++c) {
                const int ch = chlist ? chlist[g0 + c] : g0 + c;
                bulk_g2s(smem_r + c * Lp, R + (int64_t)ch * Lp, (uint32_t)(Lp * 4), &bar);
            }
        }
        const int timed_out = mbar_wait(&bar, parity, wait_ns) ? 0 : 1;
        if (__syncthreads_or(timed_out)) {
            if (threadIdx.x == 0) {
                atomicOr(status, kFlagTimeout);
                mbar_drain(&bar, parity);  // bounded: let the in-flight copy land before exiting
            }
            return;
        }
        parity ^= 1u;

        float4 rv[NB][NV];
#pragma unroll
        for (int c = 0; c < NB; ++c)
#pragma unroll
            for (int j = 0; j < NV; ++j)
                rv[c][j] = c < ng ? reinterpret_cast<const float4 *>(smem_r + c * Lp)[lane + 32 * j]
                                  : make_float4(0.f, 0.f, 0.f, 0.f);

        float best[NB];
        uint32_t bidx[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) {
            best[c] = -1.0f;
            bidx[c] = 0u;
        }

        for (int64_t row = gw; row < K; row += 2 * nw) {
            const int64_t row2 = row + nw;
            const bool has2 = row2 < K;
            float4 a[NV], b[NV];
            const float4 *pa = D4 + row * Lp4 + lane;
#pragma unroll
            for (int j = 0; j < NV; ++j) a[j] = ldg_stream(pa + 32 * j);
            if (has2) {
                const float4 *pb = D4 + row2 * Lp4 + lane;
#pragma unroll
                for (int j = 0; j < NV; ++j) b[j] = ldg_stream(pb + 32 * j);
            } else {
#pragma unroll
                for (int j = 0; j < NV; ++j) b[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            float sa[NB], sb[NB];
#pragma unroll
            for (int c = 0; c < NB; ++c) {
                float x0 = 0.f, x1 = 0.f, y0 = 0.f, y1 = 0.f;
#pragma unroll
                for (int j = 0; j < NV; ++j) {
                    x0 = fmaf(a[j].x, rv[c][j].x, x0);
                    x1 = fmaf(a[j].y, rv[c][j].y, x1);
                    x0 = fmaf(a[j].z, rv[c][j].z, x0);
                    x1 = fmaf(a[j].w, rv[c][j].w, x1);
                    y0 = fmaf(b[j].x, rv[c][j].x, y0);
                    y1 = fmaf(b[j].y, rv[c][j].y, y1);
                    y0 = fmaf(b[j].z, rv[c][j].z, y0);
                    y1 = fmaf(b[j].w, rv[c][j].w, y1);
                }
                sa[c] = x0 + x1;
                sb[c] = y0 + y1;
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
                for (int c = 0; c < NB; ++c) {
                    sa[c] += __shfl_xor_sync(0xffffffffu, sa[c], off);
                    sb[c] += __shfl_xor_sync(0xffffffffu, sb[c], off);
                }
            }
#pragma unroll
            for (int c = 0; c < NB; ++c) {
                if (c < ng) {
                    if (WRITE_SCORES) {
                        if (lane == 0) {
                            const int ch = chlist ? chlist[g0 + c] : g0 + c;
                            scores[(int64_t)ch * K + row] = sa[c];
                            if (has2) scores[(int64_t)ch * K + row2] = sb[c];
                        }
                    } else {
                        float x = fabsf(sa[c]);
                        if (x > best[c]) {
                            best[c] = x;
                            bidx[c] = (uint32_t)row;
                        }
                        if (has2) {
                            x = fabsf(sb[c]);
                            if (x > best[c]) {
                                best[c] = x;
                                bidx[c] = (uint32_t)row2;
                            }
                        }
                    }
                }
            }
        }

        if (!WRITE_SCORES) {
            if (lane == 0) {
#pragma unroll
                for (int c = 0; c < NB; ++c) {
                    red_s[wid][c] = best[c];
                    red_i[wid][c] = bidx[c];
                }
            }
            __syncthreads();
            if (threadIdx.x < ng) {
                const int c = threadIdx.x;
                float bs = -1.0f;
                uint32_t bi = 0u;
                for (int w = 0; w < kWarps; ++w) {
                    const float s = red_s[w][c];
                    const uint32_t i = red_i[w][c];
                    if (s > bs || (s == bs && i < bi)) {
                        bs = s;
                        bi = i;
                    }
                }
                if (bs >= 0.0f) {
                    const int ch = chlist ? chlist[g0 + c] : g0 + c;
                    atomicMax(keys + ch, pack_key(bs, bi));
                }
            }
        }
        __syncthreads();  // shared residuals and reduction slots are reused by the next group
    }
}

template <int NV, int NB, bool WS>
static cudaError_t gemv_instance(const float *D, int64_t K, int Lp, const float *R, int B, const int *chlist,
                                 const int *count_dev, unsigned long long *keys, float *scores, int *status,
                                 int grid_ctas, unsigned long long wait_ns, cudaStream_t st, bool pdl) {
    const size_t smem = (size_t)NB * Lp * sizeof(float);
    return launch_kernel(k_gemv<NV, NB, WS>, dim3(grid_ctas), dim3(kGemvThreads), smem, st, pdl, D, K, Lp, R, B,
                         chlist, count_dev, keys, scores, status, wait_ns);
}

template <bool WS>
static cudaError_t gemv_dispatch(const float *D, int64_t K, int Lp, const float *R, int B, const int *chlist,
                                 const int *count_dev, unsigned long long *keys, float *scores, int *status,
                                 int grid_ctas, unsigned long long wait_ns, cudaStream_t st, bool pdl = false) {
    const int nv = Lp / 128;
    // Several channels per pass over D only when the count is known on the host.
    const bool multi = (count_dev == nullptr) && B >= 4 && nv <= 4;
#define ACT_GEMV_CASE(NVV)                                                                                 \
    case NVV:                                                                                              \
        return multi ? gemv_instance<NVV, 4, WS>(D, K, Lp, R, B, chlist, count_dev, keys, scores, status, \
                                                 grid_ctas, wait_ns, st, pdl)                              \
                     : gemv_instance<NVV, 1, WS>(D, K, Lp, R, B, chlist, count_dev, keys, scores, status, \
                                                 grid_ctas, wait_ns, st, pdl);
    switch (nv) {
        ACT_GEMV_CASE(1)
        ACT_GEMV_CASE(2)
        ACT_GEMV_CASE(3)
        ACT_GEMV_CASE(4)
        case 8:
            return gemv_instance<8, 1, WS>(D, K, Lp, R, B, chlist, count_dev, keys, scores, status, grid_ctas,
                                           wait_ns, st, pdl);
        case 16:
            return gemv_instance<16, 1, WS>(D, K, Lp, R, B, chlist, count_dev, keys, scores, status, grid_ctas,
                                            wait_ns, st, pdl);
        default:
            return cudaErrorInvalidValue;
    }
#undef ACT_GEMV_CASE
}

int gemv_ctas(int sm_count, int Lp) { return sm_count * gemv_max_ctas_per_sm(Lp); }

int gemv_max_ctas_per_sm(int Lp) {
    int per_sm = 0;
    const int nv = Lp / 128;
    cudaError_t e = cudaErrorInvalidValue;
    const size_t smem = (size_t)Lp * sizeof(float);
    switch (nv) {
        case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gemv<1, 1, false>, kGemvThreads, smem); break;
        case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gemv<2, 1, false>, kGemvThreads, smem); break;
        case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gemv<3, 1, false>, kGemvThreads, smem); break;
        case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gemv<4, 1, false>, kGemvThreads, smem); break;
        case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gemv<8, 1, false>, kGemvThreads, smem); break;
        case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gemv<16, 1, false>, kGemvThreads, smem); break;
        default: break;
    }
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    if (per_sm > 4) per_sm = 4;
    return per_sm;
}

cudaError_t launch_gemv_argmax(const float *D, int64_t K, int Lp, const float *R, int B, const int *chlist,
                               const int *count_dev, unsigned long long *keys, int *status, int grid_ctas,
                               cudaStream_t st, unsigned long long wait_ns, bool pdl) {
    return gemv_dispatch<false>(D, K, Lp, R, B, chlist, count_dev, keys, nullptr, status, grid_ctas, wait_ns, st,
                                pdl);
}

cudaError_t launch_project(const float *D, int64_t K, int Lp, const float *R, int B, float *scores, int *status,
                           int grid_ctas, cudaStream_t st, unsigned long long wait_ns) {
    return gemv_dispatch<true>(D, K, Lp, R, B, nullptr, nullptr, nullptr, scores, status, grid_ctas, wait_ns, st);
}

}  // namespace act
