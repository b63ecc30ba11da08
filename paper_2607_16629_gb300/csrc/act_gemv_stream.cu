// FP32 search of the projection P = D X^T (Sec. IV-A) with the selection
// fused, the dictionary streamed by the TMA bulk-copy engine: one persistent
// CTA per SM takes chunks of whole rows (chunk k of the dictionary goes to
// CTA k mod grid, so the CTAs read neighbouring chunks at any moment) and
// brings each into shared memory with one cp.async.bulk through a ring of
// stages; eight consumer warps score the rows of each chunk with the same
// per-row arithmetic as the GEMV (row_score order), so every score has the
// same bits; the selection (largest |score|, lowest row on ties) is the same
// key whatever the row order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "act_device.cuh"
#include "act_internal.cuh"

namespace act {

namespace {

constexpr int kConsumerWarps = 8;
constexpr int kStreamThreads = (kConsumerWarps + 1) * 32;  // + one producer warp
constexpr int kMaxStreamStages = 8;
// Stage ring: 128 KB per SM (4 stages of 32 KB at N = 512).  Measured on the
// 2,097,152 x 512 dictionary: 128-144 KB in flight per SM streams at
// 7.4-7.5 TB/s; 192 KB (6 x 32 KB) at 6.95 TB/s, 64 KB (2 x 32 KB) at
// 6.2 TB/s; 16 KB chunks lose to per-chunk overhead.
constexpr int kStreamSmem = 131072;

struct StreamShape {
    int rows_per_chunk;  // whole rows per stage, a multiple of the consumer warps
    int stages;
};

StreamShape stream_shape(int Lp) {
    const int row_bytes = Lp * 4;
    int rows = 32768 / row_bytes;
    if (rows < kConsumerWarps) rows = kConsumerWarps;
    rows = rows / kConsumerWarps * kConsumerWarps;
    int st = kStreamSmem / (rows * row_bytes);
    if (st > kMaxStreamStages) st = kMaxStreamStages;
    return {rows, st};
}

template <int NV>
__global__ void __launch_bounds__(kStreamThreads, 1)
    k_gemv_stream(const float *__restrict__ D, int64_t K, int Lp, const float *__restrict__ R, int B,
                  const int *__restrict__ chlist, const int *__restrict__ count_dev,
                  unsigned long long *__restrict__ keys, int rows_per_chunk, int stages, int *status,
                  unsigned long long wait_ns) {
    extern __shared__ __align__(128) float sm[];  // stages x rows_per_chunk x Lp
    __shared__ __align__(8) uint64_t full[kMaxStreamStages], empty[kMaxStreamStages];
    __shared__ float red_s[kConsumerWarps];
    __shared__ uint32_t red_i[kConsumerWarps];
    __shared__ int abort_sh;
    __shared__ unsigned long long issued_sh;  // bulk copies issued by the producer so far (all channels)
    // launched as a programmatic dependent of the kernel before it (the
    // residual update, or the queue that count_dev counts): every block waits
    // for it before reading the residuals, the count or the keys, then lets
    // the next kernel launch
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int count = count_dev ? *count_dev : B;
    // this CTA's chunks: k-th is chunk blockIdx.x + k gridDim.x of the dictionary
    const int64_t total_chunks = (K + rows_per_chunk - 1) / rows_per_chunk;
    const int64_t n_chunks =
        total_chunks > blockIdx.x ? (total_chunks - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const size_t stage_floats = (size_t)rows_per_chunk * Lp;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        abort_sh = 0;
        issued_sh = 0ull;
        fence_mbar_init();
    }
    __syncthreads();

    for (int c = 0; c < count; ++c) {
        const int ch = chlist ? chlist[c] : c;
        if (wid == kConsumerWarps) {
            // ---------------- producer ----------------
            if (lane == 0) {
                for (int64_t k = 0; k < n_chunks; ++k) {
                    const uint64_t it = (uint64_t)c * n_chunks + k;  // chunks issued over all channels
                    const int s = (int)(it % stages);
                    const uint32_t ph = (uint32_t)((it / stages) & 1);
                    if (!mbar_wait(&empty[s], ph ^ 1u, wait_ns)) {
                        abort_sh = 1;
                        break;
                    }
                    const int64_t row = (blockIdx.x + k * gridDim.x) * rows_per_chunk;
                    const int64_t nrows = K - row < rows_per_chunk ? K - row : rows_per_chunk;
                    const uint32_t bytes = (uint32_t)(nrows * Lp * 4);
                    mbar_expect_tx(&full[s], bytes);
                    bulk_g2s(sm + s * stage_floats, D + row * Lp, bytes, &full[s]);
                    *(volatile unsigned long long *)&issued_sh = it + 1;
                }
            }
        } else {
            // ---------------- consumers: warp w scores rows w, w + 8, ... of each chunk ----------------
            const float4 *r4 = reinterpret_cast<const float4 *>(R + (size_t)ch * Lp);
            float4 rv[NV];
#pragma unroll
            for (int j = 0; j < NV; ++j) rv[j] = r4[lane + 32 * j];
            float best = -1.0f;
            uint32_t bidx = 0u;
            for (int64_t k = 0; k < n_chunks; ++k) {
                const uint64_t it = (uint64_t)c * n_chunks + k;
                const int s = (int)(it % stages);
                const uint32_t ph = (uint32_t)((it / stages) & 1);
                const int ok = mbar_wait(&full[s], ph, wait_ns) ? 1 : 0;
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) abort_sh = 1;
                    break;
                }
                const int64_t row0 = (blockIdx.x + k * gridDim.x) * rows_per_chunk;
                const int nrows = (int)(K - row0 < rows_per_chunk ? K - row0 : rows_per_chunk);
                const float *st_base = sm + s * stage_floats;
                for (int rr = wid; rr < nrows; rr += kConsumerWarps) {
                    const float4 *a = reinterpret_cast<const float4 *>(st_base + (size_t)rr * Lp);
                    float x0 = 0.f, x1 = 0.f;
#pragma unroll
                    for (int j = 0; j < NV; ++j) {
                        const float4 v = a[lane + 32 * j];
                        x0 = fmaf(v.x, rv[j].x, x0);
                        x1 = fmaf(v.y, rv[j].y, x1);
                        x0 = fmaf(v.z, rv[j].z, x0);
                        x1 = fmaf(v.w, rv[j].w, x1);
                    }
                    float sc = x0 + x1;
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) sc += __shfl_xor_sync(0xffffffffu, sc, off);
                    const float x = fabsf(sc);
                    if (x > best) {  // rows of a warp ascend: the first of equal scores stays
                        best = x;
                        bidx = (uint32_t)(row0 + rr);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
            }
            if (lane == 0) {
                red_s[wid] = best;
                red_i[wid] = bidx;
            }
        }
        __syncthreads();
        if (abort_sh) {
            if (threadIdx.x == 0) {
                atomicOr(status, kFlagTimeout);
                // let every copy in flight land before the CTA exits: stage s
                // took issue numbers s, s + stages, ...; wait for the phase of
                // its last one (a completed phase returns at once)
                const unsigned long long n = issued_sh;
                for (int s = 0; s < stages; ++s)
                    if (n > (unsigned long long)s)
                        mbar_drain(&full[s], (uint32_t)(((n - 1 - s) / (unsigned long long)stages) & 1ull));
            }
            return;
        }
        if (threadIdx.x == 0) {
            float bs = -1.0f;
            uint32_t bi = 0u;
            for (int w = 0; w < kConsumerWarps; ++w)
                if (red_s[w] > bs || (red_s[w] == bs && red_i[w] < bi)) {
                    bs = red_s[w];
                    bi = red_i[w];
                }
            if (bs >= 0.0f) atomicMax(keys + ch, pack_key(bs, bi));
        }
        __syncthreads();
    }
}

template <int NV>
cudaError_t stream_instance(const float *D, int64_t K, int Lp, const float *R, int B, const int *chlist,
                            const int *count_dev, unsigned long long *keys, int *status, int sm_count,
                            cudaStream_t st, unsigned long long wait_ns, bool pdl) {
    const StreamShape sh = stream_shape(Lp);
    if (sh.stages < 2) return cudaErrorInvalidValue;
    const size_t smem = (size_t)sh.stages * sh.rows_per_chunk * Lp * sizeof(float);
    // set for the current device on every launch (a per-process flag would
    // miss the second GPU of a process); no allocation, legal in a capture
    cudaError_t e =
        cudaFuncSetAttribute(k_gemv_stream<NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStreamSmem);
    if (e != cudaSuccess) return e;
    return launch_kernel(k_gemv_stream<NV>, dim3(sm_count), dim3(kStreamThreads), smem, st, pdl, D, K, Lp, R, B,
                         chlist, count_dev, keys, sh.rows_per_chunk, sh.stages, status, wait_ns);
}

}  // namespace

cudaError_t launch_gemv_stream_argmax(const float *D, int64_t K, int Lp, const float *R, int B, const int *chlist,
                                      const int *count_dev, unsigned long long *keys, int *status, int sm_count,
                                      cudaStream_t st, unsigned long long wait_ns, bool pdl) {
    switch (Lp / 128) {
        case 1: return stream_instance<1>(D, K, Lp, R, B, chlist, count_dev, keys, status, sm_count, st, wait_ns, pdl);
        case 2: return stream_instance<2>(D, K, Lp, R, B, chlist, count_dev, keys, status, sm_count, st, wait_ns, pdl);
        case 3: return stream_instance<3>(D, K, Lp, R, B, chlist, count_dev, keys, status, sm_count, st, wait_ns, pdl);
        case 4: return stream_instance<4>(D, K, Lp, R, B, chlist, count_dev, keys, status, sm_count, st, wait_ns, pdl);
        case 8: return stream_instance<8>(D, K, Lp, R, B, chlist, count_dev, keys, status, sm_count, st, wait_ns, pdl);
        case 16: return stream_instance<16>(D, K, Lp, R, B, chlist, count_dev, keys, status, sm_count, st, wait_ns, pdl);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace act
