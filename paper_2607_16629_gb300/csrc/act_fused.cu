// The whole greedy loop of Fig. 1 (search, selection, Eq. (4) update) over
// a stored FP32 dictionary in one cooperative launch.
//
// A one-channel decomposition over a dictionary that fits in L2 is bound by
// the latency of its P x 2 dependent launches, not by HBM; over a larger one
// by the stream of rows, which two passes of rows in flight per warp keep as
// busy as the per-order GEMV does.  Every CTA of a grid that is resident as
// a whole runs all P orders:
//  1. it scores its share of the rows against its own shared-memory copy of
//     each channel's residual (the FP32 GEMV's arithmetic: two FMA chains per
//     lane over float4 l + 32 j, a butterfly sum, the lowest row on ties) and
//     folds its best packed key into the order's key slot (atomicMax);
//  2. a bounded grid barrier;
//  3. every CTA reads the winning keys and applies the update of Eq. (4) to
//     its own residual copies with the update kernel's arithmetic (same block
//     size, same sums), so all copies stay bit-identical; CTA 0 alone writes
//     the atom, c_k and |r_{k+1}|^2.
// The kernel also forms r_0 = s and |s|^2 from the signals and writes the
// outputs where they are asked for, so a decomposition whose buffers are
// all in device memory is one memset and one launch.
// One barrier per order.  Key slots rotate over three buffers: CTA 0 clears
// slot (k + 2) mod 3 after barrier k, when every CTA has read it (order
// k - 1) and before any CTA can fold into it (order k + 2, after barrier
// k + 1).  The results equal those of the GEMV + update kernels bit for bit.
#include <cuda_runtime.h>
#include <stdint.h>

#include "act_device.cuh"
#include "act_ff.cuh"
#include "act_internal.cuh"
#include "act_update.cuh"

namespace act {

namespace {

constexpr int kFusedThreads = kUpdateThreads;  // the update's sums keep their order
constexpr int kFusedWarps = kFusedThreads / 32;

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_gpu(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_gpu(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Arrive at the grid barrier and wait until `target` arrivals (all CTAs,
// this order) have been counted, for at most limit_ns (0: one test).  A CTA
// that gives up raises the shared abort flag, which the others' waits see.
// Every thread of the block receives the outcome.
__device__ bool grid_barrier(unsigned int *arrived, int *abort, unsigned int target, unsigned long long limit_ns,
                             int *ok_sh) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();  // this block's key updates before its arrival
        atomicAdd(arrived, 1u);
        if (ld_acquire_gpu(arrived) < target) {
            const unsigned long long t0 = globaltimer_ns();
            while (ld_acquire_gpu(arrived) < target) {
                if (ld_relaxed_gpu(abort) || globaltimer_ns() - t0 >= limit_ns) {
                    ok = 0;
                    break;
                }
            }
        }
        if (!ok) atomicExch(abort, 1);
        __threadfence();
        *ok_sh = ok;
    }
    __syncthreads();
    return *ok_sh != 0;
}

// Rows a warp scores per pass (its loads are all issued before the first
// product), as many as keep the operands of two passes in registers.
template <int NV>
__host__ __device__ constexpr int fused_rows_per_pass() {
    return NV <= 2 ? 4 : (NV <= 4 ? 2 : 1);
}

// One pass: rows row + u nw (u < U, those below K) of the dictionary, lane
// l holding float4 l + 32 j of each.
template <int NV, int U>
__device__ __forceinline__ void fused_load_pass(const float4 *__restrict__ D4, int64_t K, int Lp4, int64_t row,
                                                int64_t nw, int lane, float4 (&a)[U][NV]) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t ru = row + u * nw;
        if (ru < K) {
            const float4 *pa = D4 + ru * Lp4 + lane;
#pragma unroll
            for (int j = 0; j < NV; ++j) a[u][j] = ldg_stream(pa + 32 * j);
        } else {
#pragma unroll
            for (int j = 0; j < NV; ++j) a[u][j] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

// Scores of one pass's rows in the FP32 GEMV's arithmetic (two FMA chains
// per lane, a butterfly sum), folded into the warp's best |score| with the
// lowest row winning a tie (rows arrive in increasing order).
template <int NV, int U>
__device__ __forceinline__ void fused_score_pass(const float4 (&a)[U][NV], const float4 (&rv)[NV], int64_t K,
                                                 int64_t row, int64_t nw, float &best, uint32_t &bidx) {
    float sc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        float x0 = 0.f, x1 = 0.f;
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            x0 = fmaf(a[u][j].x, rv[j].x, x0);
            x1 = fmaf(a[u][j].y, rv[j].y, x1);
            x0 = fmaf(a[u][j].z, rv[j].z, x0);
            x1 = fmaf(a[u][j].w, rv[j].w, x1);
        }
        sc[u] = x0 + x1;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int u = 0; u < U; ++u) sc[u] += __shfl_xor_sync(0xffffffffu, sc[u], off);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t ru = row + u * nw;
        const float x = fabsf(sc[u]);
        if (ru < K && x > best) {
            best = x;
            bidx = (uint32_t)ru;
        }
    }
}

// sig: the B signals, [B][L]; outputs (each may be null): atoms and coefs
// [B][P], energy [B][P + 1] (|s|^2 first), resid [B][resid_stride] (the
// first L samples of each row written).  sync: the barrier's count and
// abort flag, then the 3 x B key slots, all zero at launch.
template <int NV>
__global__ void __launch_bounds__(kFusedThreads) k_mp_fused(const float *__restrict__ D, int64_t K, int Lp, int L,
                                                            const float *__restrict__ sig, int B, int P, GridAxes ax,
                                                            unsigned long long *__restrict__ sync,
                                                            act_atom *__restrict__ atoms, float *__restrict__ coefs,
                                                            double *__restrict__ energy, float *__restrict__ resid,
                                                            int resid_stride, int *status,
                                                            unsigned long long wait_ns) {
    constexpr int U = fused_rows_per_pass<NV>();
    extern __shared__ __align__(16) float rs[];  // B x Lp residual copies
    __shared__ float red_s[kFusedWarps];
    __shared__ uint32_t red_i[kFusedWarps];
    __shared__ float shf[32];
    __shared__ double shd[32];
    __shared__ ff shp[32];
    __shared__ int ok_sh;
    unsigned int *arrived = reinterpret_cast<unsigned int *>(sync);
    int *abort = reinterpret_cast<int *>(sync) + 1;
    unsigned long long *fkeys = sync + 1;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * kFusedWarps + wid;
    const int64_t nw = (int64_t)gridDim.x * kFusedWarps;
    const float4 *D4 = reinterpret_cast<const float4 *>(D);
    const int Lp4 = Lp >> 2;

    // r_0 = s (Eq. (4)); CTA 0 also records |s|^2 in FP64 and flags a
    // non-finite sample, as the initialisation kernel does
    for (int b = 0; b < B; ++b) {
        double e = 0.0;
        int bad = 0;
        for (int n = threadIdx.x; n < Lp; n += blockDim.x) {
            const float v = n < L ? sig[(int64_t)b * L + n] : 0.0f;
            rs[(size_t)b * Lp + n] = v;
            if (!isfinite(v)) bad = 1;
            e = fma((double)v, (double)v, e);
        }
        if (blockIdx.x == 0) {
            const double tot = block_sum(e, shd);
            if (bad) atomicOr(status, kFlagNonFinite);
            if (threadIdx.x == 0 && energy) energy[(int64_t)b * (P + 1)] = tot;
        }
    }
    __syncthreads();

    for (int k = 0; k < P; ++k) {
        const int slot = k % 3;
        // 1. this CTA's rows against every channel; the best key per channel
        for (int b = 0; b < B; ++b) {
            const float4 *r4 = reinterpret_cast<const float4 *>(rs + (size_t)b * Lp);
            float4 rv[NV];
#pragma unroll
            for (int j = 0; j < NV; ++j) rv[j] = r4[lane + 32 * j];
            float best = -1.0f;
            uint32_t bidx = 0u;
            // two passes in flight: the next pass's rows load while this one's are scored
            float4 a[U][NV], c[U][NV];
            int64_t row = gw;
            fused_load_pass<NV, U>(D4, K, Lp4, row, nw, lane, a);
            while (row < K) {
                const int64_t row2 = row + U * nw;
                if (row2 < K) fused_load_pass<NV, U>(D4, K, Lp4, row2, nw, lane, c);
                fused_score_pass<NV, U>(a, rv, K, row, nw, best, bidx);
                if (row2 >= K) break;
                const int64_t row3 = row2 + U * nw;
                if (row3 < K) fused_load_pass<NV, U>(D4, K, Lp4, row3, nw, lane, a);
                fused_score_pass<NV, U>(c, rv, K, row2, nw, best, bidx);
                row = row3;
            }
            if (lane == 0) {
                red_s[wid] = best;
                red_i[wid] = bidx;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                float bs = -1.0f;
                uint32_t bi = 0u;
                for (int w = 0; w < kFusedWarps; ++w) {
                    const float s = red_s[w];
                    const uint32_t i = red_i[w];
                    if (s > bs || (s == bs && i < bi)) {
                        bs = s;
                        bi = i;
                    }
                }
                if (bs >= 0.0f) atomicMax(fkeys + (size_t)slot * B + b, pack_key(bs, bi));
            }
            __syncthreads();
        }

        // 2. every CTA's keys are in
        if (!grid_barrier(arrived, abort, (unsigned int)gridDim.x * (unsigned int)(k + 1), wait_ns, &ok_sh)) {
            if (threadIdx.x == 0) atomicOr(status, kFlagTimeout);
            return;
        }
        if (blockIdx.x == 0 && threadIdx.x < B) fkeys[(size_t)((k + 2) % 3) * B + threadIdx.x] = 0ull;

        // 3. the update of Eq. (4) on this CTA's residual copies
        for (int b = 0; b < B; ++b) {
            const unsigned long long key = ld_relaxed_gpu(fkeys + (size_t)slot * B + b);
            const uint32_t idx = key_index(key);
            const float *g = D + (int64_t)idx * Lp;
            float *r = rs + (size_t)b * Lp;
            float part = 0.0f;
            for (int n = threadIdx.x; n < L; n += blockDim.x) part = fmaf(g[n], r[n], part);
            const float c = block_sum(part, shf);
            if (blockIdx.x == 0) {
                ff e = {0.0f, 0.0f};
                for (int n = threadIdx.x; n < L; n += blockDim.x) {
                    const float v = fmaf(-c, g[n], r[n]);
                    r[n] = v;
                    ff_add_square(e, v);
                }
                const ff tot = block_sum_ff(e, shp);
                if (threadIdx.x < 32 && atoms) write_atom_lanes(ax, idx, atoms + (int64_t)b * P + k);
                if (threadIdx.x == 0) {
                    if (coefs) coefs[(int64_t)b * P + k] = c;
                    if (energy) energy[(int64_t)b * (P + 1) + k + 1] = ff_to_double(tot);
                }
            } else {
                for (int n = threadIdx.x; n < L; n += blockDim.x) r[n] = fmaf(-c, g[n], r[n]);
            }
            __syncthreads();
        }
    }
    if (blockIdx.x == 0 && resid)
        for (int b = 0; b < B; ++b)
            for (int n = threadIdx.x; n < L; n += blockDim.x) resid[(int64_t)b * resid_stride + n] = rs[(size_t)b * Lp + n];
}

template <int NV>
cudaError_t fused_occupancy(int B, int Lp, int *per_sm) {
    const size_t smem = (size_t)B * Lp * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_mp_fused<NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_mp_fused<NV>, kFusedThreads, smem);
}

template <int NV>
cudaError_t fused_instance(const float *D, int64_t K, int Lp, int L, const float *sig, int B, int P,
                           const GridAxes &ax, unsigned long long *sync, act_atom *atoms, float *coefs,
                           double *energy, float *resid, int resid_stride, int *status, int ctas,
                           unsigned long long wait_ns, cudaStream_t st) {
    const size_t smem = (size_t)B * Lp * sizeof(float);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(kFusedThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // the whole grid resident at once: its barrier can complete
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_mp_fused<NV>, D, K, Lp, L, sig, B, P, ax, sync, atoms, coefs, energy, resid,
                              resid_stride, status, wait_ns);
}

}  // namespace

int fused_max_ctas(int sm_count, int B, int Lp) {
    if (B < 1 || B > kFusedMaxB) return 0;
    int per_sm = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (Lp / 128) {
        case 1: e = fused_occupancy<1>(B, Lp, &per_sm); break;
        case 2: e = fused_occupancy<2>(B, Lp, &per_sm); break;
        case 3: e = fused_occupancy<3>(B, Lp, &per_sm); break;
        case 4: e = fused_occupancy<4>(B, Lp, &per_sm); break;
        case 8: e = fused_occupancy<8>(B, Lp, &per_sm); break;
        case 16: e = fused_occupancy<16>(B, Lp, &per_sm); break;
        default: break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * sm_count;
}

cudaError_t launch_mp_fused(const float *D, int64_t K, int Lp, int L, const float *sig, int B, int P,
                            const GridAxes &ax, unsigned long long *sync, act_atom *atoms, float *coefs,
                            double *energy, float *resid, int resid_stride, int *status, int ctas,
                            unsigned long long wait_ns, cudaStream_t st) {
    if (B < 1 || B > kFusedMaxB || P < 1 || ctas < 1 || K < 1 || K > 0xFFFFFFFFll || resid_stride < L)
        return cudaErrorInvalidValue;
    // the barrier's words and the three key slots start at zero
    cudaError_t e = cudaMemsetAsync(sync, 0, sizeof(unsigned long long) * (1 + 3 * (size_t)B), st);
    if (e != cudaSuccess) return e;
#define ACT_FUSED_CASE(NVV)                                                                                     \
    case NVV:                                                                                                   \
        return fused_instance<NVV>(D, K, Lp, L, sig, B, P, ax, sync, atoms, coefs, energy, resid, resid_stride, \
                                   status, ctas, wait_ns, st);
    switch (Lp / 128) {
        ACT_FUSED_CASE(1)
        ACT_FUSED_CASE(2)
        ACT_FUSED_CASE(3)
        ACT_FUSED_CASE(4)
        ACT_FUSED_CASE(8)
        ACT_FUSED_CASE(16)
        default:
            return cudaErrorInvalidValue;
    }
#undef ACT_FUSED_CASE
}

}  // namespace act
