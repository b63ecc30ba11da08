// Tensor-core search over the template dictionary, exact with respect to the
// FP32 template search (act_shift.cu):
//  1. the residuals are laid out as shifted rows X[(b, j)][kk] =
//     bf16(r_b[m_lo + kk + tc_j]) (zero outside the window), so that
//     <r_b, u_{t, tc_j}> = sum_kk u_t(m_lo + kk) X[(b, j)][kk]: one GEMM of
//     the BF16 templates (N = 256 templates per tile) against the shifted
//     residual rows (M = 128 rows per tile), K = Kt lags;
//  2. the tcgen05 GEMM scales every accumulator by its atom's 1/|u| and keeps,
//     per row and template tile, the largest |score|;
//  3. a select kernel bounds the BF16 error per channel and flags the
//     (lag, tile) items that can hold the FP32 template search's argmax;
//  4. the flagged items are rescored with the FP32 template search's own
//     arithmetic (same FMA chain, same scale) and folded into the packed key;
//     a channel with too many items takes the FP32 template search instead.
// Steps 3 and 4 make the selection bit-identical to the FP32 template search.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <new>

#include "act_device.cuh"
#include "act_internal.cuh"
#include "act_tc.cuh"

namespace act {

namespace {

using namespace tc;

constexpr int kBM = 128;          // shifted residual rows per tile (MMA M)
constexpr int kBN = 256;          // templates per tile (MMA N)
constexpr int kUmmaK = 16;
constexpr int kThreads = 256;
constexpr int kAChunkBytes = kBM * kBK * 2;  // 16 KB
constexpr int kBChunkBytes = kBN * kBK * 2;  // 32 KB
constexpr int kStageBytes = kAChunkBytes + kBChunkBytes;
constexpr int kMaxStages = 4;
constexpr int kMaxItems = 64;      // flagged (lag, tile) items per channel before the FP32 template search
constexpr uint32_t kTmemCols = 2 * kBN;
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

struct Smem {
    uint64_t bar_full[kMaxStages];
    uint64_t bar_empty[kMaxStages];
    uint64_t bar_acc_full[2];
    uint64_t bar_acc_empty[2];
    uint32_t tmem_base;
    int abort;
};

// Shifted residual rows: one thread per element of X[rows][Kt]; rows past
// B * Ntc stay zero (set once at allocation).
__global__ void __launch_bounds__(256) k_shift_rows(const float *__restrict__ R, int Lp, int L, int B, int Ntc,
                                                    int S, int tc0, int m_lo, int Kt,
                                                    __nv_bfloat16 *__restrict__ X) {
    const int64_t total = (int64_t)B * Ntc * Kt;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / Kt;
        const int kk = (int)(i % Kt);
        const int b = (int)(row / Ntc), j = (int)(row % Ntc);
        const int64_t n = (int64_t)m_lo + kk + tc0 + (int64_t)S * j;
        const float v = (n >= 0 && n < L) ? R[(size_t)b * Lp + n] : 0.0f;
        X[i] = __float2bfloat16_rn(v);
    }
}

// GEMM work item w: row tile w / n_tiles, template tile w % n_tiles.  Every
// stage holds one template chunk (256 x 64) and the matching residual chunk
// (128 x 64).  Warp 0: TMA producer; warp 1: MMA issuer; warp 2: tensor
// memory owner; warps 4-7: epilogue (thread = residual row).
__global__ void __launch_bounds__(kThreads, 1)
    k_shift_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int m_tiles,
                 int n_tiles, int nkc, int stages, int rows_valid, int Ntc, int T_pad,
                 const float *__restrict__ scaleT, float *__restrict__ tile_max, int *status) {
    extern __shared__ uint8_t dyn_raw[];
    __shared__ Smem sm;
    const uint32_t base = (smem_u32(dyn_raw) + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t items = (int64_t)m_tiles * n_tiles;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&sm.bar_full[s], 1);
            mbar_init(&sm.bar_empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&sm.bar_acc_full[a], 1);
            mbar_init(&sm.bar_acc_empty[a], 128);
        }
        sm.abort = 0;
        fence_mbar_init();
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;
    volatile int *abort_flag = &sm.abort;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
        uint32_t it = 0;
        for (int64_t w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x) {
            const int mt = (int)(w / n_tiles), nt = (int)(w % n_tiles);
            for (int kc = 0; kc < nkc; ++kc, ++it) {
                const int s = (int)(it % (uint32_t)stages);
                const uint32_t ph = (it / (uint32_t)stages) & 1u;
                if (!mbar_wait(&sm.bar_empty[s], ph ^ 1u)) {
                    *abort_flag = 1;
                    break;
                }
                const uint32_t b0 = base + (uint32_t)s * kStageBytes;
                mbar_expect_tx(&sm.bar_full[s], (uint32_t)kStageBytes);
                // templates: the tile-major layout seen as [tiles * nkc * 256][64]
                tma_load_2d(b0, &tmB, 0, (int)(((int64_t)nt * nkc + kc) * kBN), &sm.bar_full[s]);
                tma_load_2d(b0 + kBChunkBytes, &tmA, kc * kBK, mt * kBM, &sm.bar_full[s]);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        tc_fence_after();
        uint32_t it = 0, local = 0;
        for (int64_t w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x, ++local) {
            const uint32_t acc = local & 1u, aph = (local >> 1) & 1u;
            if (!mbar_wait(&sm.bar_acc_empty[acc], aph ^ 1u)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint32_t d_tmem = tmem + acc * kBN;
            for (int kc = 0; kc < nkc; ++kc, ++it) {
                const int s = (int)(it % (uint32_t)stages);
                const uint32_t ph = (it / (uint32_t)stages) & 1u;
                if (!mbar_wait(&sm.bar_full[s], ph)) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t b0 = base + (uint32_t)s * kStageBytes;
                const uint32_t a0 = b0 + kBChunkBytes;
#pragma unroll
                for (int k = 0; k < kBK / kUmmaK; ++k)
                    tc_mma(d_tmem, smem_desc(a0 + k * kUmmaK * 2), smem_desc(b0 + k * kUmmaK * 2), kIdesc,
                           (kc | k) != 0 ? 1u : 0u);
                tc_commit(&sm.bar_empty[s]);
            }
            tc_commit(&sm.bar_acc_full[acc]);
        }
    } else if (warp >= 4) {
        // ---------------- epilogue: thread = shifted residual row ----------------
        const int q = warp - 4;
        uint32_t local = 0;
        for (int64_t w = blockIdx.x; w < items; w += gridDim.x, ++local) {
            const int mt = (int)(w / n_tiles), nt = (int)(w % n_tiles);
            const uint32_t acc = local & 1u, aph = (local >> 1) & 1u;
            if (*abort_flag || !mbar_wait(&sm.bar_acc_full[acc], aph)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const int row = mt * kBM + q * 32 + lane;
            const bool valid = row < rows_valid;
            const float4 *sc4 =
                reinterpret_cast<const float4 *>(scaleT + (size_t)(valid ? row % Ntc : 0) * T_pad + (size_t)nt * kBN);
            float m0 = 0.0f, m1 = 0.0f;
#pragma unroll 1
            for (int c = 0; c < kBN / 32; ++c) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + acc * kBN + c * 32, v);
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float4 s = valid ? __ldg(sc4 + c * 8 + e) : make_float4(0.f, 0.f, 0.f, 0.f);
                    m0 = fmaxf(m0, fabsf(v[4 * e] * s.x));
                    m1 = fmaxf(m1, fabsf(v[4 * e + 1] * s.y));
                    m0 = fmaxf(m0, fabsf(v[4 * e + 2] * s.z));
                    m1 = fmaxf(m1, fabsf(v[4 * e + 3] * s.w));
                }
            }
            tc_fence_before();
            mbar_arrive(&sm.bar_acc_empty[acc]);
            if (valid) tile_max[(size_t)row * n_tiles + nt] = fmaxf(m0, m1);
        }
    }

    __syncthreads();
    if (*abort_flag) {
        if (threadIdx.x == 0) atomicOr(status, kFlagTimeout);
        sleep_ns(200000);  // let in-flight copies and MMAs land before releasing memory
    }
    tc_fence_after();
    if (warp == 2) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
}

// Item selection for channel b (one block).  With s the exact score, f the
// FP32 template search's score and h the tensor-core score of an atom,
//   |f - s| <= eps_r = (L + 4) 2^-23 |r|
// (one FP32 chain of L products, the FP32 scale and the final product), and
//   |h - s| <= delta = (1 + 1e-5) [eps_u (|r| + |dr|) + |dr|
//                                  + Kt 2^-23 (1 + eps_u)(|r| + |dr|)]
// (eps_u = largest |bf16(u) - u| / |u| over the atoms' windows, dr =
// bf16(r) - r, the Kt term bounds FP32 accumulation in the tensor core, the
// factor the scale product).  As for the dense BF16 search, the FP32 argmax
// lies in an item whose largest |h| is >= hmax - 2 delta - 2 eps_r.
__global__ void __launch_bounds__(256) k_shift_select(int Ntc, int n_tiles, int Kt, const float *__restrict__ tile_max,
                                                      int Lp, int L, const float *__restrict__ R,
                                                      const unsigned int *__restrict__ eps_bits,
                                                      unsigned long long *__restrict__ keys, int *__restrict__ fb_list,
                                                      int *__restrict__ counters, int *__restrict__ items,
                                                      long long *__restrict__ stats) {
    __shared__ double sh_d[32];
    __shared__ float sh_f[32];
    __shared__ int n_sh, base_sh;
    __shared__ int list[kMaxItems];
    const int b = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (int)(blockDim.x >> 5);
    const float *r = R + (size_t)b * Lp;
    const float *tm = tile_max + (size_t)b * Ntc * n_tiles;
    const int n_entries = Ntc * n_tiles;

    double e = 0.0, de = 0.0;
    for (int n = threadIdx.x; n < L; n += blockDim.x) {
        const float x = r[n];
        const float d = __bfloat162float(__float2bfloat16_rn(x)) - x;
        e = fma((double)x, (double)x, e);
        de = fma((double)d, (double)d, de);
    }
    const double rn = sqrt(block_sum(e, sh_d));
    const double drn = sqrt(block_sum(de, sh_d));
    const double eps_u = (double)__uint_as_float(*eps_bits);
    const double rr = rn + drn;
    const double ulp = 1.1920928955078125e-07;  // 2^-23
    const double delta = (1.0 + 1e-5) * (eps_u * rr + drn + (double)Kt * ulp * (1.0 + eps_u) * rr);
    const double eps_r = (double)(L + 4) * ulp * rn;

    float m = 0.0f;
    for (int i = threadIdx.x; i < n_entries; i += blockDim.x) m = fmaxf(m, tm[i]);
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (lane == 0) sh_f[warp] = m;
    if (threadIdx.x == 0) n_sh = 0;
    __syncthreads();
    float hmax = sh_f[0];
    for (int w = 1; w < nwarps; ++w) hmax = fmaxf(hmax, sh_f[w]);
    const double thr = (double)hmax - 2.0 * delta - 2.0 * eps_r;

    for (int i = threadIdx.x; i < n_entries; i += blockDim.x) {
        if ((double)tm[i] >= thr) {
            const int pos = atomicAdd(&n_sh, 1);
            if (pos < kMaxItems) list[pos] = i;  // i = j * n_tiles + tile
        }
    }
    __syncthreads();
    const int n = n_sh;
    if (n > kMaxItems) {
        if (threadIdx.x == 0) {
            keys[b] = 0ull;
            fb_list[atomicAdd(&counters[0], 1)] = b;
            atomicAdd((unsigned long long *)&stats[1], 1ull);
        }
        return;
    }
    if (threadIdx.x == 0) {
        keys[b] = 0ull;
        base_sh = atomicAdd(&counters[1], n);
        atomicAdd((unsigned long long *)&stats[0], 1ull);
        atomicAdd((unsigned long long *)&stats[2], (unsigned long long)n);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        items[2 * (base_sh + i)] = b;
        items[2 * (base_sh + i) + 1] = list[i];
    }
}

// FP32 rescore of the flagged items, one block of 256 threads (one per
// template of the tile) per item: the FMA chain over phases a and polyphase
// steps p of the FP32 template search, in its order, then its scale.
__global__ void __launch_bounds__(256) k_shift_rescan(const float *__restrict__ tpl, const float *__restrict__ scale,
                                                      int S, int Sa, int P, int rows, int NtcP, int T, int n_tiles,
                                                      int Lp, int L, const float *__restrict__ R,
                                                      const int *__restrict__ items, const int *__restrict__ counters,
                                                      unsigned long long *__restrict__ keys) {
    extern __shared__ __align__(16) float rpoly[];  // [Sa][P]
    __shared__ unsigned long long red[8];
    const int n_items = counters[1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
        const int b = items[2 * w];
        const int e = items[2 * w + 1];
        const int j = e / n_tiles, tile = e % n_tiles;
        const float *r = R + (size_t)b * Lp;
        for (int i = threadIdx.x; i < Sa * P; i += blockDim.x) {
            const int a = i / P, p = i % P;
            const int n = a + S * p;
            rpoly[i] = n < L ? r[n] : 0.0f;
        }
        __syncthreads();
        const int t = tile * 256 + (int)threadIdx.x;
        unsigned long long key = 0ull;
        if (t < T) {
            const int tb = t >> 5, tl = t & 31;
            const float *base = tpl + (size_t)tb * Sa * rows * 32 + tl;
            float acc = 0.0f;
            for (int a = 0; a < Sa; ++a) {
                const float *col = base + ((size_t)a * rows + (NtcP - 1 - j)) * 32;
                const float *rp = rpoly + a * P;
#pragma unroll 8
                for (int p = 0; p < P; ++p) acc = fmaf(rp[p], col[(size_t)p * 32], acc);
            }
            const float s = acc * scale[((size_t)tb * NtcP + j) * 32 + tl];
            const float x = fabsf(s);
            if (x == x) key = pack_key(x, (uint32_t)j * (uint32_t)T + (uint32_t)t);
        }
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, key, off);
            key = o > key ? o : key;
        }
        if (lane == 0) red[warp] = key;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long m = 0ull;
            for (int i = 0; i < 8; ++i) m = red[i] > m ? red[i] : m;
            if (m) atomicMax(keys + b, m);
        }
        __syncthreads();
    }
}

constexpr int kStaticReserve = 512;
constexpr int kSmemBudget = 232448 - kStaticReserve - 1024;

}  // namespace

struct ShiftTc {
    CUtensorMap mapB;
    int nkc = 0, n_tiles = 0, stages = 0, sm_count = 0;
    size_t smem = 0;
    float *tile_max = nullptr;      // [rows_cap][n_tiles]
    int *items = nullptr;           // [B_cap * kMaxItems][2]
    __nv_bfloat16 *X = nullptr;     // [rows_cap rounded up to 128][Kt]
    int B_cap = 0;
    int rows_alloc = 0;
};

cudaError_t shift_tc_prepare(ShiftTc **out, const ShiftPlan &sp, int sm_count) {
    *out = nullptr;
    if (!sp.tpl16 || sp.Kt < kBK || sp.Kt % kBK != 0) return cudaErrorNotSupported;
    ShiftTc *s = new (std::nothrow) ShiftTc();
    if (!s) return cudaErrorMemoryAllocation;
    s->nkc = sp.Kt / kBK;
    s->n_tiles = sp.T_pad / kBN;
    s->sm_count = sm_count;
    const uint64_t rows = (uint64_t)s->n_tiles * s->nkc * kBN;
    if (rows >= ((uint64_t)1 << 31) || !make_map(&s->mapB, sp.tpl16, (uint64_t)kBK, rows, kBN)) {
        delete s;
        return cudaErrorNotSupported;
    }
    int st = kSmemBudget / kStageBytes;
    s->stages = st > kMaxStages ? kMaxStages : st;
    s->smem = 1024 + (size_t)s->stages * kStageBytes;
    cudaError_t e = allow_max_smem((const void *)k_shift_gemm, s->smem);
    if (e != cudaSuccess) {
        delete s;
        return e;
    }
    *out = s;
    return cudaSuccess;
}

void shift_tc_free(ShiftTc *s) {
    if (!s) return;
    if (s->tile_max) cudaFree(s->tile_max);
    if (s->items) cudaFree(s->items);
    if (s->X) cudaFree(s->X);
    delete s;
}

// Buffers for B channels (kept when large enough).
cudaError_t shift_tc_reserve(ShiftTc *s, const ShiftPlan &sp, int B) {
    if (B <= s->B_cap) return cudaSuccess;
    if (s->tile_max) cudaFree(s->tile_max);
    if (s->items) cudaFree(s->items);
    if (s->X) cudaFree(s->X);
    s->tile_max = nullptr;
    s->items = nullptr;
    s->X = nullptr;
    s->B_cap = 0;
    const int64_t rows = (int64_t)B * sp.Ntc;
    const int64_t rows_alloc = (rows + kBM - 1) / kBM * kBM;
    if (rows_alloc > (1ll << 30)) return cudaErrorInvalidValue;
    cudaError_t e = cudaMalloc(&s->tile_max, sizeof(float) * (size_t)rows * s->n_tiles);
    if (e == cudaSuccess) e = cudaMalloc(&s->items, sizeof(int) * 2 * (size_t)B * kMaxItems);
    if (e == cudaSuccess) e = cudaMalloc(&s->X, sizeof(__nv_bfloat16) * (size_t)rows_alloc * sp.Kt);
    if (e == cudaSuccess) e = cudaMemset(s->X, 0, sizeof(__nv_bfloat16) * (size_t)rows_alloc * sp.Kt);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cudaErrorMemoryAllocation;
    }
    s->B_cap = B;
    s->rows_alloc = (int)rows_alloc;
    return cudaSuccess;
}

cudaError_t launch_shift_tc_gemm(ShiftTc *s, const ShiftPlan &sp, const float *R, int Lp, int L, int B, int *status,
                                 cudaStream_t st) {
    if (!s || B < 1 || B > s->B_cap) return cudaErrorInvalidValue;
    const int64_t nx = (int64_t)B * sp.Ntc * sp.Kt;
    int64_t blocks = (nx + 255) / 256;
    if (blocks > (int64_t)s->sm_count * 8) blocks = (int64_t)s->sm_count * 8;
    k_shift_rows<<<(int)blocks, 256, 0, st>>>(R, Lp, L, B, sp.Ntc, sp.S, sp.tc0, sp.m_lo, sp.Kt, s->X);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int rows_valid = B * sp.Ntc;
    const int m_tiles = (rows_valid + kBM - 1) / kBM;
    CUtensorMap mapA;
    if (!make_map(&mapA, s->X, (uint64_t)sp.Kt, (uint64_t)m_tiles * kBM, kBM)) return cudaErrorInvalidValue;
    const int64_t items = (int64_t)m_tiles * s->n_tiles;
    const int grid = (int)(items < s->sm_count ? items : s->sm_count);
    k_shift_gemm<<<grid, kThreads, s->smem, st>>>(mapA, s->mapB, m_tiles, s->n_tiles, s->nkc, s->stages, rows_valid,
                                                  sp.Ntc, sp.T_pad, sp.scaleT, s->tile_max, status);
    return cudaGetLastError();
}

cudaError_t launch_shift_tc_resolve(ShiftTc *s, const ShiftPlan &sp, const float *R, int Lp, int L, int B,
                                    unsigned long long *keys, int *fb_list, int *counters, long long *stats,
                                    int *status, cudaStream_t st) {
    if (!s || B < 1 || B > s->B_cap) return cudaErrorInvalidValue;
    k_shift_select<<<B, 256, 0, st>>>(sp.Ntc, s->n_tiles, sp.Kt, s->tile_max, Lp, L, R, sp.eps_bits, keys, fb_list,
                                      counters, s->items, stats);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t rsmem = sizeof(float) * (size_t)sp.Sa * sp.P;
    if (rsmem > 48 * 1024) {
        e = cudaFuncSetAttribute(k_shift_rescan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem);
        if (e != cudaSuccess) return e;
    }
    k_shift_rescan<<<2 * s->sm_count, 256, rsmem, st>>>(sp.tpl, sp.scale, sp.S, sp.Sa, sp.P, sp.rows, sp.NtcP, sp.T,
                                                       s->n_tiles, Lp, L, R, s->items, counters, keys);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the FP32 template search for the channels with too many flagged items
    return launch_shift_search(sp, R, Lp, L, B, keys, nullptr, status, false, st, fb_list, counters);
}


}  // namespace act
