// Tensor-core search of the batched projection P = D X^T (Sec. IV-A) for up
// to 128 channels: a persistent tcgen05 GEMM over the BF16 dictionary with
// the per-channel candidate selection fused into the epilogue, followed by a
// merge / FP32 rescore / certificate kernel and, for any channel whose
// candidate set cannot be shown to contain the FP32 argmax, the FP32 GEMV.
//
// GEMM shape per tile: M = 128 channels (rows of the residual matrix, padded
// with zero rows), N = 256 atoms, K = Lb samples.  The residual matrix (A,
// <= 128 KB of BF16) is loaded once per CTA by TMA and stays in shared
// memory; dictionary tiles (B, 256 atoms x 64 samples = 32 KB per stage) are
// streamed by TMA through a ring of stages; FP32 accumulators live in tensor
// memory (two 256-column buffers, so the epilogue of one tile overlaps the
// MMAs of the next).  Warp roles: warp 0 issues TMA, warp 1 issues MMAs,
// warp 2 owns the tensor-memory allocation, warps 4-7 read the accumulators
// (thread = channel) and keep, per channel, the KT largest |scores| seen by
// the CTA (ties to the lower atom index).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <new>

#include "act_device.cuh"
#include "act_internal.cuh"

namespace act {

namespace {

constexpr int kBM = 128;           // channels per tile (MMA M)
constexpr int kBN = 256;           // atoms per tile (MMA N)
constexpr int kBK = 64;            // samples per stage (one 128-byte swizzle row)
constexpr int kUmmaK = 16;         // K per tcgen05.mma (16-bit inputs)
constexpr int kCand = 8;           // candidates rescored per channel
constexpr int kTrack = kCand + 1;  // entries tracked per channel per CTA
constexpr int kGemmThreads = 256;
constexpr int kAChunkBytes = kBM * kBK * 2;  // 16 KB
constexpr int kStageBytes = kBN * kBK * 2;   // 32 KB
constexpr int kMaxDynSmem = 232448;
constexpr uint32_t kTmemCols = 512;          // 2 accumulators x 256 FP32 columns

// Instruction descriptor of tcgen05.mma.kind::f16: D = F32, A = B = BF16,
// both K-major, N = 256, M = 128.
constexpr uint32_t kIdesc = (1u << 4)                     // D format F32
                            | (1u << 7)                   // A format BF16
                            | (1u << 10)                  // B format BF16
                            | ((uint32_t)(kBN >> 3) << 17)  // N / 8
                            | ((uint32_t)(kBM >> 4) << 24); // M / 16

// Shared-memory matrix descriptor for a K-major operand written by TMA with
// 128-byte swizzling: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);   // start address
    d |= (uint64_t)1u << 16;                   // leading byte offset (unused with swizzle)
    d |= (uint64_t)(1024u >> 4) << 32;         // stride byte offset
    d |= (uint64_t)1u << 46;                   // descriptor version
    d |= (uint64_t)2u << 61;                   // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void tma_load_2d(uint32_t smem_dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 tensor-memory lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void sleep_ns(unsigned long long ns) {
    const unsigned long long t0 = globaltimer_ns();
    while (globaltimer_ns() - t0 < ns) {
    }
}

// Keeps vals[] sorted in decreasing order; a new entry equal to an existing
// one goes after it (entries arrive in increasing atom order).
__device__ __forceinline__ void topk_insert(float (&vals)[kTrack], uint32_t (&ids)[kTrack], float v, uint32_t id) {
#pragma unroll
    for (int q = 0; q < kTrack; ++q) {
        const bool gt = v > vals[q];
        const float tv = vals[q];
        const uint32_t ti = ids[q];
        vals[q] = gt ? v : tv;
        ids[q] = gt ? id : ti;
        v = gt ? tv : v;
        id = gt ? ti : id;
    }
}

struct GemmSmem {
    uint64_t bar_a;
    uint64_t bar_full[8];
    uint64_t bar_empty[8];
    uint64_t bar_acc_full[2];
    uint64_t bar_acc_empty[2];
    uint32_t tmem_base;
    int abort;
};

__global__ void __launch_bounds__(kGemmThreads, 1)
    k_gemm_topk(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t K, int nkc,
                int stages, float *__restrict__ part_val, uint32_t *__restrict__ part_idx, int *status) {
    extern __shared__ uint8_t dyn_raw[];
    __shared__ GemmSmem sm;
    const uint32_t dyn_base = (smem_u32(dyn_raw) + 1023u) & ~1023u;
    const uint32_t a_smem = dyn_base;
    const uint32_t b_smem = dyn_base + (uint32_t)nkc * kAChunkBytes;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = (K + kBN - 1) / kBN;

    if (threadIdx.x == 0) {
        mbar_init(&sm.bar_a, 1);
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
        mbar_expect_tx(&sm.bar_a, (uint32_t)(nkc * kAChunkBytes));
        for (int kc = 0; kc < nkc; ++kc) tma_load_2d(a_smem + kc * kAChunkBytes, &tmA, kc * kBK, 0, &sm.bar_a);
        uint32_t it = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
            for (int kc = 0; kc < nkc; ++kc, ++it) {
                const int s = (int)(it % (uint32_t)stages);
                const uint32_t ph = (it / (uint32_t)stages) & 1u;
                if (!mbar_wait(&sm.bar_empty[s], ph ^ 1u)) {
                    *abort_flag = 1;
                    break;
                }
                mbar_expect_tx(&sm.bar_full[s], kStageBytes);
                tma_load_2d(b_smem + s * kStageBytes, &tmB, kc * kBK, (int)(tile * kBN), &sm.bar_full[s]);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        if (!mbar_wait(&sm.bar_a, 0)) *abort_flag = 1;
        tc_fence_after();
        uint32_t it = 0, local = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x, ++local) {
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
                const uint32_t a0 = a_smem + kc * kAChunkBytes;
                const uint32_t b0 = b_smem + s * kStageBytes;
#pragma unroll
                for (int k = 0; k < kBK / kUmmaK; ++k)
                    tc_mma(d_tmem, smem_desc(a0 + k * kUmmaK * 2), smem_desc(b0 + k * kUmmaK * 2),
                           (kc | k) != 0 ? 1u : 0u);
                tc_commit(&sm.bar_empty[s]);
            }
            tc_commit(&sm.bar_acc_full[acc]);
        }
    } else if (warp >= 4) {
        // ---------------- epilogue: thread = channel ----------------
        const int q = warp - 4;
        const int ch = q * 32 + lane;
        float vals[kTrack];
        uint32_t ids[kTrack];
#pragma unroll
        for (int i = 0; i < kTrack; ++i) {
            vals[i] = -1.0f;
            ids[i] = 0xFFFFFFFFu;
        }
        uint32_t local = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++local) {
            const uint32_t acc = local & 1u, aph = (local >> 1) & 1u;
            if (*abort_flag || !mbar_wait(&sm.bar_acc_full[acc], aph)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const int64_t base = tile * kBN;
            const bool full_tile = base + kBN <= K;
#pragma unroll 1
            for (int c = 0; c < kBN / 32; ++c) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + acc * kBN + c * 32, v);
                const float thr0 = vals[kTrack - 1];
                bool any = false;
#pragma unroll
                for (int j = 0; j < 32; ++j) any |= fabsf(v[j]) > thr0;
                if (any) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int64_t atom = base + c * 32 + j;
                        const float s = fabsf(v[j]);
                        if (s > vals[kTrack - 1] && (full_tile || atom < K)) topk_insert(vals, ids, s, (uint32_t)atom);
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&sm.bar_acc_empty[acc]);
        }
        const size_t off = ((size_t)blockIdx.x * kBM + ch) * kTrack;
#pragma unroll
        for (int i = 0; i < kTrack; ++i) {
            part_val[off + i] = vals[i];
            part_idx[off + i] = ids[i];
        }
    }

    __syncthreads();
    if (*abort_flag) {
        if (threadIdx.x == 0) atomicOr(status, kFlagTimeout);
        sleep_ns(200000);  // let in-flight copies and MMAs land before releasing memory
    }
    tc_fence_after();
    if (warp == 2) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Merge of the per-CTA candidate lists, FP32 rescore and certificate.
// ---------------------------------------------------------------------------
// For channel b the GEMM left, per CTA c, its kTrack largest BF16 |scores|
// L_c (sorted).  The global top kTrack entries of the union all lie at or
// above T = max_c L_c[kTrack-1]; those entries are gathered, the first kCand
// become the candidates and the next one is U.  Every atom that is not a
// candidate has a BF16 |score| <= U.  With
//   delta = eps_g (|r| + |dr|) + (1 + 1e-5) |dr| + L 2^-23 (1 + eps_g)(|r| + |dr|)
// (eps_g = largest |bf16(g) - g| over the dictionary, dr = bf16(r) - r, the
// last term bounds FP32 accumulation in the tensor core), every
// non-candidate has an exact |<g, r>| <= U + delta.  The candidates are
// rescored in FP32 (error <= eps_r = L 2^-23 |r|); if the best rescored
// |score| - eps_r exceeds U + delta, the argmax of the exact scores is among
// the candidates and the best FP32 candidate is selected (near-ties within
// 1e-5 relative are settled by an FP64 rescore).  Otherwise the channel is
// queued for the FP32 full search.
constexpr int kGather = 1024;

__global__ void __launch_bounds__(256) k_rescore(int G, const float *__restrict__ part_val,
                                                 const uint32_t *__restrict__ part_idx, const float *__restrict__ D32,
                                                 int Lp, int L, const float *__restrict__ R,
                                                 const unsigned int *__restrict__ eps_bits,
                                                 unsigned long long *__restrict__ keys, int *__restrict__ fb_list,
                                                 int *__restrict__ fb_count, long long *__restrict__ stats) {
    __shared__ float g_val[kGather];
    __shared__ uint32_t g_idx[kGather];
    __shared__ int g_n;
    __shared__ float sh_f[32];
    __shared__ double sh_d[32];
    __shared__ uint32_t c_idx[kCand];
    __shared__ float c_fp[kCand];
    __shared__ int n_cand;
    __shared__ float U_sh;

    const int b = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float *r = R + (size_t)b * Lp;

    // |r|^2 and |bf16(r) - r|^2
    double e = 0.0, de = 0.0;
    for (int n = threadIdx.x; n < L; n += blockDim.x) {
        const float x = r[n];
        const float d = __bfloat162float(__float2bfloat16_rn(x)) - x;
        e = fma((double)x, (double)x, e);
        de = fma((double)d, (double)d, de);
    }
    const double rn = sqrt(block_sum(e, sh_d));
    const double drn = sqrt(block_sum(de, sh_d));

    // threshold T
    float t = -1.0f;
    for (int c = threadIdx.x; c < G; c += blockDim.x)
        t = fmaxf(t, part_val[((size_t)c * kBM + b) * kTrack + kTrack - 1]);
    for (int off = 16; off > 0; off >>= 1) t = fmaxf(t, __shfl_xor_sync(0xffffffffu, t, off));
    if (lane == 0) sh_f[warp] = t;
    if (threadIdx.x == 0) g_n = 0;
    __syncthreads();
    float T = sh_f[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) T = fmaxf(T, sh_f[w]);

    // gather every tracked entry >= T (each list is sorted, so a prefix)
    for (int c = threadIdx.x; c < G; c += blockDim.x) {
        const size_t base = ((size_t)c * kBM + b) * kTrack;
        for (int i = 0; i < kTrack; ++i) {
            const float v = part_val[base + i];
            if (v < T || v < 0.0f) break;
            const int pos = atomicAdd(&g_n, 1);
            if (pos < kGather) {
                g_val[pos] = v;
                g_idx[pos] = part_idx[base + i];
            }
        }
    }
    __syncthreads();
    const int n_all = g_n;
    const bool overflow = n_all > kGather;
    const int n = overflow ? kGather : n_all;

    // warp 0: the kCand + 1 best entries (|score| desc, index asc), in rounds
    if (warp == 0) {
        int taken = 0;
        float U = -1.0f;
        for (int round = 0; round <= kCand; ++round) {
            float bv = -2.0f;
            uint32_t bi = 0xFFFFFFFFu;
            int bp = -1;
            for (int i = lane; i < n; i += 32) {
                const float v = g_val[i];
                const uint32_t id = g_idx[i];
                if (v > bv || (v == bv && id < bi)) {
                    bv = v;
                    bi = id;
                    bp = i;
                }
            }
            for (int off = 16; off > 0; off >>= 1) {
                const float ov = __shfl_xor_sync(0xffffffffu, bv, off);
                const uint32_t oi = __shfl_xor_sync(0xffffffffu, bi, off);
                const int op = __shfl_xor_sync(0xffffffffu, bp, off);
                if (ov > bv || (ov == bv && oi < bi)) {
                    bv = ov;
                    bi = oi;
                    bp = op;
                }
            }
            if (bp < 0 || bv < 0.0f) break;
            if (round < kCand) {
                if (lane == 0) {
                    c_idx[taken] = bi;
                    g_val[bp] = -2.0f;
                }
                ++taken;
            } else {
                U = bv;
            }
            __syncwarp();
        }
        if (lane == 0) {
            n_cand = taken;
            U_sh = U;
        }
    }
    __syncthreads();
    const int nc = n_cand;

    // FP32 rescore, one warp per candidate
    for (int i = warp; i < nc; i += (int)(blockDim.x >> 5)) {
        const float *g = D32 + (size_t)c_idx[i] * Lp;
        float s = 0.0f;
        for (int k = lane; k < L; k += 32) s = fmaf(g[k], r[k], s);
        s = warp_sum(s);
        if (lane == 0) c_fp[i] = s;
    }
    __syncthreads();

    if (warp == 0) {
        // best and runner-up FP32 candidate
        int best = -1, second = -1;
        for (int i = 0; i < nc; ++i) {
            const float a = fabsf(c_fp[i]);
            if (best < 0 || a > fabsf(c_fp[best]) || (a == fabsf(c_fp[best]) && c_idx[i] < c_idx[best])) {
                second = best;
                best = i;
            } else if (second < 0 || a > fabsf(c_fp[second]) ||
                       (a == fabsf(c_fp[second]) && c_idx[i] < c_idx[second])) {
                second = i;
            }
        }
        // near-tie: settle among the candidates within 1e-5 of the best in FP64
        if (best >= 0 && second >= 0 && fabsf(c_fp[best]) - fabsf(c_fp[second]) <= 1e-5f * fabsf(c_fp[best])) {
            const float lim = fabsf(c_fp[best]) * (1.0f - 1e-5f);
            double bv = -1.0;
            int bsel = best;
            for (int i = 0; i < nc; ++i) {
                if (fabsf(c_fp[i]) < lim) continue;
                const float *g = D32 + (size_t)c_idx[i] * Lp;
                double s = 0.0;
                for (int k = lane; k < L; k += 32) s = fma((double)g[k], (double)r[k], s);
                s = fabs(warp_sum(s));
                if (s > bv || (s == bv && c_idx[i] < c_idx[bsel])) {
                    bv = s;
                    bsel = i;
                }
            }
            best = bsel;
        }
        if (lane == 0) {
            const double eps_g = (double)__uint_as_float(*eps_bits);
            const double rr = rn + drn;
            const double delta = eps_g * rr + (1.0 + 1e-5) * drn + (double)L * 1.1920928955078125e-07 * (1.0 + eps_g) * rr;
            const double eps_r = (double)L * 1.1920928955078125e-07 * rn;
            const double U = (double)U_sh;
            bool ok = !overflow && best >= 0;
            if (ok && U >= 0.0) ok = (double)fabsf(c_fp[best]) - eps_r > U + delta;
            if (ok) {
                keys[b] = pack_key(fabsf(c_fp[best]), c_idx[best]);
                atomicAdd((unsigned long long *)&stats[0], 1ull);
            } else {
                keys[b] = 0ull;
                const int pos = atomicAdd(fb_count, 1);
                fb_list[pos] = b;
                atomicAdd((unsigned long long *)&stats[1], 1ull);
            }
        }
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 2-D BF16 tensor map over a row-major [rows][cols] matrix, box [box_rows][64].
bool make_map(CUtensorMap *m, const void *base, uint64_t cols, uint64_t rows, uint32_t box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t gdim[2] = {cols, rows};
    cuuint64_t gstride[1] = {cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)kBK, box_rows};
    cuuint32_t estride[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), gdim, gstride, box, estride,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

struct Bf16Search {
    CUtensorMap mapB;
    int64_t K = 0;
    int Lb = 0;
    int nkc = 0;
    int stages = 0;
    int grid = 0;
    size_t smem = 0;
    float *part_val = nullptr;
    uint32_t *part_idx = nullptr;
    unsigned int *eps_bits = nullptr;  // owned by the caller (dictionary build)
};

cudaError_t bf16_search_prepare(Bf16Search **out, const __nv_bfloat16 *d16, int64_t K, int Lb, int sm_count,
                                unsigned int *eps_bits) {
    *out = nullptr;
    if (Lb % kBK != 0 || Lb > 512 || Lb < kBK) return cudaErrorNotSupported;
    Bf16Search *s = new (std::nothrow) Bf16Search();
    if (!s) return cudaErrorMemoryAllocation;
    s->K = K;
    s->Lb = Lb;
    s->nkc = Lb / kBK;
    const int avail = kMaxDynSmem - 1024 - s->nkc * kAChunkBytes;
    s->stages = avail / kStageBytes;
    if (s->stages > 6) s->stages = 6;
    if (s->stages < 2) {
        delete s;
        return cudaErrorNotSupported;
    }
    s->smem = 1024 + (size_t)s->nkc * kAChunkBytes + (size_t)s->stages * kStageBytes;
    const int64_t ntiles = (K + kBN - 1) / kBN;
    s->grid = (int)(ntiles < sm_count ? ntiles : sm_count);
    s->eps_bits = eps_bits;
    if (!make_map(&s->mapB, d16, (uint64_t)Lb, (uint64_t)K, kBN)) {
        delete s;
        return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaFuncSetAttribute(k_gemm_topk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem);
    if (e == cudaSuccess) e = cudaMalloc(&s->part_val, sizeof(float) * (size_t)s->grid * kBM * kTrack);
    if (e == cudaSuccess) e = cudaMalloc(&s->part_idx, sizeof(uint32_t) * (size_t)s->grid * kBM * kTrack);
    if (e != cudaSuccess) {
        bf16_search_free(s);
        return e;
    }
    *out = s;
    return cudaSuccess;
}

void bf16_search_free(Bf16Search *s) {
    if (!s) return;
    if (s->part_val) cudaFree(s->part_val);
    if (s->part_idx) cudaFree(s->part_idx);
    delete s;
}

cudaError_t launch_bf16_search(Bf16Search *s, int B, const __nv_bfloat16 *R16, const float *D32, int Lp, int L,
                               const float *R, unsigned long long *keys, int *fb_list, int *fb_count,
                               long long *stats, int *status, int gemv_grid, cudaStream_t st) {
    if (!s || B < 1 || B > kBM) return cudaErrorInvalidValue;
    CUtensorMap mapA;
    if (!make_map(&mapA, R16, (uint64_t)s->Lb, (uint64_t)kBM, kBM)) return cudaErrorInvalidValue;
    k_gemm_topk<<<s->grid, kGemmThreads, s->smem, st>>>(mapA, s->mapB, s->K, s->nkc, s->stages, s->part_val,
                                                        s->part_idx, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_rescore<<<B, 256, 0, st>>>(s->grid, s->part_val, s->part_idx, D32, Lp, L, R, s->eps_bits, keys, fb_list,
                                 fb_count, stats);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // FP32 full search for the channels the certificate did not cover
    return launch_gemv_argmax(D32, s->K, Lp, R, B, fb_list, fb_count, keys, status, gemv_grid, st);
}

}  // namespace act
