// Tensor-core search of the batched projection P = D X^T (Sec. IV-A), exact
// with respect to the FP32 search:
//  1. a persistent tcgen05 GEMM over the BF16 dictionary writes, per channel
//     and per tile of BN atoms, the largest BF16 |score| of the tile;
//  2. a select kernel bounds the BF16 error (delta) and flags, per channel,
//     every tile whose maximum lies within 2 delta + 2 eps_r of the channel's
//     largest BF16 |score| -- the FP32 argmax is provably in one of them;
//  3. the flagged tiles are scored in FP32 with the GEMV's own arithmetic
//     and folded into the packed selection key (a channel with too many
//     flagged tiles takes the FP32 full search instead).
//
// GEMM shape per tile: M = 128 channels (rows of the residual matrix, padded
// with zero rows), N = BN atoms (128 or 256, picked by the autotuner),
// K = Lb samples.  A work item is (dictionary tile, 128-channel row tile),
// row tiles fastest, so the CTAs working on one dictionary tile at a time
// read it from DRAM once and from L2 after that.  With one row tile and a
// window of up to 512 samples the residual matrix (A, <= 128 KB of BF16) is
// loaded once per CTA by TMA and stays in shared memory; otherwise its 16 KB
// chunks are streamed with the dictionary chunks (from L2: the whole residual
// matrix is B x Lb x 2 bytes).
// Dictionary chunks (B, BN atoms x 64 samples, contiguous in the tile-major
// BF16 layout) are streamed by TMA through a ring of stages; FP32
// accumulators live in tensor memory (two BN-column buffers, so the epilogue
// of one tile overlaps the MMAs of the next).  Warp roles: warp 0 issues
// TMA, warp 1 issues MMAs, warp 2 owns the tensor-memory allocation, warps
// 4-7 read the accumulators (thread = channel) and reduce each tile to its
// largest |score|.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <new>

#include "act_device.cuh"
#include "act_ff.cuh"
#include "act_internal.cuh"
#include "act_tc.cuh"

namespace act {

namespace {

using namespace tc;

constexpr int kBM = 128;           // channels per tile (MMA M)
constexpr int kBlockRows = 256;    // atoms per block of the tile-major BF16 layout
constexpr int kUmmaK = 16;         // K per tcgen05.mma (16-bit inputs)
constexpr int kMaxRescan = 512;    // flagged 32-atom blocks per channel before the FP32 full search
constexpr int kGemmThreads = 256;
constexpr int kAChunkBytes = kBM * kBK * 2;  // 16 KB
constexpr int kMaxDynSmem = 232448;
constexpr int kMaxStages = 8;

template <int BN>
struct TileCfg {
    static constexpr int kStageBytes = BN * kBK * 2;  // one dictionary chunk
    static constexpr uint32_t kTmemCols = 2 * BN;     // two accumulators (a power of two >= 32)
    // Instruction descriptor of tcgen05.mma.kind::f16: D = F32, A = B = BF16,
    // both K-major, N = BN, M = 128.
    static constexpr uint32_t kIdesc = (1u << 4)                      // D format F32
                                       | (1u << 7)                    // A format BF16
                                       | (1u << 10)                   // B format BF16
                                       | ((uint32_t)(BN >> 3) << 17)  // N / 8
                                       | ((uint32_t)(kBM >> 4) << 24);  // M / 16
};

struct GemmSmem {
    uint64_t bar_a;
    uint64_t bar_full[kMaxStages];
    uint64_t bar_empty[kMaxStages];
    uint64_t bar_acc_full[2];
    uint64_t bar_acc_empty[2];
    uint32_t tmem_base;
    int abort;
};

// a_stream = 0 (one row tile, windows up to 512 samples): the whole
// residual matrix (nkc chunks of 16 KB) is loaded once and stays resident;
// stages hold dictionary chunks only.
// a_stream = 1: every stage holds a dictionary chunk followed by the
// matching chunk of the item's residual row tile (16 KB, re-read from L2 for
// every item).
template <int BN>
__global__ void __launch_bounds__(kGemmThreads, 1)
    k_gemm_tilemax(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t K, int nkc,
                   int stages, int a_stream, int B, int m_tiles, float *__restrict__ tile_max,
                   float *__restrict__ blk_max, int *status, unsigned long long wait_ns) {
    using Cfg = TileCfg<BN>;
    extern __shared__ uint8_t dyn_raw[];
    __shared__ GemmSmem sm;
    const uint32_t dyn_base = (smem_u32(dyn_raw) + 1023u) & ~1023u;
    const uint32_t a_smem = dyn_base;
    const uint32_t b_smem = a_stream ? dyn_base : dyn_base + (uint32_t)nkc * kAChunkBytes;
    const uint32_t stage_bytes =
        a_stream ? (uint32_t)(Cfg::kStageBytes + kAChunkBytes) : (uint32_t)Cfg::kStageBytes;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = (K + BN - 1) / BN;
    const int64_t items = ntiles * m_tiles;  // item w: dictionary tile w / m_tiles, row tile w % m_tiles

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
                     "r"(Cfg::kTmemCols)
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
        if (!a_stream) {
            mbar_expect_tx(&sm.bar_a, (uint32_t)(nkc * kAChunkBytes));
            for (int kc = 0; kc < nkc; ++kc) tma_load_2d(a_smem + kc * kAChunkBytes, &tmA, kc * kBK, 0, &sm.bar_a);
        }
        uint32_t s = 0, ph = 0;  // the ring's stage and its phase parity
        for (int64_t w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x) {
            const int64_t tile = w / m_tiles;
            const int mt = (int)(w - tile * m_tiles);
            // row of this tile's first chunk in the tile-major layout viewed as [rows][64]
            const int64_t atom0 = tile * BN;
            const int64_t blk = atom0 / kBlockRows, sub = atom0 % kBlockRows;
            for (int kc = 0; kc < nkc; ++kc) {
                if (!mbar_wait(&sm.bar_empty[s], ph ^ 1u, wait_ns)) {
                    *abort_flag = 1;
                    break;
                }
                mbar_expect_tx(&sm.bar_full[s], stage_bytes);
                tma_load_2d(b_smem + s * stage_bytes, &tmB, 0, (int)((blk * nkc + kc) * kBlockRows + sub),
                            &sm.bar_full[s]);
                if (a_stream)
                    tma_load_2d(b_smem + s * stage_bytes + Cfg::kStageBytes, &tmA, kc * kBK, mt * kBM,
                                &sm.bar_full[s]);
                if (++s == (uint32_t)stages) {
                    s = 0;
                    ph ^= 1u;
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        if (!a_stream && !mbar_wait(&sm.bar_a, 0, wait_ns)) *abort_flag = 1;
        tc_fence_after();
        // the issuing thread must keep up with the tensor core (one 128 x 256 x 16
        // MMA per 128 cycles): no divisions, descriptors formed once per stage
        uint32_t s = 0, ph = 0, local = 0;
        for (int64_t w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x, ++local) {
            const uint32_t acc = local & 1u, aph = (local >> 1) & 1u;
            if (!mbar_wait(&sm.bar_acc_empty[acc], aph ^ 1u, wait_ns)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint32_t d_tmem = tmem + acc * BN;
            for (int kc = 0; kc < nkc; ++kc) {
                if (!mbar_wait(&sm.bar_full[s], ph, wait_ns)) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t b0 = b_smem + s * stage_bytes;
                const uint32_t a0 = a_stream ? b0 + Cfg::kStageBytes : a_smem + kc * kAChunkBytes;
                const uint64_t adesc = smem_desc(a0), bdesc = smem_desc(b0);
#pragma unroll
                for (int k = 0; k < kBK / kUmmaK; ++k)
                    tc_mma(d_tmem, smem_desc_k(adesc, k), smem_desc_k(bdesc, k), Cfg::kIdesc,
                           (kc | k) != 0 ? 1u : 0u);
                tc_commit(&sm.bar_empty[s]);
                if (++s == (uint32_t)stages) {
                    s = 0;
                    ph ^= 1u;
                }
            }
            tc_commit(&sm.bar_acc_full[acc]);
        }
    } else if (warp >= 4) {
        // ---------------- epilogue: thread = channel ----------------
        const int q = warp - 4;
        uint32_t local = 0;
        for (int64_t w = blockIdx.x; w < items; w += gridDim.x, ++local) {
            const int64_t tile = w / m_tiles;
            const int ch = (int)(w - tile * m_tiles) * kBM + q * 32 + lane;
            const uint32_t acc = local & 1u, aph = (local >> 1) & 1u;
            if (*abort_flag || !mbar_wait(&sm.bar_acc_full[acc], aph, wait_ns)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            // atoms past K in the last tile are zero rows: they score 0.
            // Per 32-atom block and per tile: the largest |score|
            float mx = 0.0f, bmv[BN / 32];
#pragma unroll
            for (int c = 0; c < BN / 32; ++c) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + acc * BN + c * 32, v);
                float m0 = 0.0f, m1 = 0.0f;
#pragma unroll
                for (int j = 0; j < 32; j += 2) {
                    m0 = fmaxf(m0, fabsf(v[j]));
                    m1 = fmaxf(m1, fabsf(v[j + 1]));
                }
                bmv[c] = fmaxf(m0, m1);
                mx = fmaxf(mx, bmv[c]);
            }
            tc_fence_before();
            mbar_arrive(&sm.bar_acc_empty[acc]);
            if (ch < B) {
                tile_max[(size_t)ch * ntiles + tile] = mx;
                float4 *bm4 = reinterpret_cast<float4 *>(blk_max + ((size_t)ch * ntiles + tile) * (BN / 32));
#pragma unroll
                for (int u = 0; u < BN / 128; ++u)
                    bm4[u] = make_float4(bmv[4 * u], bmv[4 * u + 1], bmv[4 * u + 2], bmv[4 * u + 3]);
            }
        }
    }

    __syncthreads();
    if (*abort_flag) {
        if (threadIdx.x == 0) atomicOr(status, kFlagTimeout);
        sleep_ns(200000);  // let in-flight copies and MMAs land before releasing memory
    }
    tc_fence_after();
    if (warp == 2) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::kTmemCols)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// Tile selection: which tiles can hold the FP32 argmax of channel b.
// ---------------------------------------------------------------------------
// Let s_j be the exact <g_j, r>, f_j the FP32 score the GEMV computes and
// h_j the tensor-core BF16 score.  With
//   delta = eps_g (|r| + |dr|) + (1 + 1e-5) |dr| + L 2^-23 (1 + eps_g)(|r| + |dr|)
// (eps_g = largest |bf16(g) - g| over the dictionary, dr = bf16(r) - r, the
// last term bounds FP32 accumulation in the tensor core) and
// eps_r = L 2^-23 |r| (FP32 accumulation of the GEMV), |h_j - s_j| <= delta
// and |f_j - s_j| <= eps_r.  If j* maximises |f| and jb maximises |h|:
//   |h_j*| >= |f_j*| - eps_r - delta >= |f_jb| - eps_r - delta
//          >= |h_jb| - 2 delta - 2 eps_r,
// so j* lies in a 32-atom block whose largest |h| is >= bmax - 2 delta -
// 2 eps_r.  The GEMM keeps both the per-tile and the per-block maxima; tiles
// at or above the threshold are narrowed to their blocks, which are queued
// for the FP32 rescan (keys[b] cleared); a channel with more than kMaxRescan
// of them is queued for the FP32 full search.  |r| and |dr| are float-float
// sums (inflated by 1e-6 for their rounding), the bound is formed in FP64
// once, and the threshold is rounded down to FP32 before the comparisons
// (the flagged set can only grow).
__global__ void __launch_bounds__(256) k_select(int64_t ntiles, int bpt, const float *__restrict__ tile_max,
                                                const float *__restrict__ blk_max, int Lp, int L,
                                                const float *__restrict__ R,
                                                const unsigned int *__restrict__ eps_bits,
                                                unsigned long long *__restrict__ keys, int *__restrict__ fb_list,
                                                int *__restrict__ counters, int *__restrict__ pairs,
                                                long long *__restrict__ stats) {
    __shared__ ff sh_e[8], sh_de[8];
    __shared__ float sh_f[8];
    __shared__ float thr_sh;
    __shared__ int n_sh;
    __shared__ int base_sh;
    __shared__ int list[kMaxRescan];
    const int b = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (int)(blockDim.x >> 5);
    const float *r = R + (size_t)b * Lp;
    const float *tm = tile_max + (size_t)b * ntiles;
    const float *bmx = blk_max + (size_t)b * ntiles * bpt;

    ff e = {0.0f, 0.0f}, de = {0.0f, 0.0f};
    for (int n = threadIdx.x; n < L; n += blockDim.x) {
        const float x = r[n];
        const float d = __bfloat162float(__float2bfloat16_rn(x)) - x;
        ff_fma_acc(e, x, x);
        ff_fma_acc(de, d, d);
    }
    e = ff_warp_sum(e);
    de = ff_warp_sum(de);
    float m = 0.0f;
    for (int64_t t = threadIdx.x; t < ntiles; t += blockDim.x) m = fmaxf(m, tm[t]);
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (lane == 0) {
        sh_e[warp] = e;
        sh_de[warp] = de;
        sh_f[warp] = m;
    }
    if (threadIdx.x == 0) n_sh = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        ff te = sh_e[0], tde = sh_de[0];
        float bmax = sh_f[0];
        for (int w = 1; w < nwarps; ++w) {
            te = ff_add(te, sh_e[w]);
            tde = ff_add(tde, sh_de[w]);
            bmax = fmaxf(bmax, sh_f[w]);
        }
        const double rn = sqrt(ff_to_double(te)) * (1.0 + 1e-6);
        const double drn = sqrt(ff_to_double(tde)) * (1.0 + 1e-6);
        const double eps_g = (double)__uint_as_float(*eps_bits);
        const double rr = rn + drn;
        const double ulp = 1.1920928955078125e-07;  // 2^-23
        const double delta = eps_g * rr + (1.0 + 1e-5) * drn + (double)L * ulp * (1.0 + eps_g) * rr;
        const double eps_r = (double)L * ulp * rn;
        thr_sh = __double2float_rd((double)bmax - 2.0 * delta - 2.0 * eps_r);
    }
    __syncthreads();
    const float thr = thr_sh;
    for (int64_t t = threadIdx.x; t < ntiles; t += blockDim.x) {
        if (tm[t] >= thr) {
            for (int k = 0; k < bpt; ++k) {
                if (bmx[t * bpt + k] < thr) continue;
                const int pos = atomicAdd(&n_sh, 1);
                if (pos < kMaxRescan) list[pos] = (int)(t * bpt + k);
            }
        }
    }
    __syncthreads();
    const int n = n_sh;
    if (n > kMaxRescan) {
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
        pairs[2 * (base_sh + i)] = b;
        pairs[2 * (base_sh + i) + 1] = list[i];
    }
}

// FP32 rescan of the flagged (channel, block) pairs: every atom of the block
// (tile_atoms of them) is scored exactly as the GEMV scores it and folded
// into keys[b] with the packed atomicMax (largest |score|, then lowest
// index).  One block of 8 warps per pair.
__global__ void __launch_bounds__(256) k_rescan(const float *__restrict__ D32, int64_t K, int Lp, int tile_atoms,
                                                const float *__restrict__ R, const int *__restrict__ pairs,
                                                const int *__restrict__ counters,
                                                unsigned long long *__restrict__ keys) {
    __shared__ float red_s[8];
    __shared__ uint32_t red_i[8];
    const int n_items = counters[1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nv = Lp / 128;
    const int rows_per_warp = tile_atoms / 8;
    for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
        const int b = pairs[2 * w];
        const int64_t tile = pairs[2 * w + 1];
        const float4 *res = reinterpret_cast<const float4 *>(R + (size_t)b * Lp);
        float best = -1.0f;
        uint32_t bidx = 0u;
        const int64_t row0 = tile * tile_atoms + warp * rows_per_warp;
        // four rows in flight per step; rows past K (last tile) are skipped
        for (int i = 0; i < rows_per_warp; i += 4) {
            float sc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t row = row0 + i + u;
                sc[u] = row < K ? fabsf(row_score(reinterpret_cast<const float4 *>(D32 + (size_t)row * Lp), res, nv,
                                                  lane))
                                : -1.0f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (sc[u] > best) {
                    best = sc[u];
                    bidx = (uint32_t)(row0 + i + u);
                }
        }
        if (lane == 0) {
            red_s[warp] = best;
            red_i[warp] = bidx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float bs = -1.0f;
            uint32_t bi = 0u;
            for (int q = 0; q < 8; ++q)
                if (red_s[q] > bs || (red_s[q] == bs && red_i[q] < bi)) {
                    bs = red_s[q];
                    bi = red_i[q];
                }
            if (bs >= 0.0f) atomicMax(keys + b, pack_key(bs, bi));
        }
        __syncthreads();
    }
}

// Dynamic shared memory the GEMM may use: the opt-in limit minus its static
// shared memory (barriers), less 1 KB of slack for 1024-byte alignment.
constexpr int kStaticSmemReserve = 512;
constexpr int kSmemBudget = kMaxDynSmem - kStaticSmemReserve - 1024;

// Largest number of stages that fits the shared memory for a tile width.
int max_stages(int bn, int nkc, bool a_stream) {
    const int chunk = bn * kBK * 2;
    int st = a_stream ? kSmemBudget / (chunk + kAChunkBytes) : (kSmemBudget - nkc * kAChunkBytes) / chunk;
    return st > kMaxStages ? kMaxStages : st;
}

}  // namespace

struct Bf16Search {
    CUtensorMap mapB[2];  // box heights 128 and 256
    int64_t K = 0;
    int Lb = 0;
    int nkc = 0;
    int a_stream = 0;     // with one row tile: 1 when the residual matrix cannot stay resident
    int sm_count = 0;
    // current configuration
    int bn = 256;
    int stages = 0;
    unsigned int *eps_bits = nullptr;  // owned by the caller (dictionary build)
};

cudaError_t bf16_search_configure(Bf16Search *s, int bn, int stages) {
    if (!s || (bn != 128 && bn != 256)) return cudaErrorInvalidValue;
    const int ms = max_stages(bn, s->nkc, s->a_stream != 0);
    if (stages <= 0) stages = ms;
    if (stages < 2 || stages > ms) return cudaErrorInvalidValue;
    // several row tiles stream the residual chunks: that form must fit too
    if (max_stages(bn, s->nkc, true) < 2) return cudaErrorInvalidValue;
    // the limit is set to everything the device allows, so every stage count
    // of either form can be launched
    cudaError_t e = bn == 256 ? allow_max_smem((const void *)k_gemm_tilemax<256>, 1024)
                              : allow_max_smem((const void *)k_gemm_tilemax<128>, 1024);
    if (e != cudaSuccess) return e;
    s->bn = bn;
    s->stages = stages;
    return cudaSuccess;
}

void bf16_search_get_config(const Bf16Search *s, int *bn, int *stages, int *max_stages_out) {
    if (bn) *bn = s->bn;
    if (stages) *stages = s->stages;
    if (max_stages_out) *max_stages_out = max_stages(s->bn, s->nkc, s->a_stream != 0);
}

int bf16_search_max_stages(const Bf16Search *s, int bn) { return max_stages(bn, s->nkc, s->a_stream != 0); }

cudaError_t bf16_search_prepare(Bf16Search **out, const __nv_bfloat16 *d16, int64_t K, int Lb, int sm_count,
                                unsigned int *eps_bits) {
    *out = nullptr;
    if (Lb % kBK != 0 || Lb > kMaxSamples || Lb < kBK) return cudaErrorNotSupported;
    const int64_t nblocks = (K + kBlockRows - 1) / kBlockRows;
    if (nblocks * (Lb / kBK) * kBlockRows >= ((int64_t)1 << 31)) return cudaErrorNotSupported;
    Bf16Search *s = new (std::nothrow) Bf16Search();
    if (!s) return cudaErrorMemoryAllocation;
    s->K = K;
    s->Lb = Lb;
    s->nkc = Lb / kBK;
    s->a_stream = s->nkc > 8 ? 1 : 0;  // a resident residual matrix must leave room for >= 3 stages
    s->sm_count = sm_count;
    s->eps_bits = eps_bits;
    // the tile-major BF16 dictionary seen as [blocks * nkc * 256 rows][64]
    const uint64_t rows = (uint64_t)nblocks * s->nkc * kBlockRows;
    if (!make_map(&s->mapB[0], d16, (uint64_t)kBK, rows, 128) ||
        !make_map(&s->mapB[1], d16, (uint64_t)kBK, rows, 256)) {
        delete s;
        return cudaErrorInvalidValue;
    }
    cudaError_t e = bf16_search_configure(s, 256, 0);
    if (e != cudaSuccess) {
        delete s;
        return e;
    }
    *out = s;
    return cudaSuccess;
}

void bf16_search_free(Bf16Search *s) { delete s; }

void bf16_scratch_free(Bf16Scratch &x) {
    if (x.tile_max) cudaFree(x.tile_max);
    if (x.blk_max) cudaFree(x.blk_max);
    if (x.pairs) cudaFree(x.pairs);
    x = Bf16Scratch();
}

cudaError_t bf16_scratch_reserve(const Bf16Search *s, int B, Bf16Scratch &x) {
    if (B <= x.B_cap) return cudaSuccess;
    bf16_scratch_free(x);
    // tile maxima at the narrowest tile (128 atoms), block maxima over whole 256-atom tiles
    cudaError_t e = dev_alloc((void **)&x.tile_max, sizeof(float) * (size_t)B * ((s->K + 127) / 128));
    if (e == cudaSuccess) e = dev_alloc((void **)&x.blk_max, sizeof(float) * (size_t)B * ((s->K + 255) / 256) * 8);
    if (e == cudaSuccess) e = dev_alloc((void **)&x.pairs, sizeof(int) * 2 * (size_t)B * kMaxRescan);
    if (e != cudaSuccess) {
        bf16_scratch_free(x);
        return e;
    }
    x.B_cap = B;
    return cudaSuccess;
}

cudaError_t launch_bf16_gemm(const Bf16Search *s, const Bf16Scratch &x, int B, const __nv_bfloat16 *R16, int *status,
                             cudaStream_t st, unsigned long long wait_ns) {
    if (!s || B < 1 || B > x.B_cap) return cudaErrorInvalidValue;
    const int m_tiles = (B + kBM - 1) / kBM;
    const bool astr = s->a_stream || m_tiles > 1;
    const int ms = max_stages(s->bn, s->nkc, astr);
    const int stages = s->stages < ms ? s->stages : ms;
    if (stages < 2) return cudaErrorInvalidValue;
    const size_t chunk = (size_t)s->bn * kBK * 2;
    const size_t smem = astr ? 1024 + (size_t)stages * (chunk + kAChunkBytes)
                             : 1024 + (size_t)s->nkc * kAChunkBytes + (size_t)stages * chunk;
    const int64_t ntiles = (s->K + s->bn - 1) / s->bn;
    const int64_t items = ntiles * m_tiles;
    const int grid = (int)(items < s->sm_count ? items : s->sm_count);
    // the residual rows [m_tiles * 128][Lb] (rows past B are zero)
    CUtensorMap mapA;
    if (!make_map(&mapA, R16, (uint64_t)s->Lb, (uint64_t)m_tiles * kBM, kBM)) return cudaErrorInvalidValue;
    if (s->bn == 256)
        k_gemm_tilemax<256><<<grid, kGemmThreads, smem, st>>>(mapA, s->mapB[1], s->K, s->nkc, stages, astr ? 1 : 0,
                                                              B, m_tiles, x.tile_max, x.blk_max, status, wait_ns);
    else
        k_gemm_tilemax<128><<<grid, kGemmThreads, smem, st>>>(mapA, s->mapB[0], s->K, s->nkc, stages, astr ? 1 : 0,
                                                              B, m_tiles, x.tile_max, x.blk_max, status, wait_ns);
    return cudaGetLastError();
}

cudaError_t launch_bf16_resolve(const Bf16Search *s, const Bf16Scratch &x, int B, const float *D32, int Lp, int L,
                                const float *R, unsigned long long *keys, int *fb_list, int *fb_count,
                                long long *stats, int *status, int gemv_grid, cudaStream_t st,
                                unsigned long long wait_ns) {
    if (!s || B < 1 || B > x.B_cap) return cudaErrorInvalidValue;
    const int64_t ntiles = (s->K + s->bn - 1) / s->bn;
    k_select<<<B, 256, 0, st>>>(ntiles, s->bn / 32, x.tile_max, x.blk_max, Lp, L, R, s->eps_bits, keys, fb_list,
                                fb_count, x.pairs, stats);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_rescan<<<2 * s->sm_count, 256, 0, st>>>(D32, s->K, Lp, 32, R, x.pairs, fb_count, keys);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // FP32 full search for the channels with too many flagged blocks
    return launch_gemv_argmax(D32, s->K, Lp, R, B, fb_list, fb_count, keys, status, gemv_grid, st, wait_ns);
}

}  // namespace act
