// Tensor-core search over the template dictionary, exact with respect to the
// FP32 template search (act_shift.cu):
//  1. the residuals are laid out as shifted rows X[(b, j)][kk] =
//     bf16(r_b[m_lo + kk + tc_j]) (zero outside the window), so that
//     <r_b, u_{t, tc_j}> = sum_kk u_t(m_lo + kk) X[(b, j)][kk]: one GEMM of
//     the BF16 templates (N = 256 templates per tile) against the shifted
//     residual rows (M = 128 rows per tile), K = Kt lags;
//  2. the tcgen05 GEMM scales every accumulator by its atom's 1/|u| and keeps,
//     per row, the largest |score| of every template tile and of every
//     32-template block;
//  3. a flag kernel bounds the BF16 error per channel and flags the
//     (time centre, 32-template block) items that can hold the FP32 template
//     search's argmax (scanning the tile maxima, then the flagged tiles' blocks);
//  4. the flagged items are rescored with the FP32 template search's own
//     arithmetic (same FMA chain, same scale) and folded into the packed key;
//     a channel with too many items has all of its items rescored that way.
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

// (a0 b0, a1 b1) by one packed FP32 multiply, each product rounded to
// nearest as a scalar multiply would be: the epilogue shares its warp
// scheduler with the MMA-issuing warp, so its instruction count matters.
__device__ __forceinline__ float2 mul_f32x2(float a0, float a1, float b0, float b1) {
    unsigned long long x, y, r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a0), "f"(a1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b0), "f"(b1));
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
    float2 o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));
    return o;
}

// Bounded wait on a phase by polling test_wait (never suspending the
// thread), with an optional pause between polls; PAIR: cluster-scope
// acquire.  The MMA-issuing thread polls without pausing, so it resumes the
// moment a stage lands; the epilogue pauses, taking fewer issue slots from
// the MMA-issuing warp that shares its scheduler.  Limit 0: one test.
template <bool PAIR>
__device__ __forceinline__ bool mbar_poll(uint64_t *bar, uint32_t parity, unsigned long long limit_ns,
                                          unsigned pause_ns) {
    auto test = [&]() { return PAIR ? mbar_test_wait_cluster(bar, parity) : mbar_test_wait(bar, parity); };
    if (test()) return true;
    if (limit_ns == 0) return false;
    const unsigned long long t0 = globaltimer_ns();
    while (!test()) {
        if (globaltimer_ns() - t0 >= limit_ns) return false;
        if (pause_ns) __nanosleep(pause_ns);
    }
    return true;
}

constexpr int kBM = 128;          // shifted residual rows per tile (MMA M)
constexpr int kBlockRows = 256;   // templates per block of the tile-major BF16 layout
constexpr int kUmmaK = 16;
constexpr int kThreads = 256;
constexpr int kAChunkBytes = kBM * kBK * 2;  // 16 KB
constexpr int kMaxStages = 6;
constexpr int kUnitTab = 1024;  // row units whose lag-chunk range is tabulated in shared memory

// Tile of BN templates (128 or 256, MMA N).  PAIR: a CTA pair shares each
// MMA (M = 256: the two CTAs' row tiles), each CTA loading BN / 2 of the
// templates; every CTA still holds a 128 x BN accumulator of its own rows.
template <int BN, bool PAIR = false>
struct ShiftTile {
    static constexpr int kBRows = PAIR ? BN / 2 : BN;  // template rows this CTA loads
    static constexpr int kBChunkBytes = kBRows * kBK * 2;
    static constexpr int kStageBytes = kAChunkBytes + kBChunkBytes;
    static constexpr uint32_t kTmemCols = 2 * BN;
    static constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                       ((uint32_t)((PAIR ? 2 * kBM : kBM) >> 4) << 24);
};
constexpr int kMaxItems = 1024;    // flagged (lag, block) items per channel before the full FP32 search
constexpr int kRescanWarps = 4;     // independent warps per rescore block

struct Smem {
    uint64_t bar_full[kMaxStages];
    uint64_t bar_empty[kMaxStages];
    uint64_t bar_acc_full[2];
    uint64_t bar_acc_empty[2];
    uint32_t tmem_base;
    int abort;
    unsigned int chan_max[2][kBM];  // per item parity: the tile's channel maxima (float bits)
    // the lag-chunk range [x, y] of row units 0 .. kUnitTab - 1, formed
    // during set-up: the single thread that issues the MMAs reads it at
    // every item instead of dividing (units past the table: computed there)
    short2 unit_chunk[kUnitTab];
};

// Named barrier 1 over the 128 epilogue threads, returning whether any of
// them passed a nonzero predicate (all of them get the same answer).
__device__ __forceinline__ int epilogue_bar_or(int pred) {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.s32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, 128, p;\n\t"
        "selp.s32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(pred)
        : "memory");
    return r;
}

// Row tiles of the GEMM: tile mt = g * n_cb + cb holds Bg = 128 / Jt
// channels (cb * Bg ..) times Jt neighbouring time centres (g * Jt ..); local
// row lr = (j - g Jt) Bg + (b - cb Bg), channels fastest, so with Bg >= 32
// the 32 rows an epilogue warp holds share one time centre (its scale loads
// are broadcasts).  Rows of one tile see the window
// only over lags [kc_lo, kc_hi] (in 64-lag chunks): L + (Jt - 1) S lags
// instead of Kt, the chunks outside hold only zero products and are skipped.
struct RowTiling {
    int B, Ntc, Jt, Bg, n_cb, m_tiles;
    int S, L, span0;  // span0 = -m_lo - tc0 = S (Ntc - 1); sample n at time centre j sits at lag n + span0 - S j
};

__host__ __device__ inline void tile_row(const RowTiling &t, int mt, int lr, int &b, int &j) {
    const int g = mt / t.n_cb, cb = mt - g * t.n_cb;
    b = cb * t.Bg + lr % t.Bg;
    j = g * t.Jt + lr / t.Bg;
}

__host__ __device__ inline void tile_chunks(const RowTiling &t, int mt, int &kc_lo, int &kc_hi) {
    const int g = mt / t.n_cb;
    const int j_first = g * t.Jt;
    const int j_last = min(j_first + t.Jt, t.Ntc) - 1;
    const int kk_min = t.span0 - t.S * j_last;           // sample 0 at the last time centre
    const int kk_max = t.L - 1 + t.span0 - t.S * j_first;  // sample L - 1 at the first
    kc_lo = kk_min / kBK;
    kc_hi = kk_max / kBK;
}

// Lag chunks of GEMM row unit u: one row tile, or (pair) the union of row
// tiles 2u and 2u + 1 (the second clamped to the last tile).  Chunks outside
// a tile's windows multiply zeros.
__host__ __device__ inline void unit_chunks(const RowTiling &t, bool pair, int u, int &kc_lo, int &kc_hi) {
    if (!pair) {
        tile_chunks(t, u, kc_lo, kc_hi);
        return;
    }
    int lo1, hi1;
    tile_chunks(t, 2 * u, kc_lo, kc_hi);
    tile_chunks(t, min(2 * u + 1, t.m_tiles - 1), lo1, hi1);
    kc_lo = min(kc_lo, lo1);
    kc_hi = max(kc_hi, hi1);
}

// Shifted residual rows X[(b, j)][kk] = bf16(r_b[m_lo + kk + tc0 + S j]),
// zero where the index leaves [0, L).  Block (g * n_seg + seg, b) writes
// channel b's rows for time centres j0 = g RJ .. j0 + RJ - 1 (those below
// Ntc), lags kk in [k0, k1) = [seg KSEG, min(Kt, (seg + 1) KSEG)).  It stages
// the samples those pieces cover, n_lo + i for i in [0, span) with
// n_lo = m_lo + tc0 + S j0 + k0 and span = S (rows - 1) + k1 - k0, as BF16
// in shared memory: once as read (global loads issued four at a time), then
// in 8 copies shifted by 0..7 samples built from it (copy s holds sample
// i + s at i): the 8 samples of any 16-byte output piece, at offset
// o = S jj + kk - k0, are one aligned 16-byte load from copy o & 7.  Padding
// rows (b >= B or j >= Ntc) are not written (the GEMM's epilogue ignores
// them).  Block (0, b) also prepares channel b's selection for this order:
// |r| and |bf16(r) - r| (for the error bound), the channel maximum and item
// count cleared.
__global__ void __launch_bounds__(256) k_shift_rows(RowTiling t, const float *__restrict__ R, int Lp, int tc0,
                                                    int m_lo, int Kt, int RJ, int KSEG, int n_seg, int span_pad,
                                                    __nv_bfloat16 *__restrict__ X, double2 *__restrict__ chan_norm,
                                                    unsigned int *__restrict__ chmax, int *__restrict__ chcount,
                                                    long long *__restrict__ stats) {
    extern __shared__ __align__(16) uint8_t rows_raw[];
    __shared__ float sh[32];
    // a programmatic dependent of the previous kernel (the residual update):
    // wait for it in every block, then let the GEMM launch
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int b = blockIdx.y, g = blockIdx.x / n_seg, seg = blockIdx.x - g * n_seg;
    const int j0 = g * RJ, nj = min(RJ, t.Ntc - j0);
    const int k0 = seg * KSEG, k1 = min(Kt, k0 + KSEG);
    const int L = t.L, S = t.S;
    const float *r = R + (size_t)b * Lp;
    if (blockIdx.x == 0) {
        // FP32 sums of at most 2048 squares are within 2048 * 2^-24 < 1.3e-4
        // (relative) of the exact ones: inflated by 1e-3 they bound them
        float e = 0.0f, de = 0.0f;
        for (int n = threadIdx.x; n < L; n += blockDim.x) {
            const float x = r[n];
            const float d = __bfloat162float(__float2bfloat16_rn(x)) - x;  // exact
            e = fmaf(x, x, e);
            de = fmaf(d, d, de);
        }
        const float te = block_sum(e, sh);
        const float tde = block_sum(de, sh);
        if (threadIdx.x == 0) {
            chan_norm[b] = make_double2(sqrt((double)te * (1.0 + 1e-3)), sqrt((double)tde * (1.0 + 1e-3)));
            chmax[b] = 0u;
            chcount[b] = 0;
            atomicAdd((unsigned long long *)&stats[0], 1ull);
        }
    }
    if (nj <= 0 || k0 >= k1) return;
    // the 8 shifted BF16 copies, span_pad (a multiple of 8, >= span) samples
    // each, then the plain staged window of span_pad + 8 samples
    __nv_bfloat16 *plain = reinterpret_cast<__nv_bfloat16 *>(rows_raw) + 8 * span_pad;
    const int n_lo = m_lo + tc0 + S * j0 + k0;
    const int total = span_pad + 8;
    for (int i0 = threadIdx.x; i0 < total; i0 += 4 * blockDim.x) {
        float x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * blockDim.x, n = n_lo + i;
            x[u] = (i < total && n >= 0 && n < L) ? r[n] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < total) plain[i] = __float2bfloat16_rn(x[u]);
        }
    }
    __syncthreads();
    // copy s, pair q = plain samples 2q + s and 2q + s + 1: as 32-bit words of
    // the plain window, word q + s / 2, shifted by a half word when s is odd
    const int half = span_pad >> 1;
    const uint32_t *pw = reinterpret_cast<const uint32_t *>(plain);
    uint32_t *cw = reinterpret_cast<uint32_t *>(rows_raw);
    for (int q = threadIdx.x; q < half; q += blockDim.x) {
        uint32_t w[5];
#pragma unroll
        for (int u = 0; u < 5; ++u) w[u] = pw[q + u];
#pragma unroll
        for (int sft = 0; sft < 8; ++sft)
            cw[sft * half + q] = (sft & 1) ? __funnelshift_r(w[sft >> 1], w[(sft >> 1) + 1], 16) : w[sft >> 1];
    }
    __syncthreads();
    const uint4 *cp16 = reinterpret_cast<const uint4 *>(rows_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = k0 >> 3, c1 = k1 >> 3;
    const int cb = b / t.Bg, bl = b - cb * t.Bg;
    for (int jj = warp; jj < nj; jj += blockDim.x >> 5) {
        const int j = j0 + jj, gt = j / t.Jt, jl = j - gt * t.Jt;
        const int row = (gt * t.n_cb + cb) * kBM + jl * t.Bg + bl;
        uint4 *out = reinterpret_cast<uint4 *>(X + (size_t)row * Kt);
        for (int c = c0 + lane; c < c1; c += 32) {
            const int o = S * jj + 8 * c - k0, sft = o & 7;
            out[c] = cp16[(sft * span_pad + (o - sft)) >> 3];
        }
    }
}

// GEMM work item w: row unit w / n_tiles, template tile w % n_tiles.  Every
// stage holds one template chunk (BN x 64) and the matching residual chunk
// (128 x 64).  Warp 0: TMA producer; warp 1: MMA issuer; warp 2: tensor
// memory owner; warps 4-7: epilogue (thread = residual row).
//
// PAIR (launched as clusters of 2): a unit is the row tiles 2u and 2u + 1,
// one per CTA of the pair, over the union of their lag chunks.  Each CTA
// loads its rows and its half of the template chunk, both copies counted on
// the leader's (rank 0) full barrier; the leader issues the M = 256 MMAs and
// its commits arrive on both CTAs' barriers; each CTA's epilogue reads its
// own accumulator and releases it on the leader's barrier.
template <int BN, bool PAIR>
__global__ void __launch_bounds__(kThreads, 1)
    k_shift_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, RowTiling tl,
                 int n_tiles, int nkc, int stages, int T_pad, const float *__restrict__ scaleT,
                 float *__restrict__ tile_max, float *__restrict__ blk_max, unsigned int *__restrict__ chmax,
                 int *status, unsigned long long wait_ns) {
    // shared memory: stages, then the item's scales [Jt][BN + 4] (the +4
    // floats of padding spread the Jt rows a warp reads over the banks)
    using Cfg = ShiftTile<BN, PAIR>;
    constexpr int kBChunkBytes = Cfg::kBChunkBytes, kStageBytes = Cfg::kStageBytes;
    constexpr uint32_t kTmemCols = Cfg::kTmemCols;
    extern __shared__ uint8_t dyn_raw[];
    __shared__ Smem sm;
    const uint32_t base = (smem_u32(dyn_raw) + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // PAIR: rank in the pair, the pair's index and count (1-D clusters of 2)
    const uint32_t rank = PAIR ? cta_rank_in_cluster() : 0u;
    const int64_t unit0 = PAIR ? blockIdx.x / 2 : blockIdx.x;
    const int64_t n_units = PAIR ? gridDim.x / 2 : gridDim.x;
    const int m_units = PAIR ? (tl.m_tiles + 1) / 2 : tl.m_tiles;
    const int64_t items = (int64_t)m_units * n_tiles;
    const int Ntc = tl.Ntc;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&sm.bar_full[s], 1);
            mbar_init(&sm.bar_empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&sm.bar_acc_full[a], 1);
            // PAIR: one arrival per epilogue warp of either CTA
            mbar_init(&sm.bar_acc_empty[a], PAIR ? 8 : 128);
        }
        sm.abort = 0;
        fence_mbar_init();
    }
    if (threadIdx.x < 2 * kBM) sm.chan_max[threadIdx.x / kBM][threadIdx.x % kBM] = 0u;
    for (int u = threadIdx.x; u < m_units && u < kUnitTab; u += blockDim.x) {
        int lo, hi;
        unit_chunks(tl, PAIR, u, lo, hi);
        sm.unit_chunk[u] = make_short2((short)lo, (short)hi);
    }
    if (warp == 2) {
        if constexpr (PAIR) {  // the same columns in both CTAs, allocated by one warp of each
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&sm.tmem_base)),
                         "r"(kTmemCols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&sm.tmem_base)),
                         "r"(kTmemCols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    // PAIR: both CTAs' barriers initialised and tensor memory allocated
    // before either copies, commits or arrives across the pair
    if constexpr (PAIR) cluster_barrier();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;
    volatile int *abort_flag = &sm.abort;
    // set-up above overlaps the shifted-row build; everything below reads its
    // rows (and the channel maxima it cleared) only after it completes
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
        uint32_t s = 0, ph = 0;  // the ring's stage and its phase parity
        for (int64_t w = unit0; w < items && !*abort_flag; w += n_units) {
            const int u = (int)(w / n_tiles), nt = (int)(w % n_tiles);
            // this CTA's row tile (PAIR: past the last tile, load the last one again)
            const int mt = PAIR ? min(2 * u + (int)rank, tl.m_tiles - 1) : u;
            int kc_lo, kc_hi;
            if (u < kUnitTab) {
                kc_lo = sm.unit_chunk[u].x;
                kc_hi = sm.unit_chunk[u].y;
            } else {
                unit_chunks(tl, PAIR, u, kc_lo, kc_hi);
            }
            for (int kc = kc_lo; kc <= kc_hi; ++kc) {
                const bool ok = PAIR ? mbar_wait_cluster(&sm.bar_empty[s], ph ^ 1u, wait_ns)
                                     : mbar_wait(&sm.bar_empty[s], ph ^ 1u, wait_ns);
                if (!ok) {
                    *abort_flag = 1;
                    break;
                }
                const uint32_t b0 = base + (uint32_t)s * kStageBytes;
                // templates: the tile-major layout seen as [blocks * nkc * 256][64]
                const int64_t t0 = (int64_t)nt * BN + (int64_t)rank * Cfg::kBRows;
                const int64_t blk = t0 / kBlockRows, sub = t0 % kBlockRows;
                const int yB = (int)((blk * nkc + kc) * kBlockRows + sub);
                if constexpr (PAIR) {
                    // both CTAs' copies complete on the leader's barrier
                    if (rank == 0) mbar_expect_tx(&sm.bar_full[s], (uint32_t)(2 * kStageBytes));
                    const uint32_t fb = cluster_addr(&sm.bar_full[s], 0);
                    tma_load_2d_pair(b0, &tmB, 0, yB, fb);
                    tma_load_2d_pair(b0 + kBChunkBytes, &tmA, kc * kBK, mt * kBM, fb);
                } else {
                    mbar_expect_tx(&sm.bar_full[s], (uint32_t)kStageBytes);
                    tma_load_2d(b0, &tmB, 0, yB, &sm.bar_full[s]);
                    tma_load_2d(b0 + kBChunkBytes, &tmA, kc * kBK, mt * kBM, &sm.bar_full[s]);
                }
                if (++s == (uint32_t)stages) {
                    s = 0;
                    ph ^= 1u;
                }
            }
        }
    } else if (warp == 1 && lane == 0 && rank == 0) {
        // ---------------- MMA issuer (PAIR: the leader only) ----------------
        tc_fence_after();
        // the issuing thread must keep up with the tensor core (one M x 256 x 16
        // MMA per 128 cycles): no divisions, descriptors formed once per stage
        uint32_t s = 0, ph = 0, local = 0;
        for (int64_t w = unit0; w < items && !*abort_flag; w += n_units, ++local) {
            const uint32_t acc = local & 1u, aph = (local >> 1) & 1u;
            const bool ok = PAIR ? mbar_wait_cluster(&sm.bar_acc_empty[acc], aph ^ 1u, wait_ns)
                                 : mbar_wait(&sm.bar_acc_empty[acc], aph ^ 1u, wait_ns);
            if (!ok) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint32_t d_tmem = tmem + acc * BN;
            int kc_lo, kc_hi;
            const int u = (int)(w / n_tiles);
            if (u < kUnitTab) {
                kc_lo = sm.unit_chunk[u].x;
                kc_hi = sm.unit_chunk[u].y;
            } else {
                unit_chunks(tl, PAIR, u, kc_lo, kc_hi);
            }
            for (int kc = kc_lo; kc <= kc_hi; ++kc) {
                const bool full = mbar_poll<PAIR>(&sm.bar_full[s], ph, wait_ns, 0);
                if (!full) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t b0 = base + s * (uint32_t)kStageBytes;
                const uint64_t bdesc = smem_desc(b0), adesc = smem_desc(b0 + kBChunkBytes);
#pragma unroll
                for (int k = 0; k < kBK / kUmmaK; ++k) {
                    const uint32_t accum = (kc != kc_lo || k != 0) ? 1u : 0u;
                    if constexpr (PAIR)
                        tc_mma_pair(d_tmem, smem_desc_k(adesc, k), smem_desc_k(bdesc, k), Cfg::kIdesc, accum);
                    else
                        tc_mma(d_tmem, smem_desc_k(adesc, k), smem_desc_k(bdesc, k), Cfg::kIdesc, accum);
                }
                if constexpr (PAIR)
                    tc_commit_pair(&sm.bar_empty[s], 0x3);
                else
                    tc_commit(&sm.bar_empty[s]);
                if (++s == (uint32_t)stages) {
                    s = 0;
                    ph ^= 1u;
                }
            }
            if constexpr (PAIR)
                tc_commit_pair(&sm.bar_acc_full[acc], 0x3);
            else
                tc_commit(&sm.bar_acc_full[acc]);
        }
    } else if (warp >= 4) {
        // ---------------- epilogue: thread = shifted residual row ----------------
        const int q = warp - 4;
        const int et = threadIdx.x - 128;  // 0..127 over the epilogue warps
        constexpr int kScaleLd = BN + 4;
        float *sc_sm = reinterpret_cast<float *>(dyn_raw + (base - smem_u32(dyn_raw)) + (size_t)stages * kStageBytes);
        uint32_t local = 0;
        for (int64_t w = unit0; w < items; w += n_units, ++local) {
            const int unit = (int)(w / n_tiles), nt = (int)(w % n_tiles);
            const int mt = PAIR ? 2 * unit + (int)rank : unit;  // PAIR: may be one past the last tile (no rows)
            // the tile's Jt scale rows (j0 .. j0 + Jt - 1, those below Ntc), BN each
            {
                const int j0 = (mt / tl.n_cb) * tl.Jt;
                const int rows = min(tl.Jt, Ntc - j0);
                const int per_row = BN / 4;  // 16-byte pieces
                for (int i = et; i < rows * per_row; i += 128) {
                    const int rr = i / per_row, cc = i % per_row;
                    const float *src = scaleT + (size_t)(j0 + rr) * T_pad + (size_t)nt * BN + 4 * cc;
                    const uint32_t dst = smem_u32(sc_sm + rr * kScaleLd + 4 * cc);
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
                }
                asm volatile("cp.async.wait_all;" ::: "memory");
                asm volatile("bar.sync 1, 128;" ::: "memory");
            }
            const uint32_t acc = local & 1u, aph = (local >> 1) & 1u;
            const bool landed = mbar_poll<PAIR>(&sm.bar_acc_full[acc], aph, wait_ns, 256);
            const int failed = (*abort_flag || !landed) ? 1 : 0;
            if (epilogue_bar_or(failed)) {  // the epilogue warps leave together
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const int lr = q * 32 + lane;
            int b, j;
            tile_row(tl, mt, lr, b, j);
            const bool valid = mt < tl.m_tiles && b < tl.B && j < Ntc;
            const float4 *sc4 = reinterpret_cast<const float4 *>(sc_sm + (valid ? lr / tl.Bg : 0) * kScaleLd);
            // per 32-template block and per tile: the largest scaled |score|
            float *bm = blk_max + ((size_t)(valid ? b : 0) * Ntc + (valid ? j : 0)) * (T_pad / 32) +
                        (size_t)nt * (BN / 32);
            float mx = 0.0f, bmv[BN / 32];
#pragma unroll
            for (int c = 0; c < BN / 32; ++c) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + acc * BN + c * 32, v);
                float m0 = 0.0f, m1 = 0.0f;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float4 s = valid ? sc4[c * 8 + e] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float2 p01 = mul_f32x2(v[4 * e], v[4 * e + 1], s.x, s.y);
                    const float2 p23 = mul_f32x2(v[4 * e + 2], v[4 * e + 3], s.z, s.w);
                    m0 = fmaxf(m0, fabsf(p01.x));
                    m1 = fmaxf(m1, fabsf(p01.y));
                    m0 = fmaxf(m0, fabsf(p23.x));
                    m1 = fmaxf(m1, fabsf(p23.y));
                }
                bmv[c] = fmaxf(m0, m1);
                mx = fmaxf(mx, bmv[c]);
            }
            tc_fence_before();
            if constexpr (PAIR) {  // one arrival per warp, on the leader's barrier
                __syncwarp();
                if (lane == 0) mbar_arrive_remote(cluster_addr(&sm.bar_acc_empty[acc], 0));
            } else {
                mbar_arrive(&sm.bar_acc_empty[acc]);
            }
            if (valid) {  // the row's BN / 32 block maxima are contiguous: 16-byte stores
                float4 *bm4 = reinterpret_cast<float4 *>(bm);
#pragma unroll
                for (int u = 0; u < BN / 128; ++u)
                    bm4[u] = make_float4(bmv[4 * u], bmv[4 * u + 1], bmv[4 * u + 2], bmv[4 * u + 3]);
                tile_max[((size_t)b * Ntc + j) * n_tiles + nt] = mx;
            }
            // channel maximum: non-negative floats order like their bits.  The
            // rows of one channel are the lanes lr % Bg equal: fold them within
            // the warp, then across the warps in shared memory; one global
            // atomic per channel and tile
            unsigned bits = valid ? __float_as_uint(mx) : 0u;
            for (int off = 16; off >= tl.Bg; off >>= 1) {
                const unsigned o = __shfl_xor_sync(0xffffffffu, bits, off);
                bits = o > bits ? o : bits;
            }
            unsigned int *cm = sm.chan_max[local & 1u];
            if (tl.Bg >= 32 || lane < tl.Bg) atomicMax(cm + lr % tl.Bg, bits);
            asm volatile("bar.sync 1, 128;" ::: "memory");  // also: the scale rows are reloaded for the next item
            if (et < tl.Bg) {
                const int bc = (mt % tl.n_cb) * tl.Bg + et;
                if (bc < tl.B) atomicMax(chmax + bc, cm[et]);
                cm[et] = 0u;  // rewritten two items later, after another barrier
            }
        }
    }

    __syncthreads();
    if (*abort_flag) {
        if (threadIdx.x == 0) atomicOr(status, kFlagTimeout);
        sleep_ns(200000);  // let in-flight copies and MMAs land before releasing memory
    }
    // PAIR: neither CTA leaves (or frees tensor memory) while the other may
    // still copy into, commit to or arrive on its shared memory
    if constexpr (PAIR) cluster_barrier();
    tc_fence_after();
    if (warp == 2) {
        if constexpr (PAIR)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                         : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                         : "memory");
    }
}

// Item selection for channel b (blockIdx.y; blockIdx.x slices its entries).
// With s the exact score, f the
// FP32 template search's score and h the tensor-core score of an atom,
//   |f - s| <= eps_r = (L + 4) 2^-23 |r|
// (one FP32 chain of L products, the FP32 scale and the final product), and
//   |h - s| <= delta = (1 + 1e-5) [eps_u (|r| + |dr|) + |dr|
//                                  + Kt 2^-23 (1 + eps_u)(|r| + |dr|)]
// (eps_u = largest |bf16(u) - u| / |u| over the atoms' windows, dr =
// bf16(r) - r, the Kt term bounds FP32 accumulation in the tensor core, the
// factor the scale product).  As for the dense BF16 search, the FP32 argmax
// lies in an item whose largest |h| is >= hmax - 2 delta - 2 eps_r.
__global__ void __launch_bounds__(256) k_shift_flag(int Ntc, int n_tiles, int bpt, int Kt, int L,
                                                    const float *__restrict__ tile_max,
                                                    const float *__restrict__ blk_max,
                                                    const double2 *__restrict__ chan_norm,
                                                    const unsigned int *__restrict__ chmax,
                                                    const unsigned int *__restrict__ eps_bits,
                                                    int *__restrict__ chcount, int *__restrict__ fb_list,
                                                    int *__restrict__ counters, int *__restrict__ items,
                                                    long long *__restrict__ stats) {
    const int b = blockIdx.y;
    __shared__ float thr_sh;
    asm volatile("griddepcontrol.wait;" ::: "memory");  // the GEMM's maxima
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (threadIdx.x == 0) {  // the bound in FP64, once per block
        const double2 nr = chan_norm[b];
        const double rn = nr.x, drn = nr.y;
        const double eps_u = (double)__uint_as_float(*eps_bits);
        const double rr = rn + drn;
        const double ulp = 1.1920928955078125e-07;  // 2^-23
        const double delta = (1.0 + 1e-5) * (eps_u * rr + drn + (double)Kt * ulp * (1.0 + eps_u) * rr);
        const double eps_r = (double)(L + 4) * ulp * rn;
        const double thr = (double)__uint_as_float(chmax[b]) - 2.0 * delta - 2.0 * eps_r;
        // FP32 compare against the threshold rounded down: a superset of the items
        thr_sh = __double2float_rd(thr);
    }
    __syncthreads();
    const float thr_f = thr_sh;
    // scan the tile maxima; a tile at or above the threshold is narrowed to
    // its 32-template blocks at or above it (the items: i = j * n_blocks + block)
    const float *tm = tile_max + (size_t)b * Ntc * n_tiles;
    const int n_entries = Ntc * n_tiles;
    const int n_blocks = n_tiles * bpt;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_entries; i += gridDim.x * blockDim.x) {
        if (tm[i] >= thr_f) {
            const int j = i / n_tiles, tile = i - j * n_tiles;
            const float *bm = blk_max + ((size_t)b * Ntc + j) * n_blocks + (size_t)tile * bpt;
            for (int k = 0; k < bpt; ++k) {
                if (bm[k] < thr_f) continue;
                const int pos = atomicAdd(chcount + b, 1);
                if (pos < kMaxItems) {
                    const int at = atomicAdd(&counters[1], 1);
                    items[2 * at] = b;
                    items[2 * at + 1] = j * n_blocks + tile * bpt + k;
                    atomicAdd((unsigned long long *)&stats[2], 1ull);
                } else if (pos == kMaxItems) {
                    // too many: the FP32 template search scores this channel in full
                    fb_list[atomicAdd(&counters[0], 1)] = b;
                    atomicAdd((unsigned long long *)&stats[1], 1ull);
                    atomicAdd((unsigned long long *)&stats[0], ~0ull);  // -1: not resolved by the items
                }
            }
        }
    }
}

// FP32 rescore, one warp per flagged (lag, 32-template block) item.  Lane =
// template.  Per phase
// a, the P template rows the FP32 template search reads for this lag
// (contiguous, P x 128 bytes) arrive by a bulk copy into one of the warp's
// two buffers (the next phase's copy is in flight while this one is used);
// each lane runs the FP32 search's FMA chain over them in its order and
// scales the sum the same way.  Each warp owns its barriers, buffers and
// residual phases; warps never wait on one another.
__global__ void __launch_bounds__(kRescanWarps * 32) k_shift_rescan(
    const float *__restrict__ tpl, const float *__restrict__ scale, int S, int Sa, int P, int rows, int NtcP,
    int Ntc, int T, int n_blocks, int Lp, int L, const float *__restrict__ R, const int *__restrict__ items,
    const int *__restrict__ counters, unsigned long long *__restrict__ keys, int *status,
    unsigned long long wait_ns) {
    extern __shared__ __align__(128) float sm[];  // per warp: the residual [Lp], then 2 x [P][32] rows
    __shared__ __align__(8) uint64_t bar[kRescanWarps][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t warp_floats = (size_t)Lp + 2 * (size_t)P * 32;
    float *rres = sm + warp * warp_floats;
    float *buf0 = rres + Lp;
    const uint32_t bytes = (uint32_t)P * 128u;
    asm volatile("griddepcontrol.wait;" ::: "memory");  // the flagged items
    const int n_tasks = counters[1];  // at most kMaxItems per channel
    // the fallback search behind this kernel may launch now: it reads
    // nothing of ours before its wait for our completion
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int nw = (int)(blockDim.x >> 5);
    if (lane == 0) {
        mbar_init(&bar[warp][0], 1);
        mbar_init(&bar[warp][1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t uses[2] = {0u, 0u};
    int cur_b = -1;
    // tasks go to the first warp of every block before the second (one task
    // per SM while there are fewer tasks than SMs)
    const int64_t stride = (int64_t)gridDim.x * nw;
    for (int64_t task = (int64_t)warp * gridDim.x + blockIdx.x; task < n_tasks; task += stride) {
        const int b = items[2 * task];
        const int e = items[2 * task + 1];  // j * n_blocks + block
        const int j = e / n_blocks, tb = e % n_blocks;
        if (tb * 32 >= T) continue;  // past the last template
        const float *src = tpl + ((size_t)tb * Sa * rows + (size_t)(NtcP - 1 - j)) * 32;
        __syncwarp();
        if (lane == 0) {  // phase 0's rows and, for a new channel, its residual on the same barrier
            const bool new_b = b != cur_b;
            mbar_expect_tx(&bar[warp][0], bytes + (new_b ? (uint32_t)Lp * 4u : 0u));
            bulk_g2s(buf0, src, bytes, &bar[warp][0]);
            if (new_b) bulk_g2s(rres, R + (size_t)b * Lp, (uint32_t)Lp * 4u, &bar[warp][0]);
        }
        cur_b = b;
        float acc = 0.0f;
        int ok = 1, fail_a = 0;
        for (int a = 0; a < Sa; ++a) {
            const int cb = a & 1;
            if (a + 1 < Sa && lane == 0) {
                // the other buffer was released by the __syncwarp ending phase a - 1
                mbar_expect_tx(&bar[warp][cb ^ 1], bytes);
                bulk_g2s(buf0 + (size_t)(cb ^ 1) * P * 32, src + (size_t)(a + 1) * rows * 32, bytes,
                         &bar[warp][cb ^ 1]);
            }
            ok = mbar_wait(&bar[warp][cb], uses[cb] & 1u, wait_ns) ? 1 : 0;
            ++uses[cb];
            if (!__all_sync(0xffffffffu, ok)) {
                ok = 0;
                fail_a = a;
                break;
            }
            // sample n = a + S p of the window (0 past it, as in the FP32 search's phases)
            const float *bp = buf0 + (size_t)cb * P * 32 + lane;
#pragma unroll 8
            for (int p = 0; p < P; ++p) {
                const int n = a + S * p;
                acc = fmaf(n < L ? rres[n] : 0.0f, bp[p * 32], acc);
            }
            __syncwarp();
        }
        if (!ok) {
            if (lane == 0) {
                atomicOr(status, kFlagTimeout);
                // bounded: let the copies in flight land before the warp leaves
                const int cb = fail_a & 1;
                mbar_drain(&bar[warp][cb], (uses[cb] - 1) & 1u);
                if (fail_a + 1 < Sa) mbar_drain(&bar[warp][cb ^ 1], uses[cb ^ 1] & 1u);
            }
            return;
        }
        const int t = tb * 32 + lane;
        unsigned long long key = 0ull;
        if (t < T) {
            const float sv = acc * scale[((size_t)tb * NtcP + j) * 32 + lane];
            const float x = fabsf(sv);
            if (x == x) key = pack_key(x, (uint32_t)j * (uint32_t)T + (uint32_t)t);
        }
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, key, off);
            key = o > key ? o : key;
        }
        if (lane == 0 && key) atomicMax(keys + b, key);
    }
}

// static shared memory of the kernels here (the GEMM's Smem is the largest)
constexpr int kStaticReserve = 6144;
static_assert(sizeof(Smem) + 256 <= kStaticReserve, "static shared memory above its reserve");
constexpr int kSmemBudget = 232448 - kStaticReserve - 1024;

}  // namespace

struct ShiftTc {
    CUtensorMap mapB[2];    // box heights 128 and 256
    int nkc = 0, sm_count = 0, T_pad = 0;
    int pair_clusters = 0;  // co-resident CTA pairs of the paired GEMM (0: not available)
    int rescan_warps = 0, rescan_blocks_per_sm = 0;
    size_t rescan_smem = 0;
};

cudaError_t shift_tc_prepare(ShiftTc **out, const ShiftPlan &sp, int sm_count) {
    *out = nullptr;
    if (!sp.tpl16 || sp.Kt < kBK || sp.Kt % kBK != 0) return cudaErrorNotSupported;
    ShiftTc *s = new (std::nothrow) ShiftTc();
    if (!s) return cudaErrorMemoryAllocation;
    s->nkc = sp.Kt / kBK;
    s->T_pad = sp.T_pad;
    s->sm_count = sm_count;
    const uint64_t rows = (uint64_t)(sp.T_pad / kBlockRows) * s->nkc * kBlockRows;
    if (rows >= ((uint64_t)1 << 31) || !make_map(&s->mapB[0], sp.tpl16, (uint64_t)kBK, rows, 128) ||
        !make_map(&s->mapB[1], sp.tpl16, (uint64_t)kBK, rows, 256)) {
        delete s;
        return cudaErrorNotSupported;
    }
    const void *gemms[3] = {(const void *)k_shift_gemm<128, false>, (const void *)k_shift_gemm<256, false>,
                            (const void *)k_shift_gemm<256, true>};
    const int stage_bytes[3] = {ShiftTile<128>::kStageBytes, ShiftTile<256>::kStageBytes,
                                ShiftTile<256, true>::kStageBytes};
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = allow_max_smem(gemms[i], 1024 + 2 * (size_t)stage_bytes[i]);
    if (e == cudaSuccess) e = allow_max_smem((const void *)k_shift_rows, 0);
    if (e == cudaSuccess) {
        // how many CTA pairs fit at once with the largest launch's shared memory
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(2 * (unsigned)sm_count);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = 1024 + (size_t)kSmemBudget;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, k_shift_gemm<256, true>, &cfg) != cudaSuccess) {
            cudaGetLastError();
            clusters = 0;
        }
        s->pair_clusters = clusters;
    }
    // rescore: per warp the residual and two P-row buffers; as many warps per
    // block (up to kRescanWarps) as fit
    const size_t per_warp = sizeof(float) * ((size_t)sp.Lp + 2 * (size_t)sp.P * 32);
    int rw = kRescanWarps;
    while (rw > 1 && rw * per_warp > (size_t)kSmemBudget) --rw;
    s->rescan_warps = rw;
    s->rescan_smem = rw * per_warp;
    if (e == cudaSuccess && s->rescan_smem > (size_t)kSmemBudget) e = cudaErrorNotSupported;
    if (e == cudaSuccess) e = allow_max_smem((const void *)k_shift_rescan, s->rescan_smem);
    if (e == cudaSuccess) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_shift_rescan, rw * 32, s->rescan_smem);
        s->rescan_blocks_per_sm = per_sm < 1 ? 1 : per_sm;
    }
    if (e != cudaSuccess) {
        delete s;
        return e;
    }
    *out = s;
    return cudaSuccess;
}

void shift_tc_free(ShiftTc *s) { delete s; }

void shift_tc_scratch_free(ShiftTcScratch &x) {
    if (x.tile_max) cudaFree(x.tile_max);
    if (x.blk_max) cudaFree(x.blk_max);
    if (x.items) cudaFree(x.items);
    if (x.X) cudaFree(x.X);
    if (x.chan_norm) cudaFree(x.chan_norm);
    if (x.chmax) cudaFree(x.chmax);
    if (x.chcount) cudaFree(x.chcount);
    x = ShiftTcScratch();
}

// Row tiling for B channels: Bg channels x Jt time centres per 128-row tile,
// Jt as small as B allows (fewer lag chunks per tile), at most the time
// centres (rounded up to a power of two).
static RowTiling make_tiling(const ShiftPlan &sp, int B) {
    RowTiling t;
    int bg = 1;
    while (bg < B && bg < 32) bg <<= 1;
    int ntc2 = 1;
    while (ntc2 < sp.Ntc) ntc2 <<= 1;
    t.Jt = kBM / bg < ntc2 ? kBM / bg : ntc2;
    t.Bg = kBM / t.Jt;
    t.B = B;
    t.Ntc = sp.Ntc;
    t.n_cb = (B + t.Bg - 1) / t.Bg;
    t.m_tiles = ((sp.Ntc + t.Jt - 1) / t.Jt) * t.n_cb;
    t.S = sp.S;
    t.L = sp.L;
    t.span0 = -sp.m_lo - sp.tc0;
    return t;
}

// Buffers for B channels (kept when large enough).
cudaError_t shift_tc_reserve(const ShiftTc *s, const ShiftPlan &sp, int B, ShiftTcScratch &x) {
    (void)s;
    if (B <= x.B_cap) return cudaSuccess;
    shift_tc_scratch_free(x);
    const int64_t rows = (int64_t)B * sp.Ntc;
    int64_t rows_alloc = 0;  // the largest row-tile count of any B' <= B
    for (int b2 = 1; b2 <= B; ++b2) {
        const int64_t r2 = (int64_t)make_tiling(sp, b2).m_tiles * kBM;
        rows_alloc = r2 > rows_alloc ? r2 : rows_alloc;
    }
    if (rows_alloc > (1ll << 30)) return cudaErrorInvalidValue;
    cudaError_t e = dev_alloc((void **)&x.tile_max, sizeof(float) * (size_t)rows * (sp.T_pad / 128));
    if (e == cudaSuccess) e = dev_alloc((void **)&x.blk_max, sizeof(float) * (size_t)rows * (sp.T_pad / 32));
    if (e == cudaSuccess) e = dev_alloc((void **)&x.items, sizeof(int) * 2 * (size_t)B * kMaxItems);
    if (e == cudaSuccess) e = dev_alloc((void **)&x.X, sizeof(__nv_bfloat16) * (size_t)rows_alloc * sp.Kt);
    if (e == cudaSuccess) e = cudaMemset(x.X, 0, sizeof(__nv_bfloat16) * (size_t)rows_alloc * sp.Kt);
    if (e == cudaSuccess) e = dev_alloc((void **)&x.chan_norm, sizeof(double2) * (size_t)B);
    if (e == cudaSuccess) e = dev_alloc((void **)&x.chmax, sizeof(unsigned int) * (size_t)B);
    if (e == cudaSuccess) e = dev_alloc((void **)&x.chcount, sizeof(int) * (size_t)B);
    if (e != cudaSuccess) {
        cudaGetLastError();
        shift_tc_scratch_free(x);
        return cudaErrorMemoryAllocation;
    }
    x.B_cap = B;
    x.rows_alloc = (int)rows_alloc;
    return cudaSuccess;
}

// GEMM form of a B-channel launch: the template tile width (256 unless that
// leaves SMs idle or leaves room for fewer than two stages beside the tile's
// scale rows) and whether CTA pairs share each MMA (256-wide tiles, at least
// two row tiles, a work unit for every pair that fits, pairs allowed).
static int shift_tc_bn(const ShiftTc *s, const ShiftPlan &sp, const RowTiling &tl, bool pairs_allowed, int *stages,
                       size_t *smem, bool *pair) {
    auto smem_for = [&](int bn, int stage_bytes, int *stg_out) {
        const size_t sc = (size_t)tl.Jt * (bn + 4) * sizeof(float);
        int stg = (int)((kSmemBudget - (int64_t)sc) / stage_bytes);
        stg = stg > kMaxStages ? kMaxStages : stg;
        *stg_out = stg;
        return 1024 + (size_t)stg * stage_bytes + sc;
    };
    *pair = false;
    int st256 = 0;
    const size_t sm256 = smem_for(256, ShiftTile<256>::kStageBytes, &st256);
    if ((int64_t)tl.m_tiles * (sp.T_pad / 256) >= s->sm_count && st256 >= 2) {
        int stp = 0;
        const size_t smp = smem_for(256, ShiftTile<256, true>::kStageBytes, &stp);
        const int64_t units = (int64_t)((tl.m_tiles + 1) / 2) * (sp.T_pad / 256);
        if (pairs_allowed && s->pair_clusters > 0 && tl.m_tiles >= 2 && units >= s->pair_clusters && stp >= 2) {
            // the whole budget: every operand read of a stage's MMAs stays
            // inside the allocation even at the last stage
            static_assert((kMaxStages - 1) * ShiftTile<256, true>::kStageBytes + 48 * 1024 <= kSmemBudget,
                          "paired stages beyond the shared-memory budget");
            (void)smp;
            *pair = true;
            *stages = stp;
            *smem = 1024 + (size_t)kSmemBudget;
            return 256;
        }
        *stages = st256;
        *smem = sm256;
        return 256;
    }
    *smem = smem_for(128, ShiftTile<128>::kStageBytes, stages);
    return 128;
}

bool shift_tc_uses_pairs(const ShiftTc *s, const ShiftPlan &sp, int B, bool pairs_allowed) {
    if (!s || B < 1) return false;
    int stages = 0;
    size_t smem = 0;
    bool pair = false;
    shift_tc_bn(s, sp, make_tiling(sp, B), pairs_allowed, &stages, &smem, &pair);
    return pair;
}

cudaError_t launch_shift_tc_gemm(const ShiftTc *s, const ShiftTcScratch &x, const ShiftPlan &sp, const float *R,
                                 int Lp, int L, int B, long long *stats, int *status, cudaStream_t st, bool pdl,
                                 unsigned long long wait_ns, bool pairs_allowed) {
    if (!s || B < 1 || B > x.B_cap) return cudaErrorInvalidValue;
    const RowTiling tl = make_tiling(sp, B);
    // rows per block: up to 16, fewer when that leaves SMs idle (at least 4);
    // lag segments keep the 8 staged copies within 64 KB of shared memory
    int RJ = (int)(((int64_t)B * sp.Ntc + 2 * s->sm_count - 1) / (2 * s->sm_count));
    RJ = RJ < 4 ? 4 : (RJ > 16 ? 16 : RJ);
    constexpr int kRowsSmemSamples = 65536 / 18;  // samples per copy in 64 KB of 8 BF16 copies + the plain one
    while (RJ > 1 && sp.S * (RJ - 1) + 8 + 64 > kRowsSmemSamples) --RJ;
    int KSEG = sp.Kt;
    if (sp.S * (RJ - 1) + 8 + KSEG > kRowsSmemSamples) KSEG = (kRowsSmemSamples - 8 - sp.S * (RJ - 1)) / 64 * 64;
    if (KSEG < 64) return cudaErrorInvalidValue;
    const int n_seg = (sp.Kt + KSEG - 1) / KSEG;
    const int span_pad = (sp.S * (RJ - 1) + KSEG + 7) & ~7;
    const size_t rows_smem = ((size_t)9 * span_pad + 8) * sizeof(__nv_bfloat16);
    const int64_t gx = (int64_t)((sp.Ntc + RJ - 1) / RJ) * n_seg;
    if (gx >= ((int64_t)1 << 31) || B > 65535) return cudaErrorInvalidValue;
    cudaError_t e = launch_kernel(k_shift_rows, dim3((unsigned)gx, B), dim3(256), rows_smem, st, pdl, tl, R, Lp,
                                  sp.tc0, sp.m_lo, sp.Kt, RJ, KSEG, n_seg, span_pad, x.X, x.chan_norm, x.chmax,
                                  x.chcount, stats);
    if (e != cudaSuccess) return e;
    const int m_tiles = tl.m_tiles;
    CUtensorMap mapA;
    if (!make_map(&mapA, x.X, (uint64_t)sp.Kt, (uint64_t)m_tiles * kBM, kBM)) return cudaErrorInvalidValue;
    int stages = 0;
    size_t smem = 0;
    bool pair = false;
    const int bn = shift_tc_bn(s, sp, tl, pairs_allowed, &stages, &smem, &pair);
    const int n_tiles = sp.T_pad / bn;
    if (stages < 2) return cudaErrorInvalidValue;
    if (pair) {
        // clusters of 2: each CTA loads 128-template halves (box height 128)
        const int64_t units = (int64_t)((m_tiles + 1) / 2) * n_tiles;
        const int pairs = (int)(units < s->pair_clusters ? units : s->pair_clusters);
        return launch_kernel_cluster(k_shift_gemm<256, true>, dim3(2 * pairs), dim3(kThreads), smem, st, true, 2, mapA,
                                     s->mapB[0], tl, n_tiles, s->nkc, stages, sp.T_pad, sp.scaleT, x.tile_max,
                                     x.blk_max, x.chmax, status, wait_ns);
    }
    const int i = bn == 256 ? 1 : 0;
    const int64_t items = (int64_t)m_tiles * n_tiles;
    const int grid = (int)(items < s->sm_count ? items : s->sm_count);
    // a programmatic dependent of the shifted-row build (set-up overlaps it)
    return launch_kernel(bn == 256 ? k_shift_gemm<256, false> : k_shift_gemm<128, false>, dim3(grid), dim3(kThreads),
                         smem, st, true, mapA, s->mapB[i], tl, n_tiles, s->nkc, stages, sp.T_pad, sp.scaleT,
                         x.tile_max, x.blk_max, x.chmax, status, wait_ns);
}

cudaError_t launch_shift_tc_resolve(const ShiftTc *s, const ShiftTcScratch &x, const ShiftPlan &sp, const float *R,
                                    int Lp, int L, int B, unsigned long long *keys, int *fb_list, int *counters,
                                    long long *stats, int *status, cudaStream_t st, bool pdl,
                                    unsigned long long wait_ns) {
    if (!s || B < 1 || B > x.B_cap) return cudaErrorInvalidValue;
    const RowTiling tl = make_tiling(sp, B);
    int stages = 0;
    size_t smem = 0;
    bool pair = false;
    const int bn = shift_tc_bn(s, sp, tl, false, &stages, &smem, &pair);  // the GEMM's tile width for B channels
    const int n_tiles = sp.T_pad / bn;
    const int entries = sp.Ntc * n_tiles;
    int slices = (entries + 255) / 256;
    const int max_slices = (4 * s->sm_count + B - 1) / B;
    if (slices > max_slices) slices = max_slices;
    cudaError_t e = launch_kernel(k_shift_flag, dim3(slices, B), dim3(256), 0, st, pdl, sp.Ntc, n_tiles, bn / 32,
                                  sp.Kt, L, (const float *)x.tile_max, (const float *)x.blk_max,
                                  (const double2 *)x.chan_norm, (const unsigned int *)x.chmax,
                                  (const unsigned int *)sp.eps_bits, x.chcount, fb_list, counters, x.items, stats);
    if (e != cudaSuccess) return e;
    e = launch_kernel(k_shift_rescan, dim3(s->sm_count * s->rescan_blocks_per_sm), dim3(s->rescan_warps * 32),
                      s->rescan_smem, st, true, (const float *)sp.tpl, (const float *)sp.scale, sp.S, sp.Sa, sp.P,
                      sp.rows, sp.NtcP, sp.Ntc, sp.T, sp.T_pad / 32, Lp, L, R, (const int *)x.items,
                      (const int *)counters, keys, status, wait_ns);
    if (e != cudaSuccess) return e;
    // channels with more than kMaxItems flagged items: the FP32 template
    // search over the queue, launched early (its CTAs become resident while
    // the rescore runs and read the queue after it; an empty queue leaves
    // them idle)
    return launch_shift_search(sp, R, Lp, L, B, keys, nullptr, status, true, st, fb_list, &counters[0], wait_ns);
}


}  // namespace act
