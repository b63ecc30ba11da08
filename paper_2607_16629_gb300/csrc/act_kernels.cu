// CUDA kernels of the FP32 path: atom generation (Eq. (1) real part with
// unit l2 norm, Sec. III-A), residual initialisation, the HBM-bound GEMV
// with the argmax of |<g_i, r>| fused (Sec. III-A, Sec. IV-A) and the
// coefficient / residual update of Eq. (4).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "act_device.cuh"
#include "act_internal.cuh"

namespace act {

// ---------------------------------------------------------------------------
// Atom generation
// ---------------------------------------------------------------------------
// One warp per atom.  Lane l owns samples 4*(l + 32 j) + e, e = 0..3, so the
// FP32 row is written with 128-bit stores.  The BF16 copy is written
// tile-major, [atom / 256][sample / 64][atom % 256][sample % 64], so that one
// 256-atom x 64-sample operand tile of the tensor-core search is a single
// contiguous 32 KB block.  The phase of Eq. (1), in cycles,
// phi = c tau^2 + fc tau with tau = (n - tc) / fs, is evaluated in FP64 and
// reduced to [-1/2, 1/2] before the FP32 cospi; the Gaussian exponent is
// formed in FP64 and exponentiated in FP32; the squared norm is summed in
// FP64.  An atom whose FP32 samples are all zero (or not finite) is
// degenerate: its row is stored as zeros and it scores 0.
template <int NV>
__global__ void __launch_bounds__(256) k_gen_atoms(GridAxes ax, int64_t K, int Lp, float *__restrict__ d32,
                                                    __nv_bfloat16 *__restrict__ d16, int Lb,
                                                    unsigned long long *__restrict__ degenerate,
                                                    unsigned int *__restrict__ eps_bits) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double inv_fs = 1.0 / ax.fs;
    for (int64_t atom = warp; atom < K; atom += nwarps) {
        double p[4];
        decode_params(ax, atom, p);
        const double tc = p[0], fc = p[1], chirp = p[3];
        const double inv_dt = exp(-p[2]);
        float u[NV][4];
        double energy = 0.0;
#pragma unroll
        for (int j = 0; j < NV; ++j) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int n = 4 * (lane + 32 * j) + e;
                float v = 0.0f;
                if (n < ax.L) {
                    const double tau = ((double)n - tc) * inv_fs;
                    double ph = fma(chirp, tau, fc) * tau;
                    ph -= rint(ph);
                    const float x = (float)(tau * inv_dt);
                    v = expf(-0.5f * x * x) * cospif(2.0f * (float)ph);
                }
                u[j][e] = v;
                energy = fma((double)v, (double)v, energy);
            }
        }
        energy = warp_sum(energy);
        float scale = 0.0f;
        const bool bad = !(energy > 0.0) || !isfinite(energy);
        if (!bad) scale = (float)(1.0 / sqrt(energy));
        if (bad && lane == 0 && degenerate) atomicAdd(degenerate, 1ull);
        float4 *row = reinterpret_cast<float4 *>(d32 + atom * (int64_t)Lp);
        double err = 0.0;  // |bf16(g) - g|^2 of this atom (BF16 layout only)
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            float4 w = make_float4(u[j][0] * scale, u[j][1] * scale, u[j][2] * scale, u[j][3] * scale);
            row[lane + 32 * j] = w;
            if (d16) {
                const int n0 = 4 * (lane + 32 * j);
                if (n0 < Lb) {
                    __nv_bfloat162 lo = __floats2bfloat162_rn(w.x, w.y);
                    __nv_bfloat162 hi = __floats2bfloat162_rn(w.z, w.w);
                    const float2 flo = __bfloat1622float2(lo), fhi = __bfloat1622float2(hi);
                    err += (double)(flo.x - w.x) * (flo.x - w.x) + (double)(flo.y - w.y) * (flo.y - w.y) +
                           (double)(fhi.x - w.z) * (fhi.x - w.z) + (double)(fhi.y - w.w) * (fhi.y - w.w);
                    uint2 packed;
                    packed.x = *reinterpret_cast<uint32_t *>(&lo);
                    packed.y = *reinterpret_cast<uint32_t *>(&hi);
                    // tile-major: [atom / 256][n0 / 64][atom % 256][n0 % 64]
                    const int64_t off = (((atom >> 8) * (Lb >> 6) + (n0 >> 6)) * 256 + (atom & 255)) * 64 + (n0 & 63);
                    *reinterpret_cast<uint2 *>(d16 + off) = packed;
                }
            }
        }
        if (d16 && eps_bits) {
            err = warp_sum(err);
            // positive floats order like their bit patterns; round the norm up
            if (lane == 0) atomicMax(eps_bits, __float_as_uint(__double2float_ru(sqrt(err) * (1.0 + 1e-6))));
        }
    }
}

cudaError_t launch_gen_atoms(const GridAxes &ax, int64_t K, int Lp, float *d32, __nv_bfloat16 *d16, int Lb,
                             unsigned long long *degenerate, unsigned int *eps_bits, int sm_count, cudaStream_t st) {
    const int nv = Lp / 128;
    int64_t blocks = (K + 7) / 8;
    const int64_t cap = (int64_t)sm_count * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    switch (nv) {
        case 1: k_gen_atoms<1><<<(int)blocks, 256, 0, st>>>(ax, K, Lp, d32, d16, Lb, degenerate, eps_bits); break;
        case 2: k_gen_atoms<2><<<(int)blocks, 256, 0, st>>>(ax, K, Lp, d32, d16, Lb, degenerate, eps_bits); break;
        case 3: k_gen_atoms<3><<<(int)blocks, 256, 0, st>>>(ax, K, Lp, d32, d16, Lb, degenerate, eps_bits); break;
        case 4: k_gen_atoms<4><<<(int)blocks, 256, 0, st>>>(ax, K, Lp, d32, d16, Lb, degenerate, eps_bits); break;
        case 8: k_gen_atoms<8><<<(int)blocks, 256, 0, st>>>(ax, K, Lp, d32, d16, Lb, degenerate, eps_bits); break;
        case 16: k_gen_atoms<16><<<(int)blocks, 256, 0, st>>>(ax, K, Lp, d32, d16, Lb, degenerate, eps_bits); break;
        default: {
            // Row strides between the instantiated ones are rounded up by the host.
            return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Residual initialisation: r_0 = s (Eq. (4)), padded rows, |s|^2 in FP64,
// finiteness check, selection keys cleared.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kUpdateThreads) k_init(const float *__restrict__ sig, int L, int Lp,
                                                         float *__restrict__ R, __nv_bfloat16 *__restrict__ R16,
                                                         int Lb, unsigned long long *__restrict__ keys,
                                                         double *__restrict__ energy, int P1, int *status) {
    __shared__ double sh[32];
    const int b = blockIdx.x;
    double e = 0.0;
    int bad = 0;
    for (int n = threadIdx.x; n < Lp; n += blockDim.x) {
        float v = n < L ? sig[(int64_t)b * L + n] : 0.0f;
        if (!isfinite(v)) bad = 1;
        R[(int64_t)b * Lp + n] = v;
        e = fma((double)v, (double)v, e);
        if (R16 && n < Lb) R16[(int64_t)b * Lb + n] = __float2bfloat16_rn(v);
    }
    const double tot = block_sum(e, sh);
    if (bad) atomicOr(status, kFlagNonFinite);
    if (threadIdx.x == 0) {
        if (energy) energy[(int64_t)b * P1] = tot;
        if (keys) keys[b] = 0ull;
    }
}

cudaError_t launch_init(const float *sig, int B, int L, int Lp, float *R, __nv_bfloat16 *R16, int Lb,
                        unsigned long long *keys, double *energy, int P1, int *status, cudaStream_t st) {
    k_init<<<B, kUpdateThreads, 0, st>>>(sig, L, Lp, R, R16, Lb, keys, energy, P1, status);
    return cudaGetLastError();
}

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
                                                       float *__restrict__ scores, int *status) {
    extern __shared__ __align__(128) float smem_r[];  // NB * Lp floats
    __shared__ __align__(8) uint64_t bar;
    __shared__ float red_s[kGemvThreads / 32][NB];
    __shared__ uint32_t red_i[kGemvThreads / 32][NB];

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
        const int timed_out = mbar_wait(&bar, parity) ? 0 : 1;
        if (__syncthreads_or(timed_out)) {
            if (threadIdx.x == 0) atomicOr(status, kFlagTimeout);
            mbar_wait(&bar, parity);  // bounded: let an in-flight copy land before exiting
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
                                 int grid_ctas, cudaStream_t st) {
    const size_t smem = (size_t)NB * Lp * sizeof(float);
    k_gemv<NV, NB, WS><<<grid_ctas, kGemvThreads, smem, st>>>(D, K, Lp, R, B, chlist, count_dev, keys, scores,
                                                              status);
    return cudaGetLastError();
}

template <bool WS>
static cudaError_t gemv_dispatch(const float *D, int64_t K, int Lp, const float *R, int B, const int *chlist,
                                 const int *count_dev, unsigned long long *keys, float *scores, int *status,
                                 int grid_ctas, cudaStream_t st) {
    const int nv = Lp / 128;
    // Several channels per pass over D only when the count is known on the host.
    const bool multi = (count_dev == nullptr) && B >= 4 && nv <= 4;
#define ACT_GEMV_CASE(NVV)                                                                                 \
    case NVV:                                                                                              \
        return multi ? gemv_instance<NVV, 4, WS>(D, K, Lp, R, B, chlist, count_dev, keys, scores, status, \
                                                 grid_ctas, st)                                            \
                     : gemv_instance<NVV, 1, WS>(D, K, Lp, R, B, chlist, count_dev, keys, scores, status, \
                                                 grid_ctas, st);
    switch (nv) {
        ACT_GEMV_CASE(1)
        ACT_GEMV_CASE(2)
        ACT_GEMV_CASE(3)
        ACT_GEMV_CASE(4)
        case 8:
            return gemv_instance<8, 1, WS>(D, K, Lp, R, B, chlist, count_dev, keys, scores, status, grid_ctas, st);
        case 16:
            return gemv_instance<16, 1, WS>(D, K, Lp, R, B, chlist, count_dev, keys, scores, status, grid_ctas,
                                            st);
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
                               cudaStream_t st) {
    return gemv_dispatch<false>(D, K, Lp, R, B, chlist, count_dev, keys, nullptr, status, grid_ctas, st);
}

cudaError_t launch_project(const float *D, int64_t K, int Lp, const float *R, int B, float *scores, int *status,
                           int grid_ctas, cudaStream_t st) {
    return gemv_dispatch<true>(D, K, Lp, R, B, nullptr, nullptr, nullptr, scores, status, grid_ctas, st);
}

// ---------------------------------------------------------------------------
// Coefficient and residual update (Eq. (4), Fig. 1): one block per channel.
// c_k = <g*, r_k> in FP32, r_{k+1} = r_k - c_k g*, |r_{k+1}|^2 in FP64,
// the selected atom's parameters decoded from its flat index, the key
// cleared for the next order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kUpdateThreads) k_update(const float *__restrict__ D32, int Lp, int L,
                                                           float *__restrict__ R, __nv_bfloat16 *__restrict__ R16,
                                                           int Lb, unsigned long long *__restrict__ keys,
                                                           GridAxes ax, int k, int P,
                                                           act_atom *__restrict__ atoms, float *__restrict__ coefs,
                                                           double *__restrict__ energy, int *fb_count) {
    __shared__ float shf[32];
    __shared__ double shd[32];
    const int b = blockIdx.x;
    const unsigned long long key = keys[b];
    const uint32_t idx = key_index(key);
    const float *g = D32 + (int64_t)idx * Lp;
    float *r = R + (int64_t)b * Lp;

    float part = 0.0f;
    for (int n = threadIdx.x; n < L; n += blockDim.x) part = fmaf(g[n], r[n], part);
    const float c = block_sum(part, shf);

    double e = 0.0;
    for (int n = threadIdx.x; n < L; n += blockDim.x) {
        const float v = fmaf(-c, g[n], r[n]);
        r[n] = v;
        e = fma((double)v, (double)v, e);
        if (R16) R16[(int64_t)b * Lb + n] = __float2bfloat16_rn(v);
    }
    const double tot = block_sum(e, shd);
    if (threadIdx.x == 0) {
        double p[4];
        decode_params(ax, (int64_t)idx, p);
        act_atom a;
        a.tc = p[0];
        a.fc = p[1];
        a.logdt = p[2];
        a.c = p[3];
        a.flat_index = (int64_t)idx;
        atoms[(int64_t)b * P + k] = a;
        coefs[(int64_t)b * P + k] = c;
        energy[(int64_t)b * (P + 1) + k + 1] = tot;
        keys[b] = 0ull;
        if (fb_count && b == 0) {
            fb_count[0] = 0;  // channels queued for the FP32 full search
            fb_count[1] = 0;  // (channel, CTA) pairs queued for an FP32 rescan
        }
    }
}

cudaError_t launch_update(const float *D32, int Lp, int L, float *R, __nv_bfloat16 *R16, int Lb, int B,
                          unsigned long long *keys, const GridAxes &ax, int k, int P, act_atom *atoms, float *coefs,
                          double *energy, int *fb_count, cudaStream_t st) {
    k_update<<<B, kUpdateThreads, 0, st>>>(D32, Lp, L, R, R16, Lb, keys, ax, k, P, atoms, coefs, energy,
                                           fb_count);
    return cudaGetLastError();
}

}  // namespace act

namespace act {

// ---------------------------------------------------------------------------
// Uneven batches: one length group's signals are gathered from the
// concatenated input, and its outputs scattered back to the callers' channel
// order (one block per channel of the group).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_ragged_gather(const float *__restrict__ src,
                                                       const int64_t *__restrict__ src_off, int L,
                                                       float *__restrict__ dst) {
    const int b = blockIdx.x;
    const float *s = src + src_off[b];
    for (int n = threadIdx.x; n < L; n += blockDim.x) dst[(int64_t)b * L + n] = s[n];
}

__global__ void __launch_bounds__(256) k_ragged_scatter(int P, int L, int Lp, const int *__restrict__ chan,
                                                        const int64_t *__restrict__ dst_off,
                                                        const act_atom *__restrict__ atoms,
                                                        const float *__restrict__ coefs,
                                                        const double *__restrict__ energy,
                                                        const float *__restrict__ R, act_atom *__restrict__ out_atoms,
                                                        float *__restrict__ out_coefs, double *__restrict__ out_energy,
                                                        float *__restrict__ out_resid) {
    const int b = blockIdx.x;
    const int64_t c = chan[b];
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        out_atoms[c * P + k] = atoms[(int64_t)b * P + k];
        out_coefs[c * P + k] = coefs[(int64_t)b * P + k];
    }
    for (int k = threadIdx.x; k <= P; k += blockDim.x) out_energy[c * (P + 1) + k] = energy[(int64_t)b * (P + 1) + k];
    for (int n = threadIdx.x; n < L; n += blockDim.x) out_resid[dst_off[b] + n] = R[(int64_t)b * Lp + n];
}

cudaError_t launch_ragged_gather(const float *src, const int64_t *src_off, int B, int L, float *dst, cudaStream_t st) {
    k_ragged_gather<<<B, 256, 0, st>>>(src, src_off, L, dst);
    return cudaGetLastError();
}

cudaError_t launch_ragged_scatter(int B, int P, int L, int Lp, const int *chan, const int64_t *dst_off,
                                  const act_atom *atoms, const float *coefs, const double *energy, const float *R,
                                  act_atom *out_atoms, float *out_coefs, double *out_energy, float *out_resid,
                                  cudaStream_t st) {
    k_ragged_scatter<<<B, 256, 0, st>>>(P, L, Lp, chan, dst_off, atoms, coefs, energy, R, out_atoms, out_coefs,
                                        out_energy, out_resid);
    return cudaGetLastError();
}

}  // namespace act
