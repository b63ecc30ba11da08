// LEM-inspired hierarchical coarse-to-fine search (Sec. VII-A, Fig. 7), with
// no stored dictionary: per channel and order,
//   1. a Latin hypercube sample of n_coarse parameter vectors over the grid's
//      box (strata ranked by SplitMix64 keys, uniform offsets inside them);
//   2. every candidate atom generated on the fly and projected onto the
//      residual; the top_k by |score| kept (lowest candidate index on ties,
//      duplicate parameter vectors skipped);
//   3. per refinement level, the local neighbourhood dictionary of each kept
//      candidate (offsets -R..R steps of that level per axis, clamped to the
//      box), all candidates pooled, projected and reranked to a new top_k;
//   4. the best candidate then starts the BFGS refinement (act_refine.cu).
// The random draws come from SplitMix64 (Steele, Lea and Flood, 2014): draw
// n of a stream seeded s is mix(s + (n + 1) 0x9E3779B97F4A7C15), with n
// packing (channel, order, axis, kind, sample).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "act_device.cuh"
#include "act_ff.cuh"
#include "act_internal.cuh"

namespace act {

namespace {

constexpr int kLemThreads = 256;

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t n) {
    uint64_t z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t lem_counter(int channel, int order, int axis, int kind, int i) {
    return (((((((uint64_t)channel << 12) | (uint64_t)order) << 2 | (uint64_t)axis) << 1) | (uint64_t)kind) << 20) |
           (uint64_t)i;
}

// 1. Latin hypercube: one block per (channel, axis); keys sorted in shared
// memory (bitonic sort over npow2 >= n entries, padding keys sort last).
__global__ void __launch_bounds__(kLemThreads) k_lem_lhs(int n, int npow2, LemBox box, uint64_t seed, int order,
                                                        int cap, double *__restrict__ cand, int *__restrict__ ncand) {
    extern __shared__ uint8_t sm_raw[];
    uint64_t *key = reinterpret_cast<uint64_t *>(sm_raw);
    uint32_t *idx = reinterpret_cast<uint32_t *>(key + npow2);
    const int b = blockIdx.x, a = blockIdx.y;
    double *out = cand + (size_t)b * cap * 4;
    for (int i = threadIdx.x; i < npow2; i += blockDim.x) {
        key[i] = i < n ? splitmix64_at(seed, lem_counter(b, order, a, 0, i)) : ~0ull;
        idx[i] = (uint32_t)i;
    }
    __syncthreads();
    for (int size = 2; size <= npow2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < npow2; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const uint64_t ki = key[i], kj = key[j];
                    if ((ki > kj) == up) {
                        key[i] = kj;
                        key[j] = ki;
                        const uint32_t t = idx[i];
                        idx[i] = idx[j];
                        idx[j] = t;
                    }
                }
            }
            __syncthreads();
        }
    }
    // sorted position p is the stratum (rank) of sample idx[p].  For n a
    // power of two the quotient (p + u) / n is the exact product with 2^-k:
    // the same correctly rounded value without an FP64 division
    const bool pow2 = (n & (n - 1)) == 0;
    const double inv_n = pow2 ? __longlong_as_double((long long)(1023 - (31 - __clz(n))) << 52) : 0.0;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const int i = (int)idx[p];
        const uint64_t h = splitmix64_at(seed, lem_counter(b, order, a, 1, i));
        const double u = (double)(h >> 11) * 0x1.0p-53;
        const double q = __dadd_rn((double)p, u);
        const double t = pow2 ? __dmul_rn(q, inv_n) : __ddiv_rn(q, (double)n);
        out[4 * i + a] = __dadd_rn(box.lo[a], __dmul_rn(t, __dadd_rn(box.hi[a], -box.lo[a])));
    }
    if (threadIdx.x == 0 && a == 0) ncand[b] = n;
}

// 2. Scores s = <r, u>/|u| of every candidate of every channel.  A block
// takes kScoreCands candidates of one channel: their per-atom constants are
// formed once (FP64, one thread per candidate), then each warp runs its
// candidates one after another, lane = sample stride 32.  A lane's samples
// n_k = lane + 32 k advance tau by D = 32 / fs, so the phase
// (c tau + fc) tau steps by d1_k = D (c (2 tau_k + D) + fc), and d1 by
// d2 = 2 c D^2: tau, the phase and d1 are carried by these recurrences in
// float-float (phase and d1 mod 1), from exact starting values at k = 0.
// The samples are FP32 from the same expressions as the dictionary
// generator's; products are summed in FP32 over 4 samples, then into
// float-float sums.
constexpr int kScoreCands = 64;  // at most 32 per warp (one lane each)

struct LemConst {
    ChirpFF k;
    ff D, d2;  // the lane stride in tau and the second difference of the phase (mod 1)
};

__global__ void __launch_bounds__(kLemThreads) k_lem_score(int cap, const double *__restrict__ cand,
                                                          const int *__restrict__ ncand, const float *__restrict__ R,
                                                          int Lp, int L, double inv_fs, double *__restrict__ score) {
    __shared__ LemConst ks[kScoreCands];
    const int b = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i0 = blockIdx.x * kScoreCands;
    const int n_here = min(kScoreCands, ncand[b] - i0);
    if (n_here <= 0) return;
    if (threadIdx.x < n_here) {
        const double *th = cand + ((size_t)b * cap + i0 + threadIdx.x) * 4;
        const double D = 32.0 * inv_fs;
        double d2 = 2.0 * th[3] * D * D;
        d2 -= rint(d2);
        ks[threadIdx.x] = {chirp_ff(th[0], inv_fs, th[1], th[3], exp(-th[2])), ff_from_double(D),
                           ff_from_double(d2)};
    }
    __syncthreads();
    const float *r = R + (size_t)b * Lp;
    // lane i keeps the sums of the warp's i-th candidate; the FP64 finish
    // then runs once for all of them (an FP64 instruction costs the same
    // pipe time however few lanes are active)
    constexpr int kWarps = kLemThreads / 32;
    ff my_ru = {0.0f, 0.0f}, my_uu = {0.0f, 0.0f};
    int i = 0;
    for (int q = warp; q < n_here; q += kWarps, ++i) {
        const LemConst kc = ks[q];
        const ChirpFF &k = kc.k;
        // k = 0: tau, the phase and its first difference, formed directly
        ff tau;
        ff ph = chirp_phase_pair(lane, k, &tau);
        const ff two_tau_d = ff_add({2.0f * tau.hi, 2.0f * tau.lo}, kc.D);
        ff d1 = ff_frac(ff_mul(ff_add(ff_mul(k.c, two_tau_d), k.fc), kc.D));
        ff ru = {0.0f, 0.0f}, uu = {0.0f, 0.0f};
        for (int n0 = lane; n0 < L; n0 += 128) {
            float pr = 0.0f, pu = 0.0f;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int n = n0 + 32 * e;
                if (n < L) {
                    const float x = chirp_x_ff(tau, k);
                    const float u = expf(-0.5f * x * x) * cospif(2.0f * (ph.hi + ph.lo));
                    pr = fmaf(__ldg(r + n), u, pr);
                    pu = fmaf(u, u, pu);
                    tau = ff_add_sloppy(tau, kc.D);
                    ph = ff_frac(ff_add_sloppy(ph, d1));
                    d1 = ff_frac(ff_add_sloppy(d1, kc.d2));
                }
            }
            ru = ff_add_f(ru, pr);
            uu = ff_add_f(uu, pu);
        }
        ru = ff_warp_sum(ru);
        uu = ff_warp_sum(uu);
        if (lane == i) {
            my_ru = ru;
            my_uu = uu;
        }
    }
    if (lane < i) {
        const double e = ff_to_double(my_uu);
        score[(size_t)b * cap + i0 + warp + lane * kWarps] = (e > 0.0 && isfinite(e)) ? ff_to_double(my_ru) / sqrt(e) : 0.0;
    }
}

// 3. Top-k by |score| with duplicates skipped: one block per channel, k
// rounds of a block-wide arg-max (largest |score|, then lowest index).  The
// compares run on the bit patterns (integer pipes; FP64 compares are slow
// on this GPU): for finite non-negative doubles the patterns order as the
// values, NaN scores are skipped, and two parameters are equal when their
// patterns are, or both are zeros.
__device__ __forceinline__ bool same_value(unsigned long long a, unsigned long long b) {
    return a == b || ((a | b) << 1) == 0ull;
}

__global__ void __launch_bounds__(kLemThreads) k_lem_topk(int cap, int k, const double *__restrict__ cand,
                                                         const int *__restrict__ ncand,
                                                         const double *__restrict__ score, double *__restrict__ kept,
                                                         double *__restrict__ kept_score, int *__restrict__ nkept) {
    constexpr unsigned long long kAbs = 0x7fffffffffffffffull, kInf = 0x7ff0000000000000ull;
    __shared__ unsigned long long kt[16][4];
    __shared__ unsigned long long bv_s[kLemThreads / 32];
    __shared__ int bi_s[kLemThreads / 32];
    __shared__ int m_sh;
    const int b = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = ncand[b];
    const unsigned long long *cb = reinterpret_cast<const unsigned long long *>(cand) + (size_t)b * cap * 4;
    const unsigned long long *sb = reinterpret_cast<const unsigned long long *>(score) + (size_t)b * cap;
    if (threadIdx.x == 0) m_sh = 0;
    __syncthreads();
    for (int round = 0; round < k; ++round) {
        const int m = m_sh;
        unsigned long long bv = 0ull;
        int bi = -1;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const unsigned long long v = sb[i] & kAbs;
            if (v > kInf || (bi >= 0 && v <= bv)) continue;  // NaN, or not above the best (the first index wins ties)
            bool dup = false;
            for (int q = 0; q < m && !dup; ++q)
                dup = same_value(cb[4 * i], kt[q][0]) && same_value(cb[4 * i + 1], kt[q][1]) &&
                      same_value(cb[4 * i + 2], kt[q][2]) && same_value(cb[4 * i + 3], kt[q][3]);
            if (!dup) {
                bv = v;
                bi = i;
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long ov = __shfl_xor_sync(0xffffffffu, bv, off);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (oi >= 0 && (bi < 0 || ov > bv || (ov == bv && oi < bi))) {
                bv = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            bv_s[warp] = bv;
            bi_s[warp] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long v = 0ull;
            int id = -1;
            for (int w = 0; w < kLemThreads / 32; ++w)
                if (bi_s[w] >= 0 && (id < 0 || bv_s[w] > v || (bv_s[w] == v && bi_s[w] < id))) {
                    v = bv_s[w];
                    id = bi_s[w];
                }
            if (id >= 0) {
                for (int a = 0; a < 4; ++a) kt[m][a] = cb[4 * id + a];
                kept_score[(size_t)b * k + m] = score[(size_t)b * cap + id];
                for (int a = 0; a < 4; ++a) kept[((size_t)b * k + m) * 4 + a] = cand[((size_t)b * cap + id) * 4 + a];
                m_sh = m + 1;
            }
        }
        __syncthreads();
        if (m_sh == m) break;  // nothing left
    }
    if (threadIdx.x == 0) nkept[b] = m_sh;
}

// 4. Neighbourhood dictionaries of the kept candidates for one level.
__global__ void __launch_bounds__(kLemThreads) k_lem_neigh(int cap, int k, LemBox box, LemLevel lev,
                                                          const double *__restrict__ kept,
                                                          const int *__restrict__ nkept, double *__restrict__ cand,
                                                          int *__restrict__ ncand) {
    const int b = blockIdx.x;
    const int m = nkept[b];
    int w[4], per = 1;
    for (int a = 0; a < 4; ++a) {
        w[a] = 2 * lev.radius[a] + 1;
        per *= w[a];
    }
    const int total = m * per;
    double *out = cand + (size_t)b * cap * 4;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int j = t / per;
        int rest = t % per;
        int o[4];
        for (int a = 3; a >= 0; --a) {
            o[a] = rest % w[a] - lev.radius[a];
            rest /= w[a];
        }
        for (int a = 0; a < 4; ++a) {
            double v = __dadd_rn(kept[((size_t)b * k + j) * 4 + a], __dmul_rn((double)o[a], lev.step[a]));
            v = v < box.lo[a] ? box.lo[a] : (v > box.hi[a] ? box.hi[a] : v);
            out[4 * t + a] = v;
        }
    }
    if (threadIdx.x == 0) ncand[b] = total;
}

}  // namespace

cudaError_t launch_lem_select(const LemConfig &cfg, int B, int order, const float *R, int Lp, int L, double fs,
                              const LemBuffers &lb, cudaStream_t st) {
    int npow2 = 1;
    while (npow2 < cfg.n_coarse) npow2 <<= 1;
    const size_t smem = (size_t)npow2 * (sizeof(uint64_t) + sizeof(uint32_t));
    if (smem > 48 * 1024) {
        cudaError_t ea = cudaFuncSetAttribute(k_lem_lhs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (ea != cudaSuccess) return ea;
    }
    k_lem_lhs<<<dim3(B, 4), kLemThreads, smem, st>>>(cfg.n_coarse, npow2, cfg.box, cfg.seed, order, lb.cap, lb.cand, lb.ncand);
    cudaError_t e = cudaGetLastError();
    const double inv_fs = 1.0 / fs;
    int n = cfg.n_coarse;
    for (int lev = 0; lev <= cfg.levels && e == cudaSuccess; ++lev) {
        if (lev > 0) {
            k_lem_neigh<<<B, kLemThreads, 0, st>>>(lb.cap, cfg.top_k, cfg.box, cfg.level[lev], lb.kept, lb.nkept,
                                                   lb.cand, lb.ncand);
            e = cudaGetLastError();
            int per = 1;
            for (int a = 0; a < 4; ++a) per *= 2 * cfg.level[lev].radius[a] + 1;
            n = cfg.top_k * per;
        }
        if (e != cudaSuccess) break;
        dim3 grid((n + kScoreCands - 1) / kScoreCands, B);
        k_lem_score<<<grid, kLemThreads, 0, st>>>(lb.cap, lb.cand, lb.ncand, R, Lp, L, inv_fs, lb.score);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        k_lem_topk<<<B, kLemThreads, 0, st>>>(lb.cap, cfg.top_k, lb.cand, lb.ncand, lb.score, lb.kept, lb.kept_score,
                                              lb.nkept);
        e = cudaGetLastError();
    }
    return e;
}

int lem_kernels(const LemConfig &cfg) { return 1 + 2 + 3 * cfg.levels; }

}  // namespace act
