// Off-grid refinement of each order's selected chirplet (Fig. 1:
// theta* = argmax_theta |<g(theta), r_k>| started from the grid winner) and
// the adjoint of the chirplet score used for it.
//
// Score and adjoint.  For the unit-norm real atom of Eq. (1) at continuous
// theta = (tc, fc, logDt, c), with u = E cos(phi), E = exp(-x^2/2),
// x = tau/Dt, phi = 2 pi (c tau^2 + fc tau), tau = (n - tc)/fs, g = u/|u|:
//   s = <r, u>/|u|,  ds/dr = g,
//   ds/dtheta_i = <r, du_i>/|u| - s <u, du_i>/|u|^2 with
//   du/dtc = (E x/Dt cos(phi) + E sin(phi) 2 pi (2 c tau + fc)) / fs,
//   du/dfc = -E sin(phi) 2 pi tau,  du/dlogDt = E x^2 cos(phi),
//   du/dc  = -E sin(phi) 2 pi tau^2.
// Samples are evaluated as the dictionary generator does (phase formed in
// FP64 and range-reduced before FP32 cospi/sinpi, Gaussian argument in
// FP64).  The standalone score kernel accumulates all ten sums in FP64; the
// refinement carries the phase and the two sums that define the objective in
// float-float and the eight gradient sums in FP32 (FP64 throughput is low on
// this GPU).
//
// Refinement.  BFGS on f(z) = -|s(w (.) z)| in coordinates scaled by the
// grid steps w, one cluster of 4 CTAs per channel: p = -H grad f (H reset to
// I when p is not a descent direction), a first step of at most half a grid
// step, Armijo backtracking (c1 = 1e-4, up to 20 halvings, evaluated four
// step sizes at a time, one per CTA), the standard BFGS inverse update when
// <y, s> > 0, parameters clamped to the grid box widened by one step; it
// stops early when no step is accepted.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "act_device.cuh"
#include "act_ff.cuh"
#include "act_internal.cuh"

namespace act {

namespace {

constexpr int kRefineThreads = 256;  // standalone score and update kernels
constexpr int kBfgsThreads = 512;    // the refinement: one block per channel
constexpr double kTwoPi = 6.283185307179586;

struct EvalOut {
    double s;
    double g[4];
    double nu;  // |u|
};

// The ten sums of one evaluation, reduced over the block; every thread
// receives the score and gradient.  sh must hold 10 * 32 doubles.
__device__ EvalOut eval_score(const double *th, const float *__restrict__ r, int L, double inv_fs, double *sh) {
    const double tc = th[0], fc = th[1], inv_dt = exp(-th[2]), c = th[3];
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};  // ru, uu, rd[4], ud[4]
    for (int n = threadIdx.x; n < L; n += blockDim.x) {
        const double tau = ((double)n - tc) * inv_fs;
        double ph = fma(c, tau, fc) * tau;
        ph -= rint(ph);
        const float C = cospif(2.0f * (float)ph);
        const float S = sinpif(2.0f * (float)ph);
        const float x = (float)(tau * inv_dt);
        const float E = expf(-0.5f * x * x);
        const float u = E * C;
        const float ES = E * S;
        const float du0 = (float)(((double)(E * x * C) * inv_dt + (double)ES * kTwoPi * (2.0 * c * tau + fc)) * inv_fs);
        const float du1 = (float)(-(double)ES * kTwoPi * tau);
        const float du2 = E * x * x * C;
        const float du3 = (float)(-(double)ES * kTwoPi * tau * tau);
        const double rv = (double)r[n];
        acc[0] = fma(rv, (double)u, acc[0]);
        acc[1] = fma((double)u, (double)u, acc[1]);
        acc[2] = fma(rv, (double)du0, acc[2]);
        acc[3] = fma(rv, (double)du1, acc[3]);
        acc[4] = fma(rv, (double)du2, acc[4]);
        acc[5] = fma(rv, (double)du3, acc[5]);
        acc[6] = fma((double)u, (double)du0, acc[6]);
        acc[7] = fma((double)u, (double)du1, acc[7]);
        acc[8] = fma((double)u, (double)du2, acc[8]);
        acc[9] = fma((double)u, (double)du3, acc[9]);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        acc[i] = warp_sum(acc[i]);
        if (lane == 0) sh[i * 32 + wid] = acc[i];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int i = 0; i < 10; ++i) {
            double t = lane < nw ? sh[i * 32 + lane] : 0.0;
            t = warp_sum(t);
            if (lane == 0) sh[i * 32] = t;
        }
    }
    __syncthreads();
    double tot[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) tot[i] = sh[i * 32];
    __syncthreads();
    EvalOut o;
    if (!(tot[1] > 0.0) || !isfinite(tot[1])) {
        o.s = 0.0;
        o.nu = 0.0;
        for (int i = 0; i < 4; ++i) o.g[i] = 0.0;
        return o;
    }
    o.nu = sqrt(tot[1]);
    o.s = tot[0] / o.nu;
    for (int i = 0; i < 4; ++i) o.g[i] = tot[2 + i] / o.nu - o.s * tot[6 + i] / tot[1];
    return o;
}

// Writes g(theta) = u/|u| for one channel (block), FP32.
__device__ void write_atom(const double *th, double nu, int L, double inv_fs, float *__restrict__ out) {
    const double tc = th[0], fc = th[1], inv_dt = exp(-th[2]), c = th[3];
    const float scale = nu > 0.0 ? (float)(1.0 / nu) : 0.0f;
    for (int n = threadIdx.x; n < L; n += blockDim.x) {
        const double tau = ((double)n - tc) * inv_fs;
        double ph = fma(c, tau, fc) * tau;
        ph -= rint(ph);
        const float x = (float)(tau * inv_dt);
        out[n] = expf(-0.5f * x * x) * cospif(2.0f * (float)ph) * scale;
    }
}

// Standalone score + adjoint: one block per channel.
__global__ void __launch_bounds__(kRefineThreads) k_chirplet_score(int L, double inv_fs, const double *__restrict__ theta,
                                                                  const float *__restrict__ R, double *__restrict__ score,
                                                                  double *__restrict__ grad, float *__restrict__ atoms) {
    __shared__ double sh[10 * 32];
    __shared__ double th[4];
    const int b = blockIdx.x;
    if (threadIdx.x < 4) th[threadIdx.x] = theta[4 * b + threadIdx.x];
    __syncthreads();
    const EvalOut o = eval_score(th, R + (size_t)b * L, L, inv_fs, sh);
    if (threadIdx.x == 0) {
        score[b] = o.s;
        if (grad)
            for (int i = 0; i < 4; ++i) grad[4 * b + i] = o.g[i];
    }
    if (atoms) write_atom(th, o.nu, L, inv_fs, atoms + (size_t)b * L);
}

struct RefineBox {
    double w[4], lo[4], hi[4];
    double inv_w[4], zlo[4], zhi[4];  // 1 / w and the box in scaled coordinates (formed on the host)
};

// Sums of one evaluation: the objective's two in float-float, the eight of
// its gradient in FP32.
struct EvalAcc {
    ff ru, uu;
    float rd[4], ud[4];
};

// Per-atom constants of an evaluation.
struct EvalConst {
    ChirpFF k;
    float inv_dt, inv_fs, c, fc;
};

// Sample n: the phase in float-float, the sample u and its four
// derivatives du in FP32 (expressions of the header comment).
__device__ __forceinline__ void eval_sample(int n, const EvalConst &e, float &u, float (&du)[4]) {
    constexpr float two_pi = (float)kTwoPi;
    ff tau;
    const float frac = chirp_phase_ff(n, e.k, &tau);
    const float t = tau.hi;
    float S, C;
    sincospif(2.0f * frac, &S, &C);
    const float x = chirp_x_ff(tau, e.k);
    const float E = expf(-0.5f * x * x);
    u = E * C;
    const float ES = E * S;
    du[0] = (E * x * C * e.inv_dt + ES * two_pi * fmaf(2.0f * e.c, t, e.fc)) * e.inv_fs;
    du[1] = -ES * two_pi * t;
    du[2] = E * x * x * C;
    du[3] = -ES * two_pi * t * t;
}

__device__ __forceinline__ void eval_accumulate(EvalAcc &a, float rv, float u, const float (&du)[4]) {
    ff_fma_acc(a.ru, rv, u);
    ff_fma_acc(a.uu, u, u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        a.rd[i] = fmaf(rv, du[i], a.rd[i]);
        a.ud[i] = fmaf(u, du[i], a.ud[i]);
    }
}

constexpr int kLineSearch = 20;  // Armijo halvings per iteration
constexpr int kRefineCluster = 4;  // CTAs per channel
constexpr int kRefineWarps = kBfgsThreads / 32;
constexpr int kCandPerCta = 2;     // line-search step sizes each CTA evaluates per round
constexpr int kCandWarps = kRefineWarps / kCandPerCta;  // warps per step size

// Sum over each group of 4 lanes (lane i of a group holds parameter i); the
// same bits in every lane of the group (FP32 addition commutes).
__device__ __forceinline__ float sum4f(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v + __shfl_xor_sync(0xffffffffu, v, 2);
}

// 2^-j for 0 <= j < 126, exact (built from the exponent bits).
__device__ __forceinline__ float pow2_negf(int j) { return __int_as_float((127 - j) << 23); }

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ bool ff_less(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
// a - b rounded to FP32 (a and b close: the pair difference is nearly exact)
__device__ __forceinline__ float ff_diff(ff a, ff b) {
    const ff d = ff_add(a, ff_neg(b));
    return d.hi + d.lo;
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Barrier over every thread of every CTA of the cluster; shared-memory
// writes before it are visible to the cluster's reads after it.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Stores v into the shared memory of CTA `rank` of this cluster, at the
// offset of p in this CTA's (C == 1: this CTA's own).  Made visible to that
// CTA by the next cluster barrier (release / acquire).
__device__ __forceinline__ void st_cluster_f32(float *p, uint32_t rank, int C, float v) {
    if (C == 1) {
        *p = v;
        return;
    }
    uint32_t addr;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(addr) : "r"(smem_u32(p)), "r"(rank));
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

// One line-search candidate's evaluation, published to the cluster:
// f = -|s| (float pair), the scaled gradient (FP32) and the candidate in
// scaled coordinates (float pairs).
struct Candidate {
    ff f;
    float valid;  // 1: a step size of this round (j < kLineSearch)
    float g[4];
    ff z[4];
};

// The per-candidate constants of Eq. (1) for lane i = parameter i of warp 0,
// formed in parallel from the parameter v as a float pair: lane 0 tc, lane 1
// fc, lane 2 1/dt = exp(-logDt), lane 3 c (1/fs is fixed).  1/dt only
// scales the envelope argument, which is rounded to FP32, so the FP32
// exponential gives it to the precision the sample uses.
__device__ __forceinline__ void put_const(EvalConst *ec, int i, ff v, ff inv_fs) {
    if (i == 0) {
        ec->k.tc = v;
        ec->k.inv_fs = inv_fs;
        ec->inv_fs = inv_fs.hi;
    } else if (i == 1) {
        ec->k.fc = v;
        ec->fc = v.hi;
    } else if (i == 2) {
        const float inv_dt = expf(-(v.hi + v.lo));
        ec->k.inv_dt = ff{inv_dt, 0.0f};
        ec->inv_dt = inv_dt;
    } else {
        ec->k.c = v;
        ec->c = v.hi;
    }
}

// The warp's sums of one evaluation by reduce-scatter: at every level a lane
// sends the half of its values its partner keeps and adds the half it keeps
// (xor 16: gradient sums 0-3 / 4-7 and ru / uu; then 8, 4 on the gradient
// sums; then plain butterflies), 19 shuffles instead of 60.  On return lane l
// holds the warp's total of gradient sum (l >> 2) (rd[0..3], ud[0..3]) in
// *gsum, and of ru (lanes 0-15) or uu (lanes 16-31) in *fsum.  Fixed order.
__device__ __forceinline__ void eval_warp_scatter(const EvalAcc &a, int lane, float *gsum, ff *fsum) {
    const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0, b2 = (lane & 4) != 0;
    const float g[8] = {a.rd[0], a.rd[1], a.rd[2], a.rd[3], a.ud[0], a.ud[1], a.ud[2], a.ud[3]};
    float w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        w[k] = (b4 ? g[4 + k] : g[k]) + __shfl_xor_sync(0xffffffffu, b4 ? g[k] : g[4 + k], 16);
    float x[2];
#pragma unroll
    for (int k = 0; k < 2; ++k)
        x[k] = (b3 ? w[2 + k] : w[k]) + __shfl_xor_sync(0xffffffffu, b3 ? w[k] : w[2 + k], 8);
    float y = (b2 ? x[1] : x[0]) + __shfl_xor_sync(0xffffffffu, b2 ? x[0] : x[1], 4);
    y += __shfl_xor_sync(0xffffffffu, y, 2);
    y += __shfl_xor_sync(0xffffffffu, y, 1);
    *gsum = y;
    ff v = ff_add(b4 ? a.uu : a.ru, ff_shfl_xor(b4 ? a.ru : a.uu, 16));
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) v = ff_add(v, ff_shfl_xor(v, off));
    *fsum = v;
}

// Score and gradient of kCandPerCta candidates at once: warp group h (warps
// h kCandWarps ..) evaluates the candidate whose constants are in ec[h],
// every thread of the group taking samples n = t, t + 32 kCandWarps, ....
// Partial sums go to red[warp]; after the barrier the group's first warp
// adds its warps' sums in warp order and finishes on the FP32 pipes.
// Returned in every lane of each group's first warp: the score s and
// component (lane & 3) of its gradient (zeros elsewhere).
__device__ __forceinline__ void eval_cands(const EvalConst *ec, const float *__restrict__ r, int L, float (*red)[12],
                                           ff *s_out, float *gi_out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int h = warp / kCandWarps, t = (int)threadIdx.x - h * kCandWarps * 32;
    EvalAcc a = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0, 0, 0, 0}, {0, 0, 0, 0}};
    {
        // kSpan samples of the thread at once: their evaluations are
        // independent (the latency of one overlaps the others), then they
        // are accumulated in sample order
        constexpr int kStride = 32 * kCandWarps, kSpan = 4;
        const EvalConst e = ec[h];
        for (int n0 = t; n0 < L; n0 += kSpan * kStride) {
            float u[kSpan], du[kSpan][4], rv[kSpan];
#pragma unroll
            for (int k = 0; k < kSpan; ++k) {
                const int n = n0 + k * kStride;
                rv[k] = n < L ? r[n] : 0.0f;
                eval_sample(n < L ? n : 0, e, u[k], du[k]);
            }
#pragma unroll
            for (int k = 0; k < kSpan; ++k)
                if (n0 + k * kStride < L) eval_accumulate(a, rv[k], u[k], du[k]);
        }
    }
    {
        // the warp's totals into red[warp]: [0..1] ru, [2..3] uu, [4 + c] gradient sum c
        float gs;
        ff fs;
        eval_warp_scatter(a, lane, &gs, &fs);
        if ((lane & 3) == 0) red[warp][4 + (lane >> 2)] = gs;
        if (lane == 0 || lane == 16) {
            red[warp][lane >> 3] = fs.hi;
            red[warp][(lane >> 3) + 1] = fs.lo;
        }
    }
    __syncthreads();
    *s_out = ff{0.0f, 0.0f};
    *gi_out = 0.0f;
    if (warp != h * kCandWarps) return;
    __syncwarp();  // the finish runs with the whole warp converged
    // lane 0: ru, lane 2: uu (float-float), lanes 4..11: the gradient sums,
    // each added over the group's warps in warp order
    ff tot = {0.0f, 0.0f};
    if (lane == 0 || lane == 2) {
        for (int w = 0; w < kCandWarps; ++w) tot = ff_add(tot, ff{red[warp + w][lane], red[warp + w][lane + 1]});
    } else if (lane >= 4 && lane < 12) {
        float t = 0.0f;
        for (int w = 0; w < kCandWarps; ++w) t += red[warp + w][lane];
        tot.hi = t;
    }
    const ff ru = ff_shfl(tot, 0), uu = ff_shfl(tot, 2);
    const int i = lane & 3;
    const float rdi = __shfl_sync(0xffffffffu, tot.hi, 4 + i);
    const float udi = __shfl_sync(0xffffffffu, tot.hi, 8 + i);
    // The finish on the FP32 pipes, uniform in the warp.  s = <r, u> / |u|
    // in float-float: 1/|u| is the FP32 reciprocal square root y0 corrected by
    // Newton-Raphson steps y <- y + y (1 - |u|^2 y^2) / 2 in float-float
    // (relative error 2^-22 -> about 2^-44 -> the pair's precision).  The gradient components come from
    // FP32 sums, so they are finished in FP32.  An atom with |u|^2 below
    // 1e-30 (every sample underflowed) scores 0.
    const bool ok = uu.hi > 1e-30f && uu.hi < 3.0e38f;
    const float y0 = rsqrtf(ok ? uu.hi : 1.0f);
    const ff y0sq = ff_fast_two_sum(y0 * y0, fmaf(y0, y0, -(y0 * y0)));
    const ff uy = ff_mul(ok ? uu : ff{1.0f, 0.0f}, y0sq);  // 1 - uy is exact in its high part
    const float e = (1.0f - uy.hi) - uy.lo;
    const ff y1 = ff_add_f(ff{y0, 0.0f}, 0.5f * y0 * e);
    // a second step in float-float brings 1/|u| to the pair's own precision
    const ff uy1 = ff_mul(ok ? uu : ff{1.0f, 0.0f}, ff_mul(y1, y1));
    const float e1 = (1.0f - uy1.hi) - uy1.lo;
    const ff y2 = ff_add_f(y1, 0.5f * y1.hi * e1);
    const ff sff = ff_mul(ru, y2);
    const float sf = sff.hi + sff.lo;
    *s_out = ok ? sff : ff{0.0f, 0.0f};
    *gi_out = ok ? fmaf(rdi, y2.hi, -sf * y2.hi * y2.hi * udi) : 0.0f;
}

// BFGS refinement of channel b's grid winner; theta_out[b][4].  A cluster of
// C CTAs serves one channel; all of them hold the same BFGS state and make
// the same decisions (they compute them from the same bits), so nothing but
// the candidates is exchanged.  Each iteration: the direction p = -H g
// (H reset to I if p is not a descent direction) and the first step alpha0
// (at most half a grid step); then rounds of line search in which CTA q
// evaluates the step alpha0 2^-(j0 + q); after a round every CTA reads the
// C candidates from the cluster's shared memory and takes the first (largest)
// step that satisfies the Armijo condition -- what sequential backtracking
// would take -- or, if none does, the next round j0 += C, up to kLineSearch
// halvings.  Then the BFGS inverse update (when <y, s> > 0).  It stops early
// when no step is accepted.  Bookkeeping runs on warp 0 (lane & 3 =
// parameter, the 4 x 4 update on 16 lanes); the other warps only evaluate.
__global__ void __launch_bounds__(kBfgsThreads) k_refine(GridAxes ax, RefineBox box, int steps, int Lp,
                                                          const float *__restrict__ R,
                                                          const unsigned long long *__restrict__ keys,
                                                          const double *__restrict__ theta_in, int theta_in_stride,
                                                          double *__restrict__ theta_out, int C) {
    // BFGS state: scaled coordinates z and objective f = -|s| as float pairs,
    // the scaled gradient, inverse Hessian, direction and step sizes in FP32
    // (FP64 runs at a small fraction of the FP32 rate on this GPU, and this
    // bookkeeping is the serial part of every iteration)
    __shared__ ff z[4], f, zlo[4], zhi[4], wff[4];
    __shared__ float gz[4], H[16], Hn[16], p[4], sv[4], yv[4], wf[4];
    __shared__ float gp, alpha0;
    __shared__ double th0[4];  // the start, returned unchanged if no step is taken
    // the round's candidates of the whole cluster (q = rank kCandPerCta + h),
    // pushed here by their owners before the round's cluster barrier; by
    // round parity
    __shared__ Candidate res[2][kRefineCluster * kCandPerCta];
    __shared__ float red[kRefineWarps][12];
    // every step size this CTA evaluates in one line search, formed with the
    // direction: slot s = round * kCandPerCta + h
    constexpr int kMaxSlots = kLineSearch * kCandPerCta;  // enough for C = 1
    __shared__ EvalConst slot_ec[kMaxSlots];
    __shared__ ff slot_z[kMaxSlots][4];
    __shared__ int done, slot0, moved;
    const int b = blockIdx.x / C;
    const uint32_t rank = C > 1 ? cluster_rank() : 0u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pi = lane & 3;  // the parameter of this lane in warp 0's bookkeeping
    const float *r = R + (size_t)b * Lp;
    const int L = ax.L;
    const ff inv_fs = ff_from_double(1.0 / ax.fs);

    if (warp == 0) {
        double p0 = 0.0;
        if (theta_in) {
            p0 = theta_in[(size_t)b * theta_in_stride + pi];
        } else {
            double pp[4];
            decode_params(ax, (int64_t)key_index(keys[b]), pp);
            p0 = pi == 0 ? pp[0] : (pi == 1 ? pp[1] : (pi == 2 ? pp[2] : pp[3]));
        }
        if (lane < 4) {
            // the clamp box in scaled coordinates, once per launch
            const double w = box.w[pi];
            wff[pi] = ff_from_double(w);
            wf[pi] = (float)w;
            zlo[pi] = ff_from_double(box.zlo[pi]);
            zhi[pi] = ff_from_double(box.zhi[pi]);
            z[pi] = ff_from_double(p0 * box.inv_w[pi]);
            th0[pi] = p0;
        }
        if (lane < 4 * kCandPerCta) put_const(&slot_ec[lane >> 2], pi, ff_from_double(p0), inv_fs);
        if (lane < 16) H[lane] = (lane % 5 == 0) ? 1.0f : 0.0f;
        if (lane == 0) {
            done = steps > 0 ? 0 : 1;
            moved = 0;
        }
    }
    __syncthreads();
    {  // the start point (every group of every CTA of the cluster evaluates it, with the same bits)
        ff s0;
        float g0;
        eval_cands(slot_ec, r, L, red, &s0, &g0);
        if (warp == 0 && lane < 4) {
            const float sg = s0.hi < 0.0f ? -1.0f : 1.0f;
            gz[pi] = -sg * g0 * wf[pi];
            if (lane == 0) f = s0.hi < 0.0f ? s0 : ff_neg(s0);
        }
    }
    int it = 0, j0 = 0, par = 0, rr = 0;
    bool new_dir = true;
    const int per_round = C * kCandPerCta;
    const int n_slots = (kLineSearch + per_round - 1) / per_round * kCandPerCta;
    for (;;) {
        if (warp == 0) {
            __syncwarp();
            if (!done && new_dir) {  // p = -H g (steepest descent, H reset, if not a descent direction)
                float v = 0.0f;
#pragma unroll
                for (int j = 0; j < 4; ++j) v = fmaf(-H[4 * pi + j], gz[j], v);
                float g_p = sum4f(gz[pi] * v);
                const bool reset = !(g_p < 0.0f);
                if (reset) {
                    v = -gz[pi];
                    g_p = sum4f(gz[pi] * v);
                }
                const float pn2 = sum4f(v * v);
                __syncwarp();
                if (lane < 4) {
                    p[pi] = v;
                    if (reset)
                        for (int k = 0; k < 4; ++k) H[4 * pi + k] = pi == k ? 1.0f : 0.0f;
                }
                if (lane == 0) {
                    gp = g_p;
                    alpha0 = pn2 > 0.25f ? 0.5f * rsqrtf(pn2) : 1.0f;
                    if (!(g_p < 0.0f)) done = 1;
                }
                new_dir = false;
                j0 = 0;
                rr = 0;
                __syncwarp();
                // the steps alpha0 2^-j of every round for this CTA, one (slot,
                // parameter) pair per lane, clamped to the box
                for (int t = lane; t < 4 * n_slots; t += 32) {
                    const int sl = t >> 2, i = t & 3;
                    const int j = (sl / kCandPerCta) * per_round + (int)rank * kCandPerCta + sl % kCandPerCta;
                    const float a = alpha0 * pow2_negf(j < kLineSearch ? j : 0);
                    ff zc = ff_add_f(z[i], a * p[i]);
                    zc = ff_less(zc, zlo[i]) ? zlo[i] : (ff_less(zhi[i], zc) ? zhi[i] : zc);
                    slot_z[sl][i] = zc;
                    put_const(&slot_ec[sl], i, ff_mul(zc, wff[i]), inv_fs);
                }
                __syncwarp();
            }
            if (lane == 0) slot0 = rr * kCandPerCta;
        }
        __syncthreads();
        if (done) break;
        const int s0 = slot0;
        ff sc;
        float gi;
        eval_cands(slot_ec + s0, r, L, red, &sc, &gi);
        if (warp % kCandWarps == 0 && lane < 4 * C) {
            // lane = (destination CTA, parameter): this candidate into every
            // CTA's list of the round
            const int hh = warp / kCandWarps, sl = s0 + hh;
            const uint32_t dst = (uint32_t)(lane >> 2);
            Candidate &cd = res[par][(int)rank * kCandPerCta + hh];
            const float sg = sc.hi < 0.0f ? -1.0f : 1.0f;
            st_cluster_f32(&cd.g[pi], dst, C, -sg * gi * wf[pi]);
            st_cluster_f32(&cd.z[pi].hi, dst, C, slot_z[sl][pi].hi);
            st_cluster_f32(&cd.z[pi].lo, dst, C, slot_z[sl][pi].lo);
            if (pi == 0) {
                const int j = (sl / kCandPerCta) * per_round + (int)rank * kCandPerCta + hh;
                const ff fq = sc.hi < 0.0f ? sc : ff_neg(sc);
                st_cluster_f32(&cd.f.hi, dst, C, fq.hi);
                st_cluster_f32(&cd.f.lo, dst, C, fq.lo);
                st_cluster_f32(&cd.valid, dst, C, j < kLineSearch ? 1.0f : 0.0f);
            }
        }
        // every CTA's candidate of this round is published
        if (C > 1)
            cluster_sync_all();
        else
            __syncthreads();
        if (warp == 0) {
            // lane q < C kCandPerCta: candidate q of the round (slot q % kCandPerCta
            // of CTA q / kCandPerCta, step alpha0 2^-(j0 + q)) and its Armijo
            // test f_q - f <= 1e-4 a_q <g, p> (the pair difference, nearly exact)
            int ok = 0;
            if (lane < C * kCandPerCta) {
                const Candidate &cq = res[par][lane];
                const float aq = alpha0 * pow2_negf(j0 + lane < kLineSearch ? j0 + lane : 0);
                ok = cq.valid != 0.0f && ff_diff(cq.f, f) <= 1e-4f * aq * gp;
            }
            const unsigned acc = __ballot_sync(0xffffffffu, ok);
            if (acc) {
                const int q = __ffs((int)acc) - 1;  // the largest accepted step
                const Candidate &cq = res[par][q];
                const ff zq = cq.z[pi];
                const float gq = cq.g[pi];
                const ff fq = cq.f;
                // BFGS inverse update H' = (I - rho s y^T) H (I - rho y s^T) + rho s s^T when <y, s> > 0
                const float si = ff_diff(zq, z[pi]), yi = gq - gz[pi];
                const float ys = sum4f(yi * si);
                const float rho = ys > 1e-30f ? 1.0f / ys : 0.0f;
                if (lane < 4) {
                    sv[pi] = si;
                    yv[pi] = yi;
                }
                __syncwarp();
                if (rho != 0.0f) {
                    if (lane < 16) {  // Hn = (I - rho s y^T) H
                        const int i = lane >> 2, j = lane & 3;
                        const float rs = rho * sv[i];
                        float t = 0.0f;
#pragma unroll
                        for (int k = 0; k < 4; ++k) t = fmaf((i == k ? 1.0f : 0.0f) - rs * yv[k], H[4 * k + j], t);
                        Hn[lane] = t;
                    }
                    __syncwarp();
                    if (lane < 16) {  // H = Hn (I - rho y s^T) + rho s s^T
                        const int i = lane >> 2, j = lane & 3;
                        const float rs = rho * sv[j];
                        float t = 0.0f;
#pragma unroll
                        for (int k = 0; k < 4; ++k) t = fmaf(Hn[4 * i + k], (j == k ? 1.0f : 0.0f) - rs * yv[k], t);
                        H[lane] = fmaf(rho * sv[i], sv[j], t);
                    }
                }
                __syncwarp();
                if (lane < 4) {
                    z[pi] = zq;
                    gz[pi] = gq;
                }
                if (lane == 0) {
                    f = fq;
                    moved = 1;
                    if (++it >= steps) done = 1;
                }
                new_dir = true;
            } else {
                j0 += per_round;
                ++rr;
                if (j0 >= kLineSearch && lane == 0) done = 1;  // no acceptable step: stop
            }
        }
        par ^= 1;
    }
    // no CTA leaves while another may still read its candidates
    if (C > 1) cluster_sync_all();
    if (rank == 0 && threadIdx.x < 4)
        theta_out[4 * b + threadIdx.x] = moved ? ff_to_double(ff_mul(z[threadIdx.x], wff[threadIdx.x])) : th0[threadIdx.x];
}

// Coefficient and residual update with the refined atom g(theta*) generated
// on the fly (Eq. (4)); the record keeps the grid winner's flat index (-1
// when the selection did not come from the grid).  The samples are those of
// the dictionary generator (float-float phase, chirp_sample_ff), formed once
// into registers; |u|^2 is a float-float sum, c = <g, r> an FP32 block sum,
// |r|^2 an FP64 sum.
__global__ void __launch_bounds__(kRefineThreads) k_update_refined(int Lp, float *__restrict__ R,
                                                                  __nv_bfloat16 *__restrict__ R16, int Lb,
                                                                  unsigned long long *__restrict__ keys, GridAxes ax,
                                                                  const double *__restrict__ theta, int k, int P,
                                                                  act_atom *__restrict__ atoms,
                                                                  float *__restrict__ coefs,
                                                                  double *__restrict__ energy, int *fb_count) {
    constexpr int kPer = kMaxSamples / kRefineThreads;
    __shared__ float shf[32];
    __shared__ double shd[32];
    __shared__ ff shff[32];
    __shared__ ChirpFF kc;
    const int b = blockIdx.x;
    const int L = ax.L;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kRefineThreads / 32;
    const double tc = theta[4 * b], fc = theta[4 * b + 1], ld = theta[4 * b + 2], cc = theta[4 * b + 3];
    if (threadIdx.x == 0) kc = chirp_ff(tc, 1.0 / ax.fs, fc, cc, exp(-ld));
    __syncthreads();
    const ChirpFF kk = kc;
    float *r = R + (size_t)b * Lp;
    float u[kPer];
    ff e = {0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int n = (int)threadIdx.x + i * kRefineThreads;
        u[i] = n < L ? chirp_sample_ff(n, kk) : 0.0f;
        ff_fma_acc(e, u[i], u[i]);
    }
    e = ff_warp_sum(e);
    if (lane == 0) shff[warp] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        ff t = shff[0];
        for (int w = 1; w < nw; ++w) t = ff_add(t, shff[w]);
        shd[0] = ff_to_double(t);
    }
    __syncthreads();
    const double uu = shd[0];
    __syncthreads();
    const float scale = (uu > 0.0 && isfinite(uu)) ? (float)(1.0 / sqrt(uu)) : 0.0f;
    float part = 0.0f;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int n = (int)threadIdx.x + i * kRefineThreads;
        u[i] *= scale;  // g
        if (n < L) part = fmaf(u[i], r[n], part);
    }
    const float c = block_sum(part, shf);
    double e2 = 0.0;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int n = (int)threadIdx.x + i * kRefineThreads;
        if (n < L) {
            const float v = fmaf(-c, u[i], r[n]);
            r[n] = v;
            e2 = fma((double)v, (double)v, e2);
            if (R16) R16[(size_t)b * Lb + n] = __float2bfloat16_rn(v);
        }
    }
    const double tot = block_sum(e2, shd);
    if (threadIdx.x == 0) {
        act_atom a;
        a.tc = tc;
        a.fc = fc;
        a.logdt = ld;
        a.c = cc;
        a.flat_index = keys ? (int64_t)key_index(keys[b]) : -1;  // -1: not a grid atom
        atoms[(size_t)b * P + k] = a;
        coefs[(size_t)b * P + k] = c;
        energy[(size_t)b * (P + 1) + k + 1] = tot;
        if (keys) keys[b] = 0ull;
        if (fb_count && b == 0) {
            fb_count[0] = 0;
            fb_count[1] = 0;
        }
    }
}

}  // namespace

cudaError_t launch_chirplet_score(int L, double fs, const double *theta, const float *R, int B, double *score,
                                  double *grad, float *atoms, cudaStream_t st) {
    k_chirplet_score<<<B, kRefineThreads, 0, st>>>(L, 1.0 / fs, theta, R, score, grad, atoms);
    return cudaGetLastError();
}

cudaError_t launch_refine(const GridAxes &ax, int steps, int Lp, const float *R, const unsigned long long *keys,
                          const double *theta_in, int theta_in_stride, int B, double *theta_out, cudaStream_t st) {
    RefineBox box;
    for (int i = 0; i < 4; ++i) {
        // scale = grid step; box = grid range widened by one step (an axis
        // with a zero step is held fixed)
        const double st_i = fabs(ax.step[i]);
        const double first = ax.lo[i], last = ax.lo[i] + (double)(ax.count[i] - 1) * ax.step[i];
        box.w[i] = st_i > 0.0 ? st_i : 1.0;
        box.lo[i] = st_i > 0.0 ? fmin(first, last) - st_i : first;
        box.hi[i] = st_i > 0.0 ? fmax(first, last) + st_i : first;
        box.inv_w[i] = 1.0 / box.w[i];
        box.zlo[i] = box.lo[i] / box.w[i];
        box.zhi[i] = box.hi[i] / box.w[i];
    }
    // a cluster of C CTAs per channel: the largest C of kRefineCluster, 2, 1
    // for which every channel's cluster is resident at once (measured: 64
    // channels refine 23 % faster on clusters of 2 in one wave than on
    // clusters of 4 in two; 32 channels fastest on clusters of 4); when no
    // size fits, clusters of kRefineCluster.  Every size takes the same
    // steps (the first that satisfies the Armijo condition), so the results
    // do not depend on it.
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kBfgsThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = attr;
    int C = 0, clusters_full = 0;
    for (int c : {kRefineCluster, 2}) {
        attr[0].val.clusterDim.x = (unsigned)c;
        cfg.gridDim = dim3((unsigned)(B * c));
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, k_refine, &cfg) != cudaSuccess) {
            cudaGetLastError();
            clusters = 0;
        }
        if (c == kRefineCluster) clusters_full = clusters;
        if (clusters >= B) {
            C = c;
            break;
        }
    }
    if (C == 0) {
        int per_sm = 0, sms = 0, dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_refine, kBfgsThreads, 0);
        if (e != cudaSuccess) cudaGetLastError();
        // one CTA per channel when that puts every channel on at once (or no
        // cluster can be placed), else full clusters over several waves
        C = (clusters_full < 1 || (e == cudaSuccess && per_sm * sms >= B)) ? 1 : kRefineCluster;
    }
    if (C > 1) {
        attr[0].val.clusterDim.x = (unsigned)C;
        cfg.gridDim = dim3((unsigned)(B * C));
        cfg.numAttrs = 1;
    } else {
        cfg.gridDim = dim3((unsigned)B);
        cfg.numAttrs = 0;
    }
    return cudaLaunchKernelEx(&cfg, k_refine, ax, box, steps, Lp, R, keys, theta_in, theta_in_stride, theta_out, C);
}

cudaError_t launch_update_refined(int Lp, float *R, __nv_bfloat16 *R16, int Lb, int B, unsigned long long *keys,
                                  const GridAxes &ax, const double *theta, int k, int P, act_atom *atoms, float *coefs,
                                  double *energy, int *fb_count, cudaStream_t st) {
    k_update_refined<<<B, kRefineThreads, 0, st>>>(Lp, R, R16, Lb, keys, ax, theta, k, P, atoms, coefs, energy,
                                                   fb_count);
    return cudaGetLastError();
}

}  // namespace act
