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
// grid steps w, one block per channel: p = -H grad f (H reset to I when p
// is not a descent direction), a first step of at most half a grid step,
// Armijo backtracking (c1 = 1e-4, up to 20 halvings, evaluated 8 at a time
// by the 8 warps), the standard BFGS inverse update when <y, s> > 0,
// parameters clamped to the grid box widened by one step; it stops early
// when no step is accepted.
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
                                                                  const float *__restrict__ R, float *__restrict__ score,
                                                                  double *__restrict__ grad, float *__restrict__ atoms) {
    __shared__ double sh[10 * 32];
    __shared__ double th[4];
    const int b = blockIdx.x;
    if (threadIdx.x < 4) th[threadIdx.x] = theta[4 * b + threadIdx.x];
    __syncthreads();
    const EvalOut o = eval_score(th, R + (size_t)b * L, L, inv_fs, sh);
    if (threadIdx.x == 0) {
        score[b] = (float)o.s;
        if (grad)
            for (int i = 0; i < 4; ++i) grad[4 * b + i] = o.g[i];
    }
    if (atoms) write_atom(th, o.nu, L, inv_fs, atoms + (size_t)b * L);
}

struct RefineBox {
    double w[4], lo[4], hi[4];
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

__device__ __forceinline__ EvalConst eval_const(const double *th, double inv_fs) {
    const double inv_dt = exp(-th[2]);
    return {chirp_ff(th[0], inv_fs, th[1], th[3], inv_dt), (float)inv_dt, (float)inv_fs, (float)th[3],
            (float)th[1]};
}

// Adds sample n: the phase in float-float, the sample and its four
// derivatives in FP32 (expressions of the header comment).
__device__ __forceinline__ void eval_add(EvalAcc &a, int n, float rv, const EvalConst &e) {
    constexpr float two_pi = (float)kTwoPi;
    ff tau;
    const float frac = chirp_phase_ff(n, e.k, &tau);
    const float t = tau.hi;
    float S, C;
    sincospif(2.0f * frac, &S, &C);
    const float x = chirp_x_ff(tau, e.k);
    const float E = expf(-0.5f * x * x);
    const float u = E * C;
    const float ES = E * S;
    const float du[4] = {(E * x * C * e.inv_dt + ES * two_pi * fmaf(2.0f * e.c, t, e.fc)) * e.inv_fs,
                         -ES * two_pi * t, E * x * x * C, -ES * two_pi * t * t};
    ff_fma_acc(a.ru, rv, u);
    ff_fma_acc(a.uu, u, u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        a.rd[i] = fmaf(rv, du[i], a.rd[i]);
        a.ud[i] = fmaf(u, du[i], a.ud[i]);
    }
}

__device__ __forceinline__ void eval_warp_reduce(EvalAcc &a) {
    a.ru = ff_warp_sum(a.ru);
    a.uu = ff_warp_sum(a.uu);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        a.rd[i] = warp_sum(a.rd[i]);
        a.ud[i] = warp_sum(a.ud[i]);
    }
}

// Score and one gradient component of an evaluation, as the lanes of the
// evaluating group's first warp hold them: s in every lane, component
// lane & 3 of the gradient in gi.
struct EvalLane {
    double s, gi;
};

// Score and gradient by a group of G consecutive warps (samples strided by
// the group, the warps' sums added in warp order); every group of the block
// calls it at once (it holds block barriers), each on its own candidate th
// (inactive groups take part without evaluating).  The result is valid in
// lanes 0..3 of the group's first warp, which all add the warps' sums and
// finish in FP64 together (an FP64 instruction costs the same pipe time
// however few lanes are active).  red holds one EvalAcc per warp; ec one slot
// of constants per group (formed once, by the group's first thread).
template <int G>
__device__ EvalLane eval_group(const double *th, bool active, const float *__restrict__ r, int L, double inv_fs,
                               EvalAcc *red, EvalConst *ec) {
    const int warp = threadIdx.x >> 5, g = warp / G, t = (int)threadIdx.x - g * G * 32;
    if (t == 0 && active) ec[g] = eval_const(th, inv_fs);
    __syncthreads();
    EvalAcc a = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0, 0, 0, 0}, {0, 0, 0, 0}};
    if (active) {
        const EvalConst e = ec[g];
        for (int n = t; n < L; n += 32 * G) eval_add(a, n, r[n], e);
    }
    eval_warp_reduce(a);
    if ((threadIdx.x & 31) == 0) red[warp] = a;
    __syncthreads();
    EvalLane o = {0.0, 0.0};
    if (warp == g * G && active) {
        EvalAcc u = red[g * G];
        for (int w = 1; w < G; ++w) {
            const EvalAcc &v = red[g * G + w];
            u.ru = ff_add(u.ru, v.ru);
            u.uu = ff_add(u.uu, v.uu);
            for (int i = 0; i < 4; ++i) {
                u.rd[i] += v.rd[i];
                u.ud[i] += v.ud[i];
            }
        }
        const double ru = ff_to_double(u.ru), uu = ff_to_double(u.uu);
        if (uu > 0.0 && isfinite(uu)) {
            const int i = threadIdx.x & 3;
            const float rdi = i == 0 ? u.rd[0] : (i == 1 ? u.rd[1] : (i == 2 ? u.rd[2] : u.rd[3]));
            const float udi = i == 0 ? u.ud[0] : (i == 1 ? u.ud[1] : (i == 2 ? u.ud[2] : u.ud[3]));
            const double inv_nu = 1.0 / sqrt(uu);
            o.s = ru * inv_nu;
            const double s_uu = o.s * inv_nu * inv_nu;
            o.gi = (double)rdi * inv_nu - s_uu * (double)udi;
        }
    }
    return o;
}

constexpr int kLineSearch = 20;  // Armijo halvings per iteration

// Sum over each group of 4 lanes (lane i of a group holds parameter i).
__device__ __forceinline__ double sum4(double v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v + __shfl_xor_sync(0xffffffffu, v, 2);
}

// BFGS refinement of channel b's grid winner; theta_out[b][4].  Each
// iteration evaluates the full step alpha0 and then, if the Armijo
// condition fails, half of it with the whole block (the usual outcomes);
// after that groups of 4 warps evaluate the next 4 step sizes alpha0 2^-j at
// once, and so on.  The first (largest) step that satisfies the condition
// is taken, which is what sequential backtracking would take.  The
// per-parameter bookkeeping runs on lanes of warp 0 (lane & 3 = parameter),
// the 4 x 4 inverse update on 16 threads.
__global__ void __launch_bounds__(kBfgsThreads) k_refine(GridAxes ax, RefineBox box, int steps, int Lp,
                                                          const float *__restrict__ R,
                                                          const unsigned long long *__restrict__ keys,
                                                          const double *__restrict__ theta_in, int theta_in_stride,
                                                          double *__restrict__ theta_out) {
    constexpr int kWarps = kBfgsThreads / 32;
    constexpr int kBlockSteps = 2;  // steps j = 0, 1 evaluated by the whole block
    constexpr int kGroupWarps = 4;  // then kSlots steps at a time, one per group of warps
    constexpr int kSlots = kWarps / kGroupWarps;
    constexpr int kNone = kSlots;   // state: no step accepted yet
    __shared__ double z[4], gz[4], H[16], Hn[16], p[4], th_cur[4], sv[4], yv[4];
    __shared__ double cz[kSlots][4], cth[kSlots][4], cg[kSlots][4], cf[kSlots], ca[kSlots];
    __shared__ double f, gp, alpha0, rho;
    __shared__ EvalAcc red[kWarps];
    __shared__ EvalConst ec[kSlots];
    __shared__ int state;  // -1: stop; otherwise the accepted slot (or kNone)
    const int b = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pi = lane & 3;  // the parameter of this lane in warp 0's bookkeeping
    const float *r = R + (size_t)b * Lp;
    const int L = ax.L;
    const double inv_fs = 1.0 / ax.fs;

    // component i of the trial point of step j into slot q
    auto trial = [&](int j, int q, int i) {
        const double a = alpha0 * ldexp(1.0, -j);
        double v = (z[i] + a * p[i]) * box.w[i];
        v = v < box.lo[i] ? box.lo[i] : (v > box.hi[i] ? box.hi[i] : v);
        cz[q][i] = v / box.w[i];
        cth[q][i] = v;
        if (i == 0) ca[q] = a;
    };
    // f and scaled gradient component i of slot q (lane i < 4 of the group's first warp)
    auto record = [&](const EvalLane &o, int q, int i) {
        const double sg = o.s < 0.0 ? -1.0 : 1.0;
        cg[q][i] = -sg * o.gi * box.w[i];
        if (i == 0) cf[q] = -fabs(o.s);
    };
    auto armijo = [&](int q) { return cf[q] <= f + 1e-4 * ca[q] * gp; };

    if (threadIdx.x == 0) {
        double p0[4];
        if (theta_in) {
            for (int i = 0; i < 4; ++i) p0[i] = theta_in[(size_t)b * theta_in_stride + i];
        } else {
            decode_params(ax, (int64_t)key_index(keys[b]), p0);
        }
        for (int i = 0; i < 4; ++i) {
            z[i] = p0[i] / box.w[i];
            th_cur[i] = p0[i];  // the parameters themselves: returned unchanged if no step is taken
        }
    }
    if (threadIdx.x < 16) H[threadIdx.x] = (threadIdx.x % 5 == 0) ? 1.0 : 0.0;
    __syncthreads();
    {
        const EvalLane o = eval_group<kWarps>(th_cur, true, r, L, inv_fs, red, ec);
        if (threadIdx.x < 4) {
            const double sg = o.s < 0.0 ? -1.0 : 1.0;
            gz[threadIdx.x] = -sg * o.gi * box.w[threadIdx.x];
            if (threadIdx.x == 0) f = -fabs(o.s);
        }
    }
    __syncthreads();
    for (int it = 0; it < steps; ++it) {
        if (warp == 0) {  // direction p = -H g (steepest descent, H reset, if not a descent direction)
            double v = 0.0;
            for (int j = 0; j < 4; ++j) v -= H[4 * pi + j] * gz[j];
            double g_p = sum4(gz[pi] * v);
            const bool reset = !(g_p < 0.0);
            if (reset) {
                v = -gz[pi];
                g_p = sum4(gz[pi] * v);
            }
            const double pn = sqrt(sum4(v * v));
            __syncwarp();
            if (lane < 4) {
                p[pi] = v;
                if (reset)
                    for (int k = 0; k < 4; ++k) H[4 * pi + k] = pi == k ? 1.0 : 0.0;
            }
            if (lane == 0) {
                gp = g_p;
                alpha0 = pn > 0.5 ? 0.5 / pn : 1.0;
                state = (g_p < 0.0) ? kNone : -1;
            }
            __syncwarp();
            if (g_p < 0.0 && lane < 4) trial(0, 0, pi);
        }
        __syncthreads();
        if (state < 0) break;
        // the full and the half step, by the whole block
        for (int j = 0; j < kBlockSteps && state == kNone; ++j) {
            if (j > 0) {
                if (threadIdx.x < 4) trial(j, 0, threadIdx.x);
                __syncthreads();
            }
            const EvalLane o = eval_group<kWarps>(cth[0], true, r, L, inv_fs, red, ec);
            if (threadIdx.x < 4) record(o, 0, threadIdx.x);
            if (threadIdx.x == 0 && armijo(0)) state = 0;
            __syncthreads();
        }
        // shorter steps, kSlots at a time (one group of warps each)
        for (int j0 = kBlockSteps; state == kNone && j0 < kLineSearch; j0 += kSlots) {
            const int g = warp / kGroupWarps, t = (int)threadIdx.x - g * kGroupWarps * 32;
            const bool active = j0 + g < kLineSearch;
            if (active && t < 4) trial(j0 + g, g, t);
            __syncwarp();  // the group's first thread reads the trial point
            const EvalLane o = eval_group<kGroupWarps>(cth[g], active, r, L, inv_fs, red, ec);
            if (active && t < 4) record(o, g, t);
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int q = 0; q < kSlots && j0 + q < kLineSearch; ++q)
                    if (armijo(q)) {
                        state = q;
                        break;
                    }
            }
            __syncthreads();
        }
        if (state >= kNone) break;  // no acceptable step
        // BFGS inverse update H' = (I - rho s y^T) H (I - rho y s^T) + rho s s^T
        // when <y, s> > 0
        const int q = state;
        if (warp == 0) {
            const double si = cz[q][pi] - z[pi], yi = cg[q][pi] - gz[pi];
            const double ys = sum4(yi * si);
            if (lane < 4) {
                sv[pi] = si;
                yv[pi] = yi;
            }
            if (lane == 0) rho = ys > 1e-300 ? 1.0 / ys : 0.0;
        }
        __syncthreads();
        if (rho != 0.0) {
            if (threadIdx.x < 16) {  // Hn = (I - rho s y^T) H
                const int i = threadIdx.x >> 2, j = threadIdx.x & 3;
                double a = 0.0;
                for (int k = 0; k < 4; ++k) a += ((i == k ? 1.0 : 0.0) - rho * sv[i] * yv[k]) * H[4 * k + j];
                Hn[threadIdx.x] = a;
            }
            __syncthreads();
            if (threadIdx.x < 16) {  // H = Hn (I - rho y s^T) + rho s s^T
                const int i = threadIdx.x >> 2, j = threadIdx.x & 3;
                double a = 0.0;
                for (int k = 0; k < 4; ++k) a += Hn[4 * i + k] * ((j == k ? 1.0 : 0.0) - rho * sv[j] * yv[k]);
                H[threadIdx.x] = a + rho * sv[i] * sv[j];
            }
        }
        if (threadIdx.x < 4) {
            z[threadIdx.x] = cz[q][threadIdx.x];
            th_cur[threadIdx.x] = cth[q][threadIdx.x];
            gz[threadIdx.x] = cg[q][threadIdx.x];
        }
        if (threadIdx.x == 0) f = cf[q];
        __syncthreads();
    }
    if (threadIdx.x < 4) theta_out[4 * b + threadIdx.x] = th_cur[threadIdx.x];
}

// Coefficient and residual update with the refined atom g(theta*) generated
// on the fly (Eq. (4)); the record keeps the grid winner's flat index (-1
// when the selection did not come from the grid).
__global__ void __launch_bounds__(kRefineThreads) k_update_refined(int Lp, float *__restrict__ R,
                                                                  __nv_bfloat16 *__restrict__ R16, int Lb,
                                                                  unsigned long long *__restrict__ keys, GridAxes ax,
                                                                  const double *__restrict__ theta, int k, int P,
                                                                  act_atom *__restrict__ atoms,
                                                                  float *__restrict__ coefs,
                                                                  double *__restrict__ energy, int *fb_count) {
    __shared__ float shf[32];
    __shared__ double shd[32];
    const int b = blockIdx.x;
    const int L = ax.L;
    const double inv_fs = 1.0 / ax.fs;
    const double tc = theta[4 * b], fc = theta[4 * b + 1], ld = theta[4 * b + 2], cc = theta[4 * b + 3];
    const double inv_dt = exp(-ld);
    float *r = R + (size_t)b * Lp;
    // |u|^2 in FP64, then g = u / |u| recomputed per sample
    double e = 0.0;
    for (int n = threadIdx.x; n < L; n += blockDim.x) {
        const double tau = ((double)n - tc) * inv_fs;
        double ph = fma(cc, tau, fc) * tau;
        ph -= rint(ph);
        const float x = (float)(tau * inv_dt);
        const float u = expf(-0.5f * x * x) * cospif(2.0f * (float)ph);
        e = fma((double)u, (double)u, e);
    }
    const double uu = block_sum(e, shd);
    const float scale = (uu > 0.0 && isfinite(uu)) ? (float)(1.0 / sqrt(uu)) : 0.0f;
    float part = 0.0f;
    for (int n = threadIdx.x; n < L; n += blockDim.x) {
        const double tau = ((double)n - tc) * inv_fs;
        double ph = fma(cc, tau, fc) * tau;
        ph -= rint(ph);
        const float x = (float)(tau * inv_dt);
        const float g = expf(-0.5f * x * x) * cospif(2.0f * (float)ph) * scale;
        part = fmaf(g, r[n], part);
    }
    const float c = block_sum(part, shf);
    double e2 = 0.0;
    for (int n = threadIdx.x; n < L; n += blockDim.x) {
        const double tau = ((double)n - tc) * inv_fs;
        double ph = fma(cc, tau, fc) * tau;
        ph -= rint(ph);
        const float x = (float)(tau * inv_dt);
        const float g = expf(-0.5f * x * x) * cospif(2.0f * (float)ph) * scale;
        const float v = fmaf(-c, g, r[n]);
        r[n] = v;
        e2 = fma((double)v, (double)v, e2);
        if (R16) R16[(size_t)b * Lb + n] = __float2bfloat16_rn(v);
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

cudaError_t launch_chirplet_score(int L, double fs, const double *theta, const float *R, int B, float *score,
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
        const double st = fabs(ax.step[i]);
        const double first = ax.lo[i], last = ax.lo[i] + (double)(ax.count[i] - 1) * ax.step[i];
        box.w[i] = st > 0.0 ? st : 1.0;
        box.lo[i] = st > 0.0 ? fmin(first, last) - st : first;
        box.hi[i] = st > 0.0 ? fmax(first, last) + st : first;
    }
    k_refine<<<B, kBfgsThreads, 0, st>>>(ax, box, steps, Lp, R, keys, theta_in, theta_in_stride, theta_out);
    return cudaGetLastError();
}

cudaError_t launch_update_refined(int Lp, float *R, __nv_bfloat16 *R16, int Lb, int B, unsigned long long *keys,
                                  const GridAxes &ax, const double *theta, int k, int P, act_atom *atoms, float *coefs,
                                  double *energy, int *fb_count, cudaStream_t st) {
    k_update_refined<<<B, kRefineThreads, 0, st>>>(Lp, R, R16, Lb, keys, ax, theta, k, P, atoms, coefs, energy,
                                                   fb_count);
    return cudaGetLastError();
}

}  // namespace act
