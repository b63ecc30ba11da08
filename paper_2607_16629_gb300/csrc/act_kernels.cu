// CUDA kernels of the FP32 path: atom generation (Eq. (1) real part with
// unit l2 norm, Sec. III-A), residual initialisation, and the coefficient /
// residual update of Eq. (4).  The GEMV search is in act_gemv.cu.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "act_device.cuh"
#include "act_ff.cuh"
#include "act_internal.cuh"
#include "act_update.cuh"

namespace act {

// ---------------------------------------------------------------------------
// Atom generation
// ---------------------------------------------------------------------------
// A warp per atom at a time.  Lane l owns samples 4*(l + 32 j) + e, e = 0..3,
// so the FP32 row is written with 128-bit stores.  The BF16 copy is written
// tile-major, [atom / 256][sample / 64][atom % 256][sample % 64], so that one
// 256-atom x 64-sample operand tile of the tensor-core search is a single
// contiguous 32 KB block.  The phase of Eq. (1), in cycles,
// phi = c tau^2 + fc tau with tau = (n - tc) / fs, is evaluated in
// float-float (about 48 bits) and reduced to [-1/2, 1/2] before the FP32
// cospi; the Gaussian argument tau / dt is rounded once to FP32 and
// exponentiated in FP32; the squared norm is a float-float sum (GB300 runs
// FP64 at a small fraction of its FP32 rate; the per-atom constants alone
// are formed in FP64).  An atom whose FP32 samples are all zero (or not
// finite) is degenerate: its row is stored as zeros and it scores 0.
template <int NV>
__global__ void __launch_bounds__(256) k_gen_atoms(GridAxes ax, int64_t K, int Lp, float *__restrict__ d32,
                                                    __nv_bfloat16 *__restrict__ d16, int Lb,
                                                    unsigned long long *__restrict__ degenerate,
                                                    unsigned int *__restrict__ eps_bits) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double inv_fs = 1.0 / ax.fs;
    // a warp takes 32 atoms at a time: lane l forms atom base + l's
    // constants (FP64, once per atom), then the warp generates the 32 atoms
    // one after another with the constants broadcast from their lane
    for (int64_t base = warp * 32; base < K; base += nwarps * 32) {
        ChirpFF mine = {};
        if (base + lane < K) {
            double p[4];
            decode_params(ax, base + lane, p);
            mine = chirp_ff(p[0], inv_fs, p[1], p[3], exp(-p[2]));
        }
        const int count = K - base < 32 ? (int)(K - base) : 32;
        for (int q = 0; q < count; ++q) {
            const int64_t atom = base + q;
            const ChirpFF k = chirp_ff_shfl(mine, q);
            float u[NV][4];
            ff energy = {0.0f, 0.0f};
#pragma unroll
            for (int j = 0; j < NV; ++j) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int n = 4 * (lane + 32 * j) + e;
                    const float v = n < ax.L ? chirp_sample_ff(n, k) : 0.0f;
                    u[j][e] = v;
                    ff_fma_acc(energy, v, v);
                }
            }
            const double en = ff_to_double(ff_warp_sum(energy));
            float scale = 0.0f;
            const bool bad = !(en > 0.0) || !isfinite(en);
            if (!bad) scale = (float)(1.0 / sqrt(en));
            if (bad && lane == 0 && degenerate) atomicAdd(degenerate, 1ull);
            float4 *row = reinterpret_cast<float4 *>(d32 + atom * (int64_t)Lp);
            ff err = {0.0f, 0.0f};  // |bf16(g) - g|^2 of this atom (BF16 layout only)
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
                        // each difference is exact (Sterbenz); squares summed in float-float
                        ff_fma_acc(err, flo.x - w.x, flo.x - w.x);
                        ff_fma_acc(err, flo.y - w.y, flo.y - w.y);
                        ff_fma_acc(err, fhi.x - w.z, fhi.x - w.z);
                        ff_fma_acc(err, fhi.y - w.w, fhi.y - w.w);
                        uint2 packed;
                        packed.x = *reinterpret_cast<uint32_t *>(&lo);
                        packed.y = *reinterpret_cast<uint32_t *>(&hi);
                        // tile-major: [atom / 256][n0 / 64][atom % 256][n0 % 64]
                        const int64_t off =
                            (((atom >> 8) * (Lb >> 6) + (n0 >> 6)) * 256 + (atom & 255)) * 64 + (n0 & 63);
                        *reinterpret_cast<uint2 *>(d16 + off) = packed;
                    }
                }
            }
            if (d16 && eps_bits) {
                const double e2 = ff_to_double(ff_warp_sum(err));
                // positive floats order like their bit patterns; round the norm up
                if (lane == 0) atomicMax(eps_bits, __float_as_uint(__double2float_ru(sqrt(e2) * (1.0 + 1e-6))));
            }
        }
    }
}

cudaError_t launch_gen_atoms(const GridAxes &ax, int64_t K, int Lp, float *d32, __nv_bfloat16 *d16, int Lb,
                             unsigned long long *degenerate, unsigned int *eps_bits, int sm_count, cudaStream_t st) {
    const int nv = Lp / 128;
    int64_t blocks = (K + 255) / 256;  // 8 warps of 32 atoms per block
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
    // the first search may launch now (it waits for this kernel's completion)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
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
// Coefficient and residual update (Eq. (4), Fig. 1): one block per channel.
// c_k = <g*, r_k> in FP32, r_{k+1} = r_k - c_k g*, |r_{k+1}|^2 summed as
// float pairs and returned in FP64, the selected atom's parameters decoded
// from its flat index, the key cleared for the next order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kUpdateThreads) k_update(const float *__restrict__ D32, int Lp, int L,
                                                           float *__restrict__ R, __nv_bfloat16 *__restrict__ R16,
                                                           int Lb, unsigned long long *__restrict__ keys,
                                                           GridAxes ax, int k, int P,
                                                           act_atom *__restrict__ atoms, float *__restrict__ coefs,
                                                           double *__restrict__ energy, int *fb_count) {
    __shared__ float shf[32];
    __shared__ ff shp[32];
    // launched as a programmatic dependent of the search: every block waits
    // for its keys, then lets the next search launch
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int b = blockIdx.x;
    const unsigned long long key = keys[b];
    const uint32_t idx = key_index(key);
    const float *g = D32 + (int64_t)idx * Lp;
    float *r = R + (int64_t)b * Lp;

    float part = 0.0f;
    for (int n = threadIdx.x; n < L; n += blockDim.x) part = fmaf(g[n], r[n], part);
    const float c = block_sum(part, shf);

    ff e = {0.0f, 0.0f};  // |r_{k+1}|^2 as a float pair (about 2^-44 relative)
    for (int n = threadIdx.x; n < L; n += blockDim.x) {
        const float v = fmaf(-c, g[n], r[n]);
        r[n] = v;
        ff_add_square(e, v);
        if (R16) R16[(int64_t)b * Lb + n] = __float2bfloat16_rn(v);
    }
    const ff tot = block_sum_ff(e, shp);
    if (threadIdx.x < 32) write_atom_lanes(ax, idx, atoms + (int64_t)b * P + k);
    if (threadIdx.x == 0) {
        coefs[(int64_t)b * P + k] = c;
        energy[(int64_t)b * (P + 1) + k + 1] = ff_to_double(tot);
        keys[b] = 0ull;
        if (fb_count && b == 0) {
            fb_count[0] = 0;  // channels queued for the FP32 full search
            fb_count[1] = 0;  // (channel, CTA) pairs queued for an FP32 rescan
        }
    }
}

cudaError_t launch_update(const float *D32, int Lp, int L, float *R, __nv_bfloat16 *R16, int Lb, int B,
                          unsigned long long *keys, const GridAxes &ax, int k, int P, act_atom *atoms, float *coefs,
                          double *energy, int *fb_count, cudaStream_t st, bool pdl) {
    return launch_kernel(k_update, dim3(B), dim3(kUpdateThreads), 0, st, pdl, D32, Lp, L, R, R16, Lb, keys, ax, k, P,
                         atoms, coefs, energy, fb_count);
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
