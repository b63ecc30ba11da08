// Template ("shift-correlation") dictionary and search.
//
// The real atom of Eq. (1) depends on the sample index n and the time centre
// tc only through m = n - tc.  On a grid whose tc values are whole samples,
// tc_j = tc0 + S j, every atom is therefore a window of one template
// u_t(m) per (fc, logDt, c) triple t, and the scores of all atoms that share
// t are a cross-correlation:
//     <r, u_{t, tc_j}> = sum_n r[n] u_t(n - tc0 - S j).
// Nothing of size K x L is stored: the templates (samples of u_t over the
// lags the window can see) and one FP32 scale 1/|u_{t,tc_j}| per atom are
// built once; the search forms every atom's samples in-kernel from its
// template held in shared memory.
//
// Polyphase form.  Writing n = a + S p (a = 0..Sa-1, Sa = min(S, L): a
// phase a >= L holds no sample) and k = p - j,
//     s_j = sum_a sum_p r_a[p] v_a[p - j],  r_a[p] = r[a + S p],
//                                           v_a[k] = u_t(a - tc0 + S k),
// one 1-D correlation per phase a with unit stride in p and j.
//
// Layouts (FP32):
//   templates [TB][Sa][rows][32]: block tb holds templates 32 tb .. 32 tb + 31
//     (lane = template), row rho holds k = rho - (NtcP - 1); rows =
//     NtcP + P - 1, NtcP = Ntc rounded up to 32, P = ceil(L / S) rounded up
//     to 16.  Zero for padding templates.
//   scales [TB][NtcP][32]: 1/|u| in FP32 from an FP64 sum over the window,
//     0 for a degenerate atom, a padding template or a padding lag.
// The flat index of (lag j, template t) is j T + t, the order of the grid.
//
// Search: persistent CTAs of W warps take units (channel b, lag group g of
// W J lags, template block tb).  Per unit and phase, one bulk copy brings
// the Kc = W J + P - 1 template rows the group needs into shared memory
// (two stages: the next copy is in flight while the current one is used).
// Warp w computes lags g W J + w J + q, q < J, for the block's 32 templates:
// each thread keeps J accumulators and a 2J-entry register ring of its
// template that slides by one row per p, so every p costs one shared load of
// the template (issued J steps ahead of its first use), a quarter of a
// broadcast 128-bit load of r_a and J FMAs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "act_device.cuh"
#include "act_ff.cuh"
#include "act_internal.cuh"
#include "act_update.cuh"

namespace act {

namespace {

constexpr int kShiftMaxThreads = 256;
constexpr int kShiftUpdateThreads = 512;
constexpr int kUpdatePerThread = kMaxSamples / kShiftUpdateThreads;
constexpr int kShiftMaxStages = 3;

struct ShiftArgs {
    const float *tpl;
    const float *scale;
    const float *R;
    int Lp, L, B;
    int S, Sa, P, T, TB, NtcP, Ntc, rows;
    int W, G, Kc, NS;
    int64_t K;
    unsigned long long *keys;
    float *scores;  // non-null: write every score to scores[b * K + flat] instead of selecting
    int *status;
    unsigned long long wait_ns;  // limit of each bounded wait
    // non-null: search only the channels chlist[0 .. *count_dev) (the count
    // is read after the wait on the previous kernel)
    const int *chlist;
    const int *count_dev;
};

// Template value u_t(m) at the integer lag m = n - tc: the dictionary
// generator's own sample routine at offset m, so on a grid of whole-sample
// time centres the template holds the unnormalised atom samples bit for bit.
__device__ __forceinline__ float template_sample(int m, const ChirpFF &k) {
    return chirp_sample_offset({(float)m, 0.0f}, k);
}

// One thread per (template block, phase, lane = template): the template's
// constants once, then its rows rho = 0 .. rows - 1 (lag k = rho - (NtcP - 1),
// m = a - tc0 + S k); a warp writes one 128-byte row per step.
__global__ void __launch_bounds__(256) k_shift_templates(GridAxes ax, int S, int Sa, int tc0, int NtcP, int rows,
                                                         int T, int64_t total, float *__restrict__ tpl) {
    const double inv_fs = 1.0 / ax.fs;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int lane = (int)(i & 31);
        const int64_t rest = i >> 5;
        const int a = (int)(rest % Sa);
        const int64_t tb = rest / Sa;
        const int64_t t = tb * 32 + lane;
        float *out = tpl + ((size_t)tb * Sa + a) * rows * 32 + lane;
        if (t < T) {
            double p[4];
            decode_params(ax, t, p);  // flat index t has i_tc = 0: p[1..3] are the template's axes
            const ChirpFF k = chirp_ff(0.0, inv_fs, p[1], p[3], exp(-p[2]));
            for (int rho = 0; rho < rows; ++rho) {
                const int m = a - tc0 + S * (rho - (NtcP - 1));
                out[(size_t)rho * 32] = template_sample(m, k);
            }
        } else {
            for (int rho = 0; rho < rows; ++rho) out[(size_t)rho * 32] = 0.0f;
        }
    }
}

// BF16 templates for the tensor-core search, tile-major like the BF16
// dictionary: element (t, kk) = bf16(u_t(m_lo + kk)) at
// [t / 256][kk / 64][t % 256][kk % 64]; zero for padding templates.  A warp
// takes 32 templates: lane l forms template l's constants once, then the
// warp writes the templates one after another, lane = kk stride 32.
__global__ void __launch_bounds__(256) k_shift_tpl16(GridAxes ax, int m_lo, int Kt, int T, int T_pad,
                                                     __nv_bfloat16 *__restrict__ tpl16) {
    const double inv_fs = 1.0 / ax.fs;
    const int nkc = Kt >> 6;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t0 = warp * 32; t0 < T_pad; t0 += nwarps * 32) {
        ChirpFF mine = {};
        if (t0 + lane < T) {
            double p[4];
            decode_params(ax, t0 + lane, p);
            mine = chirp_ff(0.0, inv_fs, p[1], p[3], exp(-p[2]));
        }
        for (int q = 0; q < 32; ++q) {
            const int64_t t = t0 + q;
            const ChirpFF k = chirp_ff_shfl(mine, q);
            for (int kk = lane; kk < Kt; kk += 32) {
                const float v = t < T ? template_sample(m_lo + kk, k) : 0.0f;
                const int64_t off = (((t >> 8) * nkc + (kk >> 6)) * 256 + (t & 255)) * 64 + (kk & 63);
                tpl16[off] = __float2bfloat16_rn(v);
            }
        }
    }
}

// One thread per (template block, lag, lane): |u|^2 over the window (a
// float-float sum),
// the scale 1/|u| in both layouts ([TB][NtcP][32] for the FP32 search,
// [NtcP][T_pad] for the tensor-core epilogue) and the largest relative BF16
// rounding error |bf16(u) - u| / |u| over all atoms (float bits, rounded up).
__global__ void __launch_bounds__(256) k_shift_scales(int S, int Sa, int L, int NtcP, int Ntc, int rows, int T,
                                                      int T_pad, int64_t total, const float *__restrict__ tpl,
                                                      float *__restrict__ scale, float *__restrict__ scaleT,
                                                      unsigned int *__restrict__ eps_bits,
                                                      unsigned long long *__restrict__ degenerate) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int lane = (int)(i & 31);
        const int64_t rest = i >> 5;
        const int j = (int)(rest % NtcP);
        const int64_t tb = rest / NtcP;
        const int64_t t = tb * 32 + lane;
        float sc = 0.0f;
        if (t < T && j < Ntc) {
            ff ef = {0.0f, 0.0f}, def = {0.0f, 0.0f};
            const float *base = tpl + (size_t)tb * Sa * rows * 32 + lane;
            // sample n = a + S p sits in phase a, row p - j + NtcP - 1
            for (int a = 0; a < Sa; ++a) {
                const float *col = base + ((size_t)a * rows + (NtcP - 1 - j)) * 32;
                for (int p = 0; a + S * p < L; ++p) {
                    const float u = col[(size_t)p * 32];
                    const float d = __bfloat162float(__float2bfloat16_rn(u)) - u;  // exact
                    ff_fma_acc(ef, u, u);
                    ff_fma_acc(def, d, d);
                }
            }
            const double e = ff_to_double(ef), de = ff_to_double(def);
            if (e > 0.0 && isfinite(e)) {
                sc = (float)(1.0 / sqrt(e));
                if (eps_bits)
                    atomicMax(eps_bits, __float_as_uint(__double2float_ru(sqrt(de / e) * (1.0 + 1e-6))));
            } else if (degenerate) {
                atomicAdd(degenerate, 1ull);
            }
        }
        scale[i] = sc;
        if (scaleT && t < T_pad) scaleT[(size_t)j * T_pad + t] = sc;
    }
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
        v = o > v ? o : v;
    }
    return v;
}

template <int J>
__global__ void __launch_bounds__(kShiftMaxThreads) k_shift_search(ShiftArgs A) {
    extern __shared__ __align__(128) float sm[];
    __shared__ __align__(8) uint64_t bar[kShiftMaxStages];
    __shared__ unsigned long long red[kShiftMaxThreads / 32];

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int W = A.W, NS = A.NS, Sa = A.Sa;
    // J slack rows: the look-ahead loads of the ring's last J steps
    const int stage_floats = (A.Kc + J + 1) * 32;
    float *rpoly = sm + NS * stage_floats;     // [Sa][P] + 4 slack floats, after the stages
    const int units_per_b = A.G * A.TB;
    int n_b = A.B;
    if (A.count_dev) {
        asm volatile("griddepcontrol.wait;" ::: "memory");
        n_b = min(*A.count_dev, A.B);
    }
    const int n_units = n_b * units_per_b;
    if ((int)blockIdx.x >= n_units) return;
    // chunk c of this CTA: phase c % Sa of its unit c / Sa
    const int my_units = (n_units - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    const int n_chunks = my_units * Sa;

    if (threadIdx.x == 0) {
        for (int i = 0; i < NS; ++i) mbar_init(&bar[i], 1);
        fence_mbar_init();
    }
    __syncthreads();

    const uint32_t chunk_bytes = (uint32_t)A.Kc * 32u * 4u;
    auto issue = [&](int cc) {  // thread 0 only
        if (cc >= n_chunks) return;
        const int u = (int)blockIdx.x + (cc / Sa) * (int)gridDim.x, a = cc % Sa;
        const int rem = u % units_per_b;
        const int g = rem / A.TB, tb = rem % A.TB;
        const int rho0 = A.NtcP - (g + 1) * W * J;
        const float *src = A.tpl + (((size_t)tb * Sa + a) * A.rows + rho0) * 32;
        const int s = cc % NS;
        mbar_expect_tx(&bar[s], chunk_bytes);
        bulk_g2s(sm + s * stage_floats, src, chunk_bytes, &bar[s]);
    };

    // prologue: chunks 0 .. NS-2 in flight; iteration c issues chunk c + NS - 1
    // into the stage that chunk c - 1 used (freed by the barrier ending it)
    if (threadIdx.x == 0)
        for (int i = 0; i + 1 < NS; ++i) issue(i);
    // Launched as a programmatic dependent of the previous update: everything
    // above (the templates are constant) overlaps it; the residuals and keys
    // it writes are read only after this wait.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    int cur_b = -1;
    unsigned long long best = 0ull;

    auto flush = [&](int b) {
        const unsigned long long v = warp_max_u64(best);
        if (lane == 0) red[w] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long m = 0ull;
            for (int i = 0; i < W; ++i) m = red[i] > m ? red[i] : m;
            if (m) atomicMax(A.keys + b, m);
        }
        best = 0ull;
    };

    int c = 0;  // chunks consumed by this CTA
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const int b = A.chlist ? A.chlist[u / units_per_b] : u / units_per_b;
        const int rem = u % units_per_b;
        const int g = rem / A.TB, tb = rem % A.TB;
        if (b != cur_b) {
            if (cur_b >= 0 && !A.scores) flush(cur_b);
            const float *r = A.R + (size_t)b * A.Lp;
            for (int i = threadIdx.x; i < Sa * A.P; i += blockDim.x) {
                const int a = i / A.P, p = i % A.P;
                const int n = a + A.S * p;
                rpoly[i] = n < A.L ? r[n] : 0.0f;
            }
            __syncthreads();
            cur_b = b;
        }
        const int t = tb * 32 + lane;
        const int j0 = g * W * J + w * J;
        const float *scl = A.scale + ((size_t)tb * A.NtcP + j0) * 32 + lane;
        float acc[J], sc[J];
#pragma unroll
        for (int q = 0; q < J; ++q) acc[q] = 0.0f;

        for (int a = 0; a < Sa; ++a, ++c) {
            if (threadIdx.x == 0) issue(c + NS - 1);
            if (a + 1 == Sa) {
                // the scales are needed after this phase: load them now
#pragma unroll
                for (int q = 0; q < J; ++q) sc[q] = scl[q * 32];
            }
            const int s = c % NS;
            const uint32_t parity = (uint32_t)((c / NS) & 1);
            const int ok = mbar_wait(&bar[s], parity, A.wait_ns);
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) {
                    atomicOr(A.status, kFlagTimeout);
                    // bounded: let the copies in flight land before exiting
                    for (int cc = c; cc < c + NS && cc < n_chunks; ++cc)
                        mbar_drain(&bar[cc % NS], (uint32_t)((cc / NS) & 1));
                }
                return;
            }
            const float *ts = sm + s * stage_floats + lane;
            const float4 *rp4 = reinterpret_cast<const float4 *>(rpoly + a * A.P);
            const int base = (W - w) * J - 1;  // chunk row of (p = 0, q = 0)
            // Register ring of M = 2J template rows: slot (rho - base) mod M
            // holds chunk row rho.  Step p uses rows base + p - q (q < J); the
            // oldest, base + p - J + 1, then dies and its slot takes row
            // base + p + J + 1, first used J steps later (load latency hidden).
            constexpr int M = 2 * J;
            float win[M];
#pragma unroll
            for (int d = 1 - J; d <= J; ++d) win[(d + M) % M] = ts[(base + d) * 32];
            float4 r_next = rp4[0];
            for (int pb = 0; pb < A.P; pb += M) {
#pragma unroll
                for (int i = 0; i < M; i += 4) {
                    const float4 r4 = r_next;
                    r_next = rp4[(pb + i + 4) >> 2];  // the next group of 4 steps (slack after the last)
                    const float rv[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
#pragma unroll
                        for (int q = 0; q < J; ++q) acc[q] = fmaf(rv[e], win[(i + e - q + M) % M], acc[q]);
                        win[(i + e + J + 1) % M] = ts[(base + pb + i + e + J + 1) * 32];
                    }
                }
            }
            __syncthreads();
        }

        // scores of this unit's atoms; the lowest lag wins ties (q ascending)
        if (t < A.T) {
#pragma unroll
            for (int q = 0; q < J; ++q) {
                const int j = j0 + q;
                if (j < A.Ntc) {
                    const float sv = acc[q] * sc[q];
                    const uint32_t flat = (uint32_t)j * (uint32_t)A.T + (uint32_t)t;
                    if (A.scores) {
                        A.scores[(size_t)b * A.K + flat] = sv;
                    } else {
                        const float x = fabsf(sv);
                        if (x == x) {
                            const unsigned long long key = pack_key(x, flat);
                            best = key > best ? key : best;
                        }
                    }
                }
            }
        }
    }
    if (cur_b >= 0 && !A.scores) flush(cur_b);
}

// One block per channel: the winner (j, t) of keys[b], g = scale * u_t
// read back from the template rows the search used, c = <g, r> (FP32),
// r -= c g, |r|^2 as a float-pair sum (returned in FP64), the atom record, the key cleared.
__global__ void __launch_bounds__(kShiftUpdateThreads) k_shift_update(const float *__restrict__ tpl,
                                                                     const float *__restrict__ scale,
                                                     int S, int Sa, int rows, int NtcP, int T, GridAxes ax, int Lp,
                                                     float *__restrict__ R, unsigned long long *__restrict__ keys,
                                                     int k, int P, act_atom *__restrict__ atoms,
                                                     float *__restrict__ coefs, double *__restrict__ energy,
                                                     int *__restrict__ counters) {
    // with a programmatic launch: the keys of the search before are read
    // only after it completes; the next search may launch now
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __shared__ float shf[32];
    __shared__ ff shp[32];
    const int b = blockIdx.x;
    const int L = ax.L;
    const uint32_t flat = key_index(keys[b]);
    const int j = (int)(flat / (uint32_t)T), t = (int)(flat % (uint32_t)T);
    const int tb = t >> 5, lane = t & 31;
    const float sc = scale[((size_t)tb * NtcP + j) * 32 + lane];
    const float *base = tpl + (size_t)tb * Sa * rows * 32 + lane;
    float *r = R + (size_t)b * Lp;
    // the atom's samples stay in registers between the two passes
    // (L <= kMaxSamples = kShiftUpdateThreads * kUpdatePerThread)
    float gv[kUpdatePerThread];
    float part = 0.0f;
#pragma unroll
    for (int i = 0; i < kUpdatePerThread; ++i) {
        const int n = threadIdx.x + i * kShiftUpdateThreads;
        gv[i] = 0.0f;
        if (n < L) {
            gv[i] = base[((size_t)(n % S) * rows + (n / S - j + NtcP - 1)) * 32] * sc;
            part = fmaf(gv[i], r[n], part);
        }
    }
    const float c = block_sum(part, shf);
    ff e2 = {0.0f, 0.0f};  // |r_{k+1}|^2 as a float pair (about 2^-44 relative)
#pragma unroll
    for (int i = 0; i < kUpdatePerThread; ++i) {
        const int n = threadIdx.x + i * kShiftUpdateThreads;
        if (n < L) {
            const float v = fmaf(-c, gv[i], r[n]);
            r[n] = v;
            ff_add_square(e2, v);
        }
    }
    const ff tot = block_sum_ff(e2, shp);
    if (threadIdx.x < 32) write_atom_lanes(ax, flat, atoms + (size_t)b * P + k);
    if (threadIdx.x == 0) {
        coefs[(size_t)b * P + k] = c;
        energy[(size_t)b * (P + 1) + k + 1] = ff_to_double(tot);
        keys[b] = 0ull;
        if (counters && b == 0) {
            counters[0] = 0;
            counters[1] = 0;
        }
    }
}

// The largest dynamic shared memory k_shift_search<J> was opted into, per
// device (the attribute belongs to the current device's context); it only
// grows, so graphs captured earlier keep a valid launch.
constexpr int kSmemDevices = 64;

template <int J>
cudaError_t set_smem(size_t smem) {
    static std::mutex mu;
    static size_t set[kSmemDevices] = {};
    if (smem <= 48 * 1024) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < kSmemDevices && smem <= set[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(k_shift_search<J>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && dev >= 0 && dev < kSmemDevices) set[dev] = smem;
    return e;
}

size_t shift_smem(const ShiftPlan &sp, int J, int W, int NS) {
    const int Kc = W * J + sp.P - 1;
    return sizeof(float) * ((size_t)NS * (Kc + J + 1) * 32 + (size_t)sp.Sa * sp.P + 4);
}

int shift_occupancy(int J, int W, size_t smem) {
    int per_sm = 0;
    cudaError_t e;
    switch (J) {
        case 8: e = set_smem<8>(smem); if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_shift_search<8>, 32 * W, smem); break;
        case 16: e = set_smem<16>(smem); if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_shift_search<16>, 32 * W, smem); break;
        case 32: e = set_smem<32>(smem); if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_shift_search<32>, 32 * W, smem); break;
        default: return 0;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm;
}

}  // namespace

int shift_max_ctas_per_sm(const ShiftPlan &sp, int J, int W, int NS) {
    if (!shift_config_valid(sp, J, W, NS)) return 0;
    return shift_occupancy(J, W, shift_smem(sp, J, W, NS));
}

bool shift_config_valid(const ShiftPlan &sp, int J, int W, int NS) {
    if (J != 8 && J != 16 && J != 32) return false;
    if (W < 1 || W > kShiftMaxThreads / 32) return false;
    if (NS < 1 || NS > kShiftMaxStages) return false;
    if (sp.NtcP % (W * J) != 0 || sp.P % (2 * J) != 0) return false;
    return shift_smem(sp, J, W, NS) <= 227 * 1024;
}

cudaError_t shift_plan(ShiftPlan &sp, const GridAxes &ax) {
    const double lo = ax.lo[0], step = ax.step[0];
    // whole-sample time centres only: tc0 and S integers, S >= 1
    if (!(step >= 1.0) || step != floor(step) || lo != floor(lo) || fabs(lo) > 1e9 || step > 1e6)
        return cudaErrorNotSupported;
    sp.S = (int)step;
    sp.Sa = sp.S < ax.L ? sp.S : ax.L;
    sp.L = ax.L;
    sp.tc0 = (int)lo;
    sp.Ntc = ax.count[0];
    sp.NtcP = (sp.Ntc + 31) / 32 * 32;
    sp.P = ((ax.L + sp.S - 1) / sp.S + 15) / 16 * 16;
    const int64_t T = (int64_t)ax.count[1] * ax.count[2] * ax.count[3];
    const int64_t K = T * ax.count[0];
    if (K >= 0xFFFFFFFFll || T > (1ll << 30)) return cudaErrorNotSupported;
    sp.T = (int)T;
    sp.TB = (int)((T + 31) / 32);
    sp.rows = sp.NtcP + sp.P - 1;
    sp.K = K;
    // tensor-core view: m = n - tc over [m_lo, m_hi], Kt = its length rounded up to 64
    const int64_t tc_last = (int64_t)sp.tc0 + (int64_t)sp.S * (sp.Ntc - 1);
    const int64_t m_lo = -tc_last, m_hi = (int64_t)ax.L - 1 - sp.tc0;
    const int64_t kt = (m_hi - m_lo + 1 + 63) / 64 * 64;
    sp.m_lo = (m_lo > -(1ll << 30)) ? (int)m_lo : 0;
    sp.Kt = kt <= (1 << 16) && m_lo > -(1ll << 30) ? (int)kt : 0;  // 0: no tensor-core view
    sp.T_pad = (int)((T + 255) / 256 * 256);
    return cudaSuccess;
}

cudaError_t shift_configure(ShiftPlan &sp, int J, int W, int NS, int sm_count, int ctas_per_sm) {
    if (!shift_config_valid(sp, J, W, NS)) return cudaErrorInvalidValue;
    const size_t smem = shift_smem(sp, J, W, NS);
    int per_sm = shift_occupancy(J, W, smem);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (ctas_per_sm > per_sm) return cudaErrorInvalidValue;
    if (ctas_per_sm > 0) per_sm = ctas_per_sm;
    sp.J = J;
    sp.W = W;
    sp.NS = NS;
    sp.G = sp.NtcP / (W * J);
    sp.Kc = W * J + sp.P - 1;
    sp.smem = smem;
    sp.ctas_per_sm = per_sm;
    sp.ctas = per_sm * sm_count;
    return cudaSuccess;
}

cudaError_t shift_default_config(ShiftPlan &sp, int sm_count) {
    // widest register window first, then the most warps that divide the lags
    static const int Js[] = {16, 32, 8};
    static const int Ws[] = {8, 4, 2, 1};
    for (int J : Js)
        for (int W : Ws)
            if (shift_config_valid(sp, J, W, 2) && shift_configure(sp, J, W, 2, sm_count, 0) == cudaSuccess)
                return cudaSuccess;
    return cudaErrorNotSupported;
}

cudaError_t launch_shift_build(const ShiftPlan &sp, const GridAxes &ax, unsigned long long *degenerate,
                               int sm_count, cudaStream_t st) {
    const int64_t nt = (int64_t)sp.TB * sp.Sa * 32;  // threads: (template block, phase, lane)
    int64_t blocks = (nt + 255) / 256;
    if (blocks > (int64_t)sm_count * 16) blocks = (int64_t)sm_count * 16;
    k_shift_templates<<<(int)blocks, 256, 0, st>>>(ax, sp.S, sp.Sa, sp.tc0, sp.NtcP, sp.rows, sp.T, nt, sp.tpl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t ns = (int64_t)sp.TB * sp.NtcP * 32;
    blocks = (ns + 255) / 256;
    if (blocks > (int64_t)sm_count * 16) blocks = (int64_t)sm_count * 16;
    k_shift_scales<<<(int)blocks, 256, 0, st>>>(sp.S, sp.Sa, ax.L, sp.NtcP, sp.Ntc, sp.rows, sp.T, sp.T_pad, ns,
                                                 sp.tpl, sp.scale, sp.scaleT, sp.eps_bits, degenerate);
    e = cudaGetLastError();
    if (e != cudaSuccess || !sp.tpl16) return e;
    blocks = ((int64_t)sp.T_pad + 255) / 256;  // 8 warps of 32 templates per block
    if (blocks > (int64_t)sm_count * 16) blocks = (int64_t)sm_count * 16;
    k_shift_tpl16<<<(int)blocks, 256, 0, st>>>(ax, sp.m_lo, sp.Kt, sp.T, sp.T_pad, sp.tpl16);
    return cudaGetLastError();
}

cudaError_t launch_shift_search(const ShiftPlan &sp, const float *R, int Lp, int L, int B, unsigned long long *keys,
                                float *scores, int *status, bool early_launch, cudaStream_t st, const int *chlist,
                                const int *count_dev, unsigned long long wait_ns) {
    if (sp.J == 0 || !sp.tpl || (count_dev && !chlist)) return cudaErrorInvalidValue;
    ShiftArgs A;
    A.tpl = sp.tpl;
    A.scale = sp.scale;
    A.R = R;
    A.Lp = Lp;
    A.L = L;
    A.B = B;
    A.S = sp.S;
    A.Sa = sp.Sa;
    A.P = sp.P;
    A.T = sp.T;
    A.TB = sp.TB;
    A.NtcP = sp.NtcP;
    A.Ntc = sp.Ntc;
    A.rows = sp.rows;
    A.W = sp.W;
    A.G = sp.G;
    A.Kc = sp.Kc;
    A.NS = sp.NS;
    A.K = sp.K;
    A.keys = keys;
    A.scores = scores;
    A.status = status;
    A.wait_ns = wait_ns;
    A.chlist = chlist;
    A.count_dev = count_dev;
    const int64_t units = (int64_t)B * sp.G * sp.TB;
    if (units > INT32_MAX) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(units < sp.ctas ? units : sp.ctas));
    cfg.blockDim = dim3(32u * sp.W);
    cfg.dynamicSmemBytes = sp.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = early_launch ? 1 : 0;
    switch (sp.J) {
        case 8: return cudaLaunchKernelEx(&cfg, k_shift_search<8>, A);
        case 16: return cudaLaunchKernelEx(&cfg, k_shift_search<16>, A);
        case 32: return cudaLaunchKernelEx(&cfg, k_shift_search<32>, A);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_shift_update(const ShiftPlan &sp, const GridAxes &ax, int Lp, float *R, int B,
                                unsigned long long *keys, int k, int P, act_atom *atoms, float *coefs, double *energy,
                                int *counters, cudaStream_t st, bool pdl) {
    return launch_kernel(k_shift_update, dim3(B), dim3(kShiftUpdateThreads), 0, st, pdl, sp.tpl, sp.scale, sp.S, sp.Sa,
                         sp.rows, sp.NtcP, sp.T, ax, Lp, R, keys, k, P, atoms, coefs, energy, counters);
}

}  // namespace act
