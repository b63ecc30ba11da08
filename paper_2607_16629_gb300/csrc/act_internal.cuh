// Internal declarations shared by the translation units of libact
// (kernels, launchers, device helpers).  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/act.h"
#include "act_device.cuh"

namespace act {

// Launch on st; with pdl, as a programmatic dependent of the previous kernel
// in the stream (it may start while that kernel runs, and must execute
// griddepcontrol.wait in every CTA before it touches what that kernel
// writes and before it exits).  Between a kernel and an event node (or at a
// stream's first kernel) pdl has to be false.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                 bool pdl, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// launch_kernel for a 1-D cluster of cluster_x CTAs (grid a multiple of it).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_kernel_cluster(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                         bool pdl, int cluster_x, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster_x;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Device-side status flags (one int per grid, OR-ed by kernels).
enum : int {
    kFlagNonFinite = 1,
    kFlagTimeout = 2,
};

// Grid axes in the form kernels take by value.
struct GridAxes {
    double lo[4];    // tc, fc, logdt, c
    double step[4];
    int32_t count[4];
    double fs;
    int32_t L;       // samples per window
};

// value = lo + i * step with one rounding per operation (never fused), so
// the device gives the same doubles as plain host arithmetic.
__host__ __device__ inline double axis_value(double lo, double step, int64_t i) {
#ifdef __CUDA_ARCH__
    return __dadd_rn(lo, __dmul_rn((double)i, step));
#else
    volatile double m = (double)i * step;
    return lo + m;
#endif
}

// Flat index -> parameters (tc slowest, c fastest).
__host__ __device__ inline void decode_params(const GridAxes &ax, int64_t flat, double *p) {
    int64_t ic = flat % ax.count[3];
    int64_t rest = flat / ax.count[3];
    int64_t il = rest % ax.count[2];
    rest /= ax.count[2];
    int64_t ifc = rest % ax.count[1];
    int64_t itc = rest / ax.count[1];
    p[0] = axis_value(ax.lo[0], ax.step[0], itc);
    p[1] = axis_value(ax.lo[1], ax.step[1], ifc);
    p[2] = axis_value(ax.lo[2], ax.step[2], il);
    p[3] = axis_value(ax.lo[3], ax.step[3], ic);
}

// Packed selection key: |score| bits in the high word, (2^32-1 - index) in
// the low word, so that an unsigned max picks the largest |score| and, among
// equal scores, the lowest index.  0 means "nothing selected yet".
__device__ inline unsigned long long pack_key(float abs_score, uint32_t idx) {
    return ((unsigned long long)__float_as_uint(abs_score) << 32) |
           (unsigned long long)(0xFFFFFFFFu - idx);
}
__host__ __device__ inline uint32_t key_index(unsigned long long key) {
    return key ? 0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull) : 0u;
}

constexpr int kGemvThreads = 256;

// Every device allocation of the library goes through dev_alloc (act_api.cu),
// so that act_inject_alloc_failure can make one of them fail as if the
// device were out of memory.
cudaError_t dev_alloc(void **p, size_t bytes);
constexpr int kUpdateThreads = 256;
constexpr int kMaxSamples = 2048;
constexpr int kRowAlign = 128;   // FP32 row stride granule (floats)
constexpr int kBf16Align = 64;   // BF16 row stride granule (elements)

// ---- launchers (act_kernels.cu) -------------------------------------------
cudaError_t launch_gen_atoms(const GridAxes &ax, int64_t K, int Lp, float *d32, __nv_bfloat16 *d16,
                             int Lb, unsigned long long *degenerate, unsigned int *eps_bits, int sm_count,
                             cudaStream_t st);
cudaError_t launch_init(const float *sig, int B, int L, int Lp, float *R, __nv_bfloat16 *R16, int Lb,
                        unsigned long long *keys, double *energy, int P1, int *status, cudaStream_t st);
// wait_ns (here and below): limit of each bounded device-side wait.
cudaError_t launch_gemv_argmax(const float *D, int64_t K, int Lp, const float *R, int B,
                               const int *chlist, const int *count_dev, unsigned long long *keys,
                               int *status, int grid_ctas, cudaStream_t st,
                               unsigned long long wait_ns = kWaitLimitNs, bool pdl = false);
cudaError_t launch_project(const float *D, int64_t K, int Lp, const float *R, int B, float *scores,
                           int *status, int grid_ctas, cudaStream_t st, unsigned long long wait_ns = kWaitLimitNs);
cudaError_t launch_update(const float *D32, int Lp, int L, float *R, __nv_bfloat16 *R16, int Lb, int B,
                          unsigned long long *keys, const GridAxes &ax, int k, int P, act_atom *atoms,
                          float *coefs, double *energy, int *fb_count, cudaStream_t st, bool pdl = false);
// The whole decomposition over a small stored FP32 dictionary in one
// cooperative launch (act_fused.cu), results equal to the initialisation,
// GEMV and update kernels'.  sync holds 1 + 3B words (the barrier's count
// and abort flag, the key slots), cleared by the launcher; outputs may be
// null; resid rows are resid_stride apart.  One or two channels: from four
// channels on the per-order kernels measured faster (their GEMV scores four
// channels per pass over the rows, the single launch one).
constexpr int kFusedMaxB = 2;
// Dictionaries up to this size: there the single launch measured at least
// 5 % faster than the per-order kernels (1.4x at 16.8 MB); from 1 GB on the
// two are within 1.5 %, and larger dictionaries keep the TMA-fed GEMV.
constexpr int64_t kFusedMaxDictBytes = 512ll << 20;
int fused_max_ctas(int sm_count, int B, int Lp);  // co-resident CTAs of the launch (0: no launch form)
cudaError_t launch_mp_fused(const float *D, int64_t K, int Lp, int L, const float *sig, int B, int P,
                            const GridAxes &ax, unsigned long long *sync, act_atom *atoms, float *coefs,
                            double *energy, float *resid, int resid_stride, int *status, int ctas,
                            unsigned long long wait_ns, cudaStream_t st);
cudaError_t launch_ragged_gather(const float *src, const int64_t *src_off, int B, int L, float *dst, cudaStream_t st);
cudaError_t launch_ragged_scatter(int B, int P, int L, int Lp, const int *chan, const int64_t *dst_off,
                                  const act_atom *atoms, const float *coefs, const double *energy, const float *R,
                                  act_atom *out_atoms, float *out_coefs, double *out_energy, float *out_resid,
                                  cudaStream_t st);
// The same search with the dictionary streamed by TMA bulk copies through
// shared memory, one CTA per SM (act_gemv_stream.cu); same scores, same keys.
cudaError_t launch_gemv_stream_argmax(const float *D, int64_t K, int Lp, const float *R, int B, const int *chlist,
                                      const int *count_dev, unsigned long long *keys, int *status, int sm_count,
                                      cudaStream_t st, unsigned long long wait_ns = kWaitLimitNs, bool pdl = false);
int gemv_ctas(int sm_count, int Lp);          // occupancy-limited, at most 4 CTAs per SM
int gemv_max_ctas_per_sm(int Lp);

// ---- hierarchical search (act_lem.cu) -------------------------------------
struct LemBox {
    double lo[4], hi[4];
};
struct LemLevel {
    double step[4];
    int radius[4];
};
struct LemConfig {
    int n_coarse = 0;  // LHS samples of the coarse level
    int top_k = 4;
    int levels = 2;
    LemBox box;
    LemLevel level[3];
    uint64_t seed = 0;
};
struct LemBuffers {
    int cap = 0;                  // candidates per channel
    double *cand = nullptr;       // [B][cap][4]
    double *score = nullptr;      // [B][cap]
    double *kept = nullptr;       // [B][top_k][4]
    double *kept_score = nullptr; // [B][top_k]
    int *ncand = nullptr;         // [B]
    int *nkept = nullptr;         // [B]
};
cudaError_t launch_lem_select(const LemConfig &cfg, int B, int order, const float *R, int Lp, int L, double fs,
                              const LemBuffers &lb, cudaStream_t st);
int lem_kernels(const LemConfig &cfg);

// ---- off-grid refinement (act_refine.cu) ----------------------------------
cudaError_t launch_chirplet_score(int L, double fs, const double *theta, const float *R, int B, double *score,
                                  double *grad, float *atoms, cudaStream_t st);
// Start: theta_in[b * theta_in_stride ..] when theta_in is given, else the
// grid winner decoded from keys[b].
cudaError_t launch_refine(const GridAxes &ax, int steps, int Lp, const float *R, const unsigned long long *keys,
                          const double *theta_in, int theta_in_stride, int B, double *theta_out, cudaStream_t st);
cudaError_t launch_update_refined(int Lp, float *R, __nv_bfloat16 *R16, int Lb, int B, unsigned long long *keys,
                                  const GridAxes &ax, const double *theta, int k, int P, act_atom *atoms, float *coefs,
                                  double *energy, int *fb_count, cudaStream_t st);

// ---- template (shift-correlation) dictionary and search (act_shift.cu) ----
struct ShiftPlan {
    int S = 0, tc0 = 0;         // tc_j = tc0 + S j, whole samples
    int Sa = 0;                 // phases holding samples: min(S, L)
    int L = 0;                  // window length
    int Lp = 0;                 // residual row stride of the grid (floats)
    int Ntc = 0, NtcP = 0;      // lags, and lags rounded up to 32
    int P = 0;                  // polyphase length ceil(L / S) rounded up to 16
    int T = 0, TB = 0;          // templates (fc, logDt, c triples) and 32-template blocks
    int rows = 0;               // template rows per phase: NtcP + P - 1
    int64_t K = 0;
    int J = 0, W = 0, G = 0;    // lags per thread, warps per CTA, lag groups (NtcP / (W J))
    int NS = 0;                 // shared-memory stages of template chunks (1..3)
    int Kc = 0;                 // template rows per staged chunk: W J + P - 1
    size_t smem = 0;
    int ctas_per_sm = 0, ctas = 0;
    float *tpl = nullptr;       // [TB][Sa][rows][32]
    float *scale = nullptr;     // [TB][NtcP][32]
    // tensor-core view (act_shift_tc.cu): templates over m = n - tc in
    // [m_lo, m_lo + Kt) as BF16 rows, tile-major [T_pad / 256][Kt / 64][256][64]
    int m_lo = 0, Kt = 0, T_pad = 0;
    __nv_bfloat16 *tpl16 = nullptr;
    float *scaleT = nullptr;         // [NtcP][T_pad]
    unsigned int *eps_bits = nullptr;  // largest |bf16(u) - u| / |u| over the atoms (float bits)
};
// Layout of the template dictionary; cudaErrorNotSupported unless the tc
// axis is whole samples (lo and step integers, step >= 1).
cudaError_t shift_plan(ShiftPlan &sp, const GridAxes &ax);
bool shift_config_valid(const ShiftPlan &sp, int J, int W, int NS);
int shift_max_ctas_per_sm(const ShiftPlan &sp, int J, int W, int NS);
// ctas_per_sm <= 0: as many as fit.
cudaError_t shift_configure(ShiftPlan &sp, int J, int W, int NS, int sm_count, int ctas_per_sm);
cudaError_t shift_default_config(ShiftPlan &sp, int sm_count);
cudaError_t launch_shift_build(const ShiftPlan &sp, const GridAxes &ax, unsigned long long *degenerate, int sm_count,
                               cudaStream_t st);
// Selection into keys[] (packed, atomicMax; keys must be clear), or with
// scores != null every score written to scores[b * K + flat].  With
// early_launch the kernel is a programmatic dependent of the previous kernel
// in the stream (its prologue overlaps that kernel).  With count_dev, only
// the channels chlist[0 .. min(*count_dev, B)) are searched (the grid is
// sized for B; the count is read after the wait on the previous kernel).
cudaError_t launch_shift_search(const ShiftPlan &sp, const float *R, int Lp, int L, int B, unsigned long long *keys,
                                float *scores, int *status, bool early_launch, cudaStream_t st,
                                const int *chlist = nullptr, const int *count_dev = nullptr,
                                unsigned long long wait_ns = kWaitLimitNs);
// Coefficient and residual update (Eq. (4)) with the selected atom read back
// from its template; lets the next search launch early (programmatic
// dependent launch).
// counters (may be null): the tensor-core search's per-order queue lengths, reset.
cudaError_t launch_shift_update(const ShiftPlan &sp, const GridAxes &ax, int Lp, float *R, int B,
                                unsigned long long *keys, int k, int P, act_atom *atoms, float *coefs, double *energy,
                                int *counters, cudaStream_t st, bool pdl = false);

// ---- tensor-core template search (act_shift_tc.cu) -------------------------
// ShiftTc holds what a template build fixes (tensor maps of the BF16
// templates, pipeline depths); ShiftTcScratch the per-call buffers, owned by
// the work buffers of whoever launches (a grid, or one group of a ragged
// plan), so that graphs recorded on different work buffers share nothing
// that can be reallocated.
struct ShiftTc;
struct ShiftTcScratch {
    float *tile_max = nullptr;      // [rows][T_pad / 128]: per (row, template tile)
    float *blk_max = nullptr;       // [rows][T_pad / 32] maxima per 32-template block
    int *items = nullptr;           // [B_cap * 1024][2] flagged (channel, item) pairs
    __nv_bfloat16 *X = nullptr;     // [rows_alloc][Kt] shifted BF16 residual rows
    double2 *chan_norm = nullptr;   // [B_cap] |r|, |bf16(r) - r|
    unsigned int *chmax = nullptr;  // [B_cap] largest tile maximum (float bits)
    int *chcount = nullptr;         // [B_cap] items flagged this order
    int B_cap = 0;
    int rows_alloc = 0;
};
// Tensor maps and pipeline depth for the BF16 templates of sp (which must
// hold tpl16, scaleT and eps_bits); cudaErrorNotSupported without them.
cudaError_t shift_tc_prepare(ShiftTc **out, const ShiftPlan &sp, int sm_count);
void shift_tc_free(ShiftTc *s);
// Grows x to hold up to B channels (frees and reallocates: the caller drops
// every graph that captured x first).
cudaError_t shift_tc_reserve(const ShiftTc *s, const ShiftPlan &sp, int B, ShiftTcScratch &x);
void shift_tc_scratch_free(ShiftTcScratch &x);
// One search order: shifted residual rows + tcgen05 GEMM (tile maxima of the
// scaled scores), then item selection and FP32 rescore of the flagged items;
// a channel with too many flagged items is queued in fb_list and searched in
// full by the FP32 template search (launch_shift_search over the queue).
// Leaves the packed key of every channel in keys[]; counters[0..1] must be
// zero on entry.
// pdl: the first kernel of each call follows a kernel node directly (no
// event node between), so it may be a programmatic dependent; the kernels
// inside a call always are.
// Whether a B-channel launch runs the paired-SM GEMM.
bool shift_tc_uses_pairs(const ShiftTc *s, const ShiftPlan &sp, int B, bool pairs_allowed);
// pairs_allowed: the paired-SM GEMM (cta_group::2) may be chosen where it applies.
cudaError_t launch_shift_tc_gemm(const ShiftTc *s, const ShiftTcScratch &x, const ShiftPlan &sp, const float *R,
                                 int Lp, int L, int B, long long *stats, int *status, cudaStream_t st, bool pdl = false,
                                 unsigned long long wait_ns = kWaitLimitNs, bool pairs_allowed = true);
cudaError_t launch_shift_tc_resolve(const ShiftTc *s, const ShiftTcScratch &x, const ShiftPlan &sp, const float *R,
                                    int Lp, int L, int B, unsigned long long *keys, int *fb_list, int *counters,
                                    long long *stats, int *status, cudaStream_t st, bool pdl = false,
                                    unsigned long long wait_ns = kWaitLimitNs);

// ---- tensor-core search (act_gemm.cu) -------------------------------------
// Bf16Search holds what a BF16 dictionary build fixes (tensor maps, tile
// configuration); Bf16Scratch the per-call maxima and rescan lists, owned by
// the caller's work buffers (as ShiftTcScratch).
struct Bf16Search;
struct Bf16Scratch {
    float *tile_max = nullptr;  // [B_cap][K / 128 rounded up]
    float *blk_max = nullptr;   // [B_cap][K / 32 rounded up to whole 256-atom tiles]
    int *pairs = nullptr;       // [B_cap * 512][2] flagged (channel, block) pairs
    int B_cap = 0;
};
// Prepares the tensor-core search over the BF16 dictionary d16 [K][Lb]
// (tensor maps, tile configuration).  Returns cudaErrorNotSupported when the
// shape is outside what the kernel handles.
// eps_bits: device word holding (as float bits) the largest |bf16(g) - g|_2
// over the dictionary, written by the atom generator.
cudaError_t bf16_search_prepare(Bf16Search **out, const __nv_bfloat16 *d16, int64_t K, int Lb, int sm_count,
                                unsigned int *eps_bits);
void bf16_search_free(Bf16Search *s);
// Tile width (128 or 256 atoms) and pipeline depth of the GEMM; stages <= 0
// picks the deepest that fits.  Invalid combinations are rejected.
cudaError_t bf16_search_configure(Bf16Search *s, int bn, int stages);
void bf16_search_get_config(const Bf16Search *s, int *bn, int *stages, int *max_stages);
int bf16_search_max_stages(const Bf16Search *s, int bn);
// Grows x to hold up to B channels (frees and reallocates, as shift_tc_reserve).
cudaError_t bf16_scratch_reserve(const Bf16Search *s, int B, Bf16Scratch &x);
void bf16_scratch_free(Bf16Scratch &x);
// One search order for B channels (any number: 128-channel row tiles), in
// two launch sequences: the tensor-core GEMM writing per-tile and per-block
// maxima, then tile selection, FP32 rescan of the flagged blocks and the FP32
// full search for channels with too many of them.  Leaves the packed
// selection key of every channel in keys[].
cudaError_t launch_bf16_gemm(const Bf16Search *s, const Bf16Scratch &x, int B, const __nv_bfloat16 *R16, int *status,
                             cudaStream_t st, unsigned long long wait_ns = kWaitLimitNs);
cudaError_t launch_bf16_resolve(const Bf16Search *s, const Bf16Scratch &x, int B, const float *D32, int Lp, int L,
                                const float *R, unsigned long long *keys, int *fb_list, int *fb_count,
                                long long *stats, int *status, int gemv_grid, cudaStream_t st,
                                unsigned long long wait_ns = kWaitLimitNs);

}  // namespace act
