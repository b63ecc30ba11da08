// Host side of the C ABI declared in include/act.h: argument checks, grid
// and buffer ownership, dictionary build, and the n_atoms loop of the
// matching pursuit (Eq. (4), Fig. 1) captured once per shape as a CUDA
// graph and replayed on the caller's stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "act_internal.cuh"

using namespace act;

namespace {

thread_local char g_last_error[256] = "";

void note_error(const char *what, cudaError_t e) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
}

// Countdown to the device allocation that is to fail (act_inject_alloc_failure):
// n > 0 means the n-th dev_alloc from now fails; 0 means none.
std::atomic<int> g_fail_at{0};

#define ACT_CK(call)                                                        \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) {                                            \
            note_error(#call, e_);                                          \
            return e_ == cudaErrorMemoryAllocation ? ACT_ERR_OOM : ACT_ERR_CUDA; \
        }                                                                   \
    } while (0)

// Makes `dev` current for the lifetime of the guard.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Memory the kernels of device `dev` may read and write directly: that
// device's own allocations, or managed memory.
bool is_local_device_ptr(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

int round_up(int x, int g) { return (x + g - 1) / g * g; }

// FP32 row stride: the smallest instantiated GEMV width that holds L.
int fp32_stride(int L) {
    static const int widths[] = {128, 256, 384, 512, 1024, 2048};
    for (int w : widths)
        if (L <= w) return w;
    return -1;
}

struct GraphEntry {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;
    std::vector<cudaEvent_t> events;  // pairs around search launches (profiling)
};

template <typename T>
void free_dev(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

}  // namespace

namespace act {
cudaError_t dev_alloc(void **p, size_t bytes) {
    *p = nullptr;
    int n = g_fail_at.load();
    while (n > 0) {
        if (g_fail_at.compare_exchange_weak(n, n - 1)) {
            if (n == 1) return cudaErrorMemoryAllocation;
            break;
        }
    }
    return cudaMalloc(p, bytes);
}
}  // namespace act

// Per-decomposition device buffers: a grid owns one set, a ragged plan one
// per length group.  Invariant: a CUDA graph captures device addresses of
// exactly one WorkBuffers (the one it was recorded with) plus the grid's
// dictionary, templates, status and statistics words.  Only
// act_dictionary_build replaces the latter (it drops the grid's graphs and
// bumps its generation, which makes ragged plans stale); whoever reallocates
// any part of a WorkBuffers first destroys every graph recorded on it.
struct WorkBuffers {
    int cap_B = 0, cap_P = 0;
    float *sig = nullptr;             // [B][L] staged input signals
    float *R = nullptr;               // [B][Lp] FP32 residuals
    __nv_bfloat16 *R16 = nullptr;     // [ceil(B/128)*128][Lb] BF16 residuals
    unsigned long long *keys = nullptr;
    act_atom *atoms = nullptr;        // [B][P]
    float *coefs = nullptr;           // [B][P]
    double *energy = nullptr;         // [B][P+1]
    int *fb_list = nullptr;           // [B] channels queued for the FP32 full search
    int *fb_count = nullptr;          // [2] full-search and rescan queue lengths
    double *theta = nullptr;          // [B][4] refined parameters of the current order
    unsigned long long *fsync = nullptr;  // [1 + 3B] single-launch decomposition: barrier words, key slots
    LemBuffers lem;                   // hierarchical-search candidates (allocated on first use)
    int lem_B = 0;
    Bf16Scratch b16;                  // dense tensor-core search maxima and rescan lists (on first use)
    ShiftTcScratch stc;               // tensor-core template search rows, maxima, items (on first use)
};

struct act_grid {
    act_grid_desc desc;
    GridAxes ax;
    int device = 0;
    int sm_count = 0;
    int64_t K = 0;
    int L = 0, Lp = 0, Lb = 0;
    int built = -1;  // act_dict_mode of the current dictionary, -1 = none
    act_search_mode search = ACT_SEARCH_AUTO;
    float *d32 = nullptr;
    __nv_bfloat16 *d16 = nullptr;
    unsigned long long *degenerate = nullptr;
    unsigned int *eps_bits = nullptr;  // largest |bf16(g) - g| (float bits)
    WorkBuffers w;
    int *status = nullptr;
    long long *stats = nullptr;
    Bf16Search *bf16 = nullptr;
    ShiftPlan shift;       // template dictionary (ACT_DICT_RECOMPUTE)
    ShiftTc *shift_tc = nullptr;  // its tensor-core search (ACT_SEARCH_SHIFT_BF16)
    int gemv_grid = 0;
    bool gemv_stream = false;  // FP32 search by the bulk-copy streaming GEMV (one CTA per SM)
    int refine_steps = 0;  // BFGS iterations per order (0: grid-only search)
    unsigned long long wait_ns = kWaitLimitNs;  // limit of each bounded device-side wait
    bool cta_pairs = true;  // the tensor-core template GEMM may pair SMs (cta_group::2)
    int fused_ctas_per_sm = 2;  // single-launch decomposition of small FP32 dictionaries (0: off)
    bool coop = false;          // the device runs cooperative launches
    uint64_t mem_budget = 0;  // bytes ACT_DICT_AUTO may give the dictionary (0: free device memory)
    LemConfig lem;         // hierarchical search settings
    cudaStream_t cap = nullptr;
    bool profiling = false;
    std::map<std::tuple<int, int, int, int, int>, GraphEntry> graphs;
    GraphEntry *last = nullptr;
    uint64_t generation = 0;  // bumped whenever the dictionary or the launch configuration changes
};

namespace {

void drop_graphs(act_grid *g) {
    for (auto &kv : g->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
        for (cudaEvent_t e : kv.second.events) cudaEventDestroy(e);
    }
    g->graphs.clear();
    g->last = nullptr;
}

void free_lem(WorkBuffers &w) {
    free_dev(w.lem.cand);
    free_dev(w.lem.score);
    free_dev(w.lem.kept);
    free_dev(w.lem.kept_score);
    free_dev(w.lem.ncand);
    free_dev(w.lem.nkept);
    w.lem.cap = 0;
    w.lem_B = 0;
}

void free_base(WorkBuffers &w) {
    free_dev(w.sig);
    free_dev(w.R);
    free_dev(w.R16);
    free_dev(w.keys);
    free_dev(w.atoms);
    free_dev(w.coefs);
    free_dev(w.energy);
    free_dev(w.fb_list);
    free_dev(w.fb_count);
    free_dev(w.theta);
    free_dev(w.fsync);
    w.cap_B = w.cap_P = 0;
}

void free_work(WorkBuffers &w) {
    free_base(w);
    free_lem(w);
    bf16_scratch_free(w.b16);
    shift_tc_scratch_free(w.stc);
}

void free_dictionary(act_grid *g) {
    if (g->bf16) bf16_search_free(g->bf16);
    g->bf16 = nullptr;
    free_dev(g->d32);
    free_dev(g->d16);
    if (g->shift_tc) shift_tc_free(g->shift_tc);
    g->shift_tc = nullptr;
    free_dev(g->shift.tpl);
    free_dev(g->shift.scale);
    free_dev(g->shift.tpl16);
    free_dev(g->shift.scaleT);
    free_dev(g->shift.eps_bits);
    g->shift = ShiftPlan();
    g->built = -1;
    // the tensor-core search scratch is sized by the dictionary's shape
    bf16_scratch_free(g->w.b16);
    shift_tc_scratch_free(g->w.stc);
}

#define ACT_AL(ptr, bytes)                                                          \
    do {                                                                           \
        cudaError_t e_ = dev_alloc((void **)&(ptr), (bytes));                     \
        if (e_ != cudaSuccess) {                                                   \
            cudaGetLastError();                                                    \
            note_error("device allocation " #ptr, e_);                             \
            return e_ == cudaErrorMemoryAllocation ? ACT_ERR_OOM : ACT_ERR_CUDA;   \
        }                                                                          \
    } while (0)

// Work buffers for B channels and P orders on a grid of window L.  The BF16
// residual copy always has a multiple of 128 rows (the tensor-core tile
// height), padded with zeros.  On failure the caller frees what was made.
act_status alloc_base(const act_grid *g, WorkBuffers &w, int B, int P) {
    const int rows16 = round_up(B, 128);
    ACT_AL(w.sig, sizeof(float) * (size_t)B * g->L);
    ACT_AL(w.R, sizeof(float) * (size_t)B * g->Lp);
    ACT_AL(w.R16, sizeof(__nv_bfloat16) * (size_t)rows16 * g->Lb);
    ACT_CK(cudaMemset(w.R16, 0, sizeof(__nv_bfloat16) * (size_t)rows16 * g->Lb));
    ACT_AL(w.keys, sizeof(unsigned long long) * (size_t)B);
    ACT_CK(cudaMemset(w.keys, 0, sizeof(unsigned long long) * (size_t)B));
    ACT_AL(w.atoms, sizeof(act_atom) * (size_t)B * P);
    ACT_AL(w.coefs, sizeof(float) * (size_t)B * P);
    ACT_AL(w.energy, sizeof(double) * (size_t)B * (P + 1));
    ACT_AL(w.fb_list, sizeof(int) * (size_t)B);
    ACT_AL(w.fb_count, 2 * sizeof(int));
    ACT_CK(cudaMemset(w.fb_count, 0, 2 * sizeof(int)));
    ACT_AL(w.theta, sizeof(double) * 4 * (size_t)B);
    ACT_AL(w.fsync, sizeof(unsigned long long) * (1 + 3 * (size_t)B));
    w.cap_B = B;
    w.cap_P = P;
    return ACT_OK;
}

int lem_capacity(const LemConfig &c) {
    int per = 1;
    for (int a = 0; a < 4; ++a) per *= 2 * c.level[1].radius[a] + 1;
    int per2 = 1;
    for (int a = 0; a < 4; ++a) per2 *= 2 * c.level[2].radius[a] + 1;
    int cap = c.n_coarse;
    if (c.levels >= 1 && c.top_k * per > cap) cap = c.top_k * per;
    if (c.levels >= 2 && c.top_k * per2 > cap) cap = c.top_k * per2;
    return cap;
}

act_status alloc_lem(const act_grid *g, WorkBuffers &w, int B) {
    const int cap = lem_capacity(g->lem);
    const int k = g->lem.top_k;
    ACT_AL(w.lem.cand, sizeof(double) * 4 * (size_t)B * cap);
    ACT_AL(w.lem.score, sizeof(double) * (size_t)B * cap);
    ACT_AL(w.lem.kept, sizeof(double) * 4 * (size_t)B * k);
    ACT_AL(w.lem.kept_score, sizeof(double) * (size_t)B * k);
    ACT_AL(w.lem.ncand, sizeof(int) * (size_t)B);
    ACT_AL(w.lem.nkept, sizeof(int) * (size_t)B);
    w.lem.cap = cap;
    w.lem_B = B;
    return ACT_OK;
}

act_status scratch_status(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return ACT_OK;
    cudaGetLastError();
    note_error(what, e);
    return e == cudaErrorMemoryAllocation ? ACT_ERR_OOM : ACT_ERR_CUDA;
}

// Whether w holds everything `mode` needs for B channels and P orders.
bool work_fits(const act_grid *g, const WorkBuffers &w, int B, int P, act_search_mode mode) {
    if (B > w.cap_B || P > w.cap_P) return false;
    if (mode == ACT_SEARCH_LEM && (w.lem.cap < lem_capacity(g->lem) || w.lem_B < B || !w.lem.cand)) return false;
    if (mode == ACT_SEARCH_BF16 && w.b16.B_cap < B) return false;
    if (mode == ACT_SEARCH_SHIFT_BF16 && w.stc.B_cap < B) return false;
    return true;
}

// Grows w to what `mode` needs for B channels and P orders (each part to at
// least its current size).  The caller has destroyed every graph recorded
// on w.  On failure the parts that could not be made are left empty.
act_status grow_work(const act_grid *g, WorkBuffers &w, int B, int P, act_search_mode mode) {
    act_status s = ACT_OK;
    if (B > w.cap_B || P > w.cap_P) {
        const int nB = B > w.cap_B ? B : w.cap_B;
        const int nP = P > w.cap_P ? P : w.cap_P;
        free_base(w);
        if ((s = alloc_base(g, w, nB, nP)) != ACT_OK) {
            free_base(w);
            return s;
        }
    }
    if (mode == ACT_SEARCH_LEM && (w.lem.cap < lem_capacity(g->lem) || w.lem_B < B || !w.lem.cand)) {
        const int nB = B > w.lem_B ? B : w.lem_B;
        free_lem(w);
        if ((s = alloc_lem(g, w, nB)) != ACT_OK) {
            free_lem(w);
            return s;
        }
    }
    if (mode == ACT_SEARCH_BF16 && w.b16.B_cap < B) {
        if ((s = scratch_status(bf16_scratch_reserve(g->bf16, B, w.b16), "bf16_scratch_reserve")) != ACT_OK)
            return s;
    }
    if (mode == ACT_SEARCH_SHIFT_BF16 && w.stc.B_cap < B) {
        if ((s = scratch_status(shift_tc_reserve(g->shift_tc, g->shift, B, w.stc), "shift_tc_reserve")) != ACT_OK)
            return s;
    }
    return ACT_OK;
}

// The grid's own work buffers: any growth first destroys the grid's graphs,
// which captured their addresses.
act_status ensure_work(act_grid *g, int B, int P, act_search_mode mode) {
    if (work_fits(g, g->w, B, P, mode)) return ACT_OK;
    drop_graphs(g);
    return grow_work(g, g->w, B, P, mode);
}

// Hierarchical-search settings from the public struct; the box is the
// grid's range on every axis.
act_status lem_configure(act_grid *g, const act_lem_params *p) {
    LemConfig c;
    if (p->top_k < 1 || p->top_k > 16 || p->levels < 0 || p->levels > 2) return ACT_ERR_INVALID_ARG;
    const act_axis *axes[4] = {&g->desc.tc, &g->desc.fc, &g->desc.logdt, &g->desc.c};
    double n_est = 1.0;
    for (int a = 0; a < 4; ++a) {
        const double first = axes[a]->lo, last = axes[a]->lo + (double)(axes[a]->count - 1) * axes[a]->step;
        c.box.lo[a] = fmin(first, last);
        c.box.hi[a] = fmax(first, last);
        for (int l = 0; l < 3; ++l) {
            if (!(p->steps[l][a] > 0.0) || !isfinite(p->steps[l][a])) return ACT_ERR_INVALID_ARG;
            c.level[l].step[a] = p->steps[l][a];
            c.level[l].radius[a] = p->radius[a];
        }
        if (p->radius[a] < 0 || p->radius[a] > 8) return ACT_ERR_INVALID_ARG;
        const double cnt = ceil((c.box.hi[a] - c.box.lo[a]) / p->steps[0][a]);
        n_est *= cnt > 1.0 ? cnt : 1.0;
    }
    c.n_coarse = p->n_coarse > 0 ? p->n_coarse : (n_est > 16384.0 ? 16384 : (int)n_est);
    if (c.n_coarse < 1 || c.n_coarse > 16384) return ACT_ERR_UNSUPPORTED;
    c.top_k = p->top_k;
    c.levels = p->levels;
    c.seed = p->seed;
    if (lem_capacity(c) > (1 << 20)) return ACT_ERR_UNSUPPORTED;
    g->lem = c;
    return ACT_OK;
}

act_search_mode effective_search(const act_grid *g) {
    if (g->search != ACT_SEARCH_AUTO) return g->search;
    if (g->built == ACT_DICT_BF16) return ACT_SEARCH_BF16;
    if (g->built == ACT_DICT_RECOMPUTE) return g->shift_tc ? ACT_SEARCH_SHIFT_BF16 : ACT_SEARCH_SHIFT;
    return ACT_SEARCH_FP32;
}

// Whether the grid holds what `mode` searches.
bool search_available(const act_grid *g, act_search_mode mode) {
    switch (mode) {
        case ACT_SEARCH_LEM: return true;
        case ACT_SEARCH_FP32: return g->d32 != nullptr;
        case ACT_SEARCH_BF16: return g->bf16 != nullptr && g->d16 != nullptr;
        case ACT_SEARCH_SHIFT: return g->shift.tpl != nullptr;
        case ACT_SEARCH_SHIFT_BF16: return g->shift_tc != nullptr;
        default: return false;
    }
}

// CTAs of the single-launch decomposition of B channels, or 0 where it does
// not apply: the FP32 search over a stored dictionary small enough to stay
// in L2, grid-only (no refinement), at most kFusedMaxB channels, no
// per-order profiling events, a device that runs cooperative launches.
int fused_ctas(const act_grid *g, int B, act_search_mode mode, bool profiling) {
    if (g->fused_ctas_per_sm <= 0 || !g->coop || profiling || mode != ACT_SEARCH_FP32 || !g->d32) return 0;
    if (g->refine_steps > 0 || B < 1 || B > kFusedMaxB) return 0;
    if (g->K * (int64_t)g->Lp * (int64_t)sizeof(float) > kFusedMaxDictBytes) return 0;
    const int most = fused_max_ctas(g->sm_count, B, g->Lp);
    const int want = g->sm_count * g->fused_ctas_per_sm;
    return want < most ? want : most;
}

// Records the whole decomposition (init + P orders) on stream st (being captured).
act_status record_decompose(act_grid *g, WorkBuffers &w, int B, int P, act_search_mode mode, GraphEntry &ge,
                            cudaStream_t st, bool profiling, bool allow_fused) {
    const bool bf16 = mode == ACT_SEARCH_BF16;
    __nv_bfloat16 *R16 = bf16 ? w.R16 : nullptr;
    int kernels = 0;
    const int fctas = allow_fused ? fused_ctas(g, B, mode, profiling) : 0;
    if (fctas > 0) {  // the single-launch form (it also initialises the residuals)
        ACT_CK(launch_mp_fused(g->d32, g->K, g->Lp, g->L, w.sig, B, P, g->ax, w.fsync, w.atoms, w.coefs, w.energy,
                               w.R, g->Lp, g->status, fctas, g->wait_ns, st));
        ge.kernels = 1;
        return ACT_OK;
    }
    ACT_CK(launch_init(w.sig, B, g->L, g->Lp, w.R, R16, g->Lb, w.keys, w.energy, P + 1, g->status, st));
    ++kernels;
    for (int k = 0; k < P; ++k) {
        // profiling: events before the search, after its dominant kernel
        // (GEMV or GEMM) and after the whole search
        cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
        if (profiling) {
            for (int i = 0; i < 3; ++i) {
                ACT_CK(cudaEventCreate(&ev[i]));
                ge.events.push_back(ev[i]);
            }
            ACT_CK(cudaEventRecordWithFlags(ev[0], st, cudaEventRecordExternal));
        }
        if (mode == ACT_SEARCH_LEM) {
            ACT_CK(launch_lem_select(g->lem, B, k, w.R, g->Lp, g->L, g->desc.fs, w.lem, st));
            if (profiling) ACT_CK(cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal));
            kernels += lem_kernels(g->lem);
        } else if (mode == ACT_SEARCH_SHIFT) {
            // early launch only between kernel nodes (not after profiling events)
            ACT_CK(launch_shift_search(g->shift, w.R, g->Lp, g->L, B, w.keys, nullptr, g->status, !profiling, st,
                                       nullptr, nullptr, g->wait_ns));
            if (profiling) ACT_CK(cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal));
            kernels += 1;
        } else if (mode == ACT_SEARCH_SHIFT_BF16) {
            // programmatic dependents between kernel nodes only (not next to profiling events)
            ACT_CK(launch_shift_tc_gemm(g->shift_tc, w.stc, g->shift, w.R, g->Lp, g->L, B, g->stats, g->status, st,
                                        !profiling, g->wait_ns, g->cta_pairs));
            if (profiling) ACT_CK(cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal));
            ACT_CK(launch_shift_tc_resolve(g->shift_tc, w.stc, g->shift, w.R, g->Lp, g->L, B, w.keys, w.fb_list,
                                           w.fb_count, g->stats, g->status, st, !profiling, g->wait_ns));
            kernels += 5;
        } else if (bf16) {
            ACT_CK(launch_bf16_gemm(g->bf16, w.b16, B, w.R16, g->status, st, g->wait_ns));
            if (profiling) ACT_CK(cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal));
            ACT_CK(launch_bf16_resolve(g->bf16, w.b16, B, g->d32, g->Lp, g->L, w.R, w.keys, w.fb_list, w.fb_count,
                                       g->stats, g->status, g->gemv_grid, st, g->wait_ns));
            kernels += 4;
        } else {
            // programmatic dependents between kernel nodes only (not next to profiling events)
            if (g->gemv_stream)
                ACT_CK(launch_gemv_stream_argmax(g->d32, g->K, g->Lp, w.R, B, nullptr, nullptr, w.keys, g->status,
                                                 g->sm_count, st, g->wait_ns, !profiling));
            else
                ACT_CK(launch_gemv_argmax(g->d32, g->K, g->Lp, w.R, B, nullptr, nullptr, w.keys, g->status,
                                          g->gemv_grid, st, g->wait_ns, !profiling));
            if (profiling) ACT_CK(cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal));
            kernels += 1;
        }
        if (profiling) ACT_CK(cudaEventRecordWithFlags(ev[2], st, cudaEventRecordExternal));
        if (mode == ACT_SEARCH_LEM) {
            // the best hierarchical candidate starts the (optional) BFGS refinement
            ACT_CK(launch_refine(g->ax, g->refine_steps, g->Lp, w.R, nullptr, w.lem.kept, 4 * g->lem.top_k, B,
                                 w.theta, st));
            ACT_CK(launch_update_refined(g->Lp, w.R, nullptr, g->Lb, B, nullptr, g->ax, w.theta, k, P, w.atoms,
                                         w.coefs, w.energy, nullptr, st));
            kernels += 2;
        } else if (g->refine_steps > 0) {
            ACT_CK(launch_refine(g->ax, g->refine_steps, g->Lp, w.R, w.keys, nullptr, 0, B, w.theta, st));
            ACT_CK(launch_update_refined(g->Lp, w.R, R16, g->Lb, B, w.keys, g->ax, w.theta, k, P, w.atoms, w.coefs,
                                         w.energy, bf16 || mode == ACT_SEARCH_SHIFT_BF16 ? w.fb_count : nullptr, st));
            kernels += 2;
        } else if (mode == ACT_SEARCH_SHIFT || mode == ACT_SEARCH_SHIFT_BF16) {
            // no stored rows: the selected atom is read back from its template
            ACT_CK(launch_shift_update(g->shift, g->ax, g->Lp, w.R, B, w.keys, k, P, w.atoms, w.coefs, w.energy,
                                       mode == ACT_SEARCH_SHIFT_BF16 ? w.fb_count : nullptr, st, !profiling));
            ++kernels;
        } else {
            ACT_CK(launch_update(g->d32, g->Lp, g->L, w.R, R16, g->Lb, B, w.keys, g->ax, k, P, w.atoms, w.coefs,
                                 w.energy, bf16 ? w.fb_count : nullptr, st, !profiling));
            ++kernels;
        }
    }
    ge.kernels = kernels;
    return ACT_OK;
}

act_status get_graph(act_grid *g, int B, int P, act_search_mode mode, GraphEntry **out) {
    auto key = std::make_tuple(B, P, (int)mode, g->profiling ? 1 : 0, g->refine_steps);
    auto it = g->graphs.find(key);
    if (it != g->graphs.end()) {
        *out = &it->second;
        return ACT_OK;
    }
    GraphEntry ge;
    ACT_CK(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
    act_status s = record_decompose(g, g->w, B, P, mode, ge, g->cap, g->profiling, true);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(g->cap, &graph);
    if (s != ACT_OK) {
        if (graph) cudaGraphDestroy(graph);
        for (cudaEvent_t ev : ge.events) cudaEventDestroy(ev);
        return s;
    }
    if (e != cudaSuccess) {
        note_error("cudaStreamEndCapture", e);
        for (cudaEvent_t ev : ge.events) cudaEventDestroy(ev);
        return ACT_ERR_CUDA;
    }
    ge.graph = graph;
    e = cudaGraphInstantiate(&ge.exec, graph, 0);
    if (e != cudaSuccess) {
        note_error("cudaGraphInstantiate", e);
        cudaGraphDestroy(graph);
        for (cudaEvent_t ev : ge.events) cudaEventDestroy(ev);
        return ACT_ERR_CUDA;
    }
    auto res = g->graphs.emplace(key, ge);
    *out = &res.first->second;
    return ACT_OK;
}

act_status copy_out(void *dst, const void *src, size_t bytes, cudaStream_t st, bool *host_seen) {
    if (!dst) return ACT_OK;
    if (!is_device_ptr(dst)) *host_seen = true;
    ACT_CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
    return ACT_OK;
}

}  // namespace

extern "C" {

const char *act_status_string(act_status s) {
    switch (s) {
        case ACT_OK: return "ACT_OK";
        case ACT_ERR_INVALID_ARG: return "ACT_ERR_INVALID_ARG";
        case ACT_ERR_OOM: return "ACT_ERR_OOM";
        case ACT_ERR_CUDA: return "ACT_ERR_CUDA";
        case ACT_ERR_NONFINITE: return "ACT_ERR_NONFINITE";
        case ACT_ERR_DEVICE_TIMEOUT: return "ACT_ERR_DEVICE_TIMEOUT";
        case ACT_ERR_NOT_BUILT: return "ACT_ERR_NOT_BUILT";
        case ACT_ERR_UNSUPPORTED: return "ACT_ERR_UNSUPPORTED";
    }
    return "ACT_ERR_UNKNOWN";
}

const char *act_last_error_message(void) { return g_last_error; }

static int64_t half_open_count(const double *r) {
    // Values start, start + step, ... strictly below stop.
    const double span = (r[1] - r[0]) / r[2];
    const double n = ceil(span);
    return n > 0.0 ? (int64_t)n : 0;
}

act_status act_grid_from_ranges(int32_t n_samples, double fs, const double tc[3], const double fc[3],
                                const double logdt[3], const double c[3], act_grid_desc *out) {
    if (!tc || !fc || !logdt || !c || !out) return ACT_ERR_INVALID_ARG;
    if (n_samples < 1 || n_samples > kMaxSamples || !(fs > 0.0)) return ACT_ERR_INVALID_ARG;
    const double *rs[4] = {tc, fc, logdt, c};
    act_axis *axes[4] = {&out->tc, &out->fc, &out->logdt, &out->c};
    for (int i = 0; i < 4; ++i) {
        if (!(rs[i][2] > 0.0) || !isfinite(rs[i][0]) || !isfinite(rs[i][1])) return ACT_ERR_INVALID_ARG;
        const int64_t n = half_open_count(rs[i]);
        if (n < 1 || n > INT32_MAX) return ACT_ERR_INVALID_ARG;
    }
    out->n_samples = n_samples;
    out->fs = fs;
    for (int i = 0; i < 4; ++i) {
        axes[i]->lo = rs[i][0];
        axes[i]->step = rs[i][2];
        axes[i]->count = (int32_t)half_open_count(rs[i]);
    }
    return ACT_OK;
}

act_status act_grid_create(const act_grid_desc *desc, int32_t device, act_grid **out) {
    if (!desc || !out) return ACT_ERR_INVALID_ARG;
    *out = nullptr;
    if (desc->n_samples < 1 || desc->n_samples > kMaxSamples || !(desc->fs > 0.0) || !isfinite(desc->fs))
        return ACT_ERR_INVALID_ARG;
    const act_axis *axes[4] = {&desc->tc, &desc->fc, &desc->logdt, &desc->c};
    int64_t K = 1;
    for (int i = 0; i < 4; ++i) {
        if (axes[i]->count < 1 || !isfinite(axes[i]->lo) || !isfinite(axes[i]->step)) return ACT_ERR_INVALID_ARG;
        K *= axes[i]->count;
        if (K > (int64_t)0xFFFFFFFEll) return ACT_ERR_INVALID_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        snprintf(g_last_error, sizeof(g_last_error), "no CUDA device %d", device);
        return ACT_ERR_CUDA;
    }
    DeviceGuard dg(device);
    if (!dg.ok) return ACT_ERR_CUDA;
    act_grid *g = new (std::nothrow) act_grid();
    if (!g) return ACT_ERR_OOM;
    g->desc = *desc;
    g->device = device;
    g->K = K;
    g->L = desc->n_samples;
    g->Lp = fp32_stride(g->L);
    g->Lb = round_up(g->L, kBf16Align);
    for (int i = 0; i < 4; ++i) {
        g->ax.lo[i] = axes[i]->lo;
        g->ax.step[i] = axes[i]->step;
        g->ax.count[i] = axes[i]->count;
    }
    g->ax.fs = desc->fs;
    g->ax.L = g->L;
    cudaError_t e = cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, device);
    int coop = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
    g->coop = coop != 0;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = dev_alloc((void **)&g->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(g->status, 0, sizeof(int));
    if (e == cudaSuccess) e = dev_alloc((void **)&g->stats, 3 * sizeof(long long));
    if (e == cudaSuccess) e = cudaMemset(g->stats, 0, 3 * sizeof(long long));
    if (e == cudaSuccess) e = dev_alloc((void **)&g->degenerate, sizeof(unsigned long long));
    if (e == cudaSuccess) e = dev_alloc((void **)&g->eps_bits, sizeof(unsigned int));
    if (e != cudaSuccess) {
        note_error("act_grid_create", e);
        act_destroy(g);
        return e == cudaErrorMemoryAllocation ? ACT_ERR_OOM : ACT_ERR_CUDA;
    }
    g->gemv_grid = gemv_ctas(g->sm_count, g->Lp);
    act_lem_params lp;
    memset(&lp, 0, sizeof(lp));
    lp.top_k = 4;
    lp.levels = 2;
    const double paper_steps[3][4] = {{64, 2, 2, 5}, {32, 1, 1, 2.5}, {16, 0.5, 0.5, 0.5}};
    for (int l = 0; l < 3; ++l)
        for (int a = 0; a < 4; ++a) lp.steps[l][a] = paper_steps[l][a];
    lp.radius[0] = 2;
    lp.radius[1] = 2;
    lp.radius[2] = 1;
    lp.radius[3] = 2;
    if (lem_configure(g, &lp) != ACT_OK) {  // a grid whose box needs more coarse samples: cap them
        lp.n_coarse = 16384;
        lem_configure(g, &lp);
    }
    *out = g;
    return ACT_OK;
}

act_status act_grid_size(const act_grid *g, int64_t *n_atoms, int32_t *row_stride) {
    if (!g) return ACT_ERR_INVALID_ARG;
    if (n_atoms) *n_atoms = g->K;
    if (row_stride) *row_stride = g->Lp;
    return ACT_OK;
}

// Template dictionary: per (fc, logDt, c) the samples the window can see,
// and one FP32 scale per atom.
static act_status build_templates(act_grid *g, cudaStream_t st) {
    ShiftPlan sp;
    if (shift_plan(sp, g->ax) != cudaSuccess) return ACT_ERR_UNSUPPORTED;
    sp.Lp = g->Lp;
    if (shift_default_config(sp, g->sm_count) != cudaSuccess) return ACT_ERR_UNSUPPORTED;
    const size_t bt = sizeof(float) * (size_t)sp.TB * sp.Sa * sp.rows * 32;
    const size_t bs = sizeof(float) * (size_t)sp.TB * sp.NtcP * 32;
    cudaError_t e = dev_alloc((void **)&sp.tpl, bt);
    if (e == cudaSuccess) e = dev_alloc((void **)&sp.scale, bs);
    if (e == cudaSuccess && sp.Kt > 0) {
        // the tensor-core view: BF16 templates, transposed scales, BF16 error bound
        const size_t b16 = sizeof(__nv_bfloat16) * (size_t)sp.T_pad * sp.Kt;
        const size_t bst = sizeof(float) * (size_t)sp.NtcP * sp.T_pad;
        e = dev_alloc((void **)&sp.tpl16, b16);
        if (e == cudaSuccess) e = dev_alloc((void **)&sp.scaleT, bst);
        if (e == cudaSuccess) e = dev_alloc((void **)&sp.eps_bits, sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemsetAsync(sp.scaleT, 0, bst, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(sp.eps_bits, 0, sizeof(unsigned int), st);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_dev(sp.tpl);
        free_dev(sp.scale);
        free_dev(sp.tpl16);
        free_dev(sp.scaleT);
        free_dev(sp.eps_bits);
        note_error("template dictionary", e);
        return ACT_ERR_OOM;
    }
    g->shift = sp;
    ACT_CK(cudaMemsetAsync(g->degenerate, 0, sizeof(unsigned long long), st));
    ACT_CK(launch_shift_build(g->shift, g->ax, g->degenerate, g->sm_count, st));
    g->built = ACT_DICT_RECOMPUTE;
    if (sp.tpl16 && shift_tc_prepare(&g->shift_tc, g->shift, g->sm_count) != cudaSuccess) {
        cudaGetLastError();
        g->shift_tc = nullptr;  // the FP32 template search stays available
    }
    return ACT_OK;
}

// Device bytes of the template dictionary of g (0 when its time centres are
// not whole samples).
static uint64_t template_bytes(const act_grid *g) {
    ShiftPlan sp;
    if (shift_plan(sp, g->ax) != cudaSuccess) return 0;
    uint64_t b = sizeof(float) * ((uint64_t)sp.TB * sp.Sa * sp.rows * 32 + (uint64_t)sp.TB * sp.NtcP * 32);
    if (sp.Kt > 0) b += sizeof(__nv_bfloat16) * (uint64_t)sp.T_pad * sp.Kt + sizeof(float) * (uint64_t)sp.NtcP * sp.T_pad;
    return b;
}

// ACT_DICT_AUTO: the FP32 rows when they fit the memory budget, else the
// template dictionary when the time centres are whole samples (Sec. IV-C
// pages a dictionary larger than VRAM through unified memory instead).
static act_status resolve_auto(act_grid *g, act_dict_mode *mode) {
    uint64_t budget = g->mem_budget;
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        ACT_CK(cudaMemGetInfo(&fr, &tot));
        budget = (uint64_t)((double)fr * 0.9);
    }
    const uint64_t b32 = sizeof(float) * (uint64_t)g->K * (uint64_t)g->Lp;
    if (b32 <= budget) {
        *mode = ACT_DICT_FP32;
        return ACT_OK;
    }
    const uint64_t bt = template_bytes(g);
    if (bt > 0 && bt <= budget) {
        *mode = ACT_DICT_RECOMPUTE;
        return ACT_OK;
    }
    snprintf(g_last_error, sizeof(g_last_error),
             "ACT_DICT_AUTO: %llu bytes of FP32 rows exceed the budget of %llu bytes and %s",
             (unsigned long long)b32, (unsigned long long)budget,
             bt ? "so does the template dictionary" : "the time centres are not whole samples (no template form)");
    return ACT_ERR_OOM;
}

act_status act_dictionary_build(act_grid *g, act_dict_mode mode, void *cuda_stream) {
    if (!g) return ACT_ERR_INVALID_ARG;
    if (mode != ACT_DICT_AUTO && mode != ACT_DICT_FP32 && mode != ACT_DICT_BF16 && mode != ACT_DICT_RECOMPUTE)
        return ACT_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    ACT_CK(cudaStreamSynchronize(st));
    drop_graphs(g);
    ++g->generation;  // ragged plans built on the old dictionary are stale
    free_dictionary(g);
    if (mode == ACT_DICT_AUTO) {
        const act_status s = resolve_auto(g, &mode);
        if (s != ACT_OK) return s;
    }
    if (mode == ACT_DICT_RECOMPUTE) return build_templates(g, st);
    const size_t b32 = sizeof(float) * (size_t)g->K * g->Lp;
    cudaError_t e = dev_alloc((void **)&g->d32, b32);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g->d32 = nullptr;
        note_error("dictionary (FP32)", e);
        return ACT_ERR_OOM;
    }
    if (mode == ACT_DICT_BF16) {
        // tile-major layout [K/256 tiles][Lb/64 chunks][256 atoms][64 samples],
        // the last tile padded with zero atoms
        const int64_t ntiles = (g->K + 255) / 256;
        const size_t b16 = sizeof(__nv_bfloat16) * (size_t)ntiles * 256 * g->Lb;
        e = dev_alloc((void **)&g->d16, b16);
        if (e == cudaSuccess) e = cudaMemset(g->d16, 0, b16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            g->d16 = nullptr;
            free_dictionary(g);
            note_error("dictionary (BF16)", e);
            return ACT_ERR_OOM;
        }
    }
    ACT_CK(cudaMemsetAsync(g->degenerate, 0, sizeof(unsigned long long), st));
    ACT_CK(cudaMemsetAsync(g->eps_bits, 0, sizeof(unsigned int), st));
    ACT_CK(launch_gen_atoms(g->ax, g->K, g->Lp, g->d32, g->d16, g->Lb, g->degenerate, g->eps_bits, g->sm_count,
                            st));
    if (mode == ACT_DICT_BF16) {
        cudaError_t pe = bf16_search_prepare(&g->bf16, g->d16, g->K, g->Lb, g->sm_count, g->eps_bits);
        if (pe != cudaSuccess) {
            note_error("bf16_search_prepare", pe);
            free_dictionary(g);
            return pe == cudaErrorNotSupported ? ACT_ERR_UNSUPPORTED : ACT_ERR_CUDA;
        }
    }
    g->built = mode;
    return ACT_OK;
}

act_status act_set_lem(act_grid *g, const act_lem_params *params) {
    if (!g || !params) return ACT_ERR_INVALID_ARG;
    act_status s = lem_configure(g, params);
    if (s != ACT_OK) return s;
    drop_graphs(g);
    ++g->generation;
    return ACT_OK;
}

act_status act_set_search(act_grid *g, act_search_mode mode) {
    if (!g || (int)mode < 0 || (int)mode > 5) return ACT_ERR_INVALID_ARG;
    g->search = mode;
    return ACT_OK;
}

act_status act_decompose(act_grid *g, const float *signals, int32_t channels, int32_t n_atoms,
                         act_atom *atoms_out, float *coeffs_out, float *residuals_out, double *energy_out,
                         void *cuda_stream) {
    if (!g || !signals || channels < 1 || n_atoms < 1) return ACT_ERR_INVALID_ARG;
    const act_search_mode mode = effective_search(g);
    if (!search_available(g, mode)) return ACT_ERR_NOT_BUILT;
    if (mode == ACT_SEARCH_LEM && n_atoms > 4096) return ACT_ERR_UNSUPPORTED;  // draw counter holds 12 bits of order
    DeviceGuard dg(g->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    act_status s = ensure_work(g, channels, n_atoms, mode);
    if (s != ACT_OK) return s;
    bool host_seen = !is_device_ptr(signals);
    // all buffers in the grid device's memory and the single-launch form
    // applies: the kernel reads the signals and writes the outputs itself
    // (no graph, no copies)
    const int fctas = fused_ctas(g, channels, mode, g->profiling);
    const int dev = g->device;
    if (fctas > 0 && is_local_device_ptr(signals, dev) && (!atoms_out || is_local_device_ptr(atoms_out, dev)) &&
        (!coeffs_out || is_local_device_ptr(coeffs_out, dev)) &&
        (!residuals_out || is_local_device_ptr(residuals_out, dev)) &&
        (!energy_out || is_local_device_ptr(energy_out, dev))) {
        ACT_CK(launch_mp_fused(g->d32, g->K, g->Lp, g->L, signals, channels, n_atoms, g->ax, g->w.fsync, atoms_out,
                               coeffs_out, energy_out, residuals_out, g->L, g->status, fctas, g->wait_ns, st));
        g->last = nullptr;
        return ACT_OK;
    }
    ACT_CK(cudaMemcpyAsync(g->w.sig, signals, sizeof(float) * (size_t)channels * g->L, cudaMemcpyDefault, st));
    GraphEntry *ge = nullptr;
    s = get_graph(g, channels, n_atoms, mode, &ge);
    if (s != ACT_OK) return s;
    ACT_CK(cudaGraphLaunch(ge->exec, st));
    g->last = ge;
    const size_t BP = (size_t)channels * n_atoms;
    if ((s = copy_out(atoms_out, g->w.atoms, sizeof(act_atom) * BP, st, &host_seen)) != ACT_OK) return s;
    if ((s = copy_out(coeffs_out, g->w.coefs, sizeof(float) * BP, st, &host_seen)) != ACT_OK) return s;
    if ((s = copy_out(energy_out, g->w.energy, sizeof(double) * (size_t)channels * (n_atoms + 1), st,
                      &host_seen)) != ACT_OK)
        return s;
    if (residuals_out) {
        if (!is_device_ptr(residuals_out)) host_seen = true;
        ACT_CK(cudaMemcpy2DAsync(residuals_out, sizeof(float) * g->L, g->w.R, sizeof(float) * g->Lp,
                                 sizeof(float) * g->L, channels, cudaMemcpyDefault, st));
    }
    if (host_seen) ACT_CK(cudaStreamSynchronize(st));
    return ACT_OK;
}

act_status act_project(act_grid *g, const float *signals, int32_t channels, float *scores, void *cuda_stream) {
    if (!g || !signals || !scores || channels < 1) return ACT_ERR_INVALID_ARG;
    if (g->built < 0) return ACT_ERR_NOT_BUILT;
    DeviceGuard dg(g->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    act_status s = ensure_work(g, channels, 1, ACT_SEARCH_FP32);
    if (s != ACT_OK) return s;
    ACT_CK(cudaMemcpyAsync(g->w.sig, signals, sizeof(float) * (size_t)channels * g->L, cudaMemcpyDefault, st));
    ACT_CK(launch_init(g->w.sig, channels, g->L, g->Lp, g->w.R, nullptr, g->Lb, nullptr, nullptr, 1, g->status, st));
    if (g->built == ACT_DICT_RECOMPUTE) {
        ACT_CK(launch_shift_search(g->shift, g->w.R, g->Lp, g->L, channels, nullptr, scores, g->status, false, st,
                                   nullptr, nullptr, g->wait_ns));
    } else {
        ACT_CK(launch_project(g->d32, g->K, g->Lp, g->w.R, channels, scores, g->status, g->gemv_grid, st,
                              g->wait_ns));
    }
    return ACT_OK;
}

act_status act_dictionary_rows(act_grid *g, int64_t first, int64_t count, float *out, void *cuda_stream) {
    if (!g || !out || first < 0 || count < 0 || first + count > g->K) return ACT_ERR_INVALID_ARG;
    if (g->built < 0) return ACT_ERR_NOT_BUILT;
    if (!g->d32) return ACT_ERR_UNSUPPORTED;  // template dictionary: no rows
    if (count == 0) return ACT_OK;
    DeviceGuard dg(g->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    ACT_CK(cudaMemcpy2DAsync(out, sizeof(float) * g->L, g->d32 + first * g->Lp, sizeof(float) * g->Lp,
                             sizeof(float) * g->L, (size_t)count, cudaMemcpyDefault, st));
    if (!is_device_ptr(out)) ACT_CK(cudaStreamSynchronize(st));
    return ACT_OK;
}

act_status act_grid_status(act_grid *g, void *cuda_stream) {
    if (!g) return ACT_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    ACT_CK(cudaStreamSynchronize((cudaStream_t)cuda_stream));
    int flags = 0;
    ACT_CK(cudaMemcpy(&flags, g->status, sizeof(int), cudaMemcpyDeviceToHost));
    ACT_CK(cudaMemset(g->status, 0, sizeof(int)));
    if (flags & kFlagTimeout) return ACT_ERR_DEVICE_TIMEOUT;
    if (flags & kFlagNonFinite) return ACT_ERR_NONFINITE;
    return ACT_OK;
}

// Template search: every valid (lags per thread, warps per CTA) pair.
static act_status autotune_shift(act_grid *g, int channels, cudaStream_t st, double *best_ms) {
    cudaEvent_t e0, e1;
    ACT_CK(cudaEventCreate(&e0));
    ACT_CK(cudaEventCreate(&e1));
    const int reps = 3;
    const ShiftPlan keep = g->shift;
    double best = 1e30;
    int bJ = keep.J, bW = keep.W, bS = keep.NS, bC = keep.ctas_per_sm;
    cudaError_t err = cudaSuccess;
    static const int Js[] = {8, 16, 32};
    for (int J : Js) {
      for (int W = 1; W <= 8 && err == cudaSuccess; ++W) {
        for (int NS = 1; NS <= 3 && err == cudaSuccess; ++NS) {
          const int maxc = shift_max_ctas_per_sm(g->shift, J, W, NS);
          for (int C = 1; C <= maxc && err == cudaSuccess; ++C) {
            if (shift_configure(g->shift, J, W, NS, g->sm_count, C) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            for (int pass = 0; pass < 2 && err == cudaSuccess; ++pass) {  // pass 0 warms up
                err = cudaEventRecord(e0, st);
                for (int r = 0; r < reps && err == cudaSuccess; ++r)
                    err = launch_shift_search(g->shift, g->w.R, g->Lp, g->L, channels, g->w.keys, nullptr, g->status,
                                              false, st, nullptr, nullptr, g->wait_ns);
                if (err == cudaSuccess) err = cudaEventRecord(e1, st);
                if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            }
            float t = 0.f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
            if (err == cudaSuccess && t / reps < best) {
                best = t / reps;
                bJ = J;
                bW = W;
                bS = NS;
                bC = C;
            }
          }
        }
      }
    }
    if (err == cudaSuccess) err = shift_configure(g->shift, bJ, bW, bS, g->sm_count, bC);
    if (err == cudaSuccess) err = cudaMemsetAsync(g->w.keys, 0, sizeof(unsigned long long) * (size_t)channels, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) {
        shift_configure(g->shift, keep.J, keep.W, keep.NS, g->sm_count, keep.ctas_per_sm);
        note_error("act_autotune", err);
        return ACT_ERR_CUDA;
    }
    drop_graphs(g);
    ++g->generation;
    if (best_ms) *best_ms = best;
    return ACT_OK;
}

act_status act_autotune(act_grid *g, const float *signals, int32_t channels, void *cuda_stream, double *best_ms) {
    if (!g || !signals || channels < 1) return ACT_ERR_INVALID_ARG;
    if (g->built < 0) return ACT_ERR_NOT_BUILT;
    DeviceGuard dg(g->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (g->built == ACT_DICT_RECOMPUTE) {
        act_status s = ensure_work(g, channels, 1, ACT_SEARCH_SHIFT);
        if (s != ACT_OK) return s;
        ACT_CK(cudaMemcpyAsync(g->w.sig, signals, sizeof(float) * (size_t)channels * g->L, cudaMemcpyDefault, st));
        ACT_CK(launch_init(g->w.sig, channels, g->L, g->Lp, g->w.R, nullptr, g->Lb, g->w.keys, nullptr, 1, g->status,
                           st));
        return autotune_shift(g, channels, st, best_ms);
    }
    const bool bf16 = g->bf16 != nullptr;
    act_status s = ensure_work(g, channels, 1, bf16 ? ACT_SEARCH_BF16 : ACT_SEARCH_FP32);
    if (s != ACT_OK) return s;
    ACT_CK(cudaMemcpyAsync(g->w.sig, signals, sizeof(float) * (size_t)channels * g->L, cudaMemcpyDefault, st));
    ACT_CK(launch_init(g->w.sig, channels, g->L, g->Lp, g->w.R, g->w.R16, g->Lb, g->w.keys, nullptr, 1, g->status, st));
    cudaEvent_t e0, e1;
    ACT_CK(cudaEventCreate(&e0));
    ACT_CK(cudaEventCreate(&e1));
    const int reps = 3;
    // one search order of the current configuration, `reps` times, in ms per order
    auto time_search = [&](bool use_bf16, double *ms) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {  // pass 0 warms up
            e = cudaEventRecord(e0, st);
            for (int r = 0; r < reps && e == cudaSuccess; ++r) {
                if (use_bf16) {
                    e = cudaMemsetAsync(g->w.fb_count, 0, 2 * sizeof(int), st);
                    if (e == cudaSuccess)
                        e = launch_bf16_gemm(g->bf16, g->w.b16, channels, g->w.R16, g->status, st, g->wait_ns);
                    if (e == cudaSuccess)
                        e = launch_bf16_resolve(g->bf16, g->w.b16, channels, g->d32, g->Lp, g->L, g->w.R, g->w.keys,
                                                g->w.fb_list, g->w.fb_count, g->stats, g->status, g->gemv_grid, st,
                                                g->wait_ns);
                } else {
                    e = g->gemv_stream
                            ? launch_gemv_stream_argmax(g->d32, g->K, g->Lp, g->w.R, channels, nullptr, nullptr,
                                                        g->w.keys, g->status, g->sm_count, st, g->wait_ns)
                            : launch_gemv_argmax(g->d32, g->K, g->Lp, g->w.R, channels, nullptr, nullptr, g->w.keys,
                                                 g->status, g->gemv_grid, st, g->wait_ns);
                }
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        }
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        *ms = t / reps;
        return e;
    };
    cudaError_t err = cudaSuccess;
    // FP32 GEMV: resident CTAs per SM of the load-streaming GEMV, and the
    // bulk-copy streaming GEMV
    double best32 = 1e30;
    int best_grid = g->gemv_grid;
    bool best_stream = false;
    g->gemv_stream = false;
    const int max_per_sm = gemv_max_ctas_per_sm(g->Lp);
    for (int per_sm = 1; per_sm <= max_per_sm && err == cudaSuccess; ++per_sm) {
        g->gemv_grid = g->sm_count * per_sm;
        double ms = 0.0;
        err = time_search(false, &ms);
        if (err == cudaSuccess && ms < best32) {
            best32 = ms;
            best_grid = g->gemv_grid;
        }
    }
    g->gemv_grid = best_grid;
    if (err == cudaSuccess) {
        g->gemv_stream = true;
        double ms = 0.0;
        err = time_search(false, &ms);
        if (err == cudaSuccess && ms < best32) {
            best32 = ms;
            best_stream = true;
        }
    }
    g->gemv_stream = best_stream;
    // tensor-core search: tile width x pipeline depth
    double best16 = 1e30;
    if (bf16 && err == cudaSuccess) {
        int best_bn = 256, best_st = 0;
        const int widths[2] = {128, 256};
        for (int wi = 0; wi < 2 && err == cudaSuccess; ++wi) {
            const int ms_max = bf16_search_max_stages(g->bf16, widths[wi]);
            for (int stg = 2; stg <= ms_max && err == cudaSuccess; ++stg) {
                err = bf16_search_configure(g->bf16, widths[wi], stg);
                double ms = 0.0;
                if (err == cudaSuccess) err = time_search(true, &ms);
                if (err == cudaSuccess && ms < best16) {
                    best16 = ms;
                    best_bn = widths[wi];
                    best_st = stg;
                }
            }
        }
        if (err == cudaSuccess) err = bf16_search_configure(g->bf16, best_bn, best_st);
    }
    // leave clean state: keys and counters zero, no stale graphs
    if (err == cudaSuccess) err = cudaMemsetAsync(g->w.keys, 0, sizeof(unsigned long long) * (size_t)channels, st);
    if (err == cudaSuccess) err = cudaMemsetAsync(g->w.fb_count, 0, 2 * sizeof(int), st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) {
        note_error("act_autotune", err);
        return ACT_ERR_CUDA;
    }
    drop_graphs(g);
    ++g->generation;
    if (best_ms) *best_ms = effective_search(g) == ACT_SEARCH_BF16 && bf16 ? best16 : best32;
    return ACT_OK;
}

act_status act_get_tuning(const act_grid *g, int32_t *gemv_ctas_out, int32_t *bf16_tile_atoms,
                          int32_t *bf16_stages) {
    if (!g) return ACT_ERR_INVALID_ARG;
    int bn = 0, stg = 0;
    if (g->bf16) bf16_search_get_config(g->bf16, &bn, &stg, nullptr);
    if (gemv_ctas_out) *gemv_ctas_out = g->gemv_stream ? -1 : g->gemv_grid;
    if (bf16_tile_atoms) *bf16_tile_atoms = bn;
    if (bf16_stages) *bf16_stages = stg;
    return ACT_OK;
}

act_status act_set_tuning(act_grid *g, int32_t gemv_ctas_in, int32_t bf16_tile_atoms, int32_t bf16_stages) {
    if (!g) return ACT_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    if (gemv_ctas_in > 0) {
        if (gemv_ctas_in > g->sm_count * gemv_max_ctas_per_sm(g->Lp)) return ACT_ERR_INVALID_ARG;
        g->gemv_grid = gemv_ctas_in;
        g->gemv_stream = false;
    } else if (gemv_ctas_in == -1) {
        g->gemv_stream = true;
    } else if (gemv_ctas_in < -1) {
        return ACT_ERR_INVALID_ARG;
    }
    if (bf16_tile_atoms > 0) {
        if (!g->bf16) return ACT_ERR_NOT_BUILT;
        cudaError_t e = bf16_search_configure(g->bf16, bf16_tile_atoms, bf16_stages);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return ACT_ERR_INVALID_ARG;
        }
    }
    drop_graphs(g);
    ++g->generation;
    return ACT_OK;
}

act_status act_get_shift_tuning(const act_grid *g, int32_t *lags_per_thread, int32_t *warps, int32_t *stages,
                                int32_t *ctas_per_sm) {
    if (!g) return ACT_ERR_INVALID_ARG;
    if (!g->shift.tpl) return ACT_ERR_NOT_BUILT;
    if (lags_per_thread) *lags_per_thread = g->shift.J;
    if (warps) *warps = g->shift.W;
    if (stages) *stages = g->shift.NS;
    if (ctas_per_sm) *ctas_per_sm = g->shift.ctas_per_sm;
    return ACT_OK;
}

act_status act_set_shift_tuning(act_grid *g, int32_t lags_per_thread, int32_t warps, int32_t stages,
                                int32_t ctas_per_sm) {
    if (!g) return ACT_ERR_INVALID_ARG;
    if (!g->shift.tpl) return ACT_ERR_NOT_BUILT;
    DeviceGuard dg(g->device);
    if (!shift_config_valid(g->shift, lags_per_thread, warps, stages) || ctas_per_sm < 0) return ACT_ERR_INVALID_ARG;
    if (shift_configure(g->shift, lags_per_thread, warps, stages, g->sm_count, ctas_per_sm) != cudaSuccess) {
        cudaGetLastError();
        return ACT_ERR_INVALID_ARG;
    }
    drop_graphs(g);
    ++g->generation;
    return ACT_OK;
}

act_status act_set_refinement(act_grid *g, int32_t steps) {
    if (!g || steps < 0 || steps > 1000) return ACT_ERR_INVALID_ARG;
    if (steps != g->refine_steps) {
        g->refine_steps = steps;
        ++g->generation;
    }
    return ACT_OK;
}

act_status act_chirplet_score(int32_t n_samples, double fs, const double *theta, const float *residuals,
                              int32_t channels, double *score, double *grad_theta, float *atoms, void *cuda_stream) {
    if (!theta || !residuals || !score || channels < 1 || n_samples < 1 || n_samples > kMaxSamples || !(fs > 0.0))
        return ACT_ERR_INVALID_ARG;
    ACT_CK(launch_chirplet_score(n_samples, fs, theta, residuals, channels, score, grad_theta, atoms,
                                 (cudaStream_t)cuda_stream));
    return ACT_OK;
}

act_status act_set_profiling(act_grid *g, int32_t enable) {
    if (!g) return ACT_ERR_INVALID_ARG;
    g->profiling = enable != 0;
    return ACT_OK;
}

act_status act_profile_read(act_grid *g, double *search_ms, double *core_ms, int32_t *search_launches,
                            int32_t *kernels) {
    if (!g) return ACT_ERR_INVALID_ARG;
    if (!g->last) return ACT_ERR_NOT_BUILT;
    DeviceGuard dg(g->device);
    double total = 0.0, core = 0.0;
    const auto &ev = g->last->events;
    for (size_t i = 0; i + 2 < ev.size(); i += 3) {
        ACT_CK(cudaEventSynchronize(ev[i + 2]));
        float a = 0.f, b = 0.f;
        ACT_CK(cudaEventElapsedTime(&a, ev[i], ev[i + 2]));
        ACT_CK(cudaEventElapsedTime(&b, ev[i], ev[i + 1]));
        total += a;
        core += b;
    }
    if (search_ms) *search_ms = total;
    if (core_ms) *core_ms = core;
    if (search_launches) *search_launches = (int32_t)(ev.size() / 3);
    if (kernels) *kernels = g->last->kernels;
    return ACT_OK;
}

act_status act_bf16_stats(act_grid *g, int64_t *resolved, int64_t *items_rescanned, int64_t *fallbacks) {
    if (!g) return ACT_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    long long h[3] = {0, 0, 0};
    ACT_CK(cudaMemcpy(h, g->stats, sizeof(h), cudaMemcpyDeviceToHost));
    if (resolved) *resolved = h[0];
    if (fallbacks) *fallbacks = h[1];
    if (items_rescanned) *items_rescanned = h[2];
    return ACT_OK;
}

// ---------------------------------------------------------------------------
// Uneven batches
// ---------------------------------------------------------------------------
struct act_ragged_plan {
    struct Group {
        act_grid *g = nullptr;
        uint64_t generation = 0;
        act_search_mode mode = ACT_SEARCH_FP32;
        std::vector<int> chan;       // caller channel ids of this group
        int64_t *src_off = nullptr;  // [B] sample offsets in the concatenated signals
        int *d_chan = nullptr;       // [B]
        WorkBuffers w;
        cudaStream_t st = nullptr;
        cudaEvent_t join = nullptr;
    };
    int device = 0;
    int channels = 0;
    int P = 0;
    int64_t total = 0;
    std::vector<Group> groups;
    float *d_sig = nullptr;       // [total] staged concatenated signals
    float *d_resid = nullptr;     // [total] concatenated residuals
    act_atom *d_atoms = nullptr;  // [channels][P]
    float *d_coefs = nullptr;     // [channels][P]
    double *d_energy = nullptr;   // [channels][P+1]
    cudaStream_t cap = nullptr;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;
};

static void ragged_free(act_ragged_plan *p) {
    if (!p) return;
    DeviceGuard dg(p->device);
    cudaDeviceSynchronize();
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (auto &gr : p->groups) {
        free_dev(gr.src_off);
        free_dev(gr.d_chan);
        free_work(gr.w);
        if (gr.st) cudaStreamDestroy(gr.st);
        if (gr.join) cudaEventDestroy(gr.join);
    }
    free_dev(p->d_sig);
    free_dev(p->d_resid);
    free_dev(p->d_atoms);
    free_dev(p->d_coefs);
    free_dev(p->d_energy);
    if (p->fork) cudaEventDestroy(p->fork);
    if (p->cap) cudaStreamDestroy(p->cap);
    delete p;
}

static act_status ragged_build(act_ragged_plan *p, act_grid *const *grids, int32_t n_grids, const int64_t *offsets) {
    // group channels by window length
    std::map<int, int> group_of_len;
    for (int i = 0; i < n_grids; ++i) {
        act_grid *g = grids[i];
        if (!g || (g->built < 0 && effective_search(g) != ACT_SEARCH_LEM)) return ACT_ERR_NOT_BUILT;
        if (g->device != p->device) return ACT_ERR_INVALID_ARG;
        if (group_of_len.count(g->L)) return ACT_ERR_INVALID_ARG;  // one grid per window length
        group_of_len[g->L] = (int)p->groups.size();
        act_ragged_plan::Group gr;
        gr.g = g;
        gr.generation = g->generation;
        p->groups.push_back(gr);
    }
    for (int c = 0; c < p->channels; ++c) {
        const int64_t len = offsets[c + 1] - offsets[c];
        auto it = group_of_len.find((int)len);
        if (len < 1 || it == group_of_len.end()) return ACT_ERR_INVALID_ARG;
        p->groups[it->second].chan.push_back(c);
    }
    p->total = offsets[p->channels];
    ACT_AL(p->d_sig, sizeof(float) * (size_t)p->total);
    ACT_AL(p->d_resid, sizeof(float) * (size_t)p->total);
    ACT_AL(p->d_atoms, sizeof(act_atom) * (size_t)p->channels * p->P);
    ACT_AL(p->d_coefs, sizeof(float) * (size_t)p->channels * p->P);
    ACT_AL(p->d_energy, sizeof(double) * (size_t)p->channels * (p->P + 1));
    ACT_CK(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
    ACT_CK(cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming));
    for (auto &gr : p->groups) {
        const int B = (int)gr.chan.size();
        if (B == 0) continue;
        act_grid *g = gr.g;
        gr.mode = effective_search(g);
        if (!search_available(g, gr.mode)) return ACT_ERR_NOT_BUILT;
        // the plan's own buffers, search scratch included: nothing the
        // plan's graph captures belongs to the grid's work buffers
        act_status s = grow_work(g, gr.w, B, p->P, gr.mode);
        if (s != ACT_OK) return s;
        std::vector<int64_t> off(B);
        for (int i = 0; i < B; ++i) off[i] = offsets[gr.chan[i]];
        ACT_AL(gr.src_off, sizeof(int64_t) * B);
        ACT_CK(cudaMemcpy(gr.src_off, off.data(), sizeof(int64_t) * B, cudaMemcpyHostToDevice));
        ACT_AL(gr.d_chan, sizeof(int) * B);
        ACT_CK(cudaMemcpy(gr.d_chan, gr.chan.data(), sizeof(int) * B, cudaMemcpyHostToDevice));
        ACT_CK(cudaStreamCreateWithFlags(&gr.st, cudaStreamNonBlocking));
        ACT_CK(cudaEventCreateWithFlags(&gr.join, cudaEventDisableTiming));
    }
    // one graph: fork, then per length group gather -> MP loop -> scatter on
    // its own branch, then join
    ACT_CK(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
    act_status s = ACT_OK;
    cudaError_t e = cudaEventRecord(p->fork, p->cap);
    for (auto &gr : p->groups) {
        const int B = (int)gr.chan.size();
        if (B == 0 || e != cudaSuccess || s != ACT_OK) continue;
        act_grid *g = gr.g;
        e = cudaStreamWaitEvent(gr.st, p->fork, 0);
        if (e == cudaSuccess) e = launch_ragged_gather(p->d_sig, gr.src_off, B, g->L, gr.w.sig, gr.st);
        GraphEntry ge;
        if (e == cudaSuccess) s = record_decompose(g, gr.w, B, p->P, gr.mode, ge, gr.st, false, false);
        p->kernels += ge.kernels + 2;
        if (e == cudaSuccess && s == ACT_OK)
            e = launch_ragged_scatter(B, p->P, g->L, g->Lp, gr.d_chan, gr.src_off, gr.w.atoms, gr.w.coefs,
                                      gr.w.energy, gr.w.R, p->d_atoms, p->d_coefs, p->d_energy, p->d_resid, gr.st);
        if (e == cudaSuccess && s == ACT_OK) e = cudaEventRecord(gr.join, gr.st);
        if (e == cudaSuccess && s == ACT_OK) e = cudaStreamWaitEvent(p->cap, gr.join, 0);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(p->cap, &graph);
    if (s != ACT_OK || e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (s != ACT_OK) return s;
        note_error("ragged capture", e != cudaSuccess ? e : e2);
        return ACT_ERR_CUDA;
    }
    p->graph = graph;
    ACT_CK(cudaGraphInstantiate(&p->exec, graph, 0));
    return ACT_OK;
}

act_status act_ragged_plan_create(act_grid *const *grids, int32_t n_grids, const int64_t *offsets, int32_t channels,
                                  int32_t n_atoms, act_ragged_plan **out) {
    if (!grids || n_grids < 1 || !offsets || channels < 1 || n_atoms < 1 || !out) return ACT_ERR_INVALID_ARG;
    *out = nullptr;
    if (offsets[0] != 0) return ACT_ERR_INVALID_ARG;
    for (int c = 0; c < channels; ++c)
        if (offsets[c + 1] <= offsets[c]) return ACT_ERR_INVALID_ARG;
    if (!grids[0]) return ACT_ERR_INVALID_ARG;
    DeviceGuard dg(grids[0]->device);
    act_ragged_plan *p = new (std::nothrow) act_ragged_plan();
    if (!p) return ACT_ERR_OOM;
    p->device = grids[0]->device;
    p->channels = channels;
    p->P = n_atoms;
    act_status s = ragged_build(p, grids, n_grids, offsets);
    if (s != ACT_OK) {
        ragged_free(p);
        return s;
    }
    *out = p;
    return ACT_OK;
}

act_status act_ragged_decompose(act_ragged_plan *p, const float *signals, act_atom *atoms_out, float *coeffs_out,
                                float *residuals_out, double *energy_out, void *cuda_stream) {
    if (!p || !signals) return ACT_ERR_INVALID_ARG;
    for (auto &gr : p->groups)
        if (gr.g->generation != gr.generation || (gr.g->built < 0 && gr.mode != ACT_SEARCH_LEM))
            return ACT_ERR_NOT_BUILT;  // stale plan
    DeviceGuard dg(p->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    bool host_seen = !is_device_ptr(signals);
    ACT_CK(cudaMemcpyAsync(p->d_sig, signals, sizeof(float) * (size_t)p->total, cudaMemcpyDefault, st));
    ACT_CK(cudaGraphLaunch(p->exec, st));
    const size_t BP = (size_t)p->channels * p->P;
    act_status s;
    if ((s = copy_out(atoms_out, p->d_atoms, sizeof(act_atom) * BP, st, &host_seen)) != ACT_OK) return s;
    if ((s = copy_out(coeffs_out, p->d_coefs, sizeof(float) * BP, st, &host_seen)) != ACT_OK) return s;
    if ((s = copy_out(energy_out, p->d_energy, sizeof(double) * (size_t)p->channels * (p->P + 1), st,
                      &host_seen)) != ACT_OK)
        return s;
    if ((s = copy_out(residuals_out, p->d_resid, sizeof(float) * (size_t)p->total, st, &host_seen)) != ACT_OK)
        return s;
    if (host_seen) ACT_CK(cudaStreamSynchronize(st));
    return ACT_OK;
}

act_status act_ragged_plan_info(const act_ragged_plan *p, int32_t *groups, int32_t *kernels) {
    if (!p) return ACT_ERR_INVALID_ARG;
    int n = 0;
    for (auto &gr : p->groups) n += gr.chan.empty() ? 0 : 1;
    if (groups) *groups = n;
    if (kernels) *kernels = p->kernels;
    return ACT_OK;
}

void act_ragged_plan_destroy(act_ragged_plan *p) { ragged_free(p); }

act_status act_dictionary_mode(const act_grid *g, int32_t *mode) {
    if (!g || !mode) return ACT_ERR_INVALID_ARG;
    *mode = g->built;
    return g->built < 0 ? ACT_ERR_NOT_BUILT : ACT_OK;
}

act_status act_set_memory_budget(act_grid *g, uint64_t bytes) {
    if (!g) return ACT_ERR_INVALID_ARG;
    g->mem_budget = bytes;
    return ACT_OK;
}

act_status act_set_wait_limit(act_grid *g, int64_t ns) {
    if (!g || ns < 0) return ACT_ERR_INVALID_ARG;
    const unsigned long long v = (unsigned long long)ns;
    if (v != g->wait_ns) {
        g->wait_ns = v;  // a kernel argument: the recorded graphs carry the old value
        drop_graphs(g);
        ++g->generation;
    }
    return ACT_OK;
}

act_status act_set_cta_pairs(act_grid *g, int32_t enable) {
    if (!g || (enable != 0 && enable != 1)) return ACT_ERR_INVALID_ARG;
    if ((enable != 0) != g->cta_pairs) {
        g->cta_pairs = enable != 0;  // the recorded graphs hold the other kernel
        drop_graphs(g);
    }
    return ACT_OK;
}

act_status act_set_fused(act_grid *g, int32_t ctas_per_sm) {
    if (!g || ctas_per_sm < 0 || ctas_per_sm > 32) return ACT_ERR_INVALID_ARG;
    if (ctas_per_sm != g->fused_ctas_per_sm) {
        g->fused_ctas_per_sm = ctas_per_sm;  // the recorded graphs hold the other launch form
        drop_graphs(g);
    }
    return ACT_OK;
}

act_status act_get_fused(const act_grid *g, int32_t channels, int32_t *ctas) {
    if (!g || !ctas || channels < 1) return ACT_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    *ctas = fused_ctas(g, channels, effective_search(g), g->profiling);
    return ACT_OK;
}

act_status act_get_cta_pairs(const act_grid *g, int32_t channels, int32_t *used) {
    if (!g || !used || channels < 1) return ACT_ERR_INVALID_ARG;
    *used = (g->shift_tc && shift_tc_uses_pairs(g->shift_tc, g->shift, channels, g->cta_pairs)) ? 1 : 0;
    return ACT_OK;
}

act_status act_inject_alloc_failure(int32_t nth) {
    if (nth < 0) return ACT_ERR_INVALID_ARG;
    g_fail_at.store(nth);
    return ACT_OK;
}

void act_destroy(act_grid *g) {
    if (!g) return;
    DeviceGuard dg(g->device);
    cudaDeviceSynchronize();
    drop_graphs(g);
    free_dictionary(g);
    free_work(g->w);
    free_dev(g->status);
    free_dev(g->stats);
    free_dev(g->degenerate);
    free_dev(g->eps_bits);
    if (g->cap) cudaStreamDestroy(g->cap);
    delete g;
}

}  // extern "C"
