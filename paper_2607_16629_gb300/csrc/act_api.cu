// Host side of the C ABI declared in include/act.h: argument checks, grid
// and buffer ownership, dictionary build, and the n_atoms loop of the
// matching pursuit (Eq. (4), Fig. 1) captured once per shape as a CUDA
// graph and replayed on the caller's stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

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
    // work buffers
    int cap_B = 0, cap_P = 0;
    float *sig = nullptr;
    float *R = nullptr;
    __nv_bfloat16 *R16 = nullptr;
    unsigned long long *keys = nullptr;
    act_atom *atoms = nullptr;
    float *coefs = nullptr;
    double *energy = nullptr;
    int *status = nullptr;
    int *fb_list = nullptr;
    int *fb_count = nullptr;
    long long *stats = nullptr;
    Bf16Search *bf16 = nullptr;
    int gemv_grid = 0;
    cudaStream_t cap = nullptr;
    bool profiling = false;
    std::map<std::tuple<int, int, int, int>, GraphEntry> graphs;
    GraphEntry *last = nullptr;
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

void free_work(act_grid *g) {
    free_dev(g->sig);
    free_dev(g->R);
    free_dev(g->R16);
    free_dev(g->keys);
    free_dev(g->atoms);
    free_dev(g->coefs);
    free_dev(g->energy);
    free_dev(g->fb_list);
    g->cap_B = g->cap_P = 0;
}

void free_dictionary(act_grid *g) {
    if (g->bf16) bf16_search_free(g->bf16);
    g->bf16 = nullptr;
    free_dev(g->d32);
    free_dev(g->d16);
    g->built = -1;
}

// Work buffers for B channels and P orders.  The BF16 residual copy always
// has at least 128 rows (the tensor-core tile height), padded with zeros.
act_status ensure_work(act_grid *g, int B, int P) {
    if (B <= g->cap_B && P <= g->cap_P) return ACT_OK;
    drop_graphs(g);
    const int nB = B > g->cap_B ? B : g->cap_B;
    const int nP = P > g->cap_P ? P : g->cap_P;
    free_work(g);
    const int rows16 = round_up(nB, 128);
    ACT_CK(cudaMalloc(&g->sig, sizeof(float) * (size_t)nB * g->L));
    ACT_CK(cudaMalloc(&g->R, sizeof(float) * (size_t)nB * g->Lp));
    ACT_CK(cudaMalloc(&g->R16, sizeof(__nv_bfloat16) * (size_t)rows16 * g->Lb));
    ACT_CK(cudaMemset(g->R16, 0, sizeof(__nv_bfloat16) * (size_t)rows16 * g->Lb));
    ACT_CK(cudaMalloc(&g->keys, sizeof(unsigned long long) * (size_t)nB));
    ACT_CK(cudaMemset(g->keys, 0, sizeof(unsigned long long) * (size_t)nB));
    ACT_CK(cudaMalloc(&g->atoms, sizeof(act_atom) * (size_t)nB * nP));
    ACT_CK(cudaMalloc(&g->coefs, sizeof(float) * (size_t)nB * nP));
    ACT_CK(cudaMalloc(&g->energy, sizeof(double) * (size_t)nB * (nP + 1)));
    ACT_CK(cudaMalloc(&g->fb_list, sizeof(int) * (size_t)nB));
    g->cap_B = nB;
    g->cap_P = nP;
    return ACT_OK;
}

act_search_mode effective_search(const act_grid *g) {
    if (g->search == ACT_SEARCH_FP32) return ACT_SEARCH_FP32;
    if (g->search == ACT_SEARCH_BF16) return ACT_SEARCH_BF16;
    return g->built == ACT_DICT_BF16 ? ACT_SEARCH_BF16 : ACT_SEARCH_FP32;
}

// Records the whole decomposition (init + P orders) on the capture stream.
act_status record_decompose(act_grid *g, int B, int P, act_search_mode mode, GraphEntry &ge) {
    cudaStream_t st = g->cap;
    const bool bf16 = mode == ACT_SEARCH_BF16;
    __nv_bfloat16 *R16 = bf16 ? g->R16 : nullptr;
    int kernels = 0;
    ACT_CK(launch_init(g->sig, B, g->L, g->Lp, g->R, R16, g->Lb, g->keys, g->energy, P + 1, g->status, st));
    ++kernels;
    for (int k = 0; k < P; ++k) {
        // profiling: events before the search, after its dominant kernel
        // (GEMV or GEMM) and after the whole search
        cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
        if (g->profiling) {
            for (int i = 0; i < 3; ++i) {
                ACT_CK(cudaEventCreate(&ev[i]));
                ge.events.push_back(ev[i]);
            }
            ACT_CK(cudaEventRecordWithFlags(ev[0], st, cudaEventRecordExternal));
        }
        if (bf16) {
            ACT_CK(launch_bf16_gemm(g->bf16, B, g->R16, g->status, st));
            if (g->profiling) ACT_CK(cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal));
            ACT_CK(launch_bf16_resolve(g->bf16, B, g->d32, g->Lp, g->L, g->R, g->keys, g->fb_list, g->fb_count,
                                       g->stats, g->status, g->gemv_grid, st));
            kernels += 4;
        } else {
            ACT_CK(launch_gemv_argmax(g->d32, g->K, g->Lp, g->R, B, nullptr, nullptr, g->keys, g->status,
                                      g->gemv_grid, st));
            if (g->profiling) ACT_CK(cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal));
            kernels += 1;
        }
        if (g->profiling) ACT_CK(cudaEventRecordWithFlags(ev[2], st, cudaEventRecordExternal));
        ACT_CK(launch_update(g->d32, g->Lp, g->L, g->R, R16, g->Lb, B, g->keys, g->ax, k, P, g->atoms, g->coefs,
                             g->energy, bf16 ? g->fb_count : nullptr, st));
        ++kernels;
    }
    ge.kernels = kernels;
    return ACT_OK;
}

act_status get_graph(act_grid *g, int B, int P, act_search_mode mode, GraphEntry **out) {
    auto key = std::make_tuple(B, P, (int)mode, g->profiling ? 1 : 0);
    auto it = g->graphs.find(key);
    if (it != g->graphs.end()) {
        *out = &it->second;
        return ACT_OK;
    }
    GraphEntry ge;
    ACT_CK(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
    act_status s = record_decompose(g, B, P, mode, ge);
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
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&g->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(g->status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&g->fb_count, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(g->fb_count, 0, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&g->stats, 3 * sizeof(long long));
    if (e == cudaSuccess) e = cudaMemset(g->stats, 0, 3 * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&g->degenerate, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&g->eps_bits, sizeof(unsigned int));
    if (e != cudaSuccess) {
        note_error("act_grid_create", e);
        act_destroy(g);
        return e == cudaErrorMemoryAllocation ? ACT_ERR_OOM : ACT_ERR_CUDA;
    }
    g->gemv_grid = gemv_ctas(g->sm_count, g->Lp);
    *out = g;
    return ACT_OK;
}

act_status act_grid_size(const act_grid *g, int64_t *n_atoms, int32_t *row_stride) {
    if (!g) return ACT_ERR_INVALID_ARG;
    if (n_atoms) *n_atoms = g->K;
    if (row_stride) *row_stride = g->Lp;
    return ACT_OK;
}

act_status act_dictionary_build(act_grid *g, act_dict_mode mode, void *cuda_stream) {
    if (!g) return ACT_ERR_INVALID_ARG;
    if (mode == ACT_DICT_RECOMPUTE) return ACT_ERR_UNSUPPORTED;
    if (mode == ACT_DICT_AUTO) mode = ACT_DICT_FP32;
    if (mode != ACT_DICT_FP32 && mode != ACT_DICT_BF16) return ACT_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    ACT_CK(cudaStreamSynchronize(st));
    drop_graphs(g);
    free_dictionary(g);
    const size_t b32 = sizeof(float) * (size_t)g->K * g->Lp;
    cudaError_t e = cudaMalloc(&g->d32, b32);
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
        e = cudaMalloc(&g->d16, b16);
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

act_status act_set_search(act_grid *g, act_search_mode mode) {
    if (!g || (int)mode < 0 || (int)mode > 2) return ACT_ERR_INVALID_ARG;
    g->search = mode;
    return ACT_OK;
}

act_status act_decompose(act_grid *g, const float *signals, int32_t channels, int32_t n_atoms,
                         act_atom *atoms_out, float *coeffs_out, float *residuals_out, double *energy_out,
                         void *cuda_stream) {
    if (!g || !signals || channels < 1 || n_atoms < 1) return ACT_ERR_INVALID_ARG;
    if (g->built < 0) return ACT_ERR_NOT_BUILT;
    DeviceGuard dg(g->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const act_search_mode mode = effective_search(g);
    if (mode == ACT_SEARCH_BF16) {
        if (!g->bf16 || !g->d16) return ACT_ERR_NOT_BUILT;
        if (channels > 128) return ACT_ERR_UNSUPPORTED;
    }
    act_status s = ensure_work(g, channels, n_atoms);
    if (s != ACT_OK) return s;
    bool host_seen = !is_device_ptr(signals);
    ACT_CK(cudaMemcpyAsync(g->sig, signals, sizeof(float) * (size_t)channels * g->L, cudaMemcpyDefault, st));
    GraphEntry *ge = nullptr;
    s = get_graph(g, channels, n_atoms, mode, &ge);
    if (s != ACT_OK) return s;
    ACT_CK(cudaGraphLaunch(ge->exec, st));
    g->last = ge;
    const size_t BP = (size_t)channels * n_atoms;
    if ((s = copy_out(atoms_out, g->atoms, sizeof(act_atom) * BP, st, &host_seen)) != ACT_OK) return s;
    if ((s = copy_out(coeffs_out, g->coefs, sizeof(float) * BP, st, &host_seen)) != ACT_OK) return s;
    if ((s = copy_out(energy_out, g->energy, sizeof(double) * (size_t)channels * (n_atoms + 1), st,
                      &host_seen)) != ACT_OK)
        return s;
    if (residuals_out) {
        if (!is_device_ptr(residuals_out)) host_seen = true;
        ACT_CK(cudaMemcpy2DAsync(residuals_out, sizeof(float) * g->L, g->R, sizeof(float) * g->Lp,
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
    act_status s = ensure_work(g, channels, 1);
    if (s != ACT_OK) return s;
    ACT_CK(cudaMemcpyAsync(g->sig, signals, sizeof(float) * (size_t)channels * g->L, cudaMemcpyDefault, st));
    ACT_CK(launch_init(g->sig, channels, g->L, g->Lp, g->R, nullptr, g->Lb, nullptr, nullptr, 1, g->status, st));
    ACT_CK(launch_project(g->d32, g->K, g->Lp, g->R, channels, scores, g->status, g->gemv_grid, st));
    return ACT_OK;
}

act_status act_dictionary_rows(act_grid *g, int64_t first, int64_t count, float *out, void *cuda_stream) {
    if (!g || !out || first < 0 || count < 0 || first + count > g->K) return ACT_ERR_INVALID_ARG;
    if (g->built < 0) return ACT_ERR_NOT_BUILT;
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

act_status act_autotune(act_grid *g, const float *signals, int32_t channels, void *cuda_stream, double *best_ms) {
    if (!g || !signals || channels < 1) return ACT_ERR_INVALID_ARG;
    if (g->built < 0) return ACT_ERR_NOT_BUILT;
    DeviceGuard dg(g->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const bool bf16 = g->bf16 != nullptr && channels <= 128;
    act_status s = ensure_work(g, channels, 1);
    if (s != ACT_OK) return s;
    ACT_CK(cudaMemcpyAsync(g->sig, signals, sizeof(float) * (size_t)channels * g->L, cudaMemcpyDefault, st));
    ACT_CK(launch_init(g->sig, channels, g->L, g->Lp, g->R, g->R16, g->Lb, g->keys, nullptr, 1, g->status, st));
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
                    e = cudaMemsetAsync(g->fb_count, 0, 2 * sizeof(int), st);
                    if (e == cudaSuccess) e = launch_bf16_gemm(g->bf16, channels, g->R16, g->status, st);
                    if (e == cudaSuccess)
                        e = launch_bf16_resolve(g->bf16, channels, g->d32, g->Lp, g->L, g->R, g->keys, g->fb_list,
                                                g->fb_count, g->stats, g->status, g->gemv_grid, st);
                } else {
                    e = launch_gemv_argmax(g->d32, g->K, g->Lp, g->R, channels, nullptr, nullptr, g->keys,
                                           g->status, g->gemv_grid, st);
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
    // FP32 GEMV: resident CTAs per SM
    double best32 = 1e30;
    int best_grid = g->gemv_grid;
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
    if (err == cudaSuccess) err = cudaMemsetAsync(g->keys, 0, sizeof(unsigned long long) * (size_t)channels, st);
    if (err == cudaSuccess) err = cudaMemsetAsync(g->fb_count, 0, 2 * sizeof(int), st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) {
        note_error("act_autotune", err);
        return ACT_ERR_CUDA;
    }
    drop_graphs(g);
    if (best_ms) *best_ms = effective_search(g) == ACT_SEARCH_BF16 && bf16 ? best16 : best32;
    return ACT_OK;
}

act_status act_get_tuning(const act_grid *g, int32_t *gemv_ctas_out, int32_t *bf16_tile_atoms,
                          int32_t *bf16_stages) {
    if (!g) return ACT_ERR_INVALID_ARG;
    int bn = 0, stg = 0;
    if (g->bf16) bf16_search_get_config(g->bf16, &bn, &stg, nullptr);
    if (gemv_ctas_out) *gemv_ctas_out = g->gemv_grid;
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

act_status act_bf16_stats(act_grid *g, int64_t *resolved, int64_t *tiles_rescanned, int64_t *fallbacks) {
    if (!g) return ACT_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    long long h[3] = {0, 0, 0};
    ACT_CK(cudaMemcpy(h, g->stats, sizeof(h), cudaMemcpyDeviceToHost));
    if (resolved) *resolved = h[0];
    if (fallbacks) *fallbacks = h[1];
    if (tiles_rescanned) *tiles_rescanned = h[2];
    return ACT_OK;
}

void act_destroy(act_grid *g) {
    if (!g) return;
    DeviceGuard dg(g->device);
    cudaDeviceSynchronize();
    drop_graphs(g);
    free_dictionary(g);
    free_work(g);
    free_dev(g->status);
    free_dev(g->fb_count);
    free_dev(g->stats);
    free_dev(g->degenerate);
    free_dev(g->eps_bits);
    if (g->cap) cudaStreamDestroy(g->cap);
    delete g;
}

}  // extern "C"
