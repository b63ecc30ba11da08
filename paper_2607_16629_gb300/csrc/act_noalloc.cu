// act_search_noalloc: the FP32 search (GEMV with the argmax fused) for callers
// that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not acceptable -- a
// latency-bound streaming loop where the implicit device synchronisation of
// an allocation would stall the pipeline, or a host process whose device
// memory is entirely reserved up front by another allocator (a framework's
// caching allocator holding the whole HBM).  Such callers own every buffer they pass; the only
// extra memory this path touches is the fixed scratch array below.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "act_internal.cuh"

namespace {

constexpr int kNoAllocMaxChannels = 256;
constexpr int kNoAllocMaxDevices = 64;

// The scratch of act_search_noalloc: one packed selection key per channel
// (largest |score| in the high word, 2^32-1 - index in the low word) and one
// status word after them.  256 * 8 + 8 bytes, resident on every GPU that
// loads this library until the process exits.  In host code this name is
// only a stand-in for the device symbol: its device address comes from
// cudaGetSymbolAddress.
static __device__ __align__(256) unsigned long long g_search_scratch[kNoAllocMaxChannels + 1];

std::mutex g_setup_mu;
unsigned long long *g_scratch_addr[kNoAllocMaxDevices] = {};
int g_sm_count[kNoAllocMaxDevices] = {};

// Converts the packed keys into outputs.  A channel whose search recorded a
// device-side timeout (status word non-zero) or found no finite score gets
// index -1 and score 0.
__global__ void k_noalloc_finish(int B, int64_t *__restrict__ best_index, float *__restrict__ best_score) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const unsigned long long key = g_search_scratch[b];
    const bool failed = g_search_scratch[kNoAllocMaxChannels] != 0ull || key == 0ull;
    best_index[b] = failed ? -1 : (int64_t)act::key_index(key);
    best_score[b] = failed ? 0.0f : __uint_as_float((unsigned int)(key >> 32));
}

}  // namespace

extern "C" act_status act_search_noalloc(const float *dictionary, int64_t n_atoms, int32_t row_stride,
                                         const float *residuals, int32_t channels, int64_t *best_index,
                                         float *best_score, void *cuda_stream) {
    if (!dictionary || !residuals || !best_index || !best_score) return ACT_ERR_INVALID_ARG;
    if (n_atoms < 1 || n_atoms > (int64_t)0xFFFFFFFEll) return ACT_ERR_INVALID_ARG;
    if (channels < 1 || channels > kNoAllocMaxChannels) return ACT_ERR_UNSUPPORTED;
    if (row_stride != 128 && row_stride != 256 && row_stride != 384 && row_stride != 512 && row_stride != 1024 &&
        row_stride != 2048)
        return ACT_ERR_UNSUPPORTED;
    if (((uintptr_t)dictionary & 15u) || ((uintptr_t)residuals & 15u)) return ACT_ERR_INVALID_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return ACT_ERR_CUDA;
    unsigned long long *scratch = nullptr;
    int sms = 0;
    {
        // one-time set-up per device, with that device current
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_search_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return ACT_ERR_CUDA;
            }
            int n = 0;
            if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
                cudaGetLastError();
                return ACT_ERR_CUDA;
            }
            g_sm_count[dev] = n;
            g_scratch_addr[dev] = (unsigned long long *)p;
        }
        scratch = g_scratch_addr[dev];
        sms = g_sm_count[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // keys must start at 0 (the search takes an atomic max) and so must the status word
    if (cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * (size_t)(kNoAllocMaxChannels + 1), st) !=
        cudaSuccess)
        return ACT_ERR_CUDA;
    int *status = reinterpret_cast<int *>(scratch + kNoAllocMaxChannels);
    // one channel: the bulk-copy streaming GEMV (the faster stream); several:
    // the load-streaming GEMV, which scores several channels per pass
    const cudaError_t e =
        channels == 1
            ? act::launch_gemv_stream_argmax(dictionary, n_atoms, row_stride, residuals, 1, nullptr, nullptr,
                                             scratch, status, sms, st)
            : act::launch_gemv_argmax(dictionary, n_atoms, row_stride, residuals, channels, nullptr, nullptr,
                                      scratch, status, act::gemv_ctas(sms, row_stride), st);
    if (e != cudaSuccess) return ACT_ERR_CUDA;
    k_noalloc_finish<<<(channels + 127) / 128, 128, 0, st>>>(channels, best_index, best_score);
    if (cudaGetLastError() != cudaSuccess) return ACT_ERR_CUDA;
    return ACT_OK;
}
