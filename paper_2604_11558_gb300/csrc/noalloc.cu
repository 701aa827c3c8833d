// sexpe_step_noalloc: the split-TF32 step with its scratch memory in a static
// device array, for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not wanted
// -- inside a region being captured into a CUDA graph under the global capture
// mode (allocation calls are prohibited there), inside a host framework that
// owns every device allocation through its own pool and forbids plugins from
// calling cudaMalloc, or in a loop with a hard memory budget that must not
// grow.  Such a caller still brings a plan made earlier (its constant tables)
// and its own state buffer; the only extra memory a step needs, the FP32
// intermediate between the mode-3 pass and the slab pass, comes from the
// array below instead.
//
// The array is g_step_scratch: kNoAllocScratchFloats FP32 values (8 MiB).
// Every GPU that loads this library holds it until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "sexpe.h"

namespace sexpe {
sexpe_status check_split_step_with_scratch(const sexpe_plan* p, const double* state, const float* Y,
                                           long long y_floats);
sexpe_status zero_scratch_padding(const sexpe_plan* p, float* Y, cudaStream_t st);
sexpe_status enqueue_split_step_with_scratch(sexpe_plan* p, double* state, float* Y, long long y_floats,
                                             cudaStream_t st);
}

namespace {

// 2^21 floats = 8 MiB: enough for species x points <= 2,097,152, with every
// rho line padded to a multiple of 4 points (the two-species 100^3 ball needs
// 2,000,000).
constexpr long long kNoAllocScratchFloats = 2LL * 1024 * 1024;

static __device__ __align__(256) float g_step_scratch[kNoAllocScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float* g_scratch_ptr[kMaxDevices] = {};   // device address of g_step_scratch, per device

// Once per device, with that device current: the host-side name of the array is
// only a stand-in, so ask the runtime for its device address.
sexpe_status scratch_for_current_device(float** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SEXPE_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return SEXPE_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_step_scratch);
        if (e != cudaSuccess || !ptr) return SEXPE_ECUDA;
        g_scratch_ptr[dev] = static_cast<float*>(ptr);
    }
    *out = g_scratch_ptr[dev];
    return SEXPE_OK;
}

}  // namespace

extern "C" sexpe_status sexpe_step_noalloc(sexpe_plan* plan, double* state_dev, int64_t n_steps, void* stream) {
    if (!plan || !state_dev || n_steps < 0) return SEXPE_EINVAL;
    float* scratch = nullptr;
    const sexpe_status s = scratch_for_current_device(&scratch);
    if (s != SEXPE_OK) return s;
    // Everything is checked before the first launch: the plan (split-TF32, single grid, made on
    // this device), the state's 8-byte alignment and the scratch capacity.
    const sexpe_status c = sexpe::check_split_step_with_scratch(plan, state_dev, scratch, kNoAllocScratchFloats);
    if (c != SEXPE_OK || n_steps == 0) return c;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Every step's first kernel writes all species x points values of the intermediate before a
    // later kernel reads them.  The padding slots of the rho lines (n_rho not a multiple of 4) are
    // never written by a step and hold whatever an earlier call with another layout left there
    // (possibly non-finite); they are zeroed here, as the plan's own buffer is at setup, so that
    // results equal sexpe_step's bit for bit.
    const sexpe_status z = sexpe::zero_scratch_padding(plan, scratch, st);
    if (z != SEXPE_OK) return z;
    for (int64_t k = 0; k < n_steps; ++k) {
        const sexpe_status r = sexpe::enqueue_split_step_with_scratch(plan, state_dev, scratch, kNoAllocScratchFloats, st);
        if (r != SEXPE_OK) return r;
    }
    return SEXPE_OK;
}
