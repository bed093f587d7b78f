// noalloc.cu -- class probabilities with no device allocation at all.
//
// Some callers cannot call cudaMalloc: a decoder host in a real-time feedback
// loop that runs under a fixed memory budget and may not take the CUDA
// allocator's device-wide locks or trigger its implicit synchronisation, or a
// host application whose device memory is owned by another framework that
// forbids raw allocations.  gp_pmerge_noalloc serves them: it combines the
// component probabilities of each error class the same way the compiler's
// grouping stage does, but its scratch accumulators live in the file-scope
// array below, which every GPU that loads the library holds until exit.
//
// Contract (also stated in gpdem.h):
//  - at most kNoAllocMaxClasses classes per call (8 MiB of accumulators);
//  - the first call on a device looks up the array's device address for that
//    device (cudaGetSymbolAddress) and caches it; make that first call before
//    any stream capture, and do not reset the device after it (the cached
//    address would be stale);
//  - every call clears the accumulators it uses before adding into them, and
//    all calls share the one array, so calls that overlap on the GPU (on
//    different streams, or from different host threads) race.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>

#include "common.cuh"

namespace gpdem {
void set_last_error(const std::string &msg);   // message returned by gp_last_error()

namespace {

constexpr uint32_t kNoAllocMaxClasses = 1u << 19;   // 524,288 classes
constexpr int kNoAllocMaxDevices = 64;

// two 64-bit words (low, high) of a 128-bit fixed-point sum per class
static __device__ __align__(256) unsigned long long g_noalloc_acc[2ull * kNoAllocMaxClasses];

// per device, the array's address once looked up; read with one acquire
// load, so calls after the first take no lock
std::mutex g_noalloc_mu;
std::atomic<unsigned long long *> g_noalloc_ptr[kNoAllocMaxDevices] = {};

__global__ void noalloc_clear(unsigned long long *acc, uint32_t n_classes) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < 2u * n_classes; i += gridDim.x * blockDim.x)
        acc[i] = 0ull;
}

// t_i = -log(1 - 2 q_i) of every member, added to its class as an exact
// 128-bit integer (scale 2^-96), so the sum does not depend on the order in
// which the atomics land.
__global__ void noalloc_accumulate(unsigned long long *acc, const int32_t *mech_class, const float *q,
                                   uint32_t n_mech, uint32_t n_classes) {
    for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < n_mech; m += gridDim.x * blockDim.x) {
        const int32_t c = mech_class[m];
        if (c < 0 || (uint32_t)c >= n_classes) continue;
        const float qi = q[m];
        if (!(qi > 0.0f)) continue;
        float t = -log1pf(-2.0f * qi);
        if (!(t < 1048576.0f)) t = 1048576.0f;          // q >= 1/2 saturates P at 1/2
        unsigned long long lo, hi;
        to_fixed(t, kProbShift, lo, hi);
        acc128_add(&acc[2 * (size_t)c], lo, hi);
    }
}

// P = (1 - exp(-T)) / 2 (Eq. pmerge in closed form), w = log((1 - P) / P)
__global__ void noalloc_finish(const unsigned long long *acc, float *prob, float *logodds, uint32_t n_classes) {
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n_classes; c += gridDim.x * blockDim.x) {
        const float T = fixed_to_float(acc[2 * (size_t)c], acc[2 * (size_t)c + 1], kProbShift);
        const float P = -0.5f * expm1f(-T);
        prob[c] = P;
        if (logodds) logodds[c] = log1pf(-P) - logf(P);
    }
}

}  // namespace
}  // namespace gpdem

using namespace gpdem;

extern "C" gp_status gp_pmerge_noalloc(const int32_t *mech_class, const float *q, uint32_t n_mech,
                                       uint32_t n_classes, float *prob, float *logodds, void *stream) {
    if (n_classes > kNoAllocMaxClasses) {
        set_last_error("gp_pmerge_noalloc: " + std::to_string(n_classes) + " classes requested, at most " +
                       std::to_string(kNoAllocMaxClasses) + " fit the built-in scratch array");
        return GP_ERR_CAPACITY;
    }
    if ((n_mech && (!mech_class || !q)) || (n_classes && !prob)) {
        set_last_error("gp_pmerge_noalloc: null input or output pointer");
        return GP_ERR_INVALID;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_last_error(std::string("gp_pmerge_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return GP_ERR_CUDA;
    }
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_last_error("gp_pmerge_noalloc: device " + std::to_string(dev) + " is beyond the " +
                       std::to_string(kNoAllocMaxDevices) + " devices this entry point supports");
        return GP_ERR_CUDA;
    }
    unsigned long long *acc = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (!acc) {
        // one-time set-up per device, with that device current
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        acc = g_noalloc_ptr[dev].load(std::memory_order_relaxed);
        if (!acc) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_acc);
            if (e != cudaSuccess || !p) {
                set_last_error(std::string("gp_pmerge_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
                return GP_ERR_CUDA;
            }
            acc = static_cast<unsigned long long *>(p);
            g_noalloc_ptr[dev].store(acc, std::memory_order_release);
        }
    }
    if (n_classes == 0) return GP_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t threads = 256;
    const uint32_t g_clear = std::min<uint32_t>((2u * n_classes + threads - 1) / threads, 4096u);
    const uint32_t g_mech = std::min<uint32_t>((n_mech + threads - 1) / threads, 4096u);
    const uint32_t g_cls = std::min<uint32_t>((n_classes + threads - 1) / threads, 4096u);
    noalloc_clear<<<g_clear, threads, 0, s>>>(acc, n_classes);
    if (n_mech) noalloc_accumulate<<<g_mech, threads, 0, s>>>(acc, mech_class, q, n_mech, n_classes);
    noalloc_finish<<<g_cls, threads, 0, s>>>(acc, prob, logodds, n_classes);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string("gp_pmerge_noalloc: launch: ") + cudaGetErrorString(e));
        return GP_ERR_CUDA;
    }
    return GP_OK;
}
