// sort_static.cu -- the (key, value) radix sort for callers that cannot
// allocate device memory.
//
// Some callers may not call cudaMalloc on the path where they sort: a host
// framework that owns every device allocation through its own pool and
// forbids raw cudaMalloc from plug-ins, or latency-critical code where the
// implicit device-wide synchronisation of cudaMalloc / cudaFree would stall
// other work.  fgs_sort_pairs needs a caller-provided scratch buffer and
// two ping-pong buffers; fgs_sort_pairs_static instead uses one scratch
// array that the library itself owns: a file-scope __device__ array of
// fixed size that every GPU loading the library holds until the process
// exits.  The caller passes only the keys and values, and gets them back
// sorted in place.
//
// The array's name is a host-side stand-in in host code, never a device
// address, so this file looks the device address up with
// cudaGetSymbolAddress once per device (with that device current) and
// passes that pointer to the kernels.  The address is cached per device
// number, for the context the CUDA runtime uses there (the primary
// context): after cudaDeviceReset, or with another context made current
// through the driver API, the cached address is no longer valid.
#include <mutex>

#include "fgs_common.cuh"

namespace fgs {
int radix_sort(unsigned long long* keys, uint32_t* vals, unsigned long long* keys_alt,
               uint32_t* vals_alt, int64_t n_max, const uint32_t* n_dev, int bits, uint32_t* hist,
               cudaStream_t st, cudaError_t* err);
cudaError_t launch_set_count(uint32_t* dst, uint32_t value, cudaStream_t st);
size_t sort_hist_bytes(int64_t n_max, int rb);

namespace {

constexpr int64_t kMaxPairs = FGS_STATIC_SORT_MAX_PAIRS;
constexpr size_t kCountBytes = 256;
constexpr size_t kKeysBytes = sizeof(unsigned long long) * (size_t)kMaxPairs;
constexpr size_t kValsBytes = sizeof(uint32_t) * (size_t)kMaxPairs;
// radix histograms: 256 digits x (kMaxPairs / 4096) tiles, digit totals, slack
constexpr size_t kHistBytes = sizeof(uint32_t) * (256 * (kMaxPairs / 4096) + 256 + 64);
constexpr size_t kScratchBytes = kCountBytes + kKeysBytes + kValsBytes + kHistBytes;

// The scratch every call shares: [count | keys ping-pong | values ping-pong | histograms].
static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
unsigned char* g_scratch_dev[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device (looked up once).
int scratch_on_current_device(unsigned char** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FGS_ERR_CUDA;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess || !p) return FGS_ERR_CUDA;
        g_scratch_dev[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_dev[dev];
    return FGS_OK;
}

}  // namespace
}  // namespace fgs

using namespace fgs;

extern "C" int fgs_sort_pairs_static(uint64_t* keys, uint32_t* vals, int64_t n, int32_t bits,
                                     void* stream)
{
    if (n < 0) return FGS_ERR_SHAPE;
    if (n > kMaxPairs) return FGS_ERR_TOO_LARGE;
    if (bits < 1 || bits > 64) return FGS_ERR_ARG;
    if (n == 0) return FGS_OK;
    if (!keys || !vals) return FGS_ERR_NULL;
    // 8-byte key and 4-byte value accesses
    if ((uintptr_t)keys % 8 != 0 || (uintptr_t)vals % 4 != 0) return FGS_ERR_ALIGN;
    if (sort_hist_bytes(n, 8) > kHistBytes) return FGS_ERR_TOO_LARGE;
    unsigned char* base = nullptr;
    const int rc = scratch_on_current_device(&base);
    if (rc != FGS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t* n_dev = reinterpret_cast<uint32_t*>(base);
    unsigned long long* keys_alt = reinterpret_cast<unsigned long long*>(base + kCountBytes);
    uint32_t* vals_alt = reinterpret_cast<uint32_t*>(base + kCountBytes + kKeysBytes);
    uint32_t* hist = reinterpret_cast<uint32_t*>(base + kCountBytes + kKeysBytes + kValsBytes);
    // Every word the sort reads is written earlier in the same call (count,
    // then each pass's histograms), so nothing needs clearing.
    if (launch_set_count(n_dev, (uint32_t)n, st) != cudaSuccess) return FGS_ERR_CUDA;
    cudaError_t e = cudaSuccess;
    const int alt = radix_sort(reinterpret_cast<unsigned long long*>(keys), vals, keys_alt, vals_alt, n,
                               n_dev, bits, hist, st, &e);
    if (e != cudaSuccess) return FGS_ERR_CUDA;
    if (alt) {
        if (cudaMemcpyAsync(keys, keys_alt, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToDevice, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(vals, vals_alt, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st) !=
                cudaSuccess)
            return FGS_ERR_CUDA;
    }
    return FGS_OK;
}
