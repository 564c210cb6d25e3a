// Allocation-free entry point: the bucket-count prefix sum of the table
// build (K2, decoupled look-back) with its scratch in a file-scope static
// device array instead of a workspace.  The paper has no counterpart; this
// exists for callers that must not allocate device memory (see
// hp_scan_noalloc in include/hashpoint.h).
#include <mutex>

#include "hp_kernels.cuh"

namespace hp {

namespace {

// Scratch layout, in 64-bit words: [0] ticket (low 32 bits), [1..2] status
// word (ErrWord), [3] unused, [4 ..] one look-back word per 2048-entry tile.
constexpr int64_t kNoAllocHead = 4;
constexpr int64_t kNoAllocMaxTiles = HP_SCAN_NOALLOC_MAX_N / kScanTile;
static_assert(HP_SCAN_NOALLOC_MAX_N % kScanTile == 0, "limit must be whole tiles");

// 8 KiWords + 4 = 65,568 bytes (8,192-entry tiles), resident on every device that loads the library.
static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoAllocHead + kNoAllocMaxTiles];

constexpr int kMaxDevices = 128;
std::mutex g_noalloc_mu;
uint64_t *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the static array on the current device.  The symbol's
// name is only a host-side stand-in, so the address is looked up once per
// device (with that device current) and cached.
hp_status noalloc_scratch(uint64_t **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return HP_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return HP_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = static_cast<uint64_t *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return HP_OK;
}

}  // namespace

}  // namespace hp

using namespace hp;

extern "C" hp_status hp_scan_noalloc(const uint32_t *d_in, uint32_t *d_out, int64_t n, int32_t *d_status,
                                     void *stream)
{
    if (n < 0) return HP_ERR_INVALID_ARG;
    if (n > HP_SCAN_NOALLOC_MAX_N) return HP_ERR_TOO_LARGE;
    if (n == 0) return HP_OK;
    if (!d_in || !d_out || ((uintptr_t)d_in & 15u) || ((uintptr_t)d_out & 15u)) return HP_ERR_INVALID_ARG;
    uint64_t *scratch = nullptr;
    hp_status s = noalloc_scratch(&scratch);
    if (s != HP_OK) return s;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t tiles = div_up(n, kScanTile);
    // the array keeps the previous call's contents: clear the ticket, the
    // status word and the look-back words this call uses
    if (cudaMemsetAsync(scratch, 0, sizeof(uint64_t) * (size_t)(kNoAllocHead + tiles), st) != cudaSuccess) {
        cudaGetLastError();
        return HP_ERR_CUDA;
    }
    uint32_t *ticket = reinterpret_cast<uint32_t *>(scratch);
    ErrWord *err = reinterpret_cast<ErrWord *>(scratch + 1);
    k_scan<<<(unsigned)tiles, kScanThreads, 0, st>>>(d_in, d_out, n, scratch + kNoAllocHead, ticket, err,
                                                     kSpinLimitDefault, -1);
    if (cudaGetLastError() != cudaSuccess) return HP_ERR_CUDA;
    if (d_status &&
        cudaMemcpyAsync(d_status, &err->status, sizeof(int32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        return HP_ERR_CUDA;
    }
    return HP_OK;
}
