// noalloc.cu -- the per-tile depth sort for callers that cannot allocate device
// memory.
//
// Some callers cannot call cudaMalloc: memory-capped tenants of a shared GPU
// whose budget is handed out by someone else, hosts that own every byte of
// device memory through their own allocator, and latency-bound loops that cannot
// afford the device-wide synchronization an allocation or a free may bring.  For them,
// tsp_sort_tiles_noalloc() sorts caller-owned per-tile key lists in place and
// keeps the merge scratch it needs for long lists in a fixed array compiled into
// the library (TSP_NOALLOC_SORT_MAX_KEYS keys, 8 MB), which every GPU that loads
// the library holds until the process exits.  Nothing here calls cudaMalloc,
// cudaFree or an allocating library routine.
#include <mutex>

#include "launch.h"

namespace tsp {

namespace {

// Shared by every call on a device; its contents are whatever the last call left.
// Nothing in it needs to start at zero: a call writes every element it reads.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[TSP_NOALLOC_SORT_MAX_KEYS];

constexpr int kCap = 4096;
constexpr int kThreads = 256;
constexpr int kMaxDevices = 128;

void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Bitonic sort of n <= kCap keys in shared memory, written back in place.
__device__ void sort_in_smem(unsigned long long* keys, uint32_t n, unsigned long long* s)
{
    uint32_t P = 2;
    while (P < n) P <<= 1;
    for (uint32_t i = threadIdx.x; i < P; i += kThreads) s[i] = i < n ? keys[i] : ~0ull;
    __syncthreads();
    for (uint32_t k = 2; k <= P; k <<= 1)
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < P; i += kThreads) {
                const uint32_t l = i ^ j;
                if (l > i) {
                    const unsigned long long a = s[i], b = s[l];
                    if ((a > b) == ((i & k) == 0)) { s[i] = b; s[l] = a; }
                }
            }
            __syncthreads();
        }
    for (uint32_t i = threadIdx.x; i < n; i += kThreads) keys[i] = s[i];
    __syncthreads();
}

// One CTA per tile.  Lists longer than kCap are sorted in kCap runs and merged
// pairwise through the static scratch (slice [off[t], off[t+1]) of it, so tiles
// never share scratch); each key finds its merged slot by binary search in the
// partner run.  A key of the left run counts the partner's keys below it, a key
// of the right run those not above it, so equal keys in the two runs land on
// distinct slots (left run first) and every slot is written once.
__global__ void __launch_bounds__(kThreads) k_sort_tiles_noalloc(unsigned long long* keys,
                                                                 const uint32_t* __restrict__ off,
                                                                 uint32_t num_keys,
                                                                 unsigned long long* scratch)
{
    __shared__ unsigned long long s[kCap];
    const uint32_t t = blockIdx.x;
    const uint32_t b = min(off[t], num_keys), e = min(off[t + 1], num_keys);
    if (e <= b + 1) return;
    const uint32_t n = e - b;
    if (n <= (uint32_t)kCap) {
        sort_in_smem(keys + b, n, s);
        return;
    }
    for (uint32_t c = 0; c < n; c += kCap) sort_in_smem(keys + b + c, min((uint32_t)kCap, n - c), s);
    unsigned long long* src = keys + b;
    unsigned long long* dst = scratch + b;
    for (uint32_t L = kCap; L < n; L <<= 1) {
        for (uint32_t i = threadIdx.x; i < n; i += kThreads) {
            const uint32_t run = i / L, start = run * L, partner = run ^ 1u;
            const unsigned long long key = src[i];
            const uint64_t ps64 = (uint64_t)partner * L;
            if (ps64 >= n) { dst[i] = key; continue; }
            const uint32_t ps = (uint32_t)ps64, pe = min(ps + L, n);
            const bool left = run < partner;
            uint32_t lo = ps, hi = pe;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                const unsigned long long m = src[mid];
                if (left ? (m < key) : (m <= key)) lo = mid + 1; else hi = mid;
            }
            dst[min(run, partner) * L + (i - start) + (lo - ps)] = key;
        }
        __syncthreads();
        unsigned long long* x = src; src = dst; dst = x;
    }
    if (src != keys + b)
        for (uint32_t i = threadIdx.x; i < n; i += kThreads) keys[b + i] = src[i];
}

}  // namespace

}  // namespace tsp

extern "C" tsp_status tsp_sort_tiles_noalloc(uint64_t* keys, const uint32_t* offsets, uint32_t num_tiles,
                                             uint32_t num_keys, void* stream)
{
    using namespace tsp;
    if (num_keys > TSP_NOALLOC_SORT_MAX_KEYS) return TSP_ERR_INVALID_ARG;
    if (num_tiles == 0 || num_keys == 0) return TSP_OK;
    if (!keys || !offsets || ((uintptr_t)keys % 8) != 0 || ((uintptr_t)offsets % 4) != 0)
        return TSP_ERR_INVALID_ARG;
    if (num_tiles > (uint32_t)INT32_MAX) return TSP_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return TSP_ERR_CUDA;
    }
    void* scratch = nullptr;
    {
        // once per device, with that device current: the device address of the
        // static array (its host-side name is only a stand-in)
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return TSP_ERR_CUDA;
            }
            g_scratch_addr[dev] = p;
        }
        scratch = g_scratch_addr[dev];
    }
    k_sort_tiles_noalloc<<<num_tiles, kThreads, 0, (cudaStream_t)stream>>>(
        (unsigned long long*)keys, offsets, num_keys, (unsigned long long*)scratch);
    return cudaGetLastError() == cudaSuccess ? TSP_OK : TSP_ERR_CUDA;
}
