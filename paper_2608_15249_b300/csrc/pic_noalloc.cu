// pic_noalloc.cu -- the per-cell sort permutation for callers that cannot
// allocate device memory.
//
// Some callers of this library may not call cudaMalloc: a host framework that
// owns all of the device's memory through its own pool, or a hot loop that
// cannot afford the device-wide synchronisation that cudaMalloc / cudaFree
// imply.  ap_pic_sort_perm_noalloc runs the same stable radix sort as
// ap_pic_sort, but its scratch (keys, indices, digit histograms, scan
// partials) lives in one fixed-size array in device global memory declared in
// this file.  Every GPU that loads the library holds the array
// (~17 MiB) until the process exits; the caller passes only its input and
// output buffers.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so the first call on each device, with that
// device current, looks the address up with cudaGetSymbolAddress and keeps it
// for the life of the process.  That first call must therefore come before any
// stream capture, and a caller that resets the device (cudaDeviceReset, which
// unloads this library's module and its array) must not call the entry point on
// that device again: the kept address would be stale.
// Every call shares the array: calls whose work overlaps on the GPU (different
// streams, or different host threads on the same device) race on it and must
// be ordered by the caller.  No word of the scratch needs to start at zero:
// each call writes every word it reads before reading it.
#include <cuda_runtime.h>

#include <mutex>

#include "ap_pic.h"
#include "pic_internal.cuh"

using namespace apk;

namespace {

constexpr int64_t MAX_NP = AP_PIC_NOALLOC_MAX_NP;
constexpr size_t TILE = SORT_TILE;                          // items per sort tile
constexpr size_t MAX_TILES = (size_t)(MAX_NP + TILE - 1) / TILE;
constexpr size_t HIST_WORDS = (size_t)SORT_MAX_RADIX * MAX_TILES;  // per-tile digit histograms
constexpr size_t SCAN_WORDS = 256;                          // scan partials (checked below)
constexpr size_t SCRATCH_WORDS = 4 * (size_t)MAX_NP + HIST_WORDS + SCAN_WORDS;
constexpr int MAX_DEVICES = 64;

std::mutex g_mu;
uint32_t *g_addr[MAX_DEVICES] = {nullptr};

}  // namespace

// The shared scratch: keys[2], indices[2] (MAX_NP words each), histograms, scan partials.
static __device__ __align__(256) uint32_t g_noalloc_scratch[SCRATCH_WORDS];

// Device address of the scratch on the current device (looked up once per device).
static ap_pic_status scratch_address(uint32_t **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return AP_PIC_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return AP_PIC_ERR_CUDA;
        }
        g_addr[dev] = static_cast<uint32_t *>(ptr);
    }
    *out = g_addr[dev];
    return AP_PIC_OK;
}

extern "C" ap_pic_status ap_pic_sort_perm_noalloc(int ndim, const int *n, const int *brick,
                                                  int64_t np, const int32_t *cell, int32_t *perm,
                                                  void *cuda_stream)
{
    if (ndim < 1 || ndim > 3 || !n || !brick || np < 0) return AP_PIC_ERR_ARG;
    if (np > MAX_NP) return AP_PIC_ERR_TOO_LARGE;
    if (np == 0) return AP_PIC_OK;
    if (!cell || !perm) return AP_PIC_ERR_ARG;
    if (sort_scan_tmp_len(HIST_WORDS) > SCAN_WORDS) return AP_PIC_ERR_TOO_LARGE;
    GridParams g{};
    g.ndim = ndim;
    int b[3] = {1, 1, 1};
    int64_t nkeys = 1;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = 1;
        if (a >= ndim) continue;
        if (n[a] < 2 || brick[a] < 0) return AP_PIC_ERR_ARG;
        g.n[a] = n[a];
        b[a] = brick[a] == 0 ? (ndim == 1 ? 64 : 8) : brick[a];
        if (b[a] > n[a]) b[a] = n[a];
        nkeys *= (int64_t)((n[a] + b[a] - 1) / b[a]) * b[a];
    }
    if (nkeys > (int64_t(1) << 32)) return AP_PIC_ERR_ARG;
    int key_bits = 0;
    for (uint64_t k = (uint64_t)(nkeys - 1); k; k >>= 1) ++key_bits;

    uint32_t *base = nullptr;
    const ap_pic_status st = scratch_address(&base);
    if (st != AP_PIC_OK) return st;
    SortScratch s{};
    s.keys[0] = base;
    s.keys[1] = base + MAX_NP;
    s.idx[0] = base + 2 * MAX_NP;
    s.idx[1] = base + 3 * MAX_NP;
    s.hist = base + 4 * MAX_NP;
    s.scan_tmp = s.hist + HIST_WORDS;
    s.scan_tmp_len = SCAN_WORDS;
    s.capacity = MAX_NP;

    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    int slot = 0;
    if (launch_sort_perm(g, b, key_bits, cell, np, s, &slot, stream) != cudaSuccess ||
        cudaMemcpyAsync(perm, s.idx[slot], (size_t)np * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                        stream) != cudaSuccess) {
        cudaGetLastError();
        return AP_PIC_ERR_CUDA;
    }
    return AP_PIC_OK;
}
