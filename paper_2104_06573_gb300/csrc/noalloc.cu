// Doublet building for one event without any device allocation.
//
// Some callers cannot let a library allocate device memory: serving loops that must never call
// cudaMalloc after start-up (it synchronises the device and stalls every other stream, which
// breaks latency targets), and applications whose device memory is entirely owned by their own
// pool allocator, leaving nothing for a library to cudaMalloc.  For them this file provides one
// entry point that uses no scratch beyond a fixed-size array in device global memory
// (`g_scratch`, a file-scope `static __device__` array that every GPU loading the library holds
// until the process exits).  The caller passes inputs and outputs; nothing is allocated.
//
// Limits: at most kNaMaxHits hits and kNaMaxCells cells per call, layers x phi bins as for the
// other entry points.  All calls share g_scratch, which keeps the last call's contents: calls
// whose work overlaps on the GPU (different streams or threads without ordering) race on it.
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/pxr.h"
#include "pxr_dev.cuh"

namespace pxr {

constexpr uint32_t kNaMaxHits = 65536;
constexpr uint32_t kNaMaxCells = 1u << 20;
constexpr uint32_t kNaMaxKeys = kMaxLayers * 2048;

// Byte layout of the scratch array (all offsets 256-aligned).
constexpr size_t na_align(size_t v) { return (v + 255) & ~size_t(255); }
constexpr size_t kNaHitOff = 0;                                         // 2 x u32
constexpr size_t kNaCellOff = na_align(kNaHitOff + 8);                  // 2 x u32
constexpr size_t kNaCnt = na_align(kNaCellOff + 8);                     // kCounters x u32
constexpr size_t kNaBkt = na_align(kNaCnt + 4 * kCounters);             // (keys + 1) x u32
constexpr size_t kNaHs = na_align(kNaBkt + 4 * (kNaMaxKeys + 1));       // hits x float4
constexpr size_t kNaR64 = na_align(kNaHs + 16 * (size_t)kNaMaxHits);     // hits x double
constexpr size_t kNaMeta = na_align(kNaR64 + 8 * (size_t)kNaMaxHits);    // hits x u32
constexpr size_t kNaItem = na_align(kNaMeta + 4 * (size_t)kNaMaxHits);   // hits x 4 x uint4
constexpr size_t kNaPhi = na_align(kNaItem + 64 * (size_t)kNaMaxHits);    // hits x float
constexpr size_t kNaHitChunk = na_align(kNaPhi + 4 * (size_t)kNaMaxHits); // hit chunks x u32
constexpr size_t kNaBytes = na_align(kNaHitChunk + 4 * (size_t)(kNaMaxHits / kHitChunk));  // ~6.4 MB

static __device__ __align__(256) unsigned char g_scratch[kNaBytes];

// Sorted hit positions of the cells -> the caller's hit indices (in place).
__global__ void k_na_to_caller(uint32_t *inner, uint32_t *outer, const uint32_t *n_cells,
                               uint32_t cap)
{
    const uint32_t *cnt = reinterpret_cast<const uint32_t *>(g_scratch + kNaCnt);
    const uint32_t *meta = reinterpret_cast<const uint32_t *>(g_scratch + kNaMeta);
    const uint32_t n = min(cnt[C_CELLS], cap);
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        inner[c] = meta[inner[c]] & kLocalMask;
        outer[c] = meta[outer[c]] & kLocalMask;
    }
    (void)n_cells;
}

// Event bounds of the single event and zeroed counters.
__global__ void k_na_init(uint32_t n_hits, uint32_t cap)
{
    uint32_t *hit_off = reinterpret_cast<uint32_t *>(g_scratch + kNaHitOff);
    uint32_t *cell_off = reinterpret_cast<uint32_t *>(g_scratch + kNaCellOff);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(g_scratch + kNaCnt);
    if (threadIdx.x == 0) {
        hit_off[0] = 0;
        hit_off[1] = n_hits;
        cell_off[0] = 0;
        cell_off[1] = cap;
    }
    if (threadIdx.x < kCounters) cnt[threadIdx.x] = 0;
    // one event: every hit chunk belongs to event 0
    uint32_t *hc = reinterpret_cast<uint32_t *>(g_scratch + kNaHitChunk);
    for (uint32_t c = threadIdx.x; c < kNaMaxHits / kHitChunk; c += blockDim.x) hc[c] = 0;
}

// Copy the cell count (and the overflow flag) to the caller.
__global__ void k_na_count(uint32_t *n_cells, uint32_t *flags)
{
    const uint32_t *cnt = reinterpret_cast<const uint32_t *>(g_scratch + kNaCnt);
    if (threadIdx.x == 0) {
        n_cells[0] = cnt[C_CELLS];
        if (flags) flags[0] = cnt[C_FLAGS];
    }
}

// Parameter derivation and error reporting shared with the other entry points.
int dev_params(const pxr_params *p, DevParams *d);
int set_error(int code, const char *msg);
inline int set_error(int code, const std::string &msg) { return set_error(code, msg.c_str()); }

}  // namespace pxr

using namespace pxr;

namespace {
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mu;
unsigned char *g_na_ptr[kNaMaxDevices] = {};
}  // namespace

extern "C" int pxr_doublets_noalloc(const float *x, const float *y, const float *z,
                                    const uint16_t *layer, uint32_t n_hits,
                                    const pxr_params *params, uint32_t *cells_inner,
                                    uint32_t *cells_outer, uint32_t cap, uint32_t *n_cells,
                                    uint32_t *flags, void *stream)
{
    if (!params || !cells_inner || !cells_outer || !n_cells || (n_hits && (!x || !y || !z || !layer)))
        return set_error(PXR_EINVAL, "null argument");
    if (n_hits > kNaMaxHits)
        return set_error(PXR_EINVAL, "n_hits exceeds the 65536-hit limit of pxr_doublets_noalloc");
    if (cap > kNaMaxCells)
        return set_error(PXR_EINVAL, "cap exceeds the 1048576-cell limit of pxr_doublets_noalloc");
    DevParams dp;
    int rc = dev_params(params, &dp);
    if (rc != PXR_OK) return rc;
    if (dp.n_keys > kNaMaxKeys) return set_error(PXR_EINVAL, "too many layer x phi-bin keys");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices)
        return set_error(PXR_ECUDA, "cudaGetDevice failed");
    unsigned char *base = nullptr;
    {
        // Once per device, with that device current: resolve the array's device address (host
        // code may not use g_scratch's host-side name as an address) and set the kernel
        // attributes.  This happens in the first call on each device.
        std::lock_guard<std::mutex> g(g_na_mu);
        if (!g_na_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess) return set_error(PXR_ECUDA, cudaGetErrorString(e));
            e = init_kernels();
            if (e != cudaSuccess) return set_error(PXR_ECUDA, cudaGetErrorString(e));
            g_na_ptr[dev] = static_cast<unsigned char *>(p);
        }
        base = g_na_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    DevBatch b;
    std::memset(&b, 0, sizeof b);
    b.E = 1;
    b.N = n_hits;
    b.C = cap;
    b.x = x;
    b.y = y;
    b.z = z;
    b.layer = layer;
    b.hit_off = reinterpret_cast<const uint32_t *>(base + kNaHitOff);
    b.cell_off = reinterpret_cast<const uint32_t *>(base + kNaCellOff);
    b.cnt = reinterpret_cast<uint32_t *>(base + kNaCnt);
    b.bkt = reinterpret_cast<uint32_t *>(base + kNaBkt);
    b.hs = reinterpret_cast<float4 *>(base + kNaHs);
    b.r64 = reinterpret_cast<double *>(base + kNaR64);
    b.hmeta = reinterpret_cast<uint32_t *>(base + kNaMeta);
    b.item = reinterpret_cast<uint4 *>(base + kNaItem);
    b.cell_in = cells_inner;
    b.cell_out = cells_outer;
    b.hphi = reinterpret_cast<float *>(base + kNaPhi);
    b.hit_chunk = reinterpret_cast<const uint32_t *>(base + kNaHitChunk);
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // An error left pending by earlier work of the process is reported as such (and left in
    // place for its owner), not blamed on the launches below.
    cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess)
        return set_error(PXR_ECUDA, std::string("CUDA error pending before the call: ") +
                                        cudaGetErrorString(pending));
    // Each launch is checked right after it is issued, so that the message names it.
    auto check = [](const char *what) {
        const cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) return PXR_OK;
        return set_error(PXR_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    };
    k_na_init<<<1, 32, 0, s>>>(n_hits, cap);
    if ((rc = check("launch of the scratch initialisation")) != PXR_OK) return rc;
    launch_sort(b, dp, s, sms);
    if ((rc = check("launch of the hit sort")) != PXR_OK) return rc;
    launch_doublets_compact(b, dp, s, sms);
    if ((rc = check("launch of the doublet kernel")) != PXR_OK) return rc;
    k_na_to_caller<<<sms * 4, 256, 0, s>>>(cells_inner, cells_outer, n_cells, cap);
    if ((rc = check("launch of the index conversion")) != PXR_OK) return rc;
    k_na_count<<<1, 32, 0, s>>>(n_cells, flags);
    return check("launch of the count copy");
}
