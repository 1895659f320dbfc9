// Per-layer phi-binned counting sort of each event's hits (count -> exclusive scan -> scatter).
//
// One CTA owns one event at a time: the (layer, phi bin) histogram lives in shared memory, the
// scan runs in the CTA, and the scatter writes the sorted hit records (x, y, z, r as float4), the
// FP64 radius and the hit's layer and caller index.  Bucket start positions are written per
// event so that later stages read a layer's phi window as one or two contiguous ranges.
// The bin of a hit is floor((atan2f(y, x) + pi) * nb / 2pi), clamped; later stages widen every
// phi window by a margin far above atan2f's error, and the exact cut decides, so the binning
// never changes a result.
#include "pxr_dev.cuh"
#include "pxr_cuts.cuh"

namespace pxr {

constexpr float kPiF = 3.14159265358979f;

__device__ __forceinline__ uint32_t phi_bin(float phi, const DevParams &p)
{
    float t = floorf((phi + kPiF) * p.bins_per_rad);
    int b = (int)t;
    b = b < 0 ? 0 : b;
    return (uint32_t)(b >= (int)p.nb ? (int)p.nb - 1 : b);
}

// Block-wide exclusive scan of s[0..n) in place; returns the total.  blockDim.x is a multiple
// of 32 and at most 1024.
__device__ uint32_t block_exclusive_scan(uint32_t *s, uint32_t n, uint32_t *warp_tot)
{
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    const uint32_t per = (n + nt - 1) / nt;
    const uint32_t b0 = min(n, tid * per), b1 = min(n, b0 + per);
    uint32_t local = 0;
    for (uint32_t k = b0; k < b1; ++k) local += s[k];
    // inclusive scan of `local` across the block
    const uint32_t lane = tid & 31u, wid = tid >> 5;
    uint32_t v = local;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= (uint32_t)o) v += t;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
        uint32_t nw = nt >> 5;
        uint32_t w = lane < nw ? warp_tot[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= (uint32_t)o) w += t;
        }
        if (lane < nw) warp_tot[lane] = w;     // inclusive warp prefix
    }
    __syncthreads();
    uint32_t excl = v - local + (wid ? warp_tot[wid - 1] : 0u);
    uint32_t total = warp_tot[(nt >> 5) - 1];
    for (uint32_t k = b0; k < b1; ++k) {
        uint32_t c = s[k];
        s[k] = excl;
        excl += c;
    }
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(1024) k_sort(DevBatch b, DevParams p)
{
    extern __shared__ uint32_t s_cnt[];
    __shared__ uint32_t s_warp[32];
    const uint32_t nk = p.n_keys;
    for (uint32_t e = blockIdx.x; e < b.E; e += gridDim.x) {
        const uint32_t h0 = b.hit_off[e], n = b.hit_off[e + 1] - h0;
        for (uint32_t k = threadIdx.x; k < nk; k += blockDim.x) s_cnt[k] = 0;
        __syncthreads();
        bool bad = false;
        for (uint32_t h = threadIdx.x; h < n; h += blockDim.x) {
            uint32_t g = h0 + h;
            uint32_t L = b.layer[g];
            if (L >= p.n_layers) { bad = true; continue; }
            atomicAdd(&s_cnt[L * p.nb + phi_bin(atan2f(b.y[g], b.x[g]), p)], 1u);
        }
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&b.cnt[C_FLAGS * b.E + e], F_LAYER);
        uint32_t total = block_exclusive_scan(s_cnt, nk, s_warp);
        uint32_t *bk = b.bkt + (size_t)e * (nk + 1);
        for (uint32_t k = threadIdx.x; k < nk; k += blockDim.x) bk[k] = h0 + s_cnt[k];
        if (threadIdx.x == 0) bk[nk] = h0 + total;
        // positions past the valid hits (inputs with a bad layer) get layer 0xFF in their record
        for (uint32_t h = total + threadIdx.x; h < n; h += blockDim.x) b.hmeta[h0 + h] = 0xFFFFFFFFu;
        __syncthreads();
        for (uint32_t h = threadIdx.x; h < n; h += blockDim.x) {
            uint32_t g = h0 + h;
            uint32_t L = b.layer[g];
            if (L >= p.n_layers) continue;
            float x = b.x[g], y = b.y[g], z = b.z[g];
            const float phi = atan2f(y, x);
            uint32_t pos = h0 + atomicAdd(&s_cnt[L * p.nb + phi_bin(phi, p)], 1u);
            double r = radius64((double)x, (double)y);
            b.hs[pos] = make_float4(x, y, z, __double2float_rn(r));
            b.r64[pos] = r;
            b.hmeta[pos] = (L << kLocalBits) | h;
            b.hphi[pos] = phi;
        }
        __syncthreads();
    }
}

cudaError_t init_kernels()
{
    // up to 16 layers x 2048 bins of 4-byte counters
    cudaError_t e = cudaFuncSetAttribute(k_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kMaxLayers * 2048 * (int)sizeof(uint32_t));
    if (e != cudaSuccess) return e;
    return init_fit_kernels();
}

void launch_sort(const DevBatch &b, const DevParams &p, cudaStream_t s, int sms)
{
    const uint32_t cap = (uint32_t)sms * p.grid_per_sm[0];
    const uint32_t grid = b.E < cap ? b.E : cap;
    if (grid == 0) return;
    k_sort<<<grid, 1024, p.n_keys * sizeof(uint32_t), s>>>(b, p);
}

// Per-event, per-layer hit counts (used once to size a plan's per-event capacities).
__global__ void k_layer_count(const uint32_t *hit_off, const uint16_t *layer, uint32_t E,
                              uint32_t n_layers, uint32_t *counts)
{
    __shared__ uint32_t s[kMaxLayers + 1];
    for (uint32_t e = blockIdx.x; e < E; e += gridDim.x) {
        if (threadIdx.x <= kMaxLayers) s[threadIdx.x] = 0;
        __syncthreads();
        for (uint32_t g = hit_off[e] + threadIdx.x; g < hit_off[e + 1]; g += blockDim.x) {
            uint32_t L = layer[g];
            atomicAdd(&s[L < n_layers ? L : kMaxLayers], 1u);
        }
        __syncthreads();
        if (threadIdx.x <= kMaxLayers) counts[(size_t)e * (kMaxLayers + 1) + threadIdx.x] = s[threadIdx.x];
        __syncthreads();
    }
}

void launch_layer_count(const uint32_t *hit_off, const uint16_t *layer, uint32_t E,
                        uint32_t n_layers, uint32_t *counts, cudaStream_t s, int sms)
{
    uint32_t grid = E < (uint32_t)(sms * 4) ? E : (uint32_t)(sms * 4);
    if (grid == 0) return;
    k_layer_count<<<grid, 256, 0, s>>>(hit_off, layer, E, n_layers, counts);
}

}  // namespace pxr
