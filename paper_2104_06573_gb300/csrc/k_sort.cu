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

// Order-preserving int encoding of floats (min / max by integer atomics).
__device__ __forceinline__ int ford_s(float f)
{
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float funord_s(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF); }

// Grid cell of a sorted hit: coarse azimuth bin (the fine bin scaled down, so a fine-bin window
// maps onto whole coarse bins) and the bin of its free coordinate (z on a barrel layer, the
// radius on a disk) over the layer's range in the event.
__device__ __forceinline__ uint32_t grid_key(uint32_t g, uint32_t fine, float f, float4 gl,
                                             const DevParams &p)
{
    const uint32_t pc = fine * p.gphi / p.nb;
    int zc = (int)floorf((f - gl.x) * gl.y);
    zc = zc < 0 ? 0 : (zc >= (int)p.gz ? (int)p.gz - 1 : zc);
    return (g * p.gphi + pc) * p.gz + (uint32_t)zc;
}

// One CTA per event.  1) (layer, phi bin) histogram, 2) scan (bucket starts), 3) scatter of the
// sorted hit records; then, when the batch carries a hit grid (the CA stage's lookup), 4) each
// layer's range of the free coordinate (binning) and of the fixed one (the r-z cone), 5) grid
// histogram, 6) scan, 7) scatter of the sorted positions and free coordinates by grid cell.
// The shared counters of steps 1-3 are reused for steps 5-7.
__global__ void __launch_bounds__(1024) k_sort(DevBatch b, DevParams p)
{
    extern __shared__ uint32_t s_cnt[];
    __shared__ uint32_t s_warp[32];
    __shared__ int s_lay[kMaxLayers][4];    // free min, free max, fixed min, fixed max (ordered)
    const uint32_t nk = p.n_keys;
    const bool grid = b.gpos != nullptr;
    for (uint32_t e = blockIdx.x; e < b.E; e += gridDim.x) {
        const uint32_t h0 = b.hit_off[e], n = b.hit_off[e + 1] - h0;
        for (uint32_t k = threadIdx.x; k < nk; k += blockDim.x) s_cnt[k] = 0;
        if (threadIdx.x < kMaxLayers * 4) {
            const uint32_t l = threadIdx.x >> 2, q = threadIdx.x & 3u;
            s_lay[l][q] = (q & 1u) ? ford_s(-3.0e38f) : ford_s(3.0e38f);
        }
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
        if (!grid) continue;
        // ---- hit grid (the grid layers' hits, each layer contiguous in the sorted order) ----
        for (uint32_t L = 0; L < p.n_layers; ++L) {
            if (p.glidx[L] == 0xFF) continue;
            const bool disk = p.is_disk[L];
            int m0 = ford_s(3.0e38f), m1 = ford_s(-3.0e38f), m2 = m0, m3 = m1;
            for (uint32_t t = bk[L * p.nb] + threadIdx.x; t < bk[(L + 1) * p.nb]; t += blockDim.x) {
                const float4 h = b.hs[t];
                const int fr = ford_s(disk ? h.w : h.z), fx = ford_s(disk ? h.z : h.w);
                m0 = min(m0, fr);
                m1 = max(m1, fr);
                m2 = min(m2, fx);
                m3 = max(m3, fx);
            }
            m0 = __reduce_min_sync(0xFFFFFFFFu, m0);
            m1 = __reduce_max_sync(0xFFFFFFFFu, m1);
            m2 = __reduce_min_sync(0xFFFFFFFFu, m2);
            m3 = __reduce_max_sync(0xFFFFFFFFu, m3);
            if ((threadIdx.x & 31u) == 0) {
                atomicMin(&s_lay[L][0], m0);
                atomicMax(&s_lay[L][1], m1);
                atomicMin(&s_lay[L][2], m2);
                atomicMax(&s_lay[L][3], m3);
            }
        }
        __syncthreads();
        const uint32_t gk = p.n_glayers * p.gphi * p.gz;
        float4 *gl = b.glay + (size_t)e * p.n_glayers;
        if (threadIdx.x < p.n_layers && p.glidx[threadIdx.x] != 0xFF) {
            const uint32_t l = threadIdx.x;
            const float f0 = funord_s(s_lay[l][0]), f1 = funord_s(s_lay[l][1]);
            const float scale = f1 > f0 ? (float)p.gz / (f1 - f0) : 0.f;
            gl[p.glidx[l]] = make_float4(f0, scale, funord_s(s_lay[l][2]), funord_s(s_lay[l][3]));
        }
        for (uint32_t k = threadIdx.x; k < gk; k += blockDim.x) s_cnt[k] = 0;
        __syncthreads();
        // the grid layers' hits, layer by layer (positions [bk[L nb], bk[(L + 1) nb]))
        auto for_grid_hits = [&](auto &&fn) {
            for (uint32_t L = 0; L < p.n_layers; ++L) {
                const uint32_t g = p.glidx[L];
                if (g == 0xFF) continue;
                const float4 glg = gl[g];
                for (uint32_t t = bk[L * p.nb] + threadIdx.x; t < bk[(L + 1) * p.nb];
                     t += blockDim.x) {
                    const float4 h = b.hs[t];
                    const float f = p.is_disk[L] ? h.w : h.z;
                    fn(t, f, grid_key(g, phi_bin(b.hphi[t], p), f, glg, p));
                }
            }
        };
        for_grid_hits([&](uint32_t, float, uint32_t key) { atomicAdd(&s_cnt[key], 1u); });
        __syncthreads();
        const uint32_t gtotal = block_exclusive_scan(s_cnt, gk, s_warp);
        uint32_t *go = b.gofs + (size_t)e * (gk + 1);
        for (uint32_t k = threadIdx.x; k < gk; k += blockDim.x) go[k] = h0 + s_cnt[k];
        if (threadIdx.x == 0) go[gk] = h0 + gtotal;
        __syncthreads();
        for_grid_hits([&](uint32_t t, float f, uint32_t key) {
            const uint32_t q = h0 + atomicAdd(&s_cnt[key], 1u);
            b.gpos[q] = t;
            b.gfree[q] = f;
        });
        __syncthreads();
    }
}

cudaError_t init_kernels()
{
    // up to 16 layers x 2048 bins of 4-byte counters (the hit grid's counters are fewer)
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
    const uint32_t gk = b.gpos ? p.n_glayers * p.gphi * p.gz : 0u;
    const size_t smem = (size_t)(p.n_keys > gk ? p.n_keys : gk) * sizeof(uint32_t);
    k_sort<<<grid, p.block_threads[0], smem, s>>>(b, p);
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
