// Per-layer phi-binned counting sort of each event's hits (count -> exclusive scan -> scatter).
//
// One thread-block cluster owns one event at a time: the (layer, phi bin) histogram lives in the
// cluster's distributed shared memory, the scan runs in the cluster, and the scatter writes the
// sorted hit records (x, y, z, r as float4), the FP64 radius and the hit's layer and caller
// index.  Bucket start positions are written per event so that later stages read a layer's phi
// window as one or two contiguous ranges.
// The bin of a hit is floor((atan2f(y, x) + pi) * nb / 2pi), clamped; later stages widen every
// phi window by a margin far above atan2f's error, and the exact cut decides, so the binning
// never changes a result.
#include <cooperative_groups.h>

#include "pxr_dev.cuh"
#include "pxr_cuts.cuh"

namespace cg = cooperative_groups;

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

// Atomic increment of counter i of CTA q's shared memory (this CTA's own: a plain shared atomic).
__device__ __forceinline__ uint32_t cl_inc(cg::cluster_group &cl, uint32_t *s, uint32_t q,
                                           uint32_t r, uint32_t i)
{
    if (q == r) return atomicAdd(s + i, 1u);
    return atomicAdd(cl.map_shared_rank(s + i, q), 1u);
}

// Exclusive scan of counters distributed over the cluster: CTA r holds keys [r S, (r + 1) S) in
// its s_cnt (its n own keys).  Each CTA scans its slice, publishes the slice total, adds the
// totals of the slices before it and writes out[k] = base + its counter k.  Returns the grand
// total.  Ends with a cluster barrier: no CTA changes a counter (the scatter's increments)
// before every CTA has written its part of `out` and read all slice totals.
__device__ uint32_t cluster_exclusive_scan(cg::cluster_group &cl, uint32_t *s_cnt, uint32_t n,
                                           uint32_t *s_warp, uint32_t *s_tot, uint32_t *out,
                                           uint32_t base)
{
    const uint32_t r = cl.block_rank(), C = cl.num_blocks();
    const uint32_t t = block_exclusive_scan(s_cnt, n, s_warp);
    if (threadIdx.x == 0) *s_tot = t;
    cl.sync();
    uint32_t off = 0, total = 0;
    for (uint32_t q = 0; q < C; ++q) {
        const uint32_t v = *cl.map_shared_rank(s_tot, q);
        off += q < r ? v : 0u;
        total += v;
    }
    for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) {
        const uint32_t c = s_cnt[k] + off;
        s_cnt[k] = c;
        out[k] = base + c;
    }
    cl.sync();
    return total;
}

// One cluster of C CTAs per event (C = 1: one CTA).  The counters of every step are spread over
// the cluster's shared memories (key k in CTA k / S, S = ceil(keys / C)); hits are spread over
// all the cluster's threads and count, or take their position, by atomics on the owning CTA's
// shared memory.  1) (layer, phi bin) histogram, 2) scan (bucket starts), 3) scatter of the
// sorted hit records; then, when the batch carries a hit grid (the CA stage's lookup), 4) each
// grid layer's range of the free coordinate (binning) and of the fixed one (the r-z cone),
// gathered in CTA 0, 5) grid histogram, 6) scan, 7) scatter of the sorted positions and free
// coordinates by grid cell.  The counters of steps 1-3 are reused for steps 5-7.  Every CTA of
// a cluster takes the same events and passes the same cluster barriers.
__global__ void __launch_bounds__(1024) k_sort(DevBatch b, DevParams p)
{
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ uint32_t s_cnt[];
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_tot;
    __shared__ int s_lay[kMaxLayers][4];    // (CTA 0) free min, free max, fixed min, fixed max
    __shared__ float4 s_gl[kMaxLayers];     // per grid layer: free min, bins per unit, fixed range
    const uint32_t r = cl.block_rank(), C = cl.num_blocks();
    const uint32_t tid = r * blockDim.x + threadIdx.x, nthr = C * blockDim.x;
    const uint32_t nk = p.n_keys, S = (nk + C - 1) / C;
    const uint32_t k0 = min(nk, r * S), kn = min(nk, k0 + S) - k0;
    const bool grid = b.gpos != nullptr;
    const uint32_t gk = grid ? p.n_glayers * p.gphi * p.gz : 0u, GS = (gk + C - 1) / C;
    const uint32_t g0 = min(gk, r * GS), gn = min(gk, g0 + GS) - g0;
    int *lay0 = cl.map_shared_rank(&s_lay[0][0], 0);
    for (uint32_t e = blockIdx.x / C; e < b.E; e += gridDim.x / C) {
        const uint32_t h0 = b.hit_off[e], n = b.hit_off[e + 1] - h0;
        for (uint32_t k = threadIdx.x; k < kn; k += blockDim.x) s_cnt[k] = 0;
        if (r == 0 && threadIdx.x < kMaxLayers * 4) {
            const uint32_t l = threadIdx.x >> 2, q = threadIdx.x & 3u;
            s_lay[l][q] = (q & 1u) ? ford_s(-3.0e38f) : ford_s(3.0e38f);
        }
        cl.sync();
        bool bad = false;
        for (uint32_t h = tid; h < n; h += nthr) {
            const uint32_t g = h0 + h;
            const uint32_t L = b.layer[g];
            if (L >= p.n_layers) { bad = true; continue; }
            const uint32_t key = L * p.nb + phi_bin(atan2f(b.y[g], b.x[g]), p), q = key / S;
            cl_inc(cl, s_cnt, q, r, key - q * S);
        }
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&b.cnt[C_FLAGS * b.E + e], F_LAYER);
        cl.sync();
        uint32_t *bk = b.bkt + (size_t)e * (nk + 1);
        const uint32_t total = cluster_exclusive_scan(cl, s_cnt, kn, s_warp, &s_tot, bk + k0, h0);
        if (tid == 0) bk[nk] = h0 + total;
        // positions past the valid hits (inputs with a bad layer) get layer 0xFF in their record
        for (uint32_t h = total + tid; h < n; h += nthr) b.hmeta[h0 + h] = 0xFFFFFFFFu;
        for (uint32_t h = tid; h < n; h += nthr) {
            const uint32_t g = h0 + h;
            const uint32_t L = b.layer[g];
            if (L >= p.n_layers) continue;
            const float x = b.x[g], y = b.y[g], z = b.z[g];
            const float phi = atan2f(y, x);
            const uint32_t key = L * p.nb + phi_bin(phi, p), q = key / S;
            const uint32_t pos = h0 + cl_inc(cl, s_cnt, q, r, key - q * S);
            const double r = radius64((double)x, (double)y);
            b.hs[pos] = make_float4(x, y, z, __double2float_rn(r));
            b.r64[pos] = r;
            b.hmeta[pos] = (L << kLocalBits) | h;
            b.hphi[pos] = phi;
        }
        cl.sync();                 // records and bucket starts written, counters free again
        if (!grid) continue;
        // ---- hit grid (the grid layers' hits, each layer contiguous in the sorted order) ----
        for (uint32_t L = 0; L < p.n_layers; ++L) {
            if (p.glidx[L] == 0xFF) continue;
            const bool disk = p.is_disk[L];
            int m0 = ford_s(3.0e38f), m1 = ford_s(-3.0e38f), m2 = m0, m3 = m1;
            for (uint32_t t = bk[L * p.nb] + tid; t < bk[(L + 1) * p.nb]; t += nthr) {
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
                atomicMin(lay0 + 4 * L + 0, m0);
                atomicMax(lay0 + 4 * L + 1, m1);
                atomicMin(lay0 + 4 * L + 2, m2);
                atomicMax(lay0 + 4 * L + 3, m3);
            }
        }
        for (uint32_t k = threadIdx.x; k < gn; k += blockDim.x) s_cnt[k] = 0;
        cl.sync();
        float4 *gl = b.glay + (size_t)e * p.n_glayers;
        if (threadIdx.x < p.n_layers && p.glidx[threadIdx.x] != 0xFF) {
            const uint32_t l = threadIdx.x;
            const float f0 = funord_s(lay0[4 * l + 0]), f1 = funord_s(lay0[4 * l + 1]);
            const float scale = f1 > f0 ? (float)p.gz / (f1 - f0) : 0.f;
            const float4 v = make_float4(f0, scale, funord_s(lay0[4 * l + 2]),
                                         funord_s(lay0[4 * l + 3]));
            s_gl[p.glidx[l]] = v;
            if (r == 0) gl[p.glidx[l]] = v;
        }
        __syncthreads();
        // the grid layers' hits, layer by layer (positions [bk[L nb], bk[(L + 1) nb]))
        auto for_grid_hits = [&](auto &&fn) {
            for (uint32_t L = 0; L < p.n_layers; ++L) {
                const uint32_t g = p.glidx[L];
                if (g == 0xFF) continue;
                const float4 glg = s_gl[g];
                for (uint32_t t = bk[L * p.nb] + tid; t < bk[(L + 1) * p.nb]; t += nthr) {
                    const float4 h = b.hs[t];
                    const float f = p.is_disk[L] ? h.w : h.z;
                    const uint32_t key = grid_key(g, phi_bin(b.hphi[t], p), f, glg, p);
                    const uint32_t q = key / GS;
                    fn(t, f, q, key - q * GS);
                }
            }
        };
        for_grid_hits([&](uint32_t, float, uint32_t q, uint32_t i) { cl_inc(cl, s_cnt, q, r, i); });
        cl.sync();
        uint32_t *go = b.gofs + (size_t)e * (gk + 1);
        const uint32_t gtotal = cluster_exclusive_scan(cl, s_cnt, gn, s_warp, &s_tot, go + g0, h0);
        if (tid == 0) go[gk] = h0 + gtotal;
        for_grid_hits([&](uint32_t t, float f, uint32_t q, uint32_t i) {
            const uint32_t pos = h0 + cl_inc(cl, s_cnt, q, r, i);
            b.gpos[pos] = t;
            b.gfree[pos] = f;
        });
        cl.sync();
    }
}

cudaError_t init_kernels()
{
    // up to 16 layers x 2048 bins of 4-byte counters (the hit grid's counters are fewer)
    cudaError_t e = cudaFuncSetAttribute(k_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kMaxLayers * 2048 * (int)sizeof(uint32_t));
    if (e != cudaSuccess) return e;
    if ((e = init_graph_kernels()) != cudaSuccess) return e;
    return init_fit_kernels();
}

// Cluster size: about PXR_SORT_HITS hits per CTA on the batch's mean event, a power of two up to
// 8 (the portable cluster size limit).
#ifndef PXR_SORT_HITS
#define PXR_SORT_HITS 4096
#endif
static uint32_t sort_cluster(const DevBatch &b)
{
    const uint64_t mean = b.E ? (uint64_t)b.N / b.E : 0;
    uint32_t C = 1;
    while (C < 8 && (uint64_t)C * PXR_SORT_HITS < mean) C <<= 1;
    return C;
}

void launch_sort(const DevBatch &b, const DevParams &p, cudaStream_t s, int sms)
{
    const uint32_t C = sort_cluster(b);
    const uint64_t cap = (uint64_t)sms * p.grid_per_sm[0] / C;    // clusters
    const uint64_t clusters = b.E < cap ? b.E : (cap ? cap : 1);
    if (b.E == 0) return;
    const uint32_t gk = b.gpos ? p.n_glayers * p.gphi * p.gz : 0u;
    const uint32_t keys = p.n_keys > gk ? p.n_keys : gk;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(clusters * C));
    cfg.blockDim = dim3(p.block_threads[0]);
    cfg.dynamicSmemBytes = (size_t)((keys + C - 1) / C) * sizeof(uint32_t);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_sort, b, p);
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
