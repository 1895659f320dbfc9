// Doublets, CA cell connection, ntuplet walk and ntuplet selection.
//
// Doublets: one warp per (inner hit, layer pair).  The outer layer's phi window is one or two
// contiguous runs of the sorted hits; the item reserves one entry per candidate with one atomic,
// the 32 lanes test 32 consecutive candidates per step (coalesced float4 loads) and write the
// outer hit, or kNone where the cut fails, to the candidate's entry.  The entries of an inner
// hit are contiguous (the CA stage reads them as one run per pair) and the cell (i, o) is found
// from o's position in i's window without a search.
//
// CA connect: one warp per junction hit j.  j's out-cells (j, k) are staged in shared memory and
// counting-sorted by the free coordinate of k (z on barrel layers, r on disks); each in-cell
// (i, j), one per lane, tests only the bins reached by the cone of r-z directions within
// asin(theta_cut) of its own, a conservative window in which the exact cuts decide.  Lanes with
// passes compute their cell's index from j's rank in i's window and append their edge lists
// through one atomic per warp.  Ntuplets: one warp per root hit walks the out-edges of its
// cells depth first.  Selection removes suffix paths and assigns output slots.
#include <cooperative_groups.h>

#include "pxr_dev.cuh"
#include "pxr_cuts.cuh"

namespace cg = cooperative_groups;

namespace pxr {

constexpr float kPiF2 = 3.14159265358979f;
constexpr int kMaxIt = 8;   // ballot masks kept per (hit, pair): 256 candidates

struct Window {
    uint32_t r0, n1, r2, n2;
    __device__ __forceinline__ uint32_t pos(uint32_t c) const { return c < n1 ? r0 + c : r2 + (c - n1); }
    __device__ __forceinline__ uint32_t size() const { return n1 + n2; }
};

// Candidates of layer Lo for an inner hit at azimuth phi: bins floor((phi -+ w_eps + pi) * nb/2pi)
// taken modulo nb (one or two runs of the sorted hits).
__device__ __forceinline__ Window phi_window(const uint32_t *__restrict__ bk, uint32_t Lo,
                                             float phi, const DevParams &p)
{
    const uint32_t *lb = bk + Lo * p.nb;
    int nb = (int)p.nb;
    Window w;
    if (!(fabsf(phi) <= 4.f)) {                // a non-finite azimuth has no window
        w.r0 = w.n1 = w.r2 = w.n2 = 0;
        return w;
    }
    int blo = (int)floorf((phi - p.w_eps + kPiF2) * p.bins_per_rad);
    int bhi = (int)floorf((phi + p.w_eps + kPiF2) * p.bins_per_rad);
    if (bhi - blo + 1 >= nb) {
        w.r0 = lb[0]; w.n1 = lb[nb] - lb[0]; w.r2 = 0; w.n2 = 0;
    } else if (blo < 0) {
        w.r0 = lb[blo + nb]; w.n1 = lb[nb] - w.r0; w.r2 = lb[0]; w.n2 = lb[bhi + 1] - w.r2;
    } else if (bhi >= nb) {
        w.r0 = lb[blo]; w.n1 = lb[nb] - w.r0; w.r2 = lb[0]; w.n2 = lb[bhi - nb + 1] - w.r2;
    } else {
        w.r0 = lb[blo]; w.n1 = lb[bhi + 1] - w.r0; w.r2 = 0; w.n2 = 0;
    }
    return w;
}

// FP64 decision of the doublet cut (every call in FP64 mode, the guard band in FP32 mode), kept
// out of line so that its double-precision registers do not weigh on the callers' hot loops.
__device__ __noinline__ bool doublet_exact(const double *r64, uint32_t g, uint32_t o, float xi,
                                           float yi, float xo, float yo, double cw)
{
    return doublet64((double)xi, (double)yi, r64[g], (double)xo, (double)yo, r64[o], cw);
}

// The kernels are instantiated per cut mode.  F64 (FP64-cut mode): a candidate is accepted or
// rejected by the FP64 formula, inline, except when the FP32 evaluation rejects it outside its
// rigorous error band (the FP64 formula rejects it too; most candidates end there).  Otherwise
// FP32 decides outside the band and the out-of-line FP64 formula inside it.
template <bool F64>
__device__ __forceinline__ bool doublet_test(const DevBatch &b, const DevParams &p, uint32_t g,
                                             float4 hi, uint32_t o, float4 ho)
{
    if constexpr (F64) {
        if (doublet32(hi, ho, p.cw32) == 0) return false;
        return doublet64((double)hi.x, (double)hi.y, b.r64[g], (double)ho.x, (double)ho.y,
                         b.r64[o], p.cw);
    } else {
        const int r = doublet32(hi, ho, p.cw32);
        if (r >= 0) return r == 1;
        return doublet_exact(b.r64, g, o, hi.x, hi.y, ho.x, ho.y, p.cw);
    }
}

// Compact form (allocation-free entry point): passing pairs only, counted first, then written
// from the ballot masks, so the cells of an inner hit are contiguous.
template <bool F64>
__global__ void __launch_bounds__(256) k_doublets_compact(DevBatch b, DevParams p, uint32_t slots)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const uint64_t n_items = (uint64_t)b.N * slots;
    const uint32_t nk = p.n_keys;
    uint64_t item = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t stride = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (; item < n_items; item += stride) {
        const uint32_t g = (uint32_t)(item / slots), slot = (uint32_t)(item % slots);
        // independent loads first (hits past an event's valid range carry layer 0xFF)
        const uint32_t meta = b.hmeta[g];
        const float4 hi = b.hs[g];
        const float phig = b.hphi[g];
        const uint32_t e = hit_event(b, g);
        const uint32_t L = meta >> kLocalBits;
        if (L >= p.n_layers || slot >= p.n_out[L]) continue;
        const uint32_t *bk = b.bkt + (size_t)e * (nk + 1);
        const uint32_t c_lo = b.cell_off[e], c_hi = b.cell_off[e + 1];
        const uint32_t Lo = p.out_layer[L][slot];
        const Window w = phi_window(bk, Lo, phig, p);
        const uint32_t nc = w.size();

        uint32_t masks[kMaxIt];
        uint32_t count = 0;
#pragma unroll
        for (int k = 0; k < kMaxIt; ++k) {
            masks[k] = 0;
            if ((uint32_t)k * 32u < nc) {
                uint32_t c = (uint32_t)k * 32u + lane;
                bool pass = false;
                if (c < nc) { const uint32_t o = w.pos(c); pass = doublet_test<F64>(b, p, g, hi, o, b.hs[o]); }
                masks[k] = __ballot_sync(0xFFFFFFFFu, pass);
                count += __popc(masks[k]);
            }
        }
        for (uint32_t c0 = kMaxIt * 32u; c0 < nc; c0 += 32u) {
            uint32_t c = c0 + lane;
            bool pass = false;
            if (c < nc) { const uint32_t o = w.pos(c); pass = doublet_test<F64>(b, p, g, hi, o, b.hs[o]); }
            count += __popc(__ballot_sync(0xFFFFFFFFu, pass));
        }

        uint32_t base = 0;
        if (lane == 0 && count) base = atomicAdd(&b.cnt[C_CELLS * b.E + e], count);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        const uint32_t cap = c_hi - c_lo;
        uint32_t nw = count;
        if (base >= cap) nw = 0;
        else if (base + count > cap) nw = cap - base;
        if (lane == 0) {
            if (nw < count) atomicOr(&b.cnt[C_FLAGS * b.E + e], F_CELLS);
            b.item[(size_t)g * kMaxOut + slot] = make_uint4(c_lo + base, nw, 0u, 0u);
        }
        if (nw == 0) continue;
        const uint32_t first = c_lo + base;
        uint32_t run = 0;
#pragma unroll
        for (int k = 0; k < kMaxIt; ++k) {
            uint32_t m = masks[k];
            if ((m >> lane) & 1u) {
                uint32_t idx = run + __popc(m & lt_mask);
                if (idx < nw) {
                    uint32_t o = w.pos((uint32_t)k * 32u + lane);
                    b.cell_in[first + idx] = g;
                    b.cell_out[first + idx] = o;
                }
            }
            run += __popc(m);
        }
        for (uint32_t c0 = kMaxIt * 32u; c0 < nc; c0 += 32u) {
            uint32_t c = c0 + lane;
            uint32_t o = c < nc ? w.pos(c) : 0u;
            bool pass = c < nc && doublet_test<F64>(b, p, g, hi, o, b.hs[o]);
            uint32_t m = __ballot_sync(0xFFFFFFFFu, pass);
            if (pass) {
                uint32_t idx = run + __popc(m & lt_mask);
                if (idx < nw) {
                    b.cell_in[first + idx] = g;
                    b.cell_out[first + idx] = o;
                }
            }
            run += __popc(m);
        }
    }
}

// Plan form: one warp per block of 32 consecutive items (inner hit, layer pair), one lane per
// item.  The lanes find their items' windows together (one round of dependent loads for 32
// items); the warp reserves one entry per candidate for all its items with one atomic per event
// present (usually one).  The items are then taken one at a time, their data broadcast from the
// owning lane: the lanes test 32 consecutive candidates per step (coalesced float4 loads) and
// write the outer hit, or kNone where the cut fails, to the candidate's entry.

template <bool F64>
__global__ void __launch_bounds__(256) k_doublets(DevBatch b, DevParams p, uint32_t slots)
{
    const uint32_t FULL = 0xFFFFFFFFu;
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t n_items = (uint64_t)b.N * slots;
    const uint64_t n_blocks = (n_items + 31) / 32;
    const uint32_t nk = p.n_keys;
    const uint64_t stride = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t blk = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; blk < n_blocks;
         blk += stride) {
        // ---- one item per lane: its window on the outer layer ----
        const uint64_t item = blk * 32 + lane;
        uint32_t g = 0, slot = 0, e = 0, nc = 0, r0 = 0, n1 = 0, r2 = 0, c_lo = 0, cap = 0;
        float4 hi = make_float4(0.f, 0.f, 0.f, 0.f);
        bool valid = false;
        if (item < n_items) {
            g = (uint32_t)(item / slots);
            slot = (uint32_t)(item % slots);
            // independent loads first (hits past an event's valid range carry layer 0xFF)
            const uint32_t meta = b.hmeta[g];
            hi = b.hs[g];
            const float phig = b.hphi[g];
            e = hit_event(b, g);
            const uint32_t L = meta >> kLocalBits;
            valid = L < p.n_layers && slot < p.n_out[L];
            if (valid) {
                c_lo = b.cell_off[e];
                cap = b.cell_off[e + 1] - c_lo;
                const Window w = phi_window(b.bkt + (size_t)e * (nk + 1), p.out_layer[L][slot],
                                            phig, p);
                r0 = w.r0;
                n1 = w.n1;
                r2 = w.r2;
                nc = w.size();
            }
        }
        // ---- reservation: one atomic per event among the lanes ----
        uint32_t excl = nc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, excl, o);
            if (lane >= (uint32_t)o) excl += t;
        }
        const uint32_t total = __shfl_sync(FULL, excl, 31);
        excl -= nc;
        uint32_t base = 0;
        for (uint32_t rem = __ballot_sync(FULL, nc > 0); rem;) {
            const int h = __ffs(rem) - 1;
            const uint32_t eh = __shfl_sync(FULL, e, h);
            const uint32_t seg = __ballot_sync(FULL, nc > 0 && e == eh);
            const uint32_t v = (seg >> lane) & 1u ? nc : 0u;
            uint32_t sc = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(FULL, sc, o);
                if (lane >= (uint32_t)o) sc += t;
            }
            const uint32_t stot = __shfl_sync(FULL, sc, 31);
            uint32_t sb = 0;
            if (lane == (uint32_t)h) sb = atomicAdd(&b.cnt[C_SLOTS * b.E + eh], stot);
            sb = __shfl_sync(FULL, sb, h);
            if ((seg >> lane) & 1u) base = sb + sc - v;
            rem &= ~seg;
        }
        const uint32_t nw = base >= cap ? 0u : min(nc, cap - base);
        const uint32_t first = c_lo + base;
        if (valid) {
            if (nw < nc) atomicOr(&b.cnt[C_FLAGS * b.E + e], F_CELLS);
            const size_t oi = (size_t)g * kMaxOut + slot;
            b.item[oi] = make_uint4(first, nw, r0, n1 - r2);
        }
        // ---- candidates, item by item (the item's data broadcast once), 32 per step ----
        const uint32_t has = __ballot_sync(FULL, nw > 0);
        const uint32_t e_main = __shfl_sync(FULL, e, has ? __ffs(has) - 1 : 0);
        uint32_t npass = 0;                       // this lane's passes of the event e_main
        for (uint32_t m = has; m; m &= m - 1) {
            const int k = __ffs(m) - 1;
            const uint32_t gk = __shfl_sync(FULL, g, k);
            const float4 hk = make_float4(__shfl_sync(FULL, hi.x, k), __shfl_sync(FULL, hi.y, k),
                                          0.f, __shfl_sync(FULL, hi.w, k));
            const uint32_t a0 = __shfl_sync(FULL, r0, k), a1 = __shfl_sync(FULL, n1, k);
            const uint32_t a2 = __shfl_sync(FULL, r2, k);
            const uint32_t fk = __shfl_sync(FULL, first, k), wk = __shfl_sync(FULL, nw, k);
            const uint32_t ek = __shfl_sync(FULL, e, k);
            uint32_t np = 0;
            for (uint32_t c = lane; c < wk; c += 32) {
                const uint32_t o = c < a1 ? a0 + c : a2 + (c - a1);
                const bool pass = doublet_test<F64>(b, p, gk, hk, o, __ldg(&b.hs[o]));
                b.cell_out[fk + c] = pass ? o : kNone;
                np += pass;
            }
            if (ek == e_main) npass += np;
            else if (np) atomicAdd(&b.cnt[C_CELLS * b.E + ek], np);   // block spans two events
        }
        npass = __reduce_add_sync(FULL, npass);
        if (lane == 0 && npass) atomicAdd(&b.cnt[C_CELLS * b.E + e_main], npass);
    }
}

void launch_doublets(const DevBatch &b, const DevParams &p, cudaStream_t s, int sms)
{
    uint32_t slots = 1;
    for (uint32_t l = 0; l < p.n_layers; ++l) slots = p.n_out[l] > slots ? p.n_out[l] : slots;
    const uint64_t warps = ((uint64_t)b.N * slots + 31) / 32;     // one warp per 32 items
    const uint32_t tpb = p.block_threads[1];
    uint64_t blocks = (warps + tpb / 32 - 1) / (tpb / 32);
    const uint64_t cap = (uint64_t)sms * p.grid_per_sm[1];
    if (blocks > cap) blocks = cap;
    if (blocks == 0) return;
    if (p.cut_mode == CUT_FP64)
        k_doublets<true><<<(unsigned)blocks, tpb, 0, s>>>(b, p, slots);
    else
        k_doublets<false><<<(unsigned)blocks, tpb, 0, s>>>(b, p, slots);
}

void launch_doublets_compact(const DevBatch &b, const DevParams &p, cudaStream_t s, int sms)
{
    uint32_t slots = 1;
    for (uint32_t l = 0; l < p.n_layers; ++l) slots = p.n_out[l] > slots ? p.n_out[l] : slots;
    uint64_t warps = (uint64_t)b.N * slots;
    uint64_t blocks = (warps + 7) / 8;
    uint64_t cap = (uint64_t)sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) return;
    if (p.cut_mode == CUT_FP64)
        k_doublets_compact<true><<<(unsigned)blocks, 256, 0, s>>>(b, p, slots);
    else
        k_doublets_compact<false><<<(unsigned)blocks, 256, 0, s>>>(b, p, slots);
}

// ------------------------------------------------------------------------------------------
// CA connect
// ------------------------------------------------------------------------------------------
// FP64 part of the triplet cut, out of line (see doublet_exact): the r-z alignment in FP64 when
// need_theta, then the DCA, decided by the FP32 result dc (1 pass, 0 fail) or else in FP64.
__device__ __noinline__ bool triplet_exact(const double *r64, const uint32_t *cell_out,
                                           const float4 *hs, uint32_t i, uint32_t j, uint32_t B,
                                           uint32_t k, float xi, float yi, float4 hj, float4 hk,
                                           bool need_theta, int dc, double theta, double dca)
{
    if (need_theta) {
        if (k == kNone) k = cell_out[B];
        const double zi = (double)hs[i].z, zj = (double)hj.z, zk = (double)hk.z;
        const double ri = r64[i], rj = r64[j], rk = r64[k];
        const double nA = seglen64(ri, zi, rj, zj);
        const double nB = seglen64(rj, zj, rk, zk);
        if (!theta64(ri, zi, rj, zj, rk, zk, nA, nB, theta)) return false;
    }
    if (dc >= 0) return dc == 1;
    return dca64((double)xi, (double)yi, (double)hj.x, (double)hj.y, (double)hk.x,
                 (double)hk.y) <= dca;
}

// Warp-aggregated count of the calling lanes into *c.
__device__ __forceinline__ void count_lanes(unsigned long long *c)
{
    const uint32_t m = __activemask();
    if ((threadIdx.x & 31u) == (uint32_t)(__ffs(m) - 1)) atomicAdd(c, (unsigned long long)__popc(m));
}

// Exact decision for the triplet (i, j, k), k the outer hit of the out-cell B = (j, k) (kNone:
// read from B's entry): r-z alignment, then DCA.  FP32 mode decides in float when outside the
// guard bands and takes the FP64 formulas otherwise (FP64 mode always).
template <bool F64>
__device__ __forceinline__ bool triplet_test(const DevBatch &b, const DevParams &p, uint32_t i,
                                             uint32_t j, uint32_t B, uint32_t k, float xi,
                                             float yi, float4 hj, float4 hk, const RZ32 &a)
{
    if (b.ca_tests) count_lanes(b.ca_tests);
    if constexpr (F64) {
        if (theta32(a, rz32(hj, hk), p.theta32) == 0) return false;
        if (k == kNone) k = b.cell_out[B];
        const double zi = (double)b.hs[i].z, zj = (double)hj.z, zk = (double)hk.z;
        const double ri = b.r64[i], rj = b.r64[j], rk = b.r64[k];
        if (!theta64(ri, zi, rj, zj, rk, zk, seglen64(ri, zi, rj, zj), seglen64(rj, zj, rk, zk),
                     p.theta))
            return false;
        if (b.ca_tests) count_lanes(b.ca_tests + 1);
        if (dca32(xi, yi, hj.x, hj.y, hk.x, hk.y, p.dca32) == 0) return false;
        return dca64((double)xi, (double)yi, (double)hj.x, (double)hj.y, (double)hk.x,
                     (double)hk.y) <= p.dca;
    } else {
        const int th = theta32(a, rz32(hj, hk), p.theta32);
        if (th == 0) return false;
        if (b.ca_tests) count_lanes(b.ca_tests + 1);
        const int dc = dca32(xi, yi, hj.x, hj.y, hk.x, hk.y, p.dca32);
        if (th == 1 && dc >= 0) return dc == 1;
        return triplet_exact(b.r64, b.cell_out, b.hs, i, j, B, k, xi, yi, hj, hk, th < 0, dc,
                             p.theta, p.dca);
    }
}

// Conservative interval of the free coordinate (z on a barrel layer, r on a disk) reachable from
// hit j along r-z directions within asin(theta_cut) of a = (ar, az), modulo pi.  With m the slope
// of a against the layer's fixed coordinate and T = tan(asin(theta_cut)), the allowed slopes are
// [(m - T)/(1 + mT), (m + T)/(1 - mT)] unless the cone contains the direction along the layer
// (then everything is reachable); the offsets along the fixed coordinate span [dlo, dhi].
// Returns false when the whole free range must be scanned.
__device__ __forceinline__ bool cone_window(float ar, float az, float base, float dlo, float dhi,
                                            bool disk, float T, float &lo, float &hi)
{
    const float u = disk ? az : ar, v = disk ? ar : az;
    dlo -= 1e-4f + 1e-5f * fabsf(dlo);
    dhi += 1e-4f + 1e-5f * fabsf(dhi);
    if (!(fabsf(u) > 1e-20f) || !(T < 1e30f)) return false;
    // approximate divisions: their ~2 ulp errors are far inside the margin below
    const float m = __fdividef(v, u);
    const float den_hi = 1.f - m * T, den_lo = 1.f + m * T;
    if (!(den_hi > 1e-4f) || !(den_lo > 1e-4f)) return false;
    const float s_hi = __fdividef(m + T, den_hi), s_lo = __fdividef(m - T, den_lo);
    const float c1 = dlo * s_lo, c2 = dlo * s_hi, c3 = dhi * s_lo, c4 = dhi * s_hi;
    lo = base + fminf(fminf(c1, c2), fminf(c3, c4));
    hi = base + fmaxf(fmaxf(c1, c2), fmaxf(c3, c4));
    const float smax = fmaxf(fabsf(s_lo), fabsf(s_hi));
    const float margin = 2e-3f + 1e-4f * (fabsf(lo) + fabsf(hi)) +
                         1e-5f * fmaxf(fabsf(dlo), fabsf(dhi)) * (1.f + smax * smax);
    lo -= margin;
    hi += margin;
    return true;
}

// The cone window of cone_window for the tile pass, with a division-free slope interval: the
// exact interval [(m - T)/(1 + mT), (m + T)/(1 - mT)] deviates from m by T(1 + m^2)/(1 -+ mT),
// and 1/(1 - x) <= 1 + 2|x| for |x| <= 1/2, so [m - d, m + d] with d = T(1 + m^2)(1 + 2|m|T)
// contains it (a wider cone only admits candidates the exact cut then rejects).  dlo, dhi come
// adjusted by the caller (the same widening cone_window applies), dmx = 1e-5 max(|dlo|, |dhi|).
// Returns false when the whole free range must be scanned (|mT| > 1/2 included).
__device__ __forceinline__ bool cone_tile(float ar, float az, float base, float dlo, float dhi,
                                          float dmx, bool disk, float T, float &lo, float &hi)
{
    const float u = disk ? az : ar, v = disk ? ar : az;
    if (!(fabsf(u) > 1e-20f)) return false;
    const float m = __fdividef(v, u);
    const float mt = fabsf(m) * T;
    if (!(mt <= 0.5f)) return false;
    const float d = T * __fmaf_rn(m, m, 1.f) * __fmaf_rn(2.f, mt, 1.f);
    const float sl = m - d, sh = m + d;
    const float c1 = dlo * sl, c2 = dlo * sh, c3 = dhi * sl, c4 = dhi * sh;
    lo = base + fminf(fminf(c1, c2), fminf(c3, c4));
    hi = base + fmaxf(fmaxf(c1, c2), fmaxf(c3, c4));
    const float smax = fabsf(m) + d;
    const float margin = 2e-3f + 1e-4f * (fabsf(lo) + fabsf(hi)) + dmx * __fmaf_rn(smax, smax, 1.f);
    lo -= margin;
    hi += margin;
    return true;
}

// Mark cell C as reached (it has an in-edge).  The first marker clears C's edge count (the walk
// reads it; a later level writes the count if C gets out-edges) and, when C is `listed` (a
// non-root cell whose outer hit starts further pairs), appends it to the event's frontier list,
// the input of the sparse pass of C's outer layer.
__device__ __forceinline__ void mark_reached(const DevBatch &b, uint32_t e, uint32_t C,
                                             uint32_t c_in, bool listed)
{
    const uint32_t bit = 1u << (C & 31u);
    if (!listed) {
        // nothing to append: the mark needs no answer, and clearing the count again is harmless
        // (C's own edges are written by a later launch)
        atomicOr(&b.live[C >> 5], bit);
        b.nbr_head[C].y = 0u;
        return;
    }
    if (atomicOr(&b.live[C >> 5], bit) & bit) return;
    b.nbr_head[C].y = 0u;
    const uint32_t cap = b.edge_off[e + 1] - b.edge_off[e];
    const uint32_t x = atomicAdd(&b.cnt[C_FRONT * b.E + e], 1u);
    if (x < cap) {
        b.front_list[b.edge_off[e] + x] = C;
        b.front_in[b.edge_off[e] + x] = c_in;
    } else {
        atomicOr(&b.cnt[C_FLAGS * b.E + e], F_EDGES);
    }
}

// The grid search of the out-cells (j, k) on layer Lk of the pair (item itj of hit j) that can
// continue the segment a (ending at j) of the cell (i, j): the hit grid's cells of j's phi
// window on Lk (whole coarse azimuth bins: j's fine-bin window as the doublet stage binned it)
// crossed with the bins of the r-z cone of directions within asin(theta_cut) of a, a
// conservative window.  Returns the number of grid ranges (one per coarse bin, at most kCaR:
// a window of at most 1 rad spans at most 7 bins of 2 pi / 32) with their starts and lengths in
// q0, qn, and the cone [lo, hi]; 0 when nothing can pass.
constexpr int kCaR = 8;

__device__ __forceinline__ uint32_t ca_ranges(const DevBatch &b, const DevParams &p, uint32_t e,
                                              uint32_t Lk, float4 hj, float phij, const RZ32 &a,
                                              uint4 itj, float &lo, float &hi,
                                              uint32_t (&q0)[kCaR], uint32_t (&qn)[kCaR])
{
    lo = -3.0e38f;
    hi = 3.0e38f;
    const uint32_t g = p.glidx[Lk];
    if (itj.y == 0 || g == 0xFF || !(fabsf(phij) <= 4.f)) return 0;   // (g: always a grid layer;
                                                                     //  phij: finite)
    const float4 gl = b.glay[(size_t)e * p.n_glayers + g];
    const bool disk = p.is_disk[Lk];
    const float jx = disk ? hj.z : hj.w;          // j's fixed coordinate relative to Lk's
    int z0 = 0, z1 = (int)p.gz - 1;
    if (cone_window(a.ar, a.az, disk ? hj.w : hj.z, gl.z - jx, gl.w - jx, disk, p.tan_win, lo,
                    hi)) {
        const float u0 = floorf((lo - gl.x) * gl.y), u1 = floorf((hi - gl.x) * gl.y);
        if (!(u1 >= 0.f) || !(u0 < (float)p.gz)) return 0;  // (also when either is not a number)
        z0 = u0 < 0.f ? 0 : (int)u0;
        z1 = u1 >= (float)p.gz ? (int)p.gz - 1 : (int)u1;
    }
    const int nb = (int)p.nb, gp = (int)p.gphi;
    const int blo = (int)floorf((phij - p.w_eps + kPiF2) * p.bins_per_rad);
    const int bhi = (int)floorf((phij + p.w_eps + kPiF2) * p.bins_per_rad);
    int c0, c1, c2 = 1, c3 = 0;                   // coarse runs [c0, c1] and [c2, c3]
    if (bhi - blo + 1 >= nb) {
        c0 = 0; c1 = gp - 1;
    } else if (blo < 0) {
        c0 = (blo + nb) * gp / nb; c1 = gp - 1;
        c2 = 0; c3 = bhi * gp / nb;
    } else if (bhi >= nb) {
        c0 = blo * gp / nb; c1 = gp - 1;
        c2 = 0; c3 = (bhi - nb) * gp / nb;
    } else {
        c0 = blo * gp / nb; c1 = bhi * gp / nb;
    }
    const uint32_t *go = b.gofs + (size_t)e * (p.n_glayers * p.gphi * p.gz + 1) +
                         (size_t)g * p.gphi * p.gz;
    uint32_t nr = 0;
    // (the bounds of all ranges are loaded together)
#pragma unroll
    for (int r = 0; r < kCaR; ++r) {
        const int n1 = c1 - c0 + 1;
        const int pc = r < n1 ? c0 + r : c2 + (r - n1);
        if (r < n1 || pc <= c3) {
            const uint32_t *gc = go + (size_t)pc * p.gz;
            q0[r] = gc[z0];
            qn[r] = gc[z1 + 1];
            nr = r + 1;
        } else {
            q0[r] = qn[r] = 0;
        }
    }
#pragma unroll
    for (int r = 0; r < kCaR; ++r) qn[r] -= q0[r];
    return nr;
}

constexpr int kEdgeBuf = 8;     // passes buffered per cell; a longer list is found again
#ifndef PXR_CA_MINB
#define PXR_CA_MINB 4           // CTAs per SM the sparse CA kernel is compiled for (registers)
#endif

// One warp's cells (one per lane), their queries and passes, in shared memory: the warp works
// through the grid candidates of all its lanes as one list, 32 at a time, so that a lane with
// many candidates does not hold up the others.
struct CaWarp {
    float4 hj[32], a[32];        // junction hit, segment into it (ar, az, |a|, error bound)
    float2 xy[32], cone[32];     // the segment's inner hit (x, y); the cone [lo, hi]
    uint4 itj[32];               // j's entries on the out-layer of the pair
    uint32_t i[32], j[32], fr[32];
    uint32_t pre[32];            // exclusive prefix of the lanes' candidates
    uint32_t q0[kCaR][32], qn[kCaR][32];
    uint32_t npass[32];
    uint32_t buf[kEdgeBuf][32];  // passes; bit 31: list the target in the frontier
};

// The exact triplet cut for a grid candidate, out of line: only candidates inside the cone get
// here, and its registers then do not weigh on the lookup loop.
template <bool F64>
__device__ __noinline__ bool ca_test(const DevBatch &b, const DevParams &p, uint32_t i, uint32_t j,
                                     uint32_t B, uint32_t k, float xi, float yi, float4 hj,
                                     float4 a4)
{
    const RZ32 a{a4.x, a4.y, a4.z, a4.w};
    return triplet_test<F64>(b, p, i, j, B, k, xi, yi, hj, b.hs[k], a);
}

// One pair (out-layer Lk of the lane's cell; lanes with active false take no part) for the
// warp's cells: each lane's grid ranges, then the flattened candidates, each checked against its
// owner's cone, j's window (the rank among j's entries) and the entry (which holds k unless the
// doublet cut failed); the exact triplet cut decides; passes go to the owner's buffer.
template <bool F64>
__device__ __forceinline__ void ca_warp_pair(const DevBatch &b, const DevParams &p, uint32_t e,
                                             CaWarp &W, uint32_t lane, bool active, uint32_t Lk,
                                             uint32_t i, uint32_t j, float xi, float yi,
                                             float4 hj, float phij, const RZ32 &a, uint4 itj,
                                             uint32_t fr)
{
    const uint32_t FULL = 0xFFFFFFFFu;
    uint32_t q0[kCaR], qn[kCaR];
    float lo = 0.f, hi = 0.f;
    uint32_t nr = 0, nc = 0;
    if (active) nr = ca_ranges(b, p, e, Lk, hj, phij, a, itj, lo, hi, q0, qn);
#pragma unroll
    for (int r = 0; r < kCaR; ++r) {
        if (r >= (int)nr) qn[r] = 0;
        nc += qn[r];
        W.q0[r][lane] = q0[r];
        W.qn[r][lane] = qn[r];
    }
    uint32_t incl = nc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, incl, o);
        if (lane >= (uint32_t)o) incl += t;
    }
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    if (total == 0) return;
    W.pre[lane] = incl - nc;
    W.hj[lane] = hj;
    W.a[lane] = make_float4(a.ar, a.az, a.na, a.Ea);
    W.xy[lane] = make_float2(xi, yi);
    W.cone[lane] = make_float2(lo, hi);
    W.itj[lane] = itj;
    W.i[lane] = i;
    W.j[lane] = j;
    W.fr[lane] = fr;
    __syncwarp();
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t f = base + lane;
        if (f < total) {
            uint32_t o = 0;                       // the last lane whose candidates start <= f
#pragma unroll
            for (uint32_t step = 16; step; step >>= 1)
                if (W.pre[o + step] <= f) o += step;
            uint32_t off = f - W.pre[o], r = 0;
            while (off >= W.qn[r][o]) off -= W.qn[r++][o];
            const uint32_t q = W.q0[r][o] + off;
            const float fz = b.gfree[q];
            const float2 cone = W.cone[o];
            if (fz >= cone.x && fz <= cone.y) {
                const uint32_t k = b.gpos[q];
                const uint4 it = W.itj[o];
                const uint32_t rank = k >= it.z ? k - it.z : k + it.w;
                if (rank < it.y) {
                    const uint32_t B = it.x + rank;
                    const float2 xy = W.xy[o];
                    if (b.cell_out[B] == k &&
                        ca_test<F64>(b, p, W.i[o], W.j[o], B, k, xy.x, xy.y, W.hj[o], W.a[o])) {
                        const uint32_t sl = atomicAdd(&W.npass[o], 1u);
                        if (sl < (uint32_t)kEdgeBuf) W.buf[sl][o] = B | W.fr[o];
                    }
                }
            }
        }
    }
    __syncwarp();
}

// Edge lists of one cell per lane (all lanes in event e): npass passes of the lane's cell A,
// buffered in W.buf when there are at most kEdgeBuf of them.  The warp's returning atomics are
// issued together: the edge reservation, the root-list reservation (a root cell with edges is
// listed), the frontier slots of the targets that start further pairs (taken before freshness
// is known: a slot of a target already reached holds kNone) and the targets' reached marks.
// Each lane writes its cell's list head and its buffered passes and clears the edge count of a
// target it reached first.  Returns the lane's list start (absolute) and sets nw to the entries
// that fit the region; a cell with more than kEdgeBuf passes is written by ca_rest.
__device__ __forceinline__ uint32_t ca_append(const DevBatch &b, uint32_t e, bool root,
                                              uint32_t A, uint32_t a_in, uint32_t a_out,
                                              uint32_t npass, const CaWarp &W, uint32_t lane,
                                              uint32_t &nw)
{
    const uint32_t FULL = 0xFFFFFFFFu;
    nw = 0;
    const uint32_t nbuf = npass <= (uint32_t)kEdgeBuf ? npass : 0u;
    uint32_t nf = 0;
    for (uint32_t t = 0; t < nbuf; ++t) nf += W.buf[t][lane] >> 31;
    uint32_t incl = npass, finc = nf;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, incl, o);
        const uint32_t u = __shfl_up_sync(FULL, finc, o);
        if (lane >= (uint32_t)o) { incl += t; finc += u; }
    }
    const uint32_t tot = __shfl_sync(FULL, incl, 31), ftot = __shfl_sync(FULL, finc, 31);
    if (tot == 0) return 0;
    const uint32_t rm = root ? __ballot_sync(FULL, npass > 0) : 0u;
    uint32_t base = 0, rbase = 0, fbase = 0;
    if (lane == 0) {
        base = atomicAdd(&b.cnt[C_EDGES * b.E + e], tot);
        if (rm) rbase = atomicAdd(&b.cnt[C_ROOTS * b.E + e], __popc(rm));
        if (ftot) fbase = atomicAdd(&b.cnt[C_FRONT * b.E + e], ftot);
    }
    uint32_t fresh = 0;                           // bit t: buffered target t reached first here
    for (uint32_t t = 0; t < nbuf; ++t) {
        const uint32_t B = W.buf[t][lane] & 0x7FFFFFFFu, bit = 1u << (B & 31u);
        if (!(atomicOr(&b.live[B >> 5], bit) & bit)) fresh |= 1u << t;
    }
    base = __shfl_sync(FULL, base, 0);
    rbase = __shfl_sync(FULL, rbase, 0) + __popc(rm & ((1u << lane) - 1u));
    fbase = __shfl_sync(FULL, fbase, 0) + finc - nf;
    if (npass == 0) return 0;
    const uint32_t g0 = b.edge_off[e], cap = b.edge_off[e + 1] - g0;
    const uint32_t my0 = base + incl - npass;
    nw = my0 >= cap ? 0u : min(npass, cap - my0);
    if (nw < npass) atomicOr(&b.cnt[C_FLAGS * b.E + e], F_EDGES);
    if (root) {
        if (rbase < cap) {
            b.root_list[g0 + rbase] = A;
            b.root_in[g0 + rbase] = a_in;
        } else {
            atomicOr(&b.cnt[C_FLAGS * b.E + e], F_EDGES);
        }
    }
    b.nbr_head[A] = make_uint2(g0 + my0, nw);
    for (uint32_t t = 0; t < nbuf; ++t) {
        const uint32_t Bf = W.buf[t][lane], B = Bf & 0x7FFFFFFFu;
        const bool fr_t = (fresh >> t) & 1u;
        if (t < nw) b.nbr[g0 + my0 + t] = B;
        if (fr_t) b.nbr_head[B].y = 0u;
        if (Bf >> 31) {
            if (fbase < cap) {
                b.front_list[g0 + fbase] = fr_t ? B : kNone;
                b.front_in[g0 + fbase] = a_out;
            } else {
                atomicOr(&b.cnt[C_FLAGS * b.E + e], F_EDGES);
            }
            ++fbase;
        }
    }
    return g0 + my0;
}

// Every pass of a cell with more than kEdgeBuf of them (rare), found again lane by lane in a
// fixed order and written, the targets marked reached.  The cell is the segment a from hit i
// (x, y = xi, yi) to its outer hit j (on layer Lj; hj, phij); its pairs start on Lj.
template <bool F64>
__device__ __noinline__ void ca_rest(const DevBatch &b, const DevParams &p, uint32_t e,
                                     uint32_t i, uint32_t j, uint32_t Lj, float xi, float yi,
                                     float4 hj, float phij, RZ32 a, uint32_t first, uint32_t nw)
{
    const bool j_root = (p.root_mask >> Lj) & 1u;
    uint32_t t = 0;
    for (uint32_t s = 0; s < p.n_out[Lj]; ++s) {
        const uint32_t Lk = p.out_layer[Lj][s];
        const bool fr = !j_root && p.n_out[Lk] > 0;
        const uint4 itj = b.item[(size_t)j * kMaxOut + s];
        uint32_t q0[kCaR], qn[kCaR];
        float lo, hi;
        const uint32_t nr = ca_ranges(b, p, e, Lk, hj, phij, a, itj, lo, hi, q0, qn);
        for (uint32_t r = 0; r < nr; ++r)
            for (uint32_t q = q0[r]; q < q0[r] + qn[r]; ++q) {
                const float fz = b.gfree[q];
                if (fz < lo || fz > hi) continue;
                const uint32_t k = b.gpos[q];
                const uint32_t rank = k >= itj.z ? k - itj.z : k + itj.w;
                if (rank >= itj.y) continue;
                const uint32_t B = itj.x + rank;
                if (b.cell_out[B] != k ||
                    !ca_test<F64>(b, p, i, j, B, k, xi, yi, hj,
                                  make_float4(a.ar, a.az, a.na, a.Ea)))
                    continue;
                if (t < nw) b.nbr[first + t] = B;
                mark_reached(b, e, B, j, fr);
                ++t;
            }
    }
}

constexpr int kStage = 256;     // out-cells of one junction staged per out-layer slot
#ifndef PXR_CONN_BINS
#define PXR_CONN_BINS 128
#endif
constexpr int kBins = PXR_CONN_BINS;   // local bins of the free coordinate (multiple of 32)

// Order-preserving int encoding of floats (for warp min / max reductions).
__device__ __forceinline__ int ford(float f)
{
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float funord(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF); }


// One junction hit j (on a layer of layer_mask, in event e), one warp.  For each out-layer
// slot, j's out-cells (j, k) are staged in shared memory (k's coordinates) and counting-sorted
// by the free coordinate of k (z on barrel layers, r on disks) into local bins over the staged
// range.  The in-cells (i, j) are found 32 at a time, one per lane, by scanning i over j's phi
// window on the inner layer with the doublet cut; each lane computes the cone of r-z directions
// that can pass the alignment cut, the bins it reaches (a conservative window: the exact cuts
// decide) and tests those out-cells itself (j's entries of failed candidates are skipped).  The
// in-cell's index is j's rank in i's window.  Lanes with passes append their edges: the round's
// returning atomics (edge and root-list reservations, frontier slots, reached marks) are issued
// together.  A slot with more than kStage entries is tested from global memory.  This is the
// dense pass's path for the junctions of a tile whose window unions exceed the tile's staging
// (k_connect_tiles); sH, sT and bin are the calling warp's staging arrays.
template <bool F64>
__device__ __noinline__ void connect_junction(const DevBatch &b, const DevParams &p, uint32_t e,
                                              uint32_t j, uint32_t layer_mask, float4 *sH,
                                              uint16_t *sT, uint32_t *bin)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nk = p.n_keys;
    {
        const uint32_t meta = b.hmeta[j];
        const float4 hj = b.hs[j];
        const float phij = b.hphi[j];
        const uint4 it0 = b.item[(size_t)j * kMaxOut];
        uint32_t f0 = it0.x, nB = it0.y;
        const uint32_t Lj = meta >> kLocalBits;
        if (Lj >= p.n_layers || !((layer_mask >> Lj) & 1u)) return;
        const uint32_t nin = p.n_in[Lj], nout = p.n_out[Lj];
        if (nin == 0 || nout == 0) return;
        const uint32_t *bk = b.bkt + (size_t)e * (nk + 1);
        const Window w0 = phi_window(bk, p.in_layer[Lj][0], phij, p);
        // out-cells that start further pairs from a non-root inner layer go to the frontier
        const bool j_root = (p.root_mask >> Lj) & 1u;
        for (uint32_t s = 0; s < nout; ++s) {
            const uint32_t Lk = p.out_layer[Lj][s];
            const bool disk = p.is_disk[Lk];
            if (s) {
                const uint4 its = b.item[(size_t)j * kMaxOut + s];
                f0 = its.x;
                nB = its.y;
            }
            if (nB == 0) continue;
            const bool staged = nB <= (uint32_t)kStage;
            // candidates of an in-cell are positions [q0, q1) of the bin-sorted passing entries
            // (staged) or of j's entries (not staged, failed candidates skipped); nq of them
            uint32_t nq = nB;
            float flo = 0.f, fhi = 0.f, dlo = 0.f, dhi = 0.f, scale = 0.f;
            if (staged) {
                int m0 = ford(3.0e38f), m1 = ford(-3.0e38f), m2 = m0, m3 = m1;
                auto take = [&](uint32_t t, uint32_t k, float4 hk) {
                    if (k == kNone) {                       // candidate that failed the cut
                        sH[t] = make_float4(__int_as_float(0x7FC00000), 0.f, 0.f, 0.f);
                        return;
                    }
                    const float fc = disk ? hk.w : hk.z, xc = disk ? hk.z : hk.w;
                    sH[t] = hk;
                    m0 = min(m0, ford(fc));
                    m1 = max(m1, ford(fc));
                    m2 = min(m2, ford(xc));
                    m3 = max(m3, ford(xc));
                };
                for (uint32_t t0 = 0; t0 < nB; t0 += 64) {      // two loads in flight per lane
                    const uint32_t ta = t0 + lane, tb = ta + 32u;
                    const uint32_t ka = ta < nB ? b.cell_out[f0 + ta] : 0u;
                    const uint32_t kb = tb < nB ? b.cell_out[f0 + tb] : 0u;
                    const float4 ha = ta < nB && ka != kNone ? b.hs[ka] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 hb = tb < nB && kb != kNone ? b.hs[kb] : make_float4(0.f, 0.f, 0.f, 0.f);
                    if (ta < nB) take(ta, ka, ha);
                    if (tb < nB) take(tb, kb, hb);
                }
                m0 = __reduce_min_sync(0xFFFFFFFFu, m0);
                m1 = __reduce_max_sync(0xFFFFFFFFu, m1);
                m2 = __reduce_min_sync(0xFFFFFFFFu, m2);
                m3 = __reduce_max_sync(0xFFFFFFFFu, m3);
                flo = funord(m0);
                fhi = funord(m1);
                dlo = funord(m2) - (disk ? hj.z : hj.w);
                dhi = funord(m3) - (disk ? hj.z : hj.w);
                scale = fhi > flo ? (float)kBins / (fhi - flo) : 0.f;
                // counting sort of the list positions by local bin: histogram, scan, scatter
#pragma unroll
                for (int q = 0; q < kBins / 32; ++q) bin[lane + 32 * q] = 0;
                __syncwarp();
                auto local_bin = [&](uint32_t t) {
                    const float4 hk = sH[t];
                    const int bb = (int)floorf(((disk ? hk.w : hk.z) - flo) * scale);
                    return bb < 0 ? 0u : (bb >= kBins ? (uint32_t)kBins - 1u : (uint32_t)bb);
                };
                // (entries of failed candidates carry x = NaN and are left out)
                for (uint32_t t = lane; t < nB; t += 32)
                    if (!isnan(sH[t].x)) atomicAdd(&bin[local_bin(t)], 1u);
                __syncwarp();
                {
                    constexpr int per = kBins / 32;      // consecutive bins per lane
                    uint32_t v[per], sum = 0;
#pragma unroll
                    for (int q = 0; q < per; ++q) { v[q] = bin[lane * per + q]; sum += v[q]; }
                    uint32_t incl = sum;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                        if (lane >= (uint32_t)o) incl += t;
                    }
                    uint32_t run = incl - sum;
                    __syncwarp();
#pragma unroll
                    for (int q = 0; q < per; ++q) { bin[lane * per + q] = run; run += v[q]; }
                    __syncwarp();
                }
                for (uint32_t t = lane; t < nB; t += 32)
                    if (!isnan(sH[t].x)) sT[atomicAdd(&bin[local_bin(t)], 1u)] = (uint16_t)t;
                __syncwarp();
                // bin[t] is now the end of bin t; the start of bin t is bin[t - 1] (0 for t = 0)
                nq = bin[kBins - 1];
            }
            const bool front = !j_root && p.n_out[Lk] > 0;
            for (uint32_t si = 0; si < nin; ++si) {
                const uint32_t Li = p.in_layer[Lj][si];
                const uint32_t slot_i = p.in_slot[Lj][si];
                // this pass takes the root in-cells; reached non-root ones go to the sparse pass
                if (!((p.root_mask >> Li) & 1u)) continue;
                const Window w = si ? phi_window(bk, Li, phij, p) : w0;
                const uint32_t nc = w.size();
                for (uint32_t c0 = 0; c0 < nc; c0 += 32) {
                    // ---- one in-cell candidate per lane ----
                    const uint32_t c = c0 + lane;
                    uint32_t i = 0, q0 = 0, q1 = 0;
                    float clo = -3.0e38f, chi = 3.0e38f;   // the cone (candidates outside skip)
                    uint4 itm = make_uint4(0u, 0u, 0u, 0u);
                    float4 hi = make_float4(0.f, 0.f, 0.f, 0.f);
                    RZ32 a{0.f, 0.f, 0.f, 0.f};
                    if (c < nc) {
                        i = w.pos(c);
                        hi = b.hs[i];
                        itm = b.item[(size_t)i * kMaxOut + slot_i];   // with hs[i]: one round trip
                        if (doublet_test<F64>(b, p, i, hi, j, hj)) {
                            a = rz32(hi, hj);
                            q1 = nq;
                            float lo, hi_;
                            if (staged && cone_window(a.ar, a.az, disk ? hj.w : hj.z, dlo, dhi,
                                                      disk, p.tan_win, lo, hi_)) {
                                if (hi_ < flo || lo > fhi) {
                                    q1 = 0;
                                } else {
                                    int b0 = (int)floorf((lo - flo) * scale);
                                    int b1 = (int)floorf((hi_ - flo) * scale);
                                    b0 = b0 < 0 ? 0 : (b0 >= kBins ? kBins - 1 : b0);
                                    b1 = b1 < 0 ? 0 : (b1 >= kBins ? kBins - 1 : b1);
                                    q0 = b0 ? bin[b0 - 1] : 0u;
                                    q1 = bin[b1];
                                    clo = lo;
                                    chi = hi_;
                                }
                            }
                        }
                    }
                    // ---- index of the in-cell (i, j): i's entry of rank(j) in its window ----
                    uint32_t A = kNone, kA = kNone;
                    if (q1 > q0) {
                        const uint32_t rank = j >= itm.z ? j - itm.z : j + itm.w;
                        if (rank < itm.y) {
                            A = itm.x + rank;
                            kA = b.cell_out[A];                 // checked after the tests
                        }
                    }
                    // ---- each lane tests its own candidates ----
                    uint32_t npass = 0, qf = 0, Bf = 0;
                    for (uint32_t q = q0; q < q1; ++q) {
                        uint32_t B;
                        float4 hk;
                        if (staged) {
                            const uint32_t t = sT[q];
                            B = f0 + t;
                            hk = sH[t];
                            const float fc = disk ? hk.w : hk.z;
                            if (fc < clo || fc > chi) continue;
                        } else {
                            B = f0 + q;
                            const uint32_t k = b.cell_out[B];
                            if (k == kNone) continue;
                            hk = b.hs[k];
                        }
                        if (triplet_test<F64>(b, p, i, j, B, kNone, hi.x, hi.y, hj, hk, a)) {
                            if (npass == 0) { qf = q; Bf = B; }
                            ++npass;
                        }
                    }
                    const uint32_t pm = __ballot_sync(0xFFFFFFFFu, npass > 0);
                    if (pm == 0) continue;
                    // the entry holds j unless the in-cell was dropped by a capacity overflow
                    // (rank beyond the written entries); any other mismatch is flagged
                    if (npass && A != kNone && kA != j) atomicOr(&b.cnt[C_FLAGS * b.E + e], F_CELLS);
                    if (kA != j) A = kNone;
                    // ---- append the edges: one atomic per warp reserves all lanes' lists ----
                    const bool ok = npass && A != kNone;   // kNone: the cell was dropped (overflow)
                    uint32_t have = 0, old = 0;
                    if (ok && s > 0) {
                        const uint2 hd = b.nbr_head[A];
                        have = hd.y;
                        old = hd.x;
                    }
                    const uint32_t need = ok ? have + npass : 0u;
                    uint32_t incl = need;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                        if (lane >= (uint32_t)o) incl += t;
                    }
                    const uint32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
                    // the round's returning atomics are issued together: the edge reservation, the
                    // root-list reservation (every in-cell of this pass is a root cell; it is listed
                    // with its first edges) and the reached mark of each lane's first pass (set
                    // before the capacity is known: under overflow, flagged, a marked cell may
                    // lack its edge, which only costs work)
                    const bool first_root = ok && have == 0;
                    const uint32_t rm = __ballot_sync(0xFFFFFFFFu, first_root);
                    const uint32_t fm = __ballot_sync(0xFFFFFFFFu, ok && front);
                    uint32_t base = 0, rbase = 0, fbase = 0, was = 0;
                    const uint32_t bit = 1u << (Bf & 31u);
                    if (lane == 0 && tot) base = atomicAdd(&b.cnt[C_EDGES * b.E + e], tot);
                    if (lane == 0 && rm) rbase = atomicAdd(&b.cnt[C_ROOTS * b.E + e], __popc(rm));
                    if (lane == 0 && fm) fbase = atomicAdd(&b.cnt[C_FRONT * b.E + e], __popc(fm));
                    if (ok) was = atomicOr(&b.live[Bf >> 5], bit);
                    const uint32_t lt = (1u << lane) - 1u;
                    base = __shfl_sync(0xFFFFFFFFu, base, 0);
                    rbase = __shfl_sync(0xFFFFFFFFu, rbase, 0) + __popc(rm & lt);
                    fbase = __shfl_sync(0xFFFFFFFFu, fbase, 0) + __popc(fm & lt);
                    const uint32_t cap = b.edge_off[e + 1] - b.edge_off[e];
                    const uint32_t my0 = base + incl - need;
                    const uint32_t nw = !ok || my0 >= cap ? 0u : min(need, cap - my0);
                    // a cell reached for the first time: its edge count cleared and, if its outer
                    // hit starts further pairs, the frontier entry (one reservation per warp)
                    const bool fresh = ok && !(was & bit);
                    if (fresh) b.nbr_head[Bf].y = 0u;
                    if (ok && front) {
                        if (fbase < cap) {
                            b.front_list[b.edge_off[e] + fbase] = fresh ? Bf : kNone;
                            b.front_in[b.edge_off[e] + fbase] = j;
                        } else {
                            atomicOr(&b.cnt[C_FLAGS * b.E + e], F_EDGES);
                        }
                    }
                    if (first_root) {
                        if (rbase < cap) {
                            b.root_list[b.edge_off[e] + rbase] = A;
                            b.root_in[b.edge_off[e] + rbase] = i;
                        } else {
                            atomicOr(&b.cnt[C_FLAGS * b.E + e], F_EDGES);
                        }
                    }
                    if (ok) {
                        if (nw < need) atomicOr(&b.cnt[C_FLAGS * b.E + e], F_EDGES);
                        const uint32_t first = b.edge_off[e] + my0;
                        uint32_t wr = 0;
                        for (uint32_t t = 0; t < have && wr < nw; ++t) b.nbr[first + wr++] = b.nbr[old + t];
                        if (wr < nw) b.nbr[first + wr++] = Bf;
                        for (uint32_t q = qf + 1; q < q1 && wr < nw && npass > 1; ++q) {
                            uint32_t B;
                            float4 hk;
                            if (staged) {
                                const uint32_t t = sT[q];
                                B = f0 + t;
                                hk = sH[t];
                                const float fc = disk ? hk.w : hk.z;
                                if (fc < clo || fc > chi) continue;
                            } else {
                                B = f0 + q;
                                const uint32_t k = b.cell_out[B];
                                if (k == kNone) continue;
                                hk = b.hs[k];
                            }
                            if (triplet_test<F64>(b, p, i, j, B, kNone, hi.x, hi.y, hj, hk, a)) {
                                b.nbr[first + wr++] = B;
                                mark_reached(b, e, B, j, front);
                            }
                        }
                        b.nbr_head[A] = make_uint2(first, wr);
                    }
                }
            }
            __syncwarp();
        }
    }
}


// ------------------------------------------------------------------------------------------
// Dense CA pass on junction tiles
// ------------------------------------------------------------------------------------------
// A tile is a run of up to 32 consecutive junction hits of one event and layer (in (layer, phi
// bin) order), one per lane of a warp.  Their phi windows on an inner (outer) layer overlap
// almost entirely, so the warp stages the union of the windows once, in shared memory, instead
// of once per junction.  The lanes then walk their junctions' inner windows in step: for the
// inner hit i of its step a lane computes the r-z cone of the segment (i, j) and looks up the
// staged outer hits inside it (counting-sorted by the free coordinate).  The few that fall
// inside the cone are queued, and the warp tests them 32 at a time with all lanes busy: a cell
// (j, k) (rank in j's window, entry holding the hit), the exact triplet cut, and the in-cell
// (i, j) itself, read from i's entry (the doublet stage decided it).  Passes are buffered in
// queue order, so the passes of one in-cell are adjacent, and appended together: one edge,
// root-list and frontier reservation per flush, each in-cell's edges a contiguous run.
constexpr uint32_t kTileJ = kCaTile;  // junction hits per tile (one per lane)
constexpr int kTileW = 4;             // warps per CTA
constexpr uint32_t kTileQ = 128;      // queued candidates per warp (a ring)
constexpr uint32_t kTileCand = 2;     // queued candidates per lane and step; more: lane alone
constexpr uint32_t kTilePass = 64;    // buffered passes per warp
constexpr uint32_t kTileAlone = 64;   // in-cells with many candidates, handled after the steps
#ifndef PXR_TILE_MINB
#define PXR_TILE_MINB 4               // CTAs per SM the tile kernel is compiled for (registers;
                                      //   its shared memory allows four)
#endif

constexpr uint32_t kZBins = 512;      // bins of the outer union's free coordinate

// The staged unions of the tile path: the inner hits' (z, r), the outer hits' free coordinate
// in staging order and in bin order with their staging indices, the bin ends (16 bits each, two
// per word; a union holds at most kStage hits).  The step loop reads nothing else.
struct TileStage {
    float2 hin[kStage];
    float zs[kStage];
    float zo[kStage];
    uint16_t sT[kStage];
    uint32_t zb[kZBins / 2];
};

// The staging of connect_junction (the tile's junctions one by one).
struct TileFallback {
    float4 sH[kStage];
    uint16_t sT[kStage];
    uint32_t bin[kBins];
};

struct TileWarp {
    union {
        TileStage t;
        TileFallback f;
    } u;
    float4 jh[32];                    // the junctions' hits
    uint4 jit[32];                    // their entries on the current out-layer
    uint32_t jpos[32];                // their sorted positions
    uint32_t q[kTileQ];               // candidates: junction lane << 16 | inner << 8 | outer
    uint32_t pA[kTilePass], pB[kTilePass], pI[kTilePass], pK[kTilePass];   // passes: in-cell,
                                      //   out-cell, inner hit, junction lane << 8 | inner index
    uint32_t pHave[kTilePass];        // a run's edges from an earlier out-layer (run start)
    uint32_t alone[kTileAlone];       // in-cells (junction lane << 8 | inner index) whose cone
                                      //   held more than kTileCand candidates
    float fix[2];                     // fixed-coordinate range of the staged outer hits
};

// End of bin x of the packed bin ends.
__device__ __forceinline__ uint32_t zbin_end(const uint32_t *zb, uint32_t x)
{
    return (zb[x >> 1] >> (16u * (x & 1u))) & 0xFFFFu;
}

constexpr int kTileSmem = kTileW * (int)sizeof(TileWarp);   // dynamic shared memory per CTA

// Hit positions of an event's layer taken as periodic in azimuth: the first hit of the
// unwrapped phi bin bb (in [-nb, 2 nb): bins below 0 and from nb on are the neighbouring turns)
// relative to the layer's first hit, tot hits per turn.
__device__ __forceinline__ int tile_v(const uint32_t *lb, int nb, int tot, int bb)
{
    if (bb < 0) return (int)(lb[bb + nb] - lb[0]) - tot;
    if (bb >= nb) return (int)(lb[bb - nb] - lb[0]) + tot;
    return (int)(lb[bb] - lb[0]);
}

// The union of the tile's windows on one layer (lb: the layer's bucket starts): staging index s
// is the hit at periodic position v0 + s; n hits (the whole layer, in natural order, when the
// union spans every bin).
struct TileSpan {
    int v0;
    uint32_t n, lb0, tot;
};

// Sorted position of staging index s.
__device__ __forceinline__ uint32_t tile_pos(const TileSpan &t, uint32_t s)
{
    int v = t.v0 + (int)s;
    if (v < 0) v += (int)t.tot;
    else if (v >= (int)t.tot) v -= (int)t.tot;
    return t.lb0 + (uint32_t)v;
}

// The union of the lanes' windows [blo, bhi] (unwrapped bins; ok false: the lane has none) and
// each lane's window as staging indices [ws, ws + wn) (modulo n when the union is the whole
// layer).  Warp-collective.
__device__ __forceinline__ TileSpan tile_span(const uint32_t *lb, int nb, bool ok, int blo,
                                              int bhi, uint32_t &ws, uint32_t &wn)
{
    TileSpan t;
    t.lb0 = lb[0];
    t.tot = lb[nb] - t.lb0;
    t.v0 = 0;
    t.n = 0;
    ws = wn = 0;
    const int ulo = __reduce_min_sync(0xFFFFFFFFu, ok ? blo : 0x7FFFFFFF);
    const int uhi = __reduce_max_sync(0xFFFFFFFFu, ok ? bhi : -0x7FFFFFFF);
    if (ulo > uhi || t.tot == 0) return t;
    const int tot = (int)t.tot;
    if (uhi - ulo + 1 >= nb) {
        t.n = t.tot;
        if (ok) {
            if (bhi - blo + 1 >= nb) {
                wn = t.tot;
            } else {
                int a = tile_v(lb, nb, tot, blo);
                wn = (uint32_t)(tile_v(lb, nb, tot, bhi + 1) - a);
                if (a < 0) a += tot;
                else if (a >= tot) a -= tot;
                ws = (uint32_t)a;
            }
        }
    } else {
        t.v0 = tile_v(lb, nb, tot, ulo);
        t.n = (uint32_t)(tile_v(lb, nb, tot, uhi + 1) - t.v0);
        if (ok) {
            const int a = tile_v(lb, nb, tot, blo);
            ws = (uint32_t)(a - t.v0);
            wn = (uint32_t)(tile_v(lb, nb, tot, bhi + 1) - a);
        }
    }
    return t;
}

// The out-cell B of j for the staged outer hit kt, and the triplet (i, j, k): kNone unless
// (j, k) is a cell (rank in j's window, entry holding k) and the exact triplet cut passes.
template <bool F64>
__device__ __forceinline__ uint32_t tile_test(const DevBatch &b, const DevParams &p, uint32_t ev,
                                              const TileSpan &tk, uint32_t kt, uint32_t i,
                                              float4 hi, uint32_t j, float4 hj, const RZ32 &a,
                                              uint4 itj)
{
    const uint32_t k = tile_pos(tk, kt);
    const uint32_t rank = k >= itj.z ? k - itj.z : k + itj.w;
    if (rank >= itj.y) return kNone;
    const uint32_t B = itj.x + rank;
    if (!PXR_IN(b, ev, B, b.C)) return kNone;
    const float4 hk = b.hs[k];
    if (!triplet_test<F64>(b, p, i, j, B, k, hi.x, hi.y, hj, hk, a)) return kNone;
    return b.cell_out[B] == k ? B : kNone;          // (j, k) failed the doublet cut: kNone
}

// The in-cell (i, j) for the pair slot slot_i of i: i's entry of rank(j) in its window, kNone
// when the doublet stage did not keep it.
__device__ __forceinline__ uint32_t tile_incell(const DevBatch &b, uint32_t ev, uint32_t i,
                                                uint32_t slot_i, uint32_t j)
{
    const uint4 iti = b.item[(size_t)i * kMaxOut + slot_i];
    const uint32_t rank = j >= iti.z ? j - iti.z : j + iti.w;
    if (rank >= iti.y) return kNone;
    const uint32_t A = iti.x + rank;
    if (!PXR_IN(b, ev, A, b.C)) return kNone;
    return b.cell_out[A] == j ? A : kNone;
}

// Every pass of one in-cell (i, j) written straight to global memory, for a lane whose cone
// held more than kTileCand candidates (rare): the candidates [q0, q1) of the bin order tested
// one by one.  more: an earlier out-layer of j may have given the in-cell edges already (copied
// first).
template <bool F64>
__device__ __noinline__ void tile_direct(const DevBatch &b, const DevParams &p, uint32_t e,
                                         const TileWarp &S, const TileSpan &tk, uint32_t q0,
                                         uint32_t q1, float lo, float hi_, bool disk,
                                         uint32_t slot_i, uint32_t i, float4 hi, uint32_t j,
                                         float4 hj, uint4 itj, bool more, bool front)
{
    const RZ32 a = rz32(hi, hj);
    uint32_t np = 0;
    for (uint32_t q = q0; q < q1; ++q) {
        const float fc = S.u.t.zo[q];
        if (fc >= lo && fc <= hi_ &&
            tile_test<F64>(b, p, e, tk, S.u.t.sT[q], i, hi, j, hj, a, itj) != kNone)
            ++np;
    }
    if (np == 0) return;
    const uint32_t A = tile_incell(b, e, i, slot_i, j);
    if (A == kNone) return;
    uint32_t have = 0, old = 0;
    if (more) {
        const uint2 hd = b.nbr_head[A];
        have = hd.y;
        old = hd.x;
    }
    const uint32_t need = have + np;
    const uint32_t g0 = b.edge_off[e], cap = b.edge_off[e + 1] - g0;
    const uint32_t my0 = atomicAdd(&b.cnt[C_EDGES * b.E + e], need);
    const uint32_t nw = my0 >= cap ? 0u : min(need, cap - my0);
    if (nw < need) atomicOr(&b.cnt[C_FLAGS * b.E + e], F_EDGES);
    if (have == 0) {
        const uint32_t r = atomicAdd(&b.cnt[C_ROOTS * b.E + e], 1u);
        if (r < cap) {
            b.root_list[g0 + r] = A;
            b.root_in[g0 + r] = i;
        } else {
            atomicOr(&b.cnt[C_FLAGS * b.E + e], F_EDGES);
        }
    }
    uint32_t wr = 0;
    for (uint32_t t = 0; t < have && wr < nw; ++t) b.nbr[g0 + my0 + wr++] = b.nbr[old + t];
    for (uint32_t q = q0; q < q1; ++q) {
        const float fc = S.u.t.zo[q];
        if (!(fc >= lo && fc <= hi_)) continue;
        const uint32_t B = tile_test<F64>(b, p, e, tk, S.u.t.sT[q], i, hi, j, hj, a, itj);
        if (B == kNone) continue;
        if (wr < nw) b.nbr[g0 + my0 + wr++] = B;
        mark_reached(b, e, B, j, front);
    }
    b.nbr_head[A] = make_uint2(g0 + my0, wr);
}

// One listed in-cell (key: junction lane << 8 | inner staging index) written by tile_direct:
// its cone recomputed from the staged hits (flo, fhi, scale: the outer union's free-coordinate
// range and bin scale).
template <bool F64>
__device__ __noinline__ void tile_alone(const DevBatch &b, const DevParams &p, uint32_t e,
                                        const TileWarp &S, TileSpan ti, TileSpan tk, uint32_t key,
                                        float flo, float fhi, float scale, bool disk,
                                        uint32_t slot_i, bool more, bool front)
{
    const uint32_t t = key >> 8, sx = key & 0xFFu;
    const float4 hi = b.hs[tile_pos(ti, sx)], hj = S.jh[t];
    const float jfix = disk ? hj.z : hj.w, jfree = disk ? hj.w : hj.z;
    float dlo = S.fix[0] - jfix, dhi = S.fix[1] - jfix;
    dlo -= 1e-4f + 1e-5f * fabsf(dlo);
    dhi += 1e-4f + 1e-5f * fabsf(dhi);
    const float dmx = 1e-5f * fmaxf(fabsf(dlo), fabsf(dhi));
    uint32_t q0 = 0, q1 = tk.n;
    float lo = -3.0e38f, hi_ = 3.0e38f;
    if (cone_tile(__fsub_rn(hj.w, hi.w), __fsub_rn(hj.z, hi.z), jfree, dlo, dhi, dmx, disk,
                  p.tan_win, lo, hi_)) {
        if (hi_ < flo || lo > fhi) return;
        int b0 = (int)floorf((lo - flo) * scale);
        int b1 = (int)floorf((hi_ - flo) * scale);
        b0 = b0 < 0 ? 0 : (b0 >= (int)kZBins ? (int)kZBins - 1 : b0);
        b1 = b1 < 0 ? 0 : (b1 >= (int)kZBins ? (int)kZBins - 1 : b1);
        q0 = b0 ? zbin_end(S.u.t.zb, b0 - 1) : 0u;
        q1 = zbin_end(S.u.t.zb, b1);
    }
    tile_direct<F64>(b, p, e, S, tk, q0, q1, lo, hi_, disk, slot_i, tile_pos(ti, sx), hi,
                     S.jpos[t], hj, S.jit[t], more, front);
}

// Append the first n buffered passes (runs of equal in-cell, each complete).  A run whose in-cell
// has no edges yet (every run when more is false) takes its place in one contiguous block of
// edges reserved for the flush and is listed as a root cell; a run whose in-cell got edges from
// an earlier out-layer is written by its first lane with the old edges copied in front.  Every
// pass marks its target reached and, when front, takes a frontier slot (taken before the target
// is known to be fresh: kNone if it is not).  Warp-collective.
__device__ __forceinline__ void tile_flush(const DevBatch &b, uint32_t e, TileWarp &S, uint32_t n,
                                           bool more, bool front, uint32_t lane)
{
    const uint32_t FULL = 0xFFFFFFFFu;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t g0 = b.edge_off[e], cap = b.edge_off[e + 1] - g0;
    __syncwarp();
    // run starts: the earlier edges of their in-cells; counts of the block and the new roots
    uint32_t nfast = 0, nroot = 0;
    for (uint32_t r0 = 0; r0 < n; r0 += 32) {
        const uint32_t x = r0 + lane;
        bool fast = false, root = false;
        if (x < n) {
            const uint32_t A = S.pA[x];
            const bool start = x == 0 || S.pA[x - 1] != A;
            uint32_t have = 0;
            if (start) {
                if (more) have = b.nbr_head[A].y;
                S.pHave[x] = have;
                root = have == 0;
            }
        }
        __syncwarp();
        if (x < n) {
            uint32_t s0 = x;
            while (s0 > 0 && S.pA[s0 - 1] == S.pA[x]) --s0;
            fast = S.pHave[s0] == 0;
        }
        nfast += __popc(__ballot_sync(FULL, fast));
        nroot += __popc(__ballot_sync(FULL, root));
    }
    uint32_t ebase = 0, rbase = 0, fbase = 0;
    if (lane == 0) {
        if (nfast) ebase = atomicAdd(&b.cnt[C_EDGES * b.E + e], nfast);
        if (nroot) rbase = atomicAdd(&b.cnt[C_ROOTS * b.E + e], nroot);
        if (front && n) fbase = atomicAdd(&b.cnt[C_FRONT * b.E + e], n);
    }
    ebase = __shfl_sync(FULL, ebase, 0);
    rbase = __shfl_sync(FULL, rbase, 0);
    fbase = __shfl_sync(FULL, fbase, 0);
    if (ebase + nfast > cap && nfast) {
        if (lane == 0) atomicOr(&b.cnt[C_FLAGS * b.E + e], F_EDGES);
    }
    for (uint32_t r0 = 0; r0 < n; r0 += 32) {
        const uint32_t x = r0 + lane;
        const bool v = x < n;
        uint32_t A = 0, B = 0, s0 = x;
        bool start = false, fast = false;
        if (v) {
            A = S.pA[x];
            B = S.pB[x];
            start = x == 0 || S.pA[x - 1] != A;
            while (s0 > 0 && S.pA[s0 - 1] == A) --s0;
            fast = S.pHave[s0] == 0;
        }
        const uint32_t fm = __ballot_sync(FULL, fast), rm = __ballot_sync(FULL, start && fast);
        const uint32_t epos = ebase + __popc(fm & lt), rpos = rbase + __popc(rm & lt);
        ebase += __popc(fm);
        rbase += __popc(rm);
        if (!v) continue;
        if (fast) {
            if (epos < cap) b.nbr[g0 + epos] = B;
            if (start) {
                // the run's length and the edges that fit the region
                uint32_t len = 1;
                while (x + len < n && S.pA[x + len] == A) ++len;
                const uint32_t nw = epos >= cap ? 0u : min(len, cap - epos);
                b.nbr_head[A] = make_uint2(g0 + epos, nw);
                if (rpos < cap) {
                    b.root_list[g0 + rpos] = A;
                    b.root_in[g0 + rpos] = S.pI[x];
                } else {
                    atomicOr(&b.cnt[C_FLAGS * b.E + e], F_EDGES);
                }
            }
        } else if (start) {
            // an in-cell with edges from an earlier out-layer: old edges, then this run
            uint32_t len = 1;
            while (x + len < n && S.pA[x + len] == A) ++len;
            const uint2 hd = b.nbr_head[A];
            const uint32_t need = hd.y + len;
            const uint32_t my0 = atomicAdd(&b.cnt[C_EDGES * b.E + e], need);
            const uint32_t nw = my0 >= cap ? 0u : min(need, cap - my0);
            if (nw < need) atomicOr(&b.cnt[C_FLAGS * b.E + e], F_EDGES);
            uint32_t wr = 0;
            for (uint32_t t = 0; t < hd.y && wr < nw; ++t) b.nbr[g0 + my0 + wr++] = b.nbr[hd.x + t];
            for (uint32_t t = 0; t < len && wr < nw; ++t) b.nbr[g0 + my0 + wr++] = S.pB[x + t];
            b.nbr_head[A] = make_uint2(g0 + my0, wr);
        }
        // the target reached; its frontier slot
        const uint32_t bit = 1u << (B & 31u);
        const bool fresh = !(atomicOr(&b.live[B >> 5], bit) & bit);
        if (fresh) b.nbr_head[B].y = 0u;
        if (front) {
            const uint32_t fpos = fbase + x;
            if (fpos < cap) {
                b.front_list[g0 + fpos] = fresh ? B : kNone;
                b.front_in[g0 + fpos] = S.jpos[S.pK[x] >> 8];
            } else {
                atomicOr(&b.cnt[C_FLAGS * b.E + e], F_EDGES);
            }
        }
    }
    __syncwarp();
}

// Stage the (z, r) of a union's hits (n <= kStage) into dst, four loads in flight per lane.
__device__ __forceinline__ void tile_stage(const DevBatch &b, const TileSpan &t, float2 *dst,
                                           uint32_t lane)
{
    for (uint32_t q0 = 0; q0 < t.n; q0 += 128) {
        float4 h[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t q = q0 + 32u * u + lane;
            if (q < t.n) h[u] = b.hs[tile_pos(t, q)];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t q = q0 + 32u * u + lane;
            if (q < t.n) dst[q] = make_float2(h[u].z, h[u].w);
        }
    }
}

template <bool F64>
__global__ void __launch_bounds__(kTileW * 32, PXR_TILE_MINB) k_connect_tiles(DevBatch b,
                                                                             DevParams p,
                                                                             uint32_t layer_mask)
{
    extern __shared__ __align__(16) unsigned char s_tile[];   // kTileW x TileWarp
    const uint32_t FULL = 0xFFFFFFFFu;
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    TileWarp &S = reinterpret_cast<TileWarp *>(s_tile)[wid];
    const uint32_t nk = p.n_keys;
    const int nb = (int)p.nb;
    const uint64_t stride = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t n_tiles = b.jbase[b.E];
    for (uint64_t tt = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; tt < n_tiles;
         tt += stride) {
        // the tile: (event, junction layer, first junction hit, junction hits)
        const uint4 tr = b.tiles[tt];
        const uint32_t e = tr.x, Lj = tr.y, J0 = tr.z, nJ = tr.w;
        const uint32_t *bk = b.bkt + (size_t)e * (nk + 1);
        const uint32_t nin = p.n_in[Lj], nout = p.n_out[Lj];
        if (nJ == 0 || nin == 0 || nout == 0) continue;
        const bool jv = lane < nJ;
        const uint32_t j = J0 + (jv ? lane : 0u);
        const float4 hj = b.hs[j];
        const float phij = b.hphi[j];
        const bool ok = jv && fabsf(phij) <= 4.f;    // (a non-finite azimuth has no window)
        const int blo = ok ? (int)floorf((phij - p.w_eps + kPiF2) * p.bins_per_rad) : 0;
        const int bhi = ok ? (int)floorf((phij + p.w_eps + kPiF2) * p.bins_per_rad) : 0;
        const uint4 itj0 = ok ? b.item[(size_t)j * kMaxOut] : make_uint4(0u, 0u, 0u, 0u);
        // the unions on the first root in-layer and the first out-layer (kept for the passes
        // below); every union must fit the staging, otherwise the tile's junctions go one by one
        uint32_t si0 = 0;
        while (si0 < nin && !((p.root_mask >> p.in_layer[Lj][si0]) & 1u)) ++si0;
        if (si0 == nin) continue;
        uint32_t ws0, wn0, os, on;
        const TileSpan ti0 = tile_span(bk + p.in_layer[Lj][si0] * p.nb, nb, ok, blo, bhi, ws0, wn0);
        const TileSpan tk0 = tile_span(bk + p.out_layer[Lj][0] * p.nb, nb, ok, blo, bhi, os, on);
        bool fits = ti0.n <= (uint32_t)kStage && tk0.n <= (uint32_t)kStage;
        for (uint32_t si = si0 + 1; si < nin && fits; ++si) {
            const uint32_t Li = p.in_layer[Lj][si];
            if (!((p.root_mask >> Li) & 1u)) continue;
            uint32_t ws, wn;
            fits = tile_span(bk + Li * p.nb, nb, ok, blo, bhi, ws, wn).n <= (uint32_t)kStage;
        }
        for (uint32_t s = 1; s < nout && fits; ++s) {
            uint32_t ws, wn;
            fits = tile_span(bk + p.out_layer[Lj][s] * p.nb, nb, ok, blo, bhi, ws, wn).n <=
                   (uint32_t)kStage;
        }
        if (!fits) {
            for (uint32_t t = 0; t < nJ; ++t)
                connect_junction<F64>(b, p, e, J0 + t, layer_mask, S.u.f.sH, S.u.f.sT, S.u.f.bin);
            continue;
        }
        const bool j_root = (p.root_mask >> Lj) & 1u;
        __syncwarp();
        S.jh[lane] = hj;
        S.jpos[lane] = j;
        for (uint32_t si = 0; si < nin; ++si) {
            const uint32_t Li = p.in_layer[Lj][si];
            // this pass takes the root in-cells; reached non-root ones go to the sparse pass
            if (!((p.root_mask >> Li) & 1u)) continue;
            const uint32_t slot_i = p.in_slot[Lj][si];
            uint32_t ws = ws0, wn = wn0;
            const TileSpan ti = si == si0 ? ti0 : tile_span(bk + Li * p.nb, nb, ok, blo, bhi, ws, wn);
            if (ti.n == 0) continue;
            __syncwarp();
            tile_stage(b, ti, S.u.t.hin, lane);
            for (uint32_t s = 0; s < nout; ++s) {
                const uint32_t Lk = p.out_layer[Lj][s];
                const bool disk = p.is_disk[Lk];
                const bool front = !j_root && p.n_out[Lk] > 0;
                const bool more = s > 0;
                const uint4 itj = s == 0 ? itj0 : (ok ? b.item[(size_t)j * kMaxOut + s]
                                                      : make_uint4(0u, 0u, 0u, 0u));
                const TileSpan tk = s == 0 ? tk0 : tile_span(bk + Lk * p.nb, nb, ok, blo, bhi, os, on);
                if (tk.n == 0) continue;
                __syncwarp();
                S.jit[lane] = itj;
                // the outer union's free (z barrel, r disk) coordinates and their range, the
                // range of the fixed coordinate
                int m0 = ford(3.0e38f), m1 = ford(-3.0e38f), m2 = m0, m3 = m1;
                for (uint32_t q0 = 0; q0 < tk.n; q0 += 128) {
                    float4 h[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const uint32_t q = q0 + 32u * u + lane;
                        if (q < tk.n) h[u] = b.hs[tile_pos(tk, q)];
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const uint32_t q = q0 + 32u * u + lane;
                        if (q < tk.n) {
                            const float fc = disk ? h[u].w : h[u].z, xc = disk ? h[u].z : h[u].w;
                            S.u.t.zs[q] = fc;
                            m0 = min(m0, ford(fc));
                            m1 = max(m1, ford(fc));
                            m2 = min(m2, ford(xc));
                            m3 = max(m3, ford(xc));
                        }
                    }
                }
                const float flo = funord(__reduce_min_sync(FULL, m0));
                const float fhi = funord(__reduce_max_sync(FULL, m1));
                const float jfix = disk ? hj.z : hj.w, jfree = disk ? hj.w : hj.z;
                const float xmin = funord(__reduce_min_sync(FULL, m2));
                const float xmax = funord(__reduce_max_sync(FULL, m3));
                if (lane == 0) {
                    S.fix[0] = xmin;
                    S.fix[1] = xmax;
                }
                float dlo = xmin - jfix, dhi = xmax - jfix;
                dlo -= 1e-4f + 1e-5f * fabsf(dlo);
                dhi += 1e-4f + 1e-5f * fabsf(dhi);
                const float dmx = 1e-5f * fmaxf(fabsf(dlo), fabsf(dhi));
                const float scale = fhi > flo ? (float)kZBins / (fhi - flo) : 0.f;
                auto local_bin = [&](float fc) {
                    const int bb = (int)floorf((fc - flo) * scale);
                    return bb < 0 ? 0u : (bb >= (int)kZBins ? kZBins - 1u : (uint32_t)bb);
                };
                // counting sort of the staged hits by bin (16-bit counters, two per word):
                // histogram, scan, scatter
                uint32_t *zb = S.u.t.zb;
#pragma unroll
                for (uint32_t q = 0; q < kZBins / 2; q += 32) zb[q + lane] = 0;
                __syncwarp();
                for (uint32_t q = lane; q < tk.n; q += 32) {
                    const uint32_t x = local_bin(S.u.t.zs[q]);
                    atomicAdd(&zb[x >> 1], 1u << (16u * (x & 1u)));
                }
                __syncwarp();
                {
                    constexpr uint32_t per = kZBins / 64;      // words per lane
                    uint32_t v[per], sum = 0;
#pragma unroll
                    for (uint32_t q = 0; q < per; ++q) {
                        v[q] = zb[lane * per + q];
                        sum += (v[q] & 0xFFFFu) + (v[q] >> 16);
                    }
                    uint32_t incl = sum;
#pragma unroll
                    for (int w = 1; w < 32; w <<= 1) {
                        const uint32_t t = __shfl_up_sync(FULL, incl, w);
                        if (lane >= (uint32_t)w) incl += t;
                    }
                    uint32_t run = incl - sum;
                    __syncwarp();
#pragma unroll
                    for (uint32_t q = 0; q < per; ++q) {
                        const uint32_t lo16 = run, hi16 = run + (v[q] & 0xFFFFu);
                        zb[lane * per + q] = lo16 | hi16 << 16;
                        run = hi16 + (v[q] >> 16);
                    }
                    __syncwarp();
                }
                for (uint32_t q = lane; q < tk.n; q += 32) {
                    const float fc = S.u.t.zs[q];
                    const uint32_t x = local_bin(fc), sh = 16u * (x & 1u);
                    const uint32_t pos = (atomicAdd(&zb[x >> 1], 1u << sh) >> sh) & 0xFFFFu;
                    S.u.t.zo[pos] = fc;
                    S.u.t.sT[pos] = (uint16_t)q;
                }
                __syncwarp();
                // zb now holds the end of each bin.  The lanes step through their junctions'
                // inner windows together; candidates in a cone are queued (ring of kTileQ,
                // positions head..tail) and tested 32 at a time; passes buffered (np of them).
                const uint32_t wme = itj.y ? wn : 0u;      // j without cells on Lk: nothing
                const uint32_t wmax = __reduce_max_sync(FULL, wme);
                uint32_t head = 0, tail = 0, np = 0;
                // test the n <= 32 candidates at the queue head, passes appended in queue order
                auto batch = [&](uint32_t n) {
                    const bool v = lane < n;
                    const uint32_t ent = v ? S.q[(head + lane) % kTileQ] : 0u;
                    head += n;
                    uint32_t A = kNone, B = kNone, pi = 0;
                    const uint32_t t = ent >> 16, sx = (ent >> 8) & 0xFFu, kt = ent & 0xFFu;
                    if (v) {
                        // the out-cell (j, k) by k's rank in j's window; the hits and i's entries
                        // record loaded together, then both cell entries together
                        pi = tile_pos(ti, sx);
                        const uint32_t k = tile_pos(tk, kt), jq = S.jpos[t];
                        const uint4 itq = S.jit[t];
                        const uint32_t rk = k >= itq.z ? k - itq.z : k + itq.w;
                        if (rk < itq.y) {
                            const float4 hi = b.hs[pi], hk = b.hs[k], hjt = S.jh[t];
                            const uint4 iti = b.item[(size_t)pi * kMaxOut + slot_i];
                            if (triplet_test<F64>(b, p, pi, jq, itq.x + rk, k, hi.x, hi.y, hjt,
                                                  hk, rz32(hi, hjt))) {
                                const uint32_t ri = jq >= iti.z ? jq - iti.z : jq + iti.w;
                                if (ri < iti.y) {
                                    const uint32_t Bc = itq.x + rk, Ac = iti.x + ri;
                                    const bool in = PXR_IN(b, e, Bc, b.C) && PXR_IN(b, e, Ac, b.C);
                                    const uint32_t ob = in ? b.cell_out[Bc] : kNone;
                                    const uint32_t oa = in ? b.cell_out[Ac] : kNone;
                                    // (j, k) and (i, j) cells: the doublet stage kept both
                                    if (ob == k && oa == jq) {
                                        A = Ac;
                                        B = Bc;
                                    }
                                }
                            }
                        }
                    }
                    const uint32_t pm = __ballot_sync(FULL, A != kNone);
                    if (A != kNone) {
                        const uint32_t x = np + __popc(pm & lt);
                        S.pA[x] = A;
                        S.pB[x] = B;
                        S.pI[x] = pi;
                        S.pK[x] = t << 8 | sx;
                    }
                    np += __popc(pm);
                };
                // append the buffered passes whose runs are complete: all but the last run when
                // the queue head belongs to the same in-cell (moved to the buffer's front)
                auto flush_complete = [&]() {
                    uint32_t keep = 0;
                    if (np && tail != head &&
                        S.pK[np - 1] == ((S.q[head % kTileQ] >> 8) & 0x1FFFu)) {
                        const uint32_t Al = S.pA[np - 1];
                        while (keep < np && S.pA[np - 1 - keep] == Al) ++keep;
                    }
                    tile_flush(b, e, S, np - keep, more, front, lane);
                    uint32_t a0 = 0, b0 = 0, i0 = 0, k0 = 0;
                    if (lane < keep) {
                        const uint32_t src = np - keep + lane;
                        a0 = S.pA[src];
                        b0 = S.pB[src];
                        i0 = S.pI[src];
                        k0 = S.pK[src];
                    }
                    __syncwarp();
                    if (lane < keep) {
                        S.pA[lane] = a0;
                        S.pB[lane] = b0;
                        S.pI[lane] = i0;
                        S.pK[lane] = k0;
                    }
                    __syncwarp();
                    np = keep;
                };
                // the steps; in-cells whose cone holds more than kTileCand candidates are listed
                // and written by their lanes alone between runs of steps (rare: kept out of the
                // step loop, whose registers a call would constrain)
                uint32_t nalone = 0;
                for (uint32_t c = 0; c < wmax;) {
                    for (; c < wmax; ++c) {
                        // ---- this step's inner hit per lane: cone, bins, candidates inside ----
                        uint32_t nq = 0, k0 = 0, k1 = 0, sx = 0;
                        if (c < wme) {
                            sx = ws + c;
                            if (sx >= ti.n) sx -= ti.n;
                            const float2 hi = S.u.t.hin[sx];     // (z, r)
                            // the segment (i, j) in r-z (norm and error bound only where tested)
                            const float ar = __fsub_rn(hj.w, hi.y), az = __fsub_rn(hj.z, hi.x);
                            uint32_t q0 = 0, q1 = tk.n;
                            float lo = -3.0e38f, hi_ = 3.0e38f;
                            if (cone_tile(ar, az, jfree, dlo, dhi, dmx, disk, p.tan_win, lo, hi_)) {
                                if (hi_ < flo || lo > fhi) {
                                    q1 = 0;
                                } else {
                                    int b0 = (int)floorf((lo - flo) * scale);
                                    int b1 = (int)floorf((hi_ - flo) * scale);
                                    b0 = b0 < 0 ? 0 : (b0 >= (int)kZBins ? (int)kZBins - 1 : b0);
                                    b1 = b1 < 0 ? 0 : (b1 >= (int)kZBins ? (int)kZBins - 1 : b1);
                                    q0 = b0 ? zbin_end(zb, b0 - 1) : 0u;
                                    q1 = zbin_end(zb, b1);
                                }
                            }
                            for (uint32_t q = q0; q < q1; ++q) {
                                const float fc = S.u.t.zo[q];
                                if (fc < lo || fc > hi_) continue;
                                const uint32_t kt = S.u.t.sT[q];
                                if (nq == 0) k0 = kt;
                                else if (nq == 1) k1 = kt;
                                ++nq;
                            }
                        }
                        const uint32_t me = lane << 16 | sx << 8;
                        const bool alone = nq > kTileCand;
                        const uint32_t am = __ballot_sync(FULL, alone);
                        if (alone) S.alone[nalone + __popc(am & lt)] = me >> 8;
                        nalone += __popc(am);
                        // ---- queue the others' candidates (0 to 2 per lane, adjacent) ----
                        const uint32_t m = alone ? 0u : nq;
                        const uint32_t m1 = __ballot_sync(FULL, m & 1u), m2 = __ballot_sync(FULL, m & 2u);
                        if (m1 | m2) {
                            const uint32_t x = tail + __popc(m1 & lt) + 2u * __popc(m2 & lt);
                            if (m > 0) S.q[x % kTileQ] = me | k0;
                            if (m > 1) S.q[(x + 1) % kTileQ] = me | k1;
                            tail += __popc(m1) + 2u * __popc(m2);
                            __syncwarp();
                        }
                        // ---- full batches; a flush keeps a run that may continue in the queue
                        while (tail - head >= 32) {
                            if (np + 32 > kTilePass) flush_complete();
                            batch(32);
                            __syncwarp();
                        }
                        if (nalone > kTileAlone - 32) {
                            ++c;
                            break;
                        }
                    }
                    __syncwarp();
                    if (lane < nalone)
                        tile_alone<F64>(b, p, e, S, ti, tk, S.alone[lane], flo, fhi, scale, disk,
                                        slot_i, more, front);
                    if (nalone > 32 && lane < nalone - 32)
                        tile_alone<F64>(b, p, e, S, ti, tk, S.alone[32 + lane], flo, fhi, scale,
                                        disk, slot_i, more, front);
                    nalone = 0;
                    __syncwarp();
                }
                // drain the queue and append everything
                while (tail != head) {
                    if (np + 32 > kTilePass) flush_complete();
                    batch(min(32u, tail - head));
                    __syncwarp();
                }
                tile_flush(b, e, S, np, more, front, lane);
            }
        }
    }
}


// The tiles of a dense CA level: per event and layer of layer_mask, its hits in runs of
// per_tile.  jbase[e] = the tiles of events before e, jbase[E] = all; tiles[] = each tile's
// (event, layer, first hit, hits).  One CTA; each thread takes a run of consecutive events.
__global__ void __launch_bounds__(1024) k_jbase(DevBatch b, DevParams p, uint32_t layer_mask,
                                                uint32_t per_tile)
{
    __shared__ uint32_t s_w[32];
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    const uint32_t per = (b.E + nt - 1) / nt;
    const uint32_t e0 = min(b.E, tid * per), e1 = min(b.E, e0 + per);
    auto count = [&](uint32_t e) {
        const uint32_t *bke = b.bkt + (size_t)e * (p.n_keys + 1);
        uint32_t c = 0;
        for (uint32_t l = 0; l < p.n_layers; ++l)
            if ((layer_mask >> l) & 1u)
                c += (bke[(l + 1) * p.nb] - bke[l * p.nb] + per_tile - 1) / per_tile;
        return c;
    };
    uint32_t mine = 0;
    for (uint32_t e = e0; e < e1; ++e) mine += count(e);
    const uint32_t lane = tid & 31u, wid = tid >> 5;
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= (uint32_t)o) incl += t;
    }
    if (lane == 31) s_w[wid] = incl;
    __syncthreads();
    uint32_t run = 0, tot = 0;
    for (uint32_t w = 0; w < nt / 32; ++w) {
        if (w < wid) run += s_w[w];
        tot += s_w[w];
    }
    run += incl - mine;
    for (uint32_t e = e0; e < e1; ++e) {
        b.jbase[e] = run;
        run += count(e);
    }
    if (tid == 0) b.jbase[b.E] = tot;
    __syncthreads();
    // the records: one warp per event, its tiles over the lanes
    for (uint32_t e = wid; e < b.E; e += nt / 32) {
        uint32_t r = b.jbase[e];
        const uint32_t *bke = b.bkt + (size_t)e * (p.n_keys + 1);
        for (uint32_t l = 0; l < p.n_layers; ++l) {
            if (!((layer_mask >> l) & 1u)) continue;
            const uint32_t lo = bke[l * p.nb], n_l = bke[(l + 1) * p.nb] - lo;
            const uint32_t ntl = (n_l + per_tile - 1) / per_tile;
            for (uint32_t k = lane; k < ntl; k += 32)
                b.tiles[r + k] = make_uint4(e, l, lo + k * per_tile, min(per_tile, n_l - k * per_tile));
            r += ntl;
        }
    }
}

void launch_connect(const DevBatch &b, const DevParams &p, uint32_t layer_mask, cudaStream_t s,
                    int sms)
{
    k_jbase<<<1, 1024, 0, s>>>(b, p, layer_mask, kTileJ);
    // tiles: at most one per kTileJ hits plus one per event and layer
    uint64_t blocks = ((uint64_t)b.N / kTileJ + (uint64_t)b.E * p.n_layers + kTileW - 1) / kTileW;
    uint64_t cap = (uint64_t)sms * p.grid_per_sm[2];
    if (blocks > cap) blocks = cap;
    if (blocks == 0) return;
    if (p.cut_mode == CUT_FP64)
        k_connect_tiles<true><<<(unsigned)blocks, kTileW * 32, kTileSmem, s>>>(b, p, layer_mask);
    else
        k_connect_tiles<false><<<(unsigned)blocks, kTileW * 32, kTileSmem, s>>>(b, p, layer_mask);
}

// Sparse CA pass of one level over the frontier: cells B = (j, k) that were reached (have an
// in-edge), are not root cells, and whose outer hit k lies on a junction layer of the level.
// One lane per frontier entry (chunks of 256 entries, all of one event per CTA): for every pair
// starting on k's layer the warp looks up the out-cells (k, l) that pass the triplet cut
// (ca_warp_pair), then appends the cells' edge lists; reached out-cells join the frontier.
template <bool F64>
__global__ void __launch_bounds__(256, PXR_CA_MINB) k_ca_front(DevBatch b, DevParams p,
                                                               uint32_t total, uint32_t layer_mask)
{
    __shared__ CaWarp s_w[8];
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    CaWarp &W = s_w[wid];
    const uint32_t n_chunks = total / kChunk;
    for (uint32_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        const uint32_t e = b.edge_chunk[ch];
        const uint32_t x0 = b.edge_off[e];
        const uint32_t nf = min(b.front_snap[e], b.edge_off[e + 1] - x0);
        if (ch * kChunk - x0 >= nf) continue;                      // uniform over the CTA
        const uint32_t x = ch * kChunk + threadIdx.x;
        uint32_t B = kNone, j = 0, k = 0, Lk = 0;
        bool valid = x - x0 < nf;
        if (valid) {
            B = b.front_list[x];
            j = b.front_in[x];
            valid = B != kNone;                                    // slot of a cell reached twice
            valid = valid && PXR_IN(b, e, B, b.C) && PXR_IN(b, e, j, b.N);
        }
        if (valid) {
            k = b.cell_out[B];
            valid = PXR_IN(b, e, k, b.N);
        }
        if (valid) {
            Lk = b.hmeta[k] >> kLocalBits;
            valid = (layer_mask >> Lk) & 1u;
        }
        float4 hj = make_float4(0.f, 0.f, 0.f, 0.f), hk = hj;
        float phik = 0.f;
        RZ32 a{0.f, 0.f, 0.f, 0.f};
        uint32_t nout = 0;
        bool k_root = false;
        if (valid) {
            hj = b.hs[j];
            hk = b.hs[k];
            phik = b.hphi[k];
            a = rz32(hj, hk);
            nout = p.n_out[Lk];
            k_root = (p.root_mask >> Lk) & 1u;
        }
        W.npass[lane] = 0;
        const uint32_t nmax = __reduce_max_sync(0xFFFFFFFFu, nout);
        for (uint32_t t = 0; t < nmax; ++t) {
            const bool act = t < nout;
            const uint32_t Ll = act ? p.out_layer[Lk][t] : 0u;
            const uint32_t fr = act && !k_root && p.n_out[Ll] > 0 ? 0x80000000u : 0u;
            const uint4 itk = act ? b.item[(size_t)k * kMaxOut + t] : make_uint4(0, 0, 0, 0);
            ca_warp_pair<F64>(b, p, e, W, lane, act, Ll, j, k, hj.x, hj.y, hk, phik, a, itk, fr);
        }
        __syncwarp();
        const uint32_t npass = W.npass[lane];
        uint32_t nw;
        const uint32_t first = ca_append(b, e, false, B, j, k, npass, W, lane, nw);
        if (npass > (uint32_t)kEdgeBuf)
            ca_rest<F64>(b, p, e, j, k, Lk, hj.x, hj.y, hk, phik, a, first, nw);
        __syncwarp();
    }
}

void launch_connect_front(const DevBatch &b, const DevParams &p, uint32_t total,
                          uint32_t layer_mask, cudaStream_t s, int sms)
{
    const uint32_t chunks = total / kChunk;
    const uint32_t cap = (uint32_t)sms * p.grid_per_sm[2];
    if (chunks == 0) return;
    const uint32_t grid = chunks < cap ? chunks : cap;
    if (p.cut_mode == CUT_FP64)
        k_ca_front<true><<<grid, 256, 0, s>>>(b, p, total, layer_mask);
    else
        k_ca_front<false><<<grid, 256, 0, s>>>(b, p, total, layer_mask);
}

// ------------------------------------------------------------------------------------------
// Ntuplets: depth-first walk from every root cell
// ------------------------------------------------------------------------------------------
// Depth-first walk from one root cell A; emits every path that has max_hits hits or ends at a
// cell without out-edges, if it has at least min_hits hits.  All lanes of a calling warp walk
// in the same event e.
__device__ __forceinline__ void walk_from(const DevBatch &b, const DevParams &p, uint32_t e,
                                          uint32_t A, uint32_t a_in)
{
    uint32_t cells[kMaxHits - 1];
    uint32_t next[kMaxHits - 1];
    int d = 0;
    cells[0] = A;
    next[0] = 0;
    const uint32_t tcap = b.tup_off[e + 1] - b.tup_off[e];
    while (d >= 0) {
        const uint32_t c = cells[d];
        const uint32_t nh = (uint32_t)d + 2u;
        if (!PXR_IN(b, e, c, b.C)) {
            --d;
            continue;
        }
        // (a path at the hit cap ends here whatever c's edges: they are not read)
        const uint2 hd = nh < p.max_hits ? b.nbr_head[c] : make_uint2(0u, 0u);
        const uint32_t ne = hd.y;
        if (next[d] == 0 && (nh >= p.max_hits || ne == 0)) {
            if (nh >= p.min_hits) {
                // one reservation for the lanes that emit together (a warp's walks share e)
                const cg::coalesced_group g = cg::coalesced_threads();
                uint32_t base = 0;
                if (g.thread_rank() == 0) base = atomicAdd(&b.cnt[C_TUPLES * b.E + e], g.size());
                const uint32_t slot = g.shfl(base, 0) + g.thread_rank();
                if (slot < tcap) {
                    const uint32_t t = b.tup_off[e] + slot;
                    uint32_t *th = b.tup_hits + (size_t)t * kMaxHits;
                    th[0] = a_in;
                    for (int q = 0; q <= d; ++q) th[q + 1] = b.cell_out[cells[q]];
                    for (int q = d + 2; q < kMaxHits; ++q) th[q] = kNone;
                    b.tup_n[t] = (uint8_t)nh;
                    b.tup_state[t] = nh < p.max_hits ? 2 : 1;
                    b.tup_first[t] = A;
                } else {
                    atomicOr(&b.cnt[C_FLAGS * b.E + e], F_TUPLES);
                }
            }
            --d;
            continue;
        }
        if (next[d] < ne) {
            if (!PXR_IN(b, e, (uint64_t)hd.x + next[d], b.G)) {
                --d;
                continue;
            }
            const uint32_t nxt = b.nbr[hd.x + next[d]];
            ++next[d];
            ++d;
            cells[d] = nxt;
            next[d] = 0;
            if (p.drop_suffixes) atomicMin(&b.mindepth[nxt], (uint32_t)d);
        } else {
            --d;
        }
    }
}

// One warp per root hit (a hit on a root layer); its lanes walk from the hit's cells.
// Walk from every root cell: one warp per root hit, the lanes over its cells.  Used when 2-hit
// paths count (min_hits <= 2), since then root cells without out-edges emit too.
__global__ void __launch_bounds__(256) k_ntuplets(DevBatch b, DevParams p)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t stride = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t gg = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gg < b.N;
         gg += stride) {
        const uint32_t g = (uint32_t)gg;
        // independent loads first (hits past an event's valid range carry layer 0xFF)
        const uint32_t L = b.hmeta[g] >> kLocalBits;
        const uint32_t e = hit_event(b, g);
        const uint4 it0 = b.item[(size_t)g * kMaxOut];
        if (L >= p.n_layers || !((p.root_mask >> L) & 1u)) continue;
        for (uint32_t s = 0; s < p.n_out[L]; ++s) {
            const uint4 its = s ? b.item[(size_t)g * kMaxOut + s] : it0;
            const uint32_t f = its.x, n = its.y;
            for (uint32_t c = lane; c < n; c += 32)
                if (b.cell_out[f + c] != kNone) walk_from(b, p, e, f + c, g);
        }
    }
}

// The chunks (kChunk entries of one event each) of the filled part of a per-event region: the
// region of event e starts at off[e], counter `which` says how much of it was filled.  Per-event
// prefix in jbase (free once the CA stage has ended; jbase[E] = all chunks), so that the walk
// visits the listed root cells (C_ROOTS of the edge regions) and the selection the emitted
// ntuplets (C_TUPLES of the ntuplet regions) without a pass over the whole capacity.  One CTA;
// each thread takes a run of consecutive events.
__global__ void __launch_bounds__(1024) k_chunks(DevBatch b, uint32_t which,
                                                 const uint32_t *__restrict__ off)
{
    __shared__ uint32_t s_w[32];
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    const uint32_t per = (b.E + nt - 1) / nt;
    const uint32_t e0 = min(b.E, tid * per), e1 = min(b.E, e0 + per);
    auto count = [&](uint32_t e) {
        const uint32_t n = min(b.cnt[which * b.E + e], off[e + 1] - off[e]);
        return (n + kChunk - 1) / kChunk;
    };
    uint32_t mine = 0;
    for (uint32_t e = e0; e < e1; ++e) mine += count(e);
    const uint32_t lane = tid & 31u, wid = tid >> 5;
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= (uint32_t)o) incl += t;
    }
    if (lane == 31) s_w[wid] = incl;
    __syncthreads();
    uint32_t run = 0, tot = 0;
    for (uint32_t w = 0; w < nt / 32; ++w) {
        if (w < wid) run += s_w[w];
        tot += s_w[w];
    }
    run += incl - mine;
    for (uint32_t e = e0; e < e1; ++e) {
        b.jbase[e] = run;
        run += count(e);
    }
    if (tid == 0) b.jbase[b.E] = tot;
}

// Walk from the root cells that have out-edges (listed per event by the CA stage): one CTA per
// chunk of an event's listed cells (k_chunks), one thread per cell.  Enough when paths need
// at least 3 hits.
__global__ void __launch_bounds__(256) k_walk_roots(DevBatch b, DevParams p)
{
    const uint32_t total = b.jbase[b.E];
    for (uint32_t v = blockIdx.x; v < total; v += gridDim.x) {
        const uint32_t e = find_event(b.jbase, b.E, v);
        const uint32_t x0 = b.edge_off[e];
        const uint32_t n = min(b.cnt[C_ROOTS * b.E + e], b.edge_off[e + 1] - x0);
        const uint32_t x = (v - b.jbase[e]) * kChunk + threadIdx.x;
        if (x < n) walk_from(b, p, e, b.root_list[x0 + x], b.root_in[x0 + x]);
    }
}

void launch_ntuplets(const DevBatch &b, const DevParams &p, uint32_t edge_total, cudaStream_t s,
                     int sms)
{
    if (p.min_hits > 2) {
        const uint32_t chunks = edge_total / kChunk;
        const uint32_t cap = (uint32_t)sms * p.grid_per_sm[3];
        if (chunks == 0) return;
        // (the edge capacity bounds the listed root cells, hence their chunks)
        k_chunks<<<1, 1024, 0, s>>>(b, C_ROOTS, b.edge_off);
        k_walk_roots<<<chunks < cap ? chunks : cap, kChunk, 0, s>>>(b, p);
        return;
    }
    uint64_t blocks = ((uint64_t)b.N + 7) / 8;
    uint64_t cap = (uint64_t)sms * 2 * p.grid_per_sm[3];
    if (blocks > cap) blocks = cap;
    if (blocks == 0) return;
    k_ntuplets<<<(unsigned)blocks, 256, 0, s>>>(b, p);
}

// ------------------------------------------------------------------------------------------
// Selection: a path that ended without an out-edge is a strict suffix of another emitted path
// exactly when a root path of m hits enters its first cell and m + (its hits) <= max_hits.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_select(DevBatch b, DevParams p)
{
    const uint32_t total = b.jbase[b.E];      // chunks of emitted ntuplets (k_chunks)
    for (uint32_t v = blockIdx.x; v < total; v += gridDim.x) {
        const uint32_t e = find_event(b.jbase, b.E, v);
        const uint32_t t0 = b.tup_off[e];
        const uint32_t nt = min(b.cnt[C_TUPLES * b.E + e], b.tup_off[e + 1] - t0);
        const uint32_t x = (v - b.jbase[e]) * kChunk + threadIdx.x;
        if (x >= nt) continue;
        const uint32_t t = t0 + x;
        bool keep = true;
        if (p.drop_suffixes && b.tup_state[t] == 2 && PXR_IN(b, e, b.tup_first[t], b.C)) {
            const uint32_t md = b.mindepth[b.tup_first[t]];
            if (md != kNone && md + b.tup_n[t] <= p.max_hits) keep = false;
        }
        const uint32_t rank = keep ? atomicAdd(&b.cnt[C_OUT * b.E + e], 1u) : kNone;
        b.tup_rank[t] = rank;
        if (keep) b.tup_list[t0 + rank] = t;
    }
}

void launch_select(const DevBatch &b, const DevParams &p, uint32_t total, cudaStream_t s, int sms)
{
    uint64_t blocks = total / kChunk;              // (bounds the chunks of emitted ntuplets)
    uint64_t cap = (uint64_t)sms * 2 * p.grid_per_sm[4];
    if (blocks > cap) blocks = cap;
    if (blocks == 0) return;
    k_chunks<<<1, 1024, 0, s>>>(b, C_TUPLES, b.tup_off);
    k_select<<<(unsigned)blocks, 256, 0, s>>>(b, p);
}

// Exclusive prefix of the per-event output counts (one CTA).
__global__ void k_out_scan(DevBatch b)
{
    __shared__ uint32_t carry;
    __shared__ uint32_t warp_tot[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    for (uint32_t e0 = 0; e0 < b.E; e0 += blockDim.x) {
        uint32_t e = e0 + threadIdx.x;
        uint32_t v = e < b.E ? b.cnt[C_OUT * b.E + e] : 0u;
        uint32_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= (uint32_t)o) incl += t;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            uint32_t nw = blockDim.x >> 5;
            uint32_t w = lane < nw ? warp_tot[lane] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t t = __shfl_up_sync(0xFFFFFFFFu, w, o);
                if (lane >= (uint32_t)o) w += t;
            }
            if (lane < nw) warp_tot[lane] = w;
        }
        __syncthreads();
        uint32_t excl = carry + incl - v + (wid ? warp_tot[wid - 1] : 0u);
        if (e < b.E) b.out_evt[e] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) b.out_evt[b.E] = carry;
}

void launch_out_scan(const DevBatch &b, cudaStream_t s)
{
    k_out_scan<<<1, 1024, 0, s>>>(b);
}

// Caller index of slot q of ntuplet t, kNone past its hits (the padding of the canonical order).
__device__ __forceinline__ uint32_t tup_caller(const DevBatch &b, uint32_t e, uint32_t t, int q)
{
    if (q >= b.tup_n[t]) return kNone;
    const uint32_t h = b.tup_hits[(size_t)t * kMaxHits + q];
    return PXR_IN(b, e, h, b.N) ? b.hmeta[h] & kLocalMask : kNone;
}

constexpr uint32_t kCanonSmem = 32768;     // events with more hits count in global memory

// Canonical order of each event's kept ntuplets: lexicographic by their hits' caller indices
// (unused slots as kNone), so that a result does not depend on the batch or on the order in
// which the walk found the ntuplets.  A counting sort by the first hit (per-hit counters of the
// event, in shared memory up to kCanonSmem hits), then each bucket (the ntuplets sharing a first
// hit: a few) by insertion on the remaining hits; tup_list receives the order, in which the fit
// writes the tracks.  One CTA per event.
__global__ void __launch_bounds__(1024) k_canon(DevBatch b)
{
    extern __shared__ uint32_t s_cnt[];        // the bucket counters of events up to kCanonSmem hits
    __shared__ uint32_t s_warp[32];
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    for (uint32_t e = blockIdx.x; e < b.E; e += gridDim.x) {
        const uint32_t h0 = b.hit_off[e], nh = b.hit_off[e + 1] - h0;
        const uint32_t t0 = b.tup_off[e];
        const uint32_t n = b.out_evt[e + 1] - b.out_evt[e];
        if (n < 2) continue;                                       // uniform over the CTA
        uint32_t *cnt = nh <= kCanonSmem ? s_cnt : b.canon_cnt + h0;   // uniform over the CTA
        uint32_t *tmp = b.tup_tmp + t0;
        for (uint32_t c = tid; c < nh; c += nt) cnt[c] = 0;
        __syncthreads();
        for (uint32_t k = tid; k < n; k += nt) atomicAdd(&cnt[tup_caller(b, e, b.tup_list[t0 + k], 0)], 1u);
        __syncthreads();
        block_exclusive_scan(cnt, nh, s_warp);
        for (uint32_t k = tid; k < n; k += nt) {
            const uint32_t t = b.tup_list[t0 + k];
            tmp[atomicAdd(&cnt[tup_caller(b, e, t, 0)], 1u)] = t;
        }
        __syncthreads();
        // cnt[c] is now the end of bucket c
        for (uint32_t c = tid; c < nh; c += nt) {
            const uint32_t lo = c ? cnt[c - 1] : 0u, hi = cnt[c];
            for (uint32_t x = lo + 1; x < hi; ++x) {
                const uint32_t t = tmp[x];
                uint32_t y = x;
                while (y > lo) {
                    const uint32_t u = tmp[y - 1];
                    int cmp = 0;
                    for (int q = 1; q < kMaxHits && cmp == 0; ++q) {
                        const uint32_t a = tup_caller(b, e, u, q), v = tup_caller(b, e, t, q);
                        cmp = a < v ? -1 : (a > v ? 1 : 0);
                    }
                    if (cmp <= 0) break;
                    tmp[y] = u;
                    --y;
                }
                tmp[y] = t;
            }
        }
        __syncthreads();
        for (uint32_t k = tid; k < n; k += nt) b.tup_list[t0 + k] = tmp[k];
        __syncthreads();
    }
}

void launch_canon(const DevBatch &b, cudaStream_t s, int sms)
{
    const uint32_t grid = b.E < (uint32_t)sms * 2 ? b.E : (uint32_t)sms * 2;
    if (grid == 0) return;
    k_canon<<<grid, 1024, kCanonSmem * sizeof(uint32_t), s>>>(b);
}

cudaError_t init_graph_kernels()
{
    cudaError_t r = cudaFuncSetAttribute(k_canon, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kCanonSmem * (int)sizeof(uint32_t));
    if (r == cudaSuccess)
        r = cudaFuncSetAttribute(k_connect_tiles<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSmem);
    if (r == cudaSuccess)
        r = cudaFuncSetAttribute(k_connect_tiles<true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSmem);
    return r;
}

}  // namespace pxr
