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
#include "pxr_dev.cuh"
#include "pxr_cuts.cuh"

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
    int blo = (int)floorf((phi - p.w_eps + kPiF2) * p.bins_per_rad);
    int bhi = (int)floorf((phi + p.w_eps + kPiF2) * p.bins_per_rad);
    Window w;
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
    uint64_t blocks = (warps + 7) / 8;
    const uint64_t cap = (uint64_t)sms * p.grid_per_sm[1];
    if (blocks > cap) blocks = cap;
    if (blocks == 0) return;
    if (p.cut_mode == CUT_FP64)
        k_doublets<true><<<(unsigned)blocks, 256, 0, s>>>(b, p, slots);
    else
        k_doublets<false><<<(unsigned)blocks, 256, 0, s>>>(b, p, slots);
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
                                           float xi, float yi, float4 hj, float4 hk,
                                           bool need_theta, int dc, double theta, double dca)
{
    if (need_theta) {
        const uint32_t k = cell_out[B];
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

// Exact decision for the triplet (i, j, k), k the outer hit of the out-cell B = (j, k):
// r-z alignment, then DCA.  FP32 mode decides in float when outside the guard bands and takes
// the FP64 formulas otherwise (FP64 mode always).
template <bool F64>
__device__ __forceinline__ bool triplet_test(const DevBatch &b, const DevParams &p, uint32_t i,
                                             uint32_t j, uint32_t B, float xi, float yi,
                                             float4 hj, float4 hk, const RZ32 &a)
{
    if constexpr (F64) {
        if (theta32(a, rz32(hj, hk), p.theta32) == 0) return false;
        const uint32_t k = b.cell_out[B];
        const double zi = (double)b.hs[i].z, zj = (double)hj.z, zk = (double)hk.z;
        const double ri = b.r64[i], rj = b.r64[j], rk = b.r64[k];
        if (!theta64(ri, zi, rj, zj, rk, zk, seglen64(ri, zi, rj, zj), seglen64(rj, zj, rk, zk),
                     p.theta))
            return false;
        if (dca32(xi, yi, hj.x, hj.y, hk.x, hk.y, p.dca32) == 0) return false;
        return dca64((double)xi, (double)yi, (double)hj.x, (double)hj.y, (double)hk.x,
                     (double)hk.y) <= p.dca;
    } else {
        const int th = theta32(a, rz32(hj, hk), p.theta32);
        if (th == 0) return false;
        const int dc = dca32(xi, yi, hj.x, hj.y, hk.x, hk.y, p.dca32);
        if (th == 1 && dc >= 0) return dc == 1;
        return triplet_exact(b.r64, b.cell_out, b.hs, i, j, B, xi, yi, hj, hk, th < 0, dc,
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

constexpr int kConnWarps = 8;
constexpr int kStage = 256;     // out-cells of one junction staged per out-layer slot
constexpr int kBins = 128;      // local bins of the free coordinate (multiple of 32)

// Order-preserving int encoding of floats (for warp min / max reductions).
__device__ __forceinline__ int ford(float f)
{
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float funord(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF); }

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
        b.nbr_n[C] = 0u;
        return;
    }
    if (atomicOr(&b.live[C >> 5], bit) & bit) return;
    b.nbr_n[C] = 0u;
    const uint32_t cap = b.edge_off[e + 1] - b.edge_off[e];
    const uint32_t x = atomicAdd(&b.cnt[C_FRONT * b.E + e], 1u);
    if (x < cap) {
        b.front_list[b.edge_off[e] + x] = C;
        b.front_in[b.edge_off[e] + x] = c_in;
    } else {
        atomicOr(&b.cnt[C_FLAGS * b.E + e], F_EDGES);
    }
}

// One warp per junction hit j.  For each out-layer slot, j's out-cells (j, k) are staged in
// shared memory (k's coordinates) and counting-sorted by the free coordinate of k (z on barrel
// layers, r on disks) into local bins over the staged range.  The in-cells (i, j) are found 32
// at a time, one per lane, by scanning i over j's phi window on the inner layer with the doublet
// cut; each lane computes the cone of r-z directions that can pass the alignment cut, the bins it
// reaches (a conservative window: the exact cuts decide) and tests those out-cells itself (j's
// entries of failed candidates are skipped).  The in-cell's index is j's rank in i's window
// (loaded alongside the tests).  Lanes with passes append their edges: the round's returning
// atomics (edge and root-list reservations, frontier slots, reached marks) are issued together,
// so a round waits on one atomic round trip.  A slot with more than kStage entries is tested
// from global memory.  Loads that do not depend on one another are issued together (the
// junction's own records, its first out-cell list and inner window) so that a junction waits on
// few memory round trips.
template <bool F64>
__global__ void __launch_bounds__(kConnWarps * 32, 4) k_connect(DevBatch b, DevParams p,
                                                                uint32_t layer_mask)
{
    __shared__ float4 s_h[kConnWarps][kStage];      // staged out-cells' outer hits (list order)
    __shared__ uint16_t s_t[kConnWarps][kStage];    // list positions sorted by local bin
    __shared__ uint32_t s_bin[kConnWarps][kBins];   // bin ends after the scan
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    float4 *sH = s_h[wid];
    uint16_t *sT = s_t[wid];
    uint32_t *bin = s_bin[wid];
    const uint32_t nk = p.n_keys;
    const uint64_t stride = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t n_junctions = b.jbase[b.E];
    for (uint64_t jj = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; jj < n_junctions;
         jj += stride) {
        // the jj-th junction hit: its event from the per-event junction prefix, its position
        // from the event's layer ranges of the layers in layer_mask
        const uint32_t g = (uint32_t)jj;
        const uint32_t e = find_event(b.jbase, b.E, g);
        uint32_t o = g - b.jbase[e];
        const uint32_t *bke = b.bkt + (size_t)e * (nk + 1);
        uint32_t j = 0;
        for (uint32_t l = 0; l < p.n_layers; ++l) {
            if (!((layer_mask >> l) & 1u)) continue;
            const uint32_t lo = bke[l * p.nb], n_l = bke[(l + 1) * p.nb] - lo;
            if (o < n_l) { j = lo + o; break; }
            o -= n_l;
        }
        const uint32_t meta = b.hmeta[j];
        const float4 hj = b.hs[j];
        const float phij = b.hphi[j];
        const uint4 it0 = b.item[(size_t)j * kMaxOut];
        uint32_t f0 = it0.x, nB = it0.y;
        const uint32_t Lj = meta >> kLocalBits;
        if (Lj >= p.n_layers || !((layer_mask >> Lj) & 1u)) continue;
        const uint32_t nin = p.n_in[Lj], nout = p.n_out[Lj];
        if (nin == 0 || nout == 0) continue;
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
                        } else {
                            B = f0 + q;
                            const uint32_t k = b.cell_out[B];
                            if (k == kNone) continue;
                            hk = b.hs[k];
                        }
                        if (triplet_test<F64>(b, p, i, j, B, hi.x, hi.y, hj, hk, a)) {
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
                    if (ok && s > 0) { have = b.nbr_n[A]; old = b.nbr_first[A]; }
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
                    if (fresh) b.nbr_n[Bf] = 0u;
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
                            } else {
                                B = f0 + q;
                                const uint32_t k = b.cell_out[B];
                                if (k == kNone) continue;
                                hk = b.hs[k];
                            }
                            if (triplet_test<F64>(b, p, i, j, B, hi.x, hi.y, hj, hk, a)) {
                                b.nbr[first + wr++] = B;
                                mark_reached(b, e, B, j, front);
                            }
                        }
                        b.nbr_first[A] = first;
                        b.nbr_n[A] = wr;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// Per-event prefix of the hits on the layers of layer_mask (the junctions of a dense CA level):
// jbase[e] = junctions of events before e, jbase[E] = all.  One CTA; each thread takes a run of
// consecutive events.
__global__ void __launch_bounds__(1024) k_jbase(DevBatch b, DevParams p, uint32_t layer_mask)
{
    __shared__ uint32_t s_w[32];
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    const uint32_t per = (b.E + nt - 1) / nt;
    const uint32_t e0 = min(b.E, tid * per), e1 = min(b.E, e0 + per);
    auto count = [&](uint32_t e) {
        const uint32_t *bke = b.bkt + (size_t)e * (p.n_keys + 1);
        uint32_t c = 0;
        for (uint32_t l = 0; l < p.n_layers; ++l)
            if ((layer_mask >> l) & 1u) c += bke[(l + 1) * p.nb] - bke[l * p.nb];
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
}

void launch_connect(const DevBatch &b, const DevParams &p, uint32_t layer_mask, cudaStream_t s,
                    int sms)
{
    k_jbase<<<1, 1024, 0, s>>>(b, p, layer_mask);
    uint64_t blocks = ((uint64_t)b.N + kConnWarps - 1) / kConnWarps;
    uint64_t cap = (uint64_t)sms * p.grid_per_sm[2];
    if (blocks > cap) blocks = cap;
    if (blocks == 0) return;
    if (p.cut_mode == CUT_FP64)
        k_connect<true><<<(unsigned)blocks, kConnWarps * 32, 0, s>>>(b, p, layer_mask);
    else
        k_connect<false><<<(unsigned)blocks, kConnWarps * 32, 0, s>>>(b, p, layer_mask);
}

// Sparse CA pass over the frontier: cells B = (j, k) that were reached (have an in-edge), are not
// root cells, and whose outer hit k lies on a layer of layer_mask.  Their out-edges go to the
// out-cells C = (k, l) of every pair starting on k's layer that pass the triplet cut.  Each warp
// takes 32 consecutive frontier entries (one chunk of 256 entries per CTA, all of one event): the
// lanes load their cells' hits together, then the warp tests the cells' out-entries one cell at
// a time, 32 entries per step (failed candidates skipped), collecting the passes in shared
// memory grouped by cell; one atomic reserves the edge lists of all 32 cells, which are
// contiguous and in the same order, so the warp copies them with coalesced stores.  A cell whose
// passes do not fit the buffer is redone on its own.  Reached out-cells join the frontier.
constexpr int kFrontBuf = 256;
constexpr int kFrontU = 3;      // entries per lane whose loads are issued together

template <bool F64>
__global__ void __launch_bounds__(256, 4) k_connect_front(DevBatch b, DevParams p, uint32_t total,
                                                          uint32_t layer_mask)
{
    __shared__ uint32_t s_pass[8][kFrontBuf];
    const uint32_t FULL = 0xFFFFFFFFu;
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5, lt = (1u << lane) - 1u;
    uint32_t *buf = s_pass[wid];
    const uint32_t n_chunks = total / kChunk;
    for (uint32_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        const uint32_t e = b.edge_chunk[ch];
        const uint32_t x0 = b.edge_off[e];
        const uint32_t nf = min(b.front_snap[e], b.edge_off[e + 1] - x0);
        if (ch * kChunk - x0 >= nf) continue;                      // uniform over the CTA
        // ---- this warp's 32 entries, one cell per lane ----
        const uint32_t x = ch * kChunk + wid * 32u + lane;
        uint32_t B = 0, j = 0, k = 0, Lk = 0;
        float4 hj = make_float4(0.f, 0.f, 0.f, 0.f), hk = hj;
        uint4 it0 = make_uint4(0u, 0u, 0u, 0u);                    // k's first pair's entries
        bool valid = x - x0 < nf;
        if (valid) {
            B = b.front_list[x];
            j = b.front_in[x];
            valid = B != kNone;                                    // slot of a cell reached twice
        }
        if (valid) {
            k = b.cell_out[B];
            hj = b.hs[j];
            hk = b.hs[k];
            it0 = b.item[(size_t)k * kMaxOut];
            Lk = b.hmeta[k] >> kLocalBits;
            valid = (layer_mask >> Lk) & 1u;
        }
        uint32_t my_cnt = 0, redo = 0;
        uint32_t nbuf = 0;                                         // warp-uniform
        for (uint32_t m = __ballot_sync(FULL, valid); m; m &= m - 1) {
            const int q = __ffs(m) - 1;
            const uint32_t jq = __shfl_sync(FULL, j, q), kq = __shfl_sync(FULL, k, q);
            const uint32_t Lq = __shfl_sync(FULL, Lk, q);
            const float4 hjq = make_float4(__shfl_sync(FULL, hj.x, q), __shfl_sync(FULL, hj.y, q),
                                           __shfl_sync(FULL, hj.z, q), __shfl_sync(FULL, hj.w, q));
            const float4 hkq = make_float4(__shfl_sync(FULL, hk.x, q), __shfl_sync(FULL, hk.y, q),
                                           __shfl_sync(FULL, hk.z, q), __shfl_sync(FULL, hk.w, q));
            const RZ32 a = rz32(hjq, hkq);
            const bool k_root = (p.root_mask >> Lq) & 1u;
            const uint32_t start = nbuf;
            uint32_t cnt = 0;
            bool fits = true;
            for (uint32_t s = 0; s < p.n_out[Lq]; ++s) {
                const uint4 it = s ? b.item[(size_t)kq * kMaxOut + s]
                                   : make_uint4(__shfl_sync(FULL, it0.x, q),
                                                __shfl_sync(FULL, it0.y, q), 0u, 0u);
                const bool front = !k_root && p.n_out[p.out_layer[Lq][s]] > 0;
                for (uint32_t c0 = 0; c0 < it.y; c0 += 32u * kFrontU) {
                    // all loads of the step first: entries, then their outer hits
                    uint32_t l[kFrontU];
                    float4 hl[kFrontU];
#pragma unroll
                    for (int u = 0; u < kFrontU; ++u) {
                        const uint32_t c = c0 + 32u * u + lane;
                        l[u] = c < it.y ? b.cell_out[it.x + c] : kNone;
                    }
#pragma unroll
                    for (int u = 0; u < kFrontU; ++u)
                        hl[u] = l[u] != kNone ? b.hs[l[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int u = 0; u < kFrontU; ++u) {
                        if (c0 + 32u * u >= it.y) break;                   // uniform
                        const uint32_t C = it.x + c0 + 32u * u + lane;
                        const bool pass = l[u] != kNone &&
                            triplet_test<F64>(b, p, jq, kq, C, hjq.x, hjq.y, hkq, hl[u], a);
                        const uint32_t pm = __ballot_sync(FULL, pass);
                        if (pass) {
                            const uint32_t idx = start + cnt + __popc(pm & lt);
                            if (idx < (uint32_t)kFrontBuf) buf[idx] = C;
                            mark_reached(b, e, C, kq, front);
                        }
                        cnt += __popc(pm);
                    }
                }
            }
            if (start + cnt > (uint32_t)kFrontBuf) fits = false;
            if (lane == (uint32_t)q) {
                my_cnt = fits ? cnt : 0u;
                redo = fits ? 0u : cnt;
            }
            if (fits) nbuf += cnt;
        }
        // ---- one reservation for the buffered lists (in lane order = buffer order) ----
        uint32_t incl = my_cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, incl, o);
            if (lane >= (uint32_t)o) incl += t;
        }
        uint32_t base = 0;
        if (lane == 0 && nbuf) base = atomicAdd(&b.cnt[C_EDGES * b.E + e], nbuf);
        base = __shfl_sync(FULL, base, 0);
        const uint32_t cap = b.edge_off[e + 1] - x0;
        const uint32_t nw = base >= cap ? 0u : min(nbuf, cap - base);
        if (nw < nbuf && lane == 0) atomicOr(&b.cnt[C_FLAGS * b.E + e], F_EDGES);
        __syncwarp();
        for (uint32_t t = lane; t < nw; t += 32) b.nbr[x0 + base + t] = buf[t];
        if (my_cnt) {
            const uint32_t o = incl - my_cnt;                      // offset in the warp's range
            b.nbr_first[B] = x0 + base + o;
            b.nbr_n[B] = o >= nw ? 0u : min(my_cnt, nw - o);
        }
        // ---- cells whose passes did not fit: their own reservation and a second sweep ----
        for (uint32_t m = __ballot_sync(FULL, redo > 0); m; m &= m - 1) {
            const int q = __ffs(m) - 1;
            const uint32_t Bq = __shfl_sync(FULL, B, q), n = __shfl_sync(FULL, redo, q);
            const uint32_t jq = __shfl_sync(FULL, j, q), kq = __shfl_sync(FULL, k, q);
            const uint32_t Lq = __shfl_sync(FULL, Lk, q);
            const float4 hjq = make_float4(__shfl_sync(FULL, hj.x, q), __shfl_sync(FULL, hj.y, q),
                                           __shfl_sync(FULL, hj.z, q), __shfl_sync(FULL, hj.w, q));
            const float4 hkq = make_float4(__shfl_sync(FULL, hk.x, q), __shfl_sync(FULL, hk.y, q),
                                           __shfl_sync(FULL, hk.z, q), __shfl_sync(FULL, hk.w, q));
            const RZ32 a = rz32(hjq, hkq);
            uint32_t rb = 0;
            if (lane == 0) rb = atomicAdd(&b.cnt[C_EDGES * b.E + e], n);
            rb = __shfl_sync(FULL, rb, 0);
            const uint32_t rw = rb >= cap ? 0u : min(n, cap - rb);
            if (lane == 0) {
                if (rw < n) atomicOr(&b.cnt[C_FLAGS * b.E + e], F_EDGES);
                b.nbr_first[Bq] = x0 + rb;
                b.nbr_n[Bq] = rw;
            }
            uint32_t run = 0;
            for (uint32_t s = 0; s < p.n_out[Lq] && run < rw; ++s) {
                const uint4 it = b.item[(size_t)kq * kMaxOut + s];
                for (uint32_t c0 = 0; c0 < it.y && run < rw; c0 += 32) {
                    const uint32_t C = it.x + c0 + lane;
                    bool pass = false;
                    if (c0 + lane < it.y) {
                        const uint32_t l = b.cell_out[C];
                        if (l != kNone)
                            pass = triplet_test<F64>(b, p, jq, kq, C, hjq.x, hjq.y, hkq, b.hs[l], a);
                    }
                    const uint32_t pm = __ballot_sync(FULL, pass);
                    const uint32_t idx = run + __popc(pm & lt);
                    if (pass && idx < rw) b.nbr[x0 + rb + idx] = C;
                    run += __popc(pm);
                }
            }
        }
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
        k_connect_front<true><<<grid, 256, 0, s>>>(b, p, total, layer_mask);
    else
        k_connect_front<false><<<grid, 256, 0, s>>>(b, p, total, layer_mask);
}

// ------------------------------------------------------------------------------------------
// Ntuplets: depth-first walk from every root cell
// ------------------------------------------------------------------------------------------
// Depth-first walk from one root cell A; emits every path that has max_hits hits or ends at a
// cell without out-edges, if it has at least min_hits hits.
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
        const uint32_t ne = b.nbr_n[c];
        if (next[d] == 0 && (nh >= p.max_hits || ne == 0)) {
            if (nh >= p.min_hits) {
                const uint32_t slot = atomicAdd(&b.cnt[C_TUPLES * b.E + e], 1u);
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
            const uint32_t nxt = b.nbr[b.nbr_first[c] + next[d]];
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

// Walk from the root cells that have out-edges (listed per event by the CA stage): one thread
// per listed cell.  Enough when paths need at least 3 hits.
__global__ void __launch_bounds__(256) k_walk_roots(DevBatch b, DevParams p, uint32_t total)
{
    const uint32_t n_chunks = total / kChunk;
    for (uint32_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        const uint32_t x = ch * kChunk + threadIdx.x;
        const uint32_t e = b.edge_chunk[ch];
        const uint32_t x0 = b.edge_off[e];
        const uint32_t n = min(b.cnt[C_ROOTS * b.E + e], b.edge_off[e + 1] - x0);
        if (x - x0 < n) walk_from(b, p, e, b.root_list[x], b.root_in[x]);
    }
}

void launch_ntuplets(const DevBatch &b, const DevParams &p, uint32_t edge_total, cudaStream_t s,
                     int sms)
{
    if (p.min_hits > 2) {
        const uint32_t chunks = edge_total / kChunk;
        const uint32_t cap = (uint32_t)sms * p.grid_per_sm[3];
        if (chunks == 0) return;
        k_walk_roots<<<chunks < cap ? chunks : cap, kChunk, 0, s>>>(b, p, edge_total);
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
__global__ void __launch_bounds__(256) k_select(DevBatch b, DevParams p, uint32_t total)
{
    const uint32_t n_chunks = total / kChunk;
    for (uint32_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        const uint32_t t = ch * kChunk + threadIdx.x;
        const uint32_t e = b.tup_chunk[ch];
        const uint32_t t0 = b.tup_off[e];
        const uint32_t nt = min(b.cnt[C_TUPLES * b.E + e], b.tup_off[e + 1] - t0);
        if (t - t0 >= nt) continue;
        bool keep = true;
        if (p.drop_suffixes && b.tup_state[t] == 2) {
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
    uint64_t blocks = total / kChunk;
    uint64_t cap = (uint64_t)sms * 2 * p.grid_per_sm[4];
    if (blocks > cap) blocks = cap;
    if (blocks == 0) return;
    k_select<<<(unsigned)blocks, 256, 0, s>>>(b, p, total);
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

}  // namespace pxr
