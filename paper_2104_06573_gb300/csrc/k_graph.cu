// Doublets, CA cell connection, ntuplet walk and ntuplet selection.
//
// Doublets: one warp per (inner hit, layer pair).  The outer layer's phi window is one or two
// contiguous runs of the sorted hits; the 32 lanes test 32 consecutive candidates per step
// (coalesced float4 loads), a ballot records the passes, one atomic per (hit, pair) reserves the
// cells, and the second sweep writes them from the ballot masks, so the cells of an inner hit are
// contiguous (the CA stage reads them as one run per pair).
//
// CA connect: one thread per cell A = (i, j).  The out-cells (j, k) that can pass the r-z
// alignment cut have k inside a cone of directions around A's direction; a second index of the
// hits (a per-layer grid over the free coordinate and phi) turns that cone into a few grid rows,
// a conservative window in which the exact cuts decide.  Passes are counted first; the cells
// that have any reserve their edge list with one atomic.  Ntuplets: one thread per root cell walks the
// out-edges depth first with an explicit stack.  Selection removes suffix paths and assigns
// output slots.
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

__device__ __forceinline__ bool doublet_test(const DevBatch &b, const DevParams &p, uint32_t g,
                                             float4 hi, uint32_t o)
{
    float4 ho = b.hs[o];
    if (p.cut_mode == CUT_FP32) {
        int r = doublet32(hi, ho, p.cw32);
        if (r >= 0) return r == 1;
    }
    return doublet64((double)hi.x, (double)hi.y, b.r64[g], (double)ho.x, (double)ho.y, b.r64[o],
                     p.cw);
}

__global__ void __launch_bounds__(256) k_doublets(DevBatch b, DevParams p, uint32_t slots)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const uint64_t n_items = (uint64_t)b.N * slots;
    const uint32_t nk = p.n_keys;
    uint64_t item = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t stride = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (; item < n_items; item += stride) {
        const uint32_t g = (uint32_t)(item / slots), slot = (uint32_t)(item % slots);
        const uint32_t e = hit_event(b, g);
        const uint32_t *bk = b.bkt + (size_t)e * (nk + 1);
        if (g >= bk[nk]) continue;                       // hit rejected by the sort (bad layer)
        const uint32_t L = b.hmeta[g] >> kLocalBits;
        if (slot >= p.n_out[L]) continue;
        const uint32_t Lo = p.out_layer[L][slot];
        const float4 hi = b.hs[g];
        const Window w = phi_window(bk, Lo, b.hphi[g], p);
        const uint32_t nc = w.size();

        uint32_t masks[kMaxIt];
        uint32_t count = 0;
#pragma unroll
        for (int k = 0; k < kMaxIt; ++k) {
            masks[k] = 0;
            if ((uint32_t)k * 32u < nc) {
                uint32_t c = (uint32_t)k * 32u + lane;
                bool pass = c < nc && doublet_test(b, p, g, hi, w.pos(c));
                masks[k] = __ballot_sync(0xFFFFFFFFu, pass);
                count += __popc(masks[k]);
            }
        }
        for (uint32_t c0 = kMaxIt * 32u; c0 < nc; c0 += 32u) {
            uint32_t c = c0 + lane;
            bool pass = c < nc && doublet_test(b, p, g, hi, w.pos(c));
            count += __popc(__ballot_sync(0xFFFFFFFFu, pass));
        }

        uint32_t base = 0;
        if (lane == 0 && count) base = atomicAdd(&b.cnt[C_CELLS * b.E + e], count);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        const uint32_t cap = b.cell_off[e + 1] - b.cell_off[e];
        uint32_t nw = count;
        if (base >= cap) nw = 0;
        else if (base + count > cap) nw = cap - base;
        if (lane == 0) {
            if (nw < count) atomicOr(&b.cnt[C_FLAGS * b.E + e], F_CELLS);
            b.out_first[(size_t)g * kMaxOut + slot] = b.cell_off[e] + base;
            b.out_n[(size_t)g * kMaxOut + slot] = nw;
        }
        if (nw == 0) continue;
        const uint32_t first = b.cell_off[e] + base;
        const bool fp64 = p.cut_mode == CUT_FP64;
        const double ri = fp64 ? b.r64[g] : 0.0;
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
                    if (fp64) b.cell_len64[first + idx] =
                        seglen64(ri, (double)hi.z, b.r64[o], (double)b.hs[o].z);
                }
            }
            run += __popc(m);
        }
        for (uint32_t c0 = kMaxIt * 32u; c0 < nc; c0 += 32u) {
            uint32_t c = c0 + lane;
            uint32_t o = c < nc ? w.pos(c) : 0u;
            bool pass = c < nc && doublet_test(b, p, g, hi, o);
            uint32_t m = __ballot_sync(0xFFFFFFFFu, pass);
            if (pass) {
                uint32_t idx = run + __popc(m & lt_mask);
                if (idx < nw) {
                    b.cell_in[first + idx] = g;
                    b.cell_out[first + idx] = o;
                    if (fp64) b.cell_len64[first + idx] =
                        seglen64(ri, (double)hi.z, b.r64[o], (double)b.hs[o].z);
                }
            }
            run += __popc(m);
        }
    }
}

void launch_doublets(const DevBatch &b, const DevParams &p, cudaStream_t s, int sms)
{
    uint32_t slots = 1;
    for (uint32_t l = 0; l < p.n_layers; ++l) slots = p.n_out[l] > slots ? p.n_out[l] : slots;
    uint64_t warps = (uint64_t)b.N * slots;
    uint64_t blocks = (warps + 7) / 8;
    uint64_t cap = (uint64_t)sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) return;
    k_doublets<<<(unsigned)blocks, 256, 0, s>>>(b, p, slots);
}

// ------------------------------------------------------------------------------------------
// CA connect
// ------------------------------------------------------------------------------------------
// Exact decision for the triplet (i, j, k): r-z alignment, then DCA.  FP32 mode decides in float
// when outside the guard band and falls back to the FP64 formulas otherwise.
__device__ __forceinline__ bool triplet_test(const DevBatch &b, const DevParams &p, uint32_t i,
                                             uint32_t j, uint32_t k, float4 hi, float4 hj,
                                             float4 hk, const RZ32 &a, double na64)
{
    bool exact_theta = p.cut_mode == CUT_FP64;
    if (!exact_theta) {
        const RZ32 bs = rz32(hj, hk);
        const int r = theta32(a, bs, p.theta32);
        if (r == 0) return false;
        exact_theta = r < 0;
    }
    if (exact_theta) {
        const double ri = b.r64[i], rj = b.r64[j], rk = b.r64[k];
        const double nA = p.cut_mode == CUT_FP64 ? na64 : seglen64(ri, (double)hi.z, rj, (double)hj.z);
        const double nB = seglen64(rj, (double)hj.z, rk, (double)hk.z);
        if (!theta64(ri, (double)hi.z, rj, (double)hj.z, rk, (double)hk.z, nA, nB, p.theta))
            return false;
    }
    if (p.cut_mode == CUT_FP32) {
        const int r = dca32(hi.x, hi.y, hj.x, hj.y, hk.x, hk.y, p.dca32);
        if (r >= 0) return r == 1;
    }
    return dca64((double)hi.x, (double)hi.y, (double)hj.x, (double)hj.y, (double)hk.x,
                 (double)hk.y) <= p.dca;
}

// Index of the cell (i, j): i's cells toward layer Lj are stored in the candidate order of i's
// phi window (run 1, then run 2), so their outer positions are increasing in that order.
__device__ __forceinline__ uint32_t find_cell(const DevBatch &b, const DevParams &p,
                                              const uint32_t *bk, uint32_t i, float4 hi,
                                              uint32_t slot, uint32_t Lj, uint32_t j)
{
    const Window w = phi_window(bk, Lj, b.hphi[i], p);
    auto rank = [&](uint32_t pos) {
        return (pos >= w.r0 && pos < w.r0 + w.n1) ? pos - w.r0 : w.n1 + (pos - w.r2);
    };
    const uint32_t f = b.out_first[(size_t)i * kMaxOut + slot];
    const uint32_t n = b.out_n[(size_t)i * kMaxOut + slot];
    const uint32_t want = rank(j);
    uint32_t lo = 0, hi_ = n;
    while (lo < hi_) {
        const uint32_t mid = (lo + hi_) >> 1;
        if (rank(b.cell_out[f + mid]) < want) lo = mid + 1; else hi_ = mid;
    }
    if (lo < n && b.cell_out[f + lo] == j) return f + lo;
    return kNone;   // dropped by a cell overflow
}

// Conservative interval of the free coordinate (z on a barrel layer, r on a disk) reachable from
// hit j along r-z directions within asin(theta_cut) of a = (ar, az), modulo pi.  With m the slope
// of a against the layer's fixed coordinate and T = tan(asin(theta_cut)), the allowed slopes are
// [(m - T)/(1 + mT), (m + T)/(1 - mT)] unless the cone contains the direction along the layer
// (then everything is reachable); the offsets along the fixed coordinate span the layer's range.
// Returns false when the whole free range must be scanned.
__device__ __forceinline__ bool cone_window(float ar, float az, float rj, float zj, bool disk,
                                            const float *lr, float T, float &lo, float &hi)
{
    const float u = disk ? az : ar, v = disk ? ar : az;
    const float base = disk ? rj : zj;
    float dlo = disk ? lr[2] - zj : lr[0] - rj;
    float dhi = disk ? lr[3] - zj : lr[1] - rj;
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

// The grid's bin of a free-coordinate value (the same expression the grid was built with).
__device__ __forceinline__ uint32_t free_bin(float v, float lo, float scale, uint32_t nf)
{
    const int b = (int)floorf((v - lo) * scale);
    return (uint32_t)(b < 0 ? 0 : (b >= (int)nf ? (int)nf - 1 : b));
}

// Visit every hit k of the grid rows of layer Lk that the in-cell's cone can reach, inside hit
// j's phi window (coarse grid bins; the doublet cut decides).
template <typename F>
__device__ __forceinline__ void visit_cone(const DevBatch &b, const DevParams &p, uint32_t e,
                                           uint32_t Lk, const RZ32 &a, float4 hj, float phij,
                                           F &&f)
{
    const float *lr = b.lrange + ((size_t)e * p.n_layers + Lk) * kLr;
    const bool disk = p.is_disk[Lk];
    const float flo = disk ? lr[0] : lr[2], fhi = disk ? lr[1] : lr[3];
    if (!(fhi >= flo)) return;                               // no hit on this layer
    float lo = flo, hi = fhi;
    if (cone_window(a.ar, a.az, hj.w, hj.z, disk, lr, p.tan_win, lo, hi)) {
        lo = fmaxf(lo, flo);
        hi = fminf(hi, fhi);
        if (lo > hi) return;
    }
    const uint32_t fb0 = free_bin(lo, lr[4], lr[5], p.nf), fb1 = free_bin(hi, lr[4], lr[5], p.nf);
    const int np2 = (int)p.np2;
    const int pb0 = (int)floorf((phij - p.w_eps + kPiF2) * p.bins2_per_rad);
    const int pb1 = (int)floorf((phij + p.w_eps + kPiF2) * p.bins2_per_rad);
    const uint32_t *b2 = b.bkt2 + (size_t)e * (p.n_keys2 + 1);
    for (uint32_t fb = fb0; fb <= fb1; ++fb) {
        const uint32_t row = (Lk * p.nf + fb) * p.np2;
        uint32_t r[4];
        int nr;
        if (pb1 - pb0 + 1 >= np2) {
            r[0] = row; r[1] = row + np2; nr = 1;
        } else if (pb0 < 0) {
            r[0] = row + pb0 + np2; r[1] = row + np2; r[2] = row; r[3] = row + pb1 + 1; nr = 2;
        } else if (pb1 >= np2) {
            r[0] = row + pb0; r[1] = row + np2; r[2] = row; r[3] = row + pb1 - np2 + 1; nr = 2;
        } else {
            r[0] = row + pb0; r[1] = row + pb1 + 1; nr = 1;
        }
        for (int q = 0; q < nr; ++q)
            for (uint32_t t = b2[r[2 * q]]; t < b2[r[2 * q + 1]]; ++t) f(b.zs[t]);
    }
}

// Grid ranges of one in-cell's cone: for every out-layer slot, the grid rows the cone reaches
// and the one or two phi runs of each row.  Calls f(slot, first, count) for each non-empty range.
template <typename F>
__device__ __forceinline__ void cone_ranges(const DevBatch &b, const DevParams &p, uint32_t e,
                                            uint32_t Lj, const RZ32 &a, float4 hj, float phij,
                                            F &&f)
{
    const uint32_t *b2 = b.bkt2 + (size_t)e * (p.n_keys2 + 1);
    const int np2 = (int)p.np2;
    const int pb0 = (int)floorf((phij - p.w_eps + kPiF2) * p.bins2_per_rad);
    const int pb1 = (int)floorf((phij + p.w_eps + kPiF2) * p.bins2_per_rad);
    for (uint32_t s = 0; s < p.n_out[Lj]; ++s) {
        const uint32_t Lk = p.out_layer[Lj][s];
        const float *lr = b.lrange + ((size_t)e * p.n_layers + Lk) * kLr;
        const bool disk = p.is_disk[Lk];
        const float flo = disk ? lr[0] : lr[2], fhi = disk ? lr[1] : lr[3];
        if (!(fhi >= flo)) continue;                             // no hit on this layer
        float lo = flo, hi = fhi;
        if (cone_window(a.ar, a.az, hj.w, hj.z, disk, lr, p.tan_win, lo, hi)) {
            lo = fmaxf(lo, flo);
            hi = fminf(hi, fhi);
            if (lo > hi) continue;
        }
        const uint32_t fb0 = free_bin(lo, lr[4], lr[5], p.nf), fb1 = free_bin(hi, lr[4], lr[5], p.nf);
        for (uint32_t fb = fb0; fb <= fb1; ++fb) {
            const uint32_t row = (Lk * p.nf + fb) * p.np2;
            uint32_t r[4];
            int nr;
            if (pb1 - pb0 + 1 >= np2) {
                r[0] = row; r[1] = row + np2; nr = 1;
            } else if (pb0 < 0) {
                r[0] = row + pb0 + np2; r[1] = row + np2; r[2] = row; r[3] = row + pb1 + 1; nr = 2;
            } else if (pb1 >= np2) {
                r[0] = row + pb0; r[1] = row + np2; r[2] = row; r[3] = row + pb1 - np2 + 1; nr = 2;
            } else {
                r[0] = row + pb0; r[1] = row + pb1 + 1; nr = 1;
            }
            for (int q = 0; q < nr; ++q) {
                const uint32_t t0 = b2[r[2 * q]], t1 = b2[r[2 * q + 1]];
                if (t1 > t0) f(s, t0, t1 - t0);
            }
        }
    }
}

constexpr int kConnWarps = 8;
constexpr int kMaxR = 6;       // candidate ranges kept per in-cell (more: sequential path)
constexpr int kPass = 96;      // passing triplets kept per warp round (more: sequential path)

// One warp per 32 consecutive cells A = (i, j).  Each lane sets up its cell and collects the
// grid ranges its cone reaches; the warp then tests all lanes' candidates together, 32 at a
// time, so that lanes with many and lanes with no candidates do not diverge.  Passing triplets
// go to a per-warp list; every cell with passes reserves its edge list with one atomic and looks
// up each out-cell's index.  Cells whose cone needs more than kMaxR ranges, or whose passes do
// not fit the list, take the sequential path.
__global__ void __launch_bounds__(256, 2) k_connect(DevBatch b, DevParams p, uint32_t total)
{
    struct Lane {
        float4 hi, hj;
        RZ32 a;
        double na64;
        uint32_t i, j, pre, cnt, nr, npass;
        uint32_t rs[kMaxR], rn[kMaxR];
        uint8_t rslot[kMaxR];
        uint8_t seq;
    };
    __shared__ Lane s_lane[kConnWarps][32];
    __shared__ uint32_t s_pk[kConnWarps][kPass];
    __shared__ uint8_t s_pown[kConnWarps][kPass], s_pslot[kConnWarps][kPass];
    __shared__ uint32_t s_np[kConnWarps];
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    Lane *L = s_lane[wid];
    Lane &me = L[lane];
    const uint32_t n_chunks = total / kChunk;
    for (uint32_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        const uint32_t A = ch * kChunk + threadIdx.x;
        const uint32_t e = b.cell_chunk[ch];
        const uint32_t c0 = b.cell_off[e];
        const uint32_t ncell = min(b.cnt[C_CELLS * b.E + e], b.cell_off[e + 1] - c0);
        // ---- per-lane set-up -----------------------------------------------------------------
        me.cnt = 0;
        me.nr = 0;
        me.npass = 0;
        me.seq = 0;
        uint32_t Lj = 0;
        bool valid = A - c0 < ncell;
        if (valid) {
            me.j = b.cell_out[A];
            Lj = b.hmeta[me.j] >> kLocalBits;
            valid = p.n_out[Lj] != 0;
        }
        if (valid) {
            me.i = b.cell_in[A];
            me.hi = b.hs[me.i];
            me.hj = b.hs[me.j];
            me.a = rz32(me.hi, me.hj);
            me.na64 = p.cut_mode == CUT_FP64 ? b.cell_len64[A] : 0.0;
            cone_ranges(b, p, e, Lj, me.a, me.hj, b.hphi[me.j],
                        [&](uint32_t s, uint32_t t0, uint32_t n) {
                            if (me.nr < (uint32_t)kMaxR) {
                                me.rs[me.nr] = t0;
                                me.rn[me.nr] = n;
                                me.rslot[me.nr] = (uint8_t)s;
                                ++me.nr;
                                me.cnt += n;
                            } else {
                                me.seq = 1;
                            }
                        });
            if (me.seq) me.cnt = 0;
        }
        // ---- flatten the candidates of the warp --------------------------------------------
        uint32_t incl = me.cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= (uint32_t)o) incl += t;
        }
        me.pre = incl - me.cnt;
        const uint32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
        if (lane == 0) s_np[wid] = 0;
        __syncwarp();
        for (uint32_t base = 0; base < tot; base += 32) {
            const uint32_t t = base + lane;
            if (t < tot) {
                uint32_t lo = 0, hi_ = 31;                      // last lane with pre <= t
                while (lo < hi_) {
                    const uint32_t mid = (lo + hi_ + 1) >> 1;
                    if (L[mid].pre <= t) lo = mid; else hi_ = mid - 1;
                }
                const Lane &ow = L[lo];
                uint32_t loc = t - ow.pre, r = 0;
                while (loc >= ow.rn[r]) { loc -= ow.rn[r]; ++r; }
                const uint32_t k = b.zs[ow.rs[r] + loc];
                const float4 hk = b.hs[k];
                if (doublet_test(b, p, ow.j, ow.hj, k) &&
                    triplet_test(b, p, ow.i, ow.j, k, ow.hi, ow.hj, hk, ow.a, ow.na64)) {
                    const uint32_t q = atomicAdd(&s_np[wid], 1u);
                    if (q < (uint32_t)kPass) {
                        s_pk[wid][q] = k;
                        s_pown[wid][q] = (uint8_t)lo;
                        s_pslot[wid][q] = ow.rslot[r];
                        atomicAdd(&L[lo].npass, 1u);
                    } else {
                        L[lo].seq = 1;                          // list full: redo this cell alone
                    }
                }
            }
        }
        __syncwarp();
        // ---- edges -------------------------------------------------------------------------
        if (!valid) continue;
        const uint32_t *bk = b.bkt + (size_t)e * (p.n_keys + 1);
        const uint32_t np = min(s_np[wid], (uint32_t)kPass);
        const uint32_t i = me.i, j = me.j;
        auto pass = [&](uint32_t k) {
            return doublet_test(b, p, j, me.hj, k) &&
                   triplet_test(b, p, i, j, k, me.hi, me.hj, b.hs[k], me.a, me.na64);
        };
        if (me.seq) {
            // sequential path: count, then write
            uint32_t npass = 0;
            for (uint32_t s = 0; s < p.n_out[Lj]; ++s)
                visit_cone(b, p, e, p.out_layer[Lj][s], me.a, me.hj, b.hphi[j],
                           [&](uint32_t k) { npass += pass(k); });
            if (!npass) continue;
            const uint32_t base = atomicAdd(&b.cnt[C_EDGES * b.E + e], npass);
            const uint32_t cap = b.edge_off[e + 1] - b.edge_off[e];
            const uint32_t nw = base >= cap ? 0u : min(npass, cap - base);
            if (nw < npass) atomicOr(&b.cnt[C_FLAGS * b.E + e], F_EDGES);
            const uint32_t first = b.edge_off[e] + base;
            uint32_t written = 0;
            for (uint32_t s = 0; s < p.n_out[Lj]; ++s) {
                const uint32_t Lk = p.out_layer[Lj][s];
                visit_cone(b, p, e, Lk, me.a, me.hj, b.hphi[j], [&](uint32_t k) {
                    if (written < nw && pass(k)) {
                        const uint32_t B = find_cell(b, p, bk, j, me.hj, s, Lk, k);
                        if (B != kNone) b.nbr[first + written++] = B;
                    }
                });
            }
            b.nbr_first[A] = first;
            b.nbr_n[A] = written;
            continue;
        }
        const uint32_t npass = me.npass;
        if (!npass) continue;
        const uint32_t base = atomicAdd(&b.cnt[C_EDGES * b.E + e], npass);
        const uint32_t cap = b.edge_off[e + 1] - b.edge_off[e];
        const uint32_t nw = base >= cap ? 0u : min(npass, cap - base);
        if (nw < npass) atomicOr(&b.cnt[C_FLAGS * b.E + e], F_EDGES);
        const uint32_t first = b.edge_off[e] + base;
        uint32_t written = 0;
        for (uint32_t q = 0; q < np && written < nw; ++q) {
            if (s_pown[wid][q] != lane) continue;
            const uint32_t s = s_pslot[wid][q];
            const uint32_t B = find_cell(b, p, bk, j, me.hj, s, p.out_layer[Lj][s], s_pk[wid][q]);
            if (B != kNone) b.nbr[first + written++] = B;
        }
        b.nbr_first[A] = first;
        b.nbr_n[A] = written;
    }
}

void launch_connect(const DevBatch &b, const DevParams &p, uint32_t total, cudaStream_t s, int sms)
{
    uint64_t blocks = total / kChunk;
    uint64_t cap = (uint64_t)sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) return;
    k_connect<<<(unsigned)blocks, kConnWarps * 32, 0, s>>>(b, p, total);
}

// ------------------------------------------------------------------------------------------
// Ntuplets: depth-first walk from every root cell
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_ntuplets(DevBatch b, DevParams p, uint32_t total)
{
    const uint32_t n_chunks = total / kChunk;
    for (uint32_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        const uint32_t A = ch * kChunk + threadIdx.x;
        const uint32_t e = b.cell_chunk[ch];
        const uint32_t c0 = b.cell_off[e];
        const uint32_t ncell = min(b.cnt[C_CELLS * b.E + e], b.cell_off[e + 1] - c0);
        if (A - c0 >= ncell) continue;
        const uint32_t Li = b.hmeta[b.cell_in[A]] >> kLocalBits;
        if (!((p.root_mask >> Li) & 1u)) continue;
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
                    uint32_t slot = atomicAdd(&b.cnt[C_TUPLES * b.E + e], 1u);
                    if (slot < tcap) {
                        const uint32_t t = b.tup_off[e] + slot;
                        uint32_t *th = b.tup_hits + (size_t)t * kMaxHits;
                        th[0] = b.cell_in[cells[0]];
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
}

void launch_ntuplets(const DevBatch &b, const DevParams &p, uint32_t total, cudaStream_t s, int sms)
{
    uint64_t blocks = total / kChunk;
    uint64_t cap = (uint64_t)sms * 32;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) return;
    k_ntuplets<<<(unsigned)blocks, 256, 0, s>>>(b, p, total);
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
        b.tup_rank[t] = keep ? atomicAdd(&b.cnt[C_OUT * b.E + e], 1u) : kNone;
    }
}

void launch_select(const DevBatch &b, const DevParams &p, uint32_t total, cudaStream_t s, int sms)
{
    uint64_t blocks = total / kChunk;
    uint64_t cap = (uint64_t)sms * 16;
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
