// Doublets, CA cell connection, ntuplet walk and ntuplet selection.
//
// Doublets: one warp per (inner hit, layer pair).  The outer layer's phi window is one or two
// contiguous runs of the sorted hits; the 32 lanes test 32 consecutive candidates per step
// (coalesced float4 loads), a ballot records the passes, one atomic per (hit, pair) reserves the
// cells, and the second sweep writes them from the ballot masks, so the cells of an inner hit are
// contiguous (the CA stage reads them as one run per pair).
//
// CA connect: one warp per junction hit j.  j's out-cells (j, k) are staged in shared memory and
// bucketed by the free coordinate of k (z on barrel layers, r on disks); each in-cell (i, j) tests
// only the buckets reached by the cone of r-z directions within asin(theta_cut) of its own, a
// conservative window in which the exact cuts decide.  Passes are counted first; in-cells with
// passes reserve their edge list with one atomic.  Ntuplets: one thread per root cell walks the
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
constexpr int kPass = 64;       // passing triplets collected per round of 32 in-cells

// Order-preserving int encoding of floats (for warp min / max reductions).
__device__ __forceinline__ int ford(float f)
{
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float funord(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF); }

// Append n out-edges of cell A (its list may already hold edges from an earlier out-layer slot).
template <typename G>
__device__ __forceinline__ void append_edges(const DevBatch &b, uint32_t e, uint32_t A, bool first_slot,
                                             uint32_t n, G &&get)
{
    const uint32_t have = first_slot ? 0u : b.nbr_n[A];
    const uint32_t old = b.nbr_first[A];
    const uint32_t need = have + n;
    const uint32_t base = atomicAdd(&b.cnt[C_EDGES * b.E + e], need);
    const uint32_t cap = b.edge_off[e + 1] - b.edge_off[e];
    const uint32_t nw = base >= cap ? 0u : min(need, cap - base);
    if (nw < need) atomicOr(&b.cnt[C_FLAGS * b.E + e], F_EDGES);
    const uint32_t first = b.edge_off[e] + base;
    uint32_t w = 0;
    for (uint32_t t = 0; t < have && w < nw; ++t) b.nbr[first + w++] = b.nbr[old + t];
    for (uint32_t t = 0; t < n && w < nw; ++t) b.nbr[first + w++] = get(t);
    b.nbr_first[A] = first;
    b.nbr_n[A] = w;
}

// One warp per junction hit j.  For each out-layer slot, j's out-cells (j, k) are staged in
// shared memory and bucketed by the free coordinate of k (z on barrel layers, r on disks) over
// the staged range.  The in-cells (i, j) are found 32 at a time by scanning i over j's phi window
// on the inner layer with the doublet cut; each computes the cone of r-z directions that can pass
// the alignment cut and the buckets it reaches (a conservative window: the exact cuts decide).
// The warp then tests all 32 in-cells' candidates together, 32 at a time, collecting passes in a
// shared list; each in-cell with passes finds its own index and appends its edge list.  A slot
// with more than kStage out-cells is tested against all of them from global memory; an in-cell
// whose passes overflow the list is redone alone.
__global__ void __launch_bounds__(kConnWarps * 32, 4) k_connect(DevBatch b, DevParams p)
{
    // per-warp staging and per-lane in-cell records (structure of arrays: lanes reading other
    // lanes' records hit distinct banks)
    __shared__ uint32_t s_B[kConnWarps][kStage], s_k[kConnWarps][kStage];
    __shared__ float s_f[kConnWarps][kStage];
    __shared__ uint32_t s_bin[kConnWarps][kBins];
    __shared__ float4 s_hi[kConnWarps][32], s_a[kConnWarps][32];
    __shared__ double s_na[kConnWarps][32];
    __shared__ uint32_t s_i[kConnWarps][32], s_q0[kConnWarps][32], s_pre[kConnWarps][32],
        s_npass[kConnWarps][32], s_seq[kConnWarps][32];
    __shared__ uint32_t s_pB[kConnWarps][kPass];
    __shared__ uint8_t s_pown[kConnWarps][kPass];
    __shared__ uint32_t s_np[kConnWarps];
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    uint32_t *sB = s_B[wid], *sK = s_k[wid], *bin = s_bin[wid];
    float *sF = s_f[wid];
    float4 *Hi = s_hi[wid], *Aa = s_a[wid];
    double *Na = s_na[wid];
    uint32_t *Ii = s_i[wid], *Q0 = s_q0[wid], *Pre = s_pre[wid], *Np = s_npass[wid],
             *Seq = s_seq[wid];
    const uint32_t nk = p.n_keys;
    const uint64_t stride = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t jj = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; jj < b.N;
         jj += stride) {
        const uint32_t j = (uint32_t)jj;
        const uint32_t e = hit_event(b, j);
        const uint32_t *bk = b.bkt + (size_t)e * (nk + 1);
        if (j >= bk[nk]) continue;
        const uint32_t Lj = b.hmeta[j] >> kLocalBits;
        const uint32_t nin = p.n_in[Lj], nout = p.n_out[Lj];
        if (nin == 0 || nout == 0) continue;
        const float4 hj = b.hs[j];
        const float phij = b.hphi[j];
        for (uint32_t s = 0; s < nout; ++s) {
            const uint32_t Lk = p.out_layer[Lj][s];
            const bool disk = p.is_disk[Lk];
            const uint32_t f0 = b.out_first[(size_t)j * kMaxOut + s];
            const uint32_t nB = b.out_n[(size_t)j * kMaxOut + s];
            if (nB == 0) continue;
            const bool staged = nB <= (uint32_t)kStage;
            float flo = 0.f, fhi = 0.f, dlo = 0.f, dhi = 0.f, scale = 0.f;
            if (staged) {
                // stage the out-cells: free coordinate and the ranges of both coordinates
                int m0 = ford(3.0e38f), m1 = ford(-3.0e38f), m2 = m0, m3 = m1;
                for (uint32_t t = lane; t < nB; t += 32) {
                    const uint32_t k = b.cell_out[f0 + t];
                    const float4 hk = b.hs[k];
                    const float fc = disk ? hk.w : hk.z, xc = disk ? hk.z : hk.w;
                    sK[t] = k;
                    sF[t] = fc;
                    m0 = min(m0, ford(fc));
                    m1 = max(m1, ford(fc));
                    m2 = min(m2, ford(xc));
                    m3 = max(m3, ford(xc));
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
                // counting sort by local bin: histogram, warp scan, scatter
                for (uint32_t t = lane; t < (uint32_t)kBins; t += 32) bin[t] = 0;
                __syncwarp();
                uint32_t mybin[kStage / 32], myk[kStage / 32];
#pragma unroll
                for (int q = 0; q < kStage / 32; ++q) {
                    const uint32_t t = lane + 32u * q;
                    if (t < nB) {
                        int bb = (int)floorf((sF[t] - flo) * scale);
                        bb = bb < 0 ? 0 : (bb >= kBins ? kBins - 1 : bb);
                        mybin[q] = (uint32_t)bb;
                        myk[q] = sK[t];
                        atomicAdd(&bin[bb], 1u);
                    }
                }
                __syncwarp();
                {
                    // exclusive scan of the kBins counts: kBins / 32 consecutive bins per lane
                    constexpr int per = kBins / 32;
                    uint32_t v[per], sum = 0;
#pragma unroll
                    for (int q = 0; q < per; ++q) { v[q] = bin[lane * per + q]; sum += v[q]; }
                    uint32_t incl = sum;
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
#pragma unroll
                for (int q = 0; q < kStage / 32; ++q) {
                    const uint32_t t = lane + 32u * q;
                    if (t < nB) {
                        const uint32_t pos = atomicAdd(&bin[mybin[q]], 1u);
                        sB[pos] = f0 + t;
                        sK[pos] = myk[q];
                    }
                }
                __syncwarp();
                // bin[t] is now the end of bin t; the start of bin t is bin[t - 1] (0 for t = 0)
            }
            for (uint32_t si = 0; si < nin; ++si) {
                const uint32_t Li = p.in_layer[Lj][si];
                const uint32_t slot_i = p.in_slot[Lj][si];
                const Window w = phi_window(bk, Li, phij, p);
                const uint32_t nc = w.size();
                for (uint32_t c0 = 0; c0 < nc; c0 += 32) {
                    // ---- set-up of one in-cell per lane ----
                    const uint32_t c = c0 + lane;
                    uint32_t q0 = 0, q1 = 0, my_i = 0;
                    float4 my_hi = make_float4(0.f, 0.f, 0.f, 0.f);
                    RZ32 my_a{0.f, 0.f, 0.f, 0.f};
                    double my_na = 0.0;
                    Np[lane] = 0;
                    Seq[lane] = 0;
                    bool valid = c < nc;
                    if (valid) {
                        my_i = w.pos(c);
                        my_hi = b.hs[my_i];
                        valid = doublet_test(b, p, my_i, my_hi, j);
                        if (valid) {
                            my_a = rz32(my_hi, hj);
                            my_na = p.cut_mode == CUT_FP64
                                        ? seglen64(b.r64[my_i], (double)my_hi.z, b.r64[j], (double)hj.z)
                                        : 0.0;
                            Ii[lane] = my_i;
                            Hi[lane] = my_hi;
                            Aa[lane] = make_float4(my_a.ar, my_a.az, my_a.na, my_a.Ea);
                            Na[lane] = my_na;
                            q1 = nB;
                            float lo, hi_;
                            if (staged && cone_window(my_a.ar, my_a.az, disk ? hj.w : hj.z, dlo,
                                                      dhi, disk, p.tan_win, lo, hi_)) {
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
                    const uint32_t cnt = q1 - q0;
                    Q0[lane] = q0;
                    uint32_t incl = cnt;
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                        if (lane >= (uint32_t)o) incl += t;
                    }
                    Pre[lane] = incl - cnt;
                    const uint32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
                    if (lane == 0) s_np[wid] = 0;
                    __syncwarp();
                    // ---- the warp tests all candidates, 32 at a time ----
                    for (uint32_t t0 = 0; t0 < tot; t0 += 32) {
                        const uint32_t t = t0 + lane;
                        if (t >= tot) continue;
                        uint32_t lo = 0, hi_ = 31;              // last lane with pre <= t
                        while (lo < hi_) {
                            const uint32_t mid = (lo + hi_ + 1) >> 1;
                            if (Pre[mid] <= t) lo = mid; else hi_ = mid - 1;
                        }
                        const uint32_t q = Q0[lo] + (t - Pre[lo]);
                        uint32_t B, k;
                        if (staged) { B = sB[q]; k = sK[q]; }
                        else { B = f0 + q; k = b.cell_out[B]; }
                        const float4 av = Aa[lo];
                        const RZ32 oa{av.x, av.y, av.z, av.w};
                        if (triplet_test(b, p, Ii[lo], j, k, Hi[lo], hj, b.hs[k], oa, Na[lo])) {
                            const uint32_t slot = atomicAdd(&s_np[wid], 1u);
                            if (slot < (uint32_t)kPass) {
                                s_pB[wid][slot] = B;
                                s_pown[wid][slot] = (uint8_t)lo;
                                atomicAdd(&Np[lo], 1u);
                            } else {
                                Seq[lo] = 1;
                            }
                        }
                    }
                    __syncwarp();
                    // ---- in-cells with passes write their edges ----
                    const uint32_t my_np = Np[lane];
                    if (valid && (my_np || Seq[lane])) {
                        const uint32_t A = find_cell(b, p, bk, my_i, my_hi, slot_i, Lj, j);
                        if (A != kNone) {
                            if (Seq[lane]) {
                                uint32_t n = 0;
                                for (uint32_t q = q0; q < q1; ++q) {
                                    const uint32_t B = staged ? sB[q] : f0 + q;
                                    const uint32_t k = staged ? sK[q] : b.cell_out[B];
                                    n += triplet_test(b, p, my_i, j, k, my_hi, hj, b.hs[k], my_a, my_na);
                                }
                                uint32_t q = q0;
                                append_edges(b, e, A, s == 0, n, [&](uint32_t) {
                                    for (;; ++q) {
                                        const uint32_t B = staged ? sB[q] : f0 + q;
                                        const uint32_t k = staged ? sK[q] : b.cell_out[B];
                                        if (triplet_test(b, p, my_i, j, k, my_hi, hj, b.hs[k], my_a, my_na)) {
                                            ++q;
                                            return B;
                                        }
                                    }
                                });
                            } else {
                                uint32_t q = 0;
                                append_edges(b, e, A, s == 0, my_np, [&](uint32_t) {
                                    while (s_pown[wid][q] != lane) ++q;
                                    return s_pB[wid][q++];
                                });
                            }
                        }
                    }
                    __syncwarp();
                }
            }
            __syncwarp();
        }
    }
}

void launch_connect(const DevBatch &b, const DevParams &p, uint32_t total, cudaStream_t s, int sms)
{
    (void)total;
    uint64_t blocks = ((uint64_t)b.N + kConnWarps - 1) / kConnWarps;
    uint64_t cap = (uint64_t)sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) return;
    k_connect<<<(unsigned)blocks, kConnWarps * 32, 0, s>>>(b, p);
}

// ------------------------------------------------------------------------------------------
// Ntuplets: depth-first walk from every root cell
// ------------------------------------------------------------------------------------------
// Depth-first walk from one root cell A; emits every path that has max_hits hits or ends at a
// cell without out-edges, if it has at least min_hits hits.
__device__ __forceinline__ void walk_from(const DevBatch &b, const DevParams &p, uint32_t e,
                                          uint32_t A)
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

// One warp per root hit (a hit on a root layer); its lanes walk from the hit's cells.
__global__ void __launch_bounds__(256) k_ntuplets(DevBatch b, DevParams p)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nk = p.n_keys;
    const uint64_t stride = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t gg = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gg < b.N;
         gg += stride) {
        const uint32_t g = (uint32_t)gg;
        const uint32_t e = hit_event(b, g);
        if (g >= b.bkt[(size_t)e * (nk + 1) + nk]) continue;
        const uint32_t L = b.hmeta[g] >> kLocalBits;
        if (!((p.root_mask >> L) & 1u)) continue;
        for (uint32_t s = 0; s < p.n_out[L]; ++s) {
            const uint32_t f = b.out_first[(size_t)g * kMaxOut + s];
            const uint32_t n = b.out_n[(size_t)g * kMaxOut + s];
            for (uint32_t c = lane; c < n; c += 32) {
                const uint32_t A = f + c;
                if (b.nbr_n[A] == 0 && p.min_hits > 2) continue;   // a 2-hit path is too short
                walk_from(b, p, e, A);
            }
        }
    }
}

void launch_ntuplets(const DevBatch &b, const DevParams &p, uint32_t total, cudaStream_t s, int sms)
{
    (void)total;
    uint64_t blocks = ((uint64_t)b.N + 7) / 8;
    uint64_t cap = (uint64_t)sms * 16;
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
