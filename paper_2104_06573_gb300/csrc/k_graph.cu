// Doublets, CA cell connection, ntuplet walk and ntuplet selection.
//
// Doublets: one warp per (inner hit, layer pair).  The outer layer's phi window is one or two
// contiguous runs of the sorted hits; the 32 lanes test 32 consecutive candidates per step
// (coalesced float4 loads), a ballot records the passes, one atomic per (hit, pair) reserves the
// cells, and the second sweep writes them from the ballot masks, so the cells of an inner hit are
// contiguous (the CA stage reads them as one run per pair).
//
// CA connect: one warp per junction hit j.  Its out-cells (j, k) are staged in shared memory and
// sorted by the direction of (k - j) in the r-z plane; each in-cell (i, j) tests only the
// out-cells whose direction lies within asin(theta_cut) of its own (modulo pi), a conservative
// window in which the exact cuts decide.  Passes are counted first; the cells that have any
// reserve their edge list with one atomic.  Ntuplets: one thread per root cell walks the
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
        const uint32_t e = find_event(b.hit_off, b.E, g);
        const uint32_t *bk = b.bkt + (size_t)e * (nk + 1);
        if (g >= bk[nk]) continue;                       // hit rejected by the sort (bad layer)
        const uint32_t L = b.hmeta[g] >> kLocalBits;
        if (slot >= p.n_out[L]) continue;
        const uint32_t Lo = p.out_layer[L][slot];
        const float4 hi = b.hs[g];
        const Window w = phi_window(bk, Lo, atan2f(hi.y, hi.x), p);
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
__device__ __forceinline__ bool triplet_test(const DevBatch &b, const DevParams &p, uint32_t i,
                                             uint32_t j, uint32_t k, float4 hi, float4 hj,
                                             const RZ32 &a, double na64, uint32_t A, uint32_t B)
{
    const float4 hk = b.hs[k];
    bool exact_theta = p.cut_mode == CUT_FP64;
    if (!exact_theta) {
        RZ32 bs = rz32(hj, hk);
        int r = theta32(a, bs, p.theta32);
        if (r == 0) return false;
        exact_theta = r < 0;
    }
    if (exact_theta) {
        double ri = b.r64[i], rj = b.r64[j], rk = b.r64[k];
        double nA = p.cut_mode == CUT_FP64 ? na64 : seglen64(ri, (double)hi.z, rj, (double)hj.z);
        double nB = p.cut_mode == CUT_FP64 ? b.cell_len64[B]
                                           : seglen64(rj, (double)hj.z, rk, (double)hk.z);
        if (!theta64(ri, (double)hi.z, rj, (double)hj.z, rk, (double)hk.z, nA, nB, p.theta))
            return false;
    }
    if (p.cut_mode == CUT_FP32) {
        int r = dca32(hi.x, hi.y, hj.x, hj.y, hk.x, hk.y, p.dca32);
        if (r >= 0) return r == 1;
    }
    return dca64((double)hi.x, (double)hi.y, (double)hj.x, (double)hj.y, (double)hk.x,
                 (double)hk.y) <= p.dca;
}

// Direction key of an r-z segment folded modulo pi: 1 - dr / (|dr| + dz) after turning the
// segment into the upper half plane.  It increases with the direction angle on [0, pi), and its
// derivative with respect to the angle lies in [1/2, 1], so two directions whose angles differ by
// d (modulo pi) have keys that differ by at most d (modulo 2).  Zero-length segments get -1.
__device__ __forceinline__ float dir_key(float dr, float dz)
{
    if (dz < 0.f || (dz == 0.f && dr < 0.f)) {
        dr = -dr;
        dz = -dz;
    }
    const float s = fabsf(dr) + dz;
    return s > 0.f ? 1.f - __fdiv_rn(dr, s) : -1.f;
}

constexpr int kStage = 256;      // out-cells of one junction hit sorted in shared memory
constexpr float kKeyPad = 3.0e38f;

// Bitonic sort of n (power of two) entries by key, one warp.
__device__ __forceinline__ void warp_bitonic(float *key, uint32_t *v1, uint32_t *v2, uint32_t n,
                                             uint32_t lane)
{
    for (uint32_t k = 2; k <= n; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = lane; i < n; i += 32) {
                const uint32_t ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const float a = key[i], c = key[ixj];
                    if ((a > c) == up) {
                        key[i] = c;
                        key[ixj] = a;
                        uint32_t t = v1[i]; v1[i] = v1[ixj]; v1[ixj] = t;
                        t = v2[i]; v2[i] = v2[ixj]; v2[ixj] = t;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// First index in [lo, hi) whose key is >= v (strict: > v).
__device__ __forceinline__ uint32_t key_bound(const float *key, uint32_t lo, uint32_t hi, float v,
                                              bool strict)
{
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const bool left = strict ? key[mid] <= v : key[mid] < v;
        if (left) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Index of the cell (i, j): i's cells toward layer Lj are stored in the candidate order of i's
// phi window (run 1, then run 2), so their outer positions are increasing in that order.
__device__ __forceinline__ uint32_t find_cell(const DevBatch &b, const DevParams &p,
                                              const uint32_t *bk, uint32_t i, float4 hi,
                                              uint32_t slot, uint32_t Lj, uint32_t j)
{
    const Window w = phi_window(bk, Lj, atan2f(hi.y, hi.x), p);
    auto rank = [&](uint32_t pos) {
        return (pos >= w.r0 && pos < w.r0 + w.n1) ? pos - w.r0 : w.n1 + (pos - w.r2);
    };
    const uint32_t f = b.out_first[(size_t)i * kMaxOut + slot];
    uint32_t lo = 0, hi_ = b.out_n[(size_t)i * kMaxOut + slot];
    const uint32_t want = rank(j);
    while (lo < hi_) {
        const uint32_t mid = (lo + hi_) >> 1;
        const uint32_t r = rank(b.cell_out[f + mid]);
        if (r < want) lo = mid + 1; else hi_ = mid;
    }
    if (lo < b.out_n[(size_t)i * kMaxOut + slot] && b.cell_out[f + lo] == j) return f + lo;
    return kNone;   // dropped by a cell overflow
}

// Candidate out-cells of one in-cell: up to three ranges of the sorted stage.
struct Ranges {
    uint32_t a0, a1, b0, b1, c0, c1;
};

__device__ __forceinline__ Ranges key_ranges(const float *key, uint32_t nzero, uint32_t cnt,
                                             float kA, float hw)
{
    Ranges r{0, nzero, 0, 0, 0, 0};              // zero-length out-cells always
    if (kA < 0.f || hw >= 1.f) {
        r.b0 = nzero;
        r.b1 = cnt;
        return r;
    }
    const float lo = kA - hw, hi = kA + hw;
    if (lo < 0.f) {
        r.b0 = key_bound(key, nzero, cnt, lo + 2.f, false);
        r.b1 = cnt;
        r.c0 = nzero;
        r.c1 = key_bound(key, nzero, cnt, hi, true);
    } else if (hi >= 2.f) {
        r.b0 = key_bound(key, nzero, cnt, lo, false);
        r.b1 = cnt;
        r.c0 = nzero;
        r.c1 = key_bound(key, nzero, cnt, hi - 2.f, true);
    } else {
        r.b0 = key_bound(key, nzero, cnt, lo, false);
        r.b1 = key_bound(key, nzero, cnt, hi, true);
    }
    return r;
}

// Write the out-edges of cell A (npass of them) after one atomic reservation.
template <typename Visit>
__device__ __forceinline__ void emit_edges(const DevBatch &b, uint32_t e, uint32_t A,
                                           uint32_t npass, Visit &&visit)
{
    const uint32_t base = atomicAdd(&b.cnt[C_EDGES * b.E + e], npass);
    const uint32_t cap = b.edge_off[e + 1] - b.edge_off[e];
    const uint32_t nw = base >= cap ? 0u : min(npass, cap - base);
    if (nw < npass) atomicOr(&b.cnt[C_FLAGS * b.E + e], F_EDGES);
    const uint32_t first = b.edge_off[e] + base;
    uint32_t written = 0;
    visit([&](uint32_t B) {
        if (written < nw) b.nbr[first + written++] = B;
    });
    b.nbr_first[A] = first;
    b.nbr_n[A] = written;
}

// One warp per junction hit j: its out-cells (j, k) are staged in shared memory sorted by the
// direction key of (k - j) in r-z; each in-cell (i, j), found by scanning i over j's phi window
// on the inner layer with the doublet cut, tests only the out-cells inside its key window.
__global__ void __launch_bounds__(256) k_connect(DevBatch b, DevParams p)
{
    __shared__ float s_key[8][kStage];
    __shared__ uint32_t s_B[8][kStage];
    __shared__ uint32_t s_k[8][kStage];
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    float *key = s_key[wid];
    uint32_t *sB = s_B[wid], *sK = s_k[wid];
    const uint32_t nk = p.n_keys;
    const uint64_t stride = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t jj = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; jj < b.N;
         jj += stride) {
        const uint32_t j = (uint32_t)jj;
        const uint32_t e = find_event(b.hit_off, b.E, j);
        const uint32_t *bk = b.bkt + (size_t)e * (nk + 1);
        if (j >= bk[nk]) continue;
        const uint32_t Lj = b.hmeta[j] >> kLocalBits;
        const uint32_t nin = p.n_in[Lj], nout = p.n_out[Lj];
        if (nin == 0 || nout == 0) continue;
        uint32_t sf[kMaxOut], sn[kMaxOut], nB = 0;
        for (uint32_t s = 0; s < kMaxOut; ++s) {
            sf[s] = s < nout ? b.out_first[(size_t)j * kMaxOut + s] : 0u;
            sn[s] = s < nout ? b.out_n[(size_t)j * kMaxOut + s] : 0u;
            nB += sn[s];
        }
        if (nB == 0) continue;
        const float4 hj = b.hs[j];
        const float phij = atan2f(hj.y, hj.x);
        const bool staged = nB <= (uint32_t)kStage;
        uint32_t n = 32, nzero = 0;
        if (staged) {
            while (n < nB) n <<= 1;
            for (uint32_t t = lane; t < n; t += 32) {
                if (t < nB) {
                    uint32_t q = t, s = 0;
                    while (q >= sn[s]) { q -= sn[s]; ++s; }
                    const uint32_t B = sf[s] + q;
                    const uint32_t k = b.cell_out[B];
                    const float4 hk = b.hs[k];
                    key[t] = dir_key(__fsub_rn(hk.w, hj.w), __fsub_rn(hk.z, hj.z));
                    sB[t] = B;
                    sK[t] = k;
                } else {
                    key[t] = kKeyPad;
                    sB[t] = kNone;
                    sK[t] = 0;
                }
            }
            __syncwarp();
            warp_bitonic(key, sB, sK, n, lane);
            nzero = key_bound(key, 0, nB, -0.5f, false);
        }
        for (uint32_t si = 0; si < nin; ++si) {
            const uint32_t Li = p.in_layer[Lj][si];
            const uint32_t slot_i = p.in_slot[Lj][si];
            const Window w = phi_window(bk, Li, phij, p);
            const uint32_t nc = w.size();
            for (uint32_t c0 = 0; c0 < nc; c0 += 32) {
                const uint32_t c = c0 + lane;
                if (c >= nc) continue;
                const uint32_t i = w.pos(c);
                const float4 hi = b.hs[i];
                if (!doublet_test(b, p, i, hi, j)) continue;
                const RZ32 a = rz32(hi, hj);
                const double na64 = p.cut_mode == CUT_FP64
                                        ? seglen64(b.r64[i], (double)hi.z, b.r64[j], (double)hj.z)
                                        : 0.0;
                if (staged) {
                    const float kA = dir_key(__fsub_rn(hj.w, hi.w), __fsub_rn(hj.z, hi.z));
                    const Ranges R = key_ranges(key, nzero, nB, kA, p.key_halfwin);
                    auto each = [&](auto &&f) {
                        for (uint32_t q = R.a0; q < R.a1; ++q) f(q);
                        for (uint32_t q = R.b0; q < R.b1; ++q) f(q);
                        for (uint32_t q = R.c0; q < R.c1; ++q) f(q);
                    };
                    uint32_t npass = 0;
                    each([&](uint32_t q) {
                        npass += triplet_test(b, p, i, j, sK[q], hi, hj, a, na64, 0, sB[q]);
                    });
                    if (!npass) continue;
                    const uint32_t A = find_cell(b, p, bk, i, hi, slot_i, Lj, j);
                    if (A == kNone) continue;
                    emit_edges(b, e, A, npass, [&](auto &&put) {
                        each([&](uint32_t q) {
                            if (triplet_test(b, p, i, j, sK[q], hi, hj, a, na64, A, sB[q]))
                                put(sB[q]);
                        });
                    });
                } else {
                    // more out-cells than the stage holds: test them all from global memory
                    auto each = [&](auto &&f) {
                        for (uint32_t s = 0; s < nout; ++s)
                            for (uint32_t B = sf[s]; B < sf[s] + sn[s]; ++B) f(B);
                    };
                    uint32_t npass = 0;
                    each([&](uint32_t B) {
                        npass += triplet_test(b, p, i, j, b.cell_out[B], hi, hj, a, na64, 0, B);
                    });
                    if (!npass) continue;
                    const uint32_t A = find_cell(b, p, bk, i, hi, slot_i, Lj, j);
                    if (A == kNone) continue;
                    emit_edges(b, e, A, npass, [&](auto &&put) {
                        each([&](uint32_t B) {
                            if (triplet_test(b, p, i, j, b.cell_out[B], hi, hj, a, na64, A, B))
                                put(B);
                        });
                    });
                }
            }
        }
        __syncwarp();
    }
}

void launch_connect(const DevBatch &b, const DevParams &p, uint32_t total, cudaStream_t s, int sms)
{
    (void)total;
    uint64_t blocks = ((uint64_t)b.N + 7) / 8;
    uint64_t cap = (uint64_t)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) return;
    k_connect<<<(unsigned)blocks, 256, 0, s>>>(b, p);
}

// ------------------------------------------------------------------------------------------
// Ntuplets: depth-first walk from every root cell
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_ntuplets(DevBatch b, DevParams p, uint32_t total)
{
    for (uint32_t A = blockIdx.x * blockDim.x + threadIdx.x; A < total;
         A += gridDim.x * blockDim.x) {
        const uint32_t e = find_event(b.cell_off, b.E, A);
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
    uint64_t blocks = ((uint64_t)total + 255) / 256;
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
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += gridDim.x * blockDim.x) {
        const uint32_t e = find_event(b.tup_off, b.E, t);
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
    uint64_t blocks = ((uint64_t)total + 255) / 256;
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
