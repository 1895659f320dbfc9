// Device-side data layout of one batch of events, shared by the library's kernels.
//
// A batch holds E events whose hits sit back to back in the caller's arrays.  Every per-event
// product (cells, CA edges, ntuplets, tracks) lives in a per-event region of a batch-wide array;
// region e starts at the prefix of the per-event capacities computed on the host, and a per-event
// counter says how much of it was filled.  Overflow of a region sets a per-event flag and drops
// the excess: nothing is ever written outside a region, and one event's overflow never affects
// another event (the result of an event does not depend on the batch it was run in).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pxr {

constexpr int kMaxLayers = 16;
constexpr int kMaxPairs = 32;
constexpr int kMaxHits = 6;      // hit slots per ntuplet / track
constexpr int kMaxOut = 4;       // layer pairs sharing one inner layer
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int kLocalBits = 24;   // hmeta = layer << 24 | index of the hit inside its event
constexpr uint32_t kLocalMask = (1u << kLocalBits) - 1u;
constexpr uint32_t kChunk = 256;     // per-event cell / ntuplet capacities are multiples of this
constexpr uint32_t kHitChunk = 32;   // granularity of the hit -> event table
constexpr uint32_t kCaTile = 32;     // junction hits per tile of the dense CA pass

// Per-event counters, laid out as kCounters consecutive arrays of E words.
enum Counter : int {
    C_CELLS = 0, C_EDGES = 1, C_TUPLES = 2, C_FLAGS = 3, C_OUT = 4,   // reported per event
    C_ROOTS = 5, C_SLOTS = 6, C_FRONT = 7, C_VERTS = 8,                // internal
    kCounters = 9
};
constexpr int kReportedCounters = 5;

// Track quality bits (the header's PXR_Q_GOOD, PXR_Q_KEPT).
constexpr uint8_t kQGood = 1u, kQKept = 2u;

// Per-event flags (C_FLAGS).
enum Flag : uint32_t {
    F_CELLS = 1u, F_EDGES = 2u, F_TUPLES = 4u, F_LAYER = 8u, F_VERTS = 16u,
    F_BOUNDS = 32u   // (checked build) an index outside its array; the access was skipped
};

enum CutMode : uint32_t { CUT_FP64 = 0, CUT_FP32 = 1 };
enum FitMode : uint32_t { FIT_FP64 = 0, FIT_MIXED = 1, FIT_FP32 = 2, FIT_RIEMANN = 3, FIT_SPLIT = 4 };

struct DevParams {
    uint32_t n_layers;
    uint32_t nb;                        // phi bins per layer
    uint32_t n_keys;                    // n_layers * nb
    uint32_t root_mask;
    uint32_t drop_suffixes;
    uint32_t min_hits, max_hits;
    uint32_t cut_mode, fit_mode;
    uint8_t is_disk[kMaxLayers];
    uint8_t n_out[kMaxLayers];          // number of pairs whose inner layer is l
    uint8_t out_layer[kMaxLayers][kMaxOut];   // their outer layers
    uint8_t n_in[kMaxLayers];           // number of pairs whose outer layer is l
    uint8_t in_layer[kMaxLayers][kMaxOut];    // their inner layers
    uint8_t in_slot[kMaxLayers][kMaxOut];     // slot of l among the inner layer's outer layers
    float bins_per_rad;                 // nb / (2 pi)
    float w_eps;                        // phi_window + margin for the bin window (radians)
    float cw32;                         // cos(w) rounded to float
    float theta32;                      // theta_cut rounded to float
    float dca32;                        // dca_cut rounded to float
    float tan_win;                      // tan(asin(theta_cut) + margin); inf when theta_cut >= 1
    uint32_t grid_per_sm[6];            // CTAs per SM at most, per stage (sort ... fit)
    uint32_t block_threads[6];          // threads per CTA per stage (fit: 0 = from the track count)
    uint32_t gphi, gz;                  // hit grid: coarse azimuth bins (bin = fine bin * gphi
                                        //   / nb) and bins of the free coordinate per layer
    uint32_t n_glayers;                 // layers in the grid: the out-layers of the pairs that
    uint8_t glidx[kMaxLayers];          //   start on a sparse CA junction layer; glidx = the
                                        //   layer's index among them, 0xFF for the others
    // CA levels: junction layers (with in- and out-pairs) ordered so that every pair's inner
    // layer comes first; per level the junction layers whose in-cells include root cells (dense
    // pass) and those with in-cells from non-root layers (sparse pass over reached cells)
    uint32_t n_levels;
    uint32_t level_dense[kMaxLayers + 1], level_sparse[kMaxLayers + 1];   // layer bit masks
    double cw;                          // cos(w) as given by the caller
    double theta, dca;
    double bfield, sigma_rphi, sigma_z, x_over_x0;
    double w_rphi, w_z, s2_rphi, s2_z, i_sz;   // 1/sigma_rphi^2, 1/sigma_z^2, sigma_rphi^2,
                                               //   sigma_z^2, 1/sigma_z (host-computed)
    double pt_min, chi2_max;            // track selection (0: no cut)
    uint32_t clean;                     // shared-hit cleaning
    uint32_t cov;                       // fit covariance wanted
    uint32_t vtx, vtx_min;              // primary vertices wanted; tracks a vertex needs
    double vtx_gap;                     // largest z gap (cm) inside a vertex cluster
};

struct DevBatch {
    uint32_t E;                         // events
    uint32_t N;                         // hits of all events
    uint32_t C, G, T;                   // cell entries, edge entries and ntuple slots of the
                                        //   batch (the extents the checked build tests against)
    // inputs (device, caller order, events back to back)
    const float *x, *y, *z;
    const uint16_t *layer;
    const uint32_t *hit_off;            // [E+1]
    // per-event capacity prefixes [E+1]
    const uint32_t *cell_off, *edge_off, *tup_off;
    uint32_t *cnt;                      // [kCounters * E]
    // counting sort of hits by (layer, phi bin)
    uint32_t *bkt;                      // [E * (n_keys + 1)] absolute positions
    float4 *hs;                         // [N] sorted hits: x, y, z, r (float)
    double *r64;                        // [N] sorted radii, FP64
    uint32_t *hmeta;                    // [N] layer << 24 | local caller index
    float *hphi;                        // [N] atan2f(y, x) of the sorted hits (the binned value)
    // hit grid of the sparse CA pass: per event and grid layer (index g = glidx[layer]), coarse
    // azimuth bins x bins of the free coordinate (z on barrel layers, r on disks);
    // gofs[e][(g * gphi + pc) * gz + zc] is the start of the cell's hits in gpos / gfree
    // (absolute, events back to back, one end entry per event); glay[e][g] = (free min, free
    // bin scale, fixed min, fixed max)
    uint32_t *gofs;                     // [E * (n_glayers * gphi * gz + 1)]
    uint32_t *gpos;                     // [N] sorted hit positions of grid layers, by grid cell
    float *gfree;                       // [N] their free coordinates
    float4 *glay;                       // [E * n_glayers]
    // event of a work chunk: cells, edges and ntuplets by 256-entry chunk; hits by 32-hit chunk
    // (first event of the chunk, bit 31 set when the chunk holds the start of a later event)
    const uint32_t *cell_chunk, *edge_chunk, *tup_chunk, *hit_chunk;
    // cells, grouped by (inner hit, pair slot).  The plan path keeps one entry per candidate of
    // the inner hit's phi window on the outer layer, in window order (run 1, then run 2), with
    // cell_out = kNone where the doublet cut failed.  item[(i, slot)] = (first entry, entries,
    // r0, d2): the cell (i, o) sits at first + rank, rank = o - r0 for o >= r0 (window run 1)
    // and o + d2 otherwise (run 2; unsigned arithmetic, d2 = run-1 length - run-2 start).  The
    // inner hit of an entry is implied by the item whose run holds it (the plan path stores no
    // per-entry inner hit: the CA lists carry it where a reader needs it).  The allocation-free
    // entry point writes passing pairs only, with their inner hits (item z, w unused).
    uint4 *item;                        // [N * kMaxOut]
    uint32_t *cell_in;                  // [entries] inner hit (allocation-free entry point only)
    uint32_t *cell_out;                 // [entries] outer hit, sorted position
    // CA graph: out-edges of each cell
    uint2 *nbr_head;                    // [cells] the cell's edge list: x first (absolute), y count
    uint32_t *nbr;                      // [edges] target cells
    uint32_t *mindepth;                 // [cells] fewest hits before the cell on a root path
    uint32_t *root_list;                // [edges] per event: root cells that have out-edges
    uint32_t *root_in;                  // [edges] their inner hits
    uint32_t *live;                     // [entries / 32] bit per cell: has an in-edge
    uint32_t *front_list;               // [edges] per event: non-root cells with in-edges whose
                                        //   outer hit starts further pairs (the sparse CA input;
                                        //   kNone: a slot reserved for a cell already listed)
    uint32_t *front_in;                 // [edges] the inner hits of the frontier cells
    uint32_t *jbase;                    // [E + 1] per-event prefix of the tiles of a dense CA level
    uint4 *tiles;                       // [N / kCaTile + E * n_layers + 1] the tiles of a dense CA
                                        //   level: (event, layer, first junction hit, hits)
    unsigned long long *ca_tests;       // [2] or null: CA candidate tests evaluated (r-z test) and
                                        //   of them the ones whose DCA was evaluated (counted
                                        //   only when non-null)
    uint32_t *front_snap;               // [E] frontier lengths when a sparse pass starts (the pass
                                        //   appends for later levels while it reads)
    // ntuplets
    uint32_t *tup_hits;                 // [tuples * kMaxHits] sorted hit positions
    uint8_t *tup_n;                     // [tuples]
    uint8_t *tup_state;                 // [tuples] 1 capped, 2 ended without edge
    uint32_t *tup_first;                // [tuples] root cell
    uint32_t *tup_rank;                 // [tuples] output slot within the event, kNone = dropped
    uint32_t *tup_list;                 // [tuples] per event: kept ntuplets in output order
                                        //   (canonical: by their hits' caller indices)
    uint32_t *tup_tmp;                  // [tuples] scratch of the canonical ordering
    uint32_t *canon_cnt;                // [N] per-hit counters of the canonical ordering
    // compact output, events back to back
    uint32_t *out_evt;                  // [E+1]
    uint32_t out_cap;                   // output slots (= tuple capacity)
    uint8_t *o_nh;
    uint32_t *o_hits;                   // [out_cap * kMaxHits] caller indices within the event
    double *o_pt, *o_phi, *o_cot, *o_dxy, *o_dz, *o_chi2;
    int8_t *o_q, *o_status;
    uint8_t *o_ql;                      // quality bits (PXR_Q_*)
    double *o_cov;                      // [out_cap * 15] covariances (only with the cov option)
    // primary vertices (only with the vertex option): per track its vertex (-1 none); per event
    // the vertices at the event's output offset, ordered by sum pT^2 (C_VERTS of them)
    int32_t *o_vtx;
    double *v_z, *v_err, *v_pt2;
    uint32_t *v_n;
    unsigned long long *best;           // [N] shared-hit cleaning: best rank key per hit (caller
                                        //   order, events back to back)
};

// Bounds checks of the checked build (compiled with PXR_CHECKED): an index that a kernel reads
// from another kernel's output, or computes from it, is compared with the extent of the array it
// addresses before the access; outside it, the event's F_BOUNDS flag is set and the access
// skipped (no trap: the context stays usable and the host reports PXR_EBOUNDS).  The normal
// build compiles every check to true.
#ifdef PXR_CHECKED
__device__ __forceinline__ bool bound_ok(const DevBatch &b, uint32_t e, uint64_t i, uint64_t n)
{
    if (i < n) return true;
    atomicOr(&b.cnt[3 * b.E + e], 32u);         // C_FLAGS, F_BOUNDS
    return false;
}
#define PXR_IN(b, e, i, n) ::pxr::bound_ok((b), (e), (uint64_t)(i), (uint64_t)(n))
#else
#define PXR_IN(b, e, i, n) true
#endif

// Event of hit g: the chunk table gives the event of the chunk's first hit.
__device__ __forceinline__ uint32_t hit_event(const DevBatch &b, uint32_t g)
{
    const uint32_t v = b.hit_chunk[g / kHitChunk];
    uint32_t e = v & 0x7FFFFFFFu;
    if (v >> 31)
        while (e + 1 < b.E && g >= b.hit_off[e + 1]) ++e;
    return e;
}

// Largest e with off[e] <= t (off non-decreasing, off[0] = 0, t < off[E]).
__device__ __forceinline__ uint32_t find_event(const uint32_t *__restrict__ off, uint32_t E,
                                               uint32_t t)
{
    uint32_t lo = 0, hi = E;  // invariant: off[lo] <= t < off[hi]
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// Block-wide exclusive scan of s[0..n) in place; returns the total.  blockDim.x is a multiple
// of 32 and at most 1024.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t *s, uint32_t n, uint32_t *warp_tot)
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

// One-time kernel attributes (large dynamic shared memory of the sort kernel).
cudaError_t init_kernels();
cudaError_t init_fit_kernels();     // (called by init_kernels)
cudaError_t init_graph_kernels();   // (called by init_kernels)

// Kernel launchers (defined in the .cu files).
void launch_sort(const DevBatch &b, const DevParams &p, cudaStream_t s, int sms);
void launch_layer_count(const uint32_t *hit_off, const uint16_t *layer, uint32_t E,
                        uint32_t n_layers, uint32_t *counts, cudaStream_t s, int sms);
void launch_doublets(const DevBatch &b, const DevParams &p, cudaStream_t s, int sms);
void launch_doublets_compact(const DevBatch &b, const DevParams &p, cudaStream_t s, int sms);
void launch_connect_front(const DevBatch &b, const DevParams &p, uint32_t edge_total,
                          uint32_t layer_mask, cudaStream_t s, int sms);
void launch_connect(const DevBatch &b, const DevParams &p, uint32_t layer_mask, cudaStream_t s,
                    int sms);
void launch_ntuplets(const DevBatch &b, const DevParams &p, uint32_t edge_total, cudaStream_t s,
                     int sms);
void launch_select(const DevBatch &b, const DevParams &p, uint32_t tup_total, cudaStream_t s,
                   int sms);
void launch_out_scan(const DevBatch &b, cudaStream_t s);
void launch_canon(const DevBatch &b, cudaStream_t s, int sms);
void launch_fit(const DevBatch &b, const DevParams &p, uint32_t tup_total, cudaStream_t s,
                int sms);
void launch_keep(const DevBatch &b, const DevParams &p, uint32_t tup_total, cudaStream_t s,
                 int sms);
void launch_vertices(const DevBatch &b, const DevParams &p, cudaStream_t s, int sms);
void launch_fit_batch(uint32_t m, const uint8_t *nh, const float *x, const float *y,
                      const float *z, const uint16_t *layer, uint32_t stride, const DevParams &p,
                      double *pt, double *phi, double *cot, double *dxy, double *dz, double *chi2,
                      int8_t *q, int8_t *status, cudaStream_t s, int sms);

}  // namespace pxr
