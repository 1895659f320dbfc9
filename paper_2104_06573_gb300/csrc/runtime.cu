// Host runtime of the pxr C ABI: parameter checks, the device arena, batch plans (memory layout,
// per-event capacities, launch sequence, CUDA graph), result readback, the fit-only path and the
// serving scheduler (continuous batching under a device-memory budget).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pxr.h"
#include "pxr_dev.cuh"

using namespace pxr;

// ------------------------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------------------------
static thread_local std::string g_err;

static int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(PXR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
    } while (0)

extern "C" const char *pxr_version(void) { return "pxr 0.1 (sm_103a)"; }
extern "C" const char *pxr_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------------------------------------
// parameters
// ------------------------------------------------------------------------------------------
extern "C" int pxr_params_init(pxr_params *p, int preset)
{
    if (!p) return fail(PXR_EINVAL, "null params");
    std::memset(p, 0, sizeof(*p));
    p->vtx_min_tracks = 2;                      // used when vertexing is switched on
    p->vtx_gap = 0.05;
    if (preset == PXR_PRESET_BARREL) {
        p->n_layers = 4;
        const uint8_t pi[] = {0, 1, 2}, po[] = {1, 2, 3};
        p->n_pairs = 3;
        std::memcpy(p->pair_inner, pi, 3);
        std::memcpy(p->pair_outer, po, 3);
        p->root_layer_mask = 1u;
        p->drop_suffixes = 0;
        p->min_hits = 4;
        p->max_hits = 4;
    } else if (preset == PXR_PRESET_PHASE1) {
        p->n_layers = 10;
        for (int l = 4; l < 10; ++l) p->layer_is_disk[l] = 1;
        const uint8_t pi[] = {0, 1, 2, 0, 1, 2, 0, 1, 2, 4, 5, 7, 8};
        const uint8_t po[] = {1, 2, 3, 4, 4, 4, 7, 7, 7, 5, 6, 8, 9};
        p->n_pairs = 13;
        std::memcpy(p->pair_inner, pi, 13);
        std::memcpy(p->pair_outer, po, 13);
        p->root_layer_mask = 3u;
        p->drop_suffixes = 1;
        p->min_hits = 3;
        p->max_hits = 5;
    } else {
        return fail(PXR_EINVAL, "unknown preset");
    }
    p->cut_mode = PXR_CUT_FP64;
    p->fit_mode = PXR_FIT_FP64;
    p->phi_window = 0.05;
    p->cos_phi_window = std::cos(0.05);
    p->theta_cut = 0.002;
    p->dca_cut = 0.15;
    p->bfield = 3.8;
    p->sigma_rphi = 10e-4;
    p->sigma_z = 20e-4;
    p->x_over_x0 = 0.02;
    return PXR_OK;
}

static uint32_t auto_bins(double w)
{
    // bins about a quarter of the window wide: the scanned bins exceed the window by < 25 %
    double nb = 2.0 * M_PI / (0.25 * w);
    uint32_t b = 64;
    while (b < nb && b < 2048) b <<= 1;
    return b;
}

static int check_params(const pxr_params *p, DevParams *d)
{
    if (!p) return fail(PXR_EINVAL, "null params");
    if (p->n_layers < 1 || p->n_layers > PXR_MAX_LAYERS) return fail(PXR_EINVAL, "n_layers out of range");
    if (p->n_pairs < 1 || p->n_pairs > PXR_MAX_PAIRS) return fail(PXR_EINVAL, "n_pairs out of range");
    if (p->min_hits < 2 || p->max_hits > PXR_MAX_HITS || p->min_hits > p->max_hits)
        return fail(PXR_EINVAL, "need 2 <= min_hits <= max_hits <= 6");
    if (p->cut_mode > PXR_CUT_FP32) return fail(PXR_EINVAL, "bad cut_mode");
    if (p->fit_mode > PXR_FIT_SPLIT) return fail(PXR_EINVAL, "bad fit_mode");
    if (!(p->phi_window > 0.0 && p->phi_window <= 0.5)) return fail(PXR_EINVAL, "phi_window must be in (0, 0.5]");
    if (!(std::fabs(p->cos_phi_window - std::cos(p->phi_window)) < 1e-12))
        return fail(PXR_EINVAL, "cos_phi_window must equal cos(phi_window)");
    if (!(p->theta_cut > 0.0) || !(p->dca_cut > 0.0) || !(p->bfield > 0.0) ||
        !(p->sigma_rphi > 0.0) || !(p->sigma_z > 0.0) || !(p->x_over_x0 >= 1e-6) ||
        !std::isfinite(p->theta_cut) || !std::isfinite(p->dca_cut))
        return fail(PXR_EINVAL, "cuts, field, errors and material must be positive and finite");
    if (p->n_phi_bins && (p->n_phi_bins < 64 || p->n_phi_bins > 2048))
        return fail(PXR_EINVAL, "n_phi_bins must be 0 or in [64, 2048]");
    for (int k = 0; k < PXR_STAGES; ++k)
        if (p->grid_per_sm[k] > 64) return fail(PXR_EINVAL, "grid_per_sm must be in [0, 64]");
    {
        // threads per CTA each stage's kernels accept (0 = built-in; a zero row: 0 only)
        static const uint32_t kBlockOk[PXR_STAGES][4] = {
            {256, 512, 1024, 0}, {64, 128, 256, 0}, {0}, {0}, {0}, {32, 64, 128, 256}};
        for (int k = 0; k < PXR_STAGES; ++k) {
            const uint32_t t = p->block_threads[k];
            bool ok = t == 0;
            for (int i = 0; i < 4 && !ok; ++i) ok = kBlockOk[k][i] == t;
            if (!ok)
                return fail(PXR_EINVAL, "block_threads: sort 256/512/1024, doublets 64/128/256, "
                                        "fit 32/64/128/256, connect/walk/select 0 only");
        }
    }
    if (!(p->pt_min >= 0.0) || !(p->chi2_max >= 0.0) || !std::isfinite(p->pt_min) ||
        !std::isfinite(p->chi2_max) || p->clean_shared > 1)
        return fail(PXR_EINVAL, "pt_min and chi2_max must be finite and >= 0, clean_shared 0 or 1");
    if (p->fit_cov > 1) return fail(PXR_EINVAL, "fit_cov must be 0 or 1");
    if (p->vertexing > 1 || (p->vertexing && (p->vtx_min_tracks < 2 || !(p->vtx_gap > 0.0) ||
                                             !std::isfinite(p->vtx_gap))))
        return fail(PXR_EINVAL, "vertexing needs vtx_min_tracks >= 2 and a finite vtx_gap > 0");
    if (!d) return PXR_OK;
    std::memset(d, 0, sizeof(*d));
    d->n_layers = p->n_layers;
    d->nb = p->n_phi_bins ? p->n_phi_bins : auto_bins(p->phi_window);
    d->n_keys = d->n_layers * d->nb;
    d->root_mask = p->root_layer_mask;
    d->drop_suffixes = p->drop_suffixes ? 1 : 0;
    d->min_hits = p->min_hits;
    d->max_hits = p->max_hits;
    d->cut_mode = p->cut_mode;
    d->fit_mode = p->fit_mode;
    for (uint32_t l = 0; l < p->n_layers; ++l) d->is_disk[l] = p->layer_is_disk[l] ? 1 : 0;
    for (uint32_t k = 0; k < p->n_pairs; ++k) {
        uint32_t a = p->pair_inner[k], b = p->pair_outer[k];
        if (a >= p->n_layers || b >= p->n_layers || a == b)
            return fail(PXR_EINVAL, "pair layer out of range or inner == outer");
        for (uint32_t s = 0; s < d->n_out[a]; ++s)
            if (d->out_layer[a][s] == b) return fail(PXR_EINVAL, "duplicate layer pair");
        if (d->n_out[a] >= kMaxOut) return fail(PXR_EINVAL, "more than 4 pairs share an inner layer");
        if (d->n_in[b] >= kMaxOut) return fail(PXR_EINVAL, "more than 4 pairs share an outer layer");
        d->in_layer[b][d->n_in[b]] = (uint8_t)a;
        d->in_slot[b][d->n_in[b]++] = d->n_out[a];
        d->out_layer[a][d->n_out[a]++] = (uint8_t)b;
    }
    d->bins_per_rad = (float)(d->nb / (2.0 * M_PI));
    d->w_eps = (float)(p->phi_window + 2e-5);
    d->cw32 = (float)p->cos_phi_window;
    d->theta32 = (float)p->theta_cut;
    d->dca32 = (float)p->dca_cut;
    // |sin(angle)| <= t  <=>  the r-z directions differ by at most asin(t) modulo pi
    d->tan_win = p->theta_cut < 0.99 ? (float)std::tan(std::asin(p->theta_cut) + 1e-5)
                                     : INFINITY;
    d->cw = p->cos_phi_window;
    d->theta = p->theta_cut;
    d->dca = p->dca_cut;
    d->bfield = p->bfield;
    d->sigma_rphi = p->sigma_rphi;
    d->sigma_z = p->sigma_z;
    d->s2_rphi = p->sigma_rphi * p->sigma_rphi;
    d->s2_z = p->sigma_z * p->sigma_z;
    d->w_rphi = 1.0 / d->s2_rphi;
    d->w_z = 1.0 / d->s2_z;
    d->i_sz = 1.0 / p->sigma_z;
    d->x_over_x0 = p->x_over_x0;
    d->pt_min = p->pt_min;
    d->chi2_max = p->chi2_max;
    d->clean = p->clean_shared;
    d->cov = p->fit_cov;
    d->vtx = p->vertexing;
    d->vtx_min = p->vtx_min_tracks;
    d->vtx_gap = p->vtx_gap;
    // CA levels: a layer's level is 1 + the highest level of its pairs' inner layers (0 without
    // in-pairs); junction layers (in- and out-pairs) are processed level by level, so that every
    // cell has all its in-edges before its own out-edges are built
    uint32_t level[kMaxLayers] = {};
    for (uint32_t pass = 0;; ++pass) {
        bool changed = false;
        for (uint32_t l = 0; l < p->n_layers; ++l)
            for (uint32_t q = 0; q < d->n_in[l]; ++q)
                if (level[d->in_layer[l][q]] + 1u > level[l]) {
                    level[l] = level[d->in_layer[l][q]] + 1u;
                    changed = true;
                }
        if (!changed) break;
        if (pass >= p->n_layers) return fail(PXR_EINVAL, "layer pairs form a cycle");
    }
    for (uint32_t l = 0; l < p->n_layers; ++l) {
        if (!d->n_in[l] || !d->n_out[l]) continue;
        d->n_levels = std::max(d->n_levels, level[l]);
        for (uint32_t q = 0; q < d->n_in[l]; ++q) {
            if ((p->root_layer_mask >> d->in_layer[l][q]) & 1u) d->level_dense[level[l]] |= 1u << l;
            else d->level_sparse[level[l]] |= 1u << l;
        }
    }
    // hit grid of the sparse CA pass: the out-layers of the pairs that start on its junction
    // layers; 32 coarse azimuth bins, free-coordinate bins up to 1024 per layer with at most
    // 32768 cells per event (its counters share the sort's shared memory)
    uint32_t gmask = 0;
    for (uint32_t lv = 1; lv <= d->n_levels; ++lv)
        for (uint32_t l = 0; l < p->n_layers; ++l)
            if ((d->level_sparse[lv] >> l) & 1u)
                for (uint32_t q = 0; q < d->n_out[l]; ++q) gmask |= 1u << d->out_layer[l][q];
    for (uint32_t l = 0; l < kMaxLayers; ++l)
        d->glidx[l] = (gmask >> l) & 1u ? (uint8_t)d->n_glayers++ : (uint8_t)0xFF;
    d->gphi = 32;
    d->gz = 1024;
    while (d->gz > 8 && d->n_glayers * d->gphi * d->gz > 32768u) d->gz >>= 1;
    // launch shapes: CTAs per SM at most (the kernels stride over their work)
    static const uint32_t kGridDefault[PXR_STAGES] = {4, 16, 16, 8, 8, 8};
    for (int k = 0; k < PXR_STAGES; ++k)
        d->grid_per_sm[k] = p->grid_per_sm[k] ? p->grid_per_sm[k] : kGridDefault[k];
    static const uint32_t kBlockDefault[PXR_STAGES] = {512, 256, 0, 0, 0, 0};
    for (int k = 0; k < PXR_STAGES; ++k)
        d->block_threads[k] = p->block_threads[k] ? p->block_threads[k] : kBlockDefault[k];
    return PXR_OK;
}

extern "C" int pxr_params_check(const pxr_params *p)
{
    DevParams d;
    return check_params(p, &d);
}

// ------------------------------------------------------------------------------------------
// per-event capacities
// ------------------------------------------------------------------------------------------
struct EventCaps {
    uint32_t cells, edges, tuples;
};

static EventCaps event_caps(const pxr_params &p, uint32_t nb, const uint32_t *lcount, uint32_t n)
{
    // Cell entries are the candidates of the inner hits' bin windows: with uniform azimuths a
    // pair has n_i n_o f of them, f = (2 w + one bin) / 2pi (the whole bins that cover an
    // interval exceed it by one bin width on average); 30 % head room plus a per-hit floor
    // covers fluctuations.  Edges: measured ~2-3 % of cells on the synthetic workloads.
    double pairs = 0.0, inner = 0.0;
    for (uint32_t k = 0; k < p.n_pairs; ++k) {
        pairs += (double)lcount[p.pair_inner[k]] * (double)lcount[p.pair_outer[k]];
        inner += lcount[p.pair_inner[k]];
    }
    double f = std::min(1.0, (2.0 * (p.phi_window + 2e-5) + 2.0 * M_PI / nb) / (2.0 * M_PI));
    double cells = p.max_cells_per_event ? (double)p.max_cells_per_event
                                         : std::ceil(1.3 * f * pairs) + 4.0 * inner + 256.0;
    cells = std::min(cells, 1.0e9);
    double edges = std::ceil(0.08 * cells) + 4.0 * n + 256.0;
    double tuples = p.max_tuples_per_event ? (double)p.max_tuples_per_event
                                           : std::ceil(0.5 * edges) + 2.0 * n + 256.0;
    // cells, edges and ntuplets in whole chunks: every chunk of the work loops belongs to one event
    auto up = [](double v) { return (uint32_t)(std::ceil(v / kChunk) * kChunk); };
    return EventCaps{up(cells), up(std::min(edges, 1.0e9)), up(std::min(tuples, 1.0e9))};
}

// ------------------------------------------------------------------------------------------
// device memory layout of one plan
// ------------------------------------------------------------------------------------------
struct Layout {
    size_t total = 0;
    size_t add(size_t bytes)
    {
        size_t off = (total + 255) & ~size_t(255);
        total = off + bytes;
        return off;
    }
};

struct PlanOffsets {
    // inputs (serving plans only) and small host-filled arrays come first: one H2D copy
    size_t x, y, z, layer, hit_off, cell_off, edge_off, tup_off, cell_chunk, edge_chunk, tup_chunk,
        hit_chunk,
        head_end;
    size_t cnt, bkt, hs, r64, hmeta, hphi, gofs, gpos, gfree, glay, item, cell_out,
        nbr_head, nbr, mindepth, root_list, root_in, live, front_list, front_in, front_snap, jbase, tiles, ca_tests, tup_hits, tup_n, tup_state, tup_first, tup_rank, tup_list, tup_tmp, canon_cnt, out_evt, o_nh,
        o_hits, o_pt, o_phi, o_cot, o_dxy, o_dz, o_chi2, o_q, o_status, o_ql, best, o_cov, o_vtx,
        v_z, v_err, v_pt2, v_n;
    size_t total;
};

static PlanOffsets plan_layout(uint32_t E, uint64_t N, uint64_t C, uint64_t G, uint64_t T,
                               const DevParams &dp, bool with_inputs)
{
    Layout L;
    PlanOffsets o{};
    uint64_t Ni = with_inputs ? N : 0;
    o.x = L.add(4 * Ni);
    o.y = L.add(4 * Ni);
    o.z = L.add(4 * Ni);
    o.layer = L.add(2 * Ni);
    o.hit_off = L.add(4 * (E + 1));
    o.cell_off = L.add(4 * (E + 1));
    o.edge_off = L.add(4 * (E + 1));
    o.tup_off = L.add(4 * (E + 1));
    o.cell_chunk = L.add(4 * (C / kChunk));
    o.edge_chunk = L.add(4 * (G / kChunk));
    o.tup_chunk = L.add(4 * (T / kChunk));
    o.hit_chunk = L.add(4 * ((N + kHitChunk - 1) / kHitChunk));
    o.head_end = L.total;
    o.cnt = L.add(4 * (size_t)kCounters * E);
    o.bkt = L.add(4 * (size_t)E * (dp.n_keys + 1));
    o.hs = L.add(16 * N);
    o.r64 = L.add(8 * N);
    o.hmeta = L.add(4 * N);
    o.hphi = L.add(4 * N);
    o.gofs = L.add(dp.n_glayers ? 4 * (size_t)E * ((size_t)dp.n_glayers * dp.gphi * dp.gz + 1) : 0);
    o.gpos = L.add(dp.n_glayers ? 4 * N : 0);
    o.gfree = L.add(dp.n_glayers ? 4 * N : 0);
    o.glay = L.add(16 * (size_t)E * dp.n_glayers);

    o.item = L.add(16 * N * kMaxOut);
    o.cell_out = L.add(4 * C);
    o.nbr_head = L.add(8 * C);
    o.nbr = L.add(4 * G);
    o.mindepth = L.add(4 * C);
    o.root_list = L.add(4 * G);
    o.root_in = L.add(4 * G);
    o.live = L.add(4 * ((C + 31) / 32));
    o.front_list = L.add(4 * G);
    o.front_in = L.add(4 * G);
    o.front_snap = L.add(4 * (size_t)E);
    o.jbase = L.add(4 * ((size_t)E + 1));
    o.tiles = L.add(16 * (N / kCaTile + (size_t)E * dp.n_layers + 1));
    o.ca_tests = L.add(16);
    o.tup_hits = L.add(4 * T * kMaxHits);
    o.tup_n = L.add(T);
    o.tup_state = L.add(T);
    o.tup_first = L.add(4 * T);
    o.tup_rank = L.add(4 * T);
    o.tup_list = L.add(4 * T);
    o.tup_tmp = L.add(4 * T);
    o.canon_cnt = L.add(4 * N);
    o.out_evt = L.add(4 * (E + 1));
    o.o_nh = L.add(T);
    o.o_hits = L.add(4 * T * kMaxHits);
    o.o_pt = L.add(8 * T);
    o.o_phi = L.add(8 * T);
    o.o_cot = L.add(8 * T);
    o.o_dxy = L.add(8 * T);
    o.o_dz = L.add(8 * T);
    o.o_chi2 = L.add(8 * T);
    o.o_q = L.add(T);
    o.o_status = L.add(T);
    o.o_ql = L.add(T);
    o.best = L.add(dp.clean ? 8 * N : 0);
    o.o_cov = L.add(dp.cov ? 8 * 15 * T : 0);
    o.o_vtx = L.add(dp.vtx ? 4 * T : 0);
    o.v_z = L.add(dp.vtx ? 8 * T : 0);
    o.v_err = L.add(dp.vtx ? 8 * T : 0);
    o.v_pt2 = L.add(dp.vtx ? 8 * T : 0);
    o.v_n = L.add(dp.vtx ? 4 * T : 0);
    o.total = L.add(0);
    return o;
}

// ------------------------------------------------------------------------------------------
// tracing and host-side fault injection
// ------------------------------------------------------------------------------------------
// NVTX range over a host scope (what a timeline profiler shows next to the kernels it launches).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

// Test hook: with PXR_FAULT_ARENA=n in the environment, the n-th arena allocation of the process
// (counting from 1) fails as if the arena were full.  Host-side only; nothing on the GPU fails.
static bool arena_fault_now()
{
    static const long at = [] {
        const char *v = std::getenv("PXR_FAULT_ARENA");
        return v ? std::atol(v) : 0L;
    }();
    static std::atomic<long> calls{0};
    return at > 0 && calls.fetch_add(1) + 1 == at;
}

// ------------------------------------------------------------------------------------------
// arena: first-fit free list over one device allocation
// ------------------------------------------------------------------------------------------
struct Arena {
    char *base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> size
    std::mutex mu;

    void init(char *b, size_t s)
    {
        base = b;
        size = s;
        free_.clear();
        free_[0] = s;
    }
    char *alloc(size_t bytes)
    {
        if (arena_fault_now()) return nullptr;
        std::lock_guard<std::mutex> g(mu);
        bytes = (bytes + 255) & ~size_t(255);
        if (bytes == 0) bytes = 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                size_t off = it->first, rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                return base + off;
            }
        }
        return nullptr;
    }
    void release(char *p, size_t bytes)
    {
        if (!p) return;
        std::lock_guard<std::mutex> g(mu);
        bytes = (bytes + 255) & ~size_t(255);
        if (bytes == 0) bytes = 256;
        size_t off = (size_t)(p - base);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

// ------------------------------------------------------------------------------------------
// context and plan
// ------------------------------------------------------------------------------------------
// Pinned host memory of the serving path: submissions' hits (copied from the caller once,
// then sent to the device straight from here) and batches' results (received from the device
// and read by the fetches in place).  Blocks are reused (pinned allocation is slow and
// synchronising), kept by size class (powers of two from 64 KiB), freed with the context.
struct PinnedPool {
    std::mutex mu;
    std::multimap<size_t, char *> free_;
    std::vector<char *> all;
    char *get(size_t bytes, size_t &got)
    {
        size_t c = size_t(1) << 16;
        while (c < bytes) c <<= 1;
        {
            std::lock_guard<std::mutex> g(mu);
            auto it = free_.lower_bound(c);
            if (it != free_.end() && it->first == c) {
                char *p = it->second;
                free_.erase(it);
                got = c;
                return p;
            }
        }
        char *p = nullptr;
        if (cudaMallocHost((void **)&p, c) != cudaSuccess) return nullptr;
        std::lock_guard<std::mutex> g(mu);
        all.push_back(p);
        got = c;
        return p;
    }
    void put(char *p, size_t n)
    {
        std::lock_guard<std::mutex> g(mu);
        free_.emplace(n, p);
    }
    ~PinnedPool()
    {
        for (char *p : all) cudaFreeHost(p);
    }
};

// A block of the pool, returned to it when the last holder lets go.
struct PinnedBlock {
    PinnedPool *pool = nullptr;
    char *p = nullptr;
    size_t n = 0;
    ~PinnedBlock()
    {
        if (p) pool->put(p, n);
    }
};

static std::shared_ptr<PinnedBlock> pinned_block(PinnedPool &pool, size_t bytes)
{
    auto b = std::make_shared<PinnedBlock>();
    b->pool = &pool;
    b->p = pool.get(bytes, b->n);
    if (!b->p) b.reset();
    return b;
}

struct Batch;

constexpr int kMaxSlots = 4;           // batches in flight at most (one stream and staging each)

struct pxr_ctx {
    pxr_config cfg{};
    int sms = 152;
    cudaStream_t stream = nullptr;      // default stream of the context
    bool own_stream = false;
    cudaStream_t slot_stream[kMaxSlots] = {};
    bool own_arena = false;
    Arena arena;
    std::mutex api_mu;                  // serialises plan API calls
    std::mutex plans_mu;
    std::unordered_set<pxr_plan *> plans;   // live plans, destroyed with the context
    // serving
    PinnedPool pool;                    // (outlives the tickets and batches holding its blocks)
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::thread sched;
    bool stop = false;
    size_t reserved = 0;
    uint64_t next_ticket = 1;
    std::deque<uint64_t> pending;
    std::deque<uint64_t> done_q;
    std::unordered_map<uint64_t, std::shared_ptr<struct Ticket>> tickets;
    std::vector<std::shared_ptr<Batch>> inflight;
    std::unique_ptr<struct SlotBuffers> slot_buf[kMaxSlots];
    std::string sched_error;
};

struct pxr_plan {
    pxr_ctx *ctx = nullptr;
    pxr_params params{};
    DevParams dp{};
    uint32_t E = 0;
    uint64_t N = 0, C = 0, G = 0, T = 0;
    std::vector<uint32_t> hit_off, cell_off, edge_off, tup_off;
    std::vector<uint32_t> cell_chunk, edge_chunk, tup_chunk, hit_chunk;   // event of each chunk
    PlanOffsets off{};
    char *region = nullptr;
    DevBatch db{};
    bool own_inputs = false;
    bool use_graph = false;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t last_stream = nullptr;
    cudaEvent_t ev_done = nullptr;
    cudaEvent_t ev_stage[8] = {};
    bool timed = false;
    bool has_run = false;
};

static void plan_bind(pxr_plan *P)
{
    char *r = P->region;
    const PlanOffsets &o = P->off;
    DevBatch &b = P->db;
    b.E = P->E;
    b.N = (uint32_t)P->N;
    b.C = (uint32_t)P->C;
    b.G = (uint32_t)P->G;
    b.T = (uint32_t)P->T;
    if (P->own_inputs) {
        b.x = (const float *)(r + o.x);
        b.y = (const float *)(r + o.y);
        b.z = (const float *)(r + o.z);
        b.layer = (const uint16_t *)(r + o.layer);
    }
    b.hit_off = (const uint32_t *)(r + o.hit_off);
    b.cell_off = (const uint32_t *)(r + o.cell_off);
    b.edge_off = (const uint32_t *)(r + o.edge_off);
    b.tup_off = (const uint32_t *)(r + o.tup_off);
    b.cnt = (uint32_t *)(r + o.cnt);
    b.bkt = (uint32_t *)(r + o.bkt);
    b.hs = (float4 *)(r + o.hs);
    b.r64 = (double *)(r + o.r64);
    b.hmeta = (uint32_t *)(r + o.hmeta);
    b.hphi = (float *)(r + o.hphi);
    b.gofs = (uint32_t *)(r + o.gofs);
    b.gpos = P->dp.n_glayers ? (uint32_t *)(r + o.gpos) : nullptr;     // (null: no grid)
    b.gfree = (float *)(r + o.gfree);
    b.glay = (float4 *)(r + o.glay);
    b.cell_chunk = (const uint32_t *)(r + o.cell_chunk);
    b.edge_chunk = (const uint32_t *)(r + o.edge_chunk);
    b.tup_chunk = (const uint32_t *)(r + o.tup_chunk);
    b.hit_chunk = (const uint32_t *)(r + o.hit_chunk);

    b.item = (uint4 *)(r + o.item);
    b.cell_in = nullptr;
    b.cell_out = (uint32_t *)(r + o.cell_out);
    b.nbr_head = (uint2 *)(r + o.nbr_head);
    b.nbr = (uint32_t *)(r + o.nbr);
    b.mindepth = (uint32_t *)(r + o.mindepth);
    b.root_list = (uint32_t *)(r + o.root_list);
    b.root_in = (uint32_t *)(r + o.root_in);
    b.live = (uint32_t *)(r + o.live);
    b.front_list = (uint32_t *)(r + o.front_list);
    b.front_in = (uint32_t *)(r + o.front_in);
    b.front_snap = (uint32_t *)(r + o.front_snap);
    b.jbase = (uint32_t *)(r + o.jbase);
    b.tiles = (uint4 *)(r + o.tiles);
    b.tup_hits = (uint32_t *)(r + o.tup_hits);
    b.tup_n = (uint8_t *)(r + o.tup_n);
    b.tup_state = (uint8_t *)(r + o.tup_state);
    b.tup_first = (uint32_t *)(r + o.tup_first);
    b.tup_rank = (uint32_t *)(r + o.tup_rank);
    b.tup_list = (uint32_t *)(r + o.tup_list);
    b.tup_tmp = (uint32_t *)(r + o.tup_tmp);
    b.canon_cnt = (uint32_t *)(r + o.canon_cnt);
    b.out_evt = (uint32_t *)(r + o.out_evt);
    b.out_cap = (uint32_t)P->T;
    b.o_nh = (uint8_t *)(r + o.o_nh);
    b.o_hits = (uint32_t *)(r + o.o_hits);
    b.o_pt = (double *)(r + o.o_pt);
    b.o_phi = (double *)(r + o.o_phi);
    b.o_cot = (double *)(r + o.o_cot);
    b.o_dxy = (double *)(r + o.o_dxy);
    b.o_dz = (double *)(r + o.o_dz);
    b.o_chi2 = (double *)(r + o.o_chi2);
    b.o_q = (int8_t *)(r + o.o_q);
    b.o_status = (int8_t *)(r + o.o_status);
    b.o_ql = (uint8_t *)(r + o.o_ql);
    b.best = (unsigned long long *)(r + o.best);
    b.o_cov = (double *)(r + o.o_cov);
    b.o_vtx = (int32_t *)(r + o.o_vtx);
    b.v_z = (double *)(r + o.v_z);
    b.v_err = (double *)(r + o.v_err);
    b.v_pt2 = (double *)(r + o.v_pt2);
    b.v_n = (uint32_t *)(r + o.v_n);
}

// Fill the per-event capacity prefixes from per-layer counts (lcount: E x (kMaxLayers+1)).
static int plan_size(pxr_plan *P, const uint32_t *lcount, bool with_inputs)
{
    const uint32_t E = P->E;
    P->cell_off.assign(E + 1, 0);
    P->edge_off.assign(E + 1, 0);
    P->tup_off.assign(E + 1, 0);
    uint64_t C = 0, G = 0, T = 0;
    for (uint32_t e = 0; e < E; ++e) {
        uint32_t n = P->hit_off[e + 1] - P->hit_off[e];
        EventCaps c = event_caps(P->params, P->dp.nb, lcount + (size_t)e * (kMaxLayers + 1), n);
        C += c.cells;
        G += c.edges;
        T += c.tuples;
        if (C >= 0x7FFFFFFFull || G >= 0x7FFFFFFFull || T >= 0x7FFFFFFFull)
            return fail(PXR_ENOMEM, "batch capacities exceed 2^31 entries; split the batch");
        P->cell_off[e + 1] = (uint32_t)C;
        P->edge_off[e + 1] = (uint32_t)G;
        P->tup_off[e + 1] = (uint32_t)T;
    }
    P->C = C;
    P->G = G;
    P->T = T;
    P->cell_chunk.assign(C / kChunk, 0);
    P->edge_chunk.assign(G / kChunk, 0);
    P->tup_chunk.assign(T / kChunk, 0);
    P->hit_chunk.assign((P->N + kHitChunk - 1) / kHitChunk, 0);
    for (uint32_t e = 0; e < E; ++e) {
        for (uint32_t c = P->cell_off[e] / kChunk; c < P->cell_off[e + 1] / kChunk; ++c)
            P->cell_chunk[c] = e;
        for (uint32_t c = P->edge_off[e] / kChunk; c < P->edge_off[e + 1] / kChunk; ++c)
            P->edge_chunk[c] = e;
        for (uint32_t c = P->tup_off[e] / kChunk; c < P->tup_off[e + 1] / kChunk; ++c)
            P->tup_chunk[c] = e;
    }
    for (size_t c = 0, e = 0; c < P->hit_chunk.size(); ++c) {
        const uint64_t g = (uint64_t)c * kHitChunk;
        while (e + 1 < E && g >= P->hit_off[e + 1]) ++e;
        // bit 31: a later event starts inside this chunk
        const bool straddle = e + 1 < E && P->hit_off[e + 1] < g + kHitChunk;
        P->hit_chunk[c] = (uint32_t)e | (straddle ? 0x80000000u : 0u);
    }
    P->off = plan_layout(E, P->N, C, G, T, P->dp, with_inputs);
    return PXR_OK;
}

// Record a stage event; inside a stream capture it becomes an event-record node of the graph.
static cudaError_t stage_mark(cudaEvent_t ev, cudaStream_t s, bool capturing)
{
    return capturing ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                     : cudaEventRecord(ev, s);
}

// Copy the chunk tables into a host image of the plan's head region.
static void fill_chunks(const pxr_plan *P, char *head)
{
    std::memcpy(head + P->off.cell_chunk, P->cell_chunk.data(), 4 * P->cell_chunk.size());
    std::memcpy(head + P->off.edge_chunk, P->edge_chunk.data(), 4 * P->edge_chunk.size());
    std::memcpy(head + P->off.tup_chunk, P->tup_chunk.data(), 4 * P->tup_chunk.size());
    std::memcpy(head + P->off.hit_chunk, P->hit_chunk.data(), 4 * P->hit_chunk.size());
}

static int plan_enqueue(pxr_plan *P, cudaStream_t s, bool capturing = false,
                        const DevBatch *db = nullptr)
{
    Range range("pxr.enqueue");
    const DevBatch &b = db ? *db : P->db;
    const DevParams &p = P->dp;
    int sms = P->ctx->sms;
    char *r = P->region;
    const bool t = P->timed;
    if (t) CK(stage_mark(P->ev_stage[0], s, capturing));
    CK(cudaMemsetAsync(r + P->off.cnt, 0, 4 * (size_t)kCounters * P->E, s));
    if (p.drop_suffixes) CK(cudaMemsetAsync(r + P->off.mindepth, 0xFF, 4 * P->C, s));
    // edge counts are written for root cells with edges and for every reached cell (0 until it
    // gets out-edges); two readers need the others cleared: the walk over all root cells (when
    // 2-hit paths count) and a junction with several out-layers appending to an in-cell's list
    bool multi_out = false;
    for (uint32_t l = 0; l < p.n_layers; ++l) multi_out |= p.n_out[l] > 1;
    if (p.min_hits <= 2 || multi_out) CK(cudaMemsetAsync(r + P->off.nbr_head, 0, 8 * P->C, s));
    CK(cudaMemsetAsync(r + P->off.live, 0, 4 * ((P->C + 31) / 32), s));
    launch_sort(b, p, s, sms);
    if (t) CK(stage_mark(P->ev_stage[1], s, capturing));
    launch_doublets(b, p, s, sms);
    if (t) CK(stage_mark(P->ev_stage[2], s, capturing));
    for (uint32_t lv = 1; lv <= p.n_levels; ++lv) {
        if (p.level_dense[lv]) launch_connect(b, p, p.level_dense[lv], s, sms);
        if (p.level_sparse[lv]) {
            CK(cudaMemcpyAsync(b.front_snap, b.cnt + (size_t)C_FRONT * P->E, 4 * (size_t)P->E,
                               cudaMemcpyDeviceToDevice, s));
            launch_connect_front(b, p, (uint32_t)P->G, p.level_sparse[lv], s, sms);
        }
    }
    if (t) CK(stage_mark(P->ev_stage[3], s, capturing));
    launch_ntuplets(b, p, (uint32_t)P->G, s, sms);
    launch_select(b, p, (uint32_t)P->T, s, sms);
    launch_out_scan(b, s);
    launch_canon(b, s, sms);
    if (t) CK(stage_mark(P->ev_stage[4], s, capturing));
    // the selection's shared-hit ranks start at the largest key (no track)
    if (p.clean) CK(cudaMemsetAsync(b.best, 0xFF, 8 * (size_t)P->N, s));
    launch_fit(b, p, (uint32_t)P->T, s, sms);
    if (p.clean) launch_keep(b, p, (uint32_t)P->T, s, sms);
    if (p.vtx) launch_vertices(b, p, s, sms);
    if (t) CK(stage_mark(P->ev_stage[5], s, capturing));
    CK(cudaGetLastError());
    return PXR_OK;
}

static int plan_launches(const pxr_plan *P)
{
    // sort, doublets, walk (with its root-chunk prefix when paths need 3 hits), select (with
    // its ntuplet-chunk prefix), scan, order, fit, keep, vertices
    int n = 8 + (P->dp.min_hits > 2 ? 1 : 0) + (P->dp.clean ? 1 : 0) + (P->dp.vtx ? 1 : 0);
    for (uint32_t lv = 1; lv <= P->dp.n_levels; ++lv)
        n += (P->dp.level_dense[lv] ? 2 : 0) + (P->dp.level_sparse[lv] ? 1 : 0);
    return n;
}

static void plan_free(pxr_plan *P)
{
    if (!P) return;
    if (P->graph) cudaGraphExecDestroy(P->graph);
    if (P->ev_done) cudaEventDestroy(P->ev_done);
    for (auto &e : P->ev_stage)
        if (e) cudaEventDestroy(e);
    if (P->region) P->ctx->arena.release(P->region, P->off.total);
    delete P;
}

static int set_device(pxr_ctx *ctx)
{
    CK(cudaSetDevice(ctx->cfg.device));
    return PXR_OK;
}

static int plan_finish_setup(pxr_plan *P)
{
    CK(cudaEventCreateWithFlags(&P->ev_done, cudaEventDisableTiming));
    P->timed = true;
    for (auto &e : P->ev_stage) CK(cudaEventCreate(&e));
    return PXR_OK;
}

extern "C" int pxr_plan_create(pxr_ctx *ctx, uint32_t n_events, const uint32_t *hit_offsets,
                               const float *x, const float *y, const float *z,
                               const uint16_t *layer, const pxr_params *params, int use_graph,
                               pxr_plan **out)
{
    if (!ctx || !out || !hit_offsets || !x || !y || !z || !layer || n_events == 0)
        return fail(PXR_EINVAL, "null argument or no events");
    std::lock_guard<std::mutex> api(ctx->api_mu);
    int rc = set_device(ctx);
    if (rc) return rc;
    std::unique_ptr<pxr_plan> P(new pxr_plan());
    P->ctx = ctx;
    P->params = *params;
    if ((rc = check_params(params, &P->dp))) return rc;
    P->E = n_events;
    P->hit_off.assign(hit_offsets, hit_offsets + n_events + 1);
    if (P->hit_off[0] != 0) return fail(PXR_EINVAL, "hit_offsets[0] must be 0");
    for (uint32_t e = 0; e < n_events; ++e) {
        if (P->hit_off[e + 1] < P->hit_off[e]) return fail(PXR_EINVAL, "hit_offsets not monotone");
        if (P->hit_off[e + 1] - P->hit_off[e] > kLocalMask) return fail(PXR_EINVAL, "event too large");
    }
    P->N = P->hit_off[n_events];
    P->db.x = x;
    P->db.y = y;
    P->db.z = z;
    P->db.layer = layer;
    cudaStream_t s = ctx->stream;
    // per-layer counts, read back once to size the per-event capacities
    std::vector<uint32_t> lcount((size_t)n_events * (kMaxLayers + 1));
    {
        const size_t cnt_at = (4 * (size_t)(n_events + 1) + 255) & ~size_t(255);
        const size_t bytes = cnt_at + 4 * lcount.size();
        char *tmp = ctx->arena.alloc(bytes);
        if (!tmp) return fail(PXR_EAGAIN, "arena full");
        uint32_t *d_off = (uint32_t *)tmp;
        uint32_t *d_cnt = (uint32_t *)(tmp + cnt_at);
        cudaError_t e1 = cudaMemcpyAsync(d_off, P->hit_off.data(), 4 * (n_events + 1),
                                         cudaMemcpyHostToDevice, s);
        launch_layer_count(d_off, layer, n_events, P->dp.n_layers, d_cnt, s, ctx->sms);
        cudaError_t e2 = cudaMemcpyAsync(lcount.data(), d_cnt, 4 * lcount.size(),
                                         cudaMemcpyDeviceToHost, s);
        cudaError_t e3 = cudaStreamSynchronize(s);
        ctx->arena.release(tmp, bytes);
        CK(e1);
        CK(e2);
        CK(e3);
    }
    if ((rc = plan_size(P.get(), lcount.data(), false))) return rc;
    P->region = ctx->arena.alloc(P->off.total);
    if (!P->region) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "plan needs %.1f MB, arena has no free block that large",
                      P->off.total / 1e6);
        return fail(P->off.total > ctx->arena.size ? PXR_ENOMEM : PXR_EAGAIN, msg);
    }
    plan_bind(P.get());
    // small host-computed arrays
    {
        const size_t e1 = 4 * (n_events + 1);
        std::vector<char> head(P->off.head_end, 0);
        std::memcpy(head.data() + P->off.hit_off, P->hit_off.data(), e1);
        std::memcpy(head.data() + P->off.cell_off, P->cell_off.data(), e1);
        std::memcpy(head.data() + P->off.edge_off, P->edge_off.data(), e1);
        std::memcpy(head.data() + P->off.tup_off, P->tup_off.data(), e1);
        fill_chunks(P.get(), head.data());
        size_t a = P->off.hit_off;
        CK(cudaMemcpyAsync(P->region + a, head.data() + a, P->off.head_end - a,
                           cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    }
    P->use_graph = use_graph != 0;
    if ((rc = plan_finish_setup(P.get()))) return rc;
    if (P->use_graph) {
        cudaStream_t cs;
        CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g;
        cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            rc = plan_enqueue(P.get(), cs, true);
            ce = cudaStreamEndCapture(cs, &g);
        }
        cudaStreamDestroy(cs);
        if (rc) return rc;
        CK(ce);
        ce = cudaGraphInstantiate(&P->graph, g, 0);
        cudaGraphDestroy(g);
        CK(ce);
    }
    {
        std::lock_guard<std::mutex> g(ctx->plans_mu);
        ctx->plans.insert(P.get());
    }
    *out = P.release();
    return PXR_OK;
}

extern "C" int pxr_plan_run(pxr_plan *P, void *stream)
{
    if (!P) return fail(PXR_EINVAL, "null plan");
    int rc = set_device(P->ctx);
    if (rc) return rc;
    cudaStream_t s = stream ? (cudaStream_t)stream : P->ctx->stream;
    if (P->use_graph) {
        CK(cudaGraphLaunch(P->graph, s));
    } else if ((rc = plan_enqueue(P, s))) {
        return rc;
    }
    CK(cudaEventRecord(P->ev_done, s));
    P->last_stream = s;
    P->has_run = true;
    return PXR_OK;
}

extern "C" int pxr_plan_launches(const pxr_plan *P) { return P ? plan_launches(P) : 0; }

extern "C" int pxr_plan_count_ca_tests(pxr_plan *P, void *stream, uint64_t *counts)
{
    if (!P || !counts) return fail(PXR_EINVAL, "null argument");
    int rc = set_device(P->ctx);
    if (rc) return rc;
    cudaStream_t s = stream ? (cudaStream_t)stream : P->ctx->stream;
    DevBatch b = P->db;
    b.ca_tests = (unsigned long long *)(P->region + P->off.ca_tests);
    CK(cudaMemsetAsync(b.ca_tests, 0, 16, s));
    if ((rc = plan_enqueue(P, s, false, &b))) return rc;
    CK(cudaMemcpyAsync(counts, b.ca_tests, 16, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaEventRecord(P->ev_done, s));
    P->last_stream = s;
    P->has_run = true;
    return PXR_OK;
}

extern "C" int pxr_plan_counts(pxr_plan *P, uint32_t *out)
{
    if (!P || !out) return fail(PXR_EINVAL, "null argument");
    if (!P->has_run) return fail(PXR_EINVAL, "plan has not run");
    int rc = set_device(P->ctx);
    if (rc) return rc;
    CK(cudaEventSynchronize(P->ev_done));
    CK(cudaMemcpy(out, P->db.cnt, 4 * (size_t)kReportedCounters * P->E, cudaMemcpyDeviceToHost));
    return PXR_OK;
}

extern "C" int pxr_plan_stage_ms(pxr_plan *P, float *ms, int cap, int *n)
{
    if (!P || !ms || !n) return fail(PXR_EINVAL, "null argument");
    *n = 0;
    if (!P->has_run) return fail(PXR_EINVAL, "plan has not run");
    CK(cudaEventSynchronize(P->ev_done));
    for (int k = 0; k < 5 && k < cap; ++k) {
        float v = 0.f;
        CK(cudaEventElapsedTime(&v, P->ev_stage[k], P->ev_stage[k + 1]));
        ms[k] = v;
        *n = k + 1;
    }
    return PXR_OK;
}

extern "C" void pxr_plan_destroy(pxr_plan *P)
{
    if (!P) return;
    {
        std::lock_guard<std::mutex> g(P->ctx->plans_mu);
        P->ctx->plans.erase(P);
    }
    if (P->has_run) cudaEventSynchronize(P->ev_done);
    plan_free(P);
}

// ---- readback -----------------------------------------------------------------------------
// The tracks of one event (canonical order: the device writes them so) and its vertices, as
// arrays somewhere in host memory.
struct TrackSrc {
    size_t n = 0, nv = 0;
    const uint8_t *nh = nullptr;
    const uint32_t *hits = nullptr;
    const double *pt = nullptr, *phi = nullptr, *cot = nullptr, *dxy = nullptr, *dz = nullptr,
                 *chi2 = nullptr;
    const int8_t *q = nullptr, *st = nullptr;
    const uint8_t *ql = nullptr;
    const double *cov = nullptr;         // 15 per track, or null (covariance not computed)
    const int32_t *vtx = nullptr;        // vertex of each track, or null (no vertex finding)
    const double *vz = nullptr, *verr = nullptr, *vpt2 = nullptr;
    const uint32_t *vn = nullptr;
};

// Host copies of one event's results (the plan path reads them back into these).
struct HostTracks {
    std::vector<uint8_t> nh;
    std::vector<uint32_t> hits;
    std::vector<double> pt, phi, cot, dxy, dz, chi2;
    std::vector<int8_t> q, st;
    std::vector<uint8_t> ql;
    std::vector<double> cov;             // 15 per track, or empty (covariance not computed)
    std::vector<int32_t> vtx;            // vertex of each track, or empty (no vertex finding)
    std::vector<double> vz, verr, vpt2;  // the event's vertices
    std::vector<uint32_t> vn;
    TrackSrc src() const
    {
        TrackSrc t;
        t.n = nh.size();
        t.nv = vz.size();
        t.nh = nh.data(); t.hits = hits.data(); t.pt = pt.data(); t.phi = phi.data();
        t.cot = cot.data(); t.dxy = dxy.data(); t.dz = dz.data(); t.chi2 = chi2.data();
        t.q = q.data(); t.st = st.data(); t.ql = ql.data();
        t.cov = cov.empty() ? nullptr : cov.data();
        t.vtx = vtx.empty() ? nullptr : vtx.data();
        t.vz = vz.data(); t.verr = verr.data(); t.vpt2 = vpt2.data(); t.vn = vn.data();
        return t;
    }
};

// Copy h into out's arrays at track row r0 and vertex row v0, one copy per array (no capacity
// check).  A covariance that was not computed reads as NaN, a missing vertex index as -1.
static void copy_tracks(const TrackSrc &h, pxr_tracks *out, size_t r0, size_t v0)
{
    const size_t n = h.n, nv = h.nv;
    auto cp = [](void *dst, size_t row, const void *src, size_t sz, size_t cnt) {
        if (dst && cnt) std::memcpy((char *)dst + sz * row, src, sz * cnt);
    };
    cp(out->vtx_z, v0, h.vz, 8, nv);
    cp(out->vtx_z_err, v0, h.verr, 8, nv);
    cp(out->vtx_sum_pt2, v0, h.vpt2, 8, nv);
    cp(out->vtx_n_tracks, v0, h.vn, 4, nv);
    cp(out->n_hits, r0, h.nh, 1, n);
    cp(out->hit_idx, r0, h.hits, 4 * kMaxHits, n);
    cp(out->pt, r0, h.pt, 8, n);
    cp(out->phi, r0, h.phi, 8, n);
    cp(out->cot_theta, r0, h.cot, 8, n);
    cp(out->dxy, r0, h.dxy, 8, n);
    cp(out->dz, r0, h.dz, 8, n);
    cp(out->chi2, r0, h.chi2, 8, n);
    cp(out->charge, r0, h.q, 1, n);
    cp(out->fit_status, r0, h.st, 1, n);
    cp(out->quality, r0, h.ql, 1, n);
    if (out->cov) {
        if (!h.cov) std::fill(out->cov + 15 * r0, out->cov + 15 * (r0 + n), NAN);
        else cp(out->cov, r0, h.cov, 15 * sizeof(double), n);
    }
    if (out->vertex) {
        if (!h.vtx) std::fill(out->vertex + r0, out->vertex + r0 + n, -1);
        else cp(out->vertex, r0, h.vtx, 4, n);
    }
}

// The tracks of one event into out (capacity checked).
static int emit_tracks(const TrackSrc &h, int32_t status, pxr_tracks *out)
{
    out->n_tracks = (uint32_t)h.n;
    out->n_vertices = (uint32_t)h.nv;
    out->status = status;
    if (h.n > out->capacity || h.nv > out->capacity)
        return fail(PXR_ETRUNC, "track capacity too small");
    copy_tracks(h, out, 0, 0);
    return PXR_OK;
}

static int32_t flags_status(uint32_t f)
{
    if (f & F_BOUNDS) return PXR_EBOUNDS;
    return (f & (F_CELLS | F_EDGES | F_TUPLES | F_VERTS)) ? PXR_EOVERFLOW
           : (f & F_LAYER)                                 ? PXR_EINVAL
                                                           : PXR_OK;
}

template <typename T>
static int d2h(std::vector<T> &v, const void *src, size_t n)
{
    v.resize(n);
    if (n) CK(cudaMemcpy(v.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost));
    return PXR_OK;
}

extern "C" int pxr_plan_tracks(pxr_plan *P, uint32_t e, pxr_tracks *out)
{
    if (!P || !out || e >= P->E) return fail(PXR_EINVAL, "bad plan, event or output");
    if (!P->has_run) return fail(PXR_EINVAL, "plan has not run");
    int rc = set_device(P->ctx);
    if (rc) return rc;
    CK(cudaEventSynchronize(P->ev_done));
    uint32_t ab[2], flags;
    CK(cudaMemcpy(ab, P->db.out_evt + e, 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&flags, P->db.cnt + C_FLAGS * P->E + e, 4, cudaMemcpyDeviceToHost));
    size_t a = ab[0], n = ab[1] - ab[0];
    HostTracks h;
    if ((rc = d2h(h.nh, P->db.o_nh + a, n)) || (rc = d2h(h.hits, P->db.o_hits + a * kMaxHits, n * kMaxHits)) ||
        (rc = d2h(h.pt, P->db.o_pt + a, n)) || (rc = d2h(h.phi, P->db.o_phi + a, n)) ||
        (rc = d2h(h.cot, P->db.o_cot + a, n)) || (rc = d2h(h.dxy, P->db.o_dxy + a, n)) ||
        (rc = d2h(h.dz, P->db.o_dz + a, n)) || (rc = d2h(h.chi2, P->db.o_chi2 + a, n)) ||
        (rc = d2h(h.q, P->db.o_q + a, n)) || (rc = d2h(h.st, P->db.o_status + a, n)) ||
        (rc = d2h(h.ql, P->db.o_ql + a, n)))
        return rc;
    if (P->dp.cov && (rc = d2h(h.cov, P->db.o_cov + 15 * a, 15 * n))) return rc;
    if (P->dp.vtx) {
        uint32_t nv = 0;
        CK(cudaMemcpy(&nv, P->db.cnt + C_VERTS * P->E + e, 4, cudaMemcpyDeviceToHost));
        if ((rc = d2h(h.vtx, P->db.o_vtx + a, n)) || (rc = d2h(h.vz, P->db.v_z + a, nv)) ||
            (rc = d2h(h.verr, P->db.v_err + a, nv)) || (rc = d2h(h.vpt2, P->db.v_pt2 + a, nv)) ||
            (rc = d2h(h.vn, P->db.v_n + a, nv)))
            return rc;
    }
    return emit_tracks(h.src(), flags_status(flags), out);
}

// Debug content of one event of a plan region (also used by the serving path).
static int region_debug(pxr_plan *P, uint32_t e, int what, uint32_t *buf, uint32_t cap,
                        uint32_t *n_out)
{
    CK(cudaEventSynchronize(P->ev_done));
    const DevBatch &b = P->db;
    uint32_t cnt[kCounters];
    for (int k = 0; k < kCounters; ++k)
        CK(cudaMemcpy(&cnt[k], b.cnt + (size_t)k * P->E + e, 4, cudaMemcpyDeviceToHost));
    const uint32_t h0 = P->hit_off[e], nh = P->hit_off[e + 1] - h0;
    std::vector<uint32_t> meta;
    int rc;
    if ((rc = d2h(meta, b.hmeta + h0, nh))) return rc;
    auto loc = [&](uint32_t pos) { return meta[pos - h0] & kLocalMask; };
    const uint32_t c0 = P->cell_off[e];
    const uint32_t nc = std::min(cnt[C_SLOTS], P->cell_off[e + 1] - c0);   // slots, holes included
    std::vector<uint32_t> out;
    if (what == 0 || what == 1) {
        std::vector<uint32_t> co, ci(nc, kNone);
        if ((rc = d2h(co, b.cell_out + c0, nc))) return rc;
        // the inner hit of each entry: the item (inner hit, pair slot) whose entry run holds it
        std::vector<uint4> items;
        if ((rc = d2h(items, b.item + (size_t)h0 * kMaxOut, (size_t)nh * kMaxOut))) return rc;
        for (uint32_t h = 0; h < nh; ++h) {
            const uint32_t L = meta[h] >> kLocalBits;
            if (L >= P->dp.n_layers) continue;
            for (uint32_t sl = 0; sl < P->dp.n_out[L]; ++sl) {
                const uint4 it = items[(size_t)h * kMaxOut + sl];
                for (uint32_t c = it.x - c0; c < it.x - c0 + it.y && c < nc; ++c) ci[c] = h0 + h;
            }
        }
        if (what == 0) {
            for (uint32_t c = 0; c < nc; ++c) {
                if (co[c] == kNone || ci[c] == kNone) continue;  // candidate that failed the cut
                out.push_back(loc(ci[c]));
                out.push_back(loc(co[c]));
            }
        } else {
            std::vector<uint32_t> live, roots;
            std::vector<uint2> hd;
            if ((rc = d2h(hd, b.nbr_head + c0, nc))) return rc;
            const uint32_t g0 = P->edge_off[e];
            const uint32_t ng = std::min(cnt[C_EDGES], P->edge_off[e + 1] - g0);
            std::vector<uint32_t> nb;
            if ((rc = d2h(nb, b.nbr + g0, ng))) return rc;
            // edge lists are valid for reached cells (live bit) and for root cells with edges
            // (the root list); other counts are not cleared
            if ((rc = d2h(live, b.live + c0 / 32, (nc + 31) / 32))) return rc;
            const uint32_t nr = std::min(cnt[C_ROOTS], P->edge_off[e + 1] - g0);
            if ((rc = d2h(roots, b.root_list + g0, nr))) return rc;
            std::vector<uint8_t> valid(nc, 0);
            for (uint32_t c = 0; c < nc; ++c)
                valid[c] = ci[c] != kNone && ((live[c / 32] >> (c % 32)) & 1u);
            for (uint32_t A : roots) valid[A - c0] = 1;
            for (uint32_t c = 0; c < nc; ++c)
                for (uint32_t k = 0; valid[c] && k < hd[c].y; ++k) {
                    uint32_t B = nb[hd[c].x - g0 + k] - c0;
                    out.push_back(loc(ci[c]));
                    out.push_back(loc(co[c]));
                    out.push_back(loc(co[B]));
                }
        }
    } else if (what == 2) {
        const uint32_t t0 = P->tup_off[e];
        const uint32_t nt = std::min(cnt[C_TUPLES], P->tup_off[e + 1] - t0);
        std::vector<uint32_t> th;
        if ((rc = d2h(th, b.tup_hits + (size_t)t0 * kMaxHits, (size_t)nt * kMaxHits))) return rc;
        for (uint32_t t = 0; t < nt; ++t)
            for (int k = 0; k < kMaxHits; ++k) {
                uint32_t v = th[(size_t)t * kMaxHits + k];
                out.push_back(v == kNone ? kNone : loc(v));
            }
    } else {
        return fail(PXR_EINVAL, "what must be 0, 1 or 2");
    }
    const uint32_t per = what == 0 ? 2 : what == 1 ? 3 : kMaxHits;
    *n_out = (uint32_t)(out.size() / per);
    if (out.size() > cap) return fail(PXR_ETRUNC, "debug buffer too small");
    if (!out.empty()) std::memcpy(buf, out.data(), 4 * out.size());
    return PXR_OK;
}

extern "C" int pxr_plan_debug(pxr_plan *P, uint32_t e, int what, uint32_t *buf, uint32_t cap,
                              uint32_t *n)
{
    if (!P || !n || e >= P->E || (cap && !buf)) return fail(PXR_EINVAL, "bad argument");
    if (!P->has_run) return fail(PXR_EINVAL, "plan has not run");
    int rc = set_device(P->ctx);
    if (rc) return rc;
    return region_debug(P, e, what, buf, cap, n);
}

// ---- fit-only path --------------------------------------------------------------------------
extern "C" int pxr_fit_batch(pxr_ctx *ctx, uint32_t m, const uint8_t *nh, const float *x,
                             const float *y, const float *z, const uint16_t *layer,
                             uint32_t stride, const pxr_params *params, double *pt, double *phi,
                             double *cot_theta, double *dxy, double *dz, double *chi2,
                             int8_t *charge, int8_t *fit_status, void *stream)
{
    if (!ctx || !nh || !x || !y || !z || !layer || !pt || !phi || !cot_theta || !dxy || !dz ||
        !chi2 || !charge || !fit_status || stride < 3 || stride > 64)
        return fail(PXR_EINVAL, "bad argument");
    DevParams dp;
    int rc = check_params(params, &dp);
    if (rc) return rc;
    if ((rc = set_device(ctx))) return rc;
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
    launch_fit_batch(m, nh, x, y, z, layer, stride, dp, pt, phi, cot_theta, dxy, dz, chi2, charge,
                     fit_status, s, ctx->sms);
    CK(cudaGetLastError());
    return PXR_OK;
}

// ------------------------------------------------------------------------------------------
// serving
// ------------------------------------------------------------------------------------------
struct Ticket {
    uint64_t id = 0;
    int state = 0;                       // 0 pending, 1 running, 2 done
    // the event's hits in its submission's block: x, y, z (float) then layer (uint16), nt
    // values of each for the whole submission, the event's nt from in_a
    std::shared_ptr<PinnedBlock> in;
    size_t in_nt = 0, in_a = 0;
    uint32_t n = 0;
    const float *x() const { return reinterpret_cast<const float *>(in->p) + in_a; }
    const float *y() const { return x() + in_nt; }
    const float *z() const { return x() + 2 * in_nt; }
    const uint16_t *layer() const
    {
        return reinterpret_cast<const uint16_t *>(reinterpret_cast<const float *>(in->p) +
                                                  3 * in_nt) + in_a;
    }
    uint32_t lcount[kMaxLayers + 1] = {};
    pxr_params params{};
    size_t bytes = 0;
    std::shared_ptr<Batch> batch;        // kept for pxr_fetch_debug
    uint32_t index = 0;
    int32_t status = PXR_OK;
    std::shared_ptr<PinnedBlock> out;    // the batch's results, which res points into
    TrackSrc res;
};

// Pinned host buffers of one in-flight slot, grown on demand and reused.
struct Pinned {
    char *p = nullptr;
    size_t n = 0;
    bool reserve(size_t bytes)
    {
        if (bytes <= n) return true;
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
        size_t want = std::max(bytes, size_t(1) << 20);
        if (cudaMallocHost((void **)&p, want) != cudaSuccess) return false;
        n = want;
        return true;
    }
    ~Pinned()
    {
        if (p) cudaFreeHost(p);
    }
};

struct Batch {
    pxr_ctx *ctx = nullptr;
    pxr_plan *plan = nullptr;
    std::vector<uint64_t> ids;           // tickets of the batch, in event order
    int slot = 0;
    int state = 0;                       // 1 launched, 2 copying, 3 done
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_counts = nullptr, ev_data = nullptr;
    size_t reserved = 0;
    uint32_t total = 0;
    std::vector<std::shared_ptr<PinnedBlock>> inputs;   // until the hits are on the device
    std::shared_ptr<PinnedBlock> results;               // the tracks, read by the fetches
    size_t o_nh = 0, o_hits = 0, o_pt = 0, o_phi = 0, o_cot = 0, o_dxy = 0, o_dz = 0,
           o_chi2 = 0, o_q = 0, o_st = 0, o_ql = 0, o_cov = 0, o_vtx = 0, v_z = 0, v_err = 0,
           v_pt2 = 0, v_n = 0;
    ~Batch()
    {
        if (ev_counts) cudaEventDestroy(ev_counts);
        if (ev_data) cudaEventDestroy(ev_data);
        if (plan) plan_free(plan);
    }
};

struct SlotBuffers {
    Pinned head, evt;
};

static size_t event_bytes(const pxr_params &p, const DevParams &dp, const uint32_t *lcount,
                          uint32_t n)
{
    EventCaps c = event_caps(p, dp.nb, lcount, n);
    PlanOffsets o = plan_layout(1, n, c.cells, c.edges, c.tuples, dp, true);
    return o.total + 64 * 256;  // alignment slack of the shared batch layout
}

static cudaStream_t slot_stream(pxr_ctx *ctx, int slot)
{
    return ctx->cfg.stream ? (cudaStream_t)ctx->cfg.stream : ctx->slot_stream[slot];
}

// Build and launch one batch (scheduler thread, ctx->mu held).
// Releases a held lock for the scope (the scheduler's host copies run without ctx->mu, so that
// submissions and fetches proceed meanwhile).
struct Unlocked {
    std::unique_lock<std::mutex> &lk;
    explicit Unlocked(std::unique_lock<std::mutex> &l) : lk(l) { lk.unlock(); }
    ~Unlocked() { lk.lock(); }
};

static int launch_batch(pxr_ctx *ctx, std::unique_lock<std::mutex> &lk,
                        std::vector<std::shared_ptr<Ticket>> &items, int slot,
                        std::shared_ptr<Batch> &out)
{
    Range range("pxr.batch.launch");
    auto B = std::make_shared<Batch>();
    B->ctx = ctx;
    B->slot = slot;
    const uint32_t E = (uint32_t)items.size();
    auto *P = new pxr_plan();
    B->plan = P;
    P->ctx = ctx;
    P->params = items[0]->params;
    int rc = check_params(&P->params, &P->dp);
    if (rc) return rc;
    P->E = E;
    P->hit_off.assign(E + 1, 0);
    std::vector<uint32_t> lcount((size_t)E * (kMaxLayers + 1));
    for (uint32_t e = 0; e < E; ++e) {
        P->hit_off[e + 1] = P->hit_off[e] + items[e]->n;
        std::memcpy(&lcount[(size_t)e * (kMaxLayers + 1)], items[e]->lcount,
                    sizeof(items[e]->lcount));
        B->reserved += items[e]->bytes;
        B->ids.push_back(items[e]->id);
    }
    P->N = P->hit_off[E];
    P->own_inputs = true;
    if ((rc = plan_size(P, lcount.data(), true))) return rc;
    SlotBuffers &sb = *ctx->slot_buf[slot];
    if (!sb.head.reserve(P->off.head_end) || !sb.evt.reserve(4 * (3 * (size_t)E + 1)))
        return fail(PXR_ENOMEM, "pinned host allocation failed");
    CK(cudaEventCreateWithFlags(&B->ev_counts, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&B->ev_data, cudaEventDisableTiming));
    if ((rc = plan_finish_setup(P))) return rc;
    P->region = ctx->arena.alloc(P->off.total);
    if (!P->region) return fail(PXR_EAGAIN, "arena fragmented");
    plan_bind(P);
    // the small arrays staged in the slot's pinned head, one H2D copy; the hits straight from
    // the submissions' pinned blocks, one copy per array for each run of events contiguous in
    // one block.  The batch's tickets are out of the pending queue and reach no other thread
    // before the batch is published
    {
    Unlocked unlocked(lk);
    char *h = sb.head.p;
    const size_t e1 = 4 * (E + 1);
    std::memcpy(h + P->off.hit_off, P->hit_off.data(), e1);
    std::memcpy(h + P->off.cell_off, P->cell_off.data(), e1);
    std::memcpy(h + P->off.edge_off, P->edge_off.data(), e1);
    std::memcpy(h + P->off.tup_off, P->tup_off.data(), e1);
    fill_chunks(P, h);
    cudaStream_t s = slot_stream(ctx, slot);
    B->stream = s;
    CK(cudaMemcpyAsync(P->region + P->off.hit_off, h + P->off.hit_off,
                       P->off.head_end - P->off.hit_off, cudaMemcpyHostToDevice, s));
    for (uint32_t e = 0; e < E;) {
        const Ticket &t = *items[e];
        uint32_t f = e + 1;
        while (f < E && items[f]->in == t.in && items[f]->in_a == items[f - 1]->in_a + items[f - 1]->n)
            ++f;
        const size_t a = P->hit_off[e], n = P->hit_off[f] - a;
        if (n) {
            CK(cudaMemcpyAsync(P->region + P->off.x + 4 * a, t.x(), 4 * n, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(P->region + P->off.y + 4 * a, t.y(), 4 * n, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(P->region + P->off.z + 4 * a, t.z(), 4 * n, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(P->region + P->off.layer + 2 * a, t.layer(), 2 * n,
                               cudaMemcpyHostToDevice, s));
        }
        if (B->inputs.empty() || B->inputs.back() != t.in) B->inputs.push_back(t.in);
        e = f;
    }
    if ((rc = plan_enqueue(P, s))) return rc;
    CK(cudaEventRecord(P->ev_done, s));
    P->has_run = true;
    P->last_stream = s;
    uint32_t *hev = (uint32_t *)sb.evt.p;
    CK(cudaMemcpyAsync(hev, P->db.out_evt, e1, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hev + E + 1, P->db.cnt + C_FLAGS * E, 4 * E, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hev + 2 * E + 1, P->db.cnt + C_VERTS * E, 4 * E, cudaMemcpyDeviceToHost,
                       s));
    CK(cudaEventRecord(B->ev_counts, s));
    }
    B->state = 1;
    for (uint32_t e = 0; e < E; ++e) {
        items[e]->state = 1;
        items[e]->index = e;
        items[e]->in.reset();                   // (the batch holds the blocks until the copies)
    }
    out = B;
    return PXR_OK;
}

// Advance one in-flight batch; returns true when it changed state.
static bool progress_batch(pxr_ctx *ctx, std::unique_lock<std::mutex> &lk,
                           const std::shared_ptr<Batch> &Bp)
{
    Batch &B = *Bp;
    pxr_plan *P = B.plan;
    cudaStream_t s = B.stream;
    SlotBuffers &sb = *ctx->slot_buf[B.slot];
    const uint32_t E = P->E;
    const uint32_t *hev = (const uint32_t *)sb.evt.p;
    if (B.state == 1 && cudaEventQuery(B.ev_counts) == cudaSuccess) {
        B.total = hev[E];
        size_t T = B.total;
        Layout L;
        B.o_nh = L.add(T);
        B.o_hits = L.add(4 * T * kMaxHits);
        B.o_pt = L.add(8 * T);
        B.o_phi = L.add(8 * T);
        B.o_cot = L.add(8 * T);
        B.o_dxy = L.add(8 * T);
        B.o_dz = L.add(8 * T);
        B.o_chi2 = L.add(8 * T);
        B.o_q = L.add(T);
        B.o_st = L.add(T);
        B.o_ql = L.add(T);
        B.o_cov = L.add(P->dp.cov ? 8 * 15 * (size_t)T : 0);
        const size_t tv = P->dp.vtx ? (size_t)T : 0;
        B.o_vtx = L.add(4 * tv);
        B.v_z = L.add(8 * tv);
        B.v_err = L.add(8 * tv);
        B.v_pt2 = L.add(8 * tv);
        B.v_n = L.add(4 * tv);
        // the results' pinned block (the fetches read it in place); the hits' blocks are done
        B.inputs.clear();
        {
            Unlocked unlocked(lk);
            B.results = pinned_block(ctx->pool, L.add(0) + 256);
        }
        bool ok = B.results != nullptr;
        const DevBatch &d = P->db;
        char *ho = ok ? B.results->p : nullptr;
        if (ok && T) {
            auto cp = [&](size_t off, const void *src, size_t bytes) {
                ok &= cudaMemcpyAsync(ho + off, src, bytes, cudaMemcpyDeviceToHost, s) == cudaSuccess;
            };
            cp(B.o_nh, d.o_nh, T);
            cp(B.o_hits, d.o_hits, 4 * T * kMaxHits);
            cp(B.o_pt, d.o_pt, 8 * T);
            cp(B.o_phi, d.o_phi, 8 * T);
            cp(B.o_cot, d.o_cot, 8 * T);
            cp(B.o_dxy, d.o_dxy, 8 * T);
            cp(B.o_dz, d.o_dz, 8 * T);
            cp(B.o_chi2, d.o_chi2, 8 * T);
            cp(B.o_q, d.o_q, T);
            cp(B.o_st, d.o_status, T);
            cp(B.o_ql, d.o_ql, T);
            if (P->dp.cov) cp(B.o_cov, d.o_cov, 8 * 15 * (size_t)T);
            if (P->dp.vtx) {
                cp(B.o_vtx, d.o_vtx, 4 * (size_t)T);
                cp(B.v_z, d.v_z, 8 * (size_t)T);
                cp(B.v_err, d.v_err, 8 * (size_t)T);
                cp(B.v_pt2, d.v_pt2, 8 * (size_t)T);
                cp(B.v_n, d.v_n, 4 * (size_t)T);
            }
        }
        ok &= cudaEventRecord(B.ev_data, s) == cudaSuccess;
        if (!ok) ctx->sched_error = "device-to-host copy failed";
        B.state = 2;
        return true;
    }
    if (B.state == 2 && cudaEventQuery(B.ev_data) == cudaSuccess) {
        // each event's results: a view of the batch's pinned block (tracks in canonical order)
        const char *ho = B.results ? B.results->p : nullptr;
        std::vector<std::shared_ptr<Ticket>> ts(E);
        for (uint32_t e = 0; e < E; ++e) {
            auto it = ctx->tickets.find(B.ids[e]);
            if (it == ctx->tickets.end()) continue;
            ts[e] = it->second;
            Ticket &t = *ts[e];
            const size_t a = hev[e];
            TrackSrc &r = t.res;
            r.n = hev[e + 1] - a;
            r.nv = P->dp.vtx ? hev[2 * E + 1 + e] : 0;
            if (ho) {
                auto at = [&](size_t off, size_t sz) { return ho + off + sz * a; };
                r.nh = (const uint8_t *)at(B.o_nh, 1);
                r.hits = (const uint32_t *)at(B.o_hits, 4 * kMaxHits);
                r.pt = (const double *)at(B.o_pt, 8);
                r.phi = (const double *)at(B.o_phi, 8);
                r.cot = (const double *)at(B.o_cot, 8);
                r.dxy = (const double *)at(B.o_dxy, 8);
                r.dz = (const double *)at(B.o_dz, 8);
                r.chi2 = (const double *)at(B.o_chi2, 8);
                r.q = (const int8_t *)at(B.o_q, 1);
                r.st = (const int8_t *)at(B.o_st, 1);
                r.ql = (const uint8_t *)at(B.o_ql, 1);
                r.cov = P->dp.cov ? (const double *)at(B.o_cov, 15 * sizeof(double)) : nullptr;
                r.vtx = P->dp.vtx ? (const int32_t *)at(B.o_vtx, 4) : nullptr;
                r.vz = (const double *)at(B.v_z, 8);
                r.verr = (const double *)at(B.v_err, 8);
                r.vpt2 = (const double *)at(B.v_pt2, 8);
                r.vn = (const uint32_t *)at(B.v_n, 4);
            } else {
                r.n = r.nv = 0;
            }
            t.out = B.results;
        }
        for (uint32_t e = 0; e < E; ++e) {
            if (!ts[e]) continue;
            Ticket &t = *ts[e];
            t.status = flags_status(hev[E + 1 + e]);
            if (!B.results && hev[e + 1] > hev[e]) t.status = PXR_ENOMEM;   // (no pinned memory)
            t.state = 2;
            if (ctx->cfg.keep_debug) t.batch = Bp;
            ctx->done_q.push_back(t.id);
        }
        B.state = 3;
        if (!ctx->cfg.keep_debug) {
            ctx->arena.release(P->region, P->off.total);
            P->region = nullptr;
        }
        ctx->reserved -= B.reserved;
        ctx->cv_done.notify_all();
        return true;
    }
    return false;
}

static void scheduler(pxr_ctx *ctx)
{
    cudaSetDevice(ctx->cfg.device);
    std::unique_lock<std::mutex> lk(ctx->mu);
    while (true) {
        bool moved = false;
        for (size_t k = 0; k < ctx->inflight.size();) {
            moved |= progress_batch(ctx, lk, ctx->inflight[k]);
            if (ctx->inflight[k]->state == 3) ctx->inflight.erase(ctx->inflight.begin() + k);
            else ++k;
        }
        const uint32_t max_inflight = ctx->cfg.max_inflight;
        while (!ctx->pending.empty() && ctx->inflight.size() < max_inflight) {
            // one batch: FIFO events with identical parameters, within the batch caps
            std::vector<std::shared_ptr<Ticket>> items;
            size_t hits = 0;
            const pxr_params p0 = ctx->tickets[ctx->pending.front()]->params;
            while (!ctx->pending.empty() && items.size() < ctx->cfg.max_batch_events) {
                auto &t = ctx->tickets[ctx->pending.front()];
                if (std::memcmp(&t->params, &p0, sizeof(pxr_params)) != 0) break;
                if (!items.empty() && hits + t->n > ctx->cfg.max_batch_hits) break;
                hits += t->n;
                items.push_back(t);
                ctx->pending.pop_front();
            }
            // the lowest slot (stream and pinned staging buffers) no batch in flight holds
            int slot = 0;
            for (bool taken = true; taken; slot += taken) {
                taken = false;
                for (auto &b : ctx->inflight) taken |= b->slot == slot;
            }
            std::shared_ptr<Batch> B;
            int rc = launch_batch(ctx, lk, items, slot, B);
            if (rc == PXR_EAGAIN && !ctx->inflight.empty()) {
                // arena fragmented by the batch in flight: retry after it completes
                for (auto it = items.rbegin(); it != items.rend(); ++it)
                    ctx->pending.push_front((*it)->id);
                break;
            }
            if (rc != PXR_OK) {
                ctx->sched_error = g_err;
                for (auto &t : items) {
                    t->state = 2;
                    t->status = rc == PXR_EAGAIN ? PXR_ENOMEM : rc;
                    ctx->reserved -= t->bytes;
                    ctx->done_q.push_back(t->id);
                }
                ctx->cv_done.notify_all();
                continue;
            }
            ctx->inflight.push_back(B);
            moved = true;
        }
        if (ctx->stop && ctx->pending.empty() && ctx->inflight.empty()) break;
        if (!moved) {
            if (ctx->inflight.empty() && ctx->pending.empty() && !ctx->stop)
                ctx->cv_sched.wait(lk);
            else
                ctx->cv_sched.wait_for(lk, std::chrono::microseconds(20));
        }
    }
}

extern "C" int pxr_create(const pxr_config *cfg, pxr_ctx **out)
{
    if (!cfg || !out) return fail(PXR_EINVAL, "null argument");
    std::unique_ptr<pxr_ctx> ctx(new pxr_ctx());
    ctx->cfg = *cfg;
    if (!ctx->cfg.mem_budget_bytes) ctx->cfg.mem_budget_bytes = size_t(2) << 30;
    if (!ctx->cfg.max_batch_events) ctx->cfg.max_batch_events = 256;
    if (!ctx->cfg.max_batch_hits) ctx->cfg.max_batch_hits = 4u << 20;
    if (!ctx->cfg.max_inflight) ctx->cfg.max_inflight = 2;
    if (ctx->cfg.max_inflight > kMaxSlots) ctx->cfg.max_inflight = kMaxSlots;
    CK(cudaSetDevice(ctx->cfg.device));
    CK(cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->cfg.device));
    int major = 0, minor = 0;
    CK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, ctx->cfg.device));
    CK(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, ctx->cfg.device));
    if (major != 10 || minor != 3)
        return fail(PXR_EINVAL, "this library is built for sm_103a (GB300) only");
    char *arena = (char *)cfg->arena;
    if (!arena) {
        CK(cudaMalloc((void **)&arena, ctx->cfg.mem_budget_bytes));
        ctx->own_arena = true;
    }
    ctx->arena.init(arena, ctx->cfg.mem_budget_bytes);
    if (cfg->stream) {
        ctx->stream = (cudaStream_t)cfg->stream;
    } else {
        CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
    }
    for (auto &s : ctx->slot_stream) CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    for (auto &b : ctx->slot_buf) b.reset(new SlotBuffers());
    CK(init_kernels());
    pxr_ctx *c = ctx.get();
    ctx->sched = std::thread(scheduler, c);
    *out = ctx.release();
    return PXR_OK;
}

extern "C" void pxr_destroy(pxr_ctx *ctx)
{
    if (!ctx) return;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->stop = true;
        ctx->cv_sched.notify_all();
    }
    if (ctx->sched.joinable()) ctx->sched.join();
    cudaSetDevice(ctx->cfg.device);
    {
        // plans the caller did not destroy go with the context (their memory is in its arena)
        std::lock_guard<std::mutex> g(ctx->plans_mu);
        for (pxr_plan *P : ctx->plans) {
            if (P->has_run) cudaEventSynchronize(P->ev_done);
            plan_free(P);
        }
        ctx->plans.clear();
    }
    ctx->tickets.clear();
    ctx->inflight.clear();
    for (auto &s : ctx->slot_stream)
        if (s) cudaStreamDestroy(s);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    if (ctx->own_arena && ctx->arena.base) cudaFree(ctx->arena.base);
    delete ctx;
}

// Host threads for a copy or check of `work` units (a few for large inputs).
static uint32_t host_threads(size_t work, size_t per_thread)
{
    const uint32_t hw = std::max(1u, std::thread::hardware_concurrency() / 2);
    return (uint32_t)std::max<size_t>(1, std::min<size_t>(std::min(8u, hw), work / per_thread));
}

// n_events events, hits back to back in the caller's arrays (event e: [off[e], off[e+1])): one
// pinned block receives all of them (x, y, z, layer), the events are checked and counted per
// layer, and admitted together (all or none).
static int submit_many(pxr_ctx *ctx, uint32_t n_events, const uint32_t *off, const float *x,
                       const float *y, const float *z, const uint16_t *layer,
                       const pxr_params *params, uint64_t *tickets)
{
    DevParams dp;
    int rc = check_params(params, &dp);
    if (rc) return rc;
    if (n_events == 0) return PXR_OK;
    const size_t nt = off[n_events] - off[0];
    for (uint32_t e = 0; e < n_events; ++e) {
        if (off[e + 1] < off[e]) return fail(PXR_EINVAL, "hit offsets must not decrease");
        if (off[e + 1] - off[e] > kLocalMask) return fail(PXR_EINVAL, "too many hits in one event");
    }
    auto blk = pinned_block(ctx->pool, 14 * nt + 64);
    if (!blk) return fail(PXR_ENOMEM, "pinned host allocation failed");
    float *bx = reinterpret_cast<float *>(blk->p);
    uint16_t *bl = reinterpret_cast<uint16_t *>(bx + 3 * nt);
    const float *sx = x + off[0], *sy = y + off[0], *sz = z + off[0];
    const uint16_t *sl = layer + off[0];
    std::vector<std::shared_ptr<Ticket>> ts(n_events);
    std::atomic<int> bad{0};
    // the copy and the checks, split over a few host threads by events
    auto work = [&](uint32_t w, uint32_t nw) {
        const uint32_t e0 = (uint32_t)((uint64_t)n_events * w / nw);
        const uint32_t e1 = (uint32_t)((uint64_t)n_events * (w + 1) / nw);
        if (e0 == e1) return;
        const size_t a = off[e0] - off[0], n = off[e1] - off[e0];
        std::memcpy(bx + a, sx + a, 4 * n);
        std::memcpy(bx + nt + a, sy + a, 4 * n);
        std::memcpy(bx + 2 * nt + a, sz + a, 4 * n);
        std::memcpy(bl + a, sl + a, 2 * n);
        for (uint32_t e = e0; e < e1; ++e) {
            auto t = std::make_shared<Ticket>();
            t->in = blk;
            t->in_nt = nt;
            t->in_a = off[e] - off[0];
            t->n = off[e + 1] - off[e];
            bool finite = true;
            uint32_t bad_layer = 0;
            uint32_t lc[4][kMaxLayers + 1] = {};
            const float *ex = t->x(), *ey = t->y(), *ez = t->z();
            const uint16_t *el = t->layer();
            for (uint32_t h = 0; h < t->n; ++h) {
                finite &= std::isfinite(ex[h]) & std::isfinite(ey[h]) & std::isfinite(ez[h]);
                const uint16_t l = el[h];
                bad_layer |= l >= params->n_layers;
                lc[h & 3][l < kMaxLayers ? l : kMaxLayers]++;
            }
            if (!finite) { bad |= 1; continue; }
            if (bad_layer) { bad |= 2; continue; }
            for (int l = 0; l <= kMaxLayers; ++l)
                t->lcount[l] = lc[0][l] + lc[1][l] + lc[2][l] + lc[3][l];
            t->params = *params;
            t->bytes = event_bytes(*params, dp, t->lcount, t->n);
            if (t->bytes > ctx->arena.size) bad |= 4;
            ts[e] = t;
        }
    };
    {
        const uint32_t nth = host_threads(nt, 1u << 18);
        std::vector<std::thread> th;
        for (uint32_t w = 1; w < nth; ++w) th.emplace_back(work, w, nth);
        work(0, nth);
        for (auto &t : th) t.join();
    }
    if (bad & 1) return fail(PXR_EINVAL, "non-finite hit coordinate");
    if (bad & 2) return fail(PXR_EINVAL, "hit layer id >= n_layers");
    if (bad & 4) return fail(PXR_ENOMEM, "event exceeds the memory budget");
    size_t bytes = 0;
    for (auto &t : ts) bytes += t->bytes;
    std::lock_guard<std::mutex> g(ctx->mu);
    if (!ctx->sched_error.empty() && ctx->inflight.empty() && ctx->pending.empty()) {
        // a failed batch is reported through its tickets; the context stays usable
        ctx->sched_error.clear();
    }
    if (ctx->reserved + bytes > ctx->arena.size) return fail(PXR_EAGAIN, "memory budget full");
    for (uint32_t e = 0; e < n_events; ++e) {
        auto &t = ts[e];
        t->id = ctx->next_ticket++;
        ctx->tickets[t->id] = t;
        ctx->pending.push_back(t->id);
        tickets[e] = t->id;
    }
    ctx->reserved += bytes;
    ctx->cv_sched.notify_all();
    return PXR_OK;
}

extern "C" int pxr_submit_event(pxr_ctx *ctx, const float *x, const float *y, const float *z,
                                const uint16_t *layer, uint32_t n_hits, const pxr_params *params,
                                uint64_t *ticket)
{
    if (!ctx || !ticket || (n_hits && (!x || !y || !z || !layer)))
        return fail(PXR_EINVAL, "null argument");
    const uint32_t off[2] = {0, n_hits};
    return submit_many(ctx, 1, off, x, y, z, layer, params, ticket);
}

extern "C" int pxr_submit_events(pxr_ctx *ctx, uint32_t n_events, const uint32_t *hit_offsets,
                                 const float *x, const float *y, const float *z,
                                 const uint16_t *layer, const pxr_params *params,
                                 uint64_t *tickets)
{
    if (!ctx || (n_events && (!hit_offsets || !tickets)))
        return fail(PXR_EINVAL, "null argument");
    if (n_events && hit_offsets[n_events] > hit_offsets[0] && (!x || !y || !z || !layer))
        return fail(PXR_EINVAL, "null argument");
    return submit_many(ctx, n_events, hit_offsets, x, y, z, layer, params, tickets);
}

extern "C" int pxr_poll(pxr_ctx *ctx, uint64_t *done, uint32_t cap, uint32_t *n_done,
                        int timeout_us)
{
    if (!ctx || !n_done || (cap && !done)) return fail(PXR_EINVAL, "null argument");
    std::unique_lock<std::mutex> lk(ctx->mu);
    *n_done = 0;
    auto ready = [&] {
        return !ctx->done_q.empty() ||
               (ctx->pending.empty() && ctx->inflight.empty());
    };
    if (timeout_us < 0) ctx->cv_done.wait(lk, ready);
    else if (timeout_us > 0)
        ctx->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    while (*n_done < cap && !ctx->done_q.empty()) {
        done[(*n_done)++] = ctx->done_q.front();
        ctx->done_q.pop_front();
    }
    return PXR_OK;
}

extern "C" int pxr_fetch_tracks(pxr_ctx *ctx, uint64_t ticket, pxr_tracks *out)
{
    if (!ctx || !out) return fail(PXR_EINVAL, "null argument");
    std::shared_ptr<Ticket> t;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        auto it = ctx->tickets.find(ticket);
        if (it == ctx->tickets.end()) return fail(PXR_ENOTFOUND, "unknown ticket");
        t = it->second;
        if (t->state != 2) return fail(PXR_EBUSY, "event not finished");
    }
    int rc = emit_tracks(t->res, t->status, out);
    if (rc) return rc;
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->tickets.erase(ticket);
    return PXR_OK;
}

extern "C" int pxr_fetch_events(pxr_ctx *ctx, uint32_t n, const uint64_t *tickets,
                                uint32_t *track_offsets, uint32_t *vertex_offsets,
                                int32_t *event_status, pxr_tracks *out)
{
    if (!ctx || !out || (n && (!tickets || !track_offsets))) return fail(PXR_EINVAL, "null argument");
    std::vector<std::shared_ptr<Ticket>> ts(n);
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        for (uint32_t k = 0; k < n; ++k) {
            auto it = ctx->tickets.find(tickets[k]);
            if (it == ctx->tickets.end()) return fail(PXR_ENOTFOUND, "unknown ticket");
            if (it->second->state != 2) return fail(PXR_EBUSY, "event not finished");
            ts[k] = it->second;
        }
    }
    std::vector<uint32_t> voff(n + 1, 0);
    track_offsets[0] = 0;
    int32_t worst = PXR_OK;
    for (uint32_t k = 0; k < n; ++k) {
        track_offsets[k + 1] = track_offsets[k] + (uint32_t)ts[k]->res.n;
        voff[k + 1] = voff[k] + (uint32_t)ts[k]->res.nv;
        if (event_status) event_status[k] = ts[k]->status;
        if (worst == PXR_OK) worst = ts[k]->status;
    }
    if (vertex_offsets) std::memcpy(vertex_offsets, voff.data(), 4 * (size_t)(n + 1));
    out->n_tracks = n ? track_offsets[n] : 0;
    out->n_vertices = voff[n];
    out->status = worst;
    if (out->n_tracks > out->capacity || out->n_vertices > out->capacity)
        return fail(PXR_ETRUNC, "track capacity too small");
    // one copy per array and event, split over a few host threads by events
    auto work = [&](uint32_t w, uint32_t nw) {
        for (uint32_t k = (uint32_t)((uint64_t)n * w / nw); k < (uint64_t)n * (w + 1) / nw; ++k)
            copy_tracks(ts[k]->res, out, track_offsets[k], voff[k]);
    };
    {
        const uint32_t nth = host_threads(out->n_tracks, 1u << 15);
        std::vector<std::thread> th;
        for (uint32_t w = 1; w < nth; ++w) th.emplace_back(work, w, nth);
        work(0, nth);
        for (auto &t : th) t.join();
    }
    std::lock_guard<std::mutex> g(ctx->mu);
    for (uint32_t k = 0; k < n; ++k) ctx->tickets.erase(tickets[k]);
    return PXR_OK;
}

extern "C" int pxr_fetch_debug(pxr_ctx *ctx, uint64_t ticket, int what, uint32_t *buf,
                               uint32_t cap, uint32_t *n)
{
    if (!ctx || !n || (cap && !buf)) return fail(PXR_EINVAL, "null argument");
    std::shared_ptr<Ticket> t;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        auto it = ctx->tickets.find(ticket);
        if (it == ctx->tickets.end()) return fail(PXR_ENOTFOUND, "unknown ticket");
        t = it->second;
        if (t->state != 2) return fail(PXR_EBUSY, "event not finished");
    }
    if (!ctx->cfg.keep_debug || !t->batch || !t->batch->plan->region)
        return fail(PXR_EINVAL, "context was created without keep_debug");
    int rc = set_device(ctx);
    if (rc) return rc;
    return region_debug(t->batch->plan, t->index, what, buf, cap, n);
}

// Shared with the allocation-free doublet entry point (noalloc.cu).
namespace pxr {
int dev_params(const pxr_params *p, DevParams *d) { return check_params(p, d); }
int set_error(int code, const char *msg) { return fail(code, msg); }
}  // namespace pxr
