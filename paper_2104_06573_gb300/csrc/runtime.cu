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
    if (p->fit_mode > PXR_FIT_RIEMANN) return fail(PXR_EINVAL, "bad fit_mode");
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
    // launch shapes: CTAs per SM at most (the kernels stride over their work)
    static const uint32_t kGridDefault[PXR_STAGES] = {4, 16, 16, 8, 8, 8};
    for (int k = 0; k < PXR_STAGES; ++k)
        d->grid_per_sm[k] = p->grid_per_sm[k] ? p->grid_per_sm[k] : kGridDefault[k];
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
    size_t cnt, bkt, hs, r64, hmeta, hphi, item, cell_out,
        nbr_first,
        nbr_n, nbr, mindepth, root_list, root_in, live, front_list, front_in, front_snap, jbase, tup_hits, tup_n, tup_state, tup_first, tup_rank, tup_list, out_evt, o_nh,
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

    o.item = L.add(16 * N * kMaxOut);
    o.cell_out = L.add(4 * C);
    o.nbr_first = L.add(4 * C);
    o.nbr_n = L.add(4 * C);
    o.nbr = L.add(4 * G);
    o.mindepth = L.add(4 * C);
    o.root_list = L.add(4 * G);
    o.root_in = L.add(4 * G);
    o.live = L.add(4 * ((C + 31) / 32));
    o.front_list = L.add(4 * G);
    o.front_in = L.add(4 * G);
    o.front_snap = L.add(4 * (size_t)E);
    o.jbase = L.add(4 * ((size_t)E + 1));
    o.tup_hits = L.add(4 * T * kMaxHits);
    o.tup_n = L.add(T);
    o.tup_state = L.add(T);
    o.tup_first = L.add(4 * T);
    o.tup_rank = L.add(4 * T);
    o.tup_list = L.add(4 * T);
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
struct Batch;

struct pxr_ctx {
    pxr_config cfg{};
    int sms = 152;
    cudaStream_t stream = nullptr;      // default stream of the context
    bool own_stream = false;
    cudaStream_t slot_stream[2] = {nullptr, nullptr};
    bool own_arena = false;
    Arena arena;
    std::mutex api_mu;                  // serialises plan API calls
    std::mutex plans_mu;
    std::unordered_set<pxr_plan *> plans;   // live plans, destroyed with the context
    // serving
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
    std::unique_ptr<struct SlotBuffers> slot_buf[2];
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
    b.cell_chunk = (const uint32_t *)(r + o.cell_chunk);
    b.edge_chunk = (const uint32_t *)(r + o.edge_chunk);
    b.tup_chunk = (const uint32_t *)(r + o.tup_chunk);
    b.hit_chunk = (const uint32_t *)(r + o.hit_chunk);

    b.item = (uint4 *)(r + o.item);
    b.cell_in = nullptr;
    b.cell_out = (uint32_t *)(r + o.cell_out);
    b.nbr_first = (uint32_t *)(r + o.nbr_first);
    b.nbr_n = (uint32_t *)(r + o.nbr_n);
    b.nbr = (uint32_t *)(r + o.nbr);
    b.mindepth = (uint32_t *)(r + o.mindepth);
    b.root_list = (uint32_t *)(r + o.root_list);
    b.root_in = (uint32_t *)(r + o.root_in);
    b.live = (uint32_t *)(r + o.live);
    b.front_list = (uint32_t *)(r + o.front_list);
    b.front_in = (uint32_t *)(r + o.front_in);
    b.front_snap = (uint32_t *)(r + o.front_snap);
    b.jbase = (uint32_t *)(r + o.jbase);
    b.tup_hits = (uint32_t *)(r + o.tup_hits);
    b.tup_n = (uint8_t *)(r + o.tup_n);
    b.tup_state = (uint8_t *)(r + o.tup_state);
    b.tup_first = (uint32_t *)(r + o.tup_first);
    b.tup_rank = (uint32_t *)(r + o.tup_rank);
    b.tup_list = (uint32_t *)(r + o.tup_list);
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

static int plan_enqueue(pxr_plan *P, cudaStream_t s, bool capturing = false)
{
    Range range("pxr.enqueue");
    const DevBatch &b = P->db;
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
    if (p.min_hits <= 2 || multi_out) CK(cudaMemsetAsync(r + P->off.nbr_n, 0, 4 * P->C, s));
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
    int n = 6 + (P->dp.clean ? 1 : 0) + (P->dp.vtx ? 1 : 0);   // sort, doublets, walk, select,
                                                                 // scan, fit, keep, vertices
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
    size_t size() const { return nh.size(); }
    void resize(size_t n, bool with_cov = false, bool with_vtx = false)
    {
        nh.resize(n); hits.resize(n * kMaxHits); pt.resize(n); phi.resize(n); cot.resize(n);
        dxy.resize(n); dz.resize(n); chi2.resize(n); q.resize(n); st.resize(n); ql.resize(n);
        cov.resize(with_cov ? 15 * n : 0);
        vtx.resize(with_vtx ? n : 0);
    }
    void resize_vertices(size_t nv)
    {
        vz.resize(nv); verr.resize(nv); vpt2.resize(nv); vn.resize(nv);
    }
};

// Canonical order of n tracks (lexicographic by their hit tuples): LSD radix sort on the packed
// first two hit indices (caller indices are < 2^24, so the key has 48 bits), then the rare runs
// of equal first two hits are ordered by the remaining hits.
static void canonical_order(const uint32_t *hits, size_t n, std::vector<uint32_t> &ord)
{
    std::vector<uint64_t> key(n), key2(n);
    std::vector<uint32_t> tmp(n);
    ord.resize(n);
    for (size_t i = 0; i < n; ++i) {
        const uint32_t *h = hits + i * kMaxHits;
        key[i] = ((uint64_t)(h[0] & 0xFFFFFFu) << 24) | (uint64_t)(h[1] & 0xFFFFFFu);
        ord[i] = (uint32_t)i;
    }
    size_t count[256];
    for (int pass = 0; pass < 6; ++pass) {
        const int sh = 8 * pass;
        std::fill(count, count + 256, 0);
        for (size_t i = 0; i < n; ++i) ++count[(key[i] >> sh) & 0xFF];
        size_t run = 0;
        for (int b = 0; b < 256; ++b) { const size_t c = count[b]; count[b] = run; run += c; }
        for (size_t i = 0; i < n; ++i) {
            const size_t d = count[(key[i] >> sh) & 0xFF]++;
            key2[d] = key[i];
            tmp[d] = ord[i];
        }
        key.swap(key2);
        ord.swap(tmp);
    }
    for (size_t a = 0; a < n;) {
        size_t b = a + 1;
        while (b < n && key[b] == key[a]) ++b;
        if (b - a > 1)
            std::sort(ord.begin() + a, ord.begin() + b, [&](uint32_t x, uint32_t y) {
                return std::lexicographical_compare(hits + (size_t)x * kMaxHits,
                                                    hits + (size_t)x * kMaxHits + kMaxHits,
                                                    hits + (size_t)y * kMaxHits,
                                                    hits + (size_t)y * kMaxHits + kMaxHits);
            });
        a = b;
    }
}

// Copy the tracks of h into out, in canonical order (in_order: h already is).  A covariance
// that was not computed reads as NaN.
static int emit_tracks(const HostTracks &h, int32_t status, pxr_tracks *out, bool in_order = false)
{
    const size_t n = h.size();
    out->n_tracks = (uint32_t)n;
    out->n_vertices = (uint32_t)h.vz.size();
    out->status = status;
    if (n > out->capacity) return fail(PXR_ETRUNC, "track capacity too small");
    // the vertices (ordered by sum pT^2, whatever the track order)
    const size_t nv = h.vz.size();
    if (nv) {
        if (out->vtx_z) std::memcpy(out->vtx_z, h.vz.data(), 8 * nv);
        if (out->vtx_z_err) std::memcpy(out->vtx_z_err, h.verr.data(), 8 * nv);
        if (out->vtx_sum_pt2) std::memcpy(out->vtx_sum_pt2, h.vpt2.data(), 8 * nv);
        if (out->vtx_n_tracks) std::memcpy(out->vtx_n_tracks, h.vn.data(), 4 * nv);
    }
    if (in_order) {                          // already canonical: one copy per array
        auto cp = [n](void *dst, const void *src, size_t sz) {
            if (dst && n) std::memcpy(dst, src, sz * n);
        };
        cp(out->n_hits, h.nh.data(), 1);
        cp(out->hit_idx, h.hits.data(), 4 * kMaxHits);
        cp(out->pt, h.pt.data(), 8);
        cp(out->phi, h.phi.data(), 8);
        cp(out->cot_theta, h.cot.data(), 8);
        cp(out->dxy, h.dxy.data(), 8);
        cp(out->dz, h.dz.data(), 8);
        cp(out->chi2, h.chi2.data(), 8);
        cp(out->charge, h.q.data(), 1);
        cp(out->fit_status, h.st.data(), 1);
        cp(out->quality, h.ql.data(), 1);
        if (out->cov) {
            if (h.cov.empty()) std::fill(out->cov, out->cov + 15 * n, NAN);
            else cp(out->cov, h.cov.data(), 15 * sizeof(double));
        }
        if (out->vertex) {
            if (h.vtx.empty()) std::fill(out->vertex, out->vertex + n, -1);
            else cp(out->vertex, h.vtx.data(), 4);
        }
        return PXR_OK;
    }
    std::vector<uint32_t> ord;
    canonical_order(h.hits.data(), n, ord);
    for (size_t k = 0; k < n; ++k) {
        const size_t s = ord[k];
        if (out->n_hits) out->n_hits[k] = h.nh[s];
        if (out->hit_idx)
            std::memcpy(out->hit_idx + k * kMaxHits, h.hits.data() + s * kMaxHits, 4 * kMaxHits);
        if (out->pt) out->pt[k] = h.pt[s];
        if (out->phi) out->phi[k] = h.phi[s];
        if (out->cot_theta) out->cot_theta[k] = h.cot[s];
        if (out->dxy) out->dxy[k] = h.dxy[s];
        if (out->dz) out->dz[k] = h.dz[s];
        if (out->chi2) out->chi2[k] = h.chi2[s];
        if (out->charge) out->charge[k] = h.q[s];
        if (out->fit_status) out->fit_status[k] = h.st[s];
        if (out->quality) out->quality[k] = h.ql[s];
        if (out->cov) {
            if (h.cov.empty()) std::fill(out->cov + 15 * k, out->cov + 15 * k + 15, NAN);
            else std::memcpy(out->cov + 15 * k, h.cov.data() + 15 * s, 15 * sizeof(double));
        }
        if (out->vertex) out->vertex[k] = h.vtx.empty() ? -1 : h.vtx[s];
    }
    return PXR_OK;
}

static int32_t flags_status(uint32_t f) { return (f & (F_CELLS | F_EDGES | F_TUPLES | F_VERTS)) ? PXR_EOVERFLOW : (f & F_LAYER) ? PXR_EINVAL : PXR_OK; }

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
    return emit_tracks(h, flags_status(flags), out);
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
            std::vector<uint32_t> nf, nn, live, roots;
            if ((rc = d2h(nf, b.nbr_first + c0, nc)) || (rc = d2h(nn, b.nbr_n + c0, nc))) return rc;
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
                for (uint32_t k = 0; valid[c] && k < nn[c]; ++k) {
                    uint32_t B = nb[nf[c] - g0 + k] - c0;
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
    // the event's hits, copied at submission: x, y, z (float) then layer (uint16), n of each
    std::unique_ptr<uint8_t[]> hits;
    uint32_t n = 0;
    const float *x() const { return reinterpret_cast<const float *>(hits.get()); }
    const float *y() const { return x() + n; }
    const float *z() const { return x() + 2 * (size_t)n; }
    const uint16_t *layer() const { return reinterpret_cast<const uint16_t *>(x() + 3 * (size_t)n); }
    uint32_t lcount[kMaxLayers + 1] = {};
    pxr_params params{};
    size_t bytes = 0;
    std::shared_ptr<Batch> batch;        // kept for pxr_fetch_debug
    uint32_t index = 0;
    int32_t status = PXR_OK;
    HostTracks res;                      // results in canonical order (copied from the slot's
                                         // pinned buffer by the scheduler thread)
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
    Pinned head, evt, out;
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
    // pinned staging of the head (inputs + small arrays), one H2D copy; the batch's tickets are
    // out of the pending queue and reach no other thread before the batch is published
    {
    Unlocked unlocked(lk);
    char *h = sb.head.p;
    auto stage = [&](uint32_t e0, uint32_t step) {
        for (uint32_t e = e0; e < E; e += step) {
            size_t a = P->hit_off[e], n = items[e]->n;
            std::memcpy(h + P->off.x + 4 * a, items[e]->x(), 4 * n);
            std::memcpy(h + P->off.y + 4 * a, items[e]->y(), 4 * n);
            std::memcpy(h + P->off.z + 4 * a, items[e]->z(), 4 * n);
            std::memcpy(h + P->off.layer + 2 * a, items[e]->layer(), 2 * n);
        }
    };
    {
        // large batches are staged by a few host threads
        const uint32_t nth = P->N > (1u << 20) ? std::min<uint32_t>(
            E, std::max(1u, std::min(8u, std::thread::hardware_concurrency() / 2))) : 1u;
        std::vector<std::thread> th;
        for (uint32_t w = 1; w < nth; ++w) th.emplace_back(stage, w, nth);
        stage(0, nth);
        for (auto &x : th) x.join();
    }
    const size_t e1 = 4 * (E + 1);
    std::memcpy(h + P->off.hit_off, P->hit_off.data(), e1);
    std::memcpy(h + P->off.cell_off, P->cell_off.data(), e1);
    std::memcpy(h + P->off.edge_off, P->edge_off.data(), e1);
    std::memcpy(h + P->off.tup_off, P->tup_off.data(), e1);
    fill_chunks(P, h);
    cudaStream_t s = slot_stream(ctx, slot);
    B->stream = s;
    CK(cudaMemcpyAsync(P->region, h, P->off.head_end, cudaMemcpyHostToDevice, s));
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
        items[e]->hits.reset();
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
        bool ok = sb.out.reserve(L.add(0) + 256);
        const DevBatch &d = P->db;
        char *ho = sb.out.p;
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
        const char *ho = sb.out.p;
        std::vector<std::shared_ptr<Ticket>> ts(E);
        for (uint32_t e = 0; e < E; ++e) {
            auto it = ctx->tickets.find(B.ids[e]);
            if (it != ctx->tickets.end()) ts[e] = it->second;
        }
        {
        // the results reach no other thread before the tickets are marked done (below)
        Unlocked unlocked(lk);
        Range range("pxr.batch.order");
        // events in parallel (a few host threads): the ordering is the heaviest host work of a
        // batch
        auto work = [&](uint32_t e0, uint32_t step) {
        std::vector<uint32_t> ord;
        for (uint32_t e = e0; e < E; e += step) {
            if (!ts[e]) continue;
            Ticket &t = *ts[e];
            const uint32_t a = hev[e], n = hev[e + 1] - a;
            t.res.resize(n, P->dp.cov != 0, P->dp.vtx != 0);
            t.res.resize_vertices(P->dp.vtx ? hev[2 * E + 1 + e] : 0);
            if (P->dp.vtx) {
                const uint32_t nv = hev[2 * E + 1 + e];
                std::memcpy(t.res.vz.data(), ho + B.v_z + 8 * (size_t)a, 8 * (size_t)nv);
                std::memcpy(t.res.verr.data(), ho + B.v_err + 8 * (size_t)a, 8 * (size_t)nv);
                std::memcpy(t.res.vpt2.data(), ho + B.v_pt2 + 8 * (size_t)a, 8 * (size_t)nv);
                std::memcpy(t.res.vn.data(), ho + B.v_n + 4 * (size_t)a, 4 * (size_t)nv);
            }
            if (n) {
                // canonical order here, on the scheduler thread, so that a fetch only copies
                auto hp = [&](size_t off) { return ho + off; };
                const uint32_t *hits = (const uint32_t *)hp(B.o_hits + 4 * (size_t)a * kMaxHits);
                canonical_order(hits, n, ord);
                const uint8_t *nh = (const uint8_t *)hp(B.o_nh + a);
                const double *pt = (const double *)hp(B.o_pt + 8 * (size_t)a);
                const double *phi = (const double *)hp(B.o_phi + 8 * (size_t)a);
                const double *cot = (const double *)hp(B.o_cot + 8 * (size_t)a);
                const double *dxy = (const double *)hp(B.o_dxy + 8 * (size_t)a);
                const double *dz = (const double *)hp(B.o_dz + 8 * (size_t)a);
                const double *chi2 = (const double *)hp(B.o_chi2 + 8 * (size_t)a);
                const int8_t *q = (const int8_t *)hp(B.o_q + a);
                const int8_t *st = (const int8_t *)hp(B.o_st + a);
                const uint8_t *ql = (const uint8_t *)hp(B.o_ql + a);
                const double *cv = (const double *)hp(B.o_cov + 8 * 15 * (size_t)a);
                for (uint32_t k = 0; k < n; ++k) {
                    const uint32_t s_ = ord[k];
                    t.res.nh[k] = nh[s_];
                    std::memcpy(&t.res.hits[(size_t)k * kMaxHits], hits + (size_t)s_ * kMaxHits,
                                4 * kMaxHits);
                    t.res.pt[k] = pt[s_];
                    t.res.phi[k] = phi[s_];
                    t.res.cot[k] = cot[s_];
                    t.res.dxy[k] = dxy[s_];
                    t.res.dz[k] = dz[s_];
                    t.res.chi2[k] = chi2[s_];
                    t.res.q[k] = q[s_];
                    t.res.st[k] = st[s_];
                    t.res.ql[k] = ql[s_];
                    if (P->dp.cov)
                        std::memcpy(&t.res.cov[15 * (size_t)k], cv + 15 * (size_t)s_,
                                    15 * sizeof(double));
                    if (P->dp.vtx)
                        t.res.vtx[k] = ((const int32_t *)(ho + B.o_vtx))[a + s_];
                }
            }
        }
        };
        const uint32_t nth = std::min<uint32_t>(E, std::max(1u, std::min(8u, std::thread::hardware_concurrency() / 2)));
        std::vector<std::thread> th;
        for (uint32_t w = 1; w < nth; ++w) th.emplace_back(work, w, nth);
        work(0, nth);
        for (auto &x : th) x.join();
        }
        for (uint32_t e = 0; e < E; ++e) {
            if (!ts[e]) continue;
            Ticket &t = *ts[e];
            t.status = flags_status(hev[E + 1 + e]);
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
            int slot = 0;
            for (auto &b : ctx->inflight)
                if (b->slot == 0) slot = 1;
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
    if (!ctx->cfg.max_inflight || ctx->cfg.max_inflight > 2) ctx->cfg.max_inflight = 2;
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

extern "C" int pxr_submit_event(pxr_ctx *ctx, const float *x, const float *y, const float *z,
                                const uint16_t *layer, uint32_t n_hits, const pxr_params *params,
                                uint64_t *ticket)
{
    if (!ctx || !ticket || (n_hits && (!x || !y || !z || !layer)))
        return fail(PXR_EINVAL, "null argument");
    DevParams dp;
    int rc = check_params(params, &dp);
    if (rc) return rc;
    if (n_hits > kLocalMask) return fail(PXR_EINVAL, "too many hits in one event");
    auto t = std::make_shared<Ticket>();
    // copy the hits into the ticket (uninitialised storage), then check them and count them per
    // layer (four interleaved counter sets keep the increments independent)
    t->n = n_hits;
    t->hits.reset(new uint8_t[14 * (size_t)n_hits + 16]);
    float *tx = const_cast<float *>(t->x());
    std::memcpy(tx, x, 4 * (size_t)n_hits);
    std::memcpy(tx + n_hits, y, 4 * (size_t)n_hits);
    std::memcpy(tx + 2 * (size_t)n_hits, z, 4 * (size_t)n_hits);
    std::memcpy(const_cast<uint16_t *>(t->layer()), layer, 2 * (size_t)n_hits);
    bool finite = true;
    uint32_t bad_layer = 0;
    uint32_t lc[4][kMaxLayers + 1] = {};
    for (uint32_t h = 0; h < n_hits; ++h) {
        finite &= std::isfinite(x[h]) & std::isfinite(y[h]) & std::isfinite(z[h]);
        const uint16_t l = layer[h];
        bad_layer |= l >= params->n_layers;
        lc[h & 3][l < kMaxLayers ? l : kMaxLayers]++;
    }
    if (!finite) return fail(PXR_EINVAL, "non-finite hit coordinate");
    if (bad_layer) return fail(PXR_EINVAL, "hit layer id >= n_layers");
    for (int l = 0; l <= kMaxLayers; ++l) t->lcount[l] = lc[0][l] + lc[1][l] + lc[2][l] + lc[3][l];
    t->params = *params;
    t->bytes = event_bytes(*params, dp, t->lcount, n_hits);
    if (t->bytes > ctx->arena.size) return fail(PXR_ENOMEM, "event exceeds the memory budget");
    std::lock_guard<std::mutex> g(ctx->mu);
    if (!ctx->sched_error.empty() && ctx->inflight.empty() && ctx->pending.empty()) {
        // a failed batch is reported through its tickets; the context stays usable
        ctx->sched_error.clear();
    }
    if (ctx->reserved + t->bytes > ctx->arena.size) return fail(PXR_EAGAIN, "memory budget full");
    t->id = ctx->next_ticket++;
    ctx->reserved += t->bytes;
    ctx->tickets[t->id] = t;
    ctx->pending.push_back(t->id);
    ctx->cv_sched.notify_all();
    *ticket = t->id;
    return PXR_OK;
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
    const HostTracks &r = t->res;
    int rc = emit_tracks(r, t->status, out, true);
    if (rc) return rc;
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->tickets.erase(ticket);
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
