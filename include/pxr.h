/*
 * pxr — pixel-track seeding and fitting on one GPU (sm_103a), C ABI.
 *
 * The library implements the data-parallel core of the "Tracks" module of the heterogeneous pixel
 * reconstruction studied in the paper (§2, "Patatrack Heterogeneous Pixel Reconstruction": the
 * module "forms n-tuplets from the hits, and fits the hit n-tuplets to obtain track parameters").
 * Per event it runs: a per-layer phi-binned counting sort of the hits, doublet (cell) building in a
 * phi window, cellular-automaton (CA) cell connection with an r-z alignment cut and a transverse
 * DCA cut, ntuplet finding by a depth-first walk from root cells, and a broken-line helix fit of
 * each ntuplet.  The paper gives no formulas for these steps; the definitions implemented are
 * stated at each entry point below and in the parameter struct.
 *
 * Events are independent (the paper's throughput comes from processing many events concurrently,
 * §5, Table 2).  The library batches many events into one set of kernel launches and serves a
 * stream of events with continuous batching under a device-memory budget.
 *
 * Conventions for every entry point:
 *   - Return value: PXR_OK (0) or a negative PXR_E* code.  pxr_last_error() gives a message.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA device memory of the
 *     context's device (for example from torch.empty(..., device="cuda")).
 *   - The library never takes ownership of caller memory.  Memory it allocates is released by
 *     the matching destroy call.
 *   - One context may be used from several threads: every entry point takes the context lock.
 *   - Units: cm, GeV, tesla, radians.  Hit indices in results are positions in the caller's
 *     input arrays of that event (0-based).
 */
#ifndef PXR_H
#define PXR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PXR_MAX_LAYERS 16
#define PXR_MAX_PAIRS 32
#define PXR_MAX_HITS 6          /* hit slots per track; max_hits must be <= 6 */

/* Return codes */
#define PXR_OK 0
#define PXR_EINVAL (-1)     /* bad argument, parameter or input value (NaN, layer id too large) */
#define PXR_EAGAIN (-2)     /* admission refused now (memory budget or batch slots full); retry
                               after pxr_poll has returned completed events */
#define PXR_ENOMEM (-3)     /* the request can never fit the context's memory budget */
#define PXR_EOVERFLOW (-4)  /* a per-event capacity (cells, edges, ntuplets) was exceeded; the
                               event's results are truncated, never written out of bounds */
#define PXR_ETIMEDOUT (-5)  /* a bounded wait gave up */
#define PXR_ECUDA (-6)      /* a CUDA call failed; the context should be destroyed */
#define PXR_ETRUNC (-7)     /* caller buffer too small; the required count is returned */
#define PXR_ENOTFOUND (-8)  /* unknown or already fetched ticket */
#define PXR_EBUSY (-9)      /* the ticket's event is not finished yet */
#define PXR_EBOUNDS (-10)   /* libpxr_checked.so only: a device-side bounds check found an index
                               outside its array (the access was skipped; the event's results
                               are not to be trusted).  The normal library never returns it */

/* Arithmetic of the three cuts. */
#define PXR_CUT_FP64 0      /* every cut quantity evaluated in FP64, in the fixed operation
                               order stated below (round to nearest, no fused multiply-add) */
#define PXR_CUT_FP32 1      /* FP32 evaluation with a rigorous error bound around each
                               threshold; a candidate inside the bound is re-evaluated exactly as
                               in PXR_CUT_FP64, so both modes take the same decisions */

/* Arithmetic of the broken-line fit. */
#define PXR_FIT_FP64 0      /* all steps in FP64 */
#define PXR_FIT_MIXED 1     /* FP64 arithmetic with FP32 transcendentals (atan2, log, cos, sin):
                               the normal matrices need FP64 (kink weights up to ~1e14 next to
                               measurement weights ~1e6) */
#define PXR_FIT_FP32 2      /* all steps in FP32; errors against FP64 are reported, not bounded */
#define PXR_FIT_RIEMANN 3   /* Riemann fit instead of the broken line, FP64: hits mapped to the
                               paraboloid w = x^2 + y^2, the plane through them (smallest
                               eigenvector of the weighted scatter matrix) gives the circle; a
                               weighted straight line in (arc length, z); no multiple scattering.
                               The track covariance is not computed for it (NaN) */
#define PXR_FIT_SPLIT 4     /* FP32 bulk: the local (chord) frame with error-free offsets from hit
                               0, the reference circle, residuals, arc lengths, multiple
                               scattering and the rows of the normal equations in FP32; the
                               normal matrices, their banded Cholesky with the curvature border
                               (Schur complement) and the conversion to track parameters in FP64.
                               A track whose fitted curvature is below a tenth of its reference
                               circle's (where FP32's error of the reference would be amplified)
                               or that the FP32 front end cannot take is refitted in FP64 */

/* Presets for pxr_params_init */
#define PXR_PRESET_BARREL 0 /* 4 barrel layers r = 2.9/6.8/10.9/16.0, pairs (0,1)(1,2)(2,3), roots
                               {0}, quadruplets only (min = max = 4) */
#define PXR_PRESET_PHASE1 1 /* barrel + 3 disks per side (ids 4-6 at +z, 7-9 at -z), 13 pairs,
                               roots {0,1} with suffix removal, 3..5 hits */

/* Stages whose grid size is tunable (index into pxr_params.grid_per_sm). */
#define PXR_STAGES 6
#define PXR_STAGE_SORT 0
#define PXR_STAGE_DOUBLETS 1
#define PXR_STAGE_CONNECT 2
#define PXR_STAGE_WALK 3
#define PXR_STAGE_SELECT 4
#define PXR_STAGE_FIT 5

/* Track quality bits (pxr_tracks.quality). */
#define PXR_Q_GOOD 1u       /* fit status 0 and the selection cuts (pt_min, chi2_max) passed */
#define PXR_Q_KEPT 2u       /* good, and (with clean_shared) no better-ranked good track shares a
                               hit with it */

/*
 * Reconstruction parameters.  All fields are inputs; pxr_params_init fills a preset.
 *
 * Doublets.  For every allowed pair p (layer pair_inner[p] -> layer pair_outer[p]; the pairs must
 *   not form a cycle of layers, and at most 4 pairs may share an inner or an outer layer) and every hit
 *   i on the inner and o on the outer layer, the cell (i, o) exists iff
 *       x_i x_o + y_i y_o >= cos_phi_window * r_i * r_o,   r = sqrt(x^2 + y^2),
 *   i.e. the azimuths differ by at most phi_window.  cos_phi_window must equal cos(phi_window)
 *   and is computed by the caller once (the library does not evaluate cos).
 * CA edges.  Cell A = (i, j) connects to cell B = (j, k) iff
 *       |a_r b_z - a_z b_r| <= theta_cut * |a| * |b|,  a = (r_j - r_i, z_j - z_i),
 *                                                       b = (r_k - r_j, z_k - z_j)
 *   and the circle through the three hits (transverse plane) passes within dca_cut of the
 *   origin: with u = p_j - p_i, v = p_k - p_i, D = 2 (u_x v_y - u_y v_x),
 *   c' = ((|u|^2 v_y - |v|^2 u_y) / D, (|v|^2 u_x - |u|^2 v_x) / D), c = p_i + c', R = |c'|,
 *       dca = |2 c.p_i - |p_i|^2| / (|c| + R)   (D == 0: distance of the origin from the line
 *                                                 through p_i and p_k).
 * Ntuplets.  From every cell whose inner hit lies on a layer in root_layer_mask, follow edges
 *   depth first; a path is emitted when it has max_hits hits or its last cell has no edge, and
 *   it has at least min_hits hits.  With drop_suffixes, a path that is a strict suffix of another
 *   emitted path is removed.
 * Fit.  Broken line (V. Blobel, NIM A 566 (2006) 14): reference circle through hits 0, n/2, n-1;
 *   transverse offsets + one curvature correction and a line in (s, z), each with multiple-
 *   scattering kinks at the inner hits (Highland angle with x_over_x0 per layer crossing,
 *   projected by 1 + cot^2 on the transverse and (1 + cot^2)^2 on the line kinks); weights
 *   1/sigma_rphi^2 and 1/sigma_z^2 (disks: 1/(sigma_z cot)^2); Cholesky solves; conversion to the
 *   point of closest approach to the z axis.  dxy = q (|C| - R) with C the fitted centre.
 * Selection.  Every fitted track stays in the output with quality bits: PXR_Q_GOOD when its fit
 *   status is 0, pT >= pt_min and chi2 / ndof <= chi2_max (ndof = max(2 n - 5, 1) for n hits; a
 *   threshold of 0 is no cut); PXR_Q_KEPT when it is good and, with clean_shared, no other good
 *   track of the event that shares a hit with it ranks strictly better (more hits, or as many and
 *   a smaller chi2 / ndof).  One round: a track is dropped by a better one even if that one is
 *   dropped in turn.  Without clean_shared, KEPT equals GOOD.
 * Covariance (fit_cov).  The fitted offsets u_0, u_1 and curvature correction of the transverse
 *   broken line and the line values v_0, v_1 have the covariance of the two linear least-squares
 *   problems (the corresponding blocks of the inverse normal matrices; the two fits are
 *   independent); it is propagated to (q/pT, phi, cot_theta, dxy, dz) through the conversion,
 *   linearised around the solution (forward-mode derivatives in FP64).
 * Vertices (vertexing).  The event's KEPT tracks with a finite dz, sorted by dz: a track joins
 *   the cluster of the one before it when their dz differ by at most vtx_gap; clusters of at
 *   least vtx_min_tracks tracks are vertices (z = mean dz, its standard error, the track count,
 *   sum pT^2), ordered by sum pT^2, largest first.  An event with more than 8192 kept tracks gets
 *   no vertices and PXR_EOVERFLOW.
 */
typedef struct pxr_params {
    uint32_t n_layers;                         /* <= PXR_MAX_LAYERS; hit layer ids < n_layers */
    uint8_t layer_is_disk[PXR_MAX_LAYERS];     /* 1 for disks (z-fixed layers) */
    uint32_t n_pairs;                          /* <= PXR_MAX_PAIRS */
    uint8_t pair_inner[PXR_MAX_PAIRS];
    uint8_t pair_outer[PXR_MAX_PAIRS];
    uint32_t root_layer_mask;                  /* bit l set: cells starting on layer l are roots */
    uint32_t drop_suffixes;                    /* 0 or 1 */
    uint32_t min_hits, max_hits;               /* 2 <= min_hits <= max_hits <= PXR_MAX_HITS */
    uint32_t cut_mode;                         /* PXR_CUT_* */
    uint32_t fit_mode;                         /* PXR_FIT_* */
    double phi_window;                         /* w, radians, (0, 0.5] */
    double cos_phi_window;                     /* cos(w), computed by the caller */
    double theta_cut;                          /* r-z alignment threshold, > 0 */
    double dca_cut;                            /* cm, > 0 */
    double bfield;                             /* tesla along +z, > 0 */
    double sigma_rphi, sigma_z;                /* cm, > 0 */
    double x_over_x0;                          /* radiation lengths per layer, >= 1e-6 */
    uint32_t n_phi_bins;                       /* phi bins per layer, 64..2048; 0 = automatic */
    uint32_t max_cells_per_event;              /* 0 = sized from the hit counts; rounded up to a
                                                  multiple of 256.  Counts doublet candidates
                                                  (pairs inside the phi window), a superset of
                                                  the cells */
    uint32_t max_tuples_per_event;             /* 0 = sized from the hit counts; rounded up to a
                                                  multiple of 256 */
    uint32_t grid_per_sm[PXR_STAGES];          /* launch shape: CTAs per SM at most for the
                                                  stage's grid (PXR_STAGE_*), 1..64; 0 = the
                                                  built-in value.  Results do not depend on it;
                                                  pxr's autotuner picks it with the bin count */
    uint32_t block_threads[PXR_STAGES];        /* launch shape: threads per CTA of the stage's
                                                  main kernel; 0 = the built-in value.  Sort:
                                                  256, 512 or 1024 (built-in 512); doublets:
                                                  64, 128 or 256 (built-in 256); fit: 32, 64,
                                                  128 or 256 (built-in: from the track count).
                                                  Connect, walk and select take 0 only (their
                                                  CTAs own fixed chunks of work and shared
                                                  staging).  Other values: PXR_EINVAL.  Results
                                                  do not depend on it; pxr's autotuner picks it */
    double pt_min;                             /* selection: GeV, >= 0; 0 = no cut */
    double chi2_max;                           /* selection: chi2 per degree of freedom, >= 0;
                                                  0 = no cut */
    uint32_t clean_shared;                     /* selection: 0 or 1 (shared-hit cleaning) */
    uint32_t fit_cov;                          /* 1: compute each track's covariance
                                                  (pxr_tracks.cov); 0: not computed */
    uint32_t vertexing;                        /* 1: find primary vertices (pxr_tracks.vtx_*) */
    uint32_t vtx_min_tracks;                   /* tracks a vertex needs, >= 2 */
    double vtx_gap;                            /* cm, > 0: largest z gap inside a vertex */
} pxr_params;

/* Context configuration. */
typedef struct pxr_config {
    int device;                 /* CUDA device ordinal */
    size_t mem_budget_bytes;    /* device arena; 0 = 2 GiB */
    void *arena;                /* optional caller device memory of mem_budget_bytes bytes (for
                                   example a torch uint8 tensor); NULL = allocate once at create */
    void *stream;               /* optional caller cudaStream_t for all work; NULL = the context
                                   creates its own streams */
    uint32_t max_batch_events;  /* dynamic batching cap (events per launch); 0 = 256 */
    uint32_t max_batch_hits;    /* dynamic batching cap (hits per launch); 0 = 4M */
    uint32_t max_inflight;      /* batches on the device at once, 1 to 4 (each on its own
                                   stream); 0 = 2 */
    uint32_t keep_debug;        /* keep cells/edges/ntuplets of served events for
                                   pxr_fetch_debug (costs memory until the fetch) */
} pxr_config;

/* Caller-owned arrays receiving the tracks of one event.  Any array pointer may be NULL: that
 * field is not copied.  The vertex arrays are indexed by vertex (n_vertices of them), the others
 * by track. */
typedef struct pxr_tracks {
    uint32_t capacity;          /* in: slots in every array below */
    uint32_t n_tracks;          /* out: tracks of the event (may exceed capacity: PXR_ETRUNC) */
    int32_t status;             /* out: PXR_OK or PXR_EOVERFLOW for this event */
    uint8_t *n_hits;            /* [capacity] hits per track */
    uint32_t *hit_idx;          /* [capacity * PXR_MAX_HITS] caller hit indices, inner to outer;
                                   unused slots 0xFFFFFFFF */
    double *pt, *phi, *cot_theta, *dxy, *dz, *chi2;   /* [capacity] */
    int8_t *charge;             /* [capacity] */
    int8_t *fit_status;         /* [capacity] 0 ok, 1 collinear, 2 zero curvature, 3 Cholesky */
    uint8_t *quality;           /* [capacity] PXR_Q_* bits of the selection */
    double *cov;                /* [capacity * 15] covariance of (q/pT [1/GeV], phi, cot_theta,
                                   dxy, dz), upper triangle row by row; NaN when fit_cov was 0
                                   or the fit failed */
    int32_t *vertex;            /* [capacity] index of the track's vertex, -1 for none (always -1
                                   without vertexing) */
    uint32_t n_vertices;        /* out: vertices of the event (<= n_tracks / 2) */
    double *vtx_z, *vtx_z_err;  /* [capacity] vertex z (cm, mean dz of its tracks) and the
                                   standard error of that mean */
    double *vtx_sum_pt2;        /* [capacity] sum of pT^2 of its tracks (GeV^2); vertices are
                                   ordered by it, largest first */
    uint32_t *vtx_n_tracks;     /* [capacity] */
} pxr_tracks;

typedef struct pxr_ctx pxr_ctx;
typedef struct pxr_plan pxr_plan;

/* Library version string (static storage).
 * Source: none (library plumbing; the paper defines no interface). */
const char *pxr_version(void);

/* Message of the last error on this thread (static thread-local storage).
 * Source: none (library plumbing; the paper defines no interface). */
const char *pxr_last_error(void);

/* Fill *p with a preset (PXR_PRESET_*), cut mode FP64 and fit mode FP64; no selection, no
 * covariance, no vertexing (vtx_min_tracks 2 and vtx_gap 0.05 cm for when it is switched on).
 * Source: the paper names the Tracks module's steps (§2) without values; the presets are this
 * library's synthetic geometries (barrel layers, Phase-1-like disks). */
int pxr_params_init(pxr_params *p, int preset);

/* Validate *p without touching any device: PXR_OK or PXR_EINVAL with a message.
 * Source: none (library plumbing). */
int pxr_params_check(const pxr_params *p);

/* Create a context on cfg->device.  Allocates the arena (unless cfg->arena is given), pinned host
 * staging memory and the scheduler thread.  *out receives the context.
 * Source: the paper's memory pool (§5, Table 2: allocation through a caching pool) is the
 * context for the one arena allocated here. */
int pxr_create(const pxr_config *cfg, pxr_ctx **out);

/* Stop the scheduler, wait for work in flight, release everything the context allocated.
 * Unfetched results are discarded; plans of the context that are still alive are destroyed
 * (their handles become invalid).
 * Source: none (library plumbing). */
void pxr_destroy(pxr_ctx *ctx);

/*
 * Serving path.  Submit one event (host arrays of n_hits elements, caller order).  The hit data
 * are copied before the call returns.  The event joins the next batch formed by the scheduler
 * thread (continuous batching: a batch is launched as soon as a device slot is free).
 * *ticket identifies the event.  Errors: PXR_EINVAL (bad params or input), PXR_EAGAIN (budget
 * full now), PXR_ENOMEM (the event alone exceeds the budget).
 * Source: the paper defines no serving interface; its throughput comes from events processed
 * concurrently (§5, Table 2), which this entry point provides by continuous batching.
 */
int pxr_submit_event(pxr_ctx *ctx, const float *x, const float *y, const float *z,
                     const uint16_t *layer, uint32_t n_hits, const pxr_params *params,
                     uint64_t *ticket);

/* Serving path, many events in one call: n_events events whose hits are back to back in the
 * host arrays x, y, z, layer, event e at [hit_offsets[e], hit_offsets[e+1]) (hit_offsets: host
 * array of n_events+1; the arrays are indexed from hit_offsets[0]).  Each event behaves as if
 * submitted by pxr_submit_event, in order; tickets[e] (host, n_events) receives its ticket.  The
 * hits are copied into the context's pinned host memory before the call returns (from there
 * they go to the device without a further host copy).  All events are admitted or none:
 * PXR_EINVAL (bad params or any event's input), PXR_ENOMEM (an event alone exceeds the budget,
 * or no pinned memory), PXR_EAGAIN (the events together exceed the free budget now).
 * Source: the paper defines no serving interface (§5, Table 2 for concurrent events). */
int pxr_submit_events(pxr_ctx *ctx, uint32_t n_events, const uint32_t *hit_offsets,
                      const float *x, const float *y, const float *z, const uint16_t *layer,
                      const pxr_params *params, uint64_t *tickets);

/* Return up to cap finished tickets in done[] (host array), *n_done = count.  Waits up to
 * timeout_us microseconds (0 = do not wait, < 0 = until at least one is done or none pending).
 * Source: the paper defines no serving interface (§5, Table 2 for concurrent events). */
int pxr_poll(pxr_ctx *ctx, uint64_t *done, uint32_t cap, uint32_t *n_done, int timeout_us);

/* Copy the tracks of a finished event into caller arrays (canonical order: lexicographic by hit
 * tuple).  On success the ticket is released.  PXR_ETRUNC: out->capacity too small, n_tracks set,
 * ticket kept.  PXR_EBUSY: not finished.  The event's own status (overflow) is in out->status.
 * Source: §2, the Tracks module's product (tracks with fitted parameters from hit n-tuplets). */
int pxr_fetch_tracks(pxr_ctx *ctx, uint64_t ticket, pxr_tracks *out);

/* The tracks of n finished events in one call, into one set of caller arrays: event k's tracks
 * at rows [track_offsets[k], track_offsets[k+1]) of every track array and its vertices at rows
 * [vertex_offsets[k], vertex_offsets[k+1]) of the vertex arrays (track_offsets: host array of
 * n+1, written; vertex_offsets, event_status: optional host arrays of n+1 and n, written).  Each
 * event's tracks are in canonical order; a track's vertex index counts within its event.
 * out->capacity is the rows of every array; out->n_tracks and out->n_vertices receive the
 * totals, out->status the first event status that is not PXR_OK (else PXR_OK).  On success every
 * ticket is released.  PXR_ETRUNC: capacity too small (totals set, tickets kept); PXR_EBUSY /
 * PXR_ENOTFOUND: a ticket not finished / unknown (nothing copied, tickets kept).
 * Source: §2, the Tracks module's product. */
int pxr_fetch_events(pxr_ctx *ctx, uint32_t n, const uint64_t *tickets, uint32_t *track_offsets,
                     uint32_t *vertex_offsets, int32_t *event_status, pxr_tracks *out);

/* Debug content of a finished event kept with cfg->keep_debug (before pxr_fetch_tracks):
 * what = 0: cells as (inner, outer) caller-index pairs (2 words each);
 * what = 1: CA edges as (i, j, k) caller-index triples (3 words each), for the cells that can
 *           lie on a root path (root cells and, transitively, their edges' targets: the edges
 *           of other cells cannot change a result and are not built);
 * what = 2: ntuplets before suffix removal as PXR_MAX_HITS words each (0xFFFFFFFF padded).
 * Writes at most cap words to buf (host), *n = number of items.
 * Source: §2, the Tracks module's intermediate products (doublets, CA graph, n-tuplets). */
int pxr_fetch_debug(pxr_ctx *ctx, uint64_t ticket, int what, uint32_t *buf, uint32_t cap,
                    uint32_t *n);

/*
 * Device-resident batch path ("plan").  A plan binds a batch of n_events events whose hits are
 * already in device memory: x, y, z, layer are device arrays holding all events back to back,
 * event e occupying [hit_offsets[e], hit_offsets[e+1]) (hit_offsets: host array of n_events+1).
 * The plan owns a region of the context arena for all intermediate data and results; it sizes
 * the per-event capacities from the per-layer hit counts (read back once here).  With
 * use_graph != 0 the launch sequence is captured once into a CUDA graph and replayed.
 * The caller keeps the input arrays alive and unchanged in shape for the plan's lifetime; their
 * contents may change between runs.
 * Source: many events per launch, the batched form of the concurrency of §5 (Table 2).
 */
int pxr_plan_create(pxr_ctx *ctx, uint32_t n_events, const uint32_t *hit_offsets,
                    const float *x, const float *y, const float *z, const uint16_t *layer,
                    const pxr_params *params, int use_graph, pxr_plan **out);

/* Run the whole hot path for the plan's batch on stream (cudaStream_t; NULL = the context's).
 * Asynchronous: returns after enqueueing.
 * Source: §2, the Tracks module (doublets, cellular automaton, n-tuplets, broken-line fit). */
int pxr_plan_run(pxr_plan *plan, void *stream);

/* Wait for the plan's last run and copy event e's tracks to the caller (same layout and order
 * as pxr_fetch_tracks).
 * Source: §2, the Tracks module's product. */
int pxr_plan_tracks(pxr_plan *plan, uint32_t e, pxr_tracks *out);

/* Debug content of event e after the last run (see pxr_fetch_debug for `what`).
 * Source: §2, the Tracks module's intermediate products. */
int pxr_plan_debug(pxr_plan *plan, uint32_t e, int what, uint32_t *buf, uint32_t cap,
                   uint32_t *n);

/* Number of kernel launches one pxr_plan_run performs (for launch accounting).
 * Source: none (measurement plumbing). */
int pxr_plan_launches(const pxr_plan *plan);

/* Run the plan once like pxr_plan_run, but without its graph and with the CA stage counting its
 * work, wait for it, and write to counts[2]: the candidate triplets whose r-z alignment test
 * was evaluated, and of them the ones whose transverse-DCA test was evaluated.  The results of
 * the run equal those of pxr_plan_run (the counting costs time; the run is not meant to be
 * timed).  Errors: PXR_EINVAL for a null argument, PXR_ECUDA.
 * Source: §2 (the CA's triplet tests); the counts size the CA stage's arithmetic roofline. */
int pxr_plan_count_ca_tests(pxr_plan *plan, void *stream, uint64_t *counts);

/* Per-event counters of the last run, copied to the host array out[5 * n_events]: out[k*E + e]
 * for k = 0 cells, 1 CA edges, 2 ntuplets before selection, 3 flags (1 cells, 2 edges,
 * 4 ntuplets overflowed; 8 bad layer id), 4 tracks.
 * Source: none (measurement plumbing). */
int pxr_plan_counts(pxr_plan *plan, uint32_t *out);

/* Device time in milliseconds of each stage of the last run, from CUDA events recorded between
 * the launches (event-record nodes when the plan replays a graph).  Stage order: hit sort,
 * doublets, CA connect, ntuplets + selection + output scan, fit; n = entries written (<= cap).
 * Source: none (measurement plumbing; the paper gives no per-kernel times, §5). */
int pxr_plan_stage_ms(pxr_plan *plan, float *ms, int cap, int *n);

/* Wait for the plan's last run and release it.  Call before pxr_destroy of its context (which
 * otherwise destroys it).
 * Source: none (library plumbing). */
void pxr_plan_destroy(pxr_plan *plan);

/*
 * Fit-only path over device-resident ntuplets (the precision study): m ntuplets of nh[t] hits
 * (3..PXR_MAX_HITS), hit h of ntuplet t at x[t*stride + h] (device float arrays), layer ids
 * likewise.  Outputs are device arrays of m elements.  fit_mode selects the arithmetic.
 * Source: §2, the Tracks module's fit of hit n-tuplets (the broken line, Blobel 2006, is this
 * library's reading; the paper names no fit).
 */
int pxr_fit_batch(pxr_ctx *ctx, uint32_t m, const uint8_t *nh, const float *x, const float *y,
                  const float *z, const uint16_t *layer, uint32_t stride,
                  const pxr_params *params, double *pt, double *phi, double *cot_theta,
                  double *dxy, double *dz, double *chi2, int8_t *charge, int8_t *fit_status,
                  void *stream);

/*
 * Allocation-free doublet building for one event.  The paper has no counterpart: this entry
 * point exists for callers that cannot let a library allocate device memory, such as serving
 * loops that must not call cudaMalloc after start-up (it synchronises the device and stalls the
 * other streams) and applications whose device memory is owned entirely by their own pool.
 * It runs the hit sort and the doublet stage of the other entry points (same cells, same
 * arithmetic) with all scratch in one fixed array in device global memory that the library
 * holds on every GPU that loads it (about 6.4 MB) until the process exits; it calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *
 * Inputs (device): x, y, z, layer of n_hits hits (n_hits <= 65536).  Outputs (device):
 * cells_inner[cap], cells_outer[cap] receive the cells as caller hit indices (cap <= 1048576),
 * *n_cells the number of cells found (may exceed cap: then only cap are written), *flags
 * (optional, may be NULL) the event's flag word: bit 1 = more cells than cap (the first cap
 * cells found are written, in no particular order), bit 8 = at least one hit has a layer id
 * >= params->n_layers (such hits are left out of every cell; the other hits' cells are
 * unaffected); other bits are 0.  stream: cudaStream_t or NULL.  Asynchronous: results are valid
 * once the stream reaches them.
 * The first call on each device resolves the scratch array's device address and sets kernel
 * attributes (with that device current); make that first call before any stream capture.
 * Every call shares the scratch array and it keeps the last call's contents: calls whose work
 * overlaps on the GPU race on it and must be ordered by the caller (one stream, or events).
 * Errors: PXR_EINVAL for sizes beyond the limits or bad parameters (nothing is launched),
 * PXR_ECUDA when a CUDA error was already pending before the call (nothing is launched; the
 * error is left pending) or a launch failed (the message names the launch).
 */
int pxr_doublets_noalloc(const float *x, const float *y, const float *z, const uint16_t *layer,
                         uint32_t n_hits, const pxr_params *params, uint32_t *cells_inner,
                         uint32_t *cells_outer, uint32_t cap, uint32_t *n_cells,
                         uint32_t *flags, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PXR_H */
