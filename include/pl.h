/* libpl: GB300 (sm_103a) area-hint refinement placement initializer.
 *
 * C ABI of the data-parallel hot path of "Bridging the Initialization Gap: A
 * Co-Optimization Framework for Mixed-Size Global Placement" (arXiv
 * 2511.10073):
 *   A1  netlist hypergraph -> static instance graph with macro pin expansion
 *       (Sec. V "Macro pin expansion"; the graph G = (V, E) of Sec. IV);
 *   A0  GSP-based initialization: multi-band normalized-adjacency filter
 *       (Sec. IV, multi-band filter H and its three-step procedure);
 *   A2  area hints: macro virtual nodes with repulsive edges and bin virtual
 *       nodes with density-aware signed edges (Sec. V);
 *   A3  signed Laplacian L_hint and its Gershgorin bound lambda_up (Sec. V,
 *       refinement filter H_r);
 *   A4  refinement filter H_r = ((lambda_up I - L_hint)/lambda_up)^k applied
 *       in the relaxed fixed-point iteration of Algorithm 1;
 *   A5  half-perimeter wirelength, the paper's quality metric (Sec. VII-VIII).
 *
 * Conventions
 *   - Every pointer in pl_netlist and every coordinate buffer is a DEVICE
 *     pointer owned by the caller, unless a parameter says "host".
 *   - Coordinates are interleaved FP32 pairs (x0, y0, x1, y1, ...).  "cells"
 *     buffers hold num_cells pairs; "nodes" buffers hold pl_graph_info()'s N
 *     pairs in node order: [cells][macro pins][star nodes][macro virtual
 *     nodes][bin nodes, row-major, x fastest].
 *   - Calls are issued on the given stream.  Calls that must learn sizes from
 *     the device (graph builds) synchronize that stream; pl_filter_init reads
 *     the device status once at its end.  No call aborts, traps or spins
 *     without bound; failures come back as a pl_status and pl_last_error().
 *   - Each pl_graph owns a second stream.  Graph builds and sparse products
 *     fork part of their work onto it (an event recorded on the given stream)
 *     and join it back (the given stream waits on an event), so every call
 *     still completes in the order of the given stream.
 *   - The library allocates no device memory.  A graph's device buffers are
 *     carved from a workspace the caller passes to pl_build_graph (sized by
 *     pl_workspace_size); pl_hpwl takes its own small workspace.  The
 *     library owns only the host-side pl_graph object, freed by
 *     pl_graph_destroy.
 *   - One pl_graph must not be used from two host threads at once; different
 *     graphs may be (pl_filter_init_batch does), and static builds on several
 *     threads take turns.
 */
#ifndef PL_H
#define PL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *pl_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  PL_OK = 0,
  PL_ERR_INVALID_ARG = 1, /* bad pointer, size, index, parameter or netlist content */
  PL_ERR_CUDA = 2,        /* a CUDA runtime call failed (message in pl_last_error) */
  PL_ERR_WORKSPACE = 3,   /* caller workspace too small */
  PL_ERR_OOM = 4,         /* device allocation failed */
  PL_ERR_SPECTRUM = 5,    /* lambda_up <= 0 or not finite: no refinement filter */
  PL_ERR_NONFINITE = 6,   /* a coordinate given to the library is NaN or infinite */
  PL_ERR_TIMEOUT = 7,     /* a bounded device-side wait gave up: the learned filter's
                             tensor-core kernels wait on their own MMAs for at most
                             about 2 s (no kernel waits on another block) */
  PL_ERR_UNSUPPORTED = 8  /* input beyond a documented size limit */
} pl_status;

typedef enum { PL_W_FP32 = 1, PL_W_BF16 = 2 } pl_wdtype;

/* The placement instance (Sec. IV problem statement): objects V = I/Os,
 * macros, standard cells; nets E as a pin -> net incidence. */
typedef struct {
  int32_t num_cells;         /* cells = movable std cells + fixed macros + fixed I/Os */
  int32_t num_nets;
  int64_t num_pins;          /* = net_ptr[num_nets] */
  const int64_t *net_ptr;    /* [num_nets+1] pin ranges, net_ptr[0] = 0, nondecreasing */
  const int32_t *pin_cell;   /* [num_pins] cell of each pin, in [0, num_cells) */
  const float *pin_dx;       /* [num_pins] pin offset from its cell centre, or NULL (0) */
  const float *pin_dy;
  const float *cell_w;       /* [num_cells] width, height (>= 0; > 0 for macros) */
  const float *cell_h;
  const uint8_t *cell_kind;  /* [num_cells] 0 movable, 1 fixed macro, 2 fixed I/O */
  const float *fixed_x;      /* [num_cells] centre, read for kind != 0 */
  const float *fixed_y;
  double xl, yl, xh, yh;     /* placement region, xh > xl, yh > yl */
} pl_netlist;

/* Table I parameters plus the readings the paper leaves open. */
typedef struct {
  int32_t clique_max;        /* nets with <= clique_max distinct nodes are cliques, 2..16 */
  int32_t wdtype;            /* pl_wdtype: storage type of edge weights */
  int32_t gift_enable;       /* run the GSP initialization filter (A0) */
  int32_t gift_center;       /* filter coordinates relative to the region centre */
  int32_t gift_k[3];         /* low, mid, high band: exponent k (Table I *_filter_k) */
  double gift_sigma[3];      /* self-loop sigma > 0 (Table I *_filter_sigma) */
  double gift_alpha[3];      /* band weights (Table I *_filter_effect) */
  int32_t t_hint;            /* refinement iterations T_hint (Table I refine_iteration) */
  int32_t nbx, nby;          /* refinement bins (Table I refine_num_bin_xy) */
  double gamma;              /* relaxation in [0, 1] (Algorithm 1) */
  double det_ratio;          /* detection window ratio (Table I detection_ratio) */
  double capacity;           /* bin capacity C (Table I bin_capacity) */
  double mu;                 /* logistic slope of phi_b (Sec. V) */
  int32_t ntaps;             /* 1..4 filter taps: g~ = sum_t alpha_t H_r^{k_t} g */
  int32_t tap_k[4];          /* strictly increasing orders, 1..64 */
  double tap_alpha[4];
  int32_t pin_every_step;    /* re-pin fixed nodes after every power of H_r */
  int32_t clamp;             /* clamp movable centres into the region */
} pl_params;

typedef struct pl_graph pl_graph;

/* Defaults: clique_max 16, FP32 weights, GiFt bands (k, sigma, alpha) =
 * (4, 4, 0.7), (2, 4, 0.2), (2, 2, 0.1), T_hint 3, 32 x 32 bins, gamma 0.5,
 * detection ratio 0.1, capacity 1, mu 4, one tap of order 8, clamping on. */
void pl_params_default(pl_params *p);

/* Device bytes that a graph of `nl` built with `p` may take from its
 * workspace: an upper bound computed on the host from the netlist's sizes and
 * the parameters (no device access).  It covers the static build (A1), any
 * number of hint builds (each reuses the same part of the workspace), GiFt and
 * the refinement filter, given that the macro-cell overlaps of one hint build
 * are at most 16 per movable cell on average.  0 for a NULL or negative-size
 * argument. */
size_t pl_workspace_size(const pl_netlist *nl, const pl_params *p);

/* A1 (+ A2/A3 when xy_nodes != NULL).  Builds the static instance graph of
 * `nl` (Sec. IV problem statement, Sec. V macro pin expansion) into *g:
 * creates the graph when *g == NULL, otherwise rebuilds it in place (the
 * netlist may differ).  ws: device memory of ws_bytes bytes, 256-byte aligned,
 * owned by the caller, holding every device buffer of the graph; it needs no
 * initialisation, must stay allocated and untouched while the graph is in use,
 * and may be released after pl_graph_destroy or after a rebuild with another
 * workspace.  pl_workspace_size(nl, p) bytes always suffice.  With xy_nodes
 * (device, N pairs) it also builds the area-hint graph for that placement (as
 * pl_build_hints).  Synchronizes `stream`.
 * Errors: INVALID_ARG (netlist, params or workspace pointer), WORKSPACE (ws_bytes
 * too small; the message gives the bytes needed so far), UNSUPPORTED (a net
 * with more than 32768 pins, 2^28 or more static nodes (cells, macro pins and
 * stars), a graph row beyond 2^31 entries), OOM (host), CUDA, NONFINITE. */
pl_status pl_build_graph(const pl_netlist *nl, const pl_params *p, const float *xy_nodes,
                         void *ws, size_t ws_bytes, pl_stream stream, pl_graph **g);

/* Sizes of a built graph, written to host out[16]:
 *   0 num_cells  1 macro pin nodes  2 star nodes  3 macros  4 bins
 *   5 static nodes  6 N (all nodes)  7 static nnz  8 augmented nnz (0 before
 *   the first hint build)  9 window half-width x  10 half-width y
 *   11 long (hub-path) rows  12 movable cells  13 workspace bytes used at
 *   most so far  14 workspace bytes given  15 bytes held by the static build
 *   (hint builds start above them) */
pl_status pl_graph_info(const pl_graph *g, int64_t *out);

/* A2 + A3 for the node placement xy_nodes (device, N pairs): bin densities
 * and phi_b, macro and bin hint edges, the augmented signed graph, degrees and
 * lambda_up (Sec. V).  The bin hints are kept without stored columns: each
 * hint cell's detection-window weights as one block, the bin rows as their
 * transpose (pl_graph_export writes them out as ordinary entries).  Its
 * buffers come from the graph's workspace, above the static build's part.
 * Synchronizes `stream`.  Errors: NONFINITE (a movable cell coordinate),
 * SPECTRUM (lambda_up <= 0), UNSUPPORTED (more than 16 macro-cell overlaps
 * per movable cell), WORKSPACE, CUDA. */
pl_status pl_build_hints(pl_graph *g, const pl_params *p, const float *xy_nodes,
                         pl_stream stream);

/* A4, one round of Algorithm 1 on the current augmented graph:
 * g~ = sum_t alpha_t H_r^{k_t} g, fixed nodes re-pinned, then
 * g' = (1 - gamma) g + gamma g~, re-pinned, movable centres clamped.
 * xy_in, xy_out: device, N pairs each, distinct buffers.  Synchronizes
 * `stream` to read the device status. */
pl_status pl_filter_apply(pl_graph *g, const pl_params *p, const float *xy_in, float *xy_out,
                          pl_stream stream);

/* A0 steps 2-3: g' = sum_b alpha_b A~_{sigma_b}^{k_b} g on the static graph,
 * fixed nodes re-pinned, movable centres clamped.  Device, N pairs each.
 * Synchronizes `stream` to read the device status. */
pl_status pl_gift(pl_graph *g, const pl_params *p, const float *xy_in, float *xy_out,
                  pl_stream stream);

/* A0 step 1: movable cells from xy0_cells (device, num_cells pairs) or, when
 * NULL, uniform in the region from splitmix64(seed, counter 2i + axis); fixed
 * objects at their positions; star nodes at the mean of their net's nodes. */
pl_status pl_init_signal(pl_graph *g, uint64_t seed, const float *xy0_cells, float *xy_nodes,
                         pl_stream stream);

/* The whole initializer: A0 (pl_init_signal, then pl_gift when gift_enable)
 * followed by T_hint rounds of A2-A4.  xy_out_cells: device, num_cells pairs.
 * Reads the device status once at the end (synchronizes `stream`). */
pl_status pl_filter_init(pl_graph *g, const pl_params *p, uint64_t seed, const float *xy0_cells,
                         float *xy_out_cells, pl_stream stream);

/* The batched serving form: the whole initializer (as pl_filter_init, from
 * the seed, no given placement) of n designs, each on its own built graph
 * (Algorithm 1 runs per design, so designs are independent).  A design's
 * result is the same bits as its pl_filter_init call.  Two forms (opts):
 *  - union_products = 1 (the default): A0 and each round's hint build run
 *    per design, on worker threads that each drive one of the caller's
 *    streams (largest design first); each round's filter then runs as one
 *    launch per kernel and power over all designs, a block-diagonal union of
 *    the designs' matrices with each design's own lambda_up and coefficients
 *    (on streams[0] and the first graph's second stream);
 *  - union_products = 0: each worker runs whole initializers, one design at a
 *    time.
 * xy_out_cells[i]: device, graphs[i]'s num_cells pairs.  Returns after every
 * design is done.  ws: device, 256-byte aligned, pl_batch_workspace_size(n, p)
 * bytes (only the union form uses it; may be NULL for the other).  Graph
 * builds do not run here: build the graphs first (pl_build_graph calls on
 * several threads take turns).  The union form needs one weight type for all
 * graphs.  Errors: INVALID_ARG, WORKSPACE, or the first failing design's
 * status (its index in pl_last_error). */
typedef struct {
  int32_t union_products;   /* 1: one launch per kernel and power over all designs; 0: per design */
  int32_t streams;          /* how many of the caller's streams to use, 1..nstreams (0: all) */
  int32_t rows_ctas_per_sm; /* CTAs per SM of the union short-row kernel, 1..5 (0: 5) */
} pl_batch_opts;

/* Defaults: union form, all streams, 5 CTAs per SM. */
void pl_batch_opts_default(pl_batch_opts *o);
size_t pl_batch_workspace_size(int32_t n, const pl_params *p);
pl_status pl_filter_init_batch(int32_t n, pl_graph *const *graphs, const pl_params *p,
                               const uint64_t *seeds, float *const *xy_out_cells,
                               int32_t nstreams, const pl_stream *streams,
                               const pl_batch_opts *opts, void *ws, size_t ws_bytes);

/* The batch form's autotuner: runs pl_filter_init_batch once for each
 * candidate (per-design form on 1, 2, 4, 8, 16 streams; union form on 4, 8,
 * 16 streams with 3, 4, 5 short-row CTAs per SM; streams at most nstreams),
 * timing each call on the host clock after a device synchronisation, and
 * writes the fastest to *best (and its time in ms to *best_ms, may be
 * NULL).  Every candidate gives the same bits, so xy_out_cells holds the
 * result.  Errors: as pl_filter_init_batch. */
pl_status pl_batch_autotune(int32_t n, pl_graph *const *graphs, const pl_params *p,
                            const uint64_t *seeds, float *const *xy_out_cells, int32_t nstreams,
                            const pl_stream *streams, void *ws, size_t ws_bytes,
                            pl_batch_opts *best, double *best_ms);

/* A5: writes sum over nets of (max - min) pin x + (max - min) pin y, pin =
 * cell centre (xy_cells, device) + offset, as one double to *hpwl (device).
 * ws: device scratch of at least pl_hpwl_workspace_size(num_nets) bytes, 256-
 * byte aligned; its contents need no initialisation and are left zeroed for
 * the next call.  Does not synchronize.  net_ptr must be valid (as checked
 * by pl_build_graph); a pin_cell outside [0, num_cells) is not read and makes
 * *hpwl NaN.  Errors: INVALID_ARG, WORKSPACE, CUDA. */
size_t pl_hpwl_workspace_size(int32_t num_nets);
pl_status pl_hpwl(const pl_netlist *nl, const float *xy_cells, double *hpwl, void *ws,
                  size_t ws_bytes, pl_stream stream);

/* pl_hpwl without a workspace, for callers that cannot allocate device memory
 * or hand scratch to a library: a host that owns all device memory through
 * its own pool and gives plug-ins no allocator, or a code path where an
 * allocation (which may synchronize the device) is not allowed.  No counterpart
 * in the paper.  Same result as pl_hpwl (same kernel and grid).  The scratch is
 * a fixed device array of about 10 KB inside the library (ticket words plus
 * one partial sum for each of at most 1216 blocks, the largest grid the HPWL
 * kernel uses); every GPU that loads the library keeps it until the process
 * exits.  Any num_nets >= 0 fits; a call that would need more than that array
 * is rejected with PL_ERR_UNSUPPORTED.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) and should be made before any
 * stream capture.  All calls share the array and each call clears its ticket
 * words first, so calls that overlap on the GPU (on different streams) race.
 * Allocates nothing; does not synchronize.  Errors: INVALID_ARG, UNSUPPORTED,
 * CUDA. */
pl_status pl_hpwl_noalloc(const pl_netlist *nl, const float *xy_cells, double *hpwl,
                          pl_stream stream);

/* Sec. VI: macro charge densities scheduled over the T iterations of global
 * placement, and their integrals over the bins (the macro part of each bin's
 * density at iteration t).  Four models, as the paper defines them:
 *   PL_RHO_GAUSS    charge redistribution: an area-normalized 2D Gaussian
 *                   truncated to the footprint, eta(t) blended from scheme A
 *                   (edge decay ratio r0 -> r1, log-linear) and scheme B (FWHM
 *                   beta_min -> beta_max, linear) by a smoothstep between
 *                   alpha0 and alpha1 of a = t / T;
 *   PL_RHO_EXP      charge restoration, exponential-like, sigma(t) =
 *                   -sigma_factor T ln(1 - t / T);
 *   PL_RHO_LINEAR   linear-like, clamped at 0, k(t) = k_factor / tan(pi t / 2T);
 *   PL_RHO_SIGMOID  sigmoid-like, the same k(t).
 * The paper gives no values besides T = 300 for its figure; the defaults are
 * readings.  panels x nodes: the composite Gauss-Legendre rule per axis of
 * the models without a closed form. */
typedef enum { PL_RHO_GAUSS = 0, PL_RHO_EXP = 1, PL_RHO_LINEAR = 2, PL_RHO_SIGMOID = 3 } pl_rho_model;
typedef struct {
  int32_t model;             /* pl_rho_model */
  int32_t T;                 /* iterations of the schedule, >= 1 */
  double r0, r1;             /* scheme A, in (0, 1) */
  double beta_min, beta_max; /* scheme B, > 0 */
  double alpha0, alpha1;     /* blend window, alpha0 < alpha1 */
  double sigma_factor;       /* > 0 */
  double k_factor;           /* > 0 */
  int32_t panels, nodes;     /* 1..64 panels, 1..32 nodes */
} pl_rho_params;

/* Defaults: Gaussian, T 300, r 0.05 -> 0.9, beta 0.25 -> 1.5, blend 0.3..0.7,
 * sigma_factor 0.002, k_factor 0.5, 4 panels of 8 nodes. */
void pl_rho_params_default(pl_rho_params *p);

/* rho[b] (device, nbx * nby doubles, bins row-major with x fastest over the
 * region) = sum over macros, ascending, of the integral of macro m's density
 * at iteration t (0 <= t <= T) over bin b, in area units.  mx, my, mw, mh:
 * device, the macros' centres and sizes.  FP64.  Needs no workspace; does not
 * synchronize.  Errors: INVALID_ARG, CUDA. */
pl_status pl_macro_density(const pl_rho_params *rp, int32_t t, int32_t num_macros,
                           const float *mx, const float *my, const float *mw, const float *mh,
                           double xl, double yl, double xh, double yh, int32_t nbx, int32_t nby,
                           double *rho, pl_stream stream);

/* ------------------------------------------------------------------------
 * The learned refinement filter: a small learned stand-in for the plain
 * refinement filter of Sec. V (Algorithm 1's filter step), with fewer sparse
 * products.  Three taps at powers k0 < k1 < k2 of H_r and a per-node MLP on
 * tensor cores.  In bin units about the region centre c (s the bin size per
 * axis), G_t = (H_r^{k_t} g - c) / s and
 *   P_v = theta_0 G0 + theta_1 G1 + theta_2 G2 + a_v (G1 - G0) + b_v (G2 - G0)
 *         + (o_v^x, o_v^y),
 *   (a_v, b_v, o_v^x, o_v^y) = W2 relu(W1 x_v + b1) + b2,  g~_v = c + s P_v,
 * x_v the node's 16 features, normalised ((f - mu) * isd) and rounded to
 * BF16; W1 (64 x 16) and W2 (4 x 64) are used as BF16, the hidden layer is
 * rounded to BF16, and both layers accumulate in FP32 (tcgen05.mma, kind::f16,
 * accumulators in TMEM).  The features: 0-1 G1 - G0, 2-3 G2 - G0, 4 D_vv /
 * lambda_up, 5 sum_j |w_vj| / lambda_up, 6 (negative weights) / lambda_up,
 * 7 phi_b of a hint cell's bin, 8 hint cell, 9 star node, 10 a movable
 * cell's area over the bin area, 11 round t / T_hint, 12-15 zero.  The round
 * then ends as the plain filter's: fixed nodes re-pinned, relaxation by gamma,
 * re-pinned, movable centres clamped.  No counterpart in the paper: the paper
 * applies the plain filter, which stays the judge of this one (the records
 * below are its outputs).
 *
 * Parameter vector (device, FP32, PL_LEARNED_SIZE floats, in this order):
 * mu[16], isd[16], theta[3], W1[64][16], b1[64], W2[4][64], b2[4]. */
#define PL_LEARNED_NF 16
#define PL_LEARNED_HID 64
#define PL_LEARNED_NOUT 4
#define PL_LW_MU 0
#define PL_LW_ISD 16
#define PL_LW_THETA 32
#define PL_LW_W1 35
#define PL_LW_B1 1059
#define PL_LW_W2 1123
#define PL_LW_B2 1379
#define PL_LEARNED_SIZE 1383
/* A training record: one free node (movable cell or star node) of one round,
 * 24 floats: raw features f[16], G0[2], G1[2], G2[2], and the target T[2] in
 * the same bin units: the filter output that the round's relaxation maps to
 * the plain round's result g' (re-pinned and clamped), (g' - (1 - gamma) g) /
 * gamma, which is the plain filter's g~ wherever clamping did not act.  (The
 * signed graph's H_r can amplify, so an unclamped g~ may lie far outside the
 * region; the clamped result is what the round keeps.) */
#define PL_LEARNED_REC 24

typedef struct {
  int32_t k[3];    /* tap powers, 0 <= k0 < k1 < k2 <= 64 */
  const float *w;  /* device, PL_LEARNED_SIZE floats */
} pl_learned;

/* One round of Algorithm 1 with the learned filter in place of the plain
 * one, on the current augmented graph (pl_build_hints at xy_in first): k2
 * refinement products, then one fused kernel (features, the MLP on tensor
 * cores, taps, relaxation, re-pinning, clamping).  round: t of Algorithm 1
 * (feature 11 = t / T_hint).  xy_in, xy_out: device, N pairs each, distinct.
 * Synchronizes `stream` to read the device status.  Errors: INVALID_ARG,
 * NONFINITE (the learned g~ of a free node is not finite), TIMEOUT, CUDA. */
pl_status pl_learned_apply(pl_graph *g, const pl_params *p, const pl_learned *m, int32_t round,
                           const float *xy_in, float *xy_out, pl_stream stream);

/* The whole initializer with the learned filter: A0 as pl_filter_init, then
 * T_hint rounds of A2, A3 and the learned round.  A round whose learned g~
 * is not finite is run again with the plain filter (the fallback); their
 * count goes to *fallbacks (host, may be NULL).  m == NULL runs the plain
 * filter in every round (the same bits as pl_filter_init).  Reads the device
 * status once per round.  Errors: as pl_filter_init, TIMEOUT. */
pl_status pl_filter_init_learned(pl_graph *g, const pl_params *p, const pl_learned *m,
                                 uint64_t seed, const float *xy0_cells, float *xy_out_cells,
                                 int32_t *fallbacks, pl_stream stream);

/* Check of the bounded waits above (no counterpart in the paper): one CTA
 * sets up as the learned kernels do (tensor memory, mbarrier), waits on an
 * mbarrier phase that nothing completes for at most `cycles` clocks
 * (1..4e9), frees its tensor memory and returns.  ws: device scratch of at
 * least 8192 bytes, 256-byte aligned.  Returns PL_ERR_TIMEOUT when the wait
 * gave up (the expected result; the context stays usable), PL_OK otherwise.
 * Synchronizes `stream`.  Errors: INVALID_ARG, WORKSPACE, CUDA. */
pl_status pl_learned_wait_check(int64_t cycles, void *ws, size_t ws_bytes, pl_stream stream);

/* The MLP alone on given raw features: out[i] (device, n x 4 floats) = the
 * four outputs for feat[i] (device, n x 16 floats), with the normalisation,
 * BF16 roundings and tensor-core arithmetic of pl_learned_apply.  w: device
 * parameter vector.  Does not synchronize.  Errors: INVALID_ARG, CUDA (a
 * timed-out wait leaves the rows of its tile as NaN). */
pl_status pl_learned_forward(const float *w, const float *feat, int64_t n, float *out,
                             pl_stream stream);

/* Training records of one round: with the hints built at xy_in, runs the
 * plain round of p (its result gives the target) and the powers k[0..2],
 * and writes one record per free node, in node order, to rec
 * (device, cap records of PL_LEARNED_REC floats); *count (host) = records
 * written.  round as in pl_learned_apply.  xy_in is not changed (advance the
 * trajectory with pl_filter_apply).  Synchronizes `stream`.  Errors:
 * INVALID_ARG (also gamma = 0: no filter output to learn), WORKSPACE (cap too
 * small; *count = records needed), CUDA. */
pl_status pl_learned_collect(pl_graph *g, const pl_params *p, const int32_t k[3], int32_t round,
                             const float *xy_in, float *rec, int64_t cap, int64_t *count,
                             pl_stream stream);

/* Training options.  Minibatches are batch_tiles tiles of 128 consecutive
 * records, the tiles in a fresh order every epoch (splitmix64 of seed and
 * epoch, Fisher-Yates); an epoch takes floor(full tiles / batch_tiles) steps
 * (at least one).  Adam (Kingma & Ba) with the learning rate on a cosine from
 * lr to lr_min over all steps.  fit_norm: set mu and isd from the records'
 * feature means and standard deviations first; fit_taps: set theta to the
 * least-squares taps first (both in FP64 over all records). */
typedef struct {
  int32_t epochs;       /* >= 1 */
  int32_t batch_tiles;  /* 1..1024 */
  double lr, lr_min, beta1, beta2, eps;
  uint64_t seed;
  int32_t fit_norm, fit_taps;
} pl_train_opts;

/* Defaults: 20 epochs, 128 tiles (16384 records), lr 2e-3 -> 1e-4, betas
 * 0.9 / 0.999, eps 1e-8, seed 1, both fits on. */
void pl_train_opts_default(pl_train_opts *o);

/* Device bytes of the workspace of pl_learned_train and pl_learned_loss for
 * nrec records (0 for a negative count). */
size_t pl_learned_train_ws(int64_t nrec);

/* Trains the parameter vector w (device, in/out; W1, W2, b1, b2 and theta
 * as initial values) on nrec >= 128 records (device) to minimise the mean
 * over records of ||P - T||^2 (bin units).  Forward on tensor cores as in
 * pl_learned_apply; backward on CUDA cores in FP32 (BF16 roundings passed
 * straight through), per-block partial gradients added in a fixed order, so
 * a run is reproducible.  epoch_loss (host, epochs doubles, may be NULL):
 * the mean minibatch loss of each epoch.  ws: device, 256-byte aligned,
 * pl_learned_train_ws(nrec) bytes.  Synchronizes `stream` once per epoch.
 * Errors: INVALID_ARG, WORKSPACE, TIMEOUT, CUDA. */
pl_status pl_learned_train(const float *rec, int64_t nrec, float *w, const pl_train_opts *o,
                           void *ws, size_t ws_bytes, double *epoch_loss, pl_stream stream);

/* The training loss over all nrec records (*loss, host) and, when grad
 * (device, PL_LEARNED_SIZE floats) is not NULL, its gradient (zero for mu
 * and isd).  Same kernels as pl_learned_train.  Synchronizes `stream`.
 * Errors: INVALID_ARG, WORKSPACE, TIMEOUT, CUDA. */
pl_status pl_learned_loss(const float *rec, int64_t nrec, const float *w, void *ws,
                          size_t ws_bytes, double *loss, float *grad, pl_stream stream);

/* Copies of the graph for exact comparison (all HOST buffers):
 * static CSR: rp[static nodes + 1], col[static nnz], w[static nnz] (stored
 * weight as double), base_w[num_cells] (baseWeight_i, FP64).
 * Synchronizes the graph's last stream. */
pl_status pl_graph_export_static(const pl_graph *g, int64_t *rp, int32_t *col, double *w,
                                 double *base_w);
/* augmented CSR in canonical order (rows ascending, columns ascending within
 * a row; the device stores a bin row as the concatenation of its window bins'
 * cell lists and this copy sorts it): rp[N+1], col[nnz], w[nnz], deg[N]
 * (signed degree D_ii), *lam_up, Db/Cb/phi[bins], cell_bin[num_cells] (-1 for
 * non-movable cells).  Any pointer may be NULL to skip that array. */
pl_status pl_graph_export(const pl_graph *g, int64_t *rp, int32_t *col, double *w, double *deg,
                          double *lam_up, double *Db, double *Cb, double *phi,
                          int32_t *cell_bin);

void pl_graph_destroy(pl_graph *g);

/* Benchmark hooks (no counterpart in the paper; for measuring this library).
 * pl_prof_enable(1) clears the records and starts counting: every kernel the
 * library launches is counted, and each sparse-product launch (A0, A4) is
 * bracketed by a CUDA event pair on its own stream.  pl_prof_enable(0) stops
 * recording and keeps the records.  pl_prof_read writes host out[8]:
 *   0 kernel launches between enable and disable (or now)
 *   1 refinement-filter (A4) launches  2 their summed time, ms
 *   3 their algorithmic bytes (indices + weights once, row pointers, x read,
 *     y written, one coefficient per row)
 *   4 GiFt (A0) launches  5 ms  6 algorithmic bytes
 * It synchronizes on the recorded events.  Process-wide, not per graph. */
void pl_prof_enable(int on);
pl_status pl_prof_read(double *out);

/* Message of the last failed call on this host thread ("" when none). */
const char *pl_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
