// Internal state of a libpl graph (host struct holding device buffers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/pl.h"
#include "pl_common.cuh"

namespace pl {

// SpMM work units: short rows (<= kLong entries) are read by a group of lanes
// each; long rows and every virtual-node row go to the hub path in chunks of
// kChunk.
constexpr int kLong = 128;
constexpr int kChunk = 512;
constexpr int kPad = 16;  // spare entries after the last one
constexpr int kRpPad = 8;  // spare row pointers after the last one
constexpr uint32_t kHubFlag = 0x80000000u;  // rp_s bit 31: the row is a hub row
constexpr uint32_t kOffMask = 0x7fffffffu;
// Macro-cell overlap pairs of one hint build, at most this many per movable
// cell on average (the workspace bound counts on it).
constexpr int kMaxCellMacros = 16;

// A split CSR matrix as the SpMM kernels read it.  Entries of short rows come
// first (row pointers rp_s; hub rows have zero length there and bit 31 set),
// entries of hub rows follow at absolute offsets lptr.  Two matrices exist:
//  * st, the static instance graph, built once per netlist;
//  * hm, the hint part of the augmented graph, rebuilt every round.  A row of
//    the augmented graph is its st part followed by its hm part; it is a hub
//    row (bit 31 of hm.rp_s) when it is a virtual node or has more than kLong
//    entries in total, and its st part then may sit in st's short region.
// Per hub row, lsb/lsl give its st piece and lhb/lhl its hm piece (absolute
// offsets, lengths); chunks of kChunk cover the concatenation.
struct SpMat {
  int64_t N = 0;
  uint64_t nnz_s = 0, nnz_l = 0;
  int32_t nlong = 0, nchunks = 0;
  Buf rp_s;     // uint32 [N+1+kRpPad], bit 31 = hub row
  Buf col;      // int32 [nnz_s + nnz_l + kPad]
  Buf w;        // float or uint16 (bf16) [same]
  Buf lrow;     // int32 [nlong] node of each hub row
  Buf lptr;     // uint64 [nlong+1] this matrix's part of each hub row (absolute)
  Buf lsb, lhb; // uint64 [nlong] st piece / hm piece of each hub row
  Buf lsl, lhl; // uint32 [nlong] their lengths
  Buf lchunk;   // int32 [nlong+1] first chunk of each hub row
  Buf chunk_lr; // int32 [nchunks] hub row of each chunk
  Buf longidx;  // int32 [N] hub index or -1
  Buf dsum;     // dfl [N] signed degree D_ii (hm: of the whole augmented row)
  Buf psum;     // dfl [N] sum of positive weights
  Buf c32;      // float [N] 1 - D_ii / lambda_up
  Buf c64l;     // double [nlong] same, FP64, hub rows
  Buf lam;      // 8-byte words: lambda_up, 1/lambda_up (double), the raw max key, the
                // count of window slots inside the grid and of hint cells (uint64)
  Buf part;     // float4 [nchunks] hub partial sums (two double-floats)
  int wbytes = 4;
};

}  // namespace pl

struct pl_graph {
  // sizes
  int32_t C = 0, M = 0;
  int64_t P = 0;
  int32_t Pm = 0, S = 0, Mm = 0, NB = 0, nbx = 0, nby = 0, hx = 0, hy = 0, nmov = 0;
  int64_t Nst = 0, N = 0;
  uint64_t nnz_static = 0;
  double xl = 0, yl = 0, xh = 0, yh = 0, wb = 0, hb = 0, abin = 0;
  int wdtype = PL_W_FP32, clique_max = 16;
  double det_ratio = 0.1;
  cudaStream_t stream = nullptr;
  bool have_hints = false;
  double lam_h[2] = {0.0, 0.0};  // lambda_up, 1 / lambda_up of the current hints

  // copies of the netlist
  pl::Buf cw, ch, ckind, cfx, cfy, net_ptr;
  pl::Buf pin_node;    // int32 [P]
  pl::Buf nd;          // int32 [P] distinct nodes of each net at its pin range start
  pl::Buf net_p;       // int32 [M] distinct node count
  pl::Buf star_of;     // int32 [M+1] scan of star flags
  pl::Buf star_net;    // int32 [S]
  pl::Buf star_p;      // int32 [S] node count of each star's net
  pl::Buf macro_cell;  // int32 [Mm]
  pl::Buf cell_macro;  // int32 [C+1] scan of macro flags
  pl::Buf srp;         // int64 [Nst+1] static row pointers (entries live in st)
  pl::Buf base_w;      // double [C]
  pl::Buf hflag;       // uint8 [C] movable with baseWeight > 0
  pl::Buf nkind;       // uint8 [N] 0 movable cell, 1 star, 2 fixed
  pl::Buf fixedp;      // float2 [N]
  pl::Buf bounds;      // float4 [N] clamp box of the centre
  pl::Buf amac, Cb;    // double [NB]
  pl::Buf carea;       // double [C] cell areas w h
  // macro lookup grid
  int32_t gnx = 1, gny = 1;
  double gsz = 1.0, gsx = 1.0, gsy = 1.0;
  pl::Buf gptr, glist; // int64 [gnx*gny+1], uint32 macro ids
  pl::Buf ggeo;        // float4 [..] centre and size of each listed macro
  pl::Buf mgeo;        // float4 [Mm] centre and size of each macro
  // per refinement round
  pl::Buf cell_bin;    // int32 [C]
  pl::Buf n_ovl;       // int32 [C]
  pl::Buf bcnt, boff, blist, bcur;  // bucket sort of movable cells by (bin, hint)
  pl::Buf mcnt, moff, mlist, mcur;  // cells overlapping each macro
  pl::Buf mtc, mtoff;  // per (macro, cell tile) counts and their scan (tiled macro lists)
  pl::Buf cmem;        // int32 [C * 8] each hint cell's macros (tiled macro lists)
  pl::Buf Db, phi;     // double [NB]
  pl::Buf slen;        // uint32 [N] short-region length (0 for hub rows)
  pl::Buf llen;        // uint64 [N] hub-region length (0 for short rows)
  pl::Buf clen;        // uint64 [N] chunked length of hub rows
  pl::Buf lflag;       // int32 [N+1] hub flag scan
  pl::Buf mac_base;    // uint64 [C] entry offset of a cell's first macro entry
  // bin hints without stored columns: each hint cell's window block and the
  // bin rows as its transpose over the bucket lists
  int W = 0;           // slots of a window, (2 hx + 1)(2 hy + 1)
  int64_t nslot = 0;   // window slots inside the bin grid, over all hint cells
  int64_t nhint = 0;   // hint cells (movable, baseWeight > 0)
  long long nbc_max = 0;  // bin-row chunks at most (grid of the chunk kernels)
  pl::Buf hbw;         // storage type [C * W] window-block weights of hint cells
  pl::Buf hbwq;        // storage type [chunks * W * kBinChunk] the blocks of each bin-row
                       // chunk's hint cells, slot-major (read slot by slot by the bin rows)
  pl::Buf hbin;        // int32 [C] bin of a hint cell, -1 for other cells
  pl::Buf bchunk;      // int32 [NB + 1] first chunk of each bin's hint bucket
  pl::Buf cown;        // int32 [chunks] bin of each chunk
  pl::Buf bdeg;        // float4 [chunks * W] degree partials of the bin rows
  pl::Buf bpart;       // float4 [chunks * W] product partials of the bin rows
  pl::Buf hubtmp;      // int32 scratch for merging bin rows
  pl::SpMat st;        // static matrix (A0)
  pl::SpMat hm;        // augmented matrix (A2-A4)
  // filter state
  pl::Buf xa, xb, xc, g0; // float2 [N]
  pl::Buf ua, ub;         // float [N * 2 * nchain]
  pl::Buf acc;            // double2 [N]
  pl::Buf gsc;            // float [6 * N] GiFt coefficients (a, b, sqrt(d)) of two chains
  pl::Buf q4a, q4b;       // float4 [N] GiFt chain pair, (x1, y1, x2, y2) per node
  pl::Buf status;         // int32 [8]
  pl::Buf stage;          // staging words of batched device-to-host reads
  pl::Buf star_w;         // double [kMaxNetPins + 1] star edge weights p / (p - 1)
  pl::Buf lscr;           // int32 [N / 1024 + 2] learned filter: free nodes per block of 1024
  // device memory: the caller's workspace.  The static build takes the bottom
  // of it (up to hint_mark); every hint build starts again at hint_mark.
  pl::Arena arena;
  size_t hint_mark = 0;
  cudaStream_t side = nullptr;  // the hint build's second stream (forked from and joined
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;  // back to the caller's stream)
  cudaStream_t side2 = nullptr;  // a third stream of the hint build, joined by ev_join2
  cudaEvent_t ev_join2 = nullptr;
  bool star_w_ok = false;
  // launch shapes of the sparse products on the graph's device (0 = not yet
  // looked up): SM count, resident blocks per SM of the short-row kernels by
  // [mode][weight type] and of the chain-pair kernel by weight type
  int nsm = 0;
  int occ_rows[2][2] = {{0, 0}, {0, 0}};
  int occ_rows4[2] = {0, 0};
  pl::Buf tmp[8];
  pl::Buf lay[4];         // layout scratch (scans of row lengths, chunk counts)
  pl::Buf hubf;           // uint8 [N] hub flags of a layout
};

namespace pl {

__global__ void k_cell_area(int32_t C, const float *cw, const float *ch, double *area);

// Every device buffer of a graph.  kind 0: all; kind 1: those a hint build
// takes anew (its own results and the scratch buffers every phase shares).
template <typename F>
void for_each_buf(pl_graph *g, int kind, F f) {
  Buf *hint[] = {&g->tmp[0], &g->tmp[1], &g->tmp[2], &g->tmp[3], &g->tmp[4], &g->tmp[5],
                 &g->tmp[6], &g->tmp[7], &g->lay[0], &g->lay[1], &g->lay[2], &g->lay[3],
                 &g->hubf, &g->slen, &g->llen, &g->clen, &g->lflag, &g->hubtmp, &g->cell_bin,
                 &g->n_ovl, &g->bcnt, &g->boff, &g->blist, &g->bcur, &g->mcnt, &g->moff,
                 &g->mlist, &g->mcur, &g->mtc, &g->mtoff, &g->cmem, &g->Db, &g->phi,
                 &g->mac_base, &g->hbw, &g->hbwq, &g->hbin, &g->bchunk, &g->cown, &g->bdeg,
                 &g->bpart};
  for (Buf *b : hint) f(*b);
  SpMat *ms[] = {&g->hm, &g->st};
  for (int i = 0; i < (kind == 0 ? 2 : 1); ++i) {
    SpMat *m = ms[i];
    Buf *mb[] = {&m->rp_s, &m->col, &m->w, &m->lrow, &m->lptr, &m->lsb, &m->lhb,
                 &m->lsl, &m->lhl, &m->lchunk, &m->chunk_lr, &m->longidx,
                 &m->dsum, &m->psum, &m->c32, &m->c64l, &m->lam, &m->part};
    for (Buf *b : mb) f(*b);
  }
  if (kind != 0) return;
  Buf *rest[] = {&g->cw, &g->ch, &g->ckind, &g->cfx, &g->cfy, &g->net_ptr, &g->pin_node,
                 &g->nd, &g->net_p, &g->star_of, &g->star_net, &g->star_p, &g->macro_cell,
                 &g->cell_macro, &g->srp, &g->base_w, &g->hflag, &g->nkind, &g->fixedp,
                 &g->bounds, &g->amac, &g->Cb, &g->carea, &g->gptr, &g->glist, &g->ggeo, &g->mgeo,
                 &g->xa, &g->xb, &g->xc, &g->g0, &g->ua, &g->ub, &g->acc, &g->gsc, &g->q4a,
                 &g->q4b, &g->status, &g->stage, &g->star_w, &g->lscr};
  for (Buf *b : rest) f(*b);
}

void set_error(const char *fmt, ...);
void clear_error();
pl_status cuda_fail(cudaError_t e, const char *what);

pl_status build_static(pl_graph *g, const pl_netlist *nl, const pl_params *p, cudaStream_t s);
pl_status take_filter_buffers(pl_graph *g);
double workspace_bound(const pl_netlist *nl, const pl_params *p);
pl_status build_hints(pl_graph *g, const pl_params *p, const float *xy, cudaStream_t s);
pl_status prepare_static_layout(pl_graph *g, cudaStream_t s);
pl_status run_init_signal(pl_graph *g, uint64_t seed, const float *xy0, float *xy, cudaStream_t s);
pl_status run_gift(pl_graph *g, const pl_params *p, const float *in, float *out, cudaStream_t s);
pl_status run_filter(pl_graph *g, const pl_params *p, const float *in, float *out, cudaStream_t s);
pl_status run_powers(pl_graph *g, const pl_params *p, const float *in, const int32_t k[3],
                     const float2 *out[3], cudaStream_t s);
pl_status clamp_nodes(pl_graph *g, const pl_params *p, const float *in, float *out, cudaStream_t s);
pl_status check_model(const pl_learned *m);
pl_status check_params(const pl_params *p);
pl_status same_layout(const pl_graph *g, const pl_params *p);
size_t batch_ws_bytes(int nd, const pl_params *p);
pl_status run_filter_batch(pl_graph *const *gs, int nd, const pl_params *p, const float *const *in,
                           float *const *out, void *ws, size_t ws_bytes, int rows_ctas,
                           cudaStream_t s, cudaStream_t sh);
pl_status run_learned(pl_graph *g, const pl_params *p, const pl_learned *m, int32_t round,
                      const float *in, float *out, cudaStream_t s);
pl_status read_status(pl_graph *g, cudaStream_t s);

}  // namespace pl

namespace pl {
// The graph's second stream and its fork/join events, created on first use.
inline cudaError_t ensure_side(pl_graph *g) {
  if (g->side) return cudaSuccess;
  cudaError_t e = cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming);
  return e;
}
// The third stream and its join event, created on first use.
inline cudaError_t ensure_side2(pl_graph *g) {
  cudaError_t e = ensure_side(g);
  if (e != cudaSuccess || g->side2) return e;
  e = cudaStreamCreateWithFlags(&g->side2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_join2, cudaEventDisableTiming);
  return e;
}
}  // namespace pl
