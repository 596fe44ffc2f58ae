// pl_workspace_size: an upper bound of the device bytes one graph takes from
// its caller's workspace, from the netlist's sizes and the parameters alone
// (no device access).  It follows every buffer request of the static build
// (pl_graph.cu), of a hint build (pl_hints.cu; each hint build starts again
// where the static build ended) and of the filters (pl_filter.cu), each at
// its largest size given:
//   macros <= cells, macro pin nodes <= pins, star nodes <= pins / (clique_max + 1),
//   entries before merging <= max(clique_max - 1, 2) * pins (a p-node clique gives
//     p (p - 1), a star 2 p),
//   macro-cell overlaps <= kMaxCellMacros per movable cell,
//   macro lookup grid <= 2048 x 2048 buckets, each macro in at most 36 (the
//     bucket is at least half the largest macro or cell side),
// and every request rounded up to 256 bytes plus 256 of alignment.
#include <algorithm>
#include <cmath>

#include "pl_bins.cuh"
#include "pl_internal.h"

namespace pl {

namespace {
struct Plan {
  double b = 0.0;  // doubles: no overflow for absurd inputs
  void add(double n) { b += std::ceil(n / 256.0) * 256.0 + 256.0; }
};
double scan_b(double n) { return (double)scan_tmp_bytes((long long)std::min(n, 9.0e18)) + 4096.0; }
double seg_b(double nseg, double nkeys) {  // 4-byte keys
  return (double)segsort_tmp_bytes((long long)std::min(nseg, 4.0e18), (long long)std::min(nkeys, 4.0e18), 4);
}
}  // namespace

double workspace_bound(const pl_netlist *nl, const pl_params *p) {
  const double C = nl->num_cells, M = nl->num_nets, NP = (double)nl->num_pins;
  const double NB = (double)p->nbx * p->nby, cq = p->clique_max;
  const double sw = p->wdtype == PL_W_BF16 ? 2.0 : 4.0;
  int nx = (int)std::floor(p->det_ratio * (double)p->nbx), ny = (int)std::floor(p->det_ratio * (double)p->nby);
  nx = std::max(nx, 1);
  ny = std::max(ny, 1);
  const double W = (double)(2 * ((nx - 1) / 2) + 1) * (double)(2 * ((ny - 1) / 2) + 1);
  const double Mm = C, Pm = NP, S = std::floor(NP / (cq + 1.0));
  const double Nst = C + Pm + S, N = Nst + Mm + NB;
  const double npre = std::max(cq - 1.0, 2.0) * NP;
  const double ng = 2048.0 * 2048.0, nreg = 36.0 * Mm;
  Plan st;
  // netlist copies, validation, macros and macro pins
  for (int k = 0; k < 4; ++k) st.add(C * 4 + 16);
  st.add(C + 16);
  st.add((M + 1) * 8);
  st.add(64);
  st.add(C + 256);
  st.add((C + 1) * 4);
  st.add(scan_b(std::max(C, NP)));
  st.add(std::max(NP, M) + 256);
  st.add((NP + 1) * 4 + 256);
  st.add(512);  // staging of device-to-host reads
  st.add(Mm * 4 + 16);
  st.add(NP * 4 + 16);
  st.add(NP * 4 + 16);
  // distinct nodes per net, star nodes
  st.add(M * 4 + 16);
  st.add(seg_b(M, NP));
  st.add((M + 1) * 4);
  st.add(scan_b(M));
  st.add(S * 4 + 16);
  st.add(S * 4 + 16);
  // expansion, sort and merge
  st.add((Nst + 1) * 4 + 256);
  st.add((Nst + 1) * 8 + 256);
  st.add(scan_b(Nst));
  st.add(std::ceil((npre + 4) * 4 / 16.0) * 16 + (Nst + 1) * 8 + 512);
  st.add(npre * 12 + 512);
  st.add(seg_b(Nst, npre));
  st.add((Nst + 1) * 8);
  // static layout (row lengths, the split matrix)
  const double nchunk_st = N + npre / kChunk + 1;
  st.add(N * 4 + 16);
  st.add(N * 8 + 16);
  st.add(N * 8 + 16);
  st.add(N + 256);
  st.add(scan_b(N + 1));
  st.add((N + 1) * 8 + 256);
  st.add((N + 1) * 8 + 256);
  st.add((N + 1) * 4 + 256);
  st.add((N + 1 + kRpPad) * 4);
  st.add((npre + kPad) * 4);
  st.add((npre + kPad) * sw);
  for (double b : {4.0, 8.0, 8.0, 4.0, 4.0}) st.add(N * b + 16);  // lrow, lsb, lhb, lsl, lhl
  st.add((N + 1) * 8);                                            // lptr
  st.add(N * 4 + 16);                                             // longidx
  st.add((N + 1) * 4);                                            // lchunk
  st.add((N + 1) * 4 + 256);                                      // chunk counts
  st.add(nchunk_st * 4 + 16);
  st.add(N * 8 + 16);
  st.add(N * 8 + 16);
  st.add(N * 4 + 16);
  st.add(N * 8 + 16);
  st.add(64);
  st.add((nchunk_st + 1) * 48);
  // baseWeight, hint flags, star weights, node tables, bins, macro geometry
  st.add(C * 8 + 16);
  st.add(C + 16);
  st.add((32768.0 + 1) * 8);
  st.add(N + 16);
  st.add(N * 8 + 16);
  st.add(N * 16 + 16);
  st.add(C * 8 + 16);  // cell areas
  st.add(NB * 8 + 16);
  st.add(NB * 8 + 16);
  st.add(Mm * 16 + 16);
  // macro lookup grid
  st.add((ng + 1) * 8 + 16);
  st.add((ng + 1) * 4 + 256);
  st.add(scan_b(ng));
  st.add(nreg * 4 + 16);
  st.add((ng + 1) * 4 + 256);
  st.add(seg_b(ng, nreg));
  st.add(nreg * 16 + 16);
  // filter buffers, taken once at the end of the static build
  for (int k = 0; k < 6; ++k) st.add(N * 8 + 64);
  st.add(N * 16 + 16);
  st.add(N * 24 + 64);
  st.add(N * 16 + 64);
  st.add(N * 16 + 64);
  st.add((std::floor(N / 1024.0) + 2) * 4 + 64);  // learned filter's block counts

  // one hint build
  Plan h;
  const double nmov = C, nml = nmov * kMaxCellMacros, nbk = 2 * NB;
  const double ntile = std::max(1.0, std::ceil(C / 4096.0));
  const double nmt = Mm * ntile, ncm = nbk * ntile;
  h.add(scan_b(N + 1));
  h.add(C * 4 + 16);
  h.add(C * 4 + 16);
  h.add((nbk + 1) * 4);
  h.add((Mm + 1) * 4);
  h.add(nmt * 4 + 16);
  h.add(C * 8 * 4 + 16);
  h.add((nbk + 1) * 8);
  h.add((Mm + 1) * 8);
  h.add((nmt + 1) * 8 + 256);
  h.add(scan_b(nmt + 1));
  h.add(ncm * 4 + 256);
  h.add((ncm + 1) * 8 + 256);
  h.add(scan_b(ncm + 1));
  h.add(nmov * 4 + 16);
  h.add(nml * 4 + 16);
  h.add((nbk + 1) * 4);
  h.add(seg_b(nbk, nmov));
  h.add((Mm + 1) * 4);
  h.add(seg_b(Mm, nml));
  h.add(NB * 8 + 16);
  h.add(NB * 8 + 16);
  h.add(NB * 4 + 256);
  {
    double tot = 0.0, prev = nmov;
    for (int k = 0; k < 8; ++k) {
      prev = std::floor(prev / 64) + NB + 2;
      tot += prev;
    }
    h.add(tot * 8 + 256);
  }
  const double hm_cap = 2 * nml + kPad;
  const double nchunk_h = N + (npre + 2 * nml) / kChunk + 1;
  h.add(N * 4 + 16);
  h.add(N * 8 + 16);
  h.add(N * 8 + 16);
  h.add(N + 256);
  h.add((N + 1) * 8 + 256);
  h.add((N + 1) * 8 + 256);
  h.add((N + 1) * 4 + 256);
  h.add((N + 1 + kRpPad) * 4);
  h.add(hm_cap * 4);
  h.add(hm_cap * sw);
  for (double b : {4.0, 8.0, 8.0, 4.0, 4.0}) h.add(N * b + 16);
  h.add((N + 1) * 8);
  h.add(N * 4 + 16);
  h.add((N + 1) * 4);
  h.add((N + 1) * 4 + 256);
  h.add(nchunk_h * 4 + 16);
  h.add(N * 8 + 16);
  h.add(N * 8 + 16);
  h.add(N * 4 + 16);
  h.add(N * 8 + 16);
  h.add(64);
  h.add((nchunk_h + 1) * 48);
  h.add(C * 8 + 16);                 // macro entry offsets
  h.add(C * W * sw + 64);            // window blocks, cell order
  h.add((std::floor(nmov / kBinChunk) + NB + 1) * kBinChunk * W * sw + 64);  // chunks' window blocks
  h.add(C * 4 + 16);
  h.add((NB + 1) * 4 + 256);
  h.add((NB + 1) * 4 + 256);
  const double nbc = std::floor(nmov / kBinChunk) + NB + 1;
  h.add(nbc * 4 + 256);
  h.add(nbc * W * 16 + 256);
  h.add(nbc * W * 16 + 256);
  h.add((nchunk_h + 1) * 2 * 8 + 256);
  return st.b + h.b + 4096.0;
}

// Taken at the end of the static build so that the filters find them in the
// static part of the workspace (a hint build restarts above them).
pl_status take_filter_buffers(pl_graph *g) {
  const size_t N = (size_t)g->N;
  Buf *b8[] = {&g->xa, &g->xb, &g->xc, &g->g0, &g->ua, &g->ub};
  for (Buf *b : b8) {
    cudaError_t e = ensure(*b, N * 8 + 64);
    if (e != cudaSuccess) return cuda_fail(e, "filter buffers");
  }
  cudaError_t e = ensure(g->acc, N * 16 + 16);
  if (e == cudaSuccess) e = ensure(g->gsc, N * 24 + 64);
  if (e == cudaSuccess) e = ensure(g->q4a, N * 16 + 64);
  if (e == cudaSuccess) e = ensure(g->q4b, N * 16 + 64);
  if (e == cudaSuccess) e = ensure(g->lscr, (N / 1024 + 2) * 4 + 64);
  if (e != cudaSuccess) return cuda_fail(e, "filter buffers");
  return PL_OK;
}

}  // namespace pl

extern "C" size_t pl_workspace_size(const pl_netlist *nl, const pl_params *p) {
  if (!nl || !p || nl->num_cells < 0 || nl->num_nets < 0 || nl->num_pins < 0) return 0;
  const double b = pl::workspace_bound(nl, p);
  if (!(b < 1.8e19)) return (size_t)-1;
  return (size_t)b;
}
