/* FP64 CPU oracle of the area-hint refinement initializer (arXiv 2511.10073).
 *
 * TEST INFRASTRUCTURE ONLY: the plain statement that the CUDA library is
 * checked against.  Sequential loops, ascending index order everywhere, FP64
 * arithmetic, compiled without FMA contraction.  Shares no code with the CUDA
 * library.  Each function names the part of the paper it follows; readings
 * taken where the paper is silent are stated at the function.
 *
 * Node numbering (a reading; the paper fixes none):
 *   [cells in input order][macro pin nodes, global pin order]
 *   [star nodes, net order][macro virtual nodes, macro order]
 *   [bin virtual nodes, row-major with x fastest]
 */
#include "orc.h"

/* Built twice: without OpenMP (liborc.so, the single-threaded oracle the
 * tests compare with) and with it (liborc_omp.so, timed as the all-cores CPU
 * baseline).  OMP_FOR marks only loops whose iterations write disjoint outputs
 * with the same arithmetic per element, so both builds give the same bits. */
#ifdef _OPENMP
#define OMP_FOR _Pragma("omp parallel for schedule(static)")
#define OMP_FOR_DYN _Pragma("omp parallel for schedule(dynamic, 64)")
#else
#define OMP_FOR
#define OMP_FOR_DYN
#endif

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define LATTICE 360360LL /* lcm(1..15): clique weights 1/(p-1) are integers on it */

struct orc_graph {
  int32_t C, M;
  int64_t P;
  int32_t Pm, S, Mm, NB, nbx, nby, hx, hy;
  int64_t Nst, N;
  double xl, yl, xh, yh, wb, hb, abin;
  int wdtype;
  /* copies of the netlist fields the later steps need */
  float *cw, *ch;
  uint8_t *ckind;
  /* per node */
  uint8_t *nkind; /* 0 movable cell, 1 star node (movable point), 2 fixed */
  double *fx, *fy, *hw, *hh;
  int32_t *pin_node;
  int32_t *macro_cell; /* [Mm] */
  int32_t *star_net;   /* [S] */
  int64_t *nd_ptr;     /* [M+1] distinct nodes of each net */
  int32_t *nd;
  /* static graph, canonical CSR */
  int64_t *srp;
  int32_t *scol;
  double *sw_exact, *sw_store, *sdeg;
  double *base_w; /* [C] */
  double *amac;   /* [NB] macro area inside each bin */
  /* current augmented graph */
  int have_hints;
  int64_t *rp;
  int32_t *col;
  double *w, *deg;
  double lam_up;
  double *Db, *Cb, *phi;
  int32_t *cell_bin;
};

/* ---------------------------------------------------------------- helpers */

static void *xcalloc(size_t n, size_t sz) {
  void *p = calloc(n ? n : 1, sz);
  if (!p) abort();
  return p;
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

typedef struct { int32_t col; int64_t lat; } ent_t;
static int cmp_ent(const void *a, const void *b) {
  const ent_t *x = (const ent_t *)a, *y = (const ent_t *)b;
  if (x->col != y->col) return (x->col > y->col) - (x->col < y->col);
  return (x->lat > y->lat) - (x->lat < y->lat);
}

/* exp(x) by Cody & Waite argument reduction (x = n ln2 + r, |r| <= ln2/2, with
 * ln2 split into a 32-significant-bit head and a tail so that n*head is exact)
 * followed by the degree-13 Taylor polynomial of e^r in Horner form and a
 * scaling by 2^n.  Written out here so that the CPU and GPU sides evaluate one
 * documented sequence of IEEE double operations; its accuracy is pinned against
 * the C library's exp in the tests. */
double orc_exp(double x) {
  static const double inv_ln2 = 0x1.71547652b82fep+0;
  static const double ln2_hi = 0x1.62e42fee00000p-1;
  static const double ln2_lo = 0x1.a39ef35793c76p-33;
  if (x != x) return x;
  if (x > 709.78) return INFINITY;
  if (x < -745.2) return 0.0;
  double n = floor(x * inv_ln2 + 0.5);
  double r = (x - n * ln2_hi) - n * ln2_lo;
  /* 1/j! for j = 13 .. 0 */
  static const double c[14] = {
      0x1.6124613a86d09p-33, 0x1.1eed8eff8d898p-29, 0x1.ae64567f544e4p-26,
      0x1.27e4fb7789f5cp-22, 0x1.71de3a556c734p-19, 0x1.a01a01a01a01ap-16,
      0x1.a01a01a01a01ap-13, 0x1.6c16c16c16c17p-10, 0x1.1111111111111p-7,
      0x1.5555555555555p-5,  0x1.5555555555555p-3,  0x1.0000000000000p-1,
      1.0, 1.0};
  double p = c[0];
  for (int j = 1; j < 14; ++j) p = p * r + c[j];
  int ni = (int)n;
  if (ni < -1020) return ldexp(ldexp(p, ni + 1020), -1020);
  if (ni > 1023) return ldexp(ldexp(p, 1023), ni - 1023);
  return ldexp(p, ni);
}

/* splitmix64 (Steele, Lea & Flood 2014) evaluated at counter ctr of stream
 * `seed`, top 53 bits mapped to [0, 1). */
double orc_u01(uint64_t seed, uint64_t ctr) {
  uint64_t z = seed + (ctr + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * 0x1.0p-53;
}

/* Value an FP64 edge weight takes once stored: unchanged, IEEE FP32 round to
 * nearest even, or bfloat16 (8 significant bits, FP32 exponent range) round to
 * nearest even directly from FP64. */
/* The sum of n positive doubles, each at least 2^-15, rounded once to the
   nearest double (ties to even).  Every such value is an integer multiple of
   2^-67, so the sum is taken exactly in 128-bit fixed point and converted
   once.  baseWeight is the mean of a cell's weights: this sum over n. */
static double exact_sum(const double *w, int64_t n) {
  unsigned __int128 acc = 0;
  for (int64_t k = 0; k < n; ++k) {
    int e;
    double m = frexp(w[k], &e); /* w = m 2^e, 0.5 <= m < 1 */
    if (!(w[k] > 0.0) || e < -14) {
      fprintf(stderr, "orc: weight %g outside the exact-sum range\n", w[k]);
      abort();
    }
    uint64_t M = (uint64_t)ldexp(m, 53); /* w = M 2^(e - 53) */
    acc += (unsigned __int128)M << (e + 14); /* w 2^67 */
  }
  /* round to 53 bits: the top 64 bits with a sticky bit, then one correctly
     rounded conversion */
  int sh = 0;
  while ((acc >> sh) >> 64) ++sh;
  uint64_t top = (uint64_t)(acc >> sh);
  if (sh && (acc & ((((unsigned __int128)1) << sh) - 1))) top |= 1;
  return ldexp((double)top, sh - 67);
}

double orc_store(double w, int dtype) {
  if (dtype == ORC_W_FP32) return (double)(float)w;
  if (dtype == ORC_W_BF16) {
    if (w == 0.0 || w != w || isinf(w)) return w;
    int e;
    frexp(w, &e);                 /* |w| in [2^(e-1), 2^e) */
    int q = e - 8;                /* quantum of an 8-bit significand */
    if (q < -133) q = -133;       /* bf16 subnormal quantum 2^-133 */
    double r = ldexp(nearbyint(ldexp(w, -q)), q);
    if (fabs(r) > 0x1.fep+127) r = copysign(INFINITY, w);
    return r;
  }
  return w;
}

static inline double clampd(double v, double lo, double hi) { return fmin(fmax(v, lo), hi); }

/* Integer decisions taken from coordinates (which bin holds a cell centre,
 * whether a cell overlaps a macro) are made in FP32, the precision the
 * coordinates are stored in, with one stated sequence of IEEE single
 * operations; the coordinate is first rounded to FP32.  Bin of a point:
 * clamp(floor((x - xl) * (nb / (xh - xl))), 0, nb - 1) with xl and the scale
 * each rounded to FP32. */
static int32_t bin_of(double x, double xl, double xh, int32_t nb) {
  float xf = (float)x;
  float xlf = (float)xl;
  float sc = (float)((double)nb / (xh - xl));
  float t = (xf - xlf) * sc;
  double f = floor((double)t);
  if (!(f >= 0.0)) return 0;
  if (f > (double)(nb - 1)) return nb - 1;
  return (int32_t)f;
}

/* Positive-area overlap of a cell (centre x, y; size w, h) with a macro
 * (centre xm, ym; size wm, hm): |x - xm| < (w + wm)/2 on both axes, in FP32. */
static int overlaps(double x, double y, float w, float h, float xm, float ym, float wm, float hm) {
  float dx = fabsf((float)x - xm), dy = fabsf((float)y - ym);
  return dx < 0.5f * (w + wm) && dy < 0.5f * (h + hm);
}

/* ------------------------------------------------------ A1: static graph */

/* Instance graph of the netlist hypergraph with macro pin expansion
 * (Sec. V "Macro pin expansion"; the graph G=(V,E) of Sec. IV).
 * Readings (the paper gives no net model or weights):
 *  - pins on macros become one fixed node each, at macro centre + pin offset;
 *    other pins map to their cell's node; repeated nodes of a net merge;
 *  - a net with p >= 2 distinct nodes and p <= clique_max is a clique with
 *    weight 1/(p-1) per pair; a larger net becomes a star: one movable star
 *    node joined to each of its nodes with weight p/(p-1);
 *  - parallel edges from different nets add; clique weights are summed
 *    exactly as integer multiples of 1/360360 and divided once;
 *  - baseWeight_i (Sec. V, macro edge weight) is the mean of cell i's static
 *    FP64 row weights, summed in column order. */
orc_graph *orc_create(const orc_netlist *nl, const orc_params *pr, int *err) {
  *err = ORC_ERR_INVALID;
  if (!nl || !pr || nl->num_cells < 0 || nl->num_nets < 0) return NULL;
  if (pr->clique_max < 2 || pr->clique_max > 16 || pr->nbx < 1 || pr->nby < 1) return NULL;
  if (!(nl->xh > nl->xl) || !(nl->yh > nl->yl)) return NULL;
  const int32_t C = nl->num_cells, M = nl->num_nets;
  const int64_t P = nl->num_pins;
  if (nl->net_ptr[0] != 0 || nl->net_ptr[M] != P) return NULL;
  for (int32_t e = 0; e < M; ++e)
    if (nl->net_ptr[e + 1] < nl->net_ptr[e]) return NULL;
  for (int64_t p = 0; p < P; ++p)
    if (nl->pin_cell[p] < 0 || nl->pin_cell[p] >= C) return NULL;
  for (int32_t c = 0; c < C; ++c) {
    if (nl->cell_kind[c] > 2) return NULL;
    if (nl->cell_kind[c] == 1 && !(nl->cell_w[c] > 0.0f && nl->cell_h[c] > 0.0f)) return NULL;
  }

  orc_graph *g = (orc_graph *)xcalloc(1, sizeof(orc_graph));
  g->C = C; g->M = M; g->P = P;
  g->xl = nl->xl; g->yl = nl->yl; g->xh = nl->xh; g->yh = nl->yh;
  g->wdtype = pr->wdtype;
  g->nbx = pr->nbx; g->nby = pr->nby;
  g->cw = (float *)xcalloc(C, sizeof(float));
  g->ch = (float *)xcalloc(C, sizeof(float));
  g->ckind = (uint8_t *)xcalloc(C, 1);
  memcpy(g->cw, nl->cell_w, sizeof(float) * C);
  memcpy(g->ch, nl->cell_h, sizeof(float) * C);
  memcpy(g->ckind, nl->cell_kind, C);

  /* macro pin nodes, in global pin order */
  g->pin_node = (int32_t *)xcalloc(P, sizeof(int32_t));
  int32_t Pm = 0;
  for (int64_t p = 0; p < P; ++p) {
    int32_t c = nl->pin_cell[p];
    g->pin_node[p] = (nl->cell_kind[c] == 1) ? C + Pm++ : c;
  }
  g->Pm = Pm;

  /* distinct nodes of every net, ascending */
  g->nd_ptr = (int64_t *)xcalloc(M + 1, sizeof(int64_t));
  g->nd = (int32_t *)xcalloc(P, sizeof(int32_t));
  int32_t *tmp = (int32_t *)xcalloc(P, sizeof(int32_t));
  int64_t w = 0;
  for (int32_t e = 0; e < M; ++e) {
    int64_t b = nl->net_ptr[e], n = nl->net_ptr[e + 1] - b;
    for (int64_t k = 0; k < n; ++k) tmp[k] = g->pin_node[b + k];
    qsort(tmp, n, sizeof(int32_t), cmp_i32);
    g->nd_ptr[e] = w;
    for (int64_t k = 0; k < n; ++k)
      if (k == 0 || tmp[k] != tmp[k - 1]) g->nd[w++] = tmp[k];
  }
  g->nd_ptr[M] = w;
  free(tmp);

  /* star nodes, in net order */
  int32_t S = 0;
  for (int32_t e = 0; e < M; ++e)
    if (g->nd_ptr[e + 1] - g->nd_ptr[e] > pr->clique_max) ++S;
  g->S = S;
  g->star_net = (int32_t *)xcalloc(S, sizeof(int32_t));
  g->Nst = (int64_t)C + Pm + S;

  /* edge list: count per row, place, sort each row, merge equal columns */
  int64_t *cnt = (int64_t *)xcalloc(g->Nst + 1, sizeof(int64_t));
  S = 0;
  for (int32_t e = 0; e < M; ++e) {
    int64_t b = g->nd_ptr[e], p = g->nd_ptr[e + 1] - b;
    if (p < 2) continue;
    if (p <= pr->clique_max) {
      for (int64_t k = 0; k < p; ++k) cnt[g->nd[b + k]] += p - 1;
    } else {
      int64_t s = (int64_t)C + Pm + S;
      g->star_net[S++] = e;
      for (int64_t k = 0; k < p; ++k) cnt[g->nd[b + k]] += 1;
      cnt[s] += p;
    }
  }
  int64_t *off = (int64_t *)xcalloc(g->Nst + 1, sizeof(int64_t));
  for (int64_t i = 0; i < g->Nst; ++i) off[i + 1] = off[i] + cnt[i];
  ent_t *ent = (ent_t *)xcalloc(off[g->Nst], sizeof(ent_t));
  int64_t *cur = (int64_t *)xcalloc(g->Nst + 1, sizeof(int64_t));
  memcpy(cur, off, sizeof(int64_t) * (g->Nst + 1));
  S = 0;
  for (int32_t e = 0; e < M; ++e) {
    int64_t b = g->nd_ptr[e], p = g->nd_ptr[e + 1] - b;
    if (p < 2) continue;
    if (p <= pr->clique_max) {
      int64_t lat = LATTICE / (p - 1);
      for (int64_t a = 0; a < p; ++a)
        for (int64_t c2 = 0; c2 < p; ++c2) {
          if (a == c2) continue;
          ent_t t = {g->nd[b + c2], lat};
          ent[cur[g->nd[b + a]]++] = t;
        }
    } else {
      int32_t s = C + Pm + S++;
      for (int64_t a = 0; a < p; ++a) {
        ent_t t1 = {s, -p};
        ent[cur[g->nd[b + a]]++] = t1;
        ent_t t2 = {g->nd[b + a], -p};
        ent[cur[s]++] = t2;
      }
    }
  }
  free(cur);
  g->srp = (int64_t *)xcalloc(g->Nst + 1, sizeof(int64_t));
  int64_t nnz = 0;
  for (int64_t i = 0; i < g->Nst; ++i) {
    ent_t *r = ent + off[i];
    int64_t n = off[i + 1] - off[i];
    qsort(r, n, sizeof(ent_t), cmp_ent);
    int64_t m = 0;
    for (int64_t k = 0; k < n; ++k) {
      if (m > 0 && r[m - 1].col == r[k].col) {
        /* a star edge is unique to its net and never meets another entry */
        if (r[k].lat < 0 || r[m - 1].lat < 0) abort();
        r[m - 1].lat += r[k].lat;
      } else {
        r[m++] = r[k];
      }
    }
    g->srp[i] = nnz;
    nnz += m;
    cnt[i] = m;
  }
  g->srp[g->Nst] = nnz;
  g->scol = (int32_t *)xcalloc(nnz, sizeof(int32_t));
  g->sw_exact = (double *)xcalloc(nnz, sizeof(double));
  g->sw_store = (double *)xcalloc(nnz, sizeof(double));
  g->sdeg = (double *)xcalloc(g->Nst, sizeof(double));
  for (int64_t i = 0; i < g->Nst; ++i) {
    for (int64_t k = 0; k < cnt[i]; ++k) {
      ent_t t = ent[off[i] + k];
      int64_t d = g->srp[i] + k;
      g->scol[d] = t.col;
      double we = (t.lat > 0) ? (double)t.lat / (double)LATTICE
                              : (double)(-t.lat) / (double)(-t.lat - 1);
      g->sw_exact[d] = we;
      g->sw_store[d] = orc_store(we, pr->wdtype);
    }
    double sd = 0.0;
    for (int64_t k = g->srp[i]; k < g->srp[i + 1]; ++k) sd += g->sw_store[k];
    g->sdeg[i] = sd;
  }
  free(ent); free(off); free(cnt);

  g->base_w = (double *)xcalloc(C, sizeof(double));
  for (int32_t i = 0; i < C; ++i) {
    int64_t n = g->srp[i + 1] - g->srp[i];
    if (n == 0) continue;
    g->base_w[i] = exact_sum(g->sw_exact + g->srp[i], n) / (double)n;
  }

  /* macros and virtual nodes */
  int32_t Mm = 0;
  for (int32_t c = 0; c < C; ++c) Mm += nl->cell_kind[c] == 1;
  g->Mm = Mm;
  g->macro_cell = (int32_t *)xcalloc(Mm, sizeof(int32_t));
  Mm = 0;
  for (int32_t c = 0; c < C; ++c)
    if (nl->cell_kind[c] == 1) g->macro_cell[Mm++] = c;
  g->NB = pr->nbx * pr->nby;
  g->N = g->Nst + g->Mm + g->NB;
  g->wb = (g->xh - g->xl) / (double)g->nbx;
  g->hb = (g->yh - g->yl) / (double)g->nby;
  g->abin = g->wb * g->hb;
  int32_t nx = (int32_t)floor(pr->det_ratio * (double)g->nbx);
  int32_t ny = (int32_t)floor(pr->det_ratio * (double)g->nby);
  if (nx < 1) nx = 1;
  if (ny < 1) ny = 1;
  g->hx = (nx - 1) / 2;
  g->hy = (ny - 1) / 2;

  /* node kinds, fixed positions, half sizes */
  const int64_t N = g->N;
  g->nkind = (uint8_t *)xcalloc(N, 1);
  g->fx = (double *)xcalloc(N, sizeof(double));
  g->fy = (double *)xcalloc(N, sizeof(double));
  g->hw = (double *)xcalloc(N, sizeof(double));
  g->hh = (double *)xcalloc(N, sizeof(double));
  for (int32_t c = 0; c < C; ++c) {
    if (nl->cell_kind[c] == 0) {
      g->nkind[c] = 0;
      g->hw[c] = (double)nl->cell_w[c] * 0.5;
      g->hh[c] = (double)nl->cell_h[c] * 0.5;
    } else {
      g->nkind[c] = 2;
      g->fx[c] = nl->fixed_x[c];
      g->fy[c] = nl->fixed_y[c];
    }
  }
  for (int64_t p = 0; p < P; ++p) {
    int32_t v = g->pin_node[p], c = nl->pin_cell[p];
    if (v < C) continue;
    g->nkind[v] = 2;
    g->fx[v] = (double)nl->fixed_x[c] + (nl->pin_dx ? (double)nl->pin_dx[p] : 0.0);
    g->fy[v] = (double)nl->fixed_y[c] + (nl->pin_dy ? (double)nl->pin_dy[p] : 0.0);
  }
  for (int32_t s = 0; s < g->S; ++s) g->nkind[C + Pm + s] = 1;
  for (int32_t m = 0; m < g->Mm; ++m) {
    int64_t v = g->Nst + m;
    g->nkind[v] = 2;
    g->fx[v] = nl->fixed_x[g->macro_cell[m]];
    g->fy[v] = nl->fixed_y[g->macro_cell[m]];
  }
  for (int32_t by = 0; by < g->nby; ++by)
    for (int32_t bx = 0; bx < g->nbx; ++bx) {
      int64_t v = g->Nst + g->Mm + (int64_t)by * g->nbx + bx;
      g->nkind[v] = 2;
      g->fx[v] = g->xl + ((double)bx + 0.5) * g->wb;
      g->fy[v] = g->yl + ((double)by + 0.5) * g->hb;
    }

  /* macro area inside every bin (fixed for the whole run), macro order */
  g->amac = (double *)xcalloc(g->NB, sizeof(double));
  for (int32_t by = 0; by < g->nby; ++by)
    for (int32_t bx = 0; bx < g->nbx; ++bx) {
      double bxl = g->xl + (double)bx * g->wb, bxh = g->xl + (double)(bx + 1) * g->wb;
      double byl = g->yl + (double)by * g->hb, byh = g->yl + (double)(by + 1) * g->hb;
      double a = 0.0;
      for (int32_t m = 0; m < g->Mm; ++m) {
        int32_t c = g->macro_cell[m];
        double hwm = (double)nl->cell_w[c] * 0.5, hhm = (double)nl->cell_h[c] * 0.5;
        double ox = fmin(bxh, (double)nl->fixed_x[c] + hwm) - fmax(bxl, (double)nl->fixed_x[c] - hwm);
        double oy = fmin(byh, (double)nl->fixed_y[c] + hhm) - fmax(byl, (double)nl->fixed_y[c] - hhm);
        if (ox > 0.0 && oy > 0.0) a += ox * oy;
      }
      g->amac[(int64_t)by * g->nbx + bx] = a;
    }
  g->Db = (double *)xcalloc(g->NB, sizeof(double));
  g->Cb = (double *)xcalloc(g->NB, sizeof(double));
  g->phi = (double *)xcalloc(g->NB, sizeof(double));
  g->cell_bin = (int32_t *)xcalloc(C, sizeof(int32_t));
  *err = ORC_OK;
  return g;
}

void orc_destroy(orc_graph *g) {
  if (!g) return;
  void *ps[] = {g->cw, g->ch, g->ckind, g->nkind, g->fx, g->fy, g->hw, g->hh, g->pin_node,
                g->macro_cell, g->star_net, g->nd_ptr, g->nd, g->srp, g->scol, g->sw_exact,
                g->sw_store, g->sdeg, g->base_w, g->amac, g->rp, g->col, g->w, g->deg,
                g->Db, g->Cb, g->phi, g->cell_bin};
  for (size_t k = 0; k < sizeof(ps) / sizeof(ps[0]); ++k) free(ps[k]);
  free(g);
}

void orc_sizes(const orc_graph *g, int64_t out[16]) {
  memset(out, 0, sizeof(int64_t) * 16);
  out[0] = g->C; out[1] = g->Pm; out[2] = g->S; out[3] = g->Mm; out[4] = g->NB;
  out[5] = g->Nst; out[6] = g->N; out[7] = g->srp[g->Nst];
  out[8] = g->have_hints ? g->rp[g->N] : 0;
  out[9] = g->hx; out[10] = g->hy; out[11] = g->M; out[12] = g->P;
}

void orc_static_export(const orc_graph *g, int64_t *rp, int32_t *col, double *w_exact,
                       double *w_store, double *base_w) {
  int64_t nnz = g->srp[g->Nst];
  memcpy(rp, g->srp, sizeof(int64_t) * (g->Nst + 1));
  memcpy(col, g->scol, sizeof(int32_t) * nnz);
  memcpy(w_exact, g->sw_exact, sizeof(double) * nnz);
  memcpy(w_store, g->sw_store, sizeof(double) * nnz);
  memcpy(base_w, g->base_w, sizeof(double) * g->C);
}

void orc_nodes_export(const orc_graph *g, uint8_t *nkind, double *fx, double *fy, double *hw,
                      double *hh, int32_t *pin_node) {
  memcpy(nkind, g->nkind, g->N);
  memcpy(fx, g->fx, sizeof(double) * g->N);
  memcpy(fy, g->fy, sizeof(double) * g->N);
  memcpy(hw, g->hw, sizeof(double) * g->N);
  memcpy(hh, g->hh, sizeof(double) * g->N);
  memcpy(pin_node, g->pin_node, sizeof(int32_t) * g->P);
}

/* ------------------------------------- A2 + A3: area hints, signed Laplacian */

/* Sum of a[0..n) in a fixed blocked order: n <= 64 values are added left to
 * right; longer sequences are cut into consecutive blocks of 64, each block
 * is added left to right, and the sequence of block sums is summed the same
 * way (recursively).  Used for bin densities. */
static double blocked_sum(const double *a, int64_t n) {
  if (n <= 64) {
    double s = 0.0;
    for (int64_t k = 0; k < n; ++k) s += a[k];
    return s;
  }
  int64_t nb = (n + 63) / 64;
  double *t = (double *)xcalloc(nb, sizeof(double));
  for (int64_t j = 0; j < nb; ++j) {
    double s = 0.0;
    for (int64_t k = 64 * j; k < n && k < 64 * j + 64; ++k) s += a[k];
    t[j] = s;
  }
  double r = blocked_sum(t, nb);
  free(t);
  return r;
}

typedef struct { int32_t cell, m; } mpair_t;
static int cmp_pair(const void *a, const void *b) {
  const mpair_t *x = (const mpair_t *)a, *y = (const mpair_t *)b;
  if (x->cell != y->cell) return (x->cell > y->cell) - (x->cell < y->cell);
  return (x->m > y->m) - (x->m < y->m);
}

/* Every (movable cell with baseWeight > 0, macro) pair whose rectangles
 * overlap with positive area (the FP32 test of overlaps()).  Cells are
 * bucketed by centre on a uniform grid only to skip pairs that cannot
 * overlap.  Sorted by (cell, macro). */
static mpair_t *macro_pairs(const orc_graph *g, const double *gx, const double *gy,
                            int64_t *npairs) {
  const int32_t C = g->C;
  double wmax = 0.0, hmax = 0.0, msz = 1.0;
  for (int32_t i = 0; i < C; ++i)
    if (g->ckind[i] == 0) { wmax = fmax(wmax, g->cw[i]); hmax = fmax(hmax, g->ch[i]); }
  for (int32_t m = 0; m < g->Mm; ++m) {
    int32_t c = g->macro_cell[m];
    msz = fmax(msz, fmax((double)g->cw[c], (double)g->ch[c]));
  }
  double G = msz;
  int32_t gnx = (int32_t)fmin(4096.0, fmax(1.0, ceil((g->xh - g->xl) / G)));
  int32_t gny = (int32_t)fmin(4096.0, fmax(1.0, ceil((g->yh - g->yl) / G)));
  int64_t nbk = (int64_t)gnx * gny;
  int64_t *bptr = (int64_t *)xcalloc(nbk + 1, sizeof(int64_t));
  int32_t *bcell = (int32_t *)xcalloc(C, sizeof(int32_t));
  int32_t *bk = (int32_t *)xcalloc(C, sizeof(int32_t));
  for (int32_t i = 0; i < C; ++i) {
    bk[i] = -1;
    if (g->ckind[i] != 0 || !(g->base_w[i] > 0.0)) continue;
    int32_t kx = (int32_t)clampd(floor((gx[i] - g->xl) / G), 0.0, gnx - 1.0);
    int32_t ky = (int32_t)clampd(floor((gy[i] - g->yl) / G), 0.0, gny - 1.0);
    bk[i] = ky * gnx + kx;
    bptr[bk[i] + 1]++;
  }
  for (int64_t k = 0; k < nbk; ++k) bptr[k + 1] += bptr[k];
  int64_t *fill = (int64_t *)xcalloc(nbk, sizeof(int64_t));
  for (int32_t i = 0; i < C; ++i)
    if (bk[i] >= 0) bcell[bptr[bk[i]] + fill[bk[i]]++] = i;
  int64_t cap = 1024, n = 0;
  mpair_t *out = (mpair_t *)xcalloc(cap, sizeof(mpair_t));
  for (int32_t m = 0; m < g->Mm; ++m) {
    int32_t c = g->macro_cell[m];
    double xm = g->fx[g->Nst + m], ym = g->fy[g->Nst + m];
    double ex = 0.5 * ((double)g->cw[c] + wmax), ey = 0.5 * ((double)g->ch[c] + hmax);
    /* one extra bucket each side covers the FP32 rounding of the test */
    int32_t kx0 = (int32_t)clampd(floor((xm - ex - g->xl) / G) - 1.0, 0.0, gnx - 1.0);
    int32_t kx1 = (int32_t)clampd(floor((xm + ex - g->xl) / G) + 1.0, 0.0, gnx - 1.0);
    int32_t ky0 = (int32_t)clampd(floor((ym - ey - g->yl) / G) - 1.0, 0.0, gny - 1.0);
    int32_t ky1 = (int32_t)clampd(floor((ym + ey - g->yl) / G) + 1.0, 0.0, gny - 1.0);
    for (int32_t ky = ky0; ky <= ky1; ++ky)
      for (int32_t kx = kx0; kx <= kx1; ++kx) {
        int64_t k = (int64_t)ky * gnx + kx;
        for (int64_t t = bptr[k]; t < bptr[k + 1]; ++t) {
          int32_t i = bcell[t];
          if (!overlaps(gx[i], gy[i], g->cw[i], g->ch[i], (float)xm, (float)ym, g->cw[c],
                        g->ch[c]))
            continue;
          if (n == cap) {
            cap *= 2;
            out = (mpair_t *)realloc(out, sizeof(mpair_t) * cap);
            if (!out) abort();
          }
          out[n].cell = i;
          out[n].m = m;
          ++n;
        }
      }
  }
  qsort(out, n, sizeof(mpair_t), cmp_pair);
  free(bptr); free(bcell); free(bk); free(fill);
  *npairs = n;
  return out;
}

/* Augmented signed graph from the current placement (Sec. V: macro virtual
 * node with repulsive edges, bin virtual node with density-aware signed edges;
 * BuildLap of Algorithm 1) and its Gershgorin bound lambda_up (Eq. of H_r).
 * Readings:
 *  - only movable cells with baseWeight > 0 get hint edges;
 *  - "overlaps macro m": the cell rectangle (centre, w, h) and the macro
 *    rectangle intersect with positive area (decided in FP32, overlaps());
 *  - D_b = (FP64 sum of w*h of the movable cells whose centre lies in b) / bin
 *    area; the cells are taken with baseWeight > 0 first, then the others,
 *    each group in ascending id, and added in the blocked order of
 *    blocked_sum(); the bin of a centre is decided in FP32 (bin_of());
 *  - capacity of b = C * (A_bin - macro area in b) / A_bin;
 *  - phi_b = 2 / (1 + exp(-mu (D_b - C_b))) - 1  (= 2 sigmoid(.) - 1);
 *  - cell i is in N(b) when its centre bin lies in the n_x x n_y window of b,
 *    n = max(1, floor(detection_ratio * numBin)), half width floor((n-1)/2);
 *  - weights are evaluated in the order  -((e^{-maxRatio} * phi_b) * bw_i)
 *    and rounded once to the storage type;
 *  - each row is its static part followed by macro columns (ascending) then
 *    bin columns (ascending); virtual rows list cells in ascending id;
 *  - L = D - A with signed D_ii = sum_j w_ij over stored weights (row order);
 *    lambda_up = max_i (D_ii + sum_j |w_ij|) (Gershgorin). */
int orc_build_hints(orc_graph *g, const orc_params *pr, const double *gx, const double *gy) {
  const int32_t C = g->C;
  const int64_t N = g->N, Nst = g->Nst;
  for (int32_t i = 0; i < C; ++i)
    if (g->ckind[i] == 0 && !(isfinite(gx[i]) && isfinite(gy[i]))) return ORC_ERR_NONFINITE;

  /* bin of each movable cell; each bin's cell sequence: its cells with
   * baseWeight > 0 in ascending id, then its other movable cells ascending */
  int64_t *bcnt = (int64_t *)xcalloc(2 * (int64_t)g->NB + 1, sizeof(int64_t));
  for (int32_t i = 0; i < C; ++i) {
    g->cell_bin[i] = -1;
    if (g->ckind[i] != 0) continue;
    int32_t bx = bin_of(gx[i], g->xl, g->xh, g->nbx);
    int32_t by = bin_of(gy[i], g->yl, g->yh, g->nby);
    int32_t b = by * g->nbx + bx;
    g->cell_bin[i] = b;
    bcnt[2 * (int64_t)b + (g->base_w[i] > 0.0 ? 0 : 1) + 1]++;
  }
  for (int64_t k = 0; k < 2 * (int64_t)g->NB; ++k) bcnt[k + 1] += bcnt[k];
  double *area = (double *)xcalloc(bcnt[2 * (int64_t)g->NB], sizeof(double));
  int64_t *fillp = (int64_t *)xcalloc(2 * (int64_t)g->NB, sizeof(int64_t));
  for (int32_t i = 0; i < C; ++i) {
    if (g->ckind[i] != 0) continue;
    int64_t k = 2 * (int64_t)g->cell_bin[i] + (g->base_w[i] > 0.0 ? 0 : 1);
    area[bcnt[k] + fillp[k]++] = (double)g->cw[i] * (double)g->ch[i];
  }
  OMP_FOR_DYN
  for (int32_t b = 0; b < g->NB; ++b) {
    int64_t a0 = bcnt[2 * (int64_t)b], a1 = bcnt[2 * (int64_t)b + 2];
    g->Db[b] = blocked_sum(area + a0, a1 - a0) / g->abin;
    g->Cb[b] = (pr->capacity * (g->abin - g->amac[b])) / g->abin;
    double t = pr->mu * (g->Db[b] - g->Cb[b]);
    g->phi[b] = 2.0 / (1.0 + orc_exp(-t)) - 1.0;
  }
  free(bcnt); free(area); free(fillp);

  /* (cell, macro) overlap pairs in ascending (cell, macro) order */
  int64_t npairs = 0;
  mpair_t *pairs = macro_pairs(g, gx, gy, &npairs);

  /* per-row hint counts */
  int64_t *hcnt = (int64_t *)xcalloc(N, sizeof(int64_t));
  for (int64_t q = 0; q < npairs; ++q) {
    hcnt[pairs[q].cell]++;
    hcnt[Nst + pairs[q].m]++;
  }
  for (int32_t i = 0; i < C; ++i) {
    if (g->ckind[i] != 0 || !(g->base_w[i] > 0.0)) continue;
    int32_t b = g->cell_bin[i], bx = b % g->nbx, by = b / g->nbx;
    for (int32_t yy = by - g->hy; yy <= by + g->hy; ++yy)
      for (int32_t xx = bx - g->hx; xx <= bx + g->hx; ++xx) {
        if (xx < 0 || yy < 0 || xx >= g->nbx || yy >= g->nby) continue;
        hcnt[i]++;
        hcnt[Nst + g->Mm + (int64_t)yy * g->nbx + xx]++;
      }
  }

  free(g->rp); free(g->col); free(g->w); free(g->deg);
  g->rp = (int64_t *)xcalloc(N + 1, sizeof(int64_t));
  for (int64_t v = 0; v < N; ++v) {
    int64_t sl = (v < Nst) ? g->srp[v + 1] - g->srp[v] : 0;
    g->rp[v + 1] = g->rp[v] + sl + hcnt[v];
  }
  int64_t nnz = g->rp[N];
  g->col = (int32_t *)xcalloc(nnz, sizeof(int32_t));
  g->w = (double *)xcalloc(nnz, sizeof(double));
  g->deg = (double *)xcalloc(N, sizeof(double));
  int64_t *cur = (int64_t *)xcalloc(N, sizeof(int64_t));
  OMP_FOR_DYN
  for (int64_t v = 0; v < N; ++v) {
    cur[v] = g->rp[v];
    if (v < Nst)
      for (int64_t k = g->srp[v]; k < g->srp[v + 1]; ++k) {
        g->col[cur[v]] = g->scol[k];
        g->w[cur[v]++] = g->sw_store[k];
      }
  }
  /* cells ascending: their own hint part, and their column in virtual rows */
  int64_t q = 0;
  for (int32_t i = 0; i < C; ++i) {
    if (g->ckind[i] != 0 || !(g->base_w[i] > 0.0)) continue;
    double x = gx[i], y = gy[i], bw = g->base_w[i];
    for (; q < npairs && pairs[q].cell == i; ++q) {
      int32_t m = pairs[q].m, c = g->macro_cell[m];
      double dx = fabs(x - g->fx[Nst + m]), dy = fabs(y - g->fy[Nst + m]);
      double r = fmax(dx / ((double)g->cw[c] * 0.5), dy / ((double)g->ch[c] * 0.5));
      double t = orc_exp(-r);
      t = t * bw;
      double wv = orc_store(-t, g->wdtype);
      int64_t vm = Nst + m;
      g->col[cur[i]] = (int32_t)vm;
      g->w[cur[i]++] = wv;
      g->col[cur[vm]] = i;
      g->w[cur[vm]++] = wv;
    }
    int32_t b = g->cell_bin[i], bx = b % g->nbx, by = b / g->nbx;
    for (int32_t yy = by - g->hy; yy <= by + g->hy; ++yy)
      for (int32_t xx = bx - g->hx; xx <= bx + g->hx; ++xx) {
        if (xx < 0 || yy < 0 || xx >= g->nbx || yy >= g->nby) continue;
        int32_t bb = yy * g->nbx + xx;
        int64_t vb = Nst + g->Mm + bb;
        double dx = fabs(x - g->fx[vb]), dy = fabs(y - g->fy[vb]);
        double r = fmax(dx / (g->wb * 0.5), dy / (g->hb * 0.5));
        double t = orc_exp(-r);
        t = t * g->phi[bb];
        t = t * bw;
        double wv = orc_store(-t, g->wdtype);
        g->col[cur[i]] = (int32_t)vb;
        g->w[cur[i]++] = wv;
        g->col[cur[vb]] = i;
        g->w[cur[vb]++] = wv;
      }
  }
  free(pairs);
  free(cur);
  free(hcnt);

  double *gersh = (double *)xcalloc(N, sizeof(double));
  OMP_FOR_DYN
  for (int64_t v = 0; v < N; ++v) {
    double d = 0.0, a = 0.0;
    for (int64_t k = g->rp[v]; k < g->rp[v + 1]; ++k) {
      d += g->w[k];
      a += fabs(g->w[k]);
    }
    g->deg[v] = d;
    gersh[v] = d + a;
  }
  double lam = 0.0;
  for (int64_t v = 0; v < N; ++v)
    if (gersh[v] > lam || v == 0) lam = gersh[v];
  free(gersh);
  g->lam_up = lam;
  g->have_hints = 1;
  if (!(lam > 0.0) || !isfinite(lam)) return ORC_ERR_SPECTRUM;
  return ORC_OK;
}

void orc_merged_export(const orc_graph *g, int64_t *rp, int32_t *col, double *w, double *deg,
                       double *lam_up, double *Db, double *Cb, double *phi, int32_t *cell_bin) {
  int64_t nnz = g->rp[g->N];
  memcpy(rp, g->rp, sizeof(int64_t) * (g->N + 1));
  memcpy(col, g->col, sizeof(int32_t) * nnz);
  memcpy(w, g->w, sizeof(double) * nnz);
  memcpy(deg, g->deg, sizeof(double) * g->N);
  *lam_up = g->lam_up;
  memcpy(Db, g->Db, sizeof(double) * g->NB);
  memcpy(Cb, g->Cb, sizeof(double) * g->NB);
  memcpy(phi, g->phi, sizeof(double) * g->NB);
  memcpy(cell_bin, g->cell_bin, sizeof(int32_t) * g->C);
}

/* ----------------------------------------- A4: refinement filter H_r */

/* One application of (lambda_up I - L_hint) / lambda_up, k times (the
 * refinement filter H_r = ((lambda_up I - L_hint)/lambda_up)^k, Sec. V). */
static void hr_step(const orc_graph *g, const double *x, double *y) {
  const double lam = g->lam_up;
  OMP_FOR_DYN
  for (int64_t v = 0; v < g->N; ++v) {
    double s = 0.0;
    for (int64_t k = g->rp[v]; k < g->rp[v + 1]; ++k) s += g->w[k] * x[g->col[k]];
    y[v] = ((lam - g->deg[v]) * x[v] + s) / lam;
  }
}

void orc_hr_steps(const orc_graph *g, int k, const double *x, double *y) {
  double *a = (double *)xcalloc(g->N, sizeof(double));
  double *b = (double *)xcalloc(g->N, sizeof(double));
  memcpy(a, x, sizeof(double) * g->N);
  for (int t = 0; t < k; ++t) {
    hr_step(g, a, b);
    double *s = a; a = b; b = s;
  }
  memcpy(y, a, sizeof(double) * g->N);
  free(a); free(b);
}

static void repin(const orc_graph *g, double *x, double *y) {
  for (int64_t v = 0; v < g->N; ++v)
    if (g->nkind[v] == 2) { x[v] = g->fx[v]; y[v] = g->fy[v]; }
}

static void clamp_movable(const orc_graph *g, double *x, double *y) {
  for (int64_t v = 0; v < g->N; ++v) {
    if (g->nkind[v] == 2) continue;
    x[v] = clampd(x[v], g->xl + g->hw[v], g->xh - g->hw[v]);
    y[v] = clampd(y[v], g->yl + g->hh[v], g->yh - g->hh[v]);
  }
}

/* Filter-and-relax step of Algorithm 1: g~ = sum_t alpha_t H_r^{k_t} g
 * (one tap with alpha 1 is the plain order-k filter), then
 * g <- (1 - gamma) g + gamma g~.  Readings: fixed nodes (I/Os, macros, macro
 * pins, virtual nodes) are re-pinned after the whole filter and after the
 * relaxation (optionally after every power); movable cells are then clamped
 * into the region, star nodes as points. */
void orc_filter(const orc_graph *g, const orc_params *pr, const double *gx, const double *gy,
                double *ox, double *oy) {
  const int64_t N = g->N;
  double *ax = (double *)xcalloc(N, sizeof(double)), *ay = (double *)xcalloc(N, sizeof(double));
  double *bx = (double *)xcalloc(N, sizeof(double)), *by = (double *)xcalloc(N, sizeof(double));
  double *tx = (double *)xcalloc(N, sizeof(double)), *ty = (double *)xcalloc(N, sizeof(double));
  memcpy(ax, gx, sizeof(double) * N);
  memcpy(ay, gy, sizeof(double) * N);
  int kmax = 0;
  for (int j = 0; j < pr->ntaps; ++j) kmax = pr->tap_k[j] > kmax ? pr->tap_k[j] : kmax;
  for (int t = 1; t <= kmax; ++t) {
    hr_step(g, ax, bx);
    hr_step(g, ay, by);
    double *s = ax; ax = bx; bx = s;
    s = ay; ay = by; by = s;
    if (pr->pin_every_step) repin(g, ax, ay);
    for (int j = 0; j < pr->ntaps; ++j)
      if (pr->tap_k[j] == t) {
        OMP_FOR
        for (int64_t v = 0; v < N; ++v) {
          tx[v] += pr->tap_alpha[j] * ax[v];
          ty[v] += pr->tap_alpha[j] * ay[v];
        }
      }
  }
  repin(g, tx, ty);
  for (int64_t v = 0; v < N; ++v) {
    ox[v] = (1.0 - pr->gamma) * gx[v] + pr->gamma * tx[v];
    oy[v] = (1.0 - pr->gamma) * gy[v] + pr->gamma * ty[v];
  }
  repin(g, ox, oy);
  if (pr->clamp) clamp_movable(g, ox, oy);
  free(ax); free(ay); free(bx); free(by); free(tx); free(ty);
}

/* -------------------------------------------- A0: GSP-based initialization */

/* tilde A_sigma^k x with tilde A_sigma = D_sigma^{-1/2} (A + sigma I) D_sigma^{-1/2},
 * D_sigma = D + sigma I, A the static instance graph with stored weights
 * (Sec. IV: normalized adjacency with self loops raised to a power). */
int orc_gift_band(const orc_graph *g, double sigma, int k, const double *x, double *y) {
  if (!(sigma > 0.0)) return ORC_ERR_INVALID;
  const int64_t N = g->N;
  double *a = (double *)xcalloc(N, sizeof(double)), *b = (double *)xcalloc(N, sizeof(double));
  double *rs = (double *)xcalloc(N, sizeof(double));
  for (int64_t v = 0; v < N; ++v) {
    double d = (v < g->Nst ? g->sdeg[v] : 0.0) + sigma;
    rs[v] = sqrt(d);
  }
  memcpy(a, x, sizeof(double) * N);
  for (int t = 0; t < k; ++t) {
    OMP_FOR_DYN
    for (int64_t v = 0; v < N; ++v) {
      double s = sigma * a[v] / rs[v];
      if (v < g->Nst)
        for (int64_t q = g->srp[v]; q < g->srp[v + 1]; ++q)
          s += g->sw_store[q] * a[g->scol[q]] / rs[g->scol[q]];
      b[v] = s / rs[v];
    }
    double *sw = a; a = b; b = sw;
  }
  memcpy(y, a, sizeof(double) * N);
  free(a); free(b); free(rs);
  return ORC_OK;
}

/* H g = alpha_low A~^{k_low}_{s_low} g + alpha_mid A~^{k_mid}_{s_mid} g
 *     + alpha_high A~^{k_high}_{s_high} g  (Sec. IV multi-band filter), then
 * step 3 of the GSP initialization: fixed objects re-pinned.  Readings:
 * movable cells are clamped into the region afterwards; with gift_center the
 * region centre is subtracted before filtering and added back after. */
int orc_gift(const orc_graph *g, const orc_params *pr, const double *gx, const double *gy,
             double *ox, double *oy) {
  const int64_t N = g->N;
  double cx = pr->gift_center ? 0.5 * (g->xl + g->xh) : 0.0;
  double cy = pr->gift_center ? 0.5 * (g->yl + g->yh) : 0.0;
  double *ix = (double *)xcalloc(N, sizeof(double)), *iy = (double *)xcalloc(N, sizeof(double));
  double *bx = (double *)xcalloc(N, sizeof(double)), *by = (double *)xcalloc(N, sizeof(double));
  for (int64_t v = 0; v < N; ++v) { ix[v] = gx[v] - cx; iy[v] = gy[v] - cy; ox[v] = 0.0; oy[v] = 0.0; }
  for (int band = 0; band < 3; ++band) {
    int e1 = orc_gift_band(g, pr->gift_sigma[band], pr->gift_k[band], ix, bx);
    int e2 = orc_gift_band(g, pr->gift_sigma[band], pr->gift_k[band], iy, by);
    if (e1 || e2) { free(ix); free(iy); free(bx); free(by); return ORC_ERR_INVALID; }
    for (int64_t v = 0; v < N; ++v) {
      ox[v] += pr->gift_alpha[band] * bx[v];
      oy[v] += pr->gift_alpha[band] * by[v];
    }
  }
  for (int64_t v = 0; v < N; ++v) { ox[v] += cx; oy[v] += cy; }
  repin(g, ox, oy);
  if (pr->clamp) clamp_movable(g, ox, oy);
  free(ix); free(iy); free(bx); free(by);
  return ORC_OK;
}

/* Step 1 of the GSP initialization (Sec. IV): movable cells sampled uniformly
 * in the region (or taken from xy0, interleaved x,y per cell), fixed objects
 * pinned.  Readings: the sample for cell i, axis a is splitmix64 counter
 * 2i+a; a star node starts at the mean of its net's distinct nodes. */
void orc_init_signal(const orc_graph *g, uint64_t seed, const float *xy0, double *gx,
                     double *gy) {
  for (int64_t v = 0; v < g->N; ++v) { gx[v] = g->fx[v]; gy[v] = g->fy[v]; }
  for (int32_t i = 0; i < g->C; ++i) {
    if (g->nkind[i] != 0) continue;
    if (xy0) {
      gx[i] = xy0[2 * (int64_t)i];
      gy[i] = xy0[2 * (int64_t)i + 1];
    } else {
      gx[i] = g->xl + orc_u01(seed, 2 * (uint64_t)i) * (g->xh - g->xl);
      gy[i] = g->yl + orc_u01(seed, 2 * (uint64_t)i + 1) * (g->yh - g->yl);
    }
  }
  for (int32_t s = 0; s < g->S; ++s) {
    int32_t e = g->star_net[s];
    double sx = 0.0, sy = 0.0;
    int64_t n = g->nd_ptr[e + 1] - g->nd_ptr[e];
    for (int64_t k = g->nd_ptr[e]; k < g->nd_ptr[e + 1]; ++k) {
      sx += gx[g->nd[k]];
      sy += gy[g->nd[k]];
    }
    gx[g->C + g->Pm + s] = sx / (double)n;
    gy[g->C + g->Pm + s] = sy / (double)n;
  }
}

/* The whole initializer: GSP initialization, then Algorithm 1 for t_hint
 * rounds (BuildLap -> ComputeFilter -> filter -> relax).  gx, gy receive all
 * N node coordinates. */
int orc_run(orc_graph *g, const orc_params *pr, uint64_t seed, const float *xy0, double *gx,
            double *gy) {
  const int64_t N = g->N;
  double *tx = (double *)xcalloc(N, sizeof(double)), *ty = (double *)xcalloc(N, sizeof(double));
  orc_init_signal(g, seed, xy0, gx, gy);
  int err = ORC_OK;
  if (pr->gift_enable) {
    err = orc_gift(g, pr, gx, gy, tx, ty);
    if (err) goto out;
    memcpy(gx, tx, sizeof(double) * N);
    memcpy(gy, ty, sizeof(double) * N);
  } else if (pr->clamp) {
    clamp_movable(g, gx, gy);
  }
  for (int t = 0; t < pr->t_hint; ++t) {
    err = orc_build_hints(g, pr, gx, gy);
    if (err) goto out;
    orc_filter(g, pr, gx, gy, tx, ty);
    memcpy(gx, tx, sizeof(double) * N);
    memcpy(gy, ty, sizeof(double) * N);
  }
out:
  free(tx); free(ty);
  return err;
}

/* ---------------------------------------------------------- A5: HPWL */

/* Half-perimeter wirelength: sum over nets of (max - min) of pin x plus
 * (max - min) of pin y, pin = cell centre + pin offset, net weight 1.  The
 * paper uses HPWL as its quality metric (Sec. VII, VIII) without restating
 * the standard definition. */
double orc_hpwl(const orc_netlist *nl, const double *cx, const double *cy) {
  double *span = (double *)xcalloc(nl->num_nets, sizeof(double));
  OMP_FOR_DYN
  for (int32_t e = 0; e < nl->num_nets; ++e) {
    int64_t b = nl->net_ptr[e], n = nl->net_ptr[e + 1] - b;
    if (n < 1) continue;
    double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
    for (int64_t k = b; k < b + n; ++k) {
      int32_t c = nl->pin_cell[k];
      double px = cx[c] + (nl->pin_dx ? (double)nl->pin_dx[k] : 0.0);
      double py = cy[c] + (nl->pin_dy ? (double)nl->pin_dy[k] : 0.0);
      x0 = fmin(x0, px); x1 = fmax(x1, px);
      y0 = fmin(y0, py); y1 = fmax(y1, py);
    }
    span[e] = (x1 - x0) + (y1 - y0);
  }
  double total = 0.0;
  for (int32_t e = 0; e < nl->num_nets; ++e) total += span[e];
  free(span);
  return total;
}

/* ------------------------------- Sec. VI: macro charge-density schedules */

#define ORC_PI 3.14159265358979323846

/* Gauss-Legendre nodes and weights on [-1, 1]: the roots of P_n by Newton's
 * method from the classical starting guesses cos(pi (i - 1/4) / (n + 1/2)),
 * P_n and P_n' from the three-term recurrence; weights 2 / ((1 - x^2) P_n'^2). */
void orc_gauss_legendre(int n, double *x, double *w) {
  for (int i = 1; i <= n; ++i) {
    double z = cos(ORC_PI * (i - 0.25) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i - 1] = -z;
    w[i - 1] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* Blended concentration eta(t) of the charge-redistribution model:
 * alpha = t / T; scheme A: log r = (1 - alpha) log r0 + alpha log r1,
 * eta_A = sqrt(-2 log r); scheme B: beta = beta_min + (beta_max - beta_min)
 * alpha, eta_B = sqrt(2 ln 2) / beta; smoothstep w(alpha) between alpha0 and
 * alpha1; eta = eta_B^(1 - w) eta_A^w. */
double orc_rho_eta(const orc_rho_params *rp, int t) {
  double a = (double)t / (double)rp->T;
  double lr = (1.0 - a) * log(rp->r0) + a * log(rp->r1);
  double ea = sqrt(-2.0 * lr);
  double beta = rp->beta_min + (rp->beta_max - rp->beta_min) * a;
  double eb = sqrt(2.0 * log(2.0)) / beta;
  double wgt;
  if (a <= rp->alpha0) wgt = 0.0;
  else if (a >= rp->alpha1) wgt = 1.0;
  else {
    double z = (a - rp->alpha0) / (rp->alpha1 - rp->alpha0);
    wgt = 3.0 * z * z - 2.0 * z * z * z;
  }
  return pow(eb, 1.0 - wgt) * pow(ea, wgt);
}

/* sigma(t) = -sigma_factor T ln(1 - t / T) of the exponential-like model
 * (infinite at t = T). */
double orc_rho_sigma(const orc_rho_params *rp, int t) {
  if (t >= rp->T) return INFINITY;
  return -rp->sigma_factor * rp->T * log(1.0 - (double)t / (double)rp->T);
}

/* k(t) = k_factor / tan(pi t / (2 T)) of the linear- and sigmoid-like models
 * (infinite at t = 0, 0 at t = T). */
double orc_rho_k(const orc_rho_params *rp, int t) {
  if (t <= 0) return INFINITY;
  if (t >= rp->T) return 0.0;
  return rp->k_factor / tan(0.5 * ORC_PI * (double)t / (double)rp->T);
}

/* The density rho_t at offset (dx, dy) from the centre of a w x h macro, zero
 * outside the macro.  Readings where the paper is silent: the linear-like
 * density is clamped at 0 (a charge density; the restored region is
 * r <= 1 / k); with sigma = 0 or k = infinity the density is 0 away from the
 * centre; with sigma = infinity or k = 0 it is 1. */
double orc_rho_value(const orc_rho_params *rp, int t, double dx, double dy, double w, double h) {
  if (fabs(dx) > 0.5 * w || fabs(dy) > 0.5 * h) return 0.0;
  double u = dx / w, v = dy / h;
  if (rp->model == ORC_RHO_GAUSS) {
    double eta = orc_rho_eta(rp, t), e = erf(eta / sqrt(2.0));
    return 2.0 * eta * eta / (ORC_PI * e * e) * exp(-2.0 * eta * eta * (u * u + v * v));
  }
  if (rp->model == ORC_RHO_EXP) {
    double sg = orc_rho_sigma(rp, t);
    if (isinf(sg)) return 1.0;
    if (!(sg > 0.0)) return 0.0;
    double tx = tan(ORC_PI * u), ty = tan(ORC_PI * v);
    return exp(-(tx * tx + ty * ty) / (2.0 * sg * sg));
  }
  double k = orc_rho_k(rp, t), r = sqrt(2.0 * (u * u + v * v));
  if (isinf(k)) return 0.0;
  if (rp->model == ORC_RHO_LINEAR) return fmax(0.0, 1.0 - k * r);
  return 2.0 / (1.0 + exp(k * r));
}

/* Composite Gauss-Legendre sum of f over [a, b]: `panels` equal panels,
 * `nodes` points each. */
static double gl_1d(double a, double b, int panels, int nodes, const double *gx, const double *gw,
                    double (*f)(double, const void *), const void *ctx) {
  double s = 0.0, hp = (b - a) / panels;
  for (int p = 0; p < panels; ++p) {
    double c = a + (p + 0.5) * hp;
    for (int i = 0; i < nodes; ++i) s += 0.5 * hp * gw[i] * f(c + 0.5 * hp * gx[i], ctx);
  }
  return s;
}

typedef struct { double scale; double w; } exp_ctx;
static double exp_1d(double d, const void *c) {
  const exp_ctx *e = (const exp_ctx *)c;
  double tv = tan(ORC_PI * d / e->w);
  return exp(-tv * tv * e->scale);
}

/* Integral of rho_t over [ax, bx] x [ay, by] (offsets from the macro centre),
 * the part inside the macro.  Gaussian: the separable closed form with erf;
 * exponential-like: separable, a composite Gauss-Legendre rule per axis;
 * linear- and sigmoid-like: the tensor rule on the rectangle. */
double orc_rho_integral(const orc_rho_params *rp, int t, double w, double h, double ax, double bx,
                        double ay, double by) {
  ax = fmax(ax, -0.5 * w); bx = fmin(bx, 0.5 * w);
  ay = fmax(ay, -0.5 * h); by = fmin(by, 0.5 * h);
  if (!(bx > ax) || !(by > ay)) return 0.0;
  if (rp->model == ORC_RHO_GAUSS) {
    double eta = orc_rho_eta(rp, t), e = erf(eta / sqrt(2.0));
    double A = 2.0 * eta * eta / (ORC_PI * e * e);
    double c = sqrt(2.0) * eta;
    /* int_a^b exp(-2 eta^2 d^2 / w^2) dd = w sqrt(pi) / (2 sqrt(2) eta) [erf(c b / w) - erf(c a / w)] */
    double ix = w * sqrt(ORC_PI) / (2.0 * c) * (erf(c * bx / w) - erf(c * ax / w));
    double iy = h * sqrt(ORC_PI) / (2.0 * c) * (erf(c * by / h) - erf(c * ay / h));
    return A * ix * iy;
  }
  int n = rp->nodes, P = rp->panels;
  double *gx = (double *)xcalloc(n, sizeof(double)), *gw = (double *)xcalloc(n, sizeof(double));
  orc_gauss_legendre(n, gx, gw);
  double r = 0.0;
  if (rp->model == ORC_RHO_EXP) {
    double sg = orc_rho_sigma(rp, t);
    if (isinf(sg)) r = (bx - ax) * (by - ay);
    else if (sg > 0.0) {
      exp_ctx cx = {1.0 / (2.0 * sg * sg), w}, cy = {1.0 / (2.0 * sg * sg), h};
      r = gl_1d(ax, bx, P, n, gx, gw, exp_1d, &cx) * gl_1d(ay, by, P, n, gx, gw, exp_1d, &cy);
    }
  } else {
    double hx = (bx - ax) / P, hy = (by - ay) / P;
    for (int px = 0; px < P; ++px)
      for (int py = 0; py < P; ++py) {
        double cx = ax + (px + 0.5) * hx, cy = ay + (py + 0.5) * hy;
        for (int i = 0; i < n; ++i)
          for (int j = 0; j < n; ++j)
            r += 0.25 * hx * hy * gw[i] * gw[j] *
                 orc_rho_value(rp, t, cx + 0.5 * hx * gx[i], cy + 0.5 * hy * gx[j], w, h);
      }
  }
  free(gx);
  free(gw);
  return r;
}

/* Delta rho_b(t) summed over macros (ascending): for every bin b of the
 * nbx x nby grid over the region, the integral over B_b of each macro's
 * rho_t (Sec. VI), in area units. */
void orc_macro_density(const orc_rho_params *rp, int t, int32_t nm, const double *mx,
                       const double *my, const double *mw, const double *mh, double xl, double yl,
                       double xh, double yh, int32_t nbx, int32_t nby, double *out) {
  double wb = (xh - xl) / nbx, hb = (yh - yl) / nby;
  for (int64_t b = 0; b < (int64_t)nbx * nby; ++b) out[b] = 0.0;
  for (int32_t b = 0; b < nbx * nby; ++b) {
    int32_t bx = b % nbx, by = b / nbx;
    double x0 = xl + bx * wb, x1 = xl + (bx + 1) * wb, y0 = yl + by * hb, y1 = yl + (by + 1) * hb;
    double s = 0.0;
    for (int32_t m = 0; m < nm; ++m)
      s += orc_rho_integral(rp, t, mw[m], mh[m], x0 - mx[m], x1 - mx[m], y0 - my[m], y1 - my[m]);
    out[b] = s;
  }
}
