/* FP64 CPU oracle of the area-hint refinement initializer.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, sequential statement of
 * what the CUDA library computes; it exists to check that library.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header or constant table with the CUDA library.
 *
 * Paper: "Bridging the Initialization Gap: A Co-Optimization Framework for
 * Mixed-Size Global Placement" (arXiv 2511.10073).
 *   Sec. II-A  graph, Laplacian, spectral filter definitions
 *   Sec. IV    GSP-based initialization (GiFt multi-band filter)
 *   Sec. V     area-hint refinement: macro pin expansion, macro / bin virtual
 *              nodes with signed edges, refinement filter H_r, Algorithm 1
 *   Sec. VII / VIII  HPWL as the quality metric
 * Readings where the paper is silent are listed at each function.
 */
#ifndef ORC_H
#define ORC_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_ERR_INVALID = 1, ORC_ERR_SPECTRUM = 5, ORC_ERR_NONFINITE = 6 };
enum { ORC_W_FP64 = 0, ORC_W_FP32 = 1, ORC_W_BF16 = 2 };

typedef struct {
  int32_t num_cells, num_nets;
  int64_t num_pins;
  const int64_t *net_ptr;   /* [num_nets+1] */
  const int32_t *pin_cell;  /* [num_pins] */
  const float *pin_dx, *pin_dy; /* [num_pins] or NULL */
  const float *cell_w, *cell_h; /* [num_cells] */
  const uint8_t *cell_kind;     /* 0 movable, 1 fixed macro, 2 fixed I/O */
  const float *fixed_x, *fixed_y;
  double xl, yl, xh, yh;
} orc_netlist;

typedef struct {
  int32_t clique_max;      /* nets with <= clique_max distinct nodes: clique model */
  int32_t wdtype;          /* storage of edge weights (ORC_W_*) */
  int32_t gift_enable;
  int32_t gift_center;
  int32_t gift_k[3];       /* bands: low, mid, high */
  double  gift_sigma[3];
  double  gift_alpha[3];
  int32_t t_hint;
  int32_t nbx, nby;
  double  gamma, det_ratio, capacity, mu;
  int32_t ntaps;
  int32_t tap_k[4];
  double  tap_alpha[4];
  int32_t pin_every_step;
  int32_t clamp;
} orc_params;

typedef struct orc_graph orc_graph;

orc_graph *orc_create(const orc_netlist *nl, const orc_params *pr, int *err);
void orc_destroy(orc_graph *g);
void orc_sizes(const orc_graph *g, int64_t out[16]);
void orc_static_export(const orc_graph *g, int64_t *rp, int32_t *col, double *w_exact,
                       double *w_store, double *base_w);
void orc_nodes_export(const orc_graph *g, uint8_t *nkind, double *fx, double *fy,
                      double *hw, double *hh, int32_t *pin_node);
int  orc_build_hints(orc_graph *g, const orc_params *pr, const double *gx, const double *gy);
void orc_merged_export(const orc_graph *g, int64_t *rp, int32_t *col, double *w, double *deg,
                       double *lam_up, double *Db, double *Cb, double *phi, int32_t *cell_bin);
void orc_hr_steps(const orc_graph *g, int k, const double *x, double *y);
void orc_filter(const orc_graph *g, const orc_params *pr, const double *gx, const double *gy,
                double *ox, double *oy);
int  orc_gift_band(const orc_graph *g, double sigma, int k, const double *x, double *y);
int  orc_gift(const orc_graph *g, const orc_params *pr, const double *gx, const double *gy,
              double *ox, double *oy);
void orc_init_signal(const orc_graph *g, uint64_t seed, const float *xy0,
                     double *gx, double *gy);
int  orc_run(orc_graph *g, const orc_params *pr, uint64_t seed, const float *xy0,
             double *gx, double *gy);
double orc_hpwl(const orc_netlist *nl, const double *cx, const double *cy);

/* Sec. VI: iteration-scheduled macro charge densities and their bin integrals */
enum { ORC_RHO_GAUSS = 0, ORC_RHO_EXP = 1, ORC_RHO_LINEAR = 2, ORC_RHO_SIGMOID = 3 };
typedef struct {
  int32_t model;          /* ORC_RHO_* */
  int32_t T;              /* iterations of the schedule */
  double r0, r1;          /* scheme A: edge decay ratio at alpha = 0 and 1 */
  double beta_min, beta_max; /* scheme B: normalized FWHM at alpha = 0 and 1 */
  double alpha0, alpha1;  /* smoothstep blend between them */
  double sigma_factor;    /* exponential-like model */
  double k_factor;        /* linear-like and sigmoid-like models */
  int32_t panels, nodes;  /* composite Gauss-Legendre rule per axis */
} orc_rho_params;
void orc_gauss_legendre(int n, double *x, double *w);
double orc_rho_eta(const orc_rho_params *rp, int t);
double orc_rho_sigma(const orc_rho_params *rp, int t);
double orc_rho_k(const orc_rho_params *rp, int t);
double orc_rho_value(const orc_rho_params *rp, int t, double dx, double dy, double w, double h);
double orc_rho_integral(const orc_rho_params *rp, int t, double w, double h, double ax, double bx,
                        double ay, double by);
void orc_macro_density(const orc_rho_params *rp, int t, int32_t nm, const double *mx,
                       const double *my, const double *mw, const double *mh, double xl, double yl,
                       double xh, double yh, int32_t nbx, int32_t nby, double *out);
double orc_exp(double x);
double orc_u01(uint64_t seed, uint64_t ctr);
double orc_store(double w, int dtype);

#ifdef __cplusplus
}
#endif
#endif
