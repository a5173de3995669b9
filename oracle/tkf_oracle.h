/*
 * ORACLE -- test infrastructure only (see tkf_oracle.c).  Plain FP64 C; no code shared with
 * the CUDA library.
 */
#ifndef TKF_ORACLE_H
#define TKF_ORACLE_H

#define ORC_MAX_LAYERS 16

enum { ORC_OK = 0, ORC_ERR_NOREACH = 1, ORC_ERR_SINGULAR = 2, ORC_ERR_INVALID = 3 };

typedef struct {
    int n_layers;
    double radius[ORC_MAX_LAYERS];
    double bz;
    double x_over_x0[ORC_MAX_LAYERS];
    double mass;
    double prior_sigma[6];
    double eta_min, eta_bin_w;
    int n_eta_bins, n_phi_bins;
    double chi2_cut;
    double window_margin;
    double tie_tol;        /* relative closeness that marks a ranking or cut decision fragile */
    int n_cand;            /* candidates kept per seed; <= 0 keeps every branch */
    int brute_force;       /* 1: examine every hit of the layer instead of the binned window;
                              2 (hit_dr > 0): also without the residual window, every hit of the
                              layer scored at its own radius */
    int first_build_layer; /* 0-based layer where building starts (3 = fourth layer) */
    double hit_dr;         /* largest |hit radius - layer radius| (cm); 0: hits lie on the cylinders.
                              > 0: the CMS-geometry variant of Sec. 2.2, states are taken to each
                              hit's own radius (see tkf_oracle.c) */
    double disk_z[ORC_MAX_LAYERS]; /* > 0: layer l is a pair of endcap disks at z = +-disk_z[l]
                                      (Sec. 2.2, "or endcap z"); 0: a cylinder of radius[l] */
} orc_geom;

typedef struct {
    double x, y, z, var_u, var_v;
    int layer;
    int disk; /* 1: a hit on an endcap disk, measured in r-phi (var_u) and r (var_v); 0: on a
                 cylinder, measured in r-phi and z */
} orc_hit;

typedef struct {
    int n_hits;
    const orc_hit *hits;   /* event-local ids 0..n_hits-1 */
    const int *order;      /* hit ids sorted by (layer, bin, id) */
    const int *bin_off;    /* [n_layers][n_bins + 1] CSR offsets into order */
    double var_u_max[ORC_MAX_LAYERS], var_v_max[ORC_MAX_LAYERS];
} orc_event;

typedef struct {
    int cap;        /* candidates the output arrays can hold */
    int n_cand;     /* candidates at the end (may exceed cap when n_cand <= 0) */
    int fragile_layer;
    double *par;    /* [cap][6] */
    double *cov;    /* [cap][36] */
    double *chi2;   /* [cap] */
    int *nhits;     /* [cap] */
    int *hits;      /* [cap][n_layers] */
} orc_seed_result;

typedef struct {
    long long n_prop, n_hits_examined, n_updates, n_kept;
    long long n_steps; /* hits off the cylinder (hit_dr > 0) taken to their own radius and scored */
} orc_stats;

int orc_propagate(const orc_geom *g, const double pin[6], double R, double pout[6], double J[36]);
/* to the plane z = Zp (an endcap disk) */
int orc_propagate_plane(const orc_geom *g, const double pin[6], double Zp, double pout[6], double J[36]);
void orc_scatter(const orc_geom *g, int layer, const double p[6], double P[36]);
double orc_chi2(const double p[6], const double P[36], const orc_hit *h);
int orc_update(double p[6], double P[36], const orc_hit *h, double *chi2);
int orc_seed_estimate(const orc_geom *g, const orc_hit *h1, const orc_hit *h2, const orc_hit *h3,
                      double p[6], double P[36]);
int orc_fit_track(const orc_geom *g, const double pin[6], const double Pin[36], const orc_hit *hits,
                  const int *hit_of_layer, int first, int last, double pout[6], double Pout[36],
                  double *chi2, int *nhits);
/* inward (backward) pass over layers last..first, first <= last; see tkf_oracle.c */
int orc_fit_backward(const orc_geom *g, const double pin[6], const double Pin[36], double cov_scale,
                     const orc_hit *hits, const int *hit_of_layer, int last, int first, double pout[6],
                     double Pout[36], double *chi2, int *nhits);
int orc_eta_bin(const orc_geom *g, int layer, double z);
/* the eta bin of a hit: asinh(z / R) on a cylinder of radius R, asinh(z / r_hit) on a disk */
int orc_hit_eta_bin(const orc_geom *g, const orc_hit *h);
int orc_phi_bin(const orc_geom *g, double phi);
int orc_hit_index(const orc_geom *g, int n, const orc_hit *hits, int *bin_of_hit, int *order, int *bin_off);
int orc_build_seed(const orc_geom *g, const orc_event *ev, const double sp[6], const double sP[36],
                   double schi2, int snhits, const int *shits, orc_seed_result *res, orc_stats *stats);

/* Seeding from hit triplets on layers 0, 1, 2 with a confirmation hit on layer 3 (the seeding
 * stage of Sec. 2, which the paper names but does not specify; the reading is in tkf_oracle.c).
 * Lengths in cm, pt_min in GeV. */
typedef struct {
    double pt_min;      /* curvature limit kappa_max = ORC_KB * bz / pt_min * (1 + kappa_slack) */
    double kappa_slack;
    double z_vertex;    /* |z at r = 0| of the r-z line through the first two hits */
    double d0_max;      /* |power of the beam line point / circle diameter| of the triplet circle */
    double dz_max;      /* |z of the third hit - the r-z line through the first two| */
    double conf_rphi;   /* |signed distance of the layer-3 hit from the triplet circle| */
    double conf_z;      /* |z of the layer-3 hit - the r-z line through the second and third hits| */
    int confirm;        /* 1: a confirmation hit on layer 3 is required */
} orc_seed_cuts;

/* The quantities of one candidate; a stage not reached keeps zeros. */
typedef struct {
    double chord01, kappa01, zv;          /* pair (first, second hit) */
    double chord12, kappa, d0, dz;        /* triplet */
    double chord23, f3, dz3;              /* confirmation hit (when one is given) */
    int collinear;                        /* the triplet's three points are collinear: rejected */
} orc_seed_quant;

/* Best triplet for one first-layer hit. */
typedef struct {
    int h1, h2, h3;   /* event-local ids of the chosen hits on layers 1, 2 and the confirmation hit
                         on layer 3 (h1 = -1: no seed) */
    int n_pass;       /* triplets that pass every cut (with a confirmation hit when required) */
    double score;     /* score of the chosen triplet */
    double margin;    /* smallest relative distance |q - cut| / cut over the decisions that could
                         change the result: every quantity of a passing candidate, the one failing
                         quantity of a candidate that fails on exactly one (1e30: none) */
    double gap;       /* second best minus best passing score (1e30: fewer than two) */
} orc_seed_pick;

double orc_seed_kappa_max(const orc_geom *g, const orc_seed_cuts *c);
/* quantities of (a, b, cc[, e]) (e may be NULL); returns 1 if every cut passes */
int orc_seed_eval(const orc_geom *g, const orc_seed_cuts *c, const orc_hit *a, const orc_hit *b, const orc_hit *cc,
                  const orc_hit *e, orc_seed_quant *q);
/* every hit of layer 0 among hits[0..n) (one event): its best triplet in pick[hit id]; entries of
 * hits on other layers get h1 = -1 */
int orc_find_seeds(const orc_geom *g, const orc_seed_cuts *c, int n, const orc_hit *hits, orc_seed_pick *pick);
/* the same for the listed first-layer hits only (pick[k] for first[k]) */
int orc_find_seeds_of(const orc_geom *g, const orc_seed_cuts *c, int n, const orc_hit *hits, int n_first,
                      const int *first, orc_seed_pick *pick);

/* batch helpers (plain loops over the single-object functions above) */
int orc_seed_batch(const orc_geom *g, const orc_hit *hits, int n, const int *seed_hits /*[n][3]*/,
                   double *par /*[n][6]*/, double *cov /*[n][36]*/);
int orc_fit_batch(const orc_geom *g, const orc_hit *hits, int n, const double *par_in, const double *cov_in,
                  const int *hit_ids /*[n][n_layers]*/, int first, int last, double *par_out, double *cov_out,
                  double *chi2, int *nhits, int *status);
int orc_fit_backward_batch(const orc_geom *g, const orc_hit *hits, int n, const double *par_in,
                           const double *cov_in, double cov_scale, const int *hit_ids, int last, int first,
                           double *par_out, double *cov_out, double *chi2, int *nhits, int *status);
int orc_build_batch(const orc_geom *g, const orc_event *ev, int n, const double *sp, const double *sP,
                    const double *schi2, const int *snhits, const int *shits /*[n][n_layers]*/, int cap,
                    int *n_cand, double *par, double *cov, double *chi2, int *nhits, int *hits,
                    int *fragile, orc_stats *stats);

#endif
