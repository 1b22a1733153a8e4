/*
 * FP64 CPU oracle (test infrastructure only): declarations for fd2d.c.
 * The propagators follow Section 2.1 Eqs. 1-2, Section 2.2 Eqs. 9-12b and
 * Section 2.3.1 Eq. 13 of arXiv 2403.17518; see fd2d.c for the discrete form.
 */
#ifndef DHFWI_ORACLE_H
#define DHFWI_ORACLE_H

typedef struct {
    int nz, nx, nb;   /* physical grid and sponge width (cells) */
    double h, dt;     /* grid spacing (m), time step (s) */
} or_grid;

typedef struct {
    int n_shots;
    const int *src_iz, *src_ix, *nt;     /* [n_shots] */
    const int *rec_off;                  /* [n_shots+1] CSR into rec_iz/rec_ix */
    const int *rec_iz, *rec_ix;          /* physical receiver nodes */
    const int *win_x0, *win_x1;          /* physical column window per shot */
    const double *wavelet;               /* [nt_max] or [n_shots][nt_max] */
    int nt_max;
    int wavelet_shared;
} or_geom;

void or_model_shots(const or_grid *g, const double *v, const or_geom *G, double *d);
double or_fwi_gradient(const or_grid *g, const double *v, const or_geom *G, const double *d_obs,
                       double *grad, double *d_syn, int seg);
void or_born_demig(const or_grid *g, const double *v0, const or_geom *G, const double *dv,
                   double *d);
void or_rtm_mig(const or_grid *g, const double *v0, const or_geom *G, const double *d,
                double *img, int seg);
void or_apply_lap(int NZ, int NX, const double *u, double *out);
void or_sponge(const or_grid *g, int win_w, double *w_out);

#endif
