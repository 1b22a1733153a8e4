/*
 * FP64 CPU oracle for the wave-equation operators of "Robust Full Waveform
 * Inversion with deep Hessian deblurring" (arXiv 2403.17518).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package's smoke check
 * and the CPU-baseline leg of the benchmark may load this library.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * What it computes (plain loops, float64, no blocking or fusion):
 *
 *   Wave equation, Section 2.1 Eq. 1:  m^-2 u_tt - lap(u) = f, m = velocity.
 *   Discretised with 2nd-order leapfrog in time and the 8th-order central
 *   second difference in space (unscaled D, so lap_h = D/h^2), a source
 *   sampled on one node (q^n = f(n dt), the discrete f(t) delta(x) with
 *   delta_h = 1/h^2), zero values outside the padded grid, and a Cerjan
 *   sponge w applied to both time levels:
 *
 *     a^n     = D u^n + q^n
 *     u^{n+1} = w (2 u^n + kappa a^n) - w^2 u^{n-1},   kappa = v^2 dt^2 / h^2
 *     d[n][r] = u^{n+1}(receiver r),   n = 0 .. nt-1,   u^0 = u^{-1} = 0
 *
 *   Misfit, Section 2.1 Eq. 2:  J = 1/2 sum (d_s - d_o)^2.
 *   Gradient dJ/dv by the exact discrete adjoint of the recurrence above
 *   (the paper's g = L~^T (d_o - d_s), Section 2.3.1 Eq. 13, is -dJ/dv):
 *     lambda^k = P^T r^{k-1} + 2 w lambda^{k+1} + D(kappa w lambda^{k+1})
 *                - w^2 lambda^{k+2},      k = nt .. 1, lambda^{nt+1,nt+2} = 0
 *     dJ/dv   += (2 v dt^2/h^2) w a^{k-1} lambda^k
 *   Born modelling, Section 2.2 Eqs. 9-12b, solved jointly (Eq. 9 and Eq. 11
 *   together, "no need to store the background wavefield"): the tangent of
 *   the recurrence with respect to v, whose secondary source is
 *   (2 v dt^2/h^2) w dv a0^n (discrete 2 dv/v^3 d_tt u0 of Eq. 11).
 *   Migration (adjoint of Born, Eq. 13 applied to arbitrary data): the
 *   adjoint recurrence above with r replaced by the input data.
 *
 * Per-shot padded domain: the physical window [x0, x1) of the model,
 * extended by nb cells on all four sides; the velocity there is taken from
 * the model with indices clamped to the model (edge replication).  Gradients
 * and images are folded back through that extension (its exact transpose).
 * The sponge factor counts distance from the window's outer edge.
 *
 * The backward passes keep checkpoints of (u^{n-1}, u^n) every `seg` steps
 * and recompute each segment forward before sweeping it backward; the
 * recomputed values are bit-identical to the first pass, so this changes
 * memory use only, not the arithmetic.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* 8th-order central second-difference weights (unit spacing). */
static const double OR_C[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};

typedef struct {
    int NZ, NX;     /* padded window size */
    int x0;         /* physical column of the window start */
    int sz, sx;     /* source node, padded coordinates */
    int nrec;
    int *rz, *rx;   /* receivers, padded coordinates */
    int nt;
    const double *wav;
    double *v;      /* extended velocity */
    double *kap;    /* v^2 dt^2 / h^2 */
    double *w;      /* sponge factor */
} shot_t;

static int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

static double cerjan(int d, int nb) {
    /* Cerjan et al. (1985) factor, d = cells from the outer edge. */
    if (d >= nb) return 1.0;
    double t = 0.015 * (double)(nb - d);
    return exp(-t * t);
}

static void shot_init(shot_t *S, const or_grid *g, const double *v, const or_geom *G, int s) {
    int nb = g->nb;
    int x0 = G->win_x0[s], x1 = G->win_x1[s];
    S->x0 = x0;
    S->NZ = g->nz + 2 * nb;
    S->NX = (x1 - x0) + 2 * nb;
    S->sz = G->src_iz[s] + nb;
    S->sx = G->src_ix[s] - x0 + nb;
    int a = G->rec_off[s], b = G->rec_off[s + 1];
    S->nrec = b - a;
    S->rz = (int *)malloc(sizeof(int) * (size_t)(S->nrec > 0 ? S->nrec : 1));
    S->rx = (int *)malloc(sizeof(int) * (size_t)(S->nrec > 0 ? S->nrec : 1));
    for (int r = 0; r < S->nrec; r++) {
        S->rz[r] = G->rec_iz[a + r] + nb;
        S->rx[r] = G->rec_ix[a + r] - x0 + nb;
    }
    S->nt = G->nt[s];
    S->wav = G->wavelet + (G->wavelet_shared ? 0 : (size_t)s * (size_t)G->nt_max);
    size_t n = (size_t)S->NZ * S->NX;
    S->v = (double *)malloc(sizeof(double) * n);
    S->kap = (double *)malloc(sizeof(double) * n);
    S->w = (double *)malloc(sizeof(double) * n);
    double c = g->dt * g->dt / (g->h * g->h);
    for (int i = 0; i < S->NZ; i++) {
        int pz = clampi(i - nb, 0, g->nz - 1);
        int dz = i < S->NZ - 1 - i ? i : S->NZ - 1 - i;
        for (int j = 0; j < S->NX; j++) {
            int px = clampi(x0 + j - nb, 0, g->nx - 1);
            int dx = j < S->NX - 1 - j ? j : S->NX - 1 - j;
            double vv = v[(size_t)pz * g->nx + px];
            S->v[(size_t)i * S->NX + j] = vv;
            S->kap[(size_t)i * S->NX + j] = vv * vv * c;
            S->w[(size_t)i * S->NX + j] = cerjan(dz, nb) * cerjan(dx, nb);
        }
    }
}

static void shot_free(shot_t *S) {
    free(S->rz); free(S->rx); free(S->v); free(S->kap); free(S->w);
}

/* Extension E: physical model -> padded window (edge replication). */
static void extend(const shot_t *S, const or_grid *g, const double *phys, double *ext) {
    for (int i = 0; i < S->NZ; i++) {
        int pz = clampi(i - g->nb, 0, g->nz - 1);
        for (int j = 0; j < S->NX; j++) {
            int px = clampi(S->x0 + j - g->nb, 0, g->nx - 1);
            ext[(size_t)i * S->NX + j] = phys[(size_t)pz * g->nx + px];
        }
    }
}

/* Transpose of the extension: sum padded cells into the model cell they copy. */
static void fold_add(const shot_t *S, const or_grid *g, const double *ext, double *phys) {
    for (int i = 0; i < S->NZ; i++) {
        int pz = clampi(i - g->nb, 0, g->nz - 1);
        for (int j = 0; j < S->NX; j++) {
            int px = clampi(S->x0 + j - g->nb, 0, g->nx - 1);
            phys[(size_t)pz * g->nx + px] += ext[(size_t)i * S->NX + j];
        }
    }
}

static double at(const double *u, int NZ, int NX, int i, int j) {
    if (i < 0 || i >= NZ || j < 0 || j >= NX) return 0.0;
    return u[(size_t)i * NX + j];
}

/* Unscaled 8th-order Laplacian D u at (i, j): both axes, zero outside. */
static double lap(const double *u, int NZ, int NX, int i, int j) {
    double s = 2.0 * OR_C[0] * u[(size_t)i * NX + j];
    for (int k = 1; k <= 4; k++) {
        s += OR_C[k] * (at(u, NZ, NX, i, j + k) + at(u, NZ, NX, i, j - k) +
                        at(u, NZ, NX, i + k, j) + at(u, NZ, NX, i - k, j));
    }
    return s;
}

/* One forward step n: unew = w (2u + kap a) - w^2 uold, a = D u + q^n. */
static void fwd_step(const shot_t *S, int n, const double *uold, const double *u, double *unew,
                     double *a_out) {
    for (int i = 0; i < S->NZ; i++) {
        for (int j = 0; j < S->NX; j++) {
            size_t c = (size_t)i * S->NX + j;
            double a = lap(u, S->NZ, S->NX, i, j);
            if (i == S->sz && j == S->sx) a += S->wav[n];
            double w = S->w[c];
            unew[c] = w * (2.0 * u[c] + S->kap[c] * a) - w * w * uold[c];
            if (a_out) a_out[c] = a;
        }
    }
}

/* Forward modelling of one shot; records d[n][r] = u^{n+1}(r).  If ck_every
 * > 0, stores checkpoints (u^{n-1}, u^n) at n = 0, seg, 2 seg, ... into ck. */
static void forward(const shot_t *S, double *d, int seg, double *ck) {
    size_t N = (size_t)S->NZ * S->NX;
    double *b0 = (double *)calloc(N, sizeof(double));
    double *b1 = (double *)calloc(N, sizeof(double));
    double *b2 = (double *)calloc(N, sizeof(double));
    double *uold = b0, *u = b1, *unew = b2;
    for (int n = 0; n < S->nt; n++) {
        if (ck && n % seg == 0) {
            size_t j = (size_t)(n / seg);
            memcpy(ck + (2 * j) * N, uold, N * sizeof(double));
            memcpy(ck + (2 * j + 1) * N, u, N * sizeof(double));
        }
        fwd_step(S, n, uold, u, unew, NULL);
        if (d)
            for (int r = 0; r < S->nrec; r++)
                d[(size_t)n * S->nrec + r] = unew[(size_t)S->rz[r] * S->NX + S->rx[r]];
        double *t = uold; uold = u; u = unew; unew = t;
    }
    free(b0); free(b1); free(b2);
}

/* Adjoint sweep.  Given residual-like data r[n][rec] (n = 0..nt-1, the
 * sample of u^{n+1}) and a recompute source for a^n, accumulates
 *   gext += sum_k (2 v dt^2/h^2) w a^{k-1} lambda^k. */
static void adjoint(const shot_t *S, const or_grid *g, const double *r, int seg,
                    const double *ck, double *gext) {
    size_t N = (size_t)S->NZ * S->NX;
    int nseg = (S->nt + seg - 1) / seg;
    double *abuf = (double *)malloc(sizeof(double) * N * (size_t)seg);
    double *l0 = (double *)calloc(N, sizeof(double));   /* lambda^k   */
    double *l1 = (double *)calloc(N, sizeof(double));   /* lambda^k+1 */
    double *l2 = (double *)calloc(N, sizeof(double));   /* lambda^k+2 */
    double *tmp = (double *)calloc(N, sizeof(double));
    double *f0 = (double *)malloc(sizeof(double) * N);
    double *f1 = (double *)malloc(sizeof(double) * N);
    double *f2 = (double *)malloc(sizeof(double) * N);
    double cg = 2.0 * g->dt * g->dt / (g->h * g->h);
    for (int js = nseg - 1; js >= 0; js--) {
        int n0 = js * seg;
        int n1 = n0 + seg < S->nt ? n0 + seg : S->nt;
        /* Recompute a^n for n in [n0, n1) from the checkpoint. */
        memcpy(f0, ck + (2 * (size_t)js) * N, N * sizeof(double));
        memcpy(f1, ck + (2 * (size_t)js + 1) * N, N * sizeof(double));
        double *uold = f0, *u = f1, *unew = f2;
        for (int n = n0; n < n1; n++) {
            fwd_step(S, n, uold, u, unew, abuf + (size_t)(n - n0) * N);
            double *t = uold; uold = u; u = unew; unew = t;
        }
        /* Backward over k = n1 .. n0+1. */
        for (int k = n1; k >= n0 + 1; k--) {
            for (size_t c = 0; c < N; c++) tmp[c] = S->kap[c] * S->w[c] * l1[c];
            for (int i = 0; i < S->NZ; i++) {
                for (int j = 0; j < S->NX; j++) {
                    size_t c = (size_t)i * S->NX + j;
                    double w = S->w[c];
                    l0[c] = 2.0 * w * l1[c] + lap(tmp, S->NZ, S->NX, i, j) - w * w * l2[c];
                }
            }
            for (int q = 0; q < S->nrec; q++)
                l0[(size_t)S->rz[q] * S->NX + S->rx[q]] += r[(size_t)(k - 1) * S->nrec + q];
            const double *a = abuf + (size_t)(k - 1 - n0) * N;
            for (size_t c = 0; c < N; c++) gext[c] += cg * S->v[c] * S->w[c] * a[c] * l0[c];
            double *t = l2; l2 = l1; l1 = l0; l0 = t;
        }
    }
    free(abuf); free(l0); free(l1); free(l2); free(tmp); free(f0); free(f1); free(f2);
}

static int seg_len(const shot_t *S, int seg) {
    if (seg > 0) return seg;
    /* Store everything when it is small, else use ~sqrt(nt) segments. */
    size_t N = (size_t)S->NZ * S->NX;
    if ((size_t)S->nt * N * sizeof(double) <= ((size_t)256 << 20)) return S->nt;
    int s = (int)ceil(sqrt((double)S->nt));
    return s < 1 ? 1 : s;
}

static size_t data_off(const or_geom *G, int s) {
    size_t o = 0;
    for (int k = 0; k < s; k++) o += (size_t)G->nt[k] * (size_t)(G->rec_off[k + 1] - G->rec_off[k]);
    return o;
}

/* ------------------------------------------------------------------------ */

void or_model_shots(const or_grid *g, const double *v, const or_geom *G, double *d) {
    int ns = G->n_shots;
#pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < ns; s++) {
        shot_t S;
        shot_init(&S, g, v, G, s);
        forward(&S, d + data_off(G, s), 1, NULL);
        shot_free(&S);
    }
}

/* Shared body of the gradient and of migration: per shot, forward pass with
 * checkpoints, then the adjoint sweep driven by r_all (packed like d). */
static void adjoint_all(const or_grid *g, const double *v, const or_geom *G, const double *r_all,
                        double *out, int seg) {
    int ns = G->n_shots;
    size_t P = (size_t)g->nz * g->nx;
    double *part = (double *)calloc(P * (size_t)ns, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < ns; s++) {
        shot_t S;
        shot_init(&S, g, v, G, s);
        size_t N = (size_t)S.NZ * S.NX;
        int sl = seg_len(&S, seg);
        int nseg = (S.nt + sl - 1) / sl;
        double *ck = (double *)malloc(sizeof(double) * N * 2 * (size_t)nseg);
        forward(&S, NULL, sl, ck);
        double *gext = (double *)calloc(N, sizeof(double));
        adjoint(&S, g, r_all + data_off(G, s), sl, ck, gext);
        fold_add(&S, g, gext, part + (size_t)s * P);
        free(gext); free(ck);
        shot_free(&S);
    }
    for (size_t c = 0; c < P; c++) out[c] = 0.0;
    for (int s = 0; s < ns; s++)
        for (size_t c = 0; c < P; c++) out[c] += part[(size_t)s * P + c];
    free(part);
}

double or_fwi_gradient(const or_grid *g, const double *v, const or_geom *G, const double *d_obs,
                       double *grad, double *d_syn, int seg) {
    size_t nd = data_off(G, G->n_shots);
    double *ds = (double *)malloc(sizeof(double) * (nd > 0 ? nd : 1));
    or_model_shots(g, v, G, ds);
    double J = 0.0;
    for (size_t i = 0; i < nd; i++) {
        ds[i] = ds[i] - d_obs[i];  /* residual r = d_s - d_o */
    }
    for (size_t i = 0; i < nd; i++) J += 0.5 * ds[i] * ds[i];
    adjoint_all(g, v, G, ds, grad, seg);
    if (d_syn)
        for (size_t i = 0; i < nd; i++) d_syn[i] = ds[i] + d_obs[i];
    free(ds);
    return J;
}

void or_rtm_mig(const or_grid *g, const double *v0, const or_geom *G, const double *d,
                double *img, int seg) {
    adjoint_all(g, v0, G, d, img, seg);
}

void or_born_demig(const or_grid *g, const double *v0, const or_geom *G, const double *dv,
                   double *d) {
    int ns = G->n_shots;
    double cg = 2.0 * g->dt * g->dt / (g->h * g->h);
#pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < ns; s++) {
        shot_t S;
        shot_init(&S, g, v0, G, s);
        size_t N = (size_t)S.NZ * S.NX;
        double *dve = (double *)malloc(sizeof(double) * N);
        extend(&S, g, dv, dve);
        double *B[6];
        for (int k = 0; k < 6; k++) B[k] = (double *)calloc(N, sizeof(double));
        double *uold = B[0], *u = B[1], *unew = B[2];
        double *pold = B[3], *p = B[4], *pnew = B[5];
        double *dd = d + data_off(G, s);
        for (int n = 0; n < S.nt; n++) {
            for (int i = 0; i < S.NZ; i++) {
                for (int j = 0; j < S.NX; j++) {
                    size_t c = (size_t)i * S.NX + j;
                    double a0 = lap(u, S.NZ, S.NX, i, j);
                    if (i == S.sz && j == S.sx) a0 += S.wav[n];
                    double w = S.w[c];
                    unew[c] = w * (2.0 * u[c] + S.kap[c] * a0) - w * w * uold[c];
                    double dk = cg * S.v[c] * dve[c];  /* d kappa = 2 v dt^2/h^2 dv */
                    pnew[c] = w * (2.0 * p[c] + S.kap[c] * lap(p, S.NZ, S.NX, i, j) + dk * a0) -
                              w * w * pold[c];
                }
            }
            for (int r = 0; r < S.nrec; r++)
                dd[(size_t)n * S.nrec + r] = pnew[(size_t)S.rz[r] * S.NX + S.rx[r]];
            double *t = uold; uold = u; u = unew; unew = t;
            t = pold; pold = p; p = pnew; pnew = t;
        }
        for (int k = 0; k < 6; k++) free(B[k]);
        free(dve);
        shot_free(&S);
    }
}

/* Single-step helpers exposed for the stencil pins. */
void or_apply_lap(int NZ, int NX, const double *u, double *out) {
    for (int i = 0; i < NZ; i++)
        for (int j = 0; j < NX; j++) out[(size_t)i * NX + j] = lap(u, NZ, NX, i, j);
}

void or_sponge(const or_grid *g, int win_w, double *w_out) {
    int NZ = g->nz + 2 * g->nb, NX = win_w + 2 * g->nb;
    for (int i = 0; i < NZ; i++) {
        int dz = i < NZ - 1 - i ? i : NZ - 1 - i;
        for (int j = 0; j < NX; j++) {
            int dx = j < NX - 1 - j ? j : NX - 1 - j;
            w_out[(size_t)i * NX + j] = cerjan(dz, g->nb) * cerjan(dx, g->nb);
        }
    }
}
