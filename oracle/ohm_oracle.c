/*
 * ohm_oracle.c -- TEST INFRASTRUCTURE ONLY (the oracle).
 *
 * A plain, slow, FP64 CPU reference for one theta-scheme (Crank-Nicolson at lambda = 1/2)
 * step of the ohmic dissipation equation dB/dt = -curl(eta curl B) on a block-structured
 * AMR hierarchy, following T. Matsumoto (2011), "An Implicit Scheme for Ohmic Dissipation
 * with Adaptive Mesh Refinement", Sec. 2.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file; the CUDA solver library shares no code
 * with it and never calls it.
 *
 * Storage is deliberately different from the GPU path: every grid is addressed by global
 * cell indices through one accessor (at()) that wraps periodically and, for a cell the
 * level does not have, interpolates from the parent level.  The base grid and its
 * coarsenings are dense arrays; refined levels store their present 8^3 blocks behind a
 * block-position lookup.  No halos, no neighbour tables.
 *
 * What is computed (paper passages in brackets):
 *   face fluxes F_x, F_y, F_z                       [Sec. 2.1, Eqs. 4-6]
 *   normal / transverse face derivatives            [Sec. 2.1, Eqs. 9-10]
 *   face resistivity, arithmetic mean               [Sec. 2.1, Eq. 11]
 *   flux divergence                                 [Sec. 2.1, Eq. 8]
 *   L B = B + lambda dt div F,  S = b - (1-lambda) dt div f    [Eqs. 7, 12-14]
 *   defect correction R = S - L B, B += MG(0, R)    [Sec. 2.2, Eqs. 16-18]
 *   red-black Gauss-Seidel, B_c += R_c / (1 + alpha_c)          [Sec. 2.3, Eqs. 19-23]
 *   averaging restriction and (trilinear) prolongation per component   [Sec. 2.2]
 *   refluxing: a coarse face flux at a coarse-fine interface is the mean of the four fine
 *   face fluxes that tile it (conserves magnetic flux)          [Sec. 4]
 *   one synchronous dt on every level                           [Sec. 2.4]
 *   explicit predictor-corrector step (reference for Sec. 3.3 comparisons)
 *
 * Readings where the paper is silent (the same readings the solver follows):
 *   - red-black: colour = parity of (i+j+k) in level-global indices; within one colour pass
 *     every update is computed from the pre-pass state (Jacobi within a colour), all three
 *     components together;
 *   - multigrid: a correction-scheme V(nu1,nu2) cycle over the AMR levels (homogeneous
 *     coarse-fine ghosts on the way down, ghosts interpolated from the coarser correction
 *     on the way up) and then over the base grid coarsened by 2 while every dimension is
 *     even and stays >= 2; n_coarse colour sweeps on the coarsest grid;
 *   - coarse operator: the same discretisation with h_c = 2h and eta_c = mean of the 8
 *     children; restriction = mean of 8 children; prolongation = trilinear (27,9,3,1)/64;
 *   - coarse-fine ghost: tri-quadratic interpolation from the parent's 3x3x3 coarse
 *     neighbourhood (exact for quadratics, so the interface truncation error is O(h));
 *   - covered coarse cells hold the mean of their 8 children (they are not unknowns);
 *   - convergence: ||R||_2 / ||S||_2 over leaf cells weighted by cell volume.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define BS 8
#define MAXL 8
#define MAXM 24

typedef struct {
    int n[3];                 /* cells per axis */
    int nb[3];                /* 8^3 blocks per axis (AMR levels) */
    double h;                 /* cell width */
    int full;                 /* 1: every cell present */
    unsigned char *present;   /* per block, AMR levels only */
    unsigned char *covered;   /* per block, AMR levels only */
    int *bid;                 /* refined levels: storage index of each block position, -1 absent */
    long nblk;                /* refined levels: blocks stored */
    int nchunk;               /* loop chunks: blocks (AMR) or z-planes (coarse grids) */
    int (*chunk)[6];          /* lo[3], hi[3] */
    /* dense arrays over the level domain; 3 components unless noted */
    double *B, *S, *R;        /* composite state (AMR levels) */
    double *e, *r, *t, *d;    /* multigrid correction, right-hand side, scratch, deltas */
    double *eta;              /* 1 component */
} grid_t;

typedef struct orc_hier {
    int nlev;                 /* AMR levels */
    grid_t lev[MAXL];
    int nmg;                  /* base multigrid grids, mg[0] is lev[0] */
    grid_t *mg[MAXM];
    grid_t mgown[MAXM];
    long nblocks;
    int32_t *blk;             /* level, bi, bj, bk per user block */
    double lambda;
} orc_hier;

/* ------------------------------------------------------------------ indexing */
static inline int wrapi(int i, int n) { i %= n; return i < 0 ? i + n : i; }
static inline long ncell(const grid_t *g) { return (long)g->n[0] * g->n[1] * g->n[2]; }
static inline long bidx(const grid_t *g, int i, int j, int k) {
    return ((long)(k / BS) * g->nb[1] + (j / BS)) * g->nb[0] + (i / BS);
}
/* Storage index of component c at cell (i,j,k): dense [c][z][y][x] for the base grid and
 * its coarsenings; [c][block][8][8][8] over the present blocks for refined levels. */
static inline long cidx(const grid_t *g, int c, int i, int j, int k) {
    if (g->bid)
        return (((long)c * g->nblk + g->bid[bidx(g, i, j, k)]) * BS + (k % BS)) * BS * BS + (j % BS) * BS + (i % BS);
    return (((long)c * g->n[2] + k) * g->n[1] + j) * g->n[0] + i;
}
static inline long nstore(const grid_t *g) { return g->bid ? g->nblk * BS * BS * BS : ncell(g); }
static inline int is_present(const grid_t *g, int i, int j, int k) {
    return g->full || g->present[bidx(g, i, j, k)];
}
static inline int is_covered(const grid_t *g, int i, int j, int k) {
    return g->covered ? g->covered[bidx(g, i, j, k)] : 0;
}

/* A field on one grid, with the coarser grid used for missing cells.
 * fc == NULL with C != NULL means homogeneous (zero) coarse-fine ghosts. */
typedef struct {
    const grid_t *g; const double *f;
    const grid_t *C; const double *fc;
} view_t;

static double coarse_at(const grid_t *C, const double *fc, int c, int i, int j, int k) {
    i = wrapi(i, C->n[0]); j = wrapi(j, C->n[1]); k = wrapi(k, C->n[2]);
    if (!is_present(C, i, j, k)) {
        fprintf(stderr, "oracle: coarse cell (%d,%d,%d) missing: hierarchy not properly nested\n", i, j, k);
        abort();
    }
    return fc[cidx(C, c, i, j, k)];
}

/* Component c of the field at cell (i,j,k) of the view's grid (periodic).  A cell that the
 * grid does not have is a coarse-fine ghost: the tri-quadratic Taylor interpolant of the
 * parent's 3x3x3 neighbourhood evaluated at the child's centre, offset s_d h_c/4 per axis:
 *   f0 + sum_d [ s_d (f+d - f-d)/8 + (f+d - 2 f0 + f-d)/32 ]
 *      + sum_{d<e} s_d s_e (f(+d+e) - f(+d-e) - f(-d+e) + f(-d-e))/64,
 * exact for quadratic data. */
static double at(const view_t *v, int c, int i, int j, int k) {
    const grid_t *g = v->g;
    i = wrapi(i, g->n[0]); j = wrapi(j, g->n[1]); k = wrapi(k, g->n[2]);
    if (is_present(g, i, j, k)) return v->f[cidx(g, c, i, j, k)];
    if (!v->C) { fprintf(stderr, "oracle: missing cell without a coarser grid\n"); abort(); }
    if (!v->fc) return 0.0;
    const grid_t *C = v->C;
    const double *fc = v->fc;
    int p[3] = {i / 2, j / 2, k / 2};
    double s[3] = {(i & 1) ? 1.0 : -1.0, (j & 1) ? 1.0 : -1.0, (k & 1) ? 1.0 : -1.0};
    double f0 = coarse_at(C, fc, c, p[0], p[1], p[2]);
    double val = f0;
    for (int d = 0; d < 3; d++) {
        int a[3] = {p[0], p[1], p[2]}, b[3] = {p[0], p[1], p[2]};
        a[d] += 1; b[d] -= 1;
        double fp = coarse_at(C, fc, c, a[0], a[1], a[2]), fm = coarse_at(C, fc, c, b[0], b[1], b[2]);
        val += s[d] * (fp - fm) / 8.0 + (fp - 2.0 * f0 + fm) / 32.0;
    }
    for (int d = 0; d < 3; d++)
        for (int e = d + 1; e < 3; e++) {
            double x4 = 0.0;
            for (int sd = -1; sd <= 1; sd += 2)
                for (int se = -1; se <= 1; se += 2) {
                    int q[3] = {p[0], p[1], p[2]};
                    q[d] += sd; q[e] += se;
                    x4 += (double)(sd * se) * coarse_at(C, fc, c, q[0], q[1], q[2]);
                }
            val += s[d] * s[e] * x4 / 64.0;
        }
    return val;
}

static inline double atv(const view_t *v, int c, const int x[3]) { return at(v, c, x[0], x[1], x[2]); }

/* ------------------------------------------------------------------ Eqs. 4-11 */
/* Flux F_a through the face between cell x and x + e_a.  For each component b != a,
 * F_a^b = eta_f ( -d_a B_b + d_b B_a )                          (Eqs. 4-6)
 * with d_a B_b the two-point normal difference across the face  (Eq. 9),
 * d_b B_a the four-point transverse difference straddling it    (Eq. 10),
 * and eta_f the arithmetic mean of the two cells' eta           (Eq. 11).
 * F_a^a = 0. */
static void face_flux(const view_t *B, const view_t *E, int a, const int x[3], double F[3]) {
    const double h = B->g->h;
    int xa[3] = {x[0], x[1], x[2]};
    xa[a] += 1;
    double eta_f = 0.5 * (atv(E, 0, x) + atv(E, 0, xa));
    F[a] = 0.0;
    for (int b = 0; b < 3; b++) {
        if (b == a) continue;
        double d_normal = (atv(B, b, xa) - atv(B, b, x)) / h;
        int p1[3] = {xa[0], xa[1], xa[2]}, p2[3] = {x[0], x[1], x[2]};
        int m1[3] = {xa[0], xa[1], xa[2]}, m2[3] = {x[0], x[1], x[2]};
        p1[b] += 1; p2[b] += 1; m1[b] -= 1; m2[b] -= 1;
        double d_trans = (atv(B, a, p1) + atv(B, a, p2) - atv(B, a, m1) - atv(B, a, m2)) / (4.0 * h);
        F[b] = eta_f * (-d_normal + d_trans);
    }
}

/* (div F)(x) on one grid, every face at this grid's resolution (Eq. 8). */
static void div_level(const view_t *B, const view_t *E, const int x[3], double div[3]) {
    const double h = B->g->h;
    div[0] = div[1] = div[2] = 0.0;
    for (int a = 0; a < 3; a++) {
        double Fp[3], Fm[3];
        int xm[3] = {x[0], x[1], x[2]};
        xm[a] -= 1;
        face_flux(B, E, a, x, Fp);
        face_flux(B, E, a, xm, Fm);
        for (int c = 0; c < 3; c++) div[c] += (Fp[c] - Fm[c]) / h;
    }
}

/* ------------------------------------------------------------------ composite operator */
static view_t state_view(orc_hier *H, int l, double *const *f) {
    view_t v = {&H->lev[l], f[l], l > 0 ? &H->lev[l - 1] : NULL, l > 0 ? f[l - 1] : NULL};
    return v;
}
static view_t eta_view(orc_hier *H, int l) {
    view_t v = {&H->lev[l], H->lev[l].eta, l > 0 ? &H->lev[l - 1] : NULL, l > 0 ? H->lev[l - 1].eta : NULL};
    return v;
}

/* Mean of the four level-(l+1) face fluxes tiling the level-l face whose high-side cell is
 * xh along axis a (refluxing, Sec. 4). */
static void reflux_flux(orc_hier *H, double *const *f, int l, int a, const int xh[3], double F[3]) {
    view_t Bf = state_view(H, l + 1, f), Ef = eta_view(H, l + 1);
    const grid_t *gc = &H->lev[l];
    int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
    F[0] = F[1] = F[2] = 0.0;
    for (int o1 = 0; o1 < 2; o1++)
        for (int o2 = 0; o2 < 2; o2++) {
            int lo[3];
            lo[a] = 2 * wrapi(xh[a], gc->n[a]) - 1;
            lo[b1] = 2 * wrapi(xh[b1], gc->n[b1]) + o1;
            lo[b2] = 2 * wrapi(xh[b2], gc->n[b2]) + o2;
            double Ff[3];
            face_flux(&Bf, &Ef, a, lo, Ff);
            for (int c = 0; c < 3; c++) F[c] += 0.25 * Ff[c];
        }
}

/* Composite (div F)(x) at a leaf cell of AMR level l: faces whose neighbour cell is covered
 * by level l+1 take the refluxed fine flux, all others the level-l flux. */
static void div_composite(orc_hier *H, double *const *f, int l, const int x[3], double div[3]) {
    const grid_t *g = &H->lev[l];
    view_t B = state_view(H, l, f), E = eta_view(H, l);
    div[0] = div[1] = div[2] = 0.0;
    for (int a = 0; a < 3; a++) {
        double Fp[3], Fm[3];
        int xp[3] = {x[0], x[1], x[2]}, xm[3] = {x[0], x[1], x[2]};
        xp[a] += 1; xm[a] -= 1;
        int cp = l + 1 < H->nlev && is_covered(g, wrapi(xp[0], g->n[0]), wrapi(xp[1], g->n[1]), wrapi(xp[2], g->n[2]));
        int cm = l + 1 < H->nlev && is_covered(g, wrapi(xm[0], g->n[0]), wrapi(xm[1], g->n[1]), wrapi(xm[2], g->n[2]));
        if (cp) reflux_flux(H, f, l, a, xp, Fp); else face_flux(&B, &E, a, x, Fp);
        if (cm) reflux_flux(H, f, l, a, x, Fm); else face_flux(&B, &E, a, xm, Fm);
        for (int c = 0; c < 3; c++) div[c] += (Fp[c] - Fm[c]) / g->h;
    }
}

#define FOR_CHUNK_CELLS(g, ch, x)                                           \
    for (int x##k = (g)->chunk[ch][2]; x##k < (g)->chunk[ch][5]; x##k++)    \
        for (int x##j = (g)->chunk[ch][1]; x##j < (g)->chunk[ch][4]; x##j++) \
            for (int x##i = (g)->chunk[ch][0]; x##i < (g)->chunk[ch][3]; x##i++)

static inline int chunk_is_leaf(const grid_t *g, int ch) {
    return !g->covered || !g->covered[bidx(g, g->chunk[ch][0], g->chunk[ch][1], g->chunk[ch][2])];
}

/* Covered cells := mean of their 8 children, finest level first. */
static void sync_down(orc_hier *H, double *const *f) {
    for (int l = H->nlev - 2; l >= 0; l--) {
        grid_t *g = &H->lev[l];
        const grid_t *gf = &H->lev[l + 1];
        double *fc = f[l];
        const double *ff = f[l + 1];
#pragma omp parallel for schedule(static)
        for (int ch = 0; ch < g->nchunk; ch++) {
            if (chunk_is_leaf(g, ch)) continue;
            FOR_CHUNK_CELLS(g, ch, x) {
                for (int c = 0; c < 3; c++) {
                    double s = 0.0;
                    for (int dk = 0; dk < 2; dk++) for (int dj = 0; dj < 2; dj++) for (int di = 0; di < 2; di++)
                        s += ff[cidx(gf, c, 2 * xi + di, 2 * xj + dj, 2 * xk + dk)];
                    fc[cidx(g, c, xi, xj, xk)] = s / 8.0;
                }
            }
        }
    }
}

/* out = a*X + cdiv*(div F)(X) + cy*Y on every leaf cell (X synced first by the caller). */
static void composite_apply(orc_hier *H, double *const *X, double a, double cdiv, double cy,
                            double *const *Y, double *const *out) {
    for (int l = 0; l < H->nlev; l++) {
        grid_t *g = &H->lev[l];
#pragma omp parallel for schedule(dynamic, 4)
        for (int ch = 0; ch < g->nchunk; ch++) {
            if (!chunk_is_leaf(g, ch)) {
                FOR_CHUNK_CELLS(g, ch, x) for (int c = 0; c < 3; c++) out[l][cidx(g, c, xi, xj, xk)] = 0.0;
                continue;
            }
            FOR_CHUNK_CELLS(g, ch, x) {
                int xv[3] = {xi, xj, xk};
                double div[3];
                div_composite(H, X, l, xv, div);
                for (int c = 0; c < 3; c++) {
                    long id = cidx(g, c, xi, xj, xk);
                    out[l][id] = a * X[l][id] + cdiv * div[c] + (Y ? cy * Y[l][id] : 0.0);
                }
            }
        }
    }
}

/* sum over leaf cells of R^2 dV, S^2 dV and max |R| */
static void leaf_norms(orc_hier *H, double *const *R, double *const *S, double out[3]) {
    double sr = 0, ss = 0, mx = 0;
    for (int l = 0; l < H->nlev; l++) {
        grid_t *g = &H->lev[l];
        double dv = g->h * g->h * g->h;
        double *pr = calloc(g->nchunk, sizeof(double)), *ps = calloc(g->nchunk, sizeof(double)),
               *pm = calloc(g->nchunk, sizeof(double));
#pragma omp parallel for schedule(static)
        for (int ch = 0; ch < g->nchunk; ch++) {
            if (!chunk_is_leaf(g, ch)) continue;
            double a = 0, b = 0, m = 0;
            FOR_CHUNK_CELLS(g, ch, x) for (int c = 0; c < 3; c++) {
                long id = cidx(g, c, xi, xj, xk);
                a += R[l][id] * R[l][id];
                if (S) b += S[l][id] * S[l][id];
                if (fabs(R[l][id]) > m) m = fabs(R[l][id]);
            }
            pr[ch] = a; ps[ch] = b; pm[ch] = m;
        }
        for (int ch = 0; ch < g->nchunk; ch++) {
            sr += pr[ch] * dv; ss += ps[ch] * dv;
            if (pm[ch] > mx) mx = pm[ch];
        }
        free(pr); free(ps); free(pm);
    }
    out[0] = sr; out[1] = ss; out[2] = mx;
}

/* ------------------------------------------------------------------ multigrid pieces */
/* alpha_c = lambda dt sum over the two axes a != c of (eta_{-1/2} + eta_{+1/2}) / h^2
 * (Eqs. 21-23), face eta by Eq. 11. */
static void alphas(const view_t *E, double lamdt, const int x[3], double al[3]) {
    const double h2 = E->g->h * E->g->h;
    double e0 = atv(E, 0, x), s[3];
    for (int a = 0; a < 3; a++) {
        int p[3] = {x[0], x[1], x[2]}, m[3] = {x[0], x[1], x[2]};
        p[a] += 1; m[a] -= 1;
        s[a] = 0.5 * (e0 + atv(E, 0, p)) + 0.5 * (e0 + atv(E, 0, m));
    }
    for (int c = 0; c < 3; c++) {
        al[c] = 0.0;
        for (int a = 0; a < 3; a++) if (a != c) al[c] += lamdt * s[a] / h2;
    }
}

/* One colour pass of red-black Gauss-Seidel on grid g (Eq. 19 with Eq. 20):
 * for cells with (i+j+k) % 2 == colour, e_c += (r - L e)_c / (1 + alpha_c), all deltas
 * computed from the pre-pass state, then applied. */
static void smooth_pass(grid_t *g, const view_t *ev, const view_t *E, double lamdt, int colour) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int ch = 0; ch < g->nchunk; ch++) {
        FOR_CHUNK_CELLS(g, ch, x) {
            if (((xi + xj + xk) & 1) != colour) continue;
            int xv[3] = {xi, xj, xk};
            double div[3], al[3];
            div_level(ev, E, xv, div);
            alphas(E, lamdt, xv, al);
            for (int c = 0; c < 3; c++) {
                long id = cidx(g, c, xi, xj, xk);
                double res = g->r[id] - (g->e[id] + lamdt * div[c]);
                g->d[id] = res / (1.0 + al[c]);
            }
        }
    }
#pragma omp parallel for schedule(static)
    for (int ch = 0; ch < g->nchunk; ch++) {
        FOR_CHUNK_CELLS(g, ch, x) {
            if (((xi + xj + xk) & 1) != colour) continue;
            for (int c = 0; c < 3; c++) g->e[cidx(g, c, xi, xj, xk)] += g->d[cidx(g, c, xi, xj, xk)];
        }
    }
}

/* t = r - (e + lamdt div F(e)) on every cell of the grid */
static void level_residual(grid_t *g, const view_t *ev, const view_t *E, double lamdt) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int ch = 0; ch < g->nchunk; ch++) {
        FOR_CHUNK_CELLS(g, ch, x) {
            int xv[3] = {xi, xj, xk};
            double div[3];
            div_level(ev, E, xv, div);
            for (int c = 0; c < 3; c++) {
                long id = cidx(g, c, xi, xj, xk);
                g->t[id] = g->r[id] - (g->e[id] + lamdt * div[c]);
            }
        }
    }
}

/* coarse(p) = mean of the 8 fine children, for the coarse cells that have children
 * (all of them for a full coarse grid, covered cells for an AMR level). */
static void restrict_to(const grid_t *gf, const double *ff, grid_t *gc, double *fc, int ncomp) {
#pragma omp parallel for schedule(static)
    for (int ch = 0; ch < gc->nchunk; ch++) {
        if (gc->covered && chunk_is_leaf(gc, ch)) continue;
        FOR_CHUNK_CELLS(gc, ch, x) for (int c = 0; c < ncomp; c++) {
            double s = 0.0;
            for (int dk = 0; dk < 2; dk++) for (int dj = 0; dj < 2; dj++) for (int di = 0; di < 2; di++)
                s += ff[cidx(gf, c, 2 * xi + di, 2 * xj + dj, 2 * xk + dk)];
            fc[cidx(gc, c, xi, xj, xk)] = s / 8.0;
        }
    }
}

/* fine += trilinear interpolation of the coarse field: weights 3/4 (own parent) and 1/4
 * (the neighbour on the child's side) per axis, i.e. 27/64, 9/64, 3/64, 1/64. */
static void prolong_add(const grid_t *gc, const double *fc, grid_t *gf, double *ff) {
#pragma omp parallel for schedule(static)
    for (int ch = 0; ch < gf->nchunk; ch++) {
        FOR_CHUNK_CELLS(gf, ch, x) for (int c = 0; c < 3; c++) {
            int p[3] = {xi / 2, xj / 2, xk / 2};
            int s[3] = {(xi & 1) ? 1 : -1, (xj & 1) ? 1 : -1, (xk & 1) ? 1 : -1};
            double v = 0.0;
            for (int ak = 0; ak < 2; ak++) for (int aj = 0; aj < 2; aj++) for (int ai = 0; ai < 2; ai++) {
                double w = (ai ? 0.25 : 0.75) * (aj ? 0.25 : 0.75) * (ak ? 0.25 : 0.75);
                v += w * coarse_at(gc, fc, c, p[0] + ai * s[0], p[1] + aj * s[1], p[2] + ak * s[2]);
            }
            ff[cidx(gf, c, xi, xj, xk)] += v;
        }
    }
}

static void zero_present(grid_t *g, double *f, int ncomp) {
#pragma omp parallel for schedule(static)
    for (int ch = 0; ch < g->nchunk; ch++)
        FOR_CHUNK_CELLS(g, ch, x) for (int c = 0; c < ncomp; c++) f[cidx(g, c, xi, xj, xk)] = 0.0;
}

typedef struct { int nu_pre, nu_post, n_coarse; } mgpar_t;

/* V-cycle on the base grid hierarchy, level m, e_m = 0 on entry (Sec. 2.2). */
static void base_vcycle(orc_hier *H, int m, double lamdt, const mgpar_t *P) {
    grid_t *g = H->mg[m];
    view_t ev = {g, g->e, NULL, NULL}, E = {g, g->eta, NULL, NULL};
    double ld = lamdt;
    if (m == H->nmg - 1) {
        for (int s = 0; s < P->n_coarse; s++) { smooth_pass(g, &ev, &E, ld, 0); smooth_pass(g, &ev, &E, ld, 1); }
        return;
    }
    for (int s = 0; s < P->nu_pre; s++) { smooth_pass(g, &ev, &E, ld, 0); smooth_pass(g, &ev, &E, ld, 1); }
    level_residual(g, &ev, &E, ld);
    grid_t *gc = H->mg[m + 1];
    restrict_to(g, g->t, gc, gc->r, 3);
    zero_present(gc, gc->e, 3);
    base_vcycle(H, m + 1, lamdt, P);
    prolong_add(gc, gc->e, g, g->e);
    for (int s = 0; s < P->nu_post; s++) { smooth_pass(g, &ev, &E, ld, 0); smooth_pass(g, &ev, &E, ld, 1); }
}

/* One correction-scheme V-cycle over the AMR levels and the base grid: returns the
 * correction in lev[l].e for the composite residual held in lev[l].R (leaf cells). */
static void amr_vcycle(orc_hier *H, double lamdt, const mgpar_t *P) {
    for (int l = H->nlev - 1; l >= 1; l--) {
        grid_t *g = &H->lev[l];
        /* leaf cells take the composite residual; covered cells were restricted from l+1 */
#pragma omp parallel for schedule(static)
        for (int ch = 0; ch < g->nchunk; ch++) {
            if (!chunk_is_leaf(g, ch)) continue;
            FOR_CHUNK_CELLS(g, ch, x) for (int c = 0; c < 3; c++) g->r[cidx(g, c, xi, xj, xk)] = g->R[cidx(g, c, xi, xj, xk)];
        }
        zero_present(g, g->e, 3);
        view_t ev = {g, g->e, &H->lev[l - 1], NULL};   /* homogeneous coarse-fine ghosts */
        view_t E = eta_view(H, l);
        for (int s = 0; s < P->nu_pre; s++) { smooth_pass(g, &ev, &E, lamdt, 0); smooth_pass(g, &ev, &E, lamdt, 1); }
        level_residual(g, &ev, &E, lamdt);
        restrict_to(g, g->t, &H->lev[l - 1], H->lev[l - 1].r, 3);
    }
    grid_t *g0 = &H->lev[0];
#pragma omp parallel for schedule(static)
    for (int ch = 0; ch < g0->nchunk; ch++) {
        if (!chunk_is_leaf(g0, ch)) continue;
        FOR_CHUNK_CELLS(g0, ch, x) for (int c = 0; c < 3; c++) g0->r[cidx(g0, c, xi, xj, xk)] = g0->R[cidx(g0, c, xi, xj, xk)];
    }
    zero_present(g0, g0->e, 3);
    base_vcycle(H, 0, lamdt, P);
    for (int l = 1; l < H->nlev; l++) {
        grid_t *g = &H->lev[l];
        prolong_add(&H->lev[l - 1], H->lev[l - 1].e, g, g->e);
        view_t ev = {g, g->e, &H->lev[l - 1], H->lev[l - 1].e};
        view_t E = eta_view(H, l);
        for (int s = 0; s < P->nu_post; s++) { smooth_pass(g, &ev, &E, lamdt, 0); smooth_pass(g, &ev, &E, lamdt, 1); }
    }
}

/* ------------------------------------------------------------------ setup */
static int alloc_grid(grid_t *g, int amr) {
    long n = nstore(g);
    g->e = calloc(3 * n, sizeof(double)); g->r = calloc(3 * n, sizeof(double));
    g->t = calloc(3 * n, sizeof(double)); g->d = calloc(3 * n, sizeof(double));
    g->eta = calloc(n, sizeof(double));
    if (amr) {
        g->B = calloc(3 * n, sizeof(double)); g->S = calloc(3 * n, sizeof(double));
        g->R = calloc(3 * n, sizeof(double));
        if (!g->B || !g->S || !g->R) return -1;
    }
    return (g->e && g->r && g->t && g->d && g->eta) ? 0 : -1;
}

static void free_grid(grid_t *g) {
    free(g->e); free(g->r); free(g->t); free(g->d); free(g->eta);
    free(g->B); free(g->S); free(g->R); free(g->present); free(g->covered); free(g->chunk); free(g->bid);
}

void orc_destroy(orc_hier *H) {
    if (!H) return;
    for (int l = 0; l < H->nlev; l++) free_grid(&H->lev[l]);
    for (int m = 1; m < H->nmg; m++) free_grid(&H->mgown[m]);
    free(H->blk);
    free(H);
}

#define FAIL(...) do { if (err) snprintf(err, errlen, __VA_ARGS__); orc_destroy(H); return NULL; } while (0)

orc_hier *orc_create(int nx, int ny, int nz, double dx0, int nlev, long nblocks, const int32_t *lijk,
                     double lambda, char *err, int errlen) {
    orc_hier *H = calloc(1, sizeof(orc_hier));
    if (!H) return NULL;
    if (nx <= 0 || ny <= 0 || nz <= 0 || nx % BS || ny % BS || nz % BS) FAIL("base cells must be positive multiples of 8");
    if (nlev < 1 || nlev > MAXL) FAIL("nlevels out of range");
    if (!(dx0 > 0)) FAIL("dx0 must be positive");
    H->nlev = nlev; H->lambda = lambda; H->nblocks = nblocks;
    H->blk = malloc(sizeof(int32_t) * 4 * (nblocks > 0 ? nblocks : 1));
    memcpy(H->blk, lijk, sizeof(int32_t) * 4 * nblocks);
    int base[3] = {nx, ny, nz};
    for (int l = 0; l < nlev; l++) {
        grid_t *g = &H->lev[l];
        for (int a = 0; a < 3; a++) { g->n[a] = base[a] << l; g->nb[a] = g->n[a] / BS; }
        g->h = dx0 / (double)(1 << l);
        g->full = 0;
        long nbk = (long)g->nb[0] * g->nb[1] * g->nb[2];
        g->present = calloc(nbk, 1); g->covered = calloc(nbk, 1);
        if (!g->present || !g->covered) FAIL("out of memory");
    }
    for (long b = 0; b < nblocks; b++) {
        int l = lijk[4 * b], bi = lijk[4 * b + 1], bj = lijk[4 * b + 2], bk = lijk[4 * b + 3];
        if (l < 0 || l >= nlev) FAIL("block %ld: level out of range", b);
        grid_t *g = &H->lev[l];
        if (bi < 0 || bj < 0 || bk < 0 || bi >= g->nb[0] || bj >= g->nb[1] || bk >= g->nb[2]) FAIL("block %ld out of range", b);
        long id = ((long)bk * g->nb[1] + bj) * g->nb[0] + bi;
        if (g->present[id]) FAIL("block %ld duplicated", b);
        g->present[id] = 1;
    }
    /* base level complete; octree: children of a refined block all present; nesting */
    {
        grid_t *g = &H->lev[0];
        for (long i = 0; i < (long)g->nb[0] * g->nb[1] * g->nb[2]; i++) if (!g->present[i]) FAIL("base level incomplete");
    }
    for (int l = 1; l < nlev; l++) {
        grid_t *g = &H->lev[l], *gp = &H->lev[l - 1];
        int any = 0;
        for (int bk = 0; bk < g->nb[2]; bk++) for (int bj = 0; bj < g->nb[1]; bj++) for (int bi = 0; bi < g->nb[0]; bi++) {
            if (!g->present[((long)bk * g->nb[1] + bj) * g->nb[0] + bi]) continue;
            any = 1;
            int pi = bi / 2, pj = bj / 2, pk = bk / 2;
            for (int c = 0; c < 8; c++) {
                int ci = 2 * pi + (c & 1), cj = 2 * pj + ((c >> 1) & 1), ck = 2 * pk + (c >> 2);
                if (!g->present[((long)ck * g->nb[1] + cj) * g->nb[0] + ci]) FAIL("level %d: incomplete octet", l);
            }
            for (int dk = -1; dk <= 1; dk++) for (int dj = -1; dj <= 1; dj++) for (int di = -1; di <= 1; di++) {
                int qi = wrapi(pi + di, gp->nb[0]), qj = wrapi(pj + dj, gp->nb[1]), qk = wrapi(pk + dk, gp->nb[2]);
                if (!gp->present[((long)qk * gp->nb[1] + qj) * gp->nb[0] + qi]) FAIL("level %d: not properly nested", l);
            }
            gp->covered[((long)pk * gp->nb[1] + pj) * gp->nb[0] + pi] = 1;
        }
        if (!any) FAIL("level %d has no blocks", l);
    }
    for (int l = 0; l < nlev; l++) {
        grid_t *g = &H->lev[l];
        long nbk = (long)g->nb[0] * g->nb[1] * g->nb[2];
        g->chunk = malloc(sizeof(*g->chunk) * nbk);
        g->nchunk = 0;
        if (l > 0) {
            g->bid = malloc(sizeof(int) * nbk);
            if (!g->bid) FAIL("out of memory");
            for (long q = 0; q < nbk; q++) g->bid[q] = -1;
        }
        for (int bk = 0; bk < g->nb[2]; bk++) for (int bj = 0; bj < g->nb[1]; bj++) for (int bi = 0; bi < g->nb[0]; bi++) {
            long pos = ((long)bk * g->nb[1] + bj) * g->nb[0] + bi;
            if (!g->present[pos]) continue;
            if (g->bid) g->bid[pos] = g->nchunk;
            int *c = g->chunk[g->nchunk++];
            c[0] = bi * BS; c[1] = bj * BS; c[2] = bk * BS; c[3] = c[0] + BS; c[4] = c[1] + BS; c[5] = c[2] + BS;
        }
        g->nblk = g->nchunk;
        if (alloc_grid(g, 1)) FAIL("out of memory");
    }
    H->lev[0].full = 1;
    /* base multigrid: halve while every dimension is even and the result stays >= 2 */
    H->mg[0] = &H->lev[0];
    H->nmg = 1;
    int n[3] = {nx, ny, nz};
    while (H->nmg < MAXM && n[0] % 2 == 0 && n[1] % 2 == 0 && n[2] % 2 == 0 && n[0] >= 4 && n[1] >= 4 && n[2] >= 4) {
        grid_t *g = &H->mgown[H->nmg];
        for (int a = 0; a < 3; a++) { n[a] /= 2; g->n[a] = n[a]; g->nb[a] = 0; }
        g->h = H->mg[H->nmg - 1]->h * 2.0;
        g->full = 1;
        g->nchunk = n[2];
        g->chunk = malloc(sizeof(*g->chunk) * n[2]);
        for (int k = 0; k < n[2]; k++) {
            int *c = g->chunk[k];
            c[0] = 0; c[1] = 0; c[2] = k; c[3] = n[0]; c[4] = n[1]; c[5] = k + 1;
        }
        if (alloc_grid(g, 0)) FAIL("out of memory");
        H->mg[H->nmg++] = g;
    }
    return H;
}

int orc_nmg(const orc_hier *H) { return H->nmg; }
int orc_mg_dims(const orc_hier *H, int m, int *dims) {
    if (m < 0 || m >= H->nmg) return -1;
    for (int a = 0; a < 3; a++) dims[a] = H->mg[m]->n[a];
    return 0;
}

/* ------------------------------------------------------------------ user layout */
static void scatter(orc_hier *H, const double *user, int ncomp, int which) {
    for (long b = 0; b < H->nblocks; b++) {
        int l = H->blk[4 * b];
        grid_t *g = &H->lev[l];
        double *dst = which == 0 ? g->B : which == 1 ? g->S : which == 2 ? g->R : which == 3 ? g->eta : g->e;
        int o[3] = {H->blk[4 * b + 1] * BS, H->blk[4 * b + 2] * BS, H->blk[4 * b + 3] * BS};
        const double *src = user + (size_t)b * ncomp * BS * BS * BS;
        for (int c = 0; c < ncomp; c++) for (int k = 0; k < BS; k++) for (int j = 0; j < BS; j++) for (int i = 0; i < BS; i++)
            dst[cidx(g, c, o[0] + i, o[1] + j, o[2] + k)] = src[((c * BS + k) * BS + j) * BS + i];
    }
}

static void gather(orc_hier *H, double *user, int ncomp, int which) {
    for (long b = 0; b < H->nblocks; b++) {
        int l = H->blk[4 * b];
        grid_t *g = &H->lev[l];
        const double *src = which == 0 ? g->B : which == 1 ? g->S : which == 2 ? g->R : which == 3 ? g->eta : g->e;
        int o[3] = {H->blk[4 * b + 1] * BS, H->blk[4 * b + 2] * BS, H->blk[4 * b + 3] * BS};
        double *dst = user + (size_t)b * ncomp * BS * BS * BS;
        for (int c = 0; c < ncomp; c++) for (int k = 0; k < BS; k++) for (int j = 0; j < BS; j++) for (int i = 0; i < BS; i++)
            dst[((c * BS + k) * BS + j) * BS + i] = src[cidx(g, c, o[0] + i, o[1] + j, o[2] + k)];
    }
}

enum { W_B = 0, W_S = 1, W_R = 2, W_ETA = 3, W_E = 4 };

static double *const *arr(orc_hier *H, int which, double **tmp) {
    for (int l = 0; l < H->nlev; l++)
        tmp[l] = which == W_B ? H->lev[l].B : which == W_S ? H->lev[l].S : which == W_R ? H->lev[l].R : H->lev[l].e;
    return tmp;
}

/* eta on every block (covered blocks included); coarse multigrid eta = mean of children */
int orc_set_eta(orc_hier *H, const double *eta_user) {
    scatter(H, eta_user, 1, W_ETA);
    for (int m = 1; m < H->nmg; m++) restrict_to(H->mg[m - 1], H->mg[m - 1]->eta, H->mg[m], H->mg[m]->eta, 1);
    return 0;
}

/* the eta of base multigrid grid m (dense [z][y][x]) as derived by orc_set_eta */
int orc_mg_eta(const orc_hier *H, int m, double *out) {
    if (m < 0 || m >= H->nmg) return -1;
    memcpy(out, H->mg[m]->eta, sizeof(double) * ncell(H->mg[m]));
    return 0;
}

/* out = (div F)(B) on leaf cells, 0 on covered blocks; B synced first (Eq. 8 + refluxing) */
int orc_div_flux(orc_hier *H, const double *B_user, double *out_user) {
    double *tb[MAXL], *tr[MAXL];
    scatter(H, B_user, 3, W_B);
    sync_down(H, arr(H, W_B, tb));
    composite_apply(H, arr(H, W_B, tb), 0.0, 1.0, 0.0, NULL, arr(H, W_R, tr));
    gather(H, out_user, 3, W_R);
    return 0;
}

/* out = L B = B + lambda dt div F(B) on leaf cells (Eq. 13); 0 on covered blocks */
int orc_apply_L(orc_hier *H, const double *B_user, double dt, double *out_user) {
    double *tb[MAXL], *tr[MAXL];
    scatter(H, B_user, 3, W_B);
    sync_down(H, arr(H, W_B, tb));
    composite_apply(H, arr(H, W_B, tb), 1.0, H->lambda * dt, 0.0, NULL, arr(H, W_R, tr));
    gather(H, out_user, 3, W_R);
    return 0;
}

/* S = b - (1 - lambda) dt div f(b) on leaf cells (Eq. 14) */
int orc_source(orc_hier *H, const double *b_user, double dt, double *S_user) {
    double *tb[MAXL], *ts[MAXL];
    scatter(H, b_user, 3, W_B);
    sync_down(H, arr(H, W_B, tb));
    composite_apply(H, arr(H, W_B, tb), 1.0, -(1.0 - H->lambda) * dt, 0.0, NULL, arr(H, W_S, ts));
    gather(H, S_user, 3, W_S);
    return 0;
}

static void compute_residual(orc_hier *H, double dt, double norms[4]) {
    double *tb[MAXL], *ts[MAXL], *tr[MAXL], nr[3];
    composite_apply(H, arr(H, W_B, tb), -1.0, -H->lambda * dt, 1.0, arr(H, W_S, ts), arr(H, W_R, tr));
    leaf_norms(H, arr(H, W_R, tr), arr(H, W_S, ts), nr);
    norms[0] = nr[1] > 0 ? sqrt(nr[0] / nr[1]) : sqrt(nr[0]);
    norms[1] = nr[2]; norms[2] = sqrt(nr[0]); norms[3] = sqrt(nr[1]);
}

/* R = S - L B on leaf cells (Eq. 20); norms = {||R||/||S||, max|R|, ||R||, ||S||} */
int orc_residual(orc_hier *H, const double *B_user, const double *S_user, double dt, double *R_user, double *norms) {
    double *tb[MAXL];
    scatter(H, B_user, 3, W_B);
    scatter(H, S_user, 3, W_S);
    sync_down(H, arr(H, W_B, tb));
    compute_residual(H, dt, norms);
    if (R_user) gather(H, R_user, 3, W_R);
    return 0;
}

/* One AMR V-cycle from a zero guess for the residual R_user (leaf cells): e_user receives
 * the correction on leaf cells, 0 on covered blocks. */
int orc_vcycle(orc_hier *H, const double *R_user, double dt, const int *params, double *e_user) {
    mgpar_t P = {params[0], params[1], params[2]};
    scatter(H, R_user, 3, W_R);
    amr_vcycle(H, H->lambda * dt, &P);
    for (int l = 0; l < H->nlev; l++) {
        grid_t *g = &H->lev[l];
        for (int ch = 0; ch < g->nchunk; ch++)
            if (!chunk_is_leaf(g, ch)) FOR_CHUNK_CELLS(g, ch, x) for (int c = 0; c < 3; c++) g->e[cidx(g, c, xi, xj, xk)] = 0.0;
    }
    gather(H, e_user, 3, W_E);
    return 0;
}

/* One theta-scheme step (Eq. 7) solved by defect correction (Eqs. 16-18).
 * params = {nu_pre, nu_post, n_coarse, max_outer}.  tol < 0: run exactly max_outer cycles.
 * hist[0..n] receives ||R||/||S|| before each cycle and after the last; *ncycles the count.
 * Returns 0 when converged (or the fixed count ran), 1 when not converged. */
int orc_cn_step(orc_hier *H, double *B_user, double dt, double tol, const int *params, double *hist, int *ncycles) {
    mgpar_t P = {params[0], params[1], params[2]};
    int max_outer = params[3];
    double *tb[MAXL];
    double lamdt = H->lambda * dt;
    scatter(H, B_user, 3, W_B);
    sync_down(H, arr(H, W_B, tb));
    {   /* S from b */
        double *ts[MAXL];
        composite_apply(H, arr(H, W_B, tb), 1.0, -(1.0 - H->lambda) * dt, 0.0, NULL, arr(H, W_S, ts));
    }
    int it = 0, status = 1;
    for (;;) {
        double nr[4];
        compute_residual(H, dt, nr);
        if (hist) hist[it] = nr[0];
        if (tol >= 0 && nr[0] <= tol) { status = 0; break; }
        if (it >= max_outer) { status = tol >= 0 ? 1 : 0; break; }
        amr_vcycle(H, lamdt, &P);
        for (int l = 0; l < H->nlev; l++) {
            grid_t *g = &H->lev[l];
#pragma omp parallel for schedule(static)
            for (int ch = 0; ch < g->nchunk; ch++) {
                if (!chunk_is_leaf(g, ch)) continue;
                FOR_CHUNK_CELLS(g, ch, x) for (int c = 0; c < 3; c++) {
                    long id = cidx(g, c, xi, xj, xk);
                    g->B[id] += g->e[id];
                }
            }
        }
        sync_down(H, arr(H, W_B, tb));
        it++;
    }
    if (ncycles) *ncycles = it;
    gather(H, B_user, 3, W_B);
    return status;
}

/* Explicit predictor-corrector (Heun) step with the same fluxes:
 * B* = B - dt div F(B);  B_new = (B + B* - dt div F(B*)) / 2. */
int orc_heun_step(orc_hier *H, double *B_user, double dt) {
    double *tb[MAXL], *ts[MAXL], *tr[MAXL];
    scatter(H, B_user, 3, W_B);
    sync_down(H, arr(H, W_B, tb));
    composite_apply(H, arr(H, W_B, tb), 1.0, -dt, 0.0, NULL, arr(H, W_S, ts));   /* S := B* */
    sync_down(H, arr(H, W_S, ts));
    composite_apply(H, arr(H, W_S, ts), 1.0, -dt, 1.0, arr(H, W_B, tb), arr(H, W_R, tr));
    for (int l = 0; l < H->nlev; l++) {
        grid_t *g = &H->lev[l];
        long n = 3 * nstore(g);
        for (long i = 0; i < n; i++) g->B[i] = 0.5 * g->R[i];
    }
    sync_down(H, arr(H, W_B, tb));
    gather(H, B_user, 3, W_B);
    return 0;
}

void orc_sync_down(orc_hier *H, double *B_user) {
    double *tb[MAXL];
    scatter(H, B_user, 3, W_B);
    sync_down(H, arr(H, W_B, tb));
    gather(H, B_user, 3, W_B);
}

/* ------------------------------------------------------------------ single-grid pieces
 * For kernel-by-kernel parity on one uniform periodic grid: all arrays are dense
 * [comp][nz][ny][nx] on base multigrid grid m. */
static void load_dense(grid_t *g, double *dst, const double *src, int ncomp) {
    memcpy(dst, src, sizeof(double) * ncomp * ncell(g));
}

/* one colour pass on grid m: e (in/out), r, eta given */
int orc_grid_smooth(orc_hier *H, int m, double *e, const double *r, const double *eta, double dt, int colour) {
    if (m < 0 || m >= H->nmg) return -1;
    grid_t *g = H->mg[m];
    load_dense(g, g->e, e, 3); load_dense(g, g->r, r, 3); load_dense(g, g->eta, eta, 1);
    view_t ev = {g, g->e, NULL, NULL}, E = {g, g->eta, NULL, NULL};
    smooth_pass(g, &ev, &E, H->lambda * dt, colour);
    memcpy(e, g->e, sizeof(double) * 3 * ncell(g));
    return 0;
}

/* t = r - L e on grid m */
int orc_grid_residual(orc_hier *H, int m, const double *e, const double *r, const double *eta, double dt, double *t) {
    if (m < 0 || m >= H->nmg) return -1;
    grid_t *g = H->mg[m];
    load_dense(g, g->e, e, 3); load_dense(g, g->r, r, 3); load_dense(g, g->eta, eta, 1);
    view_t ev = {g, g->e, NULL, NULL}, E = {g, g->eta, NULL, NULL};
    level_residual(g, &ev, &E, H->lambda * dt);
    memcpy(t, g->t, sizeof(double) * 3 * ncell(g));
    return 0;
}

/* coarse (grid m+1) = restriction of fine (grid m), ncomp components */
int orc_grid_restrict(orc_hier *H, int m, const double *fine, double *coarse, int ncomp) {
    if (m < 0 || m + 1 >= H->nmg) return -1;
    grid_t *g = H->mg[m], *gc = H->mg[m + 1];
    load_dense(g, g->t, fine, ncomp);
    restrict_to(g, g->t, gc, gc->t, ncomp);
    memcpy(coarse, gc->t, sizeof(double) * ncomp * ncell(gc));
    return 0;
}

/* fine (grid m) += prolongation of coarse (grid m+1) */
int orc_grid_prolong_add(orc_hier *H, int m, const double *coarse, double *fine) {
    if (m < 0 || m + 1 >= H->nmg) return -1;
    grid_t *g = H->mg[m], *gc = H->mg[m + 1];
    load_dense(gc, gc->t, coarse, 3); load_dense(g, g->t, fine, 3);
    prolong_add(gc, gc->t, g, g->t);
    memcpy(fine, g->t, sizeof(double) * 3 * ncell(g));
    return 0;
}
