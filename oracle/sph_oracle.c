/*
 * sph_oracle.c -- plain FP64 CPU oracle of the feature-aware SPH relaxation step.
 *
 * TEST INFRASTRUCTURE ONLY (see sph_oracle.h).  Written for a reader who checks it against
 * the paper by eye: no blocking, no fusion, no reordering beyond what the method states.
 * Brute-force sums run over particle indices in increasing order; sums over the oracle's
 * uniform grid run cell by cell.  OpenMP is used only across independent particles i, so
 * results do not depend on the thread count.
 *
 * Build: gcc -O2 -std=c11 -fopenmp -ffp-contract=off -fPIC -shared (no FMA contraction, so
 * the single-precision neighbour predicate below is evaluated operation by operation).
 *
 * Parity notes: functions with no independent pin say so here and in the design notes.
 *   parity unpinned: orc_control's ramp shape (Sec. 3.4.4 gives no formula) and the
 *   end-of-Phase-Two rule (the paper gives none); both are readings, checked only against
 *   hand-computed controller traces.
 */
#include "sph_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------------------------
 * Smoothing kernel.  The paper defers the kernel to its predecessor; this oracle uses the
 * Wendland C2 function with compact support r_c = kappa*h and the usual 1D/2D/3D
 * normalisations, so that the kernel integrates to one in d dimensions (Eq. 12 requires a
 * normalised kernel; Eq. 22 asks for 1D/2D/3D kernels for curve/surface/volume particles).
 *   W_d(r,h) = alpha_d (1-q)^4 (1+4q),  q = r/(kappa h) < 1
 *   alpha_1 = 3/(2R), alpha_2 = 7/(pi R^2), alpha_3 = 21/(2 pi R^3),  R = kappa h
 * ------------------------------------------------------------------------------------------ */
static double wendland_alpha(int d, double R) {
    if (d == 1) return 3.0 / (2.0 * R);
    if (d == 2) return 7.0 / (M_PI * R * R);
    if (d == 3) return 21.0 / (2.0 * M_PI * R * R * R);
    return 0.0;
}

double orc_W(int d, double r, double h, double kappa) {
    double R = kappa * h;
    double q = r / R;
    if (d < 1 || q >= 1.0) return 0.0;
    double t = 1.0 - q;
    return wendland_alpha(d, R) * t * t * t * t * (1.0 + 4.0 * q);
}

/* dW/dr = alpha_d * (-20 q (1-q)^3) / R */
double orc_dW(int d, double r, double h, double kappa) {
    double R = kappa * h;
    double q = r / R;
    if (d < 1 || q >= 1.0) return 0.0;
    double t = 1.0 - q;
    return wendland_alpha(d, R) * (-20.0 * q * t * t * t) / R;
}

/* ------------------------------------------------------------------------------------------
 * Geometry (Sec. 2.1 / 3.1): the volume region is phi > 0 and its boundary phi = 0.  The
 * level set is given analytically here: a box or ball minus circular/spherical holes.
 * ------------------------------------------------------------------------------------------ */
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double* a) { return sqrt(dot3(a, a)); }

static double dist_to(const double* x, const double* c, int D, double* u /* unit x-c, may be NULL */) {
    double d[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) d[a] = x[a] - c[a];
    double r = norm3(d);
    if (u) {
        if (r > 0) { for (int a = 0; a < 3; ++a) u[a] = d[a] / r; }
        else { u[0] = 1; u[1] = 0; u[2] = 0; }
    }
    return r;
}

double orc_h(const orc_sizing* s, const double* x) {
    double h;
    if (s->kind == ORC_H_CONST) return s->a;
    if (s->kind == ORC_H_HOLE_DIST) {
        double dmin = DBL_MAX;
        for (int k = 0; k < s->n_ref; ++k) {
            double r = dist_to(x, s->rc[k], 3, NULL);
            double dk = fabs(r - s->rr[k]);
            if (dk < dmin) dmin = dk;
        }
        h = s->a + s->b * dmin;
    } else { /* ORC_H_RADIAL */
        double r = dist_to(x, s->q, 3, NULL);
        h = s->a + s->b * r;
    }
    if (h < s->lo) h = s->lo;
    if (h > s->hi) h = s->hi;
    return h;
}

double orc_phi(const orc_domain* dom, const double* x, double* grad) {
    int D = dom->D;
    double phi = DBL_MAX, g[3] = {0, 0, 0};
    if (dom->base == ORC_BASE_BOX) {
        for (int a = 0; a < D; ++a) {
            double dlo = x[a] - dom->lo[a], dhi = dom->hi[a] - x[a];
            if (dlo < phi) { phi = dlo; g[0] = g[1] = g[2] = 0; g[a] = 1; }
            if (dhi < phi) { phi = dhi; g[0] = g[1] = g[2] = 0; g[a] = -1; }
        }
    } else {
        double u[3];
        double r = dist_to(x, dom->bc, D, u);
        phi = dom->br - r;
        for (int a = 0; a < 3; ++a) g[a] = -u[a];
    }
    for (int k = 0; k < dom->n_holes; ++k) {
        double u[3];
        double r = dist_to(x, dom->hc[k], D, u);
        double pk = r - dom->hr[k];
        if (pk < phi) { phi = pk; for (int a = 0; a < 3; ++a) g[a] = u[a]; }
    }
    if (grad) for (int a = 0; a < 3; ++a) grad[a] = g[a];
    return phi;
}

/* closest point on feature k (Algorithm 1: map r_{n+1} onto feature k) */
void orc_project(const orc_domain* dom, int k, double* x) {
    const orc_feature* f = &dom->feat[k];
    int D = dom->D;
    if (f->kind == ORC_POINT) {
        for (int a = 0; a < 3; ++a) x[a] = (a < D) ? f->p[a] : 0.0;
    } else if (f->kind == ORC_SEGMENT) {
        const double* A = f->p;
        const double* B = f->p + 3;
        double ab[3], ax[3];
        for (int a = 0; a < 3; ++a) { ab[a] = B[a] - A[a]; ax[a] = x[a] - A[a]; }
        double t = dot3(ax, ab) / dot3(ab, ab);
        if (t < 0) t = 0;
        if (t > 1) t = 1;
        for (int a = 0; a < 3; ++a) x[a] = A[a] + t * ab[a];
    } else if (f->kind == ORC_CIRCLE || f->kind == ORC_SPHERE) {
        double c[3] = {f->p[0], f->p[1], f->kind == ORC_SPHERE ? f->p[2] : 0.0};
        double R = f->kind == ORC_SPHERE ? f->p[3] : f->p[2];
        double u[3];
        dist_to(x, c, D, u);
        for (int a = 0; a < 3; ++a) x[a] = (a < D) ? c[a] + R * u[a] : 0.0;
    } else if (f->kind == ORC_RECT) {
        const double* o = f->p;
        const double* u = f->p + 3;
        const double* w = f->p + 6;
        double ox[3];
        for (int a = 0; a < 3; ++a) ox[a] = x[a] - o[a];
        double s = dot3(ox, u), t = dot3(ox, w);
        if (s < 0) s = 0;
        if (s > f->p[9]) s = f->p[9];
        if (t < 0) t = 0;
        if (t > f->p[10]) t = f->p[10];
        for (int a = 0; a < 3; ++a) x[a] = o[a] + s * u[a] + t * w[a];
    }
    /* ORC_VOLUME: nothing (escapes are handled by the integrator) */
}

/* nb: outward unit normal of the domain at the particle, used when the particle acts as a
 *     boundary particle b for a higher-dimensional particle (n_b of Eq. 17 / Eq. 19).
 * tg: the particle's own tangent-space descriptor: the unit tangent for curves, the unit
 *     normal for surfaces (Algorithm 1: forces and velocities are mapped onto feature k). */
void orc_frame(const orc_domain* dom, int k, const double* x, double* nb, double* tg) {
    const orc_feature* f = &dom->feat[k];
    int D = dom->D;
    for (int a = 0; a < 3; ++a) { nb[a] = 0; tg[a] = 0; }
    if (f->kind == ORC_POINT) {
        for (int a = 0; a < 3; ++a) nb[a] = f->nb[a];
    } else if (f->kind == ORC_SEGMENT) {
        double ab[3];
        for (int a = 0; a < 3; ++a) ab[a] = f->p[3 + a] - f->p[a];
        double L = norm3(ab);
        for (int a = 0; a < 3; ++a) { nb[a] = f->nb[a]; tg[a] = ab[a] / L; }
    } else if (f->kind == ORC_CIRCLE) {
        double c[3] = {f->p[0], f->p[1], 0.0}, u[3];
        dist_to(x, c, D, u);
        nb[0] = f->orient * u[0]; nb[1] = f->orient * u[1];
        tg[0] = -u[1]; tg[1] = u[0];
    } else if (f->kind == ORC_SPHERE) {
        double u[3];
        dist_to(x, f->p, D, u);
        for (int a = 0; a < 3; ++a) { nb[a] = f->orient * u[a]; tg[a] = nb[a]; }
    } else if (f->kind == ORC_RECT) {
        for (int a = 0; a < 3; ++a) { nb[a] = f->nb[a]; tg[a] = f->nb[a]; }
    }
}

/* v <- Pi_k(x) v : identity for volume particles, t t^T for curves, I - n n^T for surfaces,
 * zero for singular points (they never move). */
void orc_tangent(const orc_domain* dom, int k, const double* x, double* v) {
    const orc_feature* f = &dom->feat[k];
    double nb[3], tg[3];
    if (f->kind == ORC_VOLUME) return;
    if (f->dim == 0) { v[0] = v[1] = v[2] = 0; return; }
    orc_frame(dom, k, x, nb, tg);
    double s = dot3(v, tg);
    if (f->dim == 1) { for (int a = 0; a < 3; ++a) v[a] = s * tg[a]; }
    else { for (int a = 0; a < 3; ++a) v[a] = v[a] - s * tg[a]; }
}

/* Eqs. 10/11: total mass M_k = integral of rho_t = h^-d over feature k (midpoint rule).
 * The particle budget of feature k is M_k with unit-mass particles. */
double orc_feature_measure_density(const orc_domain* dom, const orc_sizing* s, int k, int nq) {
    const orc_feature* f = &dom->feat[k];
    int D = dom->D;
    double M = 0.0;
    if (f->kind == ORC_POINT) return 1.0;
    if (f->kind == ORC_VOLUME) {
        double dx[3] = {1, 1, 1}, cellv = 1.0;
        for (int a = 0; a < D; ++a) { dx[a] = (dom->hi[a] - dom->lo[a]) / nq; cellv *= dx[a]; }
        int64_t nz = (D == 3) ? nq : 1;
        for (int64_t iz = 0; iz < nz; ++iz)
            for (int64_t iy = 0; iy < nq; ++iy)
                for (int64_t ix = 0; ix < nq; ++ix) {
                    double x[3] = {dom->lo[0] + (ix + 0.5) * dx[0], dom->lo[1] + (iy + 0.5) * dx[1],
                                   D == 3 ? dom->lo[2] + (iz + 0.5) * dx[2] : 0.0};
                    if (orc_phi(dom, x, NULL) > 0) M += cellv * pow(orc_h(s, x), -(double)D);
                }
        return M;
    }
    if (f->kind == ORC_SEGMENT) {
        double L = 0, ab[3];
        for (int a = 0; a < 3; ++a) ab[a] = f->p[3 + a] - f->p[a];
        L = norm3(ab);
        for (int q = 0; q < nq; ++q) {
            double t = (q + 0.5) / nq, x[3];
            for (int a = 0; a < 3; ++a) x[a] = f->p[a] + t * ab[a];
            M += (L / nq) / orc_h(s, x);
        }
        return M;
    }
    if (f->kind == ORC_CIRCLE) {
        double R = f->p[2];
        for (int q = 0; q < nq; ++q) {
            double th = 2 * M_PI * (q + 0.5) / nq;
            double x[3] = {f->p[0] + R * cos(th), f->p[1] + R * sin(th), 0};
            M += (2 * M_PI * R / nq) / orc_h(s, x);
        }
        return M;
    }
    if (f->kind == ORC_RECT) {
        for (int i = 0; i < nq; ++i)
            for (int j = 0; j < nq; ++j) {
                double si = (i + 0.5) / nq * f->p[9], tj = (j + 0.5) / nq * f->p[10], x[3];
                for (int a = 0; a < 3; ++a) x[a] = f->p[a] + si * f->p[3 + a] + tj * f->p[6 + a];
                double hh = orc_h(s, x);
                M += (f->p[9] / nq) * (f->p[10] / nq) / (hh * hh);
            }
        return M;
    }
    if (f->kind == ORC_SPHERE) {
        double R = f->p[3];
        for (int i = 0; i < nq; ++i) {
            double th = M_PI * (i + 0.5) / nq;
            for (int j = 0; j < 2 * nq; ++j) {
                double ph = M_PI * (j + 0.5) / nq;
                double x[3] = {f->p[0] + R * sin(th) * cos(ph), f->p[1] + R * sin(th) * sin(ph),
                               f->p[2] + R * cos(th)};
                double hh = orc_h(s, x);
                M += R * R * sin(th) * (M_PI / nq) * (M_PI / nq) / (hh * hh);
            }
        }
        return M;
    }
    return 0.0;
}

/* ------------------------------------------------------------------------------------------
 * Neighbour search.
 * Definition (Eq. 7 / Eq. 19): j interacts with i when r_ij < kappa * h_ij, h_ij = (h_i+h_j)/2.
 * orc_neighbors_brute lists all such j != i, over every particle regardless of group, in
 * increasing index order, computed directly in FP64 on the positions.
 * ------------------------------------------------------------------------------------------ */
int64_t orc_neighbors_brute(int64_t n, int D, const double* x, const double* h, double kappa,
                            int64_t i, int32_t* out, int64_t cap) {
    int64_t cnt = 0;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        double r2 = 0;
        for (int a = 0; a < D; ++a) { double d = x[3 * i + a] - x[3 * j + a]; r2 += d * d; }
        double rc = kappa * 0.5 * (h[i] + h[j]);
        if (sqrt(r2) < rc) { if (cnt < cap) out[cnt] = (int32_t)j; ++cnt; }
    }
    return cnt;
}

/* Representation used by the data-parallel cell lists (Algorithm 1 "update the multi-level
 * data structure" and "construct Verlet neighbour list").  Specification, with m the number of
 * cells per support (1, 2 or 4: a level's cells are 1/m of the largest support it holds):
 *   c0  = kappa*h_lo*(1+2^-10)/m rounded up to a float;  level l has cell edge c_l = c0*2^l;
 *   L   = the smallest count with m*c0*2^(L-1) >= kappa*h_hi*(1+2^-10);
 *   thr[l] = m*c_l/(kappa*(1+2^-10)) rounded down to a float (l < L-1), thr[L-1] = +inf;
 *   a particle's level is the first l with h <= thr[l];
 *   with M = m*c_{L-1}: origin = (lo - M) rounded down to floats;
 *   dims_l = ceil((hi + M - origin)/c_l)+1;
 *   finest cell c = floor((x - origin) * (1/c0)) with 1/c0 rounded once in FP64 (clamped into
 *          the finest grid) and finest offset o = (x - origin) - c*c0 rounded to the working
 *          precision (it may fall an ulp outside [0, c0) where the rounded inverse puts x on
 *          the other side of a face);
 *   level l: cell = c >> l, offset = o + (c - (cell << l))*c0, each operation rounded in the
 *          working precision (the stored state is the finest cell + offset, so coarser levels
 *          are derived from it without the FP64 position); key = base_l + row-major cell. */
static float f_round_up(double v) {
    float f = (float)v;
    if ((double)f < v) f = nextafterf(f, INFINITY);
    return f;
}
static float f_round_down(double v) {
    float f = (float)v;
    if ((double)f > v) f = nextafterf(f, -INFINITY);
    return f;
}

void orc_grid_spec(int D, const double* lo, const double* hi, double h_lo, double h_hi,
                   double kappa, int cells_per_support, orc_grid* g) {
    const double m = 1.0 + ldexp(1.0, -10);
    const double cps = (double)cells_per_support;
    memset(g, 0, sizeof(*g));
    g->D = D;
    g->cps = cells_per_support;
    g->c0 = f_round_up(kappa * h_lo * m / cps);
    int L = 1;
    while (L < ORC_MAX_LEVELS && cps * ldexp((double)g->c0, L - 1) < kappa * h_hi * m) ++L;
    g->L = L;
    for (int l = 0; l < ORC_MAX_LEVELS; ++l)
        g->thr[l] = (l < L - 1) ? f_round_down(cps * ldexp((double)g->c0, l) / (kappa * m)) : INFINITY;
    double top = cps * ldexp((double)g->c0, L - 1);
    for (int a = 0; a < 3; ++a) g->origin[a] = (a < D) ? f_round_down(lo[a] - top) : 0.0f;
    int64_t base = 0;
    for (int l = 0; l < L; ++l) {
        double cl = ldexp((double)g->c0, l);
        int64_t cells = 1;
        for (int a = 0; a < 3; ++a) {
            g->dims[l][a] = (a < D) ? (int64_t)ceil((hi[a] + top - (double)g->origin[a]) / cl) + 1 : 1;
            cells *= g->dims[l][a];
        }
        g->base[l] = base;
        base += cells;
    }
    g->ncell = base;
}

static double to_prec(double v, int prec) { return prec == 32 ? (double)(float)v : v; }

static int level_of(const orc_grid* g, double h, int prec) {
    double hp = to_prec(h, prec);
    int l = 0;
    while (l < g->L - 1 && hp > (double)g->thr[l]) ++l;
    return l;
}

static void repr_one(const orc_grid* g, const double* x, double h, int prec, int* lvl,
                     int64_t* cell, double* off, int* clamped) {
    int l = level_of(g, h, prec);
    const double c0 = (double)g->c0;
    *lvl = l;
    *clamped = 0;
    for (int a = 0; a < 3; ++a) {
        if (a >= g->D) { cell[a] = 0; off[a] = 0; continue; }
        /* finest-level cell and offset, from the FP64 position */
        double rel = x[a] - (double)g->origin[a];
        int64_t c = (int64_t)floor(rel * (1.0 / c0));
        if (c < 0) { c = 0; *clamped = 1; }
        if (c > g->dims[0][a] - 1) { c = g->dims[0][a] - 1; *clamped = 1; }
        double o0 = to_prec(rel - (double)c * c0, prec);
        /* level l: cell = c >> l; offset = o0 + (c - (cell << l)) * c0, each operation rounded
         * in the working precision */
        int64_t cl = c >> l;
        int64_t rem = c - (cl << l);
        if (prec == 32) {
            float t = (float)rem * g->c0;
            off[a] = (double)((float)o0 + t);
        } else {
            off[a] = o0 + (double)rem * c0;
        }
        cell[a] = cl;
    }
}

void orc_grid_repr(const orc_grid* g, int64_t n, const double* x, const double* h, int32_t prec,
                   int32_t* level, int64_t* cell, double* off, int64_t* key, int32_t* clamped) {
    for (int64_t i = 0; i < n; ++i) {
        int l, cl;
        repr_one(g, x + 3 * i, h[i], prec, &l, cell + 3 * i, off + 3 * i, &cl);
        level[i] = l;
        clamped[i] = cl;
        key[i] = g->base[l] + (cell[3 * i + 2] * g->dims[l][1] + cell[3 * i + 1]) * g->dims[l][0] + cell[3 * i];
    }
}

/* The same neighbour predicate, evaluated on the representation in the working precision,
 * one rounded operation at a time:
 *   dx_a = (off_i,a - off_j,a) + m_a * c0,   m_a = cell_i,a * 2^l_i - cell_j,a * 2^l_j
 *   r2   = (dx_0*dx_0 + dx_1*dx_1) + dx_2*dx_2
 *   pair:   r2 < rc*rc,  rc = (h_i + h_j) * (kappa/2),  j != i
 *   self:   r2 < rc*rc,  rc = kappa * h_i               (j = i included)  */
int64_t orc_neighbors_repr(const orc_grid* g, int64_t n, const double* x, const double* h,
                           int32_t prec, double kappa, int32_t self_radius, int64_t i,
                           int32_t* out, int64_t cap) {
    int li, lj, ci_, cj_;
    int64_t cell_i[3], cell_j[3];
    double off_i[3], off_j[3];
    repr_one(g, x + 3 * i, h[i], prec, &li, cell_i, off_i, &ci_);
    int64_t cnt = 0;
    for (int64_t j = 0; j < n; ++j) {
        repr_one(g, x + 3 * j, h[j], prec, &lj, cell_j, off_j, &cj_);
        int accept;
        if (prec == 32) {
            float dx[3] = {0, 0, 0};
            for (int a = 0; a < g->D; ++a) {
                float m = (float)(cell_i[a] * ((int64_t)1 << li) - cell_j[a] * ((int64_t)1 << lj));
                float dd = (float)off_i[a] - (float)off_j[a];
                float mc = m * g->c0;
                dx[a] = dd + mc;
            }
            float r2 = dx[0] * dx[0];
            float t1 = dx[1] * dx[1];
            r2 = r2 + t1;
            if (g->D == 3) { float t2 = dx[2] * dx[2]; r2 = r2 + t2; }
            float hi = (float)h[i], hj = (float)h[j], rc;
            if (self_radius) rc = hi * (float)kappa;
            else { float hs = hi + hj; rc = hs * (float)(0.5 * kappa); }
            float rc2 = rc * rc;
            accept = r2 < rc2;
        } else {
            double dx[3] = {0, 0, 0};
            for (int a = 0; a < g->D; ++a) {
                double m = (double)(cell_i[a] * ((int64_t)1 << li) - cell_j[a] * ((int64_t)1 << lj));
                dx[a] = (off_i[a] - off_j[a]) + m * (double)g->c0;
            }
            double r2 = dx[0] * dx[0];
            double t1 = dx[1] * dx[1];
            r2 = r2 + t1;
            if (g->D == 3) { double t2 = dx[2] * dx[2]; r2 = r2 + t2; }
            double rc = self_radius ? h[i] * kappa : (h[i] + h[j]) * (0.5 * kappa);
            accept = r2 < rc * rc;
        }
        if (!self_radius && j == i) accept = 0;
        if (accept) { if (cnt < cap) out[cnt] = (int32_t)j; ++cnt; }
    }
    return cnt;
}

/* Stable counting sort by cell key: cell_start = exclusive prefix sum of the per-cell counts
 * (length ncell+1); perm lists particle indices cell by cell, ties in increasing index. */
void orc_counting_sort(int64_t n, const int64_t* key, int64_t ncell, int64_t* cell_start, int64_t* perm) {
    int64_t* cursor = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
    for (int64_t c = 0; c <= ncell; ++c) cell_start[c] = 0;
    for (int64_t i = 0; i < n; ++i) cell_start[key[i] + 1] += 1;
    for (int64_t c = 0; c < ncell; ++c) cell_start[c + 1] += cell_start[c];
    for (int64_t c = 0; c < ncell; ++c) cursor[c] = cell_start[c];
    for (int64_t i = 0; i < n; ++i) perm[cursor[key[i]]++] = i;
    free(cursor);
}

/* ------------------------------------------------------------------------------------------
 * Candidate lists for the oracle's own physics.  Either every particle (brute force) or the
 * particles of the 3^D cells around i on a uniform grid whose edge is kappa * max h; every
 * pair with r_ij < kappa*h_ij lies in those cells, so both visit the same interacting pairs.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    int D;
    double lo[3], cell;
    int64_t dims[3];
    int64_t* start;   /* per cell, length ncell+1 */
    int64_t* idx;     /* particle indices in cell order, increasing within a cell */
} ugrid;

static void ugrid_build(ugrid* u, int64_t n, int D, const double* x, const double* h, double kappa) {
    double hmax = 0, lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (int64_t i = 0; i < n; ++i) {
        if (h[i] > hmax) hmax = h[i];
        for (int a = 0; a < D; ++a) {
            if (x[3 * i + a] < lo[a]) lo[a] = x[3 * i + a];
            if (x[3 * i + a] > hi[a]) hi[a] = x[3 * i + a];
        }
    }
    u->D = D;
    u->cell = kappa * hmax * (1.0 + 1e-9);
    int64_t ncell = 1;
    for (int a = 0; a < 3; ++a) {
        if (a < D) { u->lo[a] = lo[a]; u->dims[a] = (int64_t)floor((hi[a] - lo[a]) / u->cell) + 1; }
        else { u->lo[a] = 0; u->dims[a] = 1; }
        ncell *= u->dims[a];
    }
    int64_t* key = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) c[a] = (int64_t)floor((x[3 * i + a] - u->lo[a]) / u->cell);
        key[i] = (c[2] * u->dims[1] + c[1]) * u->dims[0] + c[0];
    }
    u->start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ncell + 1));
    u->idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    orc_counting_sort(n, key, ncell, u->start, u->idx);
    free(key);
}

static void ugrid_free(ugrid* u) { free(u->start); free(u->idx); }

/* collects candidate indices for particle i into buf, cell by cell (increasing index within a
 * cell); returns the count.  Sums over these candidates equal the brute-force sums up to the
 * order of rounding. */
static int64_t ugrid_candidates(const ugrid* u, const double* xi, int64_t* buf, int64_t cap) {
    int64_t c[3] = {0, 0, 0}, cnt = 0;
    for (int a = 0; a < u->D; ++a) c[a] = (int64_t)floor((xi[a] - u->lo[a]) / u->cell);
    int zr = (u->D == 3) ? 1 : 0;
    for (int64_t dz = -zr; dz <= zr; ++dz)
        for (int64_t dy = -1; dy <= 1; ++dy)
            for (int64_t dx = -1; dx <= 1; ++dx) {
                int64_t cc[3] = {c[0] + dx, c[1] + dy, c[2] + dz};
                int ok = 1;
                for (int a = 0; a < 3; ++a) if (cc[a] < 0 || cc[a] >= u->dims[a]) ok = 0;
                if (!ok) continue;
                int64_t k = (cc[2] * u->dims[1] + cc[1]) * u->dims[0] + cc[0];
                for (int64_t p = u->start[k]; p < u->start[k + 1]; ++p)
                    if (cnt < cap) buf[cnt++] = u->idx[p];
            }
    return cnt;
}

static int feat_dim(const orc_domain* dom, int32_t g) { return dom->feat[g].dim; }

/* ------------------------------------------------------------------------------------------
 * Pressure-force pass (Algorithm 1: gamma_i, F_p, map F_p onto the feature, Delta t).
 * For particle i of group g, intrinsic dimension d, with rho = h^-d, P = p0/rho^2 = p0 h^(2d)
 * (EOS Eq. 6 with gamma = 2; the current density drops out of Eq. 7):
 *   sigma_i = sum_{j in g, r<kappa h_i} W_d(r_ij, h_i)                      (Eq. 20; j = i included)
 *   gamma_i = sum_{j in g, r<kappa h_i} W_d(r_ij, h_i) h_j^d                  (Eq. 18)
 *   F_i     = sum_{j in g, j != i} (P_i + P_j) dW_d(r_ij, h_ij) e_ij          (Eq. 19, first sum, m_j = 1)
 *           + sum_{b: d_b < d}  rho_b (P_i + P_b) W_d(r_ib, h_ib) n_b|i A_b    (Eq. 19, second sum)
 *             with rho_b = h_b^-d, P_b = p0 h_b^(2d), A_b = h_b^(d-1) and n_b|i the outward
 *             normal of b projected onto i's feature and normalised
 *   a_p,i   = Pi_i( -F_i / gamma_i )                                           (Eq. 4, Eq. 19)
 *   S_i     = (sum of the magnitudes of all terms of F_i) / gamma_i   (scale for tolerances)
 *   dta_g   = min_i 0.25 sqrt(r_c,i / |a_p,i|),  dtv_g = min_i r_c,i / (40 |v_i|)   (Eq. 24)
 * The viscous limit 0.125 r_c^2/nu of Eq. 24 equals 1.25 r_c/|v| with nu = 0.1 r_c |v|
 * (Eq. 8) and never binds against r_c/(40|v|), so it is omitted.
 * ------------------------------------------------------------------------------------------ */
void orc_interact(int64_t n, const orc_domain* dom, const orc_params* prm,
                  const double* x, const double* h, const int32_t* grp, const double* v,
                  int64_t n_sub, const int64_t* sub, int32_t use_grid,
                  double* sigma, double* gamma, double* F, double* a_p, double* S,
                  double* dta, double* dtv) {
    const int D = dom->D;
    const double kappa = prm->kappa, p0 = prm->p0;
    int64_t m = sub ? n_sub : n;
    ugrid u;
    if (use_grid) ugrid_build(&u, n, D, x, h, kappa);
    double* dta_i = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double* dtv_i = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));

#pragma omp parallel
    {
        int64_t cap = use_grid ? n : 0;
        int64_t* buf = use_grid ? (int64_t*)malloc(sizeof(int64_t) * (size_t)(cap > 0 ? cap : 1)) : NULL;
#pragma omp for schedule(dynamic, 64)
        for (int64_t s = 0; s < m; ++s) {
            int64_t i = sub ? sub[s] : s;
            int gi = grp[i], d = feat_dim(dom, gi);
            double sg = 0, gm = 0, f[3] = {0, 0, 0}, mag = 0;
            if (d > 0) {
                double Pi = p0 * pow(h[i], 2.0 * d);
                int64_t nc = use_grid ? ugrid_candidates(&u, x + 3 * i, buf, cap) : n;
                for (int64_t c = 0; c < nc; ++c) {
                    int64_t j = use_grid ? buf[c] : c;
                    double rij[3] = {0, 0, 0};
                    for (int a = 0; a < D; ++a) rij[a] = x[3 * i + a] - x[3 * j + a];
                    double r = norm3(rij);
                    double hij = 0.5 * (h[i] + h[j]);
                    int gj = grp[j], dj = feat_dim(dom, gj);
                    if (gj == gi) {
                        if (r < kappa * h[i]) {
                            double w = orc_W(d, r, h[i], kappa);
                            sg += w;
                            gm += w * pow(h[j], (double)d);
                        }
                        if (j != i && r < kappa * hij) {
                            double Pj = p0 * pow(h[j], 2.0 * d);
                            double c1 = (Pi + Pj) * orc_dW(d, r, hij, kappa);
                            for (int a = 0; a < 3; ++a) f[a] += c1 * rij[a] / r;
                            mag += fabs(c1);
                        }
                    } else if (prm->boundary_correction && dj < d && r < kappa * hij) {
                        double nb[3], tg[3];
                        orc_frame(dom, gj, x + 3 * j, nb, tg);
                        orc_tangent(dom, gi, x + 3 * i, nb);
                        double nn = norm3(nb);
                        if (nn > 1e-12) {
                            double rho_b = pow(h[j], -(double)d);
                            double Pb = p0 * pow(h[j], 2.0 * d);
                            double Ab = pow(h[j], (double)(d - 1));
                            double c2 = (prm->boundary_rho ? rho_b : 1.0) * (Pi + Pb) *
                                        orc_W(d, r, hij, kappa) * Ab;
                            for (int a = 0; a < 3; ++a) f[a] += c2 * nb[a] / nn;
                            mag += fabs(c2);
                        }
                    }
                }
            }
            double ap[3] = {0, 0, 0};
            if (d > 0 && gm > 0) {
                for (int a = 0; a < 3; ++a) ap[a] = -f[a] / gm;
                orc_tangent(dom, gi, x + 3 * i, ap);
            }
            if (sigma) sigma[s] = sg;
            if (gamma) gamma[s] = gm;
            if (F) for (int a = 0; a < 3; ++a) F[3 * s + a] = f[a];
            if (a_p) for (int a = 0; a < 3; ++a) a_p[3 * s + a] = ap[a];
            if (S) S[s] = (gm > 0) ? mag / gm : 0.0;
            double rc = kappa * h[i];
            double an = norm3(ap), vn = v ? norm3(v + 3 * i) : 0.0;
            dta_i[s] = (d > 0 && an > 0) ? prm->cfl_a * sqrt(rc / an) : INFINITY;
            dtv_i[s] = (d > 0 && vn > 0) ? prm->cfl_v * rc / vn : INFINITY;
        }
        free(buf);
    }
    if (dta || dtv) {
        for (int g = 0; g < dom->n_feat; ++g) { if (dta) dta[g] = INFINITY; if (dtv) dtv[g] = INFINITY; }
        for (int64_t s = 0; s < m; ++s) {
            int64_t i = sub ? sub[s] : s;
            int g = grp[i];
            if (dta && dta_i[s] < dta[g]) dta[g] = dta_i[s];
            if (dtv && dtv_i[s] < dtv[g]) dtv[g] = dtv_i[s];
        }
    }
    free(dta_i);
    free(dtv_i);
    if (use_grid) ugrid_free(&u);
}

void orc_ctrl_init(orc_ctrl* c) {
    memset(c, 0, sizeof(*c));
    c->phase = ORC_PHASE1;
    c->ramp_f = 1.0;
    for (int g = 0; g < ORC_MAX_FEAT; ++g) {
        c->gphase[g] = ORC_PHASE1;
        c->gf[g] = 1.0;
    }
}

static double rel_err(double a, double b) {
    if (b != 0) return fabs(a - b) / fabs(b);
    return a == 0 ? 0.0 : INFINITY;
}

static void window_reset(orc_ctrl* c) {
    c->wcount = 0;
    c->nwin = 0;
    for (int g = 0; g < ORC_MAX_FEAT; ++g) { c->wsum[g] = 0; c->A_last[g] = 0; c->A_prev[g] = 0; }
}

static void group_window_reset(orc_ctrl* c, int g) {
    c->gwcount[g] = 0;
    c->gnwin[g] = 0;
    c->wsum[g] = 0;
    c->A_last[g] = 0;
    c->A_prev[g] = 0;
}

/* the step size of one moving group from its Eq. 24 terms, its attenuation f and whether it is
 * nullified on the schedule (step 4 below) */
static void group_step(const orc_params* prm, int g, const double* dta, const double* dtv, double f,
                       int periodic, orc_ctrl* c) {
    double dv = (f > 0) ? dtv[g] / f : INFINITY;
    double cand = dta[g] < dv ? dta[g] : dv;
    int rs = periodic || (c->dt_prev[g] > 0 && cand < prm->dt_collapse * c->dt_prev[g]);
    double dt = rs ? dta[g] : cand;
    if (dt > prm->dt_cap) dt = prm->dt_cap;
    c->dt_prev[g] = dt;
    c->dt[g] = dt;
    c->reset[g] = rs;
}

/* ------------------------------------------------------------------------------------------
 * The same controller run by every group on its own (group_convergence = 1; Algorithm 1
 * skips a feature whose V-bar_k has converged).  For each moving group g at step n:
 *  1. RAMP -> PHASE2 once ramp_len steps have passed since the group's switch;
 *  2. in PHASE1 / PHASE2 on sampling steps: V-bar_g enters the group's window; with two
 *     closed windows E_g = max(|V-bar_g - A_last,g|/|A_last,g|, |A_last,g - A_prev,g|/|A_prev,g|);
 *     E_g < threshold moves the group PHASE1 -> RAMP or PHASE2 -> DONE;
 *  3. eps, f and the nullification schedule of the group's phase (as for the instance);
 *  4. the group's step size; a DONE group does not move (dt = 0).
 * The instance's phase is that of its least advanced moving group (DONE when all are);
 * E_sys is the largest E_g; ramp_start is the step at which the last group left PHASE1.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    int lowest, evaluated;
    double et, ea, es;
} group_acc;

/* steps 1-4 for the groups of intrinsic dimension `only_dim` (every moving group when 0) */
static void group_pass(const orc_params* prm, int G, const int32_t* gdim, const double* Vsum,
                       const double* dta, const double* dtv, orc_ctrl* c, int only_dim, group_acc* acc) {
    const int sampling = c->n % prm->sample_every == 0;
    for (int g = 0; g < G; ++g) {
        if (only_dim > 0 && gdim[g] != only_dim) continue;
        if (gdim[g] < 1) { c->dt[g] = 0; c->reset[g] = 1; c->geps[g] = 0; c->gf[g] = 0; continue; }
        int ph = c->gphase[g];
        if (ph == ORC_RAMP && c->n - c->gramp_start[g] >= prm->ramp_len) {
            ph = ORC_PHASE2;
            group_window_reset(c, g);
        }
        if ((ph == ORC_PHASE1 || ph == ORC_PHASE2) && sampling) {
            c->Vbar[g] = Vsum[g];
            c->wsum[g] += c->Vbar[g];
            c->gwcount[g] += 1;
            if (c->gwcount[g] == prm->window) {
                c->A_prev[g] = c->A_last[g];
                c->A_last[g] = c->wsum[g] / prm->window;
                c->wsum[g] = 0;
                c->gwcount[g] = 0;
                c->gnwin[g] += 1;
            }
            if (c->gnwin[g] >= 2) {
                double e1 = rel_err(c->Vbar[g], c->A_last[g]);
                double e2 = rel_err(c->A_last[g], c->A_prev[g]);
                c->gE[g] = e1 > e2 ? e1 : e2;
                if (e1 > acc->et) acc->et = e1;
                if (e2 > acc->ea) acc->ea = e2;
                acc->evaluated = 1;
                if (c->gE[g] < prm->threshold) {
                    if (ph == ORC_PHASE1) {
                        ph = ORC_RAMP;
                        c->gramp_start[g] = c->n;
                        group_window_reset(c, g);
                    } else {
                        ph = ORC_DONE;
                    }
                }
            }
        }
        c->gphase[g] = ph;
        if (c->gE[g] > acc->es) acc->es = c->gE[g];
        if (ph < acc->lowest) acc->lowest = ph;
        if (ph == ORC_DONE) { c->dt[g] = 0; c->reset[g] = 1; c->geps[g] = 0; c->gf[g] = 0; continue; }
        double eps = prm->eps1, f = 1.0;
        int periodic = (c->n % prm->reset_period) == 0;
        if (ph == ORC_RAMP) {
            double sr = (double)(c->n - c->gramp_start[g]) / (double)prm->ramp_len;
            eps = prm->eps1 * (1.0 - sr);
            f = 0.5 * (1.0 + cos(M_PI * sr));
        } else if (ph == ORC_PHASE2) {
            eps = 0.0;
            periodic = 1;
        }
        group_step(prm, g, dta, dtv, f, periodic, c);
        c->geps[g] = eps;
        c->gf[g] = f;
    }
}

/* the instance's summary after every group has run: its phase is that of its least advanced
 * moving group, E_sys the largest group error, ramp_start the step the last group left PHASE1 */
static void group_summary(orc_ctrl* c, const group_acc* acc) {
    if (acc->evaluated) {
        c->E_t = acc->et;
        c->E_avg = acc->ea;
    }
    c->E_sys = acc->es;
    if (c->phase == ORC_PHASE1 && acc->lowest > ORC_PHASE1) c->ramp_start = c->n;
    c->phase = acc->lowest;
}

static void control_per_group(const orc_params* prm, int G, const int32_t* gdim, const double* Vsum,
                              const double* dta, const double* dtv, orc_ctrl* c) {
    group_acc acc = {ORC_DONE, 0, 0.0, 0.0, 0.0};
    group_pass(prm, G, gdim, Vsum, dta, dtv, c, 0, &acc);
    group_summary(c, &acc);
}

/* ------------------------------------------------------------------------------------------
 * Two-phase controller and per-group step size for step n (Sec. 3.4, Sec. 3.5, Eq. 24).
 * Vsum[g] = sum of V~_i over group g from this step's pressure pass (Eq. 20, Eq. 22, V_ref = 1).
 *  1. RAMP -> PHASE2 once ramp_len steps have passed since the switch (windows restart).
 *  2. In PHASE1 / PHASE2, on steps n % sample_every == 0: push V-bar_g into the open window;
 *     a full window (window samples) closes with mean A; once two windows have closed,
 *       E_t   = max_g |V-bar_g - A_last,g| / |A_last,g|
 *       E_avg = max_g |A_last,g - A_prev,g| / |A_prev,g|,   E_sys = max(E_t, E_avg)
 *     and E_sys < threshold moves PHASE1 -> RAMP (ramp_start = n) or PHASE2 -> DONE.
 *  3. Parameters of this step: PHASE1: eps = eps1, attenuation f = 1, velocities nullified
 *     when n % reset_period == 0; RAMP: s = (n-ramp_start)/ramp_len, eps = eps1 (1-s),
 *     f = (1 + cos(pi s))/2, same nullification rule; PHASE2: eps = 0, f = 1, nullified
 *     every step.
 *  4. Per group: dt = min(dta, dtv/f); if the group is nullified, or dt < dt_collapse times
 *     the previous step of the group, velocities are set to zero and dt = dta; dt <= dt_cap.
 * Only groups with intrinsic dimension >= 1 take part.  DONE freezes the system (dt = 0).
 * ------------------------------------------------------------------------------------------ */
void orc_control(const orc_params* prm, int G, const int32_t* gdim, const double* Vsum,
                 const double* dta, const double* dtv, orc_ctrl* c) {
    if (c->phase == ORC_DONE) {
        for (int g = 0; g < G; ++g) { c->dt[g] = 0; c->reset[g] = 1; c->gphase[g] = ORC_DONE; c->geps[g] = 0; c->gf[g] = 0; }
        c->eps = 0; c->ramp_f = 0;
        return;
    }
    if (prm->group_convergence) {
        control_per_group(prm, G, gdim, Vsum, dta, dtv, c);
        return;
    }
    if (c->phase == ORC_RAMP && c->n - c->ramp_start >= prm->ramp_len) {
        c->phase = ORC_PHASE2;
        window_reset(c);
    }
    if ((c->phase == ORC_PHASE1 || c->phase == ORC_PHASE2) && c->n % prm->sample_every == 0) {
        for (int g = 0; g < G; ++g) {
            c->Vbar[g] = gdim[g] > 0 ? Vsum[g] : 0.0;
            c->wsum[g] += c->Vbar[g];
        }
        c->wcount += 1;
        if (c->wcount == prm->window) {
            for (int g = 0; g < G; ++g) {
                c->A_prev[g] = c->A_last[g];
                c->A_last[g] = c->wsum[g] / prm->window;
                c->wsum[g] = 0;
            }
            c->wcount = 0;
            c->nwin += 1;
        }
        if (c->nwin >= 2) {
            double et = 0, ea = 0;
            for (int g = 0; g < G; ++g) {
                if (gdim[g] < 1) continue;
                double e1 = rel_err(c->Vbar[g], c->A_last[g]);
                double e2 = rel_err(c->A_last[g], c->A_prev[g]);
                if (e1 > et) et = e1;
                if (e2 > ea) ea = e2;
            }
            c->E_t = et;
            c->E_avg = ea;
            c->E_sys = et > ea ? et : ea;
            if (c->E_sys < prm->threshold) {
                if (c->phase == ORC_PHASE1) {
                    c->phase = ORC_RAMP;
                    c->ramp_start = c->n;
                    window_reset(c);
                } else {
                    c->phase = ORC_DONE;
                    for (int g = 0; g < G; ++g) { c->dt[g] = 0; c->reset[g] = 1; c->gphase[g] = ORC_DONE; c->geps[g] = 0; c->gf[g] = 0; }
                    c->eps = 0; c->ramp_f = 0;
                    return;
                }
            }
        }
    }
    double eps = prm->eps1, f = 1.0;
    int periodic = (c->n % prm->reset_period) == 0;
    if (c->phase == ORC_RAMP) {
        double s = (double)(c->n - c->ramp_start) / (double)prm->ramp_len;
        eps = prm->eps1 * (1.0 - s);
        f = 0.5 * (1.0 + cos(M_PI * s));
    } else if (c->phase == ORC_PHASE2) {
        eps = 0.0;
        periodic = 1;
    }
    for (int g = 0; g < G; ++g) {
        c->gphase[g] = c->phase;
        c->geps[g] = eps;
        c->gf[g] = f;
        if (gdim[g] < 1) { c->dt[g] = 0; c->reset[g] = 1; continue; }
        group_step(prm, g, dta, dtv, f, periodic, c);
    }
    c->eps = eps;
    c->ramp_f = f;
}

/* ------------------------------------------------------------------------------------------
 * Viscous pass and position update (Algorithm 1: mid-point velocity, viscous force, map,
 * predicted velocity, position, map).  With dt = dt_g, f and eps from orc_control:
 *   v'_i   = 0 if the group is nullified, else f v_i
 *   v~_i   = v'_i + dt (a_p,i - eps v'_i)                                     (Eq. 23)
 *   nu_i   = visc r_c,i |v~_i|,  eta_i = rho_i nu_i                            (Eq. 8)
 *   a_v,i  = Pi_i sum_{j in g, j != i} [2 eta_i eta_j/(eta_i+eta_j)] (rho_i^-2 + rho_j^-2)
 *                          dW_d(r_ij,h_ij) (v~_i - v~_j) / r_ij                 (Eq. 7, second sum)
 *   v+_i   = v~_i + dt a_v,i,    x+_i = x_i + dt v+_i
 *   curves / surfaces: x+ projected onto the feature, v+ <- Pi(x+) v+;
 *   volume: if phi(x+) < 0 the particle is moved back to phi = 0.01 h_i along grad phi,
 *   its velocity is zeroed and the escape is counted;  h+ = h_t(x+).
 * Singular particles keep their position and zero velocity; the particles of a group that has
 * converged on its own (group_convergence = 1, Algorithm 1) keep position, velocity and h.
 * ------------------------------------------------------------------------------------------ */
void orc_integrate(int64_t n, const orc_domain* dom, const orc_sizing* siz, const orc_params* prm,
                   const orc_ctrl* c, const double* x, const double* h, const int32_t* grp,
                   const double* v, const double* a_p, int64_t n_sub, const int64_t* sub,
                   int32_t use_grid, double* x_out, double* v_out, double* h_out, double* a_v,
                   int64_t* escapes) {
    const int D = dom->D;
    const double kappa = prm->kappa;
    int64_t m = sub ? n_sub : n;
    double* vt = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    for (int64_t j = 0; j < n; ++j) {
        int g = grp[j];
        double dt = c->dt[g];
        for (int a = 0; a < 3; ++a) {
            double vp = c->reset[g] ? 0.0 : c->gf[g] * v[3 * j + a];
            vt[3 * j + a] = vp + dt * (a_p[3 * j + a] - c->geps[g] * vp);
        }
    }
    ugrid u;
    if (use_grid) ugrid_build(&u, n, D, x, h, kappa);
    int64_t esc = 0;
#pragma omp parallel reduction(+ : esc)
    {
        int64_t cap = use_grid ? n : 0;
        int64_t* buf = use_grid ? (int64_t*)malloc(sizeof(int64_t) * (size_t)(cap > 0 ? cap : 1)) : NULL;
#pragma omp for schedule(dynamic, 64)
        for (int64_t s = 0; s < m; ++s) {
            int64_t i = sub ? sub[s] : s;
            int gi = grp[i], d = feat_dim(dom, gi);
            double xo[3], vo[3], av[3] = {0, 0, 0};
            /* a converged group (group_convergence = 1) keeps its state as it is */
            const int frozen = d > 0 && c->gphase[gi] == ORC_DONE;
            for (int a = 0; a < 3; ++a) { xo[a] = x[3 * i + a]; vo[a] = frozen ? v[3 * i + a] : 0; }
            if (d > 0 && !frozen) {
                double dt = c->dt[gi];
                double rci = kappa * h[i];
                double eta_i = pow(h[i], -(double)d) * prm->visc * rci * norm3(vt + 3 * i);
                double ri2 = pow(h[i], 2.0 * d);
                int64_t nc = use_grid ? ugrid_candidates(&u, x + 3 * i, buf, cap) : n;
                for (int64_t cc = 0; cc < nc; ++cc) {
                    int64_t j = use_grid ? buf[cc] : cc;
                    if (j == i || grp[j] != gi) continue;
                    double rij[3] = {0, 0, 0};
                    for (int a = 0; a < D; ++a) rij[a] = x[3 * i + a] - x[3 * j + a];
                    double r = norm3(rij);
                    double hij = 0.5 * (h[i] + h[j]);
                    if (!(r < kappa * hij)) continue;
                    double eta_j = pow(h[j], -(double)d) * prm->visc * kappa * h[j] * norm3(vt + 3 * j);
                    if (eta_i + eta_j == 0) continue;
                    double eb = 2.0 * eta_i * eta_j / (eta_i + eta_j);
                    double coef = eb * (ri2 + pow(h[j], 2.0 * d)) * orc_dW(d, r, hij, kappa) / r;
                    for (int a = 0; a < 3; ++a) av[a] += coef * (vt[3 * i + a] - vt[3 * j + a]);
                }
                orc_tangent(dom, gi, x + 3 * i, av);
                for (int a = 0; a < 3; ++a) {
                    vo[a] = vt[3 * i + a] + dt * av[a];
                    xo[a] = x[3 * i + a] + dt * vo[a];
                }
                if (dom->feat[gi].kind == ORC_VOLUME) {
                    double gph[3];
                    double ph = orc_phi(dom, xo, gph);
                    if (ph < 0) {
                        double target = 0.01 * h[i];
                        for (int it = 0; it < prm->max_newton && ph < target * 0.5; ++it) {
                            double g2 = dot3(gph, gph);
                            for (int a = 0; a < D; ++a) xo[a] += (target - ph) * gph[a] / g2;
                            ph = orc_phi(dom, xo, gph);
                        }
                        for (int a = 0; a < 3; ++a) vo[a] = 0;
                        esc += 1;
                    }
                } else {
                    orc_project(dom, gi, xo);
                    orc_tangent(dom, gi, xo, vo);
                }
            }
            for (int a = 0; a < 3; ++a) {
                x_out[3 * s + a] = xo[a];
                v_out[3 * s + a] = vo[a];
                if (a_v) a_v[3 * s + a] = av[a];
            }
            h_out[s] = (d > 0 && !frozen) ? orc_h(siz, xo) : h[i];
        }
        free(buf);
    }
    if (escapes) *escapes = esc;
    free(vt);
    if (use_grid) ugrid_free(&u);
}

/* n_steps full steps of the relaxation (Jacobi over groups: every group reads state n). */
/* One step in Algorithm 1's feature order (feature_order = 1): the groups are taken class by
 * class in increasing intrinsic dimension (curves, surfaces, volume; singular points never
 * move).  A class's pressure pass reads the positions that the lower classes reached in this
 * step (they act on it as boundary particles, Eq. 19), its groups' controllers run on their own
 * errors (group_convergence), and its viscous pass and update follow; groups of one class do
 * not act on each other, so the order inside a class does not matter. */
static void step_feature_order(int64_t n, const orc_domain* dom, const orc_sizing* siz, const orc_params* prm,
                               orc_ctrl* c, double* x, double* v, double* h, const int32_t* grp, int32_t use_grid,
                               const int32_t* gdim, double* sigma, double* ap, double* x2, double* v2, double* h2,
                               int64_t* sub) {
    const int G = dom->n_feat, D = dom->D;
    group_acc acc = {ORC_DONE, 0, 0.0, 0.0, 0.0};
    for (int d = 1; d <= D; ++d) {
        int64_t m = 0;
        for (int64_t i = 0; i < n; ++i)
            if (gdim[grp[i]] == d) sub[m++] = i;
        double dta[ORC_MAX_FEAT], dtv[ORC_MAX_FEAT], Vsum[ORC_MAX_FEAT];
        for (int g = 0; g < G; ++g) { dta[g] = INFINITY; dtv[g] = INFINITY; Vsum[g] = 0; }
        if (m > 0) {
            orc_interact(n, dom, prm, x, h, grp, v, m, sub, use_grid, sigma, NULL, NULL, ap, NULL, dta, dtv);
            for (int64_t s = 0; s < m; ++s)
                if (sigma[s] > 0) Vsum[grp[sub[s]]] += 1.0 / sigma[s];
        }
        group_pass(prm, G, gdim, Vsum, dta, dtv, c, d, &acc);
        if (m == 0) continue;
        /* the viscous pass reads a_p of the class's particles by particle index */
        double* ap_full = x2;   /* scratch: 3n doubles */
        for (int64_t s = 0; s < m; ++s)
            for (int a = 0; a < 3; ++a) ap_full[3 * sub[s] + a] = ap[3 * s + a];
        int64_t esc = 0;
        double* xo = ap;        /* scratch reuse: 3m doubles each */
        orc_integrate(n, dom, siz, prm, c, x, h, grp, v, ap_full, m, sub, use_grid, xo, v2, h2, NULL, &esc);
        for (int64_t s = 0; s < m; ++s) {
            for (int a = 0; a < 3; ++a) {
                x[3 * sub[s] + a] = xo[3 * s + a];
                v[3 * sub[s] + a] = v2[3 * s + a];
            }
            h[sub[s]] = h2[s];
        }
        c->escapes += esc;
    }
    group_summary(c, &acc);
    c->n += 1;
}

void orc_step(int64_t n, const orc_domain* dom, const orc_sizing* siz, const orc_params* prm,
              orc_ctrl* c, double* x, double* v, double* h, const int32_t* grp,
              int32_t use_grid, int32_t n_steps) {
    const int G = dom->n_feat;
    int32_t gdim[ORC_MAX_FEAT];
    for (int g = 0; g < G; ++g) gdim[g] = dom->feat[g].dim;
    size_t nn = (size_t)(n > 0 ? n : 1);
    if (prm->feature_order == 1) {
        double* sigma = (double*)malloc(sizeof(double) * nn);
        double* ap = (double*)malloc(sizeof(double) * 3 * nn);
        double* x2 = (double*)malloc(sizeof(double) * 3 * nn);
        double* v2 = (double*)malloc(sizeof(double) * 3 * nn);
        double* h2 = (double*)malloc(sizeof(double) * nn);
        int64_t* sub = (int64_t*)malloc(sizeof(int64_t) * nn);
        for (int s = 0; s < n_steps && c->phase != ORC_DONE; ++s)
            step_feature_order(n, dom, siz, prm, c, x, v, h, grp, use_grid, gdim, sigma, ap, x2, v2, h2, sub);
        free(sigma); free(ap); free(x2); free(v2); free(h2); free(sub);
        return;
    }
    double* sigma = (double*)malloc(sizeof(double) * nn);
    double* ap = (double*)malloc(sizeof(double) * 3 * nn);
    double* x2 = (double*)malloc(sizeof(double) * 3 * nn);
    double* v2 = (double*)malloc(sizeof(double) * 3 * nn);
    double* h2 = (double*)malloc(sizeof(double) * nn);
    for (int s = 0; s < n_steps; ++s) {
        double dta[ORC_MAX_FEAT], dtv[ORC_MAX_FEAT], Vsum[ORC_MAX_FEAT];
        orc_interact(n, dom, prm, x, h, grp, v, 0, NULL, use_grid, sigma, NULL, NULL, ap, NULL, dta, dtv);
        for (int g = 0; g < G; ++g) Vsum[g] = 0;
        for (int64_t i = 0; i < n; ++i)
            if (sigma[i] > 0) Vsum[grp[i]] += 1.0 / sigma[i];
        orc_control(prm, G, gdim, Vsum, dta, dtv, c);
        if (c->phase == ORC_DONE) break;
        int64_t esc = 0;
        orc_integrate(n, dom, siz, prm, c, x, h, grp, v, ap, 0, NULL, use_grid, x2, v2, h2, NULL, &esc);
        memcpy(x, x2, sizeof(double) * 3 * (size_t)n);
        memcpy(v, v2, sizeof(double) * 3 * (size_t)n);
        memcpy(h, h2, sizeof(double) * (size_t)n);
        c->escapes += esc;
        c->n += 1;
    }
    free(sigma); free(ap); free(x2); free(v2); free(h2);
}

/* ------------------------------------------------------------------------------------------
 * Initial particle sampling (Sec. 3.6): particles of feature k are drawn at random with
 * probability proportional to the target density rho_t = h_t^-d, by rejection.  The random
 * numbers come from a counter-based generator, so that any candidate's numbers can be drawn
 * on their own: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC 2011) -- ten rounds of its S-box on a 128-bit counter under a 64-bit key,
 * the key advanced by the two Weyl constants between rounds.
 * ------------------------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0, hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Candidate c of feature k: counter (c low word, c high word, k, 0), key = the seed's two words;
 * its four numbers as uniforms in (0, 1): u = (x + 1/2) 2^-32 (exact in FP64). */
static void candidate_uniforms(uint64_t seed, int k, int64_t c, double u[4]) {
    uint32_t ctr[4] = {(uint32_t)c, (uint32_t)((uint64_t)c >> 32), (uint32_t)k, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    for (int a = 0; a < 4; ++a) u[a] = ((double)o[a] + 0.5) * (1.0 / 4294967296.0);
}

/* Whether candidate u of feature k is accepted, and its position.  Acceptance probability
 * (h_min/h_t(x))^d, h_min the sizing's lower bound:
 *   VOLUME  x uniform in the bounding box; also phi(x) > h_t(x)/4 (away from the boundary);
 *   SEGMENT x = a + u0 (b - a);
 *   CIRCLE / SPHERE  p = 2u - 1 (2 or 3 components) kept when 0 < |p|^2 <= 1, x = c + r p/|p|;
 *   RECT    (s, t) = (u0 l_u, u1 l_w), kept at least h_t(x)/4 inside the face's edges,
 *           x = o + s e_u + t e_w;
 *   POINT   the point itself. */
static int candidate_accept(const orc_domain* dom, const orc_sizing* s, int k, const double u[4], double x[3]) {
    const orc_feature* f = &dom->feat[k];
    const int D = dom->D;
    x[0] = x[1] = x[2] = 0.0;
    double h, acc;
    switch (f->kind) {
        case ORC_VOLUME: {
            for (int a = 0; a < D; ++a) x[a] = dom->lo[a] + u[a] * (dom->hi[a] - dom->lo[a]);
            h = orc_h(s, x);
            if (!(orc_phi(dom, x, NULL) > 0.25 * h)) return 0;
            double r = s->lo / h;
            double rd = r * r;
            if (D == 3) rd = rd * r;
            return u[3] < rd;
        }
        case ORC_SEGMENT:
            for (int a = 0; a < 3; ++a) x[a] = f->p[a] + u[0] * (f->p[3 + a] - f->p[a]);
            h = orc_h(s, x);
            return u[1] < s->lo / h;
        case ORC_CIRCLE: {
            double p0 = 2.0 * u[0] - 1.0, p1 = 2.0 * u[1] - 1.0;
            double q = p0 * p0 + p1 * p1;
            if (!(q > 0.0 && q <= 1.0)) return 0;
            double r = sqrt(q);
            x[0] = f->p[0] + f->p[2] * (p0 / r);
            x[1] = f->p[1] + f->p[2] * (p1 / r);
            h = orc_h(s, x);
            return u[2] < s->lo / h;
        }
        case ORC_SPHERE: {
            double p0 = 2.0 * u[0] - 1.0, p1 = 2.0 * u[1] - 1.0, p2 = 2.0 * u[2] - 1.0;
            double q = (p0 * p0 + p1 * p1) + p2 * p2;
            if (!(q > 0.0 && q <= 1.0)) return 0;
            double r = sqrt(q);
            x[0] = f->p[0] + f->p[3] * (p0 / r);
            x[1] = f->p[1] + f->p[3] * (p1 / r);
            x[2] = f->p[2] + f->p[3] * (p2 / r);
            h = orc_h(s, x);
            acc = s->lo / h;
            return u[3] < acc * acc;
        }
        case ORC_RECT: {
            double sv = u[0] * f->p[9], tv = u[1] * f->p[10];
            for (int a = 0; a < 3; ++a) x[a] = (f->p[a] + sv * f->p[3 + a]) + tv * f->p[6 + a];
            h = orc_h(s, x);
            double m = 0.25 * h;
            if (!(sv > m && sv < f->p[9] - m && tv > m && tv < f->p[10] - m)) return 0;
            acc = s->lo / h;
            return u[2] < acc * acc;
        }
        default: /* ORC_POINT */
            for (int a = 0; a < D; ++a) x[a] = f->p[a];
            return 1;
    }
}

int64_t orc_sample_feature(const orc_domain* dom, const orc_sizing* s, int k, uint64_t seed, int64_t n,
                           double* x_out) {
    int64_t got = 0, c = 0;
    while (got < n) {
        double u[4], x[3];
        candidate_uniforms(seed, k, c, u);
        if (candidate_accept(dom, s, k, u, x)) {
            for (int a = 0; a < 3; ++a) x_out[3 * got + a] = x[a];
            ++got;
        }
        ++c;
    }
    return c;
}
