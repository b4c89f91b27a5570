/*
 * idugks_oracle.c -- plain, slow, FP64 CPU oracle of explicit DUGKS and of one
 * IDUGKS iteration (Pan, Zhong & Zhuo, arXiv 1709.01819, Section 2).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, by the smoke check and by the
 * CPU baseline leg of the benchmark, never by the product path.  It shares no
 * code with the CUDA library.  Every step follows the paper's order and
 * notation with plain loops; OpenMP only splits independent velocities (or
 * independent faces/cells), every sum runs serially in a fixed order, so the
 * result does not depend on the thread count.
 *
 * Readings of the paper taken here (the GPU library takes the same ones):
 *  - reduced distributions G = int f dxi, H = int xi^2 f dxi (Eq. 5), K internal dof;
 *  - Shakhov reduced equilibria derived from the full Shakhov model for
 *    D = 2 + K degrees of freedom (Eq. 20 prints a garbled H line):
 *      P   = (1-Pr) (c.q) / ((D+2) p RT)
 *      G^S = G^eq [1 + P (c^2/RT - 4)],  H^S = H^eq [1 + P (c^2/RT - 2)];
 *  - f-bar-plus from the stored f-tilde (Eq. 10 inverted, then Eq. 12):
 *      fb+ = (2tau - h)/(2tau + dt) f~ + 3h/(2tau + dt) f^S,  h = dt/2;
 *  - heat flux of f from the transformed distributions: q = 2 tau q~ /(2 tau + dt Pr)
 *    at cells and q = 2 tau qbar/(2 tau + h Pr) at faces;
 *  - Eq. (22)-(23): the collision residual is -(2 Omega/(2 tau + dt)) (f~ - f^S);
 *  - Eq. (30): matrix-free LU-SGS with off-diagonal 1/2 (dF S - w Lambda dW),
 *    w = 2 by default, Lambda = (|V.n| + c) S at the face average;
 *  - the point relaxation the conclusions name as the other predictor (no
 *    equation printed): Jacobi sweeps on the same predictor equations
 *    D dW_c + sum_nb 1/2 (dF_nb S - w Lambda dW_nb) = R_c, from dW = 0;
 *  - diffuse wall (Eq. 34-35 in non-delta form) on f-bar with zero net mass
 *    flux; the mass component of the wall flux moment is set to zero;
 *  - ghost increments are zero in both sweeps (end of Section 2.3), or, with
 *    implicit_wall, the wall ghost of Eq. (34)-(35) built from the inner
 *    cell's increment of the previous iteration (zero after a restart).
 */
#include "idugks_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int L, R;            /* cells on each side (-1 = ghost)                     */
    double nx, ny, S;    /* unit normal from L to R, length                      */
    double rLx, rLy;     /* face midpoint minus L centroid (L's copy of the face) */
    double rRx, rRy;     /* face midpoint minus R centroid                        */
    int bc, side;        /* boundary kind / side for ghost faces, -1 otherwise    */
} orc_face;

struct orc_state {
    orc_problem p;
    double *nodes_x, *nodes_y;
    int N, Nv, nf;
    /* geometry */
    double *cx, *cy, *area, *hcell, *dtimp;
    orc_face *face;
    int *cell_face;     /* [N][4]: west, east, south, north face index (structured);
                           unstructured: the edges node m -> m+1 */
    int *nslot;         /* [N] faces of the cell (4; 3 for a triangle) */
    int *cell_sign;     /* [N][4]: +1 if the cell is L of that face, -1 if R */
    double *lsinv;      /* [N][4] inverse of the 2x2 least-squares matrix (row-major) */
    /* velocity space */
    double *ux, *uy, *w;
    double xi_max, dt, h, mu_ref, gam;
    /* state */
    double *G, *H, *W;
    /* work */
    double *fbG, *fbH, *grG, *grH, *limG, *limH;
    double *FG, *FH, *phi, *rw, *qcell, *tau;
    double *RG, *RH, *Dm, *dG, *dH, *dW;
    double *eqG, *eqH;  /* per-thread scratch is avoided: [N][Nv] equilibria */
};

/* ------------------------------------------------------------------------- */
/* quadrature (Section 2.2 closing paragraph: Gauss-Hermite or Newton-Cotes)  */
/* ------------------------------------------------------------------------- */

/* orthonormal Hermite polynomials p_0..p_n at x for the weight exp(-x^2) */
static void hermite_orthonormal(int n, double x, double *pk)
{
    pk[0] = pow(M_PI, -0.25);
    if (n >= 1) pk[1] = sqrt(2.0) * x * pk[0];
    for (int k = 1; k < n; ++k)
        pk[k + 1] = sqrt(2.0 / (k + 1)) * x * pk[k] - sqrt((double)k / (k + 1)) * pk[k - 1];
}

/* Gauss-Hermite nodes (roots of H_n) found by a sign scan plus bisection, and
 * Christoffel weights 1 / sum_{k<n} p_k(x)^2.  Returns weights for exp(-x^2). */
static int gauss_hermite(int n, double *x, double *wt)
{
    if (n < 1 || n > 400) return -1;
    double *pk = (double *)malloc(sizeof(double) * (n + 1));
    double lim = sqrt(2.0 * n + 1.0) + 1.0;
    double step = 1e-3;
    int found = 0;
    hermite_orthonormal(n, -lim, pk);
    double xa = -lim, fa = pk[n];
    for (double xb = -lim + step; xb <= lim + 0.5 * step && found < n; xb += step) {
        hermite_orthonormal(n, xb, pk);
        double fb = pk[n];
        if (fa == 0.0) { x[found++] = xa; }
        else if (fa * fb < 0.0) {
            double lo = xa, hi = xb, flo = fa;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi);
                if (mid == lo || mid == hi) break;
                hermite_orthonormal(n, mid, pk);
                if (flo * pk[n] <= 0.0) hi = mid; else { lo = mid; flo = pk[n]; }
            }
            x[found++] = 0.5 * (lo + hi);
        }
        xa = xb; fa = fb;
    }
    if (found != n) { free(pk); return -2; }
    /* the roots are symmetric: average the pairs so the rule is exactly symmetric */
    for (int i = 0; i < n / 2; ++i) {
        double a = 0.5 * (x[n - 1 - i] - x[i]);
        x[i] = -a; x[n - 1 - i] = a;
    }
    if (n % 2) x[n / 2] = 0.0;
    for (int i = 0; i < n; ++i) {
        hermite_orthonormal(n, x[i], pk);
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += pk[k] * pk[k];
        wt[i] = 1.0 / s;
    }
    for (int i = 0; i < n / 2; ++i) {
        double a = 0.5 * (wt[i] + wt[n - 1 - i]);
        wt[i] = a; wt[n - 1 - i] = a;
    }
    free(pk);
    return 0;
}

/* 1-D rule on [a, b].  Trapezoid: closed 2-point Newton-Cotes, composite.
 * Simpson: composite, n odd.  Gauss-Hermite: xi = b * x, w = b * W e^{x^2}
 * (b is the velocity unit sqrt(2 RT_ref); a is ignored).  Returns 0 on success. */
int orc_quadrature(int rule, int n, double a, double b, double *x, double *w)
{
    if (rule == ORC_NC_TRAP) {
        if (n < 2) return -1;
        double hh = (b - a) / (n - 1);
        for (int i = 0; i < n; ++i) {
            x[i] = a + hh * i;
            w[i] = (i == 0 || i == n - 1) ? 0.5 * hh : hh;
        }
        /* exact symmetry of the nodes about the midpoint */
        for (int i = 0; i < n / 2; ++i) {
            double m = 0.5 * (a + b), d = 0.5 * ((x[n - 1 - i] - m) - (x[i] - m));
            x[i] = m - d; x[n - 1 - i] = m + d;
        }
        return 0;
    }
    if (rule == ORC_NC_SIMPSON) {
        if (n < 3 || n % 2 == 0) return -1;
        double hh = (b - a) / (n - 1);
        for (int i = 0; i < n; ++i) {
            x[i] = a + hh * i;
            if (i == 0 || i == n - 1) w[i] = hh / 3.0;
            else w[i] = (i % 2) ? 4.0 * hh / 3.0 : 2.0 * hh / 3.0;
        }
        for (int i = 0; i < n / 2; ++i) {
            double m = 0.5 * (a + b), d = 0.5 * ((x[n - 1 - i] - m) - (x[i] - m));
            x[i] = m - d; x[n - 1 - i] = m + d;
        }
        if (n % 2) x[n / 2] = 0.5 * (a + b);
        return 0;
    }
    if (rule == ORC_GAUSS_HERMITE) {
        if (b <= 0.0) return -1;
        int rc = gauss_hermite(n, x, w);
        if (rc) return rc;
        for (int i = 0; i < n; ++i) {
            w[i] = b * w[i] * exp(x[i] * x[i]);
            x[i] = b * x[i];
        }
        return 0;
    }
    return -1;
}

/* ------------------------------------------------------------------------- */
/* kinetic model: Eq. (2), (4), (5), (20)                                     */
/* ------------------------------------------------------------------------- */

static double viscosity(const orc_state *s, double RT)
{
    /* mu = mu_ref (T/T_ref)^omega; mu_ref from the VHS mean free path (Eq. 36) */
    return s->mu_ref * pow(RT / s->p.RT_ref, s->p.omega);
}

static void primitives(const orc_state *s, const double *W, double *rho, double *U,
                       double *V, double *RT)
{
    /* Eq. (4): rho E = 1/2 rho (U^2 + V^2 + (K+2) RT), lambda = 1/(2RT) */
    *rho = W[0];
    *U = W[1] / W[0];
    *V = W[2] / W[0];
    *RT = (2.0 * W[3] / W[0] - (*U) * (*U) - (*V) * (*V)) / (s->p.K + 2);
}

/* Reduced Maxwellian (Eq. 2 integrated over the K internal dof, Eq. 5) with the
 * Shakhov correction (Eq. 20, reading given in the header), at every discrete
 * velocity.  Optional discrete mass normalisation of the Maxwellian part. */
static void equilibrium(const orc_state *s, double rho, double U, double V, double RT,
                        double qx, double qy, double *G, double *H)
{
    const int Nv = s->Nv, K = s->p.K;
    const double lam = 1.0 / (2.0 * RT);
    double mass = 0.0;
    for (int k = 0; k < Nv; ++k) {
        double cx = s->ux[k] - U, cy = s->uy[k] - V;
        G[k] = rho * (lam / M_PI) * exp(-lam * (cx * cx + cy * cy));
        mass += s->w[k] * G[k];
    }
    double scale = 1.0;
    if (s->p.flags & ORC_FLAG_FEQ_MASS_NORMALIZE) scale = rho / mass;
    const int D = 2 + K;
    const double p = rho * RT;
    for (int k = 0; k < Nv; ++k) {
        double cx = s->ux[k] - U, cy = s->uy[k] - V, c2 = cx * cx + cy * cy;
        double g = G[k] * scale;
        double hq = K * RT * g;
        double gs = g, hs = hq;
        if (s->p.shakhov) {
            double P = (1.0 - s->p.Pr) * (cx * qx + cy * qy) / ((D + 2) * p * RT);
            gs = g * (1.0 + P * (c2 / RT - 4.0));
            hs = hq * (1.0 + P * (c2 / RT - 2.0));
        }
        G[k] = gs;
        H[k] = hs;
    }
}

void orc_equilibrium(const orc_state *s, double rho, double u, double v, double RT,
                     double qx, double qy, double *G, double *H)
{
    equilibrium(s, rho, u, v, RT, qx, qy, G, H);
}

/* conserved moments of (G, H), Eq. (4) */
static void moments_W(const orc_state *s, const double *G, const double *H, double *W)
{
    double m0 = 0, m1 = 0, m2 = 0, m3 = 0;
    for (int k = 0; k < s->Nv; ++k) {
        double wk = s->w[k], ux = s->ux[k], uy = s->uy[k];
        m0 += wk * G[k];
        m1 += wk * ux * G[k];
        m2 += wk * uy * G[k];
        m3 += 0.5 * wk * ((ux * ux + uy * uy) * G[k] + H[k]);
    }
    W[0] = m0; W[1] = m1; W[2] = m2; W[3] = m3;
}

/* heat flux q = 1/2 sum w c (c^2 G + H), c = xi - U */
static void heat_flux(const orc_state *s, const double *G, const double *H, double U,
                      double V, double *qx, double *qy)
{
    double ax = 0, ay = 0;
    for (int k = 0; k < s->Nv; ++k) {
        double cx = s->ux[k] - U, cy = s->uy[k] - V, c2 = cx * cx + cy * cy;
        double e = c2 * G[k] + H[k];
        ax += 0.5 * s->w[k] * cx * e;
        ay += 0.5 * s->w[k] * cy * e;
    }
    *qx = ax; *qy = ay;
}

double orc_venkat_theta(double x)
{
    /* Eq. (17) */
    return (x * x + 2.0 * x) / (x * x + x + 2.0);
}

/* ------------------------------------------------------------------------- */
/* geometry of the structured block                                           */
/* ------------------------------------------------------------------------- */

static int nfi_row(const orc_state *s) { return s->p.bc_kind[ORC_IMIN] == ORC_BC_PERIODIC ? s->p.ni : s->p.ni + 1; }
static int nfj_rows(const orc_state *s) { return s->p.bc_kind[ORC_JMIN] == ORC_BC_PERIODIC ? s->p.nj : s->p.nj + 1; }
static int iface_index(const orc_state *s, int i, int j) { return j * nfi_row(s) + i; }
static int jface_index(const orc_state *s, int i, int j) { return s->p.nj * nfi_row(s) + j * s->p.ni + i; }

static double NX(const orc_state *s, int i, int j) { return s->nodes_x[j * (s->p.ni + 1) + i]; }
static double NY(const orc_state *s, int i, int j) { return s->nodes_y[j * (s->p.ni + 1) + i]; }

static void finish_geometry(orc_state *s);

static void build_geometry(orc_state *s)
{
    const int ni = s->p.ni, nj = s->p.nj;
    for (int c = 0; c < s->N; ++c) s->nslot[c] = 4;
    const int per_i = s->p.bc_kind[ORC_IMIN] == ORC_BC_PERIODIC;
    const int per_j = s->p.bc_kind[ORC_JMIN] == ORC_BC_PERIODIC;
    /* cells: area by the polygon (shoelace) formula, centroid of the polygon,
     * in coordinates relative to the cell's first node (the formulas are
     * translation invariant; in absolute coordinates a small cell far from
     * the origin would lose ~eps |x|^2 / area to cancellation) */
    for (int j = 0; j < nj; ++j)
        for (int i = 0; i < ni; ++i) {
            const double ox = NX(s, i, j), oy = NY(s, i, j);
            double px[4] = {0.0, NX(s, i + 1, j) - ox, NX(s, i + 1, j + 1) - ox, NX(s, i, j + 1) - ox};
            double py[4] = {0.0, NY(s, i + 1, j) - oy, NY(s, i + 1, j + 1) - oy, NY(s, i, j + 1) - oy};
            double a = 0, gx = 0, gy = 0;
            for (int m = 0; m < 4; ++m) {
                int n2 = (m + 1) % 4;
                double cr = px[m] * py[n2] - px[n2] * py[m];
                a += 0.5 * cr;
                gx += (px[m] + px[n2]) * cr;
                gy += (py[m] + py[n2]) * cr;
            }
            int c = j * ni + i;
            s->area[c] = a;
            s->cx[c] = ox + gx / (6.0 * a);
            s->cy[c] = oy + gy / (6.0 * a);
        }
    /* faces */
    int f = 0;
    for (int j = 0; j < nj; ++j)
        for (int i = 0; i < nfi_row(s); ++i, ++f) {
            orc_face *F = &s->face[f];
            double x0 = NX(s, i, j), y0 = NY(s, i, j), x1 = NX(s, i, j + 1), y1 = NY(s, i, j + 1);
            double tx = x1 - x0, ty = y1 - y0, S = sqrt(tx * tx + ty * ty);
            F->S = S; F->nx = ty / S; F->ny = -tx / S;
            double mx = 0.5 * (x0 + x1), my = 0.5 * (y0 + y1);
            F->bc = -1; F->side = -1;
            if (per_i) {
                F->L = j * ni + (i + ni - 1) % ni;
                F->R = j * ni + i;
                /* L's copy of a wrapped face sits on node column ni */
                double mxL = mx, myL = my;
                if (i == 0) {
                    mxL = 0.5 * (NX(s, ni, j) + NX(s, ni, j + 1));
                    myL = 0.5 * (NY(s, ni, j) + NY(s, ni, j + 1));
                }
                F->rLx = mxL - s->cx[F->L]; F->rLy = myL - s->cy[F->L];
                F->rRx = mx - s->cx[F->R]; F->rRy = my - s->cy[F->R];
            } else {
                F->L = (i > 0) ? j * ni + i - 1 : -1;
                F->R = (i < ni) ? j * ni + i : -1;
                if (F->L < 0) { F->bc = s->p.bc_kind[ORC_IMIN]; F->side = ORC_IMIN; }
                if (F->R < 0) { F->bc = s->p.bc_kind[ORC_IMAX]; F->side = ORC_IMAX; }
                if (F->L >= 0) { F->rLx = mx - s->cx[F->L]; F->rLy = my - s->cy[F->L]; } else { F->rLx = F->rLy = 0; }
                if (F->R >= 0) { F->rRx = mx - s->cx[F->R]; F->rRy = my - s->cy[F->R]; } else { F->rRx = F->rRy = 0; }
            }
        }
    for (int j = 0; j < nfj_rows(s); ++j)
        for (int i = 0; i < ni; ++i, ++f) {
            orc_face *F = &s->face[f];
            double x0 = NX(s, i, j), y0 = NY(s, i, j), x1 = NX(s, i + 1, j), y1 = NY(s, i + 1, j);
            double tx = x1 - x0, ty = y1 - y0, S = sqrt(tx * tx + ty * ty);
            F->S = S; F->nx = -ty / S; F->ny = tx / S;
            double mx = 0.5 * (x0 + x1), my = 0.5 * (y0 + y1);
            F->bc = -1; F->side = -1;
            if (per_j) {
                F->L = ((j + nj - 1) % nj) * ni + i;
                F->R = j * ni + i;
                double mxL = mx, myL = my;
                if (j == 0) {
                    mxL = 0.5 * (NX(s, i, nj) + NX(s, i + 1, nj));
                    myL = 0.5 * (NY(s, i, nj) + NY(s, i + 1, nj));
                }
                F->rLx = mxL - s->cx[F->L]; F->rLy = myL - s->cy[F->L];
                F->rRx = mx - s->cx[F->R]; F->rRy = my - s->cy[F->R];
            } else {
                F->L = (j > 0) ? (j - 1) * ni + i : -1;
                F->R = (j < nj) ? j * ni + i : -1;
                if (F->L < 0) { F->bc = s->p.bc_kind[ORC_JMIN]; F->side = ORC_JMIN; }
                if (F->R < 0) { F->bc = s->p.bc_kind[ORC_JMAX]; F->side = ORC_JMAX; }
                if (F->L >= 0) { F->rLx = mx - s->cx[F->L]; F->rLy = my - s->cy[F->L]; } else { F->rLx = F->rLy = 0; }
                if (F->R >= 0) { F->rRx = mx - s->cx[F->R]; F->rRy = my - s->cy[F->R]; } else { F->rRx = F->rRy = 0; }
            }
        }
    /* cell -> faces: west, east, south, north */
    for (int j = 0; j < nj; ++j)
        for (int i = 0; i < ni; ++i) {
            int c = j * ni + i;
            s->cell_face[4 * c + 0] = iface_index(s, i, j);
            s->cell_sign[4 * c + 0] = -1;
            s->cell_face[4 * c + 1] = iface_index(s, per_i ? (i + 1) % ni : i + 1, j);
            s->cell_sign[4 * c + 1] = +1;
            s->cell_face[4 * c + 2] = jface_index(s, i, j);
            s->cell_sign[4 * c + 2] = -1;
            s->cell_face[4 * c + 3] = jface_index(s, i, per_j ? (j + 1) % nj : j + 1);
            s->cell_sign[4 * c + 3] = +1;
        }
    finish_geometry(s);
}

/* node pair of a cell edge, for matching the two cells of an interior edge */
typedef struct {
    int a, b, cell, slot;
} orc_edge;

static int edge_cmp(const void *x, const void *y)
{
    const orc_edge *p = (const orc_edge *)x, *q = (const orc_edge *)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    if (p->cell != q->cell) return p->cell < q->cell ? -1 : 1;
    return p->slot - q->slot;
}

/* Unstructured block of triangles and quadrilaterals (nodes counter-clockwise).
 * Face f between the two cells sharing an edge; L is the cell that runs along
 * the edge counter-clockwise first in cell order (its outward normal is the
 * face normal), R the other one or -1 on the boundary.  Slot m of a cell is
 * its edge node m -> m+1.  Faces are numbered in order of first appearance
 * (cell by cell, slot by slot).  Returns 0, or -1 for a malformed mesh (an edge
 * shared by more than two cells or twice in one direction, a cell of
 * non-positive area, a boundary group out of range or periodic). */
static int build_geometry_unstructured(orc_state *s)
{
    const orc_problem *p = &s->p;
    const int N = p->n_ucells;
    int ne = 0;
    for (int c = 0; c < N; ++c) {
        int k = p->ucell_nodes[4 * c + 3] < 0 ? 3 : 4;
        s->nslot[c] = k;
        /* shoelace area and polygon centroid relative to the first node */
        const int o0 = p->ucell_nodes[4 * c];
        if (o0 < 0 || o0 >= p->n_unodes) return -1;
        const double ox = s->nodes_x[o0], oy = s->nodes_y[o0];
        double a = 0, gx = 0, gy = 0;
        for (int m = 0; m < k; ++m) {
            int n0 = p->ucell_nodes[4 * c + m], n1 = p->ucell_nodes[4 * c + (m + 1) % k];
            if (n0 < 0 || n1 < 0 || n0 >= p->n_unodes || n1 >= p->n_unodes || n0 == n1) return -1;
            double x0 = s->nodes_x[n0] - ox, y0 = s->nodes_y[n0] - oy;
            double x1 = s->nodes_x[n1] - ox, y1 = s->nodes_y[n1] - oy;
            double cr = x0 * y1 - x1 * y0;
            a += 0.5 * cr;
            gx += (x0 + x1) * cr;
            gy += (y0 + y1) * cr;
        }
        if (!(a > 0)) return -1;
        s->area[c] = a;
        s->cx[c] = ox + gx / (6.0 * a);
        s->cy[c] = oy + gy / (6.0 * a);
        ne += k;
    }
    orc_edge *E = (orc_edge *)malloc(sizeof(orc_edge) * (size_t)ne);
    int q = 0;
    for (int c = 0; c < N; ++c)
        for (int m = 0; m < s->nslot[c]; ++m) {
            int n0 = p->ucell_nodes[4 * c + m], n1 = p->ucell_nodes[4 * c + (m + 1) % s->nslot[c]];
            E[q].a = n0 < n1 ? n0 : n1;
            E[q].b = n0 < n1 ? n1 : n0;
            E[q].cell = c;
            E[q].slot = m;
            ++q;
        }
    qsort(E, (size_t)ne, sizeof(orc_edge), edge_cmp);
    /* partner of each cell slot (-1: boundary) */
    int *partner = (int *)malloc(sizeof(int) * 4 * (size_t)N);
    for (int i = 0; i < 4 * N; ++i) partner[i] = -1;
    for (int i = 0; i < ne;) {
        int j = i + 1;
        while (j < ne && E[j].a == E[i].a && E[j].b == E[i].b) ++j;
        if (j - i > 2) { free(E); free(partner); return -1; }
        if (j - i == 2) {
            partner[4 * E[i].cell + E[i].slot] = 4 * E[i + 1].cell + E[i + 1].slot;
            partner[4 * E[i + 1].cell + E[i + 1].slot] = 4 * E[i].cell + E[i].slot;
        }
        i = j;
    }
    free(E);
    int nf = 0;
    for (int i = 0; i < 4 * N; ++i) s->cell_face[i] = -1;
    for (int c = 0; c < N; ++c)
        for (int m = 0; m < s->nslot[c]; ++m) {
            if (s->cell_face[4 * c + m] >= 0) continue; /* the partner created it */
            int k = s->nslot[c];
            int n0 = p->ucell_nodes[4 * c + m], n1 = p->ucell_nodes[4 * c + (m + 1) % k];
            orc_face *F = &s->face[nf];
            double x0 = s->nodes_x[n0], y0 = s->nodes_y[n0], x1 = s->nodes_x[n1], y1 = s->nodes_y[n1];
            double tx = x1 - x0, ty = y1 - y0, S = sqrt(tx * tx + ty * ty);
            double mx = 0.5 * (x0 + x1), my = 0.5 * (y0 + y1);
            F->S = S; F->nx = ty / S; F->ny = -tx / S; /* outward of c (counter-clockwise) */
            F->L = c;
            F->rLx = mx - s->cx[c]; F->rLy = my - s->cy[c];
            F->bc = -1; F->side = -1;
            s->cell_face[4 * c + m] = nf;
            s->cell_sign[4 * c + m] = +1;
            int pr = partner[4 * c + m];
            if (pr >= 0) {
                int c2 = pr / 4, m2 = pr % 4, k2 = s->nslot[c2];
                /* the neighbour must run along the edge the other way */
                if (p->ucell_nodes[4 * c2 + m2] != n1 || p->ucell_nodes[4 * c2 + (m2 + 1) % k2] != n0) {
                    free(partner); return -1;
                }
                F->R = c2;
                F->rRx = mx - s->cx[c2]; F->rRy = my - s->cy[c2];
                s->cell_face[pr] = nf;
                s->cell_sign[pr] = -1;
            } else {
                int side = p->uedge_side[4 * c + m];
                if (side < 0 || side > 3 || p->bc_kind[side] == ORC_BC_PERIODIC) { free(partner); return -1; }
                F->R = -1;
                F->rRx = F->rRy = 0;
                F->bc = p->bc_kind[side];
                F->side = side;
            }
            ++nf;
        }
    free(partner);
    s->nf = nf;
    /* a triangle's unused slot 3 keeps a valid face index; nslot excludes it */
    for (int c = 0; c < N; ++c)
        if (s->nslot[c] == 3) { s->cell_face[4 * c + 3] = s->cell_face[4 * c]; s->cell_sign[4 * c + 3] = 0; }
    finish_geometry(s);
    return 0;
}

/* cell size, pseudo time step, least-squares matrices (Eq. 15) */
static void finish_geometry(orc_state *s)
{
    double hmin = 1e300;
    for (int c = 0; c < s->N; ++c) {
        double smax = 0;
        double a11 = 0, a12 = 0, a22 = 0;
        for (int m = 0; m < s->nslot[c]; ++m) {
            const orc_face *F = &s->face[s->cell_face[4 * c + m]];
            if (F->S > smax) smax = F->S;
            if (F->L < 0 || F->R < 0) continue; /* one-sided at boundaries */
            int sg = s->cell_sign[4 * c + m];
            double dx = sg > 0 ? F->rLx - F->rRx : F->rRx - F->rLx;
            double dy = sg > 0 ? F->rLy - F->rRy : F->rRy - F->rLy;
            a11 += dx * dx; a12 += dx * dy; a22 += dy * dy;
        }
        double det = a11 * a22 - a12 * a12;
        if (!(det > 1e-10 * (a11 + a22) * (a11 + a22))) {
            /* fewer than two neighbours in independent directions (a mesh
             * corner of triangles): no gradient, first-order reconstruction */
            for (int q = 0; q < 4; ++q) s->lsinv[4 * c + q] = 0.0;
        } else {
            s->lsinv[4 * c + 0] = a22 / det;
            s->lsinv[4 * c + 1] = -a12 / det;
            s->lsinv[4 * c + 2] = -a12 / det;
            s->lsinv[4 * c + 3] = a11 / det;
        }
        s->hcell[c] = s->area[c] / smax;
        if (s->hcell[c] < hmin) hmin = s->hcell[c];
    }
    s->dt = s->p.cfl_phys * hmin / s->xi_max;
    s->h = 0.5 * s->dt;
    for (int c = 0; c < s->N; ++c) s->dtimp[c] = s->p.cfl_imp * s->hcell[c] / s->xi_max;
}

/* ------------------------------------------------------------------------- */

static double *dalloc(size_t n) { return (double *)calloc(n ? n : 1, sizeof(double)); }

orc_state *orc_create(const orc_problem *p)
{
    const int unstructured = p->n_ucells > 0;
    if (unstructured) {
        if (p->n_unodes < 3 || !p->ucell_nodes || !p->uedge_side) return NULL;
    } else {
        if (p->ni < 1 || p->nj < 1) return NULL;
        if ((p->bc_kind[ORC_IMIN] == ORC_BC_PERIODIC) != (p->bc_kind[ORC_IMAX] == ORC_BC_PERIODIC)) return NULL;
        if ((p->bc_kind[ORC_JMIN] == ORC_BC_PERIODIC) != (p->bc_kind[ORC_JMAX] == ORC_BC_PERIODIC)) return NULL;
    }
    orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
    s->p = *p;
    size_t nn = unstructured ? (size_t)p->n_unodes : (size_t)(p->ni + 1) * (p->nj + 1);
    s->nodes_x = dalloc(nn); s->nodes_y = dalloc(nn);
    memcpy(s->nodes_x, p->nodes_x, nn * sizeof(double));
    memcpy(s->nodes_y, p->nodes_y, nn * sizeof(double));
    s->p.nodes_x = s->nodes_x; s->p.nodes_y = s->nodes_y;
    s->p.ucell_nodes = NULL; s->p.uedge_side = NULL; /* read during creation only */
    s->N = unstructured ? p->n_ucells : p->ni * p->nj;
    /* velocity grid: tensor product, k = ky * nvx + kx */
    double *x1 = dalloc(p->nvx), *w1 = dalloc(p->nvx), *y1 = dalloc(p->nvy), *v1 = dalloc(p->nvy);
    double unit = sqrt(2.0 * p->RT_ref);
    int rc = orc_quadrature(p->vrule, p->nvx, p->vxmin, p->vrule == ORC_GAUSS_HERMITE ? unit : p->vxmax, x1, w1);
    rc |= orc_quadrature(p->vrule, p->nvy, p->vymin, p->vrule == ORC_GAUSS_HERMITE ? unit : p->vymax, y1, v1);
    if (rc) { free(x1); free(w1); free(y1); free(v1); free(s->nodes_x); free(s->nodes_y); free(s); return NULL; }
    s->Nv = p->nvx * p->nvy;
    s->ux = dalloc(s->Nv); s->uy = dalloc(s->Nv); s->w = dalloc(s->Nv);
    s->xi_max = 0;
    for (int ky = 0; ky < p->nvy; ++ky)
        for (int kx = 0; kx < p->nvx; ++kx) {
            int k = ky * p->nvx + kx;
            s->ux[k] = x1[kx]; s->uy[k] = y1[ky]; s->w[k] = w1[kx] * v1[ky];
            double sp = sqrt(x1[kx] * x1[kx] + y1[ky] * y1[ky]);
            if (sp > s->xi_max) s->xi_max = sp;
        }
    free(x1); free(w1); free(y1); free(v1);
    /* gas constants: VHS reference viscosity for rho_ref = L_ref = 1 */
    double om = p->omega;
    s->mu_ref = 15.0 * sqrt(2.0 * M_PI * p->RT_ref) * p->Kn / (2.0 * (5.0 - 2.0 * om) * (7.0 - 2.0 * om));
    s->gam = (double)(p->K + 4) / (double)(p->K + 2);
    /* faces (unstructured: at most 4 per cell, the count is known after the build) */
    if (unstructured) {
        s->nf = 4 * s->N;
    } else {
        int nfi = (p->bc_kind[ORC_IMIN] == ORC_BC_PERIODIC ? p->ni : p->ni + 1) * p->nj;
        int nfj = (p->bc_kind[ORC_JMIN] == ORC_BC_PERIODIC ? p->nj : p->nj + 1) * p->ni;
        s->nf = nfi + nfj;
    }
    size_t N = s->N, Nv = s->Nv, NNv = N * Nv;
    s->cx = dalloc(N); s->cy = dalloc(N); s->area = dalloc(N); s->hcell = dalloc(N); s->dtimp = dalloc(N);
    s->face = (orc_face *)calloc((size_t)s->nf, sizeof(orc_face));
    s->cell_face = (int *)calloc(4 * N, sizeof(int));
    s->cell_sign = (int *)calloc(4 * N, sizeof(int));
    s->nslot = (int *)calloc(N, sizeof(int));
    s->lsinv = dalloc(4 * N);
    if (unstructured) {
        s->p.ucell_nodes = p->ucell_nodes; s->p.uedge_side = p->uedge_side;
        int bad = build_geometry_unstructured(s);
        s->p.ucell_nodes = NULL; s->p.uedge_side = NULL;
        if (bad) {
            free(s->nodes_x); free(s->nodes_y); free(s->ux); free(s->uy); free(s->w);
            free(s->cx); free(s->cy); free(s->area); free(s->hcell); free(s->dtimp);
            free(s->face); free(s->cell_face); free(s->cell_sign); free(s->nslot); free(s->lsinv);
            free(s);
            return NULL;
        }
    } else {
        build_geometry(s);
    }
    size_t nf = s->nf;
    s->G = dalloc(NNv); s->H = dalloc(NNv); s->W = dalloc(4 * N);
    s->fbG = dalloc(NNv); s->fbH = dalloc(NNv);
    s->grG = dalloc(2 * NNv); s->grH = dalloc(2 * NNv);
    s->limG = dalloc(NNv); s->limH = dalloc(NNv);
    s->FG = dalloc(nf * Nv); s->FH = dalloc(nf * Nv);
    s->phi = dalloc(4 * nf); s->rw = dalloc(4 * N); s->qcell = dalloc(2 * N); s->tau = dalloc(N);
    s->RG = dalloc(NNv); s->RH = dalloc(NNv); s->Dm = dalloc(NNv);
    s->dG = dalloc(NNv); s->dH = dalloc(NNv); s->dW = dalloc(4 * N);
    s->eqG = dalloc(NNv); s->eqH = dalloc(NNv);
    return s;
}

void orc_destroy(orc_state *s)
{
    if (!s) return;
    double *arrs[] = {s->nodes_x, s->nodes_y, s->cx, s->cy, s->area, s->hcell, s->dtimp, s->lsinv,
                      s->ux, s->uy, s->w, s->G, s->H, s->W, s->fbG, s->fbH, s->grG, s->grH,
                      s->limG, s->limH, s->FG, s->FH, s->phi, s->rw, s->qcell, s->tau, s->RG,
                      s->RH, s->Dm, s->dG, s->dH, s->dW, s->eqG, s->eqH};
    for (size_t i = 0; i < sizeof(arrs) / sizeof(arrs[0]); ++i) free(arrs[i]);
    free(s->face); free(s->cell_face); free(s->cell_sign); free(s->nslot);
    free(s);
}

int orc_num_cells(const orc_state *s) { return s->N; }
int orc_num_vel(const orc_state *s) { return s->Nv; }
int orc_num_faces(const orc_state *s) { return s->nf; }
double orc_dt(const orc_state *s) { return s->dt; }

void orc_velocity_grid(const orc_state *s, double *ux, double *uy, double *w)
{
    memcpy(ux, s->ux, s->Nv * sizeof(double));
    memcpy(uy, s->uy, s->Nv * sizeof(double));
    memcpy(w, s->w, s->Nv * sizeof(double));
}

void orc_get_geometry(const orc_state *s, double *cx, double *cy, double *area)
{
    memcpy(cx, s->cx, s->N * sizeof(double));
    memcpy(cy, s->cy, s->N * sizeof(double));
    memcpy(area, s->area, s->N * sizeof(double));
}

void orc_get_faces(const orc_state *s, int *L, int *R, int *bc, int *side, double *nx,
                   double *ny, double *S)
{
    for (int f = 0; f < s->nf; ++f) {
        L[f] = s->face[f].L; R[f] = s->face[f].R; bc[f] = s->face[f].bc; side[f] = s->face[f].side;
        nx[f] = s->face[f].nx; ny[f] = s->face[f].ny; S[f] = s->face[f].S;
    }
}

/* a (re)start has no last increment: the wall ghost terms start from zero */
static void clear_increments(orc_state *s)
{
    size_t NNv = (size_t)s->N * s->Nv;
    memset(s->dG, 0, NNv * sizeof(double));
    memset(s->dH, 0, NNv * sizeof(double));
}

void orc_init_uniform(orc_state *s, double rho, double u, double v, double T)
{
    /* W0 = exact continuous moments of the uniform Maxwellian; f~0 = f^eq(W0) */
    double RT = T * s->p.RT_ref;
    for (int c = 0; c < s->N; ++c) {
        double *W = s->W + 4 * c;
        W[0] = rho; W[1] = rho * u; W[2] = rho * v;
        W[3] = 0.5 * rho * (u * u + v * v + (s->p.K + 2) * RT);
        equilibrium(s, rho, u, v, RT, 0.0, 0.0, s->G + (size_t)c * s->Nv, s->H + (size_t)c * s->Nv);
    }
    clear_increments(s);
}

void orc_set_state(orc_state *s, const double *G, const double *H, const double *W)
{
    size_t NNv = (size_t)s->N * s->Nv;
    memcpy(s->G, G, NNv * sizeof(double));
    memcpy(s->H, H, NNv * sizeof(double));
    memcpy(s->W, W, 4 * s->N * sizeof(double));
    clear_increments(s);
}

void orc_get_state(const orc_state *s, double *G, double *H, double *W)
{
    size_t NNv = (size_t)s->N * s->Nv;
    if (G) memcpy(G, s->G, NNv * sizeof(double));
    if (H) memcpy(H, s->H, NNv * sizeof(double));
    if (W) memcpy(W, s->W, 4 * s->N * sizeof(double));
}

void orc_get_face_phi(const orc_state *s, double *phi4) { memcpy(phi4, s->phi, 4 * s->nf * sizeof(double)); }
void orc_get_rw(const orc_state *s, double *rw4) { memcpy(rw4, s->rw, 4 * s->N * sizeof(double)); }

/* least-squares gradient of a cell scalar, Eq. (14)-(15) (phi = 1 there) */
static void ls_grad_cell(const orc_state *s, int c, const double *val, size_t stride, size_t off,
                         double *gx, double *gy)
{
    double bx = 0, by = 0;
    double v0 = val[(size_t)c * stride + off];
    for (int m = 0; m < s->nslot[c]; ++m) {
        const orc_face *F = &s->face[s->cell_face[4 * c + m]];
        if (F->L < 0 || F->R < 0) continue;
        int sg = s->cell_sign[4 * c + m];
        int nb = sg > 0 ? F->R : F->L;
        double dx = sg > 0 ? F->rLx - F->rRx : F->rRx - F->rLx;
        double dy = sg > 0 ? F->rLy - F->rRy : F->rRy - F->rLy;
        double dv = val[(size_t)nb * stride + off] - v0;
        bx += dx * dv; by += dy * dv;
    }
    const double *A = s->lsinv + 4 * c;
    *gx = A[0] * bx + A[1] * by;
    *gy = A[2] * bx + A[3] * by;
}

void orc_ls_gradient(const orc_state *s, const double *phi, double *grad2)
{
    for (int c = 0; c < s->N; ++c) ls_grad_cell(s, c, phi, 1, 0, &grad2[2 * c], &grad2[2 * c + 1]);
}

/* Venkatakrishnan limiter of one scalar in one cell, Eq. (16)-(17): the face
 * value is the unlimited extrapolation to each face midpoint; the max and min
 * run over the least-squares neighbours and the cell itself; phi is the
 * minimum over the faces.  With a smoothing constant K > 0 (the form of the
 * limiter's source, Venkatakrishnan's steady-convergence paper, that the
 * paper cites for it) each face's factor is, with D the extrapolated
 * increment and P the increment to the neighbourhood's max (D > 0) or min
 * (D < 0), (P^2 + eps^2 + 2 D P) / (P^2 + 2 D^2 + P D + eps^2), eps^2 =
 * (K h)^3, h = sqrt(area); eps = 0 gives theta(P / D) of Eq. (17). */
static double limiter_cell(const orc_state *s, int c, const double *val, size_t stride, size_t off,
                           double gx, double gy)
{
    double v0 = val[(size_t)c * stride + off], vmax = v0, vmin = v0;
    for (int m = 0; m < s->nslot[c]; ++m) {
        const orc_face *F = &s->face[s->cell_face[4 * c + m]];
        if (F->L < 0 || F->R < 0) continue;
        int nb = s->cell_sign[4 * c + m] > 0 ? F->R : F->L;
        double v = val[(size_t)nb * stride + off];
        if (v > vmax) vmax = v;
        if (v < vmin) vmin = v;
    }
    double phi = 1.0;
    const double Kh = s->p.venkat_k * sqrt(s->area[c]);
    const double e2 = Kh * Kh * Kh;
    for (int m = 0; m < s->nslot[c]; ++m) {
        const orc_face *F = &s->face[s->cell_face[4 * c + m]];
        int sg = s->cell_sign[4 * c + m];
        double rx = sg > 0 ? F->rLx : F->rRx, ry = sg > 0 ? F->rLy : F->rRy;
        double d = gx * rx + gy * ry;
        double t = 1.0;
        if (d != 0) {
            double P = d > 0 ? vmax - v0 : vmin - v0;
            if (e2 > 0) t = (P * P + e2 + 2.0 * d * P) / (P * P + 2.0 * d * d + P * d + e2);
            else t = orc_venkat_theta(P / d);
        }
        if (t < phi) phi = t;
    }
    return phi;
}

/* Venkatakrishnan limiter of a cell scalar field, Eq. (16)-(17), as applied
 * inside the flux (LS gradient, then the minimum over the faces) */
void orc_limiter(const orc_state *s, const double *phi, double *lim)
{
    for (int c = 0; c < s->N; ++c) {
        double gx, gy;
        ls_grad_cell(s, c, phi, 1, 0, &gx, &gy);
        lim[c] = limiter_cell(s, c, phi, 1, 0, gx, gy);
    }
}

/* ------------------------------------------------------------------------- */
/* one DUGKS flux evaluation (Eq. 10-19): cell prep, gradients, faces          */
/* ------------------------------------------------------------------------- */

/* Cell prep (Eq. 10, Eq. 12): primitives from W, q from the stored f~,
 * equilibrium, fb+.  W is the conservative state (IDUGKS) or the moments of
 * f~ (explicit DUGKS, filled by the caller). */
static void cell_prep(orc_state *s)
{
    const int Nv = s->Nv;
    const double dt = s->dt, h = s->h;
    const double Pr = s->p.shakhov ? s->p.Pr : 1.0;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < s->N; ++c) {
        double rho, U, V, RT;
        primitives(s, s->W + 4 * c, &rho, &U, &V, &RT);
        double tau = viscosity(s, RT) / (rho * RT);
        double qtx, qty;
        const double *G = s->G + (size_t)c * Nv, *H = s->H + (size_t)c * Nv;
        heat_flux(s, G, H, U, V, &qtx, &qty);
        double qx = 2.0 * tau * qtx / (2.0 * tau + dt * Pr);
        double qy = 2.0 * tau * qty / (2.0 * tau + dt * Pr);
        s->qcell[2 * c] = qx; s->qcell[2 * c + 1] = qy; s->tau[c] = tau;
        double *eG = s->eqG + (size_t)c * Nv, *eH = s->eqH + (size_t)c * Nv;
        equilibrium(s, rho, U, V, RT, qx, qy, eG, eH);
        double c1 = (2.0 * tau - h) / (2.0 * tau + dt), c2 = 3.0 * h / (2.0 * tau + dt);
        for (int k = 0; k < Nv; ++k) {
            s->fbG[(size_t)c * Nv + k] = c1 * G[k] + c2 * eG[k];
            s->fbH[(size_t)c * Nv + k] = c1 * H[k] + c2 * eH[k];
        }
    }
}

static void gradients(orc_state *s)
{
    const int Nv = s->Nv;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < s->N; ++c)
        for (int k = 0; k < Nv; ++k) {
            size_t ck = (size_t)c * Nv + k;
            double gx, gy;
            ls_grad_cell(s, c, s->fbG, Nv, k, &gx, &gy);
            s->grG[2 * ck] = gx; s->grG[2 * ck + 1] = gy;
            s->limG[ck] = s->p.limiter ? limiter_cell(s, c, s->fbG, Nv, k, gx, gy) : 1.0;
            ls_grad_cell(s, c, s->fbH, Nv, k, &gx, &gy);
            s->grH[2 * ck] = gx; s->grH[2 * ck + 1] = gy;
            s->limH[ck] = s->p.limiter ? limiter_cell(s, c, s->fbH, Nv, k, gx, gy) : 1.0;
        }
}

/* reconstruction of fb at the face from one side along the characteristic,
 * Eq. (11), (13), (14): fb(x_f, t+h) = fb+_c + phi sigma_c . (x_f - xi h - x_c) */
static void reconstruct(const orc_state *s, int c, double rx, double ry, int k, double *g, double *hh)
{
    size_t ck = (size_t)c * s->Nv + k;
    double ax = rx - s->ux[k] * s->h, ay = ry - s->uy[k] * s->h;
    *g = s->fbG[ck] + s->limG[ck] * (s->grG[2 * ck] * ax + s->grG[2 * ck + 1] * ay);
    *hh = s->fbH[ck] + s->limH[ck] * (s->grH[2 * ck] * ax + s->grH[2 * ck + 1] * ay);
}

/* face distribution at the half step, face equilibrium and flux, Eq. (11)-(19) */
static void face_fluxes(orc_state *s)
{
    const int Nv = s->Nv;
    const double h = s->h;
    const double Pr = s->p.shakhov ? s->p.Pr : 1.0;
#pragma omp parallel
    {
        double *gb = dalloc(Nv), *hb = dalloc(Nv), *ge = dalloc(Nv), *he = dalloc(Nv);
        double *gw = dalloc(Nv), *hw = dalloc(Nv);
#pragma omp for schedule(dynamic, 4)
        for (int f = 0; f < s->nf; ++f) {
            const orc_face *F = &s->face[f];
            const double nx = F->nx, ny = F->ny, S = F->S;
            if (F->L >= 0 && F->R >= 0) {
                for (int k = 0; k < Nv; ++k) {
                    double sn = s->ux[k] * nx + s->uy[k] * ny;
                    double g1, h1, g2, h2;
                    if (sn > 0) reconstruct(s, F->L, F->rLx, F->rLy, k, &gb[k], &hb[k]);
                    else if (sn < 0) reconstruct(s, F->R, F->rRx, F->rRy, k, &gb[k], &hb[k]);
                    else {
                        reconstruct(s, F->L, F->rLx, F->rLy, k, &g1, &h1);
                        reconstruct(s, F->R, F->rRx, F->rRy, k, &g2, &h2);
                        gb[k] = 0.5 * (g1 + g2); hb[k] = 0.5 * (h1 + h2);
                    }
                }
            } else {
                /* boundary face: interior cell c, outward normal (from c) */
                int c = F->L >= 0 ? F->L : F->R;
                double on = F->L >= 0 ? 1.0 : -1.0;
                double rx = F->L >= 0 ? F->rLx : F->rRx, ry = F->L >= 0 ? F->rLy : F->rRy;
                const int sd = F->side;
                double bw = 1.0;
                if (F->bc == ORC_BC_WALL) {
                    equilibrium(s, 1.0, s->p.bc_u[sd], s->p.bc_v[sd], s->p.bc_T[sd] * s->p.RT_ref, 0, 0, gw, hw);
                    double out = 0, in = 0;
                    for (int k = 0; k < Nv; ++k) {
                        double so = on * (s->ux[k] * nx + s->uy[k] * ny);
                        double g1, h1;
                        if (so > 0) {
                            reconstruct(s, c, rx, ry, k, &g1, &h1);
                            out += s->w[k] * so * g1;
                        } else if (so < 0) {
                            in += s->w[k] * (-so) * gw[k];
                        }
                    }
                    bw = out / in; /* Eq. (35): zero net mass flux through the wall */
                } else {
                    equilibrium(s, s->p.bc_rho[sd], s->p.bc_u[sd], s->p.bc_v[sd],
                                s->p.bc_T[sd] * s->p.RT_ref, 0, 0, gw, hw);
                }
                for (int k = 0; k < Nv; ++k) {
                    double so = on * (s->ux[k] * nx + s->uy[k] * ny);
                    double g1, h1;
                    if (so > 0) reconstruct(s, c, rx, ry, k, &gb[k], &hb[k]);
                    else if (so < 0) { gb[k] = bw * gw[k]; hb[k] = bw * hw[k]; }
                    else {
                        reconstruct(s, c, rx, ry, k, &g1, &h1);
                        gb[k] = 0.5 * (g1 + bw * gw[k]); hb[k] = 0.5 * (h1 + bw * hw[k]);
                    }
                }
            }
            /* face macroscopic state from the moments of fb (text after Eq. 12) */
            double Wf[4], rho, U, V, RT, qbx, qby;
            moments_W(s, gb, hb, Wf);
            primitives(s, Wf, &rho, &U, &V, &RT);
            heat_flux(s, gb, hb, U, V, &qbx, &qby);
            double tau = viscosity(s, RT) / (rho * RT);
            double qx = 2.0 * tau * qbx / (2.0 * tau + h * Pr);
            double qy = 2.0 * tau * qby / (2.0 * tau + h * Pr);
            equilibrium(s, rho, U, V, RT, qx, qy, ge, he);
            /* Eq. (18) then Eq. (19) */
            double a = 2.0 * tau / (2.0 * tau + h), b = h / (2.0 * tau + h);
            double p0 = 0, p1 = 0, p2 = 0, p3 = 0;
            for (int k = 0; k < Nv; ++k) {
                double sn = s->ux[k] * nx + s->uy[k] * ny;
                double fg = sn * S * (a * gb[k] + b * ge[k]);
                double fh = sn * S * (a * hb[k] + b * he[k]);
                s->FG[(size_t)f * Nv + k] = fg;
                s->FH[(size_t)f * Nv + k] = fh;
                double wk = s->w[k];
                p0 += wk * fg;
                p1 += wk * s->ux[k] * fg;
                p2 += wk * s->uy[k] * fg;
                p3 += 0.5 * wk * ((s->ux[k] * s->ux[k] + s->uy[k] * s->uy[k]) * fg + fh);
            }
            if (F->bc == ORC_BC_WALL) p0 = 0.0; /* impermeable wall */
            s->phi[4 * f + 0] = p0; s->phi[4 * f + 1] = p1;
            s->phi[4 * f + 2] = p2; s->phi[4 * f + 3] = p3;
        }
        free(gb); free(hb); free(ge); free(he); free(gw); free(hw);
    }
}

/* ------------------------------------------------------------------------- */
/* macroscopic predictor: Eq. (27)-(31), LU-SGS                               */
/* ------------------------------------------------------------------------- */

static void euler_flux(const orc_state *s, const double *W, double nx, double ny, double *F)
{
    double rho = W[0], u = W[1] / rho, v = W[2] / rho;
    double p = (s->gam - 1.0) * (W[3] - 0.5 * rho * (u * u + v * v));
    double vn = u * nx + v * ny;
    F[0] = rho * vn;
    F[1] = W[1] * vn + p * nx;
    F[2] = W[2] * vn + p * ny;
    F[3] = (W[3] + p) * vn;
}

static double face_lambda(const orc_state *s, const orc_face *F)
{
    double uL = 0, vL = 0, cL = 0, uR = 0, vR = 0, cR = 0, rho, RT;
    int have = 0;
    if (F->L >= 0) { primitives(s, s->W + 4 * F->L, &rho, &uL, &vL, &RT); cL = sqrt(s->gam * RT); have |= 1; }
    if (F->R >= 0) { primitives(s, s->W + 4 * F->R, &rho, &uR, &vR, &RT); cR = sqrt(s->gam * RT); have |= 2; }
    double u, v, c;
    if (have == 3) { u = 0.5 * (uL + uR); v = 0.5 * (vL + vR); c = 0.5 * (cL + cR); }
    else if (have == 1) { u = uL; v = vL; c = cL; }
    else { u = uR; v = vR; c = cR; }
    return (fabs(u * F->nx + v * F->ny) + c) * F->S;
}

/* off-diagonal term of the predictor equations between cell c and the
 * neighbour across slot m with increment dn: 1/2 (dF S - w Lambda dn), dF the
 * change of the Euler flux of the neighbour's state along c's outward normal;
 * 0 (returns 0) when the slot has no neighbour cell or wraps c onto itself */
static int offdiag(const orc_state *s, const double *lam, int c, int m, const double *dnW, double *o)
{
    int fi = s->cell_face[4 * c + m];
    const orc_face *F = &s->face[fi];
    if (F->L < 0 || F->R < 0 || F->L == F->R) return 0;
    int sg = s->cell_sign[4 * c + m];
    int nb = sg > 0 ? F->R : F->L;
    double nx = sg * F->nx, ny = sg * F->ny;
    double Wn[4], F1[4], F0[4];
    for (int q = 0; q < 4; ++q) Wn[q] = s->W[4 * nb + q] + dnW[4 * nb + q];
    euler_flux(s, Wn, nx, ny, F1);
    euler_flux(s, s->W + 4 * nb, nx, ny, F0);
    for (int q = 0; q < 4; ++q) o[q] = 0.5 * ((F1[q] - F0[q]) * F->S - s->p.lusgs_omega * lam[fi] * dnW[4 * nb + q]);
    return 1;
}

/* point relaxation: n Jacobi sweeps, every cell from the previous sweep's
 * increments of all its neighbours, starting from dW = 0 (one sweep gives
 * dW = R / D) */
static void point_relaxation(orc_state *s, const double *Dd, const double *lam, int n)
{
    const int N = s->N;
    double *prev = dalloc(4 * N), *next = dalloc(4 * N);
    for (int k = 0; k < n; ++k) {
        for (int c = 0; c < N; ++c) {
            double acc[4] = {s->rw[4 * c], s->rw[4 * c + 1], s->rw[4 * c + 2], s->rw[4 * c + 3]};
            for (int m = 0; m < s->nslot[c]; ++m) {
                double o[4];
                if (!offdiag(s, lam, c, m, prev, o)) continue;
                for (int q = 0; q < 4; ++q) acc[q] -= o[q];
            }
            for (int q = 0; q < 4; ++q) next[4 * c + q] = acc[q] / Dd[c];
        }
        double *t = prev; prev = next; next = t;
    }
    memcpy(s->dW, prev, 4 * (size_t)N * sizeof(double));
    free(prev); free(next);
}

static void macro_predictor(orc_state *s)
{
    const int N = s->N;
    const double om = s->p.lusgs_omega;
    double *Dd = dalloc(N);
    double *lam = dalloc(s->nf);
    for (int f = 0; f < s->nf; ++f) lam[f] = face_lambda(s, &s->face[f]);
    for (int c = 0; c < N; ++c) {
        double d = s->area[c] / s->dtimp[c];
        for (int m = 0; m < s->nslot[c]; ++m) {
            const orc_face *F = &s->face[s->cell_face[4 * c + m]];
            if (F->L == F->R) continue; /* a cell wrapped onto itself: no net term */
            d += 0.5 * om * lam[s->cell_face[4 * c + m]];
        }
        Dd[c] = d;
    }
    if (s->p.relax_sweeps > 0) {
        point_relaxation(s, Dd, lam, s->p.relax_sweeps);
        free(Dd); free(lam);
        return;
    }
    /* forward sweep, lexicographic order idx = j*ni + i */
    for (int c = 0; c < N; ++c) {
        double acc[4] = {s->rw[4 * c], s->rw[4 * c + 1], s->rw[4 * c + 2], s->rw[4 * c + 3]};
        for (int m = 0; m < s->nslot[c]; ++m) {
            int fi = s->cell_face[4 * c + m];
            const orc_face *F = &s->face[fi];
            if (F->L < 0 || F->R < 0 || F->L == F->R) continue;
            int sg = s->cell_sign[4 * c + m];
            int nb = sg > 0 ? F->R : F->L;
            if (nb >= c) continue;
            double nx = sg * F->nx, ny = sg * F->ny;
            double Wn[4], F1[4], F0[4];
            for (int q = 0; q < 4; ++q) Wn[q] = s->W[4 * nb + q] + s->dW[4 * nb + q];
            euler_flux(s, Wn, nx, ny, F1);
            euler_flux(s, s->W + 4 * nb, nx, ny, F0);
            for (int q = 0; q < 4; ++q)
                acc[q] -= 0.5 * ((F1[q] - F0[q]) * F->S - om * lam[fi] * s->dW[4 * nb + q]);
        }
        for (int q = 0; q < 4; ++q) s->dW[4 * c + q] = acc[q] / Dd[c];
    }
    /* backward sweep */
    for (int c = N - 1; c >= 0; --c) {
        double acc[4] = {0, 0, 0, 0};
        for (int m = 0; m < s->nslot[c]; ++m) {
            int fi = s->cell_face[4 * c + m];
            const orc_face *F = &s->face[fi];
            if (F->L < 0 || F->R < 0 || F->L == F->R) continue;
            int sg = s->cell_sign[4 * c + m];
            int nb = sg > 0 ? F->R : F->L;
            if (nb <= c) continue;
            double nx = sg * F->nx, ny = sg * F->ny;
            double Wn[4], F1[4], F0[4];
            for (int q = 0; q < 4; ++q) Wn[q] = s->W[4 * nb + q] + s->dW[4 * nb + q];
            euler_flux(s, Wn, nx, ny, F1);
            euler_flux(s, s->W + 4 * nb, nx, ny, F0);
            for (int q = 0; q < 4; ++q)
                acc[q] += 0.5 * ((F1[q] - F0[q]) * F->S - om * lam[fi] * s->dW[4 * nb + q]);
        }
        for (int q = 0; q < 4; ++q) s->dW[4 * c + q] -= acc[q] / Dd[c];
    }
    free(Dd); free(lam);
}

/* ------------------------------------------------------------------------- */
/* one IDUGKS iteration                                                        */
/* ------------------------------------------------------------------------- */

/* macroscopic residual M_W = -sum_k int psi F_k (Eq. 27) per cell from the
 * last face fluxes; returns ||R_W / Omega||_2 */
static double macro_residual(orc_state *s)
{
    double r2 = 0.0;
    for (int c = 0; c < s->N; ++c) {
        double acc[4] = {0, 0, 0, 0};
        for (int m = 0; m < s->nslot[c]; ++m) {
            int fi = s->cell_face[4 * c + m];
            double sg = s->cell_sign[4 * c + m];
            for (int q = 0; q < 4; ++q) acc[q] -= sg * s->phi[4 * fi + q];
        }
        for (int q = 0; q < 4; ++q) {
            s->rw[4 * c + q] = acc[q];
            double r = acc[q] / s->area[c];
            r2 += r * r;
        }
    }
    return sqrt(r2);
}

/* micro residual M + Q (Eq. 23 with the Omega/dt factor) and LU-SGS
 * diagonal (Eq. 26), equilibrium at the predicted W^{n+1} = W + dW */
static void micro_residual(orc_state *s)
{
    const int N = s->N, Nv = s->Nv;
    const double dt = s->dt;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < N; ++c) {
        double Wn[4];
        for (int q = 0; q < 4; ++q) Wn[q] = s->W[4 * c + q] + s->dW[4 * c + q];
        double rho, U, V, RT;
        primitives(s, Wn, &rho, &U, &V, &RT);
        double taup = viscosity(s, RT) / (rho * RT);
        double *eG = s->eqG + (size_t)c * Nv, *eH = s->eqH + (size_t)c * Nv;
        equilibrium(s, rho, U, V, RT, s->qcell[2 * c], s->qcell[2 * c + 1], eG, eH);
        double cq = 2.0 * s->area[c] / (2.0 * taup + dt);
        double d0 = s->area[c] / s->dtimp[c] + cq;
        for (int k = 0; k < Nv; ++k) {
            size_t ck = (size_t)c * Nv + k;
            double mg = 0, mh = 0, dd = d0;
            for (int m = 0; m < s->nslot[c]; ++m) {
                int fi = s->cell_face[4 * c + m];
                const orc_face *F = &s->face[fi];
                double sg = s->cell_sign[4 * c + m];
                mg -= sg * s->FG[(size_t)fi * Nv + k];
                mh -= sg * s->FH[(size_t)fi * Nv + k];
                if (F->L == F->R) continue;
                double so = sg * (s->ux[k] * F->nx + s->uy[k] * F->ny);
                if (so > 0) dd += so * F->S;
            }
            s->RG[ck] = mg - cq * (s->G[ck] - eG[k]);
            s->RH[ck] = mh - cq * (s->H[ck] - eH[k]);
            s->Dm[ck] = dd;
        }
    }
}

/* Linearised diffuse wall in the micro sweeps (Eq. 33-35).  The ghost cell
 * behind a wall face takes, in each velocity coming into the domain, the
 * increment drho_g M_w (Eq. 34: M_w the unit-density wall Maxwellian, with
 * the wall's velocity and temperature), drho_g fixed by Eq. (35): the ghost
 * increment carries back the mass flux of the inner cell's outgoing
 * increments.  The inner increments are the last iteration's (dG still holds
 * them; zero after a restart, the start the end of Section 2.3 prescribes),
 * so the ghost term is known before the sweeps and enters both of them as
 * the upwind neighbour term |xi.n| S Delta_ghost, i.e. on the right-hand side. */
static void wall_ghost_terms(orc_state *s)
{
    const int Nv = s->Nv;
    double *gw = dalloc(Nv), *hw = dalloc(Nv);
    for (int f = 0; f < s->nf; ++f) {
        const orc_face *F = &s->face[f];
        if (F->bc != ORC_BC_WALL) continue;
        const int c = F->L >= 0 ? F->L : F->R, sd = F->side;
        const double on = F->L >= 0 ? 1.0 : -1.0;
        equilibrium(s, 1.0, s->p.bc_u[sd], s->p.bc_v[sd], s->p.bc_T[sd] * s->p.RT_ref, 0, 0, gw, hw);
        double out = 0, in = 0;
        for (int k = 0; k < Nv; ++k) {
            double so = on * (s->ux[k] * F->nx + s->uy[k] * F->ny);
            if (so > 0) out += s->w[k] * so * s->dG[(size_t)c * Nv + k];
            else if (so < 0) in += s->w[k] * (-so) * gw[k];
        }
        const double drho = out / in;
        for (int k = 0; k < Nv; ++k) {
            double so = on * (s->ux[k] * F->nx + s->uy[k] * F->ny);
            if (so < 0) {
                size_t ck = (size_t)c * Nv + k;
                s->RG[ck] += -so * F->S * drho * gw[k];
                s->RH[ck] += -so * F->S * drho * hw[k];
            }
        }
    }
    free(gw); free(hw);
}

/* LU-SGS sweeps of the micro equations (Eq. 26) for (RG, RH) with the
 * diagonal Dm: (D - L) D^-1 (D - U) Delta = R, L and U the upwind couplings
 * |xi.n| S of the lower and upper neighbours in the cell numbering (Eq. 25);
 * each velocity independent; the ghost increments are zero here (their wall
 * part, if any, is on the right-hand side).  Forward: Delta* = (R + sum over
 * lower inflow neighbours of |xi.n| S Delta*_nb) / D; backward: Delta =
 * Delta* + sum over upper inflow neighbours of |xi.n| S Delta_nb / D. */
static void micro_sweeps(orc_state *s)
{
    const int N = s->N, Nv = s->Nv;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < Nv; ++k) {
        for (int c = 0; c < N; ++c) {
            size_t ck = (size_t)c * Nv + k;
            double ag = s->RG[ck], ah = s->RH[ck];
            for (int m = 0; m < s->nslot[c]; ++m) {
                const orc_face *F = &s->face[s->cell_face[4 * c + m]];
                if (F->L < 0 || F->R < 0 || F->L == F->R) continue;
                int sg = s->cell_sign[4 * c + m];
                int nb = sg > 0 ? F->R : F->L;
                if (nb >= c) continue;
                double so = sg * (s->ux[k] * F->nx + s->uy[k] * F->ny);
                if (so < 0) {
                    ag += -so * F->S * s->dG[(size_t)nb * Nv + k];
                    ah += -so * F->S * s->dH[(size_t)nb * Nv + k];
                }
            }
            s->dG[ck] = ag / s->Dm[ck];
            s->dH[ck] = ah / s->Dm[ck];
        }
        for (int c = N - 1; c >= 0; --c) {
            size_t ck = (size_t)c * Nv + k;
            double ag = 0, ah = 0;
            for (int m = 0; m < s->nslot[c]; ++m) {
                const orc_face *F = &s->face[s->cell_face[4 * c + m]];
                if (F->L < 0 || F->R < 0 || F->L == F->R) continue;
                int sg = s->cell_sign[4 * c + m];
                int nb = sg > 0 ? F->R : F->L;
                if (nb <= c) continue;
                double so = sg * (s->ux[k] * F->nx + s->uy[k] * F->ny);
                if (so < 0) {
                    ag += -so * F->S * s->dG[(size_t)nb * Nv + k];
                    ah += -so * F->S * s->dH[(size_t)nb * Nv + k];
                }
            }
            s->dG[ck] += ag / s->Dm[ck];
            s->dH[ck] += ah / s->Dm[ck];
        }
    }
}

static double idugks_iteration(orc_state *s)
{
    const int N = s->N, Nv = s->Nv;
    /* DUGKS flux at the half step from f~^n and W^n */
    cell_prep(s);
    gradients(s);
    face_fluxes(s);
    double res = macro_residual(s);
    /* macroscopic predictor -> W^{n+1} */
    macro_predictor(s);
    micro_residual(s);
    if (s->p.implicit_wall) wall_ghost_terms(s);
    micro_sweeps(s);
    /* simultaneous update, Eq. (32) */
    size_t NNv = (size_t)N * Nv;
    for (size_t i = 0; i < NNv; ++i) { s->G[i] += s->dG[i]; s->H[i] += s->dH[i]; }
    for (int i = 0; i < 4 * N; ++i) s->W[i] += s->dW[i];
    return res;
}

void orc_iterate(orc_state *s, int n, double *res_abs)
{
    for (int it = 0; it < n; ++it) {
        double r = idugks_iteration(s);
        if (res_abs) res_abs[it] = r;
    }
}

/* explicit DUGKS step, Eq. (10) and Eq. (21); W is the moment set of f~ */
void orc_explicit_step(orc_state *s, int n)
{
    const int N = s->N, Nv = s->Nv;
    const double dt = s->dt;
    for (int it = 0; it < n; ++it) {
        for (int c = 0; c < N; ++c)
            moments_W(s, s->G + (size_t)c * Nv, s->H + (size_t)c * Nv, s->W + 4 * c);
        cell_prep(s);
        gradients(s);
        face_fluxes(s);
#pragma omp parallel for schedule(static)
        for (int c = 0; c < N; ++c) {
            double tau = s->tau[c];
            double a = (2.0 * tau - dt) / (2.0 * tau + dt), b = 2.0 * dt / (2.0 * tau + dt);
            for (int k = 0; k < Nv; ++k) {
                size_t ck = (size_t)c * Nv + k;
                double mg = 0, mh = 0;
                for (int m = 0; m < s->nslot[c]; ++m) {
                    int fi = s->cell_face[4 * c + m];
                    double sg = s->cell_sign[4 * c + m];
                    mg += sg * s->FG[(size_t)fi * Nv + k];
                    mh += sg * s->FH[(size_t)fi * Nv + k];
                }
                s->G[ck] = a * s->G[ck] + b * s->eqG[ck] - dt / s->area[c] * mg;
                s->H[ck] = a * s->H[ck] + b * s->eqH[ck] - dt / s->area[c] * mh;
            }
        }
    }
    for (int c = 0; c < N; ++c)
        moments_W(s, s->G + (size_t)c * Nv, s->H + (size_t)c * Nv, s->W + 4 * c);
    clear_increments(s);
}

/* the macroscopic residual R_W (Eq. 27) of the current state and the
 * predictor's increment dW (Eq. 28-31, LU-SGS or point relaxation as
 * configured); the state itself is not advanced */
void orc_debug_predictor(orc_state *s, double *rw, double *dW)
{
    const int N = s->N;
    cell_prep(s);
    gradients(s);
    face_fluxes(s);
    macro_residual(s);
    macro_predictor(s);
    memcpy(rw, s->rw, 4 * (size_t)N * sizeof(double));
    memcpy(dW, s->dW, 4 * (size_t)N * sizeof(double));
}

/* the right-hand side of the micro sweeps of the current state (the steps
 * of one iteration up to the sweeps); the state is not advanced */
void orc_debug_micro_residual(orc_state *s, double *RG, double *RH)
{
    size_t NNv = (size_t)s->N * s->Nv;
    cell_prep(s);
    gradients(s);
    face_fluxes(s);
    macro_residual(s);
    macro_predictor(s);
    micro_residual(s);
    if (s->p.implicit_wall) wall_ghost_terms(s);
    memcpy(RG, s->RG, NNv * sizeof(double));
    memcpy(RH, s->RH, NNv * sizeof(double));
}

/* the micro LU-SGS sweeps (Eq. 26) of the current state applied to a given
 * right-hand side (RG, RH): the diagonal D of the state's iteration and the
 * increments Delta the sweeps return; the state and its last increments are
 * left as they were */
void orc_debug_micro_sweeps(orc_state *s, const double *RG, const double *RH, double *dG, double *dH,
                            double *D)
{
    size_t NNv = (size_t)s->N * s->Nv;
    double *kg = dalloc(NNv), *kh = dalloc(NNv);
    memcpy(kg, s->dG, NNv * sizeof(double));
    memcpy(kh, s->dH, NNv * sizeof(double));
    cell_prep(s);
    gradients(s);
    face_fluxes(s);
    macro_residual(s);
    macro_predictor(s);
    micro_residual(s);
    memcpy(s->RG, RG, NNv * sizeof(double));
    memcpy(s->RH, RH, NNv * sizeof(double));
    micro_sweeps(s);
    memcpy(dG, s->dG, NNv * sizeof(double));
    memcpy(dH, s->dH, NNv * sizeof(double));
    memcpy(D, s->Dm, NNv * sizeof(double));
    memcpy(s->dG, kg, NNv * sizeof(double));
    memcpy(s->dH, kh, NNv * sizeof(double));
    free(kg);
    free(kh);
}

void orc_debug_cell_prep(orc_state *s, double *fbG, double *fbH, double *q, double *tau)
{
    size_t NNv = (size_t)s->N * s->Nv;
    cell_prep(s);
    memcpy(fbG, s->fbG, NNv * sizeof(double));
    memcpy(fbH, s->fbH, NNv * sizeof(double));
    memcpy(q, s->qcell, 2 * s->N * sizeof(double));
    memcpy(tau, s->tau, s->N * sizeof(double));
}

void orc_get_moments(orc_state *s, double *out6)
{
    const double Pr = s->p.shakhov ? s->p.Pr : 1.0;
    for (int c = 0; c < s->N; ++c) {
        double rho, U, V, RT, qtx, qty;
        primitives(s, s->W + 4 * c, &rho, &U, &V, &RT);
        double tau = viscosity(s, RT) / (rho * RT);
        heat_flux(s, s->G + (size_t)c * s->Nv, s->H + (size_t)c * s->Nv, U, V, &qtx, &qty);
        out6[6 * c + 0] = rho;
        out6[6 * c + 1] = U;
        out6[6 * c + 2] = V;
        out6[6 * c + 3] = RT / s->p.RT_ref;
        out6[6 * c + 4] = 2.0 * tau * qtx / (2.0 * tau + s->dt * Pr);
        out6[6 * c + 5] = 2.0 * tau * qty / (2.0 * tau + s->dt * Pr);
    }
}
