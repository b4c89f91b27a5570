// idugks_host.cpp -- host side of libidugks: the C ABI of include/idugks.h,
// problem validation, structured-mesh geometry, discrete velocity quadrature,
// workspace layout, state transfer and the iteration driver.
#include "idugks.h"
#include "idugks_internal.h"
#include "idugks_adjoint.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <string>
#include <vector>

using idg::KParams;

struct idg_ctx {
    int precision = IDG_FP64;
    int device = 0;
    std::string err;
    // problem description
    int ni = 0, nj = 0;
    std::vector<double> nodes_x, nodes_y;
    // unstructured mesh (idg_set_mesh_unstructured): ni = cells, nj = 1
    bool unstr = false;
    std::vector<int> ucell, uside;                 // [N][4] nodes, boundary groups
    std::vector<int> sched, sptr;                  // sweep schedules (see KParams)
    int nsteps_f = 0, nsteps_b = 0, sched_pc = 0;  // steps, cells per step at most
    int vrule = -1, nvx = 0, nvy = 0;
    double vx0 = 0, vx1 = 0, vy0 = 0, vy1 = 0;
    bool gas_set = false;
    int K = 1, model = IDG_BGK;
    double Pr = 1.0, omega = 0.5, Kn = 0.1, RT_ref = 0.5;
    int bc_kind[4] = {-1, -1, -1, -1};
    double bc_rho[4] = {0, 0, 0, 0}, bc_u[4] = {0, 0, 0, 0}, bc_v[4] = {0, 0, 0, 0},
           bc_T[4] = {0, 0, 0, 0};
    double cfl_imp = 100.0, cfl_phys = 0.5, lusgs_omega = 2.0;
    int limiter = 0, flags = 0;
    int relax_sweeps = 0;  // macroscopic predictor: 0 LU-SGS, n point-relaxation sweeps
    int implicit_wall = 0; // 1: linearised diffuse-wall ghost increments in the micro sweeps (Eq. 33-35)
    // derived on the host
    bool built = false;
    // Nvu: discrete velocities of the caller's grid; Nv: velocities stored per
    // cell and face, Nvu rounded up to a multiple of 4 with ghost velocities
    // of zero weight at xi = 0 (they enter no moment and no flux, and let every
    // row start on a 16-byte boundary for the vectorised sweeps)
    int N = 0, Nv = 0, Nvu = 0, nf = 0;
    std::vector<double> area, cxc, cyc, hcell, dtimp, cr, clsg, fgeo;
    std::vector<int> cface, cnb, csign, fL, fR, fbc, fside;
    std::vector<double> ux, uy, w;
    double xi_max = 0, dt = 0, mu_ref = 0;
    // reference Maxwellian of the storage
    double ref_rho = 1.0, ref_u = 0.0, ref_v = 0.0, ref_T = 1.0;
    // device
    bool bound = false;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    KParams kp{};
    KParams *kp_dev = nullptr;  // device copy of kp read by the iteration kernels
    idg::Plan plan{};           // single-instance launch plan
    double *moments_dev = nullptr;
    double *stage = nullptr;  // staging for host<->device state copies (aliases F)
    size_t stage_bytes = 0;
    // CUDA graph of kGraphChunk iterations, replayed on a library-owned stream
    // that is event-ordered with the caller's stream
    int use_graph = 1;
    cudaStream_t gstream = nullptr;
    cudaGraphExec_t gexec = nullptr;   // kGraphChunk iterations
    cudaGraphExec_t gexec1 = nullptr;  // one iteration
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // iteration bookkeeping
    long long host_iter = 0;   // iterations launched since bind
    long long start_iter = 0;  // iteration index of the last (re)start
    std::vector<double> hist;  // absolute residuals since the last (re)start
    // adjoint solver: IDG_ADJ_FIXED_POINT or IDG_ADJ_GMRES with restart adj_restart
    int adj_method = 0, adj_restart = 20;
    int adj_lim_frozen = 0;  // idg_set_adjoint_limiter: 1 holds the limiter factor at the linearisation
    double venkat_k = 0.0;   // idg_set_limiter_smoothing
    // last idg_adjoint: number of right-hand sides and the mass multiplier
    int adj_nrhs = 0;
    double adj_beta = 0.0;
};

namespace {

idg_status fail(idg_ctx *c, idg_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

idg_status cuda_fail(idg_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, IDG_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

// -------------------------------------------------------------------------
// discrete velocity quadrature (Section 2.2, closing paragraph)
// -------------------------------------------------------------------------

// Gauss-Hermite rule for the weight exp(-x^2) by the Golub-Welsch idea: the
// nodes are the eigenvalues of the symmetric Jacobi matrix of the Hermite
// recurrence (off-diagonal sqrt(k/2)).  The eigenvalues come from cyclic
// Jacobi rotations, then one or two Newton steps on the orthonormal
// recurrence polish them; the weights use W_i = 1 / (n p_{n-1}(x_i)^2).
bool gauss_hermite(int n, std::vector<double> &x, std::vector<double> &wt)
{
    if (n < 1 || n > 512) return false;
    std::vector<double> A((size_t)n * n, 0.0);
    for (int k = 1; k < n; ++k) A[(size_t)(k - 1) * n + k] = A[(size_t)k * n + k - 1] = std::sqrt(0.5 * k);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
        if (off < 1e-300) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[(size_t)p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
                for (int r = 0; r < n; ++r) {
                    double arp = A[(size_t)r * n + p], arq = A[(size_t)r * n + q];
                    A[(size_t)r * n + p] = cs * arp - sn * arq;
                    A[(size_t)r * n + q] = sn * arp + cs * arq;
                }
                for (int r = 0; r < n; ++r) {
                    double apr = A[(size_t)p * n + r], aqr = A[(size_t)q * n + r];
                    A[(size_t)p * n + r] = cs * apr - sn * aqr;
                    A[(size_t)q * n + r] = sn * apr + cs * aqr;
                }
            }
    }
    x.resize(n);
    wt.resize(n);
    for (int i = 0; i < n; ++i) x[i] = A[(size_t)i * n + i];
    std::sort(x.begin(), x.end());
    auto orth = [n](double xv, double &pn, double &pn1) {
        double p0 = std::pow(M_PI, -0.25), p1 = std::sqrt(2.0) * xv * p0;
        if (n == 1) { pn = p1; pn1 = p0; return; }
        for (int k = 1; k < n; ++k) {
            double p2 = std::sqrt(2.0 / (k + 1)) * xv * p1 - std::sqrt((double)k / (k + 1)) * p0;
            p0 = p1;
            p1 = p2;
        }
        pn = p1;
        pn1 = p0;
    };
    for (int i = 0; i < n; ++i) {
        for (int it = 0; it < 3; ++it) {
            double pn, pn1;
            orth(x[i], pn, pn1);
            double d = std::sqrt(2.0 * n) * pn1;  // p_n' = sqrt(2n) p_{n-1}
            if (d == 0.0) break;
            x[i] -= pn / d;
        }
    }
    for (int i = 0; i < n / 2; ++i) {  // exact symmetry
        double a = 0.5 * (x[n - 1 - i] - x[i]);
        x[i] = -a;
        x[n - 1 - i] = a;
    }
    if (n % 2) x[n / 2] = 0.0;
    for (int i = 0; i < n; ++i) {
        double pn, pn1;
        orth(x[i], pn, pn1);
        wt[i] = 1.0 / (n * pn1 * pn1);
    }
    for (int i = 0; i < n / 2; ++i) {
        double a = 0.5 * (wt[i] + wt[n - 1 - i]);
        wt[i] = wt[n - 1 - i] = a;
    }
    return true;
}

bool rule_1d(int rule, int n, double a, double b, double unit, std::vector<double> &x,
             std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    if (rule == IDG_NC_TRAP || rule == IDG_NC_SIMPSON) {
        if (n < 2 || !(b > a)) return false;
        if (rule == IDG_NC_SIMPSON && (n < 3 || n % 2 == 0)) return false;
        double step = (b - a) / (n - 1), mid = 0.5 * (a + b);
        for (int i = 0; i < n; ++i) {
            // symmetric about the midpoint by construction
            int m = i - (n - 1) / 2;
            double off = (n % 2) ? m * step : (i - 0.5 * (n - 1)) * step;
            x[i] = mid + off;
            if (rule == IDG_NC_TRAP) w[i] = (i == 0 || i == n - 1) ? 0.5 * step : step;
            else w[i] = (i == 0 || i == n - 1) ? step / 3.0 : ((i % 2) ? 4.0 : 2.0) * step / 3.0;
        }
        return true;
    }
    if (rule == IDG_GAUSS_HERMITE) {
        std::vector<double> gx, gw;
        if (!gauss_hermite(n, gx, gw)) return false;
        for (int i = 0; i < n; ++i) {
            x[i] = unit * gx[i];
            w[i] = unit * gw[i] * std::exp(gx[i] * gx[i]);
        }
        return true;
    }
    return false;
}

// -------------------------------------------------------------------------
// unstructured mesh of triangles and quadrilaterals
// -------------------------------------------------------------------------
// Faces are the edges: the first cell (in cell order) running along an edge
// counter-clockwise is its L side (the face normal is L's outward normal),
// the other cell R, or none on the boundary (the boundary group of that slot
// gives the condition).  Slot m of a cell is its edge node m -> m+1; a
// triangle's slot 3 is unused (sign 0, no neighbour, no geometry, the face
// index of its slot 0).  Least squares over the face neighbours; a cell
// without two neighbours in independent directions has no gradient.  The
// sweep schedules group the cells by level in the graph of lower (forward:
// smaller index) or upper (backward) neighbours -- the dependency order of
// the lexicographic sweeps -- in steps of at most sched_pc cells.
idg_status build_unstructured(idg_ctx *c, double &hmin)
{
    const int N = c->N;
    const std::vector<double> &X = c->nodes_x, &Y = c->nodes_y;
    std::vector<int> ns(N);
    c->area.assign(N, 0);
    c->cxc.assign(N, 0);
    c->cyc.assign(N, 0);
    for (int q = 0; q < N; ++q) {
        const int *cn = &c->ucell[4 * (size_t)q];
        ns[q] = cn[3] < 0 ? 3 : 4;
        // shoelace area and polygon centroid relative to the first node
        const double ox = X[cn[0]], oy = Y[cn[0]];
        double a2 = 0, sx = 0, sy = 0;
        for (int m = 0; m < ns[q]; ++m) {
            const int a = cn[m], b = cn[(m + 1) % ns[q]];
            if (a == b) return fail(c, IDG_ERR_ARG, "cell %d repeats node %d", q, a);
            const double xa = X[a] - ox, ya = Y[a] - oy, xb = X[b] - ox, yb = Y[b] - oy;
            const double cr = xa * yb - xb * ya;
            a2 += cr;
            sx += (xa + xb) * cr;
            sy += (ya + yb) * cr;
        }
        if (!(a2 > 0)) return fail(c, IDG_ERR_ARG, "cell %d has non-positive area (nodes must run counter-clockwise)", q);
        c->area[q] = 0.5 * a2;
        c->cxc[q] = ox + sx / (3.0 * a2);
        c->cyc[q] = oy + sy / (3.0 * a2);
    }
    // match the two slots of every interior edge by its sorted node pair
    struct Edge {
        int a, b, slot;  // slot = 4 cell + m
    };
    std::vector<Edge> E;
    E.reserve(4 * (size_t)N);
    for (int q = 0; q < N; ++q)
        for (int m = 0; m < ns[q]; ++m) {
            const int a = c->ucell[4 * q + m], b = c->ucell[4 * q + (m + 1) % ns[q]];
            E.push_back({std::min(a, b), std::max(a, b), 4 * q + m});
        }
    std::sort(E.begin(), E.end(), [](const Edge &u, const Edge &v) {
        return u.a != v.a ? u.a < v.a : (u.b != v.b ? u.b < v.b : u.slot < v.slot);
    });
    std::vector<int> partner(4 * (size_t)N, -1);
    for (size_t i = 0; i < E.size();) {
        size_t j = i + 1;
        while (j < E.size() && E[j].a == E[i].a && E[j].b == E[i].b) ++j;
        if (j - i > 2) return fail(c, IDG_ERR_ARG, "edge (%d,%d) is shared by %d cells", E[i].a, E[i].b, (int)(j - i));
        if (j - i == 2) {
            partner[E[i].slot] = E[i + 1].slot;
            partner[E[i + 1].slot] = E[i].slot;
        }
        i = j;
    }
    c->cface.assign(4 * N, -1);
    c->cnb.assign(4 * N, -1);
    c->csign.assign(4 * N, 0);
    c->cr.assign((size_t)8 * N, 0.0);
    c->clsg.assign((size_t)8 * N, 0.0);
    c->fL.clear(); c->fR.clear(); c->fbc.clear(); c->fside.clear(); c->fgeo.clear();
    int nf = 0;
    for (int q = 0; q < N; ++q)
        for (int m = 0; m < ns[q]; ++m) {
            const int sl = 4 * q + m;
            if (c->cface[sl] >= 0) continue;
            const int a = c->ucell[sl], b = c->ucell[4 * q + (m + 1) % ns[q]];
            const double tx = X[b] - X[a], ty = Y[b] - Y[a], S = std::sqrt(tx * tx + ty * ty);
            const double mx = 0.5 * (X[a] + X[b]), my = 0.5 * (Y[a] + Y[b]);
            double g[7] = {ty / S, -tx / S, S, mx - c->cxc[q], my - c->cyc[q], 0.0, 0.0};
            int R = -1, bc = -1, side = -1;
            const int pr = partner[sl];
            if (pr >= 0) {
                const int q2 = pr / 4, m2 = pr % 4;
                if (c->ucell[pr] != b || c->ucell[4 * q2 + (m2 + 1) % ns[q2]] != a)
                    return fail(c, IDG_ERR_ARG, "cells %d and %d run along edge (%d,%d) the same way", q, q2, a, b);
                R = q2;
                g[5] = mx - c->cxc[q2];
                g[6] = my - c->cyc[q2];
                c->cface[pr] = nf;
                c->csign[pr] = -1;
                c->cnb[pr] = q;
                c->cnb[sl] = q2;
            } else {
                side = c->uside[sl];
                if (side < 0 || c->bc_kind[side] == IDG_BC_PERIODIC)
                    return fail(c, IDG_ERR_ARG, "boundary edge (%d,%d) of cell %d needs a wall or far-field group, has %d", a, b, q, side);
                bc = c->bc_kind[side];
            }
            c->cface[sl] = nf;
            c->csign[sl] = +1;
            c->fL.push_back(q);
            c->fR.push_back(R);
            c->fbc.push_back(bc);
            c->fside.push_back(side);
            c->fgeo.insert(c->fgeo.end(), g, g + 7);
            ++nf;
        }
    c->nf = nf;
    c->hcell.assign(N, 0.0);
    c->dtimp.assign(N, 0.0);
    for (int q = 0; q < N; ++q) {
        if (ns[q] == 3) c->cface[4 * q + 3] = c->cface[4 * q];
        double smax = 0, a11 = 0, a12 = 0, a22 = 0, d[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
        for (int m = 0; m < ns[q]; ++m) {
            const int fi = c->cface[4 * q + m];
            const double *g = &c->fgeo[(size_t)7 * fi];
            const bool own_L = c->csign[4 * q + m] > 0;
            c->cr[8 * q + 2 * m] = own_L ? g[3] : g[5];
            c->cr[8 * q + 2 * m + 1] = own_L ? g[4] : g[6];
            smax = std::max(smax, g[2]);
            if (c->cnb[4 * q + m] < 0) continue;
            d[m][0] = own_L ? g[3] - g[5] : g[5] - g[3];
            d[m][1] = own_L ? g[4] - g[6] : g[6] - g[4];
            a11 += d[m][0] * d[m][0];
            a12 += d[m][0] * d[m][1];
            a22 += d[m][1] * d[m][1];
        }
        const double det = a11 * a22 - a12 * a12;
        if (det > 1e-10 * (a11 + a22) * (a11 + a22))
            for (int m = 0; m < ns[q]; ++m) {
                if (c->cnb[4 * q + m] < 0) continue;
                c->clsg[8 * q + 2 * m] = (a22 * d[m][0] - a12 * d[m][1]) / det;
                c->clsg[8 * q + 2 * m + 1] = (-a12 * d[m][0] + a11 * d[m][1]) / det;
            }
        c->hcell[q] = c->area[q] / smax;
        hmin = std::min(hmin, c->hcell[q]);
    }
    // sweep schedules
    std::vector<int> lev(N);
    int maxlevel = 0;
    std::vector<std::vector<int>> levels[2];
    for (int dir = 0; dir < 2; ++dir) {
        int nl = 0;
        for (int k = 0; k < N; ++k) {
            const int q = dir == 0 ? k : N - 1 - k;
            int l = 0;
            for (int m = 0; m < 4; ++m) {
                const int nb = c->cnb[4 * q + m];
                if (nb >= 0 && nb != q && (dir == 0 ? nb < q : nb > q)) l = std::max(l, lev[nb] + 1);
            }
            lev[q] = l;
            nl = std::max(nl, l + 1);
        }
        levels[dir].assign(nl, {});
        for (int q = 0; q < N; ++q) levels[dir][lev[q]].push_back(q);
        for (auto &lv : levels[dir]) maxlevel = std::max(maxlevel, (int)lv.size());
    }
    c->sched_pc = std::min(maxlevel, 128);
    c->sched.clear();
    c->sptr.clear();
    for (int dir = 0; dir < 2; ++dir) {
        int steps = 0;
        c->sptr.push_back(0);
        const int base = (int)c->sched.size();
        for (auto &lv : levels[dir])
            for (size_t o = 0; o < lv.size(); o += c->sched_pc) {
                for (size_t x = o; x < std::min(lv.size(), o + c->sched_pc); ++x) c->sched.push_back(lv[x]);
                c->sptr.push_back((int)c->sched.size() - base);
                ++steps;
            }
        (dir == 0 ? c->nsteps_f : c->nsteps_b) = steps;
    }
    return IDG_OK;
}

// -------------------------------------------------------------------------
// structured block geometry (Fig. 1, Section 2.3)
// -------------------------------------------------------------------------
idg_status build(idg_ctx *c)
{
    if (c->built) return IDG_OK;
    if (c->ni < 1 || c->nj < 1) return fail(c, IDG_ERR_STATE, "mesh not set");
    if (c->vrule < 0) return fail(c, IDG_ERR_STATE, "velocity grid not set");
    if (!c->gas_set) return fail(c, IDG_ERR_STATE, "gas not set");
    for (int s = 0; s < 4; ++s)
        if (c->bc_kind[s] < 0) return fail(c, IDG_ERR_STATE, "boundary of side %d not set", s);
    const bool per_i = !c->unstr && c->bc_kind[IDG_IMIN] == IDG_BC_PERIODIC;
    const bool per_j = !c->unstr && c->bc_kind[IDG_JMIN] == IDG_BC_PERIODIC;
    if (!c->unstr && (per_i != (c->bc_kind[IDG_IMAX] == IDG_BC_PERIODIC) || per_j != (c->bc_kind[IDG_JMAX] == IDG_BC_PERIODIC)))
        return fail(c, IDG_ERR_ARG, "a periodic direction needs IDG_BC_PERIODIC on both sides");
    // the wavefront kernels hold one hyperplane (up to min(ni, nj) cells) in
    // one thread block: refused here, before any workspace is sized
    if (!c->unstr && std::min(c->ni, c->nj) > 256)
        return fail(c, IDG_ERR_ARG, "min(ni, nj) = %d exceeds 256", std::min(c->ni, c->nj));
    const int ni = c->ni, nj = c->nj;
    c->N = ni * nj;
    // velocities
    std::vector<double> x1, w1, y1, v1;
    double unit = std::sqrt(2.0 * c->RT_ref);
    if (!rule_1d(c->vrule, c->nvx, c->vx0, c->vx1, unit, x1, w1) ||
        !rule_1d(c->vrule, c->nvy, c->vy0, c->vy1, unit, y1, v1))
        return fail(c, IDG_ERR_ARG, "invalid velocity quadrature (rule %d, %d x %d)", c->vrule, c->nvx, c->nvy);
    c->Nvu = c->nvx * c->nvy;
    c->Nv = (c->Nvu + 3) & ~3;
    c->ux.assign(c->Nv, 0.0);
    c->uy.assign(c->Nv, 0.0);
    c->w.assign(c->Nv, 0.0);
    c->xi_max = 0;
    for (int ky = 0; ky < c->nvy; ++ky)
        for (int kx = 0; kx < c->nvx; ++kx) {
            int k = ky * c->nvx + kx;
            c->ux[k] = x1[kx];
            c->uy[k] = y1[ky];
            c->w[k] = w1[kx] * v1[ky];
            c->xi_max = std::max(c->xi_max, std::sqrt(x1[kx] * x1[kx] + y1[ky] * y1[ky]));
        }
    double hmin = 1e300;
    if (c->unstr) {
        idg_status su = build_unstructured(c, hmin);
        if (su) return su;
    } else {
    auto X = [&](int i, int j) { return c->nodes_x[(size_t)j * (ni + 1) + i]; };
    auto Y = [&](int i, int j) { return c->nodes_y[(size_t)j * (ni + 1) + i]; };
    // cells: shoelace area and polygon centroid, relative to the cell's first
    // node (translation invariant; absolute coordinates would cancel to
    // ~eps |x|^2 / area in a small cell far from the origin)
    c->area.assign(c->N, 0);
    c->cxc.assign(c->N, 0);
    c->cyc.assign(c->N, 0);
    for (int j = 0; j < nj; ++j)
        for (int i = 0; i < ni; ++i) {
            const double ox = X(i, j), oy = Y(i, j);
            double px[4] = {0.0, X(i + 1, j) - ox, X(i + 1, j + 1) - ox, X(i, j + 1) - ox};
            double py[4] = {0.0, Y(i + 1, j) - oy, Y(i + 1, j + 1) - oy, Y(i, j + 1) - oy};
            double a2 = 0, sx = 0, sy = 0;
            for (int m = 0; m < 4; ++m) {
                int n2 = (m + 1) & 3;
                double cr = px[m] * py[n2] - px[n2] * py[m];
                a2 += cr;
                sx += (px[m] + px[n2]) * cr;
                sy += (py[m] + py[n2]) * cr;
            }
            int cc = j * ni + i;
            if (!(a2 > 0)) return fail(c, IDG_ERR_ARG, "cell (%d,%d) has non-positive area", i, j);
            c->area[cc] = 0.5 * a2;
            c->cxc[cc] = ox + sx / (3.0 * a2);
            c->cyc[cc] = oy + sy / (3.0 * a2);
        }
    // faces: i-faces row by row, then j-faces row by row
    const int nfi_row = per_i ? ni : ni + 1;
    const int nfj_rows = per_j ? nj : nj + 1;
    c->nf = nfi_row * nj + nfj_rows * ni;
    c->fL.assign(c->nf, -1);
    c->fR.assign(c->nf, -1);
    c->fbc.assign(c->nf, -1);
    c->fside.assign(c->nf, -1);
    c->fgeo.assign((size_t)7 * c->nf, 0.0);
    auto set_face = [&](int f, double x0, double y0, double x1_, double y1_, bool ifc, int L, int R,
                        double mLx, double mLy, double mRx, double mRy, int side) {
        double tx = x1_ - x0, ty = y1_ - y0, S = std::sqrt(tx * tx + ty * ty);
        double *g = &c->fgeo[(size_t)7 * f];
        g[0] = ifc ? ty / S : -ty / S;
        g[1] = ifc ? -tx / S : tx / S;
        g[2] = S;
        c->fL[f] = L;
        c->fR[f] = R;
        if (L >= 0) { g[3] = mLx - c->cxc[L]; g[4] = mLy - c->cyc[L]; }
        if (R >= 0) { g[5] = mRx - c->cxc[R]; g[6] = mRy - c->cyc[R]; }
        if (side >= 0) { c->fside[f] = side; c->fbc[f] = c->bc_kind[side]; }
    };
    int f = 0;
    for (int j = 0; j < nj; ++j)
        for (int i = 0; i < nfi_row; ++i, ++f) {
            double x0 = X(i, j), y0 = Y(i, j), x1_ = X(i, j + 1), y1_ = Y(i, j + 1);
            double mx = 0.5 * (x0 + x1_), my = 0.5 * (y0 + y1_);
            if (per_i) {
                int L = j * ni + (i + ni - 1) % ni, R = j * ni + i;
                double mLx = mx, mLy = my;
                if (i == 0) { mLx = 0.5 * (X(ni, j) + X(ni, j + 1)); mLy = 0.5 * (Y(ni, j) + Y(ni, j + 1)); }
                set_face(f, x0, y0, x1_, y1_, true, L, R, mLx, mLy, mx, my, -1);
            } else {
                int L = i > 0 ? j * ni + i - 1 : -1, R = i < ni ? j * ni + i : -1;
                int side = L < 0 ? IDG_IMIN : (R < 0 ? IDG_IMAX : -1);
                set_face(f, x0, y0, x1_, y1_, true, L, R, mx, my, mx, my, side);
            }
        }
    for (int j = 0; j < nfj_rows; ++j)
        for (int i = 0; i < ni; ++i, ++f) {
            double x0 = X(i, j), y0 = Y(i, j), x1_ = X(i + 1, j), y1_ = Y(i + 1, j);
            double mx = 0.5 * (x0 + x1_), my = 0.5 * (y0 + y1_);
            if (per_j) {
                int L = ((j + nj - 1) % nj) * ni + i, R = j * ni + i;
                double mLx = mx, mLy = my;
                if (j == 0) { mLx = 0.5 * (X(i, nj) + X(i + 1, nj)); mLy = 0.5 * (Y(i, nj) + Y(i + 1, nj)); }
                set_face(f, x0, y0, x1_, y1_, false, L, R, mLx, mLy, mx, my, -1);
            } else {
                int L = j > 0 ? (j - 1) * ni + i : -1, R = j < nj ? j * ni + i : -1;
                int side = L < 0 ? IDG_JMIN : (R < 0 ? IDG_JMAX : -1);
                set_face(f, x0, y0, x1_, y1_, false, L, R, mx, my, mx, my, side);
            }
        }
    // cell slots: west, east, south, north
    c->cface.assign(4 * c->N, 0);
    c->cnb.assign(4 * c->N, -1);
    c->csign.assign(4 * c->N, 0);
    c->cr.assign((size_t)8 * c->N, 0.0);
    c->clsg.assign((size_t)8 * c->N, 0.0);
    c->hcell.assign(c->N, 0.0);
    c->dtimp.assign(c->N, 0.0);
    for (int j = 0; j < nj; ++j)
        for (int i = 0; i < ni; ++i) {
            int cc = j * ni + i;
            int fw = j * nfi_row + i;
            int fe = j * nfi_row + (per_i ? (i + 1) % ni : i + 1);
            int fs = nfi_row * nj + j * ni + i;
            int fn = nfi_row * nj + (per_j ? (j + 1) % nj : j + 1) * ni + i;
            int fs4[4] = {fw, fe, fs, fn}, sg4[4] = {-1, +1, -1, +1};
            double smax = 0, a11 = 0, a12 = 0, a22 = 0, d[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
            for (int m = 0; m < 4; ++m) {
                int fi = fs4[m];
                const double *g = &c->fgeo[(size_t)7 * fi];
                c->cface[4 * cc + m] = fi;
                c->csign[4 * cc + m] = sg4[m];
                bool own_L = sg4[m] > 0;
                c->cr[8 * cc + 2 * m] = own_L ? g[3] : g[5];
                c->cr[8 * cc + 2 * m + 1] = own_L ? g[4] : g[6];
                smax = std::max(smax, g[2]);
                int other = own_L ? c->fR[fi] : c->fL[fi];
                c->cnb[4 * cc + m] = other;
                if (other < 0) continue;
                // neighbour displacement through the face: r_own - r_other
                d[m][0] = own_L ? g[3] - g[5] : g[5] - g[3];
                d[m][1] = own_L ? g[4] - g[6] : g[6] - g[4];
                a11 += d[m][0] * d[m][0];
                a12 += d[m][0] * d[m][1];
                a22 += d[m][1] * d[m][1];
            }
            double det = a11 * a22 - a12 * a12;
            if (!(det > 0)) return fail(c, IDG_ERR_ARG, "singular least-squares stencil at cell (%d,%d)", i, j);
            for (int m = 0; m < 4; ++m) {
                if (c->cnb[4 * cc + m] < 0) continue;
                c->clsg[8 * cc + 2 * m] = (a22 * d[m][0] - a12 * d[m][1]) / det;
                c->clsg[8 * cc + 2 * m + 1] = (-a12 * d[m][0] + a11 * d[m][1]) / det;
            }
            c->hcell[cc] = c->area[cc] / smax;
            hmin = std::min(hmin, c->hcell[cc]);
        }
    }
    c->dt = c->cfl_phys * hmin / c->xi_max;
    for (int q = 0; q < c->N; ++q) c->dtimp[q] = c->cfl_imp * c->hcell[q] / c->xi_max;
    const double om = c->omega;
    c->mu_ref = 15.0 * std::sqrt(2.0 * M_PI * c->RT_ref) * c->Kn / (2.0 * (5.0 - 2.0 * om) * (7.0 - 2.0 * om));
    c->built = true;
    return IDG_OK;
}

// -------------------------------------------------------------------------
// workspace layout
// -------------------------------------------------------------------------
struct Layout {
    size_t off = 0;
    char *base = nullptr;
    template <class P> P *take(size_t bytes)
    {
        off = (off + 255) & ~(size_t)255;
        P *p = base ? (P *)(base + off) : nullptr;
        off += bytes;
        return p;
    }
};

size_t layout(idg_ctx *c, char *base, KParams *kp)
{
    Layout L;
    L.base = base;
    const size_t N = c->N, Nv = c->Nv, nf = c->nf;
    const size_t ts = c->precision == IDG_FP64 ? 8 : 4;  // storage scalar
    const size_t t2 = 2 * ts;
    KParams k{};
    k.area = L.take<double>(8 * N);
    k.dtimp = L.take<double>(8 * N);
    k.cface = L.take<int>(16 * N);
    k.cnb = L.take<int>(16 * N);
    k.csign = L.take<int>(16 * N);
    k.crT = L.take<char>(8 * ts * N);
    k.clsgT = L.take<char>(8 * ts * N);
    k.cslotT = L.take<char>(8 * ts * N);
    k.scode = L.take<int>(32 * N);
    k.sched = c->unstr ? L.take<int>(4 * c->sched.size()) : nullptr;
    k.sptr = c->unstr ? L.take<int>(4 * c->sptr.size()) : nullptr;
    k.fL = L.take<int>(4 * nf);
    k.fR = L.take<int>(4 * nf);
    k.fgeo = L.take<double>(56 * nf);
    k.fgeoT = L.take<char>(8 * ts * nf);
    k.fbc = L.take<int>(4 * nf);
    k.fside = L.take<int>(4 * nf);
    k.bconst = L.take<double>(16 * nf);
    k.ux = L.take<double>(8 * Nv);
    k.uy = L.take<double>(8 * Nv);
    k.w = L.take<double>(8 * Nv);
    k.gref = L.take<double>(8 * Nv);
    k.uxf = L.take<float>(4 * Nv);
    k.uyf = L.take<float>(4 * Nv);
    k.wf = L.take<float>(4 * Nv);
    k.greff = L.take<float>(4 * Nv);
    k.bdevG = L.take<char>(4 * ts * Nv);
    k.bdevH = L.take<char>(4 * ts * Nv);
    k.f = L.take<char>(t2 * N * Nv);
    k.fbp = L.take<char>(t2 * N * Nv);
    k.grad = c->limiter ? L.take<char>(4 * ts * N * Nv) : nullptr;
    k.dst = L.take<char>(t2 * N * Nv);
    // the face-flux buffer doubles as the float64 staging area of
    // idg_set_state / idg_get_state (G and H of every cell): on an unstructured
    // mesh (about 1.5 faces per cell for triangles) that can be the larger need
    k.F = L.take<char>(std::max(t2 * nf * Nv, 16 * N * Nv));
    k.W = L.take<double>(32 * N);
    k.cellraw = L.take<char>(8 * idg::kRaw * N);
    k.cellA = L.take<char>(ts * idg::kCellP * N);
    k.cellq = L.take<double>(16 * N);
    k.cellp = L.take<double>(8 * idg::kCellP * N);
    k.cellpT = L.take<char>(ts * idg::kCellP * N);
    k.faceraw = L.take<char>(8 * 12 * nf);
    k.facerw = L.take<double>(8 * nf);
    k.faceA = L.take<char>(ts * idg::kCellP * nf);
    k.phiraw = L.take<char>(32 * nf);
    k.phi = L.take<double>(32 * nf);
    k.rw = L.take<double>(32 * N);
    k.mrec = L.take<char>(24 * ts * N);
    k.mdW = L.take<char>(4 * ts * N);
    k.mdW2 = c->relax_sweeps > 0 ? L.take<char>(4 * ts * N) : nullptr;
    k.wallS = c->implicit_wall ? L.take<double>(8 * nf) : nullptr;
    k.walldrg = c->implicit_wall ? L.take<double>(8 * nf) : nullptr;
    k.mpart = L.take<double>(8 * (N / 32 + 2));
    k.res = L.take<double>(8 * (size_t)idg::kMaxHist);
    k.iter = L.take<int>(256);
    k.status = k.iter + 1;
    k.wallok = k.iter + 2;
    double *mom = L.take<double>(48 * N);
    KParams *kdev = L.take<KParams>(sizeof(KParams));
    if (kp) {
        *kp = k;
        c->moments_dev = mom;
        c->kp_dev = kdev;
    }
    return L.off + 256;
}

// tables of the reference Maxwellian and its float64 moments
void reference_tables(idg_ctx *c, std::vector<double> &gref, KParams &k)
{
    const int Nv = c->Nv;
    const double RTr = c->ref_T * c->RT_ref, lamr = 0.5 / RTr;
    gref.resize(Nv);
    for (int q = 0; q < idg::kRaw; ++q) k.mref_raw[q] = 0.0;
    for (int a = 0; a < 4; ++a) k.mref_flux[a][0] = k.mref_flux[a][1] = 0.0;
    const double kRTr = c->K * RTr;
    for (int q = 0; q < Nv; ++q) {
        double cx = c->ux[q] - c->ref_u, cy = c->uy[q] - c->ref_v;
        gref[q] = c->ref_rho * lamr / M_PI * std::exp(-lamr * (cx * cx + cy * cy));
        double G = gref[q], H = kRTr * G, x = c->ux[q], y = c->uy[q], wq = c->w[q], s2 = x * x + y * y;
        double r[idg::kRaw] = {G, x * G, y * G, x * x * G, x * y * G, y * y * G, x * s2 * G, y * s2 * G, H, x * H, y * H};
        for (int m = 0; m < idg::kRaw; ++m) k.mref_raw[m] += wq * r[m];
        double psi[4] = {G, x * G, y * G, 0.5 * (s2 * G + H)};
        for (int a = 0; a < 4; ++a) {
            k.mref_flux[a][0] += wq * psi[a] * x;
            k.mref_flux[a][1] += wq * psi[a] * y;
        }
    }
    k.rho_r = c->ref_rho;
    k.U_r = c->ref_u;
    k.V_r = c->ref_v;
    k.RT_r = RTr;
}

template <class T> cudaError_t up(T *dst, const std::vector<T> &src)
{
    return cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

template <class T> std::vector<T> cast(const std::vector<double> &v) { return std::vector<T>(v.begin(), v.end()); }

template <class T> cudaError_t upT(const void *dst, const std::vector<double> &src)
{
    std::vector<T> t = cast<T>(src);
    return cudaMemcpy(const_cast<void *>(dst), t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice);
}

cudaError_t up_storage(idg_ctx *c, const void *dst, const std::vector<double> &src)
{
    return c->precision == IDG_FP64 ? upT<double>(dst, src) : upT<float>(dst, src);
}

// Everything that depends on the reference Maxwellian: its table and moments,
// the boundary Maxwellians relative to it, and the per-face half-range sums
// of the diffuse wall (Eq. 35).
idg_status upload_reference(idg_ctx *c)
{
    std::vector<double> gref;
    reference_tables(c, gref, c->kp);
    const int Nv = c->Nv;
    const double kRTr = c->K * c->ref_T * c->RT_ref;
    std::vector<double> bG((size_t)4 * Nv, 0.0), bH((size_t)4 * Nv, 0.0), dG((size_t)4 * Nv, 0.0),
        dH((size_t)4 * Nv, 0.0);
    for (int sd = 0; sd < 4; ++sd) {
        if (c->bc_kind[sd] == IDG_BC_PERIODIC) continue;
        double RT = c->bc_T[sd] * c->RT_ref, lam = 0.5 / RT;
        double rho = c->bc_kind[sd] == IDG_BC_WALL ? 1.0 : c->bc_rho[sd];
        for (int q = 0; q < Nv; ++q) {
            double cx = c->ux[q] - c->bc_u[sd], cy = c->uy[q] - c->bc_v[sd];
            double G = rho * lam / M_PI * std::exp(-lam * (cx * cx + cy * cy));
            size_t i = (size_t)sd * Nv + q;
            bG[i] = G;
            bH[i] = c->K * RT * G;
            dG[i] = G - gref[q];
            dH[i] = c->K * RT * G - kRTr * gref[q];
        }
    }
    std::vector<double> bconst((size_t)2 * c->nf, 0.0);
    for (int f = 0; f < c->nf; ++f) {
        if (c->fbc[f] < 0) continue;
        const double *g = &c->fgeo[(size_t)7 * f];
        double on = c->fL[f] >= 0 ? 1.0 : -1.0;
        int sd = c->fside[f];
        double out = 0.0, in = 0.0;
        for (int q = 0; q < Nv; ++q) {
            double so = on * (c->ux[q] * g[0] + c->uy[q] * g[1]);
            if (so > 0) out += c->w[q] * so * gref[q];
            else if (so < 0) in += c->w[q] * (-so) * bG[(size_t)sd * Nv + q];
        }
        bconst[2 * f] = out;
        bconst[2 * f + 1] = in;
    }
    std::vector<float> gf(gref.begin(), gref.end());
    cudaError_t e;
    if ((e = up((double *)c->kp.gref, gref)) != cudaSuccess) return cuda_fail(c, e, "upload gref");
    if ((e = up((float *)c->kp.greff, gf)) != cudaSuccess) return cuda_fail(c, e, "upload greff");
    if ((e = up_storage(c, c->kp.bdevG, dG)) != cudaSuccess) return cuda_fail(c, e, "upload bdevG");
    if ((e = up_storage(c, c->kp.bdevH, dH)) != cudaSuccess) return cuda_fail(c, e, "upload bdevH");
    if ((e = up((double *)c->kp.bconst, bconst)) != cudaSuccess) return cuda_fail(c, e, "upload bconst");
    return IDG_OK;
}

idg_status check_ready(idg_ctx *c)
{
    if (!c) return IDG_ERR_ARG;
    if (!c->bound) return fail(c, IDG_ERR_STATE, "workspace not bound");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    return IDG_OK;
}

constexpr int kGraphChunk = 16;

void drop_graph(idg_ctx *c)
{
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->gexec1) cudaGraphExecDestroy(c->gexec1);
    c->gexec = c->gexec1 = nullptr;
}

void free_graph_state(idg_ctx *c)
{
    drop_graph(c);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    c->ev_in = c->ev_out = nullptr;
    c->gstream = nullptr;
}

// n (kGraphChunk or 1) iterations captured once (the launch parameters are
// baked in; any change of them drops the graphs)
idg_status launch_chunk_graph(idg_ctx *c, cudaStream_t st, int n)
{
    cudaGraphExec_t &gx = n == 1 ? c->gexec1 : c->gexec;
    cudaError_t e;
    if (!c->gstream) {
        if ((e = cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(c, e, "cudaStreamCreate");
        if ((e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(c, e, "cudaEventCreate");
        if ((e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(c, e, "cudaEventCreate");
    }
    if (!gx) {
        cudaGraph_t g = nullptr;
        if ((e = cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cuda_fail(c, e, "cudaStreamBeginCapture");
        int rc = 0;
        for (int q = 0; q < n && !rc; ++q)
            rc = idg::launch_iteration(c->plan, c->precision == IDG_FP64, c->gstream);
        e = cudaStreamEndCapture(c->gstream, &g);
        if (rc || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(c, rc ? (cudaError_t)rc : e, "graph capture");
        }
        e = cudaGraphInstantiate(&gx, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            gx = nullptr;
            return cuda_fail(c, e, "cudaGraphInstantiate");
        }
    }
    if ((e = cudaEventRecord(c->ev_in, st)) != cudaSuccess) return cuda_fail(c, e, "event");
    if ((e = cudaStreamWaitEvent(c->gstream, c->ev_in, 0)) != cudaSuccess) return cuda_fail(c, e, "wait");
    if ((e = cudaGraphLaunch(gx, c->gstream)) != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
    if ((e = cudaEventRecord(c->ev_out, c->gstream)) != cudaSuccess) return cuda_fail(c, e, "event");
    if ((e = cudaStreamWaitEvent(st, c->ev_out, 0)) != cudaSuccess) return cuda_fail(c, e, "wait");
    return IDG_OK;
}

// Single-instance launch plan and the device copy of the parameters; call
// whenever kp changes (no iteration may be in flight: the library's own
// stream is drained first).
idg_status refresh_plan(idg_ctx *c)
{
    idg::Plan pl{};
    pl.dparams = c->kp_dev;
    pl.doff = nullptr;
    pl.dactive = nullptr;
    pl.ninst = 1;
    idg::blocks_per_instance(c->kp, pl.nblocks);
    if (idg::plan_shapes(&c->kp, 1, c->precision == IDG_FP64, pl))
        return fail(c, IDG_ERR_ARG, "launch shape does not fit in shared memory");
    c->kp.macro_stages = pl.macro_stages;
    c->kp.sweep_stages = pl.sweep_stages;
    pl.explicit_dugks = (c->flags & IDG_NUM_EXPLICIT) ? 1 : 0;
    cudaError_t e;
    if (c->gstream && (e = cudaStreamSynchronize(c->gstream)) != cudaSuccess) return cuda_fail(c, e, "sync");
    if ((e = cudaMemcpy(c->kp_dev, &c->kp, sizeof(KParams), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(c, e, "upload parameters");
    c->plan = pl;
    drop_graph(c);
    return IDG_OK;
}

void restart(idg_ctx *c)
{
    c->start_iter = c->host_iter;
    c->hist.clear();
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

idg_status idg_create(idg_ctx **out, int precision, int device)
{
    if (!out) return IDG_ERR_ARG;
    *out = nullptr;
    if (precision != IDG_FP64 && precision != IDG_MIXED) return IDG_ERR_ARG;
    if (device < 0) return IDG_ERR_ARG;
    idg_ctx *c = new idg_ctx();
    c->precision = precision;
    c->device = device;
    *out = c;
    return IDG_OK;
}

void idg_destroy(idg_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->bound) {
        cudaSetDevice(ctx->device);
        free_graph_state(ctx);
    }
    delete ctx;
}

const char *idg_last_error(const idg_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

idg_status idg_set_mesh_structured(idg_ctx *c, int ni, int nj, const double *nodes_x,
                                   const double *nodes_y)
{
    if (!c) return IDG_ERR_ARG;
    if (c->bound) return fail(c, IDG_ERR_STATE, "setters are closed after idg_bind_workspace");
    if (ni < 1 || nj < 1 || (long long)ni * nj > (1LL << 26) || !nodes_x || !nodes_y)
        return fail(c, IDG_ERR_ARG, "invalid mesh size %d x %d or null nodes", ni, nj);
    size_t nn = (size_t)(ni + 1) * (nj + 1);
    for (size_t q = 0; q < nn; ++q)
        if (!std::isfinite(nodes_x[q]) || !std::isfinite(nodes_y[q]))
            return fail(c, IDG_ERR_ARG, "non-finite node coordinate at %zu", q);
    c->ni = ni;
    c->nj = nj;
    c->unstr = false;
    c->ucell.clear();
    c->uside.clear();
    c->nodes_x.assign(nodes_x, nodes_x + nn);
    c->nodes_y.assign(nodes_y, nodes_y + nn);
    c->built = false;
    return IDG_OK;
}

idg_status idg_set_mesh_unstructured(idg_ctx *c, int nnodes, const double *x, const double *y, int ncells,
                                     const int *cell_nodes, const int *edge_side)
{
    if (!c) return IDG_ERR_ARG;
    if (c->bound) return fail(c, IDG_ERR_STATE, "setters are closed after idg_bind_workspace");
    if (nnodes < 3 || ncells < 1 || ncells > (1 << 24) || !x || !y || !cell_nodes || !edge_side)
        return fail(c, IDG_ERR_ARG, "invalid unstructured mesh sizes (%d nodes, %d cells) or null arrays", nnodes, ncells);
    for (int q = 0; q < nnodes; ++q)
        if (!std::isfinite(x[q]) || !std::isfinite(y[q])) return fail(c, IDG_ERR_ARG, "non-finite node coordinate at %d", q);
    for (int q = 0; q < ncells; ++q) {
        for (int m = 0; m < 4; ++m) {
            const int nd = cell_nodes[4 * q + m];
            if (nd >= nnodes || (nd < 0 && m < 3) || (nd < 0 && nd != -1))
                return fail(c, IDG_ERR_ARG, "cell %d: node %d of slot %d invalid", q, nd, m);
            const int sd = edge_side[4 * q + m];
            if (sd < -1 || sd > 3) return fail(c, IDG_ERR_ARG, "cell %d: boundary group %d of slot %d invalid", q, sd, m);
        }
    }
    c->unstr = true;
    c->ni = ncells;
    c->nj = 1;
    c->nodes_x.assign(x, x + nnodes);
    c->nodes_y.assign(y, y + nnodes);
    c->ucell.assign(cell_nodes, cell_nodes + 4 * (size_t)ncells);
    c->uside.assign(edge_side, edge_side + 4 * (size_t)ncells);
    c->built = false;
    return IDG_OK;
}

idg_status idg_set_velocity_grid(idg_ctx *c, int rule, int nx, int ny, double xmin, double xmax,
                                 double ymin, double ymax)
{
    if (!c) return IDG_ERR_ARG;
    if (c->bound) return fail(c, IDG_ERR_STATE, "setters are closed after idg_bind_workspace");
    if (rule < IDG_NC_TRAP || rule > IDG_GAUSS_HERMITE || nx < 1 || ny < 1 ||
        (long long)nx * ny > idg::kMaxVel)
        return fail(c, IDG_ERR_ARG, "invalid velocity grid (rule %d, %d x %d)", rule, nx, ny);
    std::vector<double> a, b;
    if (!rule_1d(rule, nx, xmin, xmax, 1.0, a, b) || !rule_1d(rule, ny, ymin, ymax, 1.0, a, b))
        return fail(c, IDG_ERR_ARG, "invalid velocity grid (rule %d, %d x %d)", rule, nx, ny);
    c->vrule = rule;
    c->nvx = nx;
    c->nvy = ny;
    c->vx0 = xmin; c->vx1 = xmax; c->vy0 = ymin; c->vy1 = ymax;
    c->built = false;
    return IDG_OK;
}

idg_status idg_set_gas(idg_ctx *c, int K, double Pr, double omega, double Kn, double RT_ref, int model)
{
    if (!c) return IDG_ERR_ARG;
    if (c->bound) return fail(c, IDG_ERR_STATE, "setters are closed after idg_bind_workspace");
    if (K < 0 || K > 16 || !(Pr > 0) || !(omega >= 0 && omega <= 1.5) || !(Kn > 0) || !(RT_ref > 0) ||
        (model != IDG_BGK && model != IDG_SHAKHOV))
        return fail(c, IDG_ERR_ARG, "invalid gas parameters");
    c->K = K; c->Pr = Pr; c->omega = omega; c->Kn = Kn; c->RT_ref = RT_ref; c->model = model;
    c->gas_set = true;
    c->built = false;
    return IDG_OK;
}

idg_status idg_set_boundary(idg_ctx *c, int side, int kind, double rho, double u, double v, double T)
{
    if (!c) return IDG_ERR_ARG;
    if (c->bound) return fail(c, IDG_ERR_STATE, "setters are closed after idg_bind_workspace");
    if (side < 0 || side > 3 || kind < IDG_BC_PERIODIC || kind > IDG_BC_FARFIELD)
        return fail(c, IDG_ERR_ARG, "invalid boundary side %d / kind %d", side, kind);
    if (kind != IDG_BC_PERIODIC && (!(T > 0) || !std::isfinite(u) || !std::isfinite(v)))
        return fail(c, IDG_ERR_ARG, "invalid boundary state");
    if (kind == IDG_BC_FARFIELD && !(rho > 0)) return fail(c, IDG_ERR_ARG, "far field needs rho > 0");
    c->bc_kind[side] = kind;
    c->bc_rho[side] = rho; c->bc_u[side] = u; c->bc_v[side] = v; c->bc_T[side] = T;
    c->built = false;
    return IDG_OK;
}

idg_status idg_set_numerics(idg_ctx *c, double cfl_imp, double cfl_phys, int limiter,
                            double lusgs_omega, int flags)
{
    if (!c) return IDG_ERR_ARG;
    if (c->bound) return fail(c, IDG_ERR_STATE, "setters are closed after idg_bind_workspace");
    if (!(cfl_imp > 0) || !(cfl_phys > 0) || (limiter != 0 && limiter != 1) || !(lusgs_omega >= 1.0) ||
        (flags & ~IDG_NUM_EXPLICIT) != 0)
        return fail(c, IDG_ERR_ARG, "invalid numerics");
    c->cfl_imp = cfl_imp; c->cfl_phys = cfl_phys; c->limiter = limiter;
    c->lusgs_omega = lusgs_omega; c->flags = flags;
    c->built = false;
    return IDG_OK;
}

idg_status idg_set_limiter_smoothing(idg_ctx *c, double K)
{
    if (!c) return IDG_ERR_ARG;
    if (c->bound) return fail(c, IDG_ERR_STATE, "setters are closed after idg_bind_workspace");
    if (!(K >= 0.0) || !std::isfinite(K)) return fail(c, IDG_ERR_ARG, "limiter smoothing constant %g", K);
    c->venkat_k = K;
    c->built = false;
    return IDG_OK;
}

idg_status idg_set_predictor(idg_ctx *c, int relax_sweeps)
{
    if (!c) return IDG_ERR_ARG;
    if (c->bound) return fail(c, IDG_ERR_STATE, "setters are closed after idg_bind_workspace");
    if (relax_sweeps < 0 || relax_sweeps > 64) return fail(c, IDG_ERR_ARG, "relax_sweeps %d outside 0..64", relax_sweeps);
    c->relax_sweeps = relax_sweeps;
    c->built = false;
    return IDG_OK;
}

idg_status idg_set_implicit_wall(idg_ctx *c, int on)
{
    if (!c) return IDG_ERR_ARG;
    if (c->bound) return fail(c, IDG_ERR_STATE, "setters are closed after idg_bind_workspace");
    if (on != 0 && on != 1) return fail(c, IDG_ERR_ARG, "implicit_wall %d is not 0 or 1", on);
    c->implicit_wall = on;
    c->built = false;
    return IDG_OK;
}

idg_status idg_workspace_size(idg_ctx *c, size_t *bytes)
{
    if (!c || !bytes) return IDG_ERR_ARG;
    idg_status s = build(c);
    if (s) return s;
    *bytes = layout(c, nullptr, nullptr);
    return IDG_OK;
}

idg_status idg_get_sizes(const idg_ctx *cc, int *ncell, int *nvel, int *nface)
{
    idg_ctx *c = const_cast<idg_ctx *>(cc);
    if (!c) return IDG_ERR_ARG;
    idg_status s = build(c);
    if (s) return s;
    if (ncell) *ncell = c->N;
    if (nvel) *nvel = c->Nvu;
    if (nface) *nface = c->nf;
    return IDG_OK;
}

idg_status idg_get_dt(const idg_ctx *cc, double *dt)
{
    idg_ctx *c = const_cast<idg_ctx *>(cc);
    if (!c || !dt) return IDG_ERR_ARG;
    idg_status s = build(c);
    if (s) return s;
    *dt = c->dt;
    return IDG_OK;
}

idg_status idg_velocity_grid(const idg_ctx *cc, double *ux, double *uy, double *w)
{
    idg_ctx *c = const_cast<idg_ctx *>(cc);
    if (!c) return IDG_ERR_ARG;
    idg_status s = build(c);
    if (s) return s;
    if (ux) std::memcpy(ux, c->ux.data(), c->Nvu * sizeof(double));
    if (uy) std::memcpy(uy, c->uy.data(), c->Nvu * sizeof(double));
    if (w) std::memcpy(w, c->w.data(), c->Nvu * sizeof(double));
    return IDG_OK;
}

idg_status idg_bind_workspace(idg_ctx *c, void *dev_ptr, size_t bytes)
{
    if (!c || !dev_ptr) return IDG_ERR_ARG;
    if (c->implicit_wall && (c->flags & IDG_NUM_EXPLICIT))
        return fail(c, IDG_ERR_ARG, "the linearised wall belongs to the implicit sweeps, not to explicit DUGKS");
    idg_status s = build(c);
    if (s) return s;
    size_t need = layout(c, nullptr, nullptr);
    if (bytes < need) return fail(c, IDG_ERR_OOM, "workspace of %zu bytes, need %zu", bytes, need);
    if (((uintptr_t)dev_ptr) & 255) return fail(c, IDG_ERR_ARG, "workspace must be 256-byte aligned");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    cudaPointerAttributes at{};
    e = cudaPointerGetAttributes(&at, dev_ptr);
    if (e != cudaSuccess || at.type != cudaMemoryTypeDevice || at.device != c->device) {
        cudaGetLastError();
        return fail(c, IDG_ERR_ARG, "workspace is not device memory of device %d", c->device);
    }
    c->ws = (char *)dev_ptr;
    c->ws_bytes = bytes;
    KParams &k = c->kp;
    layout(c, c->ws, &k);
    k.N = c->N; k.Nv = c->Nv; k.nf = c->nf; k.ni = c->ni; k.nj = c->nj; k.nvx = c->nvx;
    k.K = c->K; k.shakhov = c->model == IDG_SHAKHOV; k.limiter = c->limiter;
    k.venkat_k3 = c->venkat_k * c->venkat_k * c->venkat_k;
    k.per_i = c->bc_kind[IDG_IMIN] == IDG_BC_PERIODIC;
    k.per_j = c->bc_kind[IDG_JMIN] == IDG_BC_PERIODIC;
    k.dt = c->dt; k.h = 0.5 * c->dt; k.mu_ref = c->mu_ref; k.RT_ref = c->RT_ref; k.omega = c->omega;
    k.Pr = c->Pr; k.gam = (double)(c->K + 4) / (double)(c->K + 2); k.lusgs_omega = c->lusgs_omega;
    k.relax_sweeps = c->relax_sweeps;
    k.implicit_wall = c->implicit_wall;
    if (c->unstr) {
        k.per_i = k.per_j = 0;
        k.nsteps_f = c->nsteps_f;
        k.nsteps_b = c->nsteps_b;
    }
    // sweep launch shape: cell slots cover the longest hyperplane up to 64
    // micro sweeps: one thread per cell of the longest hyperplane (of the
    // longest schedule step on an unstructured mesh) and tv velocities per
    // CTA (8 by default, more on very narrow blocks)
    int maxlen = c->unstr ? c->sched_pc : std::min(c->ni, c->nj);
    if (maxlen > 256) return fail(c, IDG_ERR_ARG, "min(ni, nj) = %d exceeds 256", maxlen);
    k.sweep_pc = maxlen;
    k.sweep_vpt = 1;
    k.sweep_tv = 8;
    while (k.sweep_tv > 1 && k.sweep_tv * k.sweep_pc > 512) k.sweep_tv /= 2;
    while (k.sweep_tv < 32 && 2 * k.sweep_tv * k.sweep_pc <= 256) k.sweep_tv *= 2;
    // prefetch depth: 8 hyperplanes where shared memory allows (the plan
    // falls back to 4)
    k.macro_stages = 8;
    k.sweep_stages = 8;
    // float64: the hyperplane-slot kernel (two threads per cell halve each
    // step's float64 chain); float32 storage: one thread per line of cells
    k.macro_kind = c->precision == IDG_FP64 ? 0 : 1;
    // uploads
    std::vector<float> uxf(c->ux.begin(), c->ux.end()), uyf(c->uy.begin(), c->uy.end()),
        wf(c->w.begin(), c->w.end());
    std::vector<double> fgeo8((size_t)8 * c->nf, 0.0), cslot((size_t)8 * c->N, 0.0);
    // micro sweeps: the role of each slot's neighbour in the forward (dir +1)
    // and backward (dir -1) sweep: its slot in the previous hyperplane (>= 0),
    // -2 a ghost or not yet swept, -3 the cell itself, -4 - nb the neighbour
    // nb across a periodic seam
    std::vector<int> scode((size_t)8 * c->N, -2);
    for (int dir = 1, o = 0; dir >= -1; dir -= 2, o += 4 * c->N)
        for (int q = 0; q < c->N; ++q) {
            const int d = q % c->ni + q / c->ni;
            for (int m = 0; m < 4; ++m) {
                const int nb = c->cnb[4 * q + m];
                int code = -2;
                if (nb == q) code = -3;
                else if (nb >= 0 && (dir > 0 ? nb < q : nb > q)) {
                    if (c->unstr) {
                        code = -4 - nb;  // scheduled sweeps read every neighbour from global memory
                    } else {
                        const int nbi = nb % c->ni, dp = d - dir;
                        code = nbi + nb / c->ni == dp ? nbi - std::max(0, dp - (c->nj - 1)) : -4 - nb;
                    }
                }
                scode[o + 4 * q + m] = code;
            }
        }
    for (int q = 0; q < c->nf; ++q)
        for (int m = 0; m < 7; ++m) fgeo8[(size_t)8 * q + m] = c->fgeo[(size_t)7 * q + m];
    // micro sweeps: per slot the outward normal scaled by the face length
    for (int q = 0; q < c->N; ++q)
        for (int m = 0; m < 4; ++m) {
            int fi = c->cface[4 * q + m];
            double s = c->csign[4 * q + m], S = c->fgeo[(size_t)7 * fi + 2];
            cslot[8 * q + 2 * m] = s * c->fgeo[(size_t)7 * fi] * S;
            cslot[8 * q + 2 * m + 1] = s * c->fgeo[(size_t)7 * fi + 1] * S;
        }
    cudaError_t errs[] = {
        up((double *)k.area, c->area), up((double *)k.dtimp, c->dtimp), up((int *)k.cface, c->cface),
        up((int *)k.cnb, c->cnb), up((int *)k.csign, c->csign), up_storage(c, k.crT, c->cr),
        up_storage(c, k.clsgT, c->clsg), up_storage(c, k.cslotT, cslot), up((int *)k.scode, scode), up((int *)k.fL, c->fL),
        up((int *)k.fR, c->fR), up((double *)k.fgeo, c->fgeo), up_storage(c, k.fgeoT, fgeo8),
        up((int *)k.fbc, c->fbc), up((int *)k.fside, c->fside),
        up((double *)k.ux, c->ux), up((double *)k.uy, c->uy), up((double *)k.w, c->w),
        up((float *)k.uxf, uxf), up((float *)k.uyf, uyf), up((float *)k.wf, wf),
        cudaMemset(k.iter, 0, 256), cudaMemset(k.phi, 0, 32 * (size_t)c->nf),
        c->unstr ? up((int *)k.sched, c->sched) : cudaSuccess, c->unstr ? up((int *)k.sptr, c->sptr) : cudaSuccess};
    for (cudaError_t x : errs)
        if (x != cudaSuccess) return cuda_fail(c, x, "workspace upload");
    int rcfg = idg::configure_kernels(c->precision == IDG_FP64);
    if (rcfg) return cuda_fail(c, (cudaError_t)rcfg, "configure kernels");
    c->stage = (double *)k.F;
    c->stage_bytes = std::max((c->precision == IDG_FP64 ? 16 : 8) * (size_t)c->nf * c->Nv, 16 * (size_t)c->N * c->Nv);
    c->bound = true;
    idg_status st = upload_reference(c);
    if (!st) st = refresh_plan(c);
    if (st) { c->bound = false; return st; }
    c->host_iter = 0;
    restart(c);
    return IDG_OK;
}

idg_status idg_init_uniform(idg_ctx *c, double rho, double u, double v, double T, void *stream)
{
    idg_status s = check_ready(c);
    if (s) return s;
    if (!(rho > 0) || !(T > 0) || !std::isfinite(u) || !std::isfinite(v))
        return fail(c, IDG_ERR_ARG, "invalid uniform state");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "sync");
    c->ref_rho = rho; c->ref_u = u; c->ref_v = v; c->ref_T = T;
    if ((s = upload_reference(c))) return s;
    if ((s = refresh_plan(c))) return s;
    const size_t t2 = c->precision == IDG_FP64 ? 16 : 8;
    // f~ = M_ref exactly: deviation zero
    if ((e = cudaMemsetAsync(c->kp.f, 0, t2 * (size_t)c->N * c->Nv, st)) != cudaSuccess)
        return cuda_fail(c, e, "memset f");
    double RT = T * c->RT_ref;
    std::vector<double> W((size_t)4 * c->N);
    for (int q = 0; q < c->N; ++q) {
        W[4 * q] = rho; W[4 * q + 1] = rho * u; W[4 * q + 2] = rho * v;
        W[4 * q + 3] = 0.5 * rho * (u * u + v * v + (c->K + 2) * RT);
    }
    if ((e = cudaMemcpyAsync(c->kp.W, W.data(), W.size() * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(c, e, "upload W");
    if ((e = cudaMemsetAsync(c->kp.status, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(c, e, "status");
    // a restart has no last increment: the wall ghost terms start from zero
    if ((e = cudaMemsetAsync(c->kp.wallok, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(c, e, "wallok");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(c, e, "sync");
    restart(c);
    return IDG_OK;
}

idg_status idg_set_state(idg_ctx *c, const double *G, const double *H, const double *W, void *stream)
{
    idg_status s = check_ready(c);
    if (s) return s;
    if (!G || !H || !W) return fail(c, IDG_ERR_ARG, "null state array");
    cudaStream_t st = (cudaStream_t)stream;
    size_t n = (size_t)c->N * c->Nvu;
    cudaError_t e;
    // page-locked host arrays that the runtime maps into the device's address
    // space are read in place by the conversion kernel over the host link;
    // other host memory is staged as float64 in the face-flux buffer (large
    // enough: nf >= 2N)
    const double *gG = nullptr, *gH = nullptr;
    cudaPointerAttributes aG{}, aH{};
    if (cudaPointerGetAttributes(&aG, G) == cudaSuccess && aG.type == cudaMemoryTypeHost && aG.devicePointer &&
        cudaPointerGetAttributes(&aH, H) == cudaSuccess && aH.type == cudaMemoryTypeHost && aH.devicePointer) {
        gG = (const double *)aG.devicePointer;
        gH = (const double *)aH.devicePointer;
    } else {
        (void)cudaGetLastError();  // a query of plain host memory leaves no error behind
        double *dG = c->stage, *dH = c->stage + n;
        if (2 * n * sizeof(double) > c->stage_bytes) return fail(c, IDG_ERR_STATE, "staging buffer too small");
        if ((e = cudaMemcpyAsync(dG, G, n * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_fail(c, e, "H2D G");
        if ((e = cudaMemcpyAsync(dH, H, n * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_fail(c, e, "H2D H");
        gG = dG;
        gH = dH;
    }
    if ((e = cudaMemcpyAsync(c->kp.W, W, (size_t)c->N * 32, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(c, e, "H2D W");
    int rc = idg::launch_to_dev(c->kp, c->precision == IDG_FP64, gG, gH, c->Nvu, st);
    if (rc) return cuda_fail(c, (cudaError_t)rc, "to_dev");
    if ((e = cudaMemsetAsync(c->kp.wallok, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(c, e, "wallok");
    // a new state clears a divergence recorded by an earlier run
    if ((e = cudaMemsetAsync(c->kp.status, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(c, e, "status");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(c, e, "sync");
    restart(c);
    return IDG_OK;
}

idg_status idg_get_state(idg_ctx *c, double *G, double *H, double *W, void *stream)
{
    idg_status s = check_ready(c);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    size_t n = (size_t)c->N * c->Nvu;
    cudaError_t e;
    double *dG = c->stage, *dH = c->stage + n;
    if (2 * n * sizeof(double) > c->stage_bytes) return fail(c, IDG_ERR_STATE, "staging buffer too small");
    if (G || H) {
        int rc = idg::launch_from_dev(c->kp, c->precision == IDG_FP64, dG, dH, c->Nvu, st);
        if (rc) return cuda_fail(c, (cudaError_t)rc, "from_dev");
        if (G && (e = cudaMemcpyAsync(G, dG, n * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cuda_fail(c, e, "D2H G");
        if (H && (e = cudaMemcpyAsync(H, dH, n * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cuda_fail(c, e, "D2H H");
    }
    if (W && (e = cudaMemcpyAsync(W, c->kp.W, (size_t)c->N * 32, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(c, e, "D2H W");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(c, e, "sync");
    return IDG_OK;
}

// Checkpoint file: a 48-byte header (8-byte magic "IDGCKPT1", int32 format
// version 1, int32 precision, int64 cells, int64 velocities, int64 iterations
// since the last restart, int64 reserved 0); G, H [cells][velocities] and W
// [cells][4] (the idg_get_state view); the reference Maxwellian (rho, u, v,
// T) the storage is taken relative to; and the stored deviations f~ - M_ref
// of G and H.  All float64, little-endian.
namespace {
struct CkptHeader {
    char magic[8];
    int32_t version, precision;
    int64_t ncell, nvel, iters, reserved;
};
static_assert(sizeof(CkptHeader) == 48, "checkpoint header layout");
const char kCkptMagic[8] = {'I', 'D', 'G', 'C', 'K', 'P', 'T', '1'};

// 64-bit FNV-1a over the bytes of the discretisation the state lives on:
// the mesh (node coordinates, unstructured cell lists), the discrete
// velocities and weights, and the internal degrees of freedom K (the
// meaning of H).  Gas, boundary and numerical settings are not part of it:
// a checkpoint may start a run at another Kn or wall state (continuation).
struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void bytes(const void *p, size_t n)
    {
        const unsigned char *b = (const unsigned char *)p;
        for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    }
    void vec(const std::vector<double> &v) { bytes(v.data(), v.size() * sizeof(double)); }
    void vec(const std::vector<int> &v) { bytes(v.data(), v.size() * sizeof(int)); }
};

int64_t discretisation_hash(const idg_ctx *c)
{
    Fnv f;
    const int32_t dims[5] = {c->ni, c->nj, c->unstr ? 1 : 0, c->K, c->Nvu};
    f.bytes(dims, sizeof dims);
    f.vec(c->nodes_x);
    f.vec(c->nodes_y);
    f.vec(c->ucell);
    f.vec(c->uside);
    f.bytes(c->ux.data(), (size_t)c->Nvu * 8);
    f.bytes(c->uy.data(), (size_t)c->Nvu * 8);
    f.bytes(c->w.data(), (size_t)c->Nvu * 8);
    return (int64_t)(f.h & 0x7fffffffffffffffull);
}

bool write_all(FILE *fp, const std::vector<double> &v) { return std::fwrite(v.data(), 8, v.size(), fp) == v.size(); }
bool read_all(FILE *fp, std::vector<double> &v) { return std::fread(v.data(), 8, v.size(), fp) == v.size(); }
}  // namespace

idg_status idg_save(idg_ctx *c, const char *path, void *stream)
{
    idg_status s = check_ready(c);
    if (s) return s;
    if (!path) return fail(c, IDG_ERR_ARG, "null path");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)c->N * c->Nvu;
    std::vector<double> G(n), H(n), W((size_t)4 * c->N), dG(n), dH(n);
    if ((s = idg_get_state(c, G.data(), H.data(), W.data(), stream))) return s;
    // the deviations as stored (exact in float64 for either storage type)
    double *sG = c->stage, *sH = c->stage + n;
    int rc = idg::launch_from_dev(c->kp, c->precision == IDG_FP64, sG, sH, c->Nvu, st, true);
    if (rc) return cuda_fail(c, (cudaError_t)rc, "from_dev");
    cudaError_t e;
    if ((e = cudaMemcpyAsync(dG.data(), sG, n * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dH.data(), sH, n * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(c, e, "D2H deviations");
    CkptHeader h{};
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = 2;
    h.precision = c->precision;
    h.reserved = discretisation_hash(c);
    h.ncell = c->N;
    h.nvel = c->Nvu;
    h.iters = c->host_iter - c->start_iter;
    const std::vector<double> ref = {c->ref_rho, c->ref_u, c->ref_v, c->ref_T};
    FILE *fp = std::fopen(path, "wb");
    if (!fp) return fail(c, IDG_ERR_ARG, "cannot open %s for writing", path);
    bool ok = std::fwrite(&h, sizeof h, 1, fp) == 1 && write_all(fp, G) && write_all(fp, H) && write_all(fp, W) &&
              write_all(fp, ref) && write_all(fp, dG) && write_all(fp, dH);
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok) return fail(c, IDG_ERR_ARG, "short write to %s", path);
    return IDG_OK;
}

idg_status idg_load(idg_ctx *c, const char *path, void *stream)
{
    idg_status s = check_ready(c);
    if (s) return s;
    if (!path) return fail(c, IDG_ERR_ARG, "null path");
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return fail(c, IDG_ERR_ARG, "cannot open %s", path);
    CkptHeader h{};
    if (std::fread(&h, sizeof h, 1, fp) != 1 || std::memcmp(h.magic, kCkptMagic, 8) != 0 ||
        (h.version != 1 && h.version != 2)) {
        std::fclose(fp);
        return fail(c, IDG_ERR_ARG, "%s is not a version-1 or -2 checkpoint", path);
    }
    if (h.version == 2 && h.reserved != discretisation_hash(c)) {
        std::fclose(fp);
        return fail(c, IDG_ERR_ARG, "%s was saved on another mesh, velocity grid or K", path);
    }
    if (h.ncell != c->N || h.nvel != c->Nvu) {
        std::fclose(fp);
        return fail(c, IDG_ERR_ARG, "checkpoint of %lld cells x %lld velocities, context has %d x %d",
                    (long long)h.ncell, (long long)h.nvel, c->N, c->Nvu);
    }
    const size_t n = (size_t)c->N * c->Nvu;
    std::vector<double> G(n), H(n), W((size_t)4 * c->N), ref(4), dG(n), dH(n);
    bool ok = read_all(fp, G) && read_all(fp, H) && read_all(fp, W) && read_all(fp, ref) && read_all(fp, dG) &&
              read_all(fp, dH);
    std::fclose(fp);
    if (!ok) return fail(c, IDG_ERR_ARG, "%s is truncated", path);
    if (!(ref[0] > 0) || !(ref[3] > 0) || !std::isfinite(ref[1]) || !std::isfinite(ref[2]))
        return fail(c, IDG_ERR_ARG, "%s holds an invalid reference Maxwellian", path);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "sync");
    // the storage's reference Maxwellian, then the deviations as stored
    c->ref_rho = ref[0]; c->ref_u = ref[1]; c->ref_v = ref[2]; c->ref_T = ref[3];
    if ((s = upload_reference(c))) return s;
    if ((s = refresh_plan(c))) return s;
    double *sG = c->stage, *sH = c->stage + n;
    if (2 * n * sizeof(double) > c->stage_bytes) return fail(c, IDG_ERR_STATE, "staging buffer too small");
    if ((e = cudaMemcpyAsync(sG, dG.data(), n * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(sH, dH.data(), n * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c->kp.W, W.data(), W.size() * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(c, e, "H2D checkpoint");
    int rc = idg::launch_to_dev(c->kp, c->precision == IDG_FP64, sG, sH, c->Nvu, st, true);
    if (rc) return cuda_fail(c, (cudaError_t)rc, "to_dev");
    if ((e = cudaMemsetAsync(c->kp.wallok, 0, sizeof(int), st)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->kp.status, 0, sizeof(int), st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(c, e, "restart");
    restart(c);
    return IDG_OK;
}

idg_status idg_iterate(idg_ctx *c, int max_iter, double tol, void *stream, int *iters_done,
                       double *residual)
{
    idg_status s = check_ready(c);
    if (s) return s;
    if (max_iter < 0) return fail(c, IDG_ERR_ARG, "max_iter < 0");
    cudaStream_t st = (cudaStream_t)stream;
    const bool fp64 = c->precision == IDG_FP64;
    const int chunk = kGraphChunk;
    if (c->plan.explicit_dugks && max_iter > 0) {
        int rc = idg::launch_explicit_prologue(c->plan, fp64, st);
        if (rc) return cuda_fail(c, (cudaError_t)rc, "launch");
    }
    int done = 0;
    double rel = NAN;
    std::vector<double> buf(chunk);
    int status = 0;
    bool converged = false;
    while (done < max_iter) {
        int n = std::min(chunk, max_iter - done);
        // near the tolerance, step one iteration at a time so the run stops at
        // the crossing: the remaining iterations are predicted from the
        // geometric rate of the last (up to) 16 residuals
        if (tol > 0 && n > 1 && c->hist.size() >= 2) {
            const size_t h = c->hist.size(), m = std::min<size_t>(h - 1, 16);
            const double r1 = c->hist.front(), rl = c->hist.back(), r0 = c->hist[h - 1 - m];
            if (r1 > 0 && rl > 0 && r0 > 0 && rl < r0) {
                const double rate = std::pow(rl / r0, 1.0 / (double)m);
                const double need = std::log(tol * r1 / rl) / std::log(rate);
                if (need < (double)chunk) n = 1;
            }
        }
        long long it0 = c->host_iter;
        if ((n == kGraphChunk || n == 1) && c->use_graph) {
            if ((s = launch_chunk_graph(c, st, n))) return s;
        } else {
            for (int q = 0; q < n; ++q) {
                int rc = idg::launch_iteration(c->plan, fp64, st);
                if (rc) return cuda_fail(c, (cudaError_t)rc, "launch");
            }
        }
        c->host_iter += n;
        done += n;
        // residuals of this chunk from the device ring
        cudaError_t e;
        for (int q = 0; q < n; ++q) {
            long long slot = (it0 + q) & (idg::kMaxHist - 1);
            e = cudaMemcpyAsync(&buf[q], c->kp.res + slot, 8, cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) return cuda_fail(c, e, "D2H residual");
        }
        if ((e = cudaMemcpyAsync(&status, c->kp.status, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_fail(c, e, "D2H status");
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(c, e, "iteration");
        for (int q = 0; q < n; ++q) c->hist.push_back(buf[q]);
        if (status) {
            if (iters_done) *iters_done = done;
            return fail(c, IDG_ERR_NONFINITE, "residual became non-finite");
        }
        double r1 = c->hist.front();
        rel = r1 > 0 ? c->hist.back() / r1 : c->hist.back();
        if (tol > 0 && rel <= tol) { converged = true; break; }
    }
    if (iters_done) *iters_done = done;
    if (residual) *residual = rel;
    if (tol > 0 && !converged) return fail(c, IDG_ERR_NOT_CONVERGED, "residual %.3e above tol %.3e", rel, tol);
    return IDG_OK;
}

idg_status idg_iterate_profiled(idg_ctx *c, void *stream, double *kernel_ms)
{
    idg_status s = check_ready(c);
    if (s) return s;
    if (!kernel_ms) return IDG_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t ev[7];
    for (int q = 0; q < 7; ++q) {
        cudaError_t e = cudaEventCreate(&ev[q]);
        if (e != cudaSuccess) {
            for (int u = 0; u < q; ++u) cudaEventDestroy(ev[u]);
            return cuda_fail(c, e, "cudaEventCreate");
        }
    }
    int rc = c->plan.explicit_dugks ? idg::launch_explicit_prologue(c->plan, c->precision == IDG_FP64, st) : 0;
    if (!rc) rc = idg::launch_iteration(c->plan, c->precision == IDG_FP64, st, (void **)ev);
    cudaError_t e = rc ? (cudaError_t)rc : cudaStreamSynchronize(st);
    double r = 0.0;
    if (e == cudaSuccess) {
        for (int q = 0; q < 6; ++q) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[q], ev[q + 1]);
            kernel_ms[q] = ms;
        }
        long long slot = c->host_iter & (idg::kMaxHist - 1);
        e = cudaMemcpy(&r, c->kp.res + slot, 8, cudaMemcpyDeviceToHost);
    }
    for (int q = 0; q < 7; ++q) cudaEventDestroy(ev[q]);
    if (e != cudaSuccess) return cuda_fail(c, e, "profiled iteration");
    c->host_iter += 1;
    c->hist.push_back(r);
    return IDG_OK;
}

idg_status idg_set_tuning(idg_ctx *c, int key, int value)
{
    idg_status s = check_ready(c);
    if (s) return s;
    KParams k = c->kp;
    if (key == IDG_TUNE_GRAPH) {
        if (value != 0 && value != 1) return fail(c, IDG_ERR_ARG, "graph flag must be 0 or 1");
        c->use_graph = value;
        return IDG_OK;
    }
    if (key == IDG_TUNE_SWEEP_TV) {
        if (value < 1 || value > 32 || (value & (value - 1)) || value * k.sweep_pc > 512)
            return fail(c, IDG_ERR_ARG, "sweep velocities per block %d invalid for %d cell slots", value, k.sweep_pc);
        k.sweep_tv = value;
    } else if (key == IDG_TUNE_SWEEP_VPT) {
        if ((value != 1 && value != 2 && value != 4) || k.Nv % value)
            return fail(c, IDG_ERR_ARG, "velocities per thread %d must be 1, 2 or 4 and divide %d", value, k.Nv);
        k.sweep_vpt = value;
    } else if (key == IDG_TUNE_SWEEP_STAGES) {
        if (value != 2 && value != 4 && value != 8) return fail(c, IDG_ERR_ARG, "sweep stages must be 2, 4 or 8");
        k.sweep_stages = value;
    } else if (key == IDG_TUNE_MACRO_STAGES) {
        if (value != 2 && value != 4 && value != 8) return fail(c, IDG_ERR_ARG, "macro stages must be 2, 4 or 8");
        k.macro_stages = value;
    } else if (key == IDG_TUNE_MACRO_KIND) {
        if (value != 0 && value != 1) return fail(c, IDG_ERR_ARG, "macro kind must be 0 or 1");
        k.macro_kind = value;
        // the prefetch depth is re-derived for the other kernel's records
        k.macro_stages = 8;
    } else {
        return fail(c, IDG_ERR_ARG, "unknown tuning key %d", key);
    }
    idg::Plan trial{};
    idg::blocks_per_instance(k, trial.nblocks);
    if (key == IDG_TUNE_MACRO_KIND && !idg::plan_shapes(&k, 1, c->precision == IDG_FP64, trial))
        k.macro_stages = trial.macro_stages;
    if (idg::plan_shapes(&k, 1, c->precision == IDG_FP64, trial) ||
        trial.sweep_stages != k.sweep_stages || trial.macro_stages != k.macro_stages)
        return fail(c, IDG_ERR_ARG, "launch shape does not fit in shared memory");
    KParams old = c->kp;
    c->kp = k;
    if ((s = refresh_plan(c))) {
        c->kp = old;
        return s;
    }
    return IDG_OK;
}

idg_status idg_get_tuning(const idg_ctx *c, int key, int *value)
{
    if (!c || !value) return IDG_ERR_ARG;
    if (!c->bound) return IDG_ERR_STATE;
    if (key == IDG_TUNE_GRAPH) *value = c->use_graph;
    else if (key == IDG_TUNE_SWEEP_TV) *value = c->kp.sweep_tv;
    else if (key == IDG_TUNE_SWEEP_VPT) *value = c->kp.sweep_vpt;
    else if (key == IDG_TUNE_SWEEP_STAGES) *value = c->plan.sweep_stages;
    else if (key == IDG_TUNE_MACRO_STAGES) *value = c->plan.macro_stages;
    else if (key == IDG_TUNE_MACRO_KIND) *value = c->kp.macro_kind;
    else return IDG_ERR_ARG;
    return IDG_OK;
}

idg_status idg_get_moments(idg_ctx *c, double *out6, void *stream)
{
    idg_status s = check_ready(c);
    if (s) return s;
    if (!out6) return IDG_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = idg::launch_cell_moments(c->kp, c->precision == IDG_FP64, c->moments_dev, st);
    if (rc) return cuda_fail(c, (cudaError_t)rc, "moments");
    cudaError_t e = cudaMemcpyAsync(out6, c->moments_dev, (size_t)c->N * 48, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "D2H moments");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(c, e, "sync");
    return IDG_OK;
}

idg_status idg_get_moments_noalloc(idg_ctx *c, double *out6_dev, void *stream)
{
    idg_status s = check_ready(c);
    if (s) return s;
    if (!out6_dev) return fail(c, IDG_ERR_ARG, "null output");
    if (c->N > idg::kNoAllocMaxCells)
        return fail(c, IDG_ERR_ARG, "idg_get_moments_noalloc handles at most %d cells (this mesh has %d)",
                    idg::kNoAllocMaxCells, c->N);
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, out6_dev);
    if (e != cudaSuccess || at.type != cudaMemoryTypeDevice || at.device != c->device) {
        cudaGetLastError();
        return fail(c, IDG_ERR_ARG, "output is not device memory of device %d", c->device);
    }
    int rc = idg::launch_cell_moments_noalloc(c->kp, c->precision == IDG_FP64, c->device, out6_dev, stream);
    if (rc) return cuda_fail(c, (cudaError_t)rc, "moments (no-allocation variant)");
    return IDG_OK;
}

idg_status idg_get_residual_history(idg_ctx *c, double *out, int cap, int *n)
{
    if (!c || (!out && cap > 0) || cap < 0) return IDG_ERR_ARG;
    int m = std::min<int>(cap, (int)c->hist.size());
    if (m > 0) std::memcpy(out, c->hist.data(), m * sizeof(double));
    if (n) *n = m;
    return IDG_OK;
}

idg_status idg_get_face_flux_moments(idg_ctx *c, double *phi4, void *stream)
{
    idg_status s = check_ready(c);
    if (s) return s;
    if (!phi4) return IDG_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(phi4, c->kp.phi, (size_t)c->nf * 32, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "D2H phi");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(c, e, "sync");
    return IDG_OK;
}

idg_status idg_get_wall_force(idg_ctx *c, int side_mask, double *force2, void *stream)
{
    idg_status s = check_ready(c);
    if (s) return s;
    if (!force2 || side_mask <= 0 || side_mask > 15) return fail(c, IDG_ERR_ARG, "invalid wall-force arguments");
    for (int sd = 0; sd < 4; ++sd)
        if (((side_mask >> sd) & 1) && c->bc_kind[sd] != IDG_BC_WALL)
            return fail(c, IDG_ERR_ARG, "side %d is not a wall", sd);
    std::vector<double> phi((size_t)4 * c->nf);
    if ((s = idg_get_face_flux_moments(c, phi.data(), stream))) return s;
    double fx = 0.0, fy = 0.0;
    for (int f = 0; f < c->nf; ++f) {
        if (c->fbc[f] != IDG_BC_WALL || !((side_mask >> c->fside[f]) & 1)) continue;
        const double on = c->fL[f] >= 0 ? 1.0 : -1.0;  // from the gas into the wall
        fx += on * phi[(size_t)4 * f + 1];
        fy += on * phi[(size_t)4 * f + 2];
    }
    force2[0] = fx;
    force2[1] = fy;
    return IDG_OK;
}

idg_status idg_get_wall(idg_ctx *c, int side, double *out5, int cap, int *nfaces, void *stream)
{
    idg_status s = check_ready(c);
    if (s) return s;
    if (side < 0 || side > 3 || cap < 0 || (cap > 0 && !out5) || !nfaces)
        return fail(c, IDG_ERR_ARG, "invalid wall arguments");
    if (c->bc_kind[side] != IDG_BC_WALL) return fail(c, IDG_ERR_ARG, "side %d is not a wall", side);
    std::vector<double> phi((size_t)4 * c->nf);
    if ((s = idg_get_face_flux_moments(c, phi.data(), stream))) return s;
    const double Uw = c->bc_u[side], Vw = c->bc_v[side];
    int n = 0;
    for (int f = 0; f < c->nf; ++f) {
        if (c->fbc[f] != IDG_BC_WALL || c->fside[f] != side) continue;
        if (n < cap) {
            const double *g = &c->fgeo[(size_t)7 * f];
            const double on = c->fL[f] >= 0 ? 1.0 : -1.0;  // from the gas into the wall
            const int in = c->fL[f] >= 0 ? c->fL[f] : c->fR[f];
            const double nx = on * g[0], ny = on * g[1], S = g[2];
            // momentum flux into the wall per unit length, Pi n
            const double px = on * phi[(size_t)4 * f + 1] / S, py = on * phi[(size_t)4 * f + 2] / S;
            const double en = on * phi[(size_t)4 * f + 3] / S;
            double *o = out5 + (size_t)5 * n;
            o[0] = c->cxc[in] + (c->fL[f] >= 0 ? g[3] : g[5]);
            o[1] = c->cyc[in] + (c->fL[f] >= 0 ? g[4] : g[6]);
            o[2] = px * nx + py * ny;
            o[3] = -px * ny + py * nx;
            o[4] = en - (Uw * px + Vw * py);
        }
        ++n;
    }
    *nfaces = n;
    return IDG_OK;
}

}  // extern "C"

// ===========================================================================
// batches: many contexts advanced by one launch per kernel
// ===========================================================================
struct idg_batch {
    std::vector<idg_ctx *> ctx;
    int precision = IDG_FP64, device = 0;
    std::string err;
    bool bound = false;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    KParams *dparams = nullptr;
    int *doff = nullptr, *dactive = nullptr;
    int *dstatus = nullptr;     // [n] gathered status words
    double *dres = nullptr;     // [n][kGraphChunk] gathered residuals of the last chunk
    std::vector<KParams> hparams;
    std::vector<int> active;
    idg::Plan plan{};
    int use_graph = 1;
    cudaStream_t gstream = nullptr;
    cudaGraphExec_t gexec = nullptr, gexec1 = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

namespace idg {
int launch_batch_gather(const KParams *dparams, int n, int last, double *dres, int *dstatus, void *stream);
}

namespace {

idg_status bfail(idg_batch *b, idg_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    return s;
}

size_t batch_layout(idg_batch *b, char *base)
{
    Layout L;
    L.base = base;
    const size_t n = b->ctx.size();
    KParams *dp = L.take<KParams>(n * sizeof(KParams));
    int *doff = L.take<int>((size_t)idg::KT_COUNT * (n + 1) * sizeof(int));
    int *dact = L.take<int>(n * sizeof(int));
    int *dst = L.take<int>(n * sizeof(int));
    double *dres = L.take<double>(n * kGraphChunk * sizeof(double));
    if (base) {
        b->dparams = dp;
        b->doff = doff;
        b->dactive = dact;
        b->dstatus = dst;
        b->dres = dres;
    }
    return L.off + 256;
}

void batch_drop_graph(idg_batch *b)
{
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->gexec1) cudaGraphExecDestroy(b->gexec1);
    b->gexec = b->gexec1 = nullptr;
}

// (re)upload the instances' parameters and offsets, rebuild the plan
idg_status batch_refresh(idg_batch *b)
{
    const int n = (int)b->ctx.size();
    b->hparams.resize(n);
    std::vector<int> off((size_t)idg::KT_COUNT * (n + 1), 0);
    idg::Plan pl{};
    for (int i = 0; i < n; ++i) {
        b->hparams[i] = b->ctx[i]->kp;
        int nbk[idg::KT_COUNT];
        idg::blocks_per_instance(b->hparams[i], nbk);
        for (int t = 0; t < idg::KT_COUNT; ++t) off[(size_t)t * (n + 1) + i + 1] = off[(size_t)t * (n + 1) + i] + nbk[t];
    }
    for (int t = 0; t < idg::KT_COUNT; ++t) pl.nblocks[t] = off[(size_t)t * (n + 1) + n];
    if (idg::plan_shapes(b->hparams.data(), n, b->precision == IDG_FP64, pl))
        return bfail(b, IDG_ERR_ARG, "batch launch shape does not fit in shared memory");
    pl.dparams = b->dparams;
    pl.doff = b->doff;
    pl.dactive = b->dactive;
    pl.ninst = n;
    cudaError_t e;
    if (b->gstream && (e = cudaStreamSynchronize(b->gstream)) != cudaSuccess)
        return bfail(b, IDG_ERR_CUDA, "sync: %s", cudaGetErrorString(e));
    if ((e = cudaMemcpy(b->dparams, b->hparams.data(), n * sizeof(KParams), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->doff, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->dactive, b->active.data(), n * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess)
        return bfail(b, IDG_ERR_CUDA, "batch upload: %s", cudaGetErrorString(e));
    b->plan = pl;
    batch_drop_graph(b);
    return IDG_OK;
}

idg_status batch_launch(idg_batch *b, cudaStream_t st, int n)
{
    const bool fp64 = b->precision == IDG_FP64;
    if (!b->use_graph || (n != 1 && n != kGraphChunk)) {
        for (int q = 0; q < n; ++q) {
            int rc = idg::launch_iteration(b->plan, fp64, st);
            if (rc) return bfail(b, IDG_ERR_CUDA, "launch: %s", cudaGetErrorString((cudaError_t)rc));
        }
        return IDG_OK;
    }
    cudaError_t e;
    if (!b->gstream) {
        if ((e = cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming)) != cudaSuccess)
            return bfail(b, IDG_ERR_CUDA, "stream/event: %s", cudaGetErrorString(e));
    }
    cudaGraphExec_t &gx = n == 1 ? b->gexec1 : b->gexec;
    if (!gx) {
        cudaGraph_t g = nullptr;
        if ((e = cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return bfail(b, IDG_ERR_CUDA, "capture: %s", cudaGetErrorString(e));
        int rc = 0;
        for (int q = 0; q < n && !rc; ++q) rc = idg::launch_iteration(b->plan, fp64, b->gstream);
        e = cudaStreamEndCapture(b->gstream, &g);
        if (rc || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return bfail(b, IDG_ERR_CUDA, "graph capture failed");
        }
        e = cudaGraphInstantiate(&gx, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            gx = nullptr;
            return bfail(b, IDG_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e));
        }
    }
    if ((e = cudaEventRecord(b->ev_in, st)) != cudaSuccess || (e = cudaStreamWaitEvent(b->gstream, b->ev_in, 0)) != cudaSuccess ||
        (e = cudaGraphLaunch(gx, b->gstream)) != cudaSuccess || (e = cudaEventRecord(b->ev_out, b->gstream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(st, b->ev_out, 0)) != cudaSuccess)
        return bfail(b, IDG_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
    return IDG_OK;
}

}  // namespace

extern "C" {

idg_status idg_batch_create(idg_batch **out, idg_ctx *const *ctxs, int n)
{
    if (!out || !ctxs || n < 1) return IDG_ERR_ARG;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i] || !ctxs[i]->bound) return IDG_ERR_STATE;
        if (ctxs[i]->precision != ctxs[0]->precision || ctxs[i]->device != ctxs[0]->device) return IDG_ERR_ARG;
        if (ctxs[i]->flags & IDG_NUM_EXPLICIT) return IDG_ERR_ARG;  // batches run IDUGKS iterations
        if (ctxs[i]->relax_sweeps != ctxs[0]->relax_sweeps) return IDG_ERR_ARG;  // one predictor per batch
        if (ctxs[i]->unstr) return IDG_ERR_ARG;  // batches hold structured blocks
        if (ctxs[i]->implicit_wall) return IDG_ERR_ARG;  // batches keep zero ghost increments
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return IDG_ERR_ARG;
    }
    idg_batch *b = new idg_batch();
    b->ctx.assign(ctxs, ctxs + n);
    b->precision = ctxs[0]->precision;
    b->device = ctxs[0]->device;
    b->active.assign(n, 1);
    *out = b;
    return IDG_OK;
}

void idg_batch_destroy(idg_batch *b)
{
    if (!b) return;
    if (b->bound) {
        cudaSetDevice(b->device);
        batch_drop_graph(b);
        if (b->ev_in) cudaEventDestroy(b->ev_in);
        if (b->ev_out) cudaEventDestroy(b->ev_out);
        if (b->gstream) cudaStreamDestroy(b->gstream);
    }
    delete b;
}

const char *idg_batch_last_error(const idg_batch *b) { return b ? b->err.c_str() : "null batch"; }

idg_status idg_batch_workspace_size(idg_batch *b, size_t *bytes)
{
    if (!b || !bytes) return IDG_ERR_ARG;
    *bytes = batch_layout(b, nullptr);
    return IDG_OK;
}

idg_status idg_batch_bind_workspace(idg_batch *b, void *dev_ptr, size_t bytes)
{
    if (!b || !dev_ptr) return IDG_ERR_ARG;
    size_t need = batch_layout(b, nullptr);
    if (bytes < need) return bfail(b, IDG_ERR_OOM, "batch workspace of %zu bytes, need %zu", bytes, need);
    if (((uintptr_t)dev_ptr) & 255) return bfail(b, IDG_ERR_ARG, "workspace must be 256-byte aligned");
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return bfail(b, IDG_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    b->ws = (char *)dev_ptr;
    b->ws_bytes = bytes;
    batch_layout(b, b->ws);
    b->bound = true;
    idg_status s = batch_refresh(b);
    if (s) b->bound = false;
    return s;
}

idg_status idg_batch_iterate(idg_batch *b, int max_iter, double tol, void *stream, int *iters_done,
                             double *max_residual, int *converged)
{
    if (!b || max_iter < 0) return IDG_ERR_ARG;
    if (!b->bound) return bfail(b, IDG_ERR_STATE, "batch workspace not bound");
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return bfail(b, IDG_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;
    const int n = (int)b->ctx.size();
    // pick up any change of an instance (restart, tuning) since the last call
    bool stale = false;
    for (int i = 0; i < n; ++i)
        if (std::memcmp(&b->hparams[i], &b->ctx[i]->kp, sizeof(KParams))) stale = true;
    std::vector<int> act(n);
    for (int i = 0; i < n; ++i) {
        const idg_ctx *c = b->ctx[i];
        double rel = c->hist.empty() ? INFINITY : (c->hist.front() > 0 ? c->hist.back() / c->hist.front() : c->hist.back());
        act[i] = !(tol > 0 && rel <= tol);
    }
    if (stale || act != b->active) {
        b->active = act;
        idg_status s = batch_refresh(b);
        if (s) return s;
    }
    std::vector<double> res((size_t)n * kGraphChunk);
    std::vector<int> status(n);
    int done = 0;
    idg_status ret = IDG_OK;
    while (done < max_iter) {
        int any = 0;
        for (int i = 0; i < n; ++i) any |= b->active[i];
        if (!any) break;
        int m = std::min(kGraphChunk, max_iter - done);
        idg_status s = batch_launch(b, st, m);
        if (s) return s;
        done += m;
        int rc = idg::launch_batch_gather(b->dparams, n, m, b->dres, b->dstatus, st);
        if (rc) return bfail(b, IDG_ERR_CUDA, "gather: %s", cudaGetErrorString((cudaError_t)rc));
        if ((e = cudaMemcpyAsync(res.data(), b->dres, res.size() * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(status.data(), b->dstatus, n * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return bfail(b, IDG_ERR_CUDA, "batch residuals: %s", cudaGetErrorString(e));
        bool changed = false;
        for (int i = 0; i < n; ++i) {
            if (!b->active[i]) continue;
            idg_ctx *c = b->ctx[i];
            for (int q = 0; q < m; ++q) c->hist.push_back(res[(size_t)i * kGraphChunk + q]);
            c->host_iter += m;
            if (status[i]) {
                ret = IDG_ERR_NONFINITE;
                fail(c, IDG_ERR_NONFINITE, "residual became non-finite");
                b->active[i] = 0;
                changed = true;
                continue;
            }
            double r1 = c->hist.front();
            double rel = r1 > 0 ? c->hist.back() / r1 : c->hist.back();
            if (tol > 0 && rel <= tol) {
                b->active[i] = 0;
                changed = true;
            }
        }
        if (changed && done < max_iter) {
            if ((e = cudaMemcpyAsync(b->dactive, b->active.data(), n * sizeof(int), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess)
                return bfail(b, IDG_ERR_CUDA, "active flags: %s", cudaGetErrorString(e));
        }
    }
    double worst = 0.0;
    int all = 1;
    for (int i = 0; i < n; ++i) {
        const idg_ctx *c = b->ctx[i];
        double rel = c->hist.empty() ? INFINITY : (c->hist.front() > 0 ? c->hist.back() / c->hist.front() : c->hist.back());
        int conv = tol > 0 && rel <= tol;
        if (converged) converged[i] = conv;
        all &= conv;
        worst = std::max(worst, rel);
    }
    if (iters_done) *iters_done = done;
    if (max_residual) *max_residual = worst;
    if (ret) return bfail(b, ret, "an instance became non-finite");
    if (tol > 0 && !all) return bfail(b, IDG_ERR_NOT_CONVERGED, "largest residual %.3e above tol %.3e", worst, tol);
    return IDG_OK;
}

}  // extern "C"

// -------------------------------------------------------------------------
// discrete adjoint of the steady solve
// -------------------------------------------------------------------------
namespace {

idg::AParams adjoint_shape(const idg_ctx *c)
{
    idg::AParams a{};
    a.N = c->N; a.Nv = c->Nv; a.nf = c->nf; a.ni = c->ni; a.nj = c->nj;
    return a;
}

// A domain bounded by walls and periodic sides only conserves mass in its
// steady equations (the mass residuals sum to zero identically), so its
// steady states form a one-parameter family indexed by the total mass.  The
// adjoint then solves a second right-hand side, the total mass, and returns
// gradients at fixed total mass.
int adjoint_rhs(const idg_ctx *c)
{
    for (int sd = 0; sd < 4; ++sd)
        if (c->bc_kind[sd] == IDG_BC_FARFIELD) return 1;
    return 2;
}

// float64 length of the packed adjoint vector (lambda_G, lambda_H, lambda_W)
size_t krylov_n(const idg_ctx *c) { return (size_t)2 * c->N * c->Nv + (size_t)4 * c->N; }

// the Krylov solve's vectors after the adjoint workspace proper: the basis
// (restart + 1 vectors), x, b, w, and the dot-product partials
size_t krylov_bytes(const idg_ctx *c)
{
    if (c->adj_method != IDG_ADJ_GMRES) return 0;
    return ((size_t)(c->adj_restart + 4) * krylov_n(c) + idg::vec_dot_blocks()) * sizeof(double) + 512;
}

}  // namespace

extern "C" {

idg_status idg_adjoint_workspace_size(idg_ctx *c, size_t *bytes)
{
    if (!c || !bytes) return IDG_ERR_ARG;
    idg_status s = build(c);
    if (s) return s;
    *bytes = idg::adjoint_layout(adjoint_shape(c), adjoint_rhs(c), nullptr, nullptr) + krylov_bytes(c);
    return IDG_OK;
}

idg_status idg_set_adjoint_solver(idg_ctx *c, int method, int restart)
{
    if (!c) return IDG_ERR_ARG;
    if (method != IDG_ADJ_FIXED_POINT && method != IDG_ADJ_GMRES)
        return fail(c, IDG_ERR_ARG, "unknown adjoint solver %d", method);
    if (method == IDG_ADJ_GMRES && (restart < 2 || restart > 64))
        return fail(c, IDG_ERR_ARG, "GMRES restart %d out of [2, 64]", restart);
    c->adj_method = method;
    if (method == IDG_ADJ_GMRES) c->adj_restart = restart;
    return IDG_OK;
}

idg_status idg_set_adjoint_limiter(idg_ctx *c, int mode)
{
    if (!c) return IDG_ERR_ARG;
    if (mode != IDG_ADJ_LIMITER_EXACT && mode != IDG_ADJ_LIMITER_FROZEN)
        return fail(c, IDG_ERR_ARG, "unknown adjoint limiter mode %d", mode);
    c->adj_lim_frozen = mode == IDG_ADJ_LIMITER_FROZEN;
    return IDG_OK;
}

idg_status idg_adjoint(idg_ctx *c, int objective, int side_mask, const int *params, int nparam,
                       void *workspace, size_t bytes, int max_iter, double tol, void *stream, double *J,
                       double *grad, int *iters_done, double *residual)
{
    idg_status s = check_ready(c);
    if (s) return s;
    if (objective != IDG_OBJ_FORCE_X && objective != IDG_OBJ_FORCE_Y)
        return fail(c, IDG_ERR_ARG, "unknown objective %d", objective);
    if (side_mask <= 0 || side_mask > 15) return fail(c, IDG_ERR_ARG, "side mask %d out of range", side_mask);
    for (int sd = 0; sd < 4; ++sd)
        if (((side_mask >> sd) & 1) && c->bc_kind[sd] != IDG_BC_WALL)
            return fail(c, IDG_ERR_ARG, "objective side %d is not a wall", sd);
    if (nparam < 0 || (nparam > 0 && (!params || !grad))) return fail(c, IDG_ERR_ARG, "invalid parameter list");
    for (int i = 0; i < nparam; ++i) {
        int kind = params[i] & 0xff, mask = params[i] >> 8;
        if (kind == IDG_PAR_KN) {
            if (mask) return fail(c, IDG_ERR_ARG, "parameter %d: Kn takes no side mask", i);
            continue;
        }
        if (kind < IDG_PAR_WALL_T || kind > IDG_PAR_WALL_V || mask <= 0 || mask > 15)
            return fail(c, IDG_ERR_ARG, "parameter %d: invalid id 0x%x", i, params[i]);
        for (int sd = 0; sd < 4; ++sd)
            if (((mask >> sd) & 1) && c->bc_kind[sd] != IDG_BC_WALL)
                return fail(c, IDG_ERR_ARG, "parameter %d: side %d is not a wall", i, sd);
    }
    if (c->flags) return fail(c, IDG_ERR_ARG, "the adjoint does not support numerics flags 0x%x", c->flags);
    if (c->relax_sweeps) return fail(c, IDG_ERR_ARG, "the adjoint transposes the LU-SGS predictor only");
    if (c->unstr) return fail(c, IDG_ERR_ARG, "the adjoint runs on structured blocks only");
    if (c->implicit_wall) return fail(c, IDG_ERR_ARG, "the adjoint transposes sweeps with zero ghost increments only");
    if (max_iter < 1 || max_iter > idg::kMaxHist) return fail(c, IDG_ERR_ARG, "max_iter out of [1, %d]", idg::kMaxHist);
    if (!workspace) return fail(c, IDG_ERR_ARG, "null adjoint workspace");
    if (((uintptr_t)workspace) & 255) return fail(c, IDG_ERR_ARG, "adjoint workspace must be 256-byte aligned");
    const int nrhs = adjoint_rhs(c);
    if (c->adj_method == IDG_ADJ_GMRES && nrhs != 1)
        return fail(c, IDG_ERR_ARG, "the GMRES adjoint solves one right-hand side: a domain with a far field");
    const size_t base_need = idg::adjoint_layout(adjoint_shape(c), nrhs, nullptr, nullptr);
    const size_t need = base_need + krylov_bytes(c);
    if (bytes < need) return fail(c, IDG_ERR_OOM, "adjoint workspace of %zu bytes, need %zu", bytes, need);

    idg::AParams base = adjoint_shape(c);
    const KParams &k = c->kp;
    base.K = c->K; base.shakhov = c->model == IDG_SHAKHOV; base.limiter = c->limiter;
    base.lim_frozen = c->adj_lim_frozen;
    base.venkat_k3 = c->venkat_k * c->venkat_k * c->venkat_k;
    base.dt = k.dt; base.h = k.h; base.mu_ref = k.mu_ref; base.RT_ref = k.RT_ref; base.omega = k.omega;
    base.Pr = k.Pr; base.gam = k.gam; base.lusgs_omega = k.lusgs_omega;
    base.kappa = base.shakhov ? (1.0 - c->Pr) / (c->K + 4) : 0.0;
    base.area = k.area; base.dtimp = k.dtimp; base.fgeo = k.fgeo; base.ux = k.ux; base.uy = k.uy; base.w = k.w;
    base.cface = k.cface; base.cnb = k.cnb; base.csign = k.csign; base.fL = k.fL; base.fR = k.fR;
    base.fbc = k.fbc; base.fside = k.fside; base.W = k.W;
    for (int sd = 0; sd < 4; ++sd) {
        base.b_kind[sd] = c->bc_kind[sd];
        base.b_rho[sd] = c->bc_kind[sd] == IDG_BC_WALL ? 1.0 : c->bc_rho[sd];
        base.b_u[sd] = c->bc_u[sd];
        base.b_v[sd] = c->bc_v[sd];
        base.b_RT[sd] = c->bc_T[sd] * c->RT_ref;
    }
    base.obj_axis = objective == IDG_OBJ_FORCE_X ? 0 : 1;
    base.obj_mask = side_mask;
    idg::AParams A[2];
    idg::adjoint_layout(base, nrhs, (char *)workspace, A);

    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(A[0].lsw, c->clsg.data(), c->clsg.size() * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(A[0].crv, c->cr.data(), c->cr.size() * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(c, e, "adjoint geometry upload");
    int rc = idg::launch_from_dev(c->kp, c->precision == IDG_FP64, A[0].G, A[0].H, c->Nv, st);
    if (!rc) rc = idg::launch_adjoint_setup(A[0], st);
    for (int r = 0; r < nrhs && !rc; ++r) rc = idg::launch_adjoint_zero(A[r], st);
    if (rc) return cuda_fail(c, (cudaError_t)rc, "adjoint setup");

    const int chunk = 32;
    const size_t N4 = (size_t)4 * c->N;
    std::vector<double> buf[2], dW[2];
    double first = -1.0, rel = NAN, beta = 0.0;
    int done = 0;
    bool converged = false;
    if (c->adj_method == IDG_ADJ_GMRES) {
        // Restarted GMRES on (I - M^T) lambda = dJ/du.  One pass of the
        // transposed iteration maps lambda to F(lambda) = dJ/du + M^T lambda,
        // so A v = v - F(v) + F(0) and b = F(0); A does not need the spectral
        // radius of M^T below one, as the fixed-point iteration does.  The
        // vectors pack (lambda_G, lambda_H, lambda_W); dot products are summed
        // in a fixed order.  The last pass runs at the solution, leaving the
        // gradient's intermediates as the fixed-point iteration's last pass does.
        const size_t n = krylov_n(c), NNv = (size_t)c->N * c->Nv;
        const int m = c->adj_restart;
        double *kv = (double *)(((uintptr_t)workspace + base_need + 255) & ~(uintptr_t)255);
        double *V = kv, *xv = V + (size_t)(m + 1) * n, *bv = xv + n, *wv = bv + n, *dpart = wv + n;
        const int nblk = idg::vec_dot_blocks();
        std::vector<double> part(nblk);
        auto cpy = [&](double *dst, const double *src, size_t cnt) {
            return cudaMemcpyAsync(dst, src, cnt * 8, cudaMemcpyDeviceToDevice, st);
        };
        auto pack = [&](double *v) {
            cudaError_t x = cpy(v, A[0].lamG, NNv);
            if (x == cudaSuccess) x = cpy(v + NNv, A[0].lamH, NNv);
            if (x == cudaSuccess) x = cpy(v + 2 * NNv, A[0].lamW, N4);
            return x;
        };
        auto unpack = [&](const double *v) {
            cudaError_t x = cpy(A[0].lamG, v, NNv);
            if (x == cudaSuccess) x = cpy(A[0].lamH, v + NNv, NNv);
            if (x == cudaSuccess) x = cpy(A[0].lamW, v + 2 * NNv, N4);
            return x;
        };
        int err = 0;
        auto pass = [&]() {
            if (!err) err = idg::launch_adjoint_iteration(A[0], done % idg::kMaxHist, st);
            ++done;
        };
        auto F = [&](const double *in, double *out) {  // out = F(in)
            if (!err) err = (int)unpack(in);
            pass();
            if (!err) err = (int)pack(out);
        };
        auto axpby = [&](double a, const double *x, double b, double *y) {
            if (!err) err = idg::launch_vec_axpby(a, x, b, y, n, st);
        };
        auto dot = [&](const double *x, const double *y) {
            if (!err) err = idg::launch_vec_dot(x, y, n, dpart, st);
            if (!err) err = (int)cudaMemcpyAsync(part.data(), dpart, nblk * 8, cudaMemcpyDeviceToHost, st);
            if (!err) err = (int)cudaStreamSynchronize(st);
            double t = 0.0;
            for (int q = 0; q < nblk; ++q) t += part[q];
            return err ? NAN : t;
        };
        // b = F(0) (lambda is zero after launch_adjoint_zero); x = 0
        pass();
        if (!err) err = (int)pack(bv);
        if (!err) err = (int)cudaMemsetAsync(xv, 0, n * 8, st);
        const double bnorm = std::sqrt(dot(bv, bv));
        std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
        rel = 1.0;
        while (!err && done < max_iter) {
            // r = b - A x = F(x) - x
            F(xv, wv);
            axpby(-1.0, xv, 1.0, wv);
            const double r0 = std::sqrt(dot(wv, wv));
            rel = bnorm > 0 ? r0 / bnorm : 0.0;
            if (!std::isfinite(rel)) break;
            if ((tol > 0 && rel <= tol) || r0 == 0.0) break;
            axpby(1.0 / r0, wv, 0.0, V);
            std::fill(g.begin(), g.end(), 0.0);
            g[0] = r0;
            int k = 0;
            for (int j = 0; j < m && done < max_iter && !err; ++j) {
                double *vj = V + (size_t)j * n, *w = V + (size_t)(j + 1) * n;
                F(vj, w);                  // w = F(v_j)
                axpby(1.0, vj, -1.0, w);   // w = v_j - F(v_j)
                axpby(1.0, bv, 1.0, w);    // w = A v_j
                for (int i = 0; i <= j; ++i) {  // modified Gram-Schmidt
                    const double hij = dot(w, V + (size_t)i * n);
                    H[(size_t)i * m + j] = hij;
                    axpby(-hij, V + (size_t)i * n, 1.0, w);
                }
                const double hn = std::sqrt(dot(w, w));
                H[(size_t)(j + 1) * m + j] = hn;
                if (hn > 0) axpby(1.0 / hn, w, 0.0, w);
                for (int i = 0; i < j; ++i) {  // earlier rotations on column j
                    const double a0 = H[(size_t)i * m + j], a1 = H[(size_t)(i + 1) * m + j];
                    H[(size_t)i * m + j] = cs[i] * a0 + sn[i] * a1;
                    H[(size_t)(i + 1) * m + j] = -sn[i] * a0 + cs[i] * a1;
                }
                const double a0 = H[(size_t)j * m + j], a1 = H[(size_t)(j + 1) * m + j];
                const double rr = std::hypot(a0, a1);
                cs[j] = rr > 0 ? a0 / rr : 1.0;
                sn[j] = rr > 0 ? a1 / rr : 0.0;
                H[(size_t)j * m + j] = rr;
                H[(size_t)(j + 1) * m + j] = 0.0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                k = j + 1;
                rel = bnorm > 0 ? std::fabs(g[j + 1]) / bnorm : 0.0;
                if (!std::isfinite(rel) || (tol > 0 && rel <= tol) || hn == 0.0) break;
            }
            for (int i = k - 1; i >= 0; --i) {  // H y = g, upper triangular
                double t = g[i];
                for (int q = i + 1; q < k; ++q) t -= H[(size_t)i * m + q] * y[q];
                y[i] = t / H[(size_t)i * m + i];
            }
            for (int i = 0; i < k; ++i) axpby(y[i], V + (size_t)i * n, 1.0, xv);
        }
        if (err) return cuda_fail(c, (cudaError_t)err, "adjoint GMRES");
        if (!std::isfinite(rel)) {
            if (iters_done) *iters_done = done;
            return fail(c, IDG_ERR_NONFINITE, "adjoint GMRES residual became non-finite");
        }
        converged = tol > 0 && rel <= tol;
        // the last pass at the solution: the gradient's intermediates
        if ((e = unpack(xv)) != cudaSuccess) return cuda_fail(c, e, "adjoint GMRES");
        pass();
        if (err) return cuda_fail(c, (cudaError_t)err, "adjoint GMRES");
    } else {
    // Transposed fixed-point iterations, checked every chunk.  With two
    // right-hand sides both lambdas grow linearly along the neutral mode
    // (whose lambda_f part is zero); the multiplier beta = -<dW_J, dW_m> /
    // <dW_m, dW_m> of the lambda_W increments cancels the growth, and
    // lambda_J + beta lambda_m is the fixed-mass adjoint.
    while (done < max_iter) {
        int n = std::min(chunk, max_iter - done);
        for (int q = 0; q < n; ++q)
            for (int r = 0; r < nrhs; ++r)
                if ((rc = idg::launch_adjoint_iteration(A[r], done + q, st))) return cuda_fail(c, (cudaError_t)rc, "adjoint");
        for (int r = 0; r < nrhs; ++r) {
            buf[r].assign(n, 0.0);
            dW[r].assign(N4, 0.0);
            if ((e = cudaMemcpyAsync(buf[r].data(), A[r].res + done, n * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                (e = cudaMemcpyAsync(dW[r].data(), A[r].dlamW, N4 * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                return cuda_fail(c, e, "adjoint residual");
        }
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(c, e, "adjoint iteration");
        done += n;
        double fnorm = buf[0][n - 1], w2 = 0.0, ww = 0.0, wm = 0.0;
        bool finite = std::isfinite(fnorm);
        if (nrhs == 2) {
            for (size_t i = 0; i < N4; ++i) { ww += dW[1][i] * dW[1][i]; wm += dW[0][i] * dW[1][i]; }
            beta = ww > 0 ? -wm / ww : 0.0;
            fnorm += std::fabs(beta) * buf[1][n - 1];
            finite = finite && std::isfinite(buf[1][n - 1]);
        }
        for (size_t i = 0; i < N4; ++i) {
            double d = dW[0][i] + (nrhs == 2 ? beta * dW[1][i] : 0.0);
            w2 += d * d;
        }
        const double upd = fnorm + std::sqrt(w2);
        if (!finite || !std::isfinite(upd)) {
            if (iters_done) *iters_done = done;
            return fail(c, IDG_ERR_NONFINITE, "adjoint update became non-finite");
        }
        // relative to the lambda_f part of the first update, dJ/df
        if (first < 0) first = buf[0][0] > 0 ? buf[0][0] : 1.0;
        rel = upd / first;
        if (tol > 0 && rel <= tol) { converged = true; break; }
    }
    }

    // objective at the linearisation state and the parameter gradients of
    // the last pass: sums in a fixed order on the host
    std::vector<double> fpar((size_t)idg::kFP * c->nf), fpp[2], cpp[2];
    if ((e = cudaMemcpyAsync(fpar.data(), A[0].fpar, fpar.size() * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(c, e, "adjoint results");
    for (int r = 0; r < nrhs; ++r) {
        fpp[r].assign((size_t)idg::kFPar * c->nf, 0.0);
        cpp[r].assign((size_t)2 * c->N, 0.0);
        if ((e = cudaMemcpyAsync(fpp[r].data(), A[r].fpp, fpp[r].size() * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(cpp[r].data(), A[r].cpp, cpp[r].size() * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_fail(c, e, "adjoint results");
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(c, e, "adjoint results");
    double Jv = 0.0, knsum = 0.0, side_par[4][3] = {};
    for (int f = 0; f < c->nf; ++f) {
        const double *fp = &fpar[(size_t)idg::kFP * f];
        const int sd = c->fside[f];
        if (c->fbc[f] == IDG_BC_WALL && ((side_mask >> sd) & 1)) Jv += fp[idg::FP_ON] * fp[idg::FP_PHI1 + base.obj_axis];
    }
    for (int r = 0; r < nrhs; ++r) {
        const double wr = r == 0 ? 1.0 : beta;
        for (int f = 0; f < c->nf; ++f) {
            knsum += wr * fpp[r][(size_t)idg::kFPar * f + 3];
            if (c->fbc[f] == IDG_BC_WALL)
                for (int q = 0; q < 3; ++q) side_par[c->fside[f]][q] += wr * fpp[r][(size_t)idg::kFPar * f + q];
        }
        for (int q = 0; q < c->N; ++q) knsum += wr * (cpp[r][2 * q] + cpp[r][2 * q + 1]);
    }
    for (int i = 0; i < nparam; ++i) {
        int kind = params[i] & 0xff, mask = params[i] >> 8;
        double g = 0.0;
        if (kind == IDG_PAR_KN) g = knsum / c->Kn;
        else
            for (int sd = 0; sd < 4; ++sd) {
                if (!((mask >> sd) & 1)) continue;
                if (kind == IDG_PAR_WALL_U) g += side_par[sd][0];
                else if (kind == IDG_PAR_WALL_V) g += side_par[sd][1];
                else g += side_par[sd][2] * c->RT_ref;
            }
        grad[i] = g;
    }
    c->adj_beta = beta;
    c->adj_nrhs = nrhs;
    if (J) *J = Jv;
    if (iters_done) *iters_done = done;
    if (residual) *residual = rel;
    if (tol > 0 && !converged) return fail(c, IDG_ERR_NOT_CONVERGED, "adjoint update %.3e above tol %.3e", rel, tol);
    return IDG_OK;
}

idg_status idg_adjoint_state(idg_ctx *c, const void *workspace, int which, double *lamG, double *lamH,
                             double *lamW, void *stream)
{
    idg_status s = check_ready(c);
    if (s) return s;
    if (!workspace || (((uintptr_t)workspace) & 255)) return fail(c, IDG_ERR_ARG, "invalid adjoint workspace");
    if (c->adj_nrhs < 1) return fail(c, IDG_ERR_STATE, "no adjoint has been run");
    if (which < 0 || which > c->adj_nrhs || (which == 2 && c->adj_nrhs < 2))
        return fail(c, IDG_ERR_ARG, "adjoint solve %d not available", which);
    const double wJ = which == 2 ? 0.0 : 1.0;
    const double wm = which == 0 ? c->adj_beta : (which == 2 ? 1.0 : 0.0);
    idg::AParams A[2];
    idg::adjoint_layout(adjoint_shape(c), c->adj_nrhs, (char *)workspace, A);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)c->N * c->Nv, n4 = (size_t)4 * c->N;
    double *out[3] = {lamG, lamH, lamW};
    const size_t cnt[3] = {n, n, n4};
    // per-velocity multipliers are stored with the ghost velocities; the
    // caller's arrays have Nvu entries per cell
    auto dst = [&](int q, size_t i) -> double * {
        if (q == 2) return out[q] + i;
        const size_t cc = i / c->Nv, k = i % c->Nv;
        return k < (size_t)c->Nvu ? out[q] + cc * c->Nvu + k : nullptr;
    };
    for (int q = 0; q < 3; ++q) {
        if (!out[q]) continue;
        std::vector<double> v[2];
        for (int r = 0; r < c->adj_nrhs; ++r) {
            v[r].assign(cnt[q], 0.0);
            const double *src = q == 0 ? A[r].lamG : (q == 1 ? A[r].lamH : A[r].lamW);
            cudaError_t e = cudaMemcpyAsync(v[r].data(), src, cnt[q] * 8, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(c, e, "adjoint state");
        }
        for (size_t i = 0; i < cnt[q]; ++i)
            if (double *o = dst(q, i)) *o = wJ * v[0][i] + (c->adj_nrhs == 2 ? wm * v[1][i] : 0.0);
    }
    return IDG_OK;
}

}  // extern "C"
