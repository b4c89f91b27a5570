// idugks_adjoint.cu -- sm_103a kernels of the discrete adjoint of the steady
// IDUGKS solve (float64).
//
// One forward iteration (Section 2.3) maps u = (f~, W) to
//     W'  = W + P_W^-1 R_W(f~, W)                          macroscopic predictor
//     f~' = f~ + P_f^-1 R_f(f~, W, W')                     micro LU-SGS
// with R_W = -sum_f Phi_f (Eq. 27), R_f = -sum_f F_f - 2 Omega/(2 tau' + dt)
// (f~ - f^S(W', q)) (Eq. 23), P_W the LU-SGS operator of Eq. (28)-(31) and
// P_f the one of Eq. (26).  At the steady state R = 0, so the Jacobian of the
// iteration is M = I + P^-1 dR/du (staged as above) and the derivative of P
// drops out.  For an objective J(u, p) the transposed fixed-point iteration
//     lambda <- dJ/du + M^T lambda
// converges at the rate of the forward iteration, and its fixed point gives
//     dJ/dp = dJ/dp|_u + bar_a^T dR_W/dp + bar_b^T dR_f/dp
// with bar_b = P_f^-T lambda_f and bar_a = P_W^-T (lambda_W + (dR_f/dW')^T bar_b).
// One adjoint iteration, in launch order:
//   k_adj_micro_asc, k_adj_micro_desc   bar_b = P_f^-T lambda_f: the transposed
//       factors of Eq. (26) couple each cell to its downwind neighbours; the
//       lower transposed factor runs last, over the hyperplanes in descending order
//   k_adj_wprime    (dR_f/dW')^T bar_b: collision term at the predicted state
//   k_adj_macro     bar_a = P_W^-T (...): transposed block LU-SGS with the Euler
//       flux Jacobians of the own cell, ascending then descending hyperplanes
//   k_adj_face      VJP of the face flux (Eq. 18-19), face state and
//       equilibrium (Eq. 20), wall density (Eq. 35) and the boundary Maxwellian
//   k_adj_gather    VJP of the characteristic reconstruction (Eq. 11, 13), the
//       limiter (Eq. 16-17) and the own part of the least-squares gradient
//   k_adj_cell      neighbour part of the gradient (Eq. 14-15), VJP of fb+
//       (Eq. 12) and of the cell equilibrium, heat flux and tau; update of lambda
//   k_adj_res       norm of the update of lambda
// The limiter is differentiated where it is smooth (binding face and extreme
// neighbour fixed at the linearisation point).
#include "idugks_adjoint.h"

#include "adjoint_math.h"
#include "idugks.h"

#include <cuda_runtime.h>
#include <math.h>

namespace idg {
namespace {

constexpr int kTB = 256;  // threads of the per-cell / per-face kernels

__device__ __forceinline__ double xdn(double ux, double uy, double nx, double ny)
{
    return __dadd_rn(__dmul_rn(ux, nx), __dmul_rn(uy, ny));
}

// fixed-tree block sum (deterministic); every thread gets the result
template <int NV>
__device__ void bsum(double (&v)[NV], double *sm /* >= 32*NV + NV */)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) sm[wid * NV + q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 0; q < NV; ++q) {
            double a = 0.0;
            for (int u = 0; u < nw; ++u) a += sm[u * NV + q];
            sm[32 * NV + q] = a;
        }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = sm[32 * NV + q];
    __syncthreads();
}

__device__ __forceinline__ double pr_eff(const AParams &a) { return a.shakhov ? a.Pr : 1.0; }

__device__ __forceinline__ adj::Eq cell_eq(const AParams &a, const double *cp)
{
    adj::Eq e;
    e.rho = cp[CP_RHO]; e.U = cp[CP_U]; e.V = cp[CP_V]; e.RT = cp[CP_RT];
    e.qx = cp[CP_QX]; e.qy = cp[CP_QY]; e.kappa = a.kappa; e.K = a.K;
    return e;
}

__device__ __forceinline__ adj::Eq face_eq(const AParams &a, const double *fp)
{
    adj::Eq e;
    e.rho = fp[FP_RHO]; e.U = fp[FP_U]; e.V = fp[FP_V]; e.RT = fp[FP_RT];
    e.qx = fp[FP_QX]; e.qy = fp[FP_QY]; e.kappa = a.kappa; e.K = a.K;
    return e;
}

// reconstruction of fb+ of cell c at a face (Eq. 11, 13) for velocity k
__device__ __forceinline__ double recon(const AParams &a, int comp, int c, int k, double rx, double ry)
{
    const size_t ck = (size_t)c * a.Nv + k, NNv = (size_t)a.N * a.Nv;
    const double *fb = comp ? a.fbH : a.fbG;
    const double *sg = a.sig + 2 * (comp * NNv + ck);
    const double phi = a.lim[3 * (comp * NNv + ck)];
    const double ax = rx - a.ux[k] * a.h, ay = ry - a.uy[k] * a.h;
    return fb[ck] + phi * (sg[0] * ax + sg[1] * ay);
}

// ---------------------------------------------------------------------------
// linearisation point
// ---------------------------------------------------------------------------

// per cell: primitives, tau, heat flux of f~, q (Eq. 20), coefficients of
// fb+ (Eq. 12) and of the collision term; then fb+ itself
__global__ void __launch_bounds__(kTB) k_adj_cell_lin(AParams a)
{
    __shared__ double sm[32 * 6 + 6];
    const int c = blockIdx.x, Nv = a.Nv;
    const adj::Prim p = adj::prim_of(a.W + 4 * c, a.K);
    const double tau = adj::tau_of(p.rho, p.RT, a.mu_ref, a.RT_ref, a.omega);
    const double *G = a.G + (size_t)c * Nv, *H = a.H + (size_t)c * Nv;
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < Nv; k += blockDim.x) {
        const double cx = a.ux[k] - p.U, cy = a.uy[k] - p.V, c2 = cx * cx + cy * cy, wk = a.w[k];
        const double e = c2 * G[k] + H[k];
        s[0] += 0.5 * wk * cx * e;
        s[1] += 0.5 * wk * cy * e;
        s[2] += wk * e;
        s[3] += wk * cx * cx * G[k];
        s[4] += wk * cx * cy * G[k];
        s[5] += wk * cy * cy * G[k];
    }
    bsum<6>(s, sm);
    const double Pr = pr_eff(a), dt = a.dt, h = a.h;
    double cp[kCP];
    cp[CP_RHO] = p.rho; cp[CP_U] = p.U; cp[CP_V] = p.V; cp[CP_RT] = p.RT; cp[CP_TAU] = tau;
    cp[CP_QTX] = s[0]; cp[CP_QTY] = s[1];
    cp[CP_QX] = 2.0 * tau * s[0] / (2.0 * tau + dt * Pr);
    cp[CP_QY] = 2.0 * tau * s[1] / (2.0 * tau + dt * Pr);
    cp[CP_C1] = (2.0 * tau - h) / (2.0 * tau + dt);
    cp[CP_C2] = 3.0 * h / (2.0 * tau + dt);
    cp[CP_CQ] = 2.0 * a.area[c] / (2.0 * tau + dt);
    cp[CP_E1] = s[2]; cp[CP_SXX] = s[3]; cp[CP_SXY] = s[4]; cp[CP_SYY] = s[5];
    if (threadIdx.x < kCP) a.cpar[(size_t)kCP * c + threadIdx.x] = cp[threadIdx.x];
    const adj::Eq e = cell_eq(a, cp);
    for (int k = threadIdx.x; k < Nv; k += blockDim.x) {
        double eg, eh;
        adj::eq_eval(e, a.ux[k], a.uy[k], eg, eh);
        a.fbG[(size_t)c * Nv + k] = cp[CP_C1] * G[k] + cp[CP_C2] * eg;
        a.fbH[(size_t)c * Nv + k] = cp[CP_C1] * H[k] + cp[CP_C2] * eh;
    }
}

// per (component, cell, velocity): least-squares gradient (Eq. 14-15) and
// the Venkatakrishnan limiter (Eq. 16-17) with its binding face and extreme
// neighbour
__global__ void k_adj_grad_lin(AParams a)
{
    const size_t NNv = (size_t)a.N * a.Nv;
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= 2 * NNv) return;
    const int comp = t >= NNv;
    const size_t ck = t - comp * NNv;
    const int c = (int)(ck / a.Nv), k = (int)(ck % a.Nv);
    const double *fb = comp ? a.fbH : a.fbG;
    const double v0 = fb[ck];
    double gx = 0.0, gy = 0.0, vmax = v0, vmin = v0;
    int emax = -1, emin = -1;
    for (int m = 0; m < 4; ++m) {
        const int nb = a.cnb[4 * c + m];
        if (nb < 0) continue;
        const double v = fb[(size_t)nb * a.Nv + k];
        gx += a.lsw[8 * c + 2 * m] * (v - v0);
        gy += a.lsw[8 * c + 2 * m + 1] * (v - v0);
        if (v > vmax) { vmax = v; emax = m; }
        if (v < vmin) { vmin = v; emin = m; }
    }
    double phi = 1.0, A = 0.0, B = 0.0;
    int ms = -1, es = -1;
    if (a.limiter) {
        // the smoothing constant's eps^2 = (K h)^3, h = sqrt(area) (0: Eq. 16-17)
        const double e2 = a.venkat_k3 > 0.0 ? a.venkat_k3 * a.area[c] * sqrt(a.area[c]) : 0.0;
        for (int m = 0; m < 4; ++m) {
            const double d = gx * a.crv[8 * c + 2 * m] + gy * a.crv[8 * c + 2 * m + 1];
            double x = 0.0, th = 1.0, P = 0.0;
            int e = -1;
            if (d > 0) { P = vmax - v0; e = emax; }
            else if (d < 0) { P = vmin - v0; e = emin; }
            if (d != 0) {
                x = P / d;
                th = e2 > 0 ? adj::venkat_eps(P, d, e2) : adj::venkat(x);
            }
            if (th < phi) {
                phi = th;
                ms = m;
                es = e;
                // A = dphi / dP, B = dphi / dD at the binding face
                if (a.lim_frozen) {
                    A = B = 0.0;
                } else if (e2 > 0) {
                    adj::venkat_eps_d(P, d, e2, A, B);
                } else {
                    A = adj::venkat_d(x) / d;
                    B = -x * A;
                }
            }
        }
    }
    a.sig[2 * t] = gx;
    a.sig[2 * t + 1] = gy;
    a.lim[3 * t] = phi;
    a.lim[3 * t + 1] = A;
    a.lim[3 * t + 2] = B;
    a.lsl[2 * t] = (signed char)ms;
    a.lsl[2 * t + 1] = (signed char)es;
}

// per face: fb at the half step (Eq. 11, 13 and the boundary conditions),
// its moments, face state, tau, q (Eq. 20), weights of Eq. (18), Phi (Eq. 27)
// and the macroscopic spectral radius of the face
__global__ void __launch_bounds__(kTB) k_adj_face_lin(AParams a)
{
    __shared__ double sm[32 * 6 + 6];
    const int f = blockIdx.x, Nv = a.Nv;
    const int L = a.fL[f], R = a.fR[f], bc = a.fbc[f], sd = a.fside[f];
    const double *g = a.fgeo + 7 * f;
    const double nx = g[0], ny = g[1], S = g[2];
    const bool inner = L >= 0 && R >= 0;
    const int c = L >= 0 ? L : R;
    const double on = inner ? 0.0 : (L >= 0 ? 1.0 : -1.0);
    const double rx = L >= 0 ? g[3] : g[5], ry = L >= 0 ? g[4] : g[6];
    const bool wall = !inner && bc == IDG_BC_WALL;
    double brho = 1.0, bu = 0, bv = 0, bRT = 1.0;
    if (!inner) { brho = a.b_rho[sd]; bu = a.b_u[sd]; bv = a.b_v[sd]; bRT = a.b_RT[sd]; }
    // wall density (Eq. 35)
    double rw = 1.0, in = 0.0, out = 0.0;
    if (wall) {
        double s[2] = {0, 0};
        for (int k = threadIdx.x; k < Nv; k += blockDim.x) {
            const double so = on * xdn(a.ux[k], a.uy[k], nx, ny);
            if (so > 0) s[0] += a.w[k] * so * recon(a, 0, c, k, rx, ry);
            else if (so < 0) {
                double gG, gH;
                adj::bnd_eval(1.0, bu, bv, bRT, a.K, a.ux[k], a.uy[k], gG, gH);
                s[1] += a.w[k] * (-so) * gG;
            }
        }
        bsum<2>(s, sm);
        out = s[0];
        in = s[1];
        rw = out / in;
    }
    // fb at the face and its conserved moments
    double m[4] = {0, 0, 0, 0};
    for (int k = threadIdx.x; k < Nv; k += blockDim.x) {
        const double sn = xdn(a.ux[k], a.uy[k], nx, ny);
        double fg, fh;
        if (inner) {
            if (sn > 0) { fg = recon(a, 0, L, k, g[3], g[4]); fh = recon(a, 1, L, k, g[3], g[4]); }
            else if (sn < 0) { fg = recon(a, 0, R, k, g[5], g[6]); fh = recon(a, 1, R, k, g[5], g[6]); }
            else {
                fg = 0.5 * (recon(a, 0, L, k, g[3], g[4]) + recon(a, 0, R, k, g[5], g[6]));
                fh = 0.5 * (recon(a, 1, L, k, g[3], g[4]) + recon(a, 1, R, k, g[5], g[6]));
            }
        } else {
            const double so = on * sn;
            double gG, gH;
            adj::bnd_eval(wall ? 1.0 : brho, bu, bv, bRT, a.K, a.ux[k], a.uy[k], gG, gH);
            if (so > 0) { fg = recon(a, 0, c, k, rx, ry); fh = recon(a, 1, c, k, rx, ry); }
            else if (so < 0) { fg = rw * gG; fh = rw * gH; }
            else {
                fg = 0.5 * (recon(a, 0, c, k, rx, ry) + rw * gG);
                fh = 0.5 * (recon(a, 1, c, k, rx, ry) + rw * gH);
            }
        }
        a.fbarG[(size_t)f * Nv + k] = fg;
        a.fbarH[(size_t)f * Nv + k] = fh;
        const double x = a.ux[k], y = a.uy[k], wk = a.w[k];
        m[0] += wk * fg;
        m[1] += wk * x * fg;
        m[2] += wk * y * fg;
        m[3] += 0.5 * wk * ((x * x + y * y) * fg + fh);
    }
    bsum<4>(m, sm);
    const adj::Prim p = adj::prim_of(m, a.K);
    const double tau = adj::tau_of(p.rho, p.RT, a.mu_ref, a.RT_ref, a.omega);
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < Nv; k += blockDim.x) {
        const double fg = a.fbarG[(size_t)f * Nv + k], fh = a.fbarH[(size_t)f * Nv + k];
        const double cx = a.ux[k] - p.U, cy = a.uy[k] - p.V, c2 = cx * cx + cy * cy, wk = a.w[k];
        const double e = c2 * fg + fh;
        s[0] += 0.5 * wk * cx * e;
        s[1] += 0.5 * wk * cy * e;
        s[2] += wk * e;
        s[3] += wk * cx * cx * fg;
        s[4] += wk * cx * cy * fg;
        s[5] += wk * cy * cy * fg;
    }
    bsum<6>(s, sm);
    const double Pr = pr_eff(a), h = a.h;
    double fp[kFP];
    fp[FP_RHO] = p.rho; fp[FP_U] = p.U; fp[FP_V] = p.V; fp[FP_RT] = p.RT; fp[FP_TAU] = tau;
    fp[FP_QBX] = s[0]; fp[FP_QBY] = s[1];
    fp[FP_QX] = 2.0 * tau * s[0] / (2.0 * tau + h * Pr);
    fp[FP_QY] = 2.0 * tau * s[1] / (2.0 * tau + h * Pr);
    fp[FP_A] = 2.0 * tau / (2.0 * tau + h);
    fp[FP_B] = h / (2.0 * tau + h);
    fp[FP_RW] = rw; fp[FP_IN] = in; fp[FP_OUT] = out;
    fp[FP_E1] = s[2]; fp[FP_SXX] = s[3]; fp[FP_SXY] = s[4]; fp[FP_SYY] = s[5];
    fp[FP_ON] = on;
    // flux moments Phi (Eq. 19, 27)
    const adj::Eq e = face_eq(a, fp);
    double ph[4] = {0, 0, 0, 0};
    for (int k = threadIdx.x; k < Nv; k += blockDim.x) {
        double eg, eh;
        adj::eq_eval(e, a.ux[k], a.uy[k], eg, eh);
        const double sn = xdn(a.ux[k], a.uy[k], nx, ny);
        const double Fg = sn * S * (fp[FP_A] * a.fbarG[(size_t)f * Nv + k] + fp[FP_B] * eg);
        const double Fh = sn * S * (fp[FP_A] * a.fbarH[(size_t)f * Nv + k] + fp[FP_B] * eh);
        const double x = a.ux[k], y = a.uy[k], wk = a.w[k];
        ph[0] += wk * Fg;
        ph[1] += wk * x * Fg;
        ph[2] += wk * y * Fg;
        ph[3] += 0.5 * wk * ((x * x + y * y) * Fg + Fh);
    }
    bsum<4>(ph, sm);
    fp[FP_PHI0] = wall ? 0.0 : ph[0];
    fp[FP_PHI1] = ph[1]; fp[FP_PHI2] = ph[2]; fp[FP_PHI3] = ph[3];
    // spectral radius (|V.n| + c) S of the macroscopic LU-SGS, averaged over
    // the cells of the face
    double uu = 0, vv = 0, cc = 0;
    int nc = 0;
    for (int side = 0; side < 2; ++side) {
        const int q = side ? R : L;
        if (q < 0) continue;
        const adj::Prim pq = adj::prim_of(a.W + 4 * q, a.K);
        uu += pq.U; vv += pq.V; cc += sqrt(a.gam * pq.RT);
        ++nc;
    }
    if (nc == 2) { uu *= 0.5; vv *= 0.5; cc *= 0.5; }
    fp[FP_LAM] = (fabs(uu * nx + vv * ny) + cc) * S;
    if (threadIdx.x < kFP) a.fpar[(size_t)kFP * f + threadIdx.x] = fp[threadIdx.x];
}

// per cell: diagonal of the macroscopic LU-SGS, Omega/dt_imp + (omega/2) sum Lambda
__global__ void k_adj_macro_lin(AParams a)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.N) return;
    double d = a.area[c] / a.dtimp[c];
    for (int m = 0; m < 4; ++m) {
        const int f = a.cface[4 * c + m];
        if (a.fL[f] == a.fR[f]) continue;
        d += 0.5 * a.lusgs_omega * a.fpar[(size_t)kFP * f + FP_LAM];
    }
    a.DW[c] = d;
}

// ---------------------------------------------------------------------------
// adjoint iteration
// ---------------------------------------------------------------------------

// micro LU-SGS diagonal of Eq. (26) and the cell range of hyperplane d
__device__ __forceinline__ double micro_diag(const AParams &a, int c, int k)
{
    double d = a.area[c] / a.dtimp[c] + a.cpar[(size_t)kCP * c + CP_CQ];
    for (int m = 0; m < 4; ++m) {
        const int f = a.cface[4 * c + m];
        if (a.fL[f] == a.fR[f]) continue;
        const double *g = a.fgeo + 7 * f;
        const double so = a.csign[4 * c + m] * xdn(a.ux[k], a.uy[k], g[0], g[1]);
        if (so > 0) d += so * g[2];
    }
    return d;
}

// sum over neighbours nb (lower: nb < c, else nb > c) of (xi.n_out)^+ S y_nb
template <bool LOWER>
__device__ __forceinline__ double micro_couple(const AParams &a, const double *y, int c, int k)
{
    double acc = 0.0;
    for (int m = 0; m < 4; ++m) {
        const int nb = a.cnb[4 * c + m];
        if (nb < 0 || nb == c || (LOWER ? nb > c : nb < c)) continue;
        const int f = a.cface[4 * c + m];
        if (a.fL[f] == a.fR[f]) continue;
        const double *g = a.fgeo + 7 * f;
        const double so = a.csign[4 * c + m] * xdn(a.ux[k], a.uy[k], g[0], g[1]);
        if (so > 0) acc += so * g[2] * y[(size_t)nb * a.Nv + k];
    }
    return acc;
}

// y = (D - U~^T)^-1 lambda_f: ascending hyperplanes.  Block = 32 velocities x
// 8 warps; blockIdx.y = component.  Dependencies stay inside the block.
__global__ void __launch_bounds__(kTB) k_adj_micro_asc(AParams a)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int k = blockIdx.x * 32 + lane;
    const double *x = blockIdx.y ? a.lamH : a.lamG;
    double *y = blockIdx.y ? a.bbH : a.bbG;
    const int ni = a.ni, nj = a.nj;
    for (int d = 0; d <= ni + nj - 2; ++d) {
        const int i0 = max(0, d - nj + 1), i1 = min(d, ni - 1);
        if (k < a.Nv)
            for (int i = i0 + wid; i <= i1; i += nw) {
                const int c = (d - i) * ni + i;
                const double acc = x[(size_t)c * a.Nv + k] + micro_couple<true>(a, y, c, k);
                y[(size_t)c * a.Nv + k] = acc / micro_diag(a, c, k);
            }
        __syncthreads();
    }
}

// w = (D - L~^T)^-1 D y: descending hyperplanes, in place
__global__ void __launch_bounds__(kTB) k_adj_micro_desc(AParams a)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int k = blockIdx.x * 32 + lane;
    double *y = blockIdx.y ? a.bbH : a.bbG;
    const int ni = a.ni, nj = a.nj;
    for (int d = ni + nj - 2; d >= 0; --d) {
        const int i0 = max(0, d - nj + 1), i1 = min(d, ni - 1);
        if (k < a.Nv)
            for (int i = i0 + wid; i <= i1; i += nw) {
                const int c = (d - i) * ni + i;
                const double up = micro_couple<false>(a, y, c, k);
                y[(size_t)c * a.Nv + k] += up / micro_diag(a, c, k);
            }
        __syncthreads();
    }
}

// per cell: bar W' = (dR_f/dW')^T bar_b from the collision term
// -cq (f~ - f^S(W', q)), cq = 2 Omega/(2 tau' + dt); bar q of the cell from the
// same term; bwp = lambda_W + bar W'
__global__ void __launch_bounds__(kTB) k_adj_wprime(AParams a)
{
    __shared__ double sm[32 * 7 + 7];
    const int c = blockIdx.x, Nv = a.Nv;
    const double *cp = a.cpar + (size_t)kCP * c;
    const adj::Eq e = cell_eq(a, cp);
    const double cq = cp[CP_CQ];
    const double *G = a.G + (size_t)c * Nv, *H = a.H + (size_t)c * Nv;
    const double *bG = a.bbG + (size_t)c * Nv, *bH = a.bbH + (size_t)c * Nv;
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < Nv; k += blockDim.x) {
        double eg, eh;
        adj::eq_eval(e, a.ux[k], a.uy[k], eg, eh);
        s[6] -= bG[k] * (G[k] - eg) + bH[k] * (H[k] - eh);
        adj::eq_vjp(e, a.ux[k], a.uy[k], cq * bG[k], cq * bH[k], s);
    }
    bsum<7>(s, sm);
    if (threadIdx.x == 0) {
        const double tau = cp[CP_TAU];
        double brho = s[0], bRT = s[3], kn = 0.0;
        const double btau = s[6] * (-2.0 * cq / (2.0 * tau + a.dt));
        adj::tau_vjp(tau, cp[CP_RHO], cp[CP_RT], a.omega, btau, brho, bRT, kn);
        double bW[4] = {0, 0, 0, 0};
        adj::prim_vjp(a.W + 4 * c, a.K, brho, s[1], s[2], bRT, bW);
        for (int q = 0; q < 4; ++q) a.bwp[4 * c + q] = a.lamW[4 * c + q] + bW[q];
        a.bqc[2 * c] = s[4];
        a.bqc[2 * c + 1] = s[5];
        a.cpp[2 * c] = kn;
    }
}

// bar_a = P_W^-T bwp: (D + U^T)^-1 ascending, times D, (D + L^T)^-1 descending.
// The transposed blocks of cell c toward neighbour nb are
// -(1/2)(S A(W_c; n_out)^T + omega Lambda I), A the Euler flux Jacobian.
__device__ __forceinline__ void macro_couple(const AParams &a, int c, bool lower, double *acc)
{
    const double *Wc = a.W + 4 * c;
    for (int m = 0; m < 4; ++m) {
        const int nb = a.cnb[4 * c + m];
        if (nb < 0 || nb == c || (lower ? nb > c : nb < c)) continue;
        const int f = a.cface[4 * c + m];
        if (a.fL[f] == a.fR[f]) continue;
        const double *g = a.fgeo + 7 * f;
        const double sgn = a.csign[4 * c + m];
        const double lam = a.fpar[(size_t)kFP * f + FP_LAM];
        const double *y = a.ba + 4 * nb;
        double t[4];
        adj::euler_jacT(Wc, a.gam, sgn * g[0], sgn * g[1], y, t);
        for (int q = 0; q < 4; ++q) acc[q] += 0.5 * (g[2] * t[q] + a.lusgs_omega * lam * y[q]);
    }
}

__global__ void __launch_bounds__(kTB) k_adj_macro(AParams a)
{
    const int ni = a.ni, nj = a.nj;
    for (int d = 0; d <= ni + nj - 2; ++d) {
        const int i0 = max(0, d - nj + 1), i1 = min(d, ni - 1);
        for (int i = i0 + threadIdx.x; i <= i1; i += blockDim.x) {
            const int c = (d - i) * ni + i;
            double acc[4] = {a.bwp[4 * c], a.bwp[4 * c + 1], a.bwp[4 * c + 2], a.bwp[4 * c + 3]};
            macro_couple(a, c, true, acc);
            for (int q = 0; q < 4; ++q) a.ba[4 * c + q] = acc[q] / a.DW[c];
        }
        __syncthreads();
    }
    for (int d = ni + nj - 2; d >= 0; --d) {
        const int i0 = max(0, d - nj + 1), i1 = min(d, ni - 1);
        for (int i = i0 + threadIdx.x; i <= i1; i += blockDim.x) {
            const int c = (d - i) * ni + i;
            double acc[4] = {0, 0, 0, 0};
            macro_couple(a, c, false, acc);
            for (int q = 0; q < 4; ++q) a.ba[4 * c + q] += acc[q] / a.DW[c];
        }
        __syncthreads();
    }
}

// per face: seeds bar F (from bar_b of the two cells), bar Phi (from bar_a and
// the objective), then the VJP of Eq. (18)-(20), the face moments and the
// boundary; writes the adjoint weight of each cell's reconstruction at the face
__global__ void __launch_bounds__(kTB) k_adj_face(AParams a)
{
    __shared__ double sm[32 * 8 + 8];
    __shared__ double bc_sh[8];
    const int f = blockIdx.x, Nv = a.Nv;
    const int L = a.fL[f], R = a.fR[f], bc = a.fbc[f], sd = a.fside[f];
    const double *g = a.fgeo + 7 * f;
    const double nx = g[0], ny = g[1], S = g[2];
    const double *fp = a.fpar + (size_t)kFP * f;
    const bool inner = L >= 0 && R >= 0;
    const bool wall = !inner && bc == IDG_BC_WALL;
    const double on = fp[FP_ON];
    // bar Phi
    double bP[4] = {0, 0, 0, 0};
    for (int q = 0; q < 4; ++q) {
        if (L >= 0) bP[q] -= a.ba[4 * L + q];
        if (R >= 0) bP[q] += a.ba[4 * R + q];
    }
    if (wall) {
        bP[0] = 0.0;
        if (a.seed == 0 && ((a.obj_mask >> sd) & 1)) bP[1 + a.obj_axis] += on;
    }
    const adj::Eq e = face_eq(a, fp);
    const double A = fp[FP_A], Bc = fp[FP_B];
    const double *fbG = a.fbarG + (size_t)f * Nv, *fbH = a.fbarH + (size_t)f * Nv;
    auto barF = [&](int k, double &bg, double &bh) {
        const double x = a.ux[k], y = a.uy[k], wk = a.w[k];
        bg = wk * (bP[0] + x * bP[1] + y * bP[2] + 0.5 * (x * x + y * y) * bP[3]);
        bh = 0.5 * wk * bP[3];
        if (L >= 0) { bg -= a.bbG[(size_t)L * Nv + k]; bh -= a.bbH[(size_t)L * Nv + k]; }
        if (R >= 0) { bg += a.bbG[(size_t)R * Nv + k]; bh += a.bbH[(size_t)R * Nv + k]; }
    };
    // pass 1: weights of the face equilibrium and of a, b
    double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < Nv; k += blockDim.x) {
        double bg, bh, eg, eh;
        barF(k, bg, bh);
        adj::eq_eval(e, a.ux[k], a.uy[k], eg, eh);
        const double snS = xdn(a.ux[k], a.uy[k], nx, ny) * S;
        s[6] += snS * (fbG[k] * bg + fbH[k] * bh);
        s[7] += snS * (eg * bg + eh * bh);
        adj::eq_vjp(e, a.ux[k], a.uy[k], snS * Bc * bg, snS * Bc * bh, s);
    }
    bsum<8>(s, sm);
    if (threadIdx.x == 0) {
        const double tau = fp[FP_TAU], h = a.h, Pr = pr_eff(a);
        const double d1 = 2.0 * tau + h, d2 = 2.0 * tau + h * Pr;
        double btau = (s[6] - s[7]) * 2.0 * h / (d1 * d1);
        const double bqbx = s[4] * 2.0 * tau / d2, bqby = s[5] * 2.0 * tau / d2;
        btau += (s[4] * fp[FP_QBX] + s[5] * fp[FP_QBY]) * 2.0 * h * Pr / (d2 * d2);
        double brho = s[0], bU = s[1], bV = s[2], bRT = s[3], kn = 0.0;
        adj::heat_uv_vjp(fp[FP_E1], fp[FP_SXX], fp[FP_SXY], fp[FP_SYY], bqbx, bqby, bU, bV);
        adj::tau_vjp(tau, fp[FP_RHO], fp[FP_RT], a.omega, btau, brho, bRT, kn);
        // W_f of the face moments: rebuild it from the primitives
        double Wf[4];
        Wf[0] = fp[FP_RHO];
        Wf[1] = fp[FP_RHO] * fp[FP_U];
        Wf[2] = fp[FP_RHO] * fp[FP_V];
        Wf[3] = 0.5 * fp[FP_RHO] * (fp[FP_U] * fp[FP_U] + fp[FP_V] * fp[FP_V] + (a.K + 2) * fp[FP_RT]);
        double bW[4] = {0, 0, 0, 0};
        adj::prim_vjp(Wf, a.K, brho, bU, bV, bRT, bW);
        for (int q = 0; q < 4; ++q) bc_sh[q] = bW[q];
        bc_sh[4] = bqbx;
        bc_sh[5] = bqby;
        bc_sh[6] = kn;
    }
    __syncthreads();
    const double bW0 = bc_sh[0], bW1 = bc_sh[1], bW2 = bc_sh[2], bW3 = bc_sh[3];
    const double bqx = bc_sh[4], bqy = bc_sh[5], kn = bc_sh[6];
    // pass 2: adjoint weight of fb at the face, split to the reconstruction
    // and (boundary faces) the incoming Maxwellian
    const double rw = fp[FP_RW];
    double brw = 0.0, bpar[3] = {0, 0, 0};
    double bnd[4] = {0, 0, 0, 0};
    if (!inner) {
        bnd[0] = wall ? 1.0 : a.b_rho[sd];
        bnd[1] = a.b_u[sd]; bnd[2] = a.b_v[sd]; bnd[3] = a.b_RT[sd];
    }
    for (int k = threadIdx.x; k < Nv; k += blockDim.x) {
        double bg, bh;
        barF(k, bg, bh);
        const double x = a.ux[k], y = a.uy[k], wk = a.w[k];
        const double sn = xdn(x, y, nx, ny);
        const double cx = x - fp[FP_U], cy = y - fp[FP_V], cq = 0.5 * wk * (cx * bqx + cy * bqy);
        const double wm = wk * (bW0 + x * bW1 + y * bW2 + 0.5 * (x * x + y * y) * bW3);
        double tg = sn * S * A * bg + wm + (cx * cx + cy * cy) * cq;
        double th = sn * S * A * bh + 0.5 * wk * bW3 + cq;
        if (!inner) {
            const double so = on * sn;
            const double fr = so < 0 ? 1.0 : (so == 0 ? 0.5 : 0.0);
            if (fr > 0) {
                double gG, gH;
                adj::bnd_eval(bnd[0], bnd[1], bnd[2], bnd[3], a.K, x, y, gG, gH);
                if (wall) {
                    brw += fr * (gG * tg + gH * th);
                    adj::bnd_vjp(1.0, bnd[1], bnd[2], bnd[3], a.K, x, y, fr * rw * tg, fr * rw * th, bpar[0],
                                 bpar[1], bpar[2]);
                }
            }
            if (so < 0) tg = th = 0.0;
        }
        a.bfG[(size_t)f * Nv + k] = tg;
        a.bfH[(size_t)f * Nv + k] = th;
    }
    if (wall) {
        // pass 3: rho_w = out / in (Eq. 35)
        double t[4] = {brw, bpar[0], bpar[1], bpar[2]};
        bsum<4>(t, sm);
        const double bout = t[0] / fp[FP_IN], bin = -t[0] * fp[FP_OUT] / (fp[FP_IN] * fp[FP_IN]);
        double u[3] = {0, 0, 0};
        for (int k = threadIdx.x; k < Nv; k += blockDim.x) {
            const double x = a.ux[k], y = a.uy[k], wk = a.w[k];
            const double so = on * xdn(x, y, nx, ny);
            if (so > 0) a.bfG[(size_t)f * Nv + k] += wk * so * bout;
            else if (so < 0)
                adj::bnd_vjp(1.0, bnd[1], bnd[2], bnd[3], a.K, x, y, wk * (-so) * bin, 0.0, u[0], u[1], u[2]);
        }
        bsum<3>(u, sm);
        if (threadIdx.x == 0) {
            a.fpp[kFPar * f + 0] = t[1] + u[0];
            a.fpp[kFPar * f + 1] = t[2] + u[1];
            a.fpp[kFPar * f + 2] = t[3] + u[2];
        }
    } else if (threadIdx.x == 0) {
        a.fpp[kFPar * f + 0] = a.fpp[kFPar * f + 1] = a.fpp[kFPar * f + 2] = 0.0;
    }
    if (threadIdx.x == 0) a.fpp[kFPar * f + 3] = kn;
}

// per (component, cell, velocity): collect the weights of the cell's
// reconstructions at the faces where it is upwind (half at xi.n = 0), then the
// VJP of fb+_c + phi sigma.(x_f - xi h - x_c), of the limiter and of the own
// term of the least-squares gradient
__global__ void k_adj_gather(AParams a)
{
    const size_t NNv = (size_t)a.N * a.Nv;
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= 2 * NNv) return;
    const int comp = t >= NNv;
    const size_t ck = t - comp * NNv;
    const int c = (int)(ck / a.Nv), k = (int)(ck % a.Nv);
    const double *bf = comp ? a.bfH : a.bfG;
    const double sx = a.sig[2 * t], sy = a.sig[2 * t + 1], phi = a.lim[3 * t];
    const double ux = a.ux[k], uy = a.uy[k], h = a.h;
    double bself = 0.0, bsx = 0.0, bsy = 0.0, bphi = 0.0;
    for (int m = 0; m < 4; ++m) {
        const int f = a.cface[4 * c + m];
        const double *g = a.fgeo + 7 * f;
        const double so = a.csign[4 * c + m] * xdn(ux, uy, g[0], g[1]);
        const double wt = so > 0 ? 1.0 : (so == 0 ? 0.5 : 0.0);
        if (wt == 0.0) continue;
        const double b = wt * bf[(size_t)f * a.Nv + k];
        const double ax = a.crv[8 * c + 2 * m] - ux * h, ay = a.crv[8 * c + 2 * m + 1] - uy * h;
        bself += b;
        bsx += phi * b * ax;
        bsy += phi * b * ay;
        bphi += b * (sx * ax + sy * ay);
    }
    double bext = 0.0;
    const int ms = a.lsl[2 * t], es = a.lsl[2 * t + 1];
    if (ms >= 0) {
        const double A = a.lim[3 * t + 1], B = a.lim[3 * t + 2];
        bself -= A * bphi;
        if (es >= 0) bext = A * bphi;
        else bself += A * bphi;
        bsx += a.crv[8 * c + 2 * ms] * B * bphi;
        bsy += a.crv[8 * c + 2 * ms + 1] * B * bphi;
    }
    for (int m = 0; m < 4; ++m) {
        const int nb = a.cnb[4 * c + m];
        if (nb < 0 || nb == c) continue;
        bself -= a.lsw[8 * c + 2 * m] * bsx + a.lsw[8 * c + 2 * m + 1] * bsy;
    }
    double *r = a.crec + 4 * t;
    r[0] = bself;
    r[1] = bsx;
    r[2] = bsy;
    r[3] = bext;
}

// per cell: adjoint weight of fb+ (own record plus the neighbours' gradient
// and limiter terms), VJP of fb+ = c1 f~ + c2 f^S (Eq. 12), of the equilibrium,
// q (Eq. 20), the heat flux and tau; lambda <- lambda + increment
__global__ void __launch_bounds__(kTB) k_adj_cell(AParams a)
{
    __shared__ double sm[32 * 8 + 8];
    __shared__ double bc_sh[2];
    const int c = blockIdx.x, Nv = a.Nv;
    const size_t NNv = (size_t)a.N * Nv;
    const double *cp = a.cpar + (size_t)kCP * c;
    const adj::Eq e = cell_eq(a, cp);
    const double c1 = cp[CP_C1], c2 = cp[CP_C2], cq = cp[CP_CQ];
    const double *G = a.G + (size_t)c * Nv, *H = a.H + (size_t)c * Nv;
    int nbs[4], opp[4];
    double lwx[4], lwy[4];
    for (int m = 0; m < 4; ++m) {
        int nb = a.cnb[4 * c + m];
        if (nb == c) nb = -1;
        nbs[m] = nb;
        opp[m] = m ^ 1;
        lwx[m] = nb >= 0 ? a.lsw[8 * nb + 2 * opp[m]] : 0.0;
        lwy[m] = nb >= 0 ? a.lsw[8 * nb + 2 * opp[m] + 1] : 0.0;
    }
    double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < Nv; k += blockDim.x) {
        double b[2];
        for (int comp = 0; comp < 2; ++comp) {
            const size_t t = comp * NNv + (size_t)c * Nv + k;
            double v = a.crec[4 * t];
            for (int m = 0; m < 4; ++m) {
                if (nbs[m] < 0) continue;
                const size_t tn = comp * NNv + (size_t)nbs[m] * Nv + k;
                const double *r = a.crec + 4 * tn;
                v += lwx[m] * r[1] + lwy[m] * r[2];
                if (a.lsl[2 * tn + 1] == opp[m]) v += r[3];
            }
            b[comp] = v;
        }
        a.bfb[(size_t)c * Nv + k] = b[0];
        a.bfb[NNv + (size_t)c * Nv + k] = b[1];
        double eg, eh;
        adj::eq_eval(e, a.ux[k], a.uy[k], eg, eh);
        s[6] += G[k] * b[0] + H[k] * b[1];
        s[7] += eg * b[0] + eh * b[1];
        adj::eq_vjp(e, a.ux[k], a.uy[k], c2 * b[0], c2 * b[1], s);
    }
    bsum<8>(s, sm);
    if (threadIdx.x == 0) {
        const double tau = cp[CP_TAU], dt = a.dt, h = a.h, Pr = pr_eff(a);
        const double d1 = 2.0 * tau + dt, d2 = 2.0 * tau + dt * Pr;
        const double bqx = s[4] + a.bqc[2 * c], bqy = s[5] + a.bqc[2 * c + 1];
        const double bqtx = bqx * 2.0 * tau / d2, bqty = bqy * 2.0 * tau / d2;
        double btau = s[6] * 2.0 * (dt + h) / (d1 * d1) - s[7] * 6.0 * h / (d1 * d1) +
                      (bqx * cp[CP_QTX] + bqy * cp[CP_QTY]) * 2.0 * dt * Pr / (d2 * d2);
        double brho = s[0], bU = s[1], bV = s[2], bRT = s[3], kn = 0.0;
        adj::heat_uv_vjp(cp[CP_E1], cp[CP_SXX], cp[CP_SXY], cp[CP_SYY], bqtx, bqty, bU, bV);
        adj::tau_vjp(tau, cp[CP_RHO], cp[CP_RT], a.omega, btau, brho, bRT, kn);
        double bW[4] = {0, 0, 0, 0};
        adj::prim_vjp(a.W + 4 * c, a.K, brho, bU, bV, bRT, bW);
        if (a.seed == 1) bW[0] += a.area[c];  // d(sum Omega W_0)/dW
        for (int q = 0; q < 4; ++q) {
            const double nw = a.bwp[4 * c + q] + bW[q];
            a.dlamW[4 * c + q] = nw - a.lamW[4 * c + q];
            a.lamW[4 * c + q] = nw;
        }
        a.cpp[2 * c + 1] = kn;
        bc_sh[0] = bqtx;
        bc_sh[1] = bqty;
    }
    __syncthreads();
    const double bqtx = bc_sh[0], bqty = bc_sh[1];
    double r[1] = {0.0};
    for (int k = threadIdx.x; k < Nv; k += blockDim.x) {
        const size_t ck = (size_t)c * Nv + k;
        const double cx = a.ux[k] - e.U, cy = a.uy[k] - e.V, hq = 0.5 * a.w[k] * (cx * bqtx + cy * bqty);
        const double dg = c1 * a.bfb[ck] - cq * a.bbG[ck] + (cx * cx + cy * cy) * hq;
        const double dh = c1 * a.bfb[NNv + ck] - cq * a.bbH[ck] + hq;
        a.lamG[ck] += dg;
        a.lamH[ck] += dh;
        r[0] += dg * dg + dh * dh;
    }
    bsum<1>(r, sm);
    if (threadIdx.x == 0) a.rpart[c] = r[0];
}

__global__ void __launch_bounds__(kTB) k_adj_res(AParams a, int it)
{
    __shared__ double sm[32 + 1];
    double r[1] = {0.0};
    for (int c = threadIdx.x; c < a.N; c += blockDim.x) r[0] += a.rpart[c];
    bsum<1>(r, sm);
    if (threadIdx.x == 0) a.res[it] = sqrt(r[0]);
}

unsigned nblk(size_t n, int tb) { return (unsigned)((n + tb - 1) / tb); }

}  // namespace

size_t adjoint_layout(const AParams &s, int nrhs, char *base, AParams *out)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        off = (off + 255) & ~(size_t)255;
        char *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    const size_t N = s.N, Nv = s.Nv, nf = s.nf, NNv = N * Nv, d = sizeof(double);
    AParams a = s;
    // linearisation, shared by the solves
    a.lsw = (double *)take(8 * N * d);
    a.crv = (double *)take(8 * N * d);
    a.G = (double *)take(NNv * d);
    a.H = (double *)take(NNv * d);
    a.cpar = (double *)take(kCP * N * d);
    a.fbG = (double *)take(NNv * d);
    a.fbH = (double *)take(NNv * d);
    a.sig = (double *)take(4 * NNv * d);
    a.lim = (double *)take(6 * NNv * d);
    a.lsl = (signed char *)take(4 * NNv);
    a.fpar = (double *)take(kFP * nf * d);
    a.fbarG = (double *)take(nf * Nv * d);
    a.fbarH = (double *)take(nf * Nv * d);
    a.DW = (double *)take(N * d);
    for (int r = 0; r < nrhs; ++r) {
        a.seed = r;
        a.lamG = (double *)take(NNv * d);
        a.lamH = (double *)take(NNv * d);
        a.lamW = (double *)take(4 * N * d);
        a.bbG = (double *)take(NNv * d);
        a.bbH = (double *)take(NNv * d);
        a.bwp = (double *)take(4 * N * d);
        a.ba = (double *)take(4 * N * d);
        a.bqc = (double *)take(2 * N * d);
        a.bfG = (double *)take(nf * Nv * d);
        a.bfH = (double *)take(nf * Nv * d);
        a.crec = (double *)take(8 * NNv * d);
        a.bfb = (double *)take(2 * NNv * d);
        a.fpp = (double *)take(kFPar * nf * d);
        a.cpp = (double *)take(2 * N * d);
        a.rpart = (double *)take(N * d);
        a.res = (double *)take(kMaxHist * d);
        a.dlamW = (double *)take(4 * N * d);
        if (out) out[r] = a;
    }
    return off + 256;
}

int launch_adjoint_setup(const AParams &a, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    const size_t NNv = (size_t)a.N * a.Nv;
    k_adj_cell_lin<<<a.N, kTB, 0, st>>>(a);
    k_adj_grad_lin<<<nblk(2 * NNv, 256), 256, 0, st>>>(a);
    k_adj_face_lin<<<a.nf, kTB, 0, st>>>(a);
    k_adj_macro_lin<<<nblk(a.N, 128), 128, 0, st>>>(a);
    return (int)cudaGetLastError();
}

int launch_adjoint_zero(const AParams &a, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    const size_t NNv = (size_t)a.N * a.Nv;
    cudaMemsetAsync(a.lamG, 0, NNv * sizeof(double), st);
    cudaMemsetAsync(a.lamH, 0, NNv * sizeof(double), st);
    cudaMemsetAsync(a.lamW, 0, 4 * (size_t)a.N * sizeof(double), st);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// vector operations of the Krylov solve (float64, deterministic: fixed grid,
// per-block partial sums summed by the host in block order)
// ---------------------------------------------------------------------------
constexpr int kVecBlocks = 1024, kVecThreads = 256;

__global__ void __launch_bounds__(kVecThreads) k_vec_dot(const double *x, const double *y, size_t n, double *part)
{
    __shared__ double sm[kVecThreads / 32];
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)kVecThreads + threadIdx.x; i < n; i += (size_t)kVecBlocks * kVecThreads)
        s += x[i] * y[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kVecThreads / 32; ++w) t += sm[w];
        part[blockIdx.x] = t;
    }
}

// y = a x + b y
__global__ void k_vec_axpby(double a, const double *x, double b, double *y, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}

int launch_vec_dot(const double *x, const double *y, size_t n, double *dpart, void *stream)
{
    k_vec_dot<<<kVecBlocks, kVecThreads, 0, (cudaStream_t)stream>>>(x, y, n, dpart);
    return (int)cudaGetLastError();
}

int launch_vec_axpby(double a, const double *x, double b, double *y, size_t n, void *stream)
{
    k_vec_axpby<<<kVecBlocks, kVecThreads, 0, (cudaStream_t)stream>>>(a, x, b, y, n);
    return (int)cudaGetLastError();
}

int vec_dot_blocks() { return kVecBlocks; }

int launch_adjoint_iteration(const AParams &a, int it, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    const size_t NNv = (size_t)a.N * a.Nv;
    const dim3 sweep_grid(nblk(a.Nv, 32), 2);
    k_adj_micro_asc<<<sweep_grid, kTB, 0, st>>>(a);
    k_adj_micro_desc<<<sweep_grid, kTB, 0, st>>>(a);
    k_adj_wprime<<<a.N, kTB, 0, st>>>(a);
    k_adj_macro<<<1, kTB, 0, st>>>(a);
    k_adj_face<<<a.nf, kTB, 0, st>>>(a);
    k_adj_gather<<<nblk(2 * NNv, 256), 256, 0, st>>>(a);
    k_adj_cell<<<a.N, kTB, 0, st>>>(a);
    k_adj_res<<<1, kTB, 0, st>>>(a, it);
    return (int)cudaGetLastError();
}

}  // namespace idg
