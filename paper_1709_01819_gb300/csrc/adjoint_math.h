// adjoint_math.h -- local chain rules of the steady IDUGKS residual, written
// as host/device functions so that they can be checked against finite
// differences on the CPU.  Every function takes the forward inputs and the
// adjoint weights of its outputs and accumulates the adjoint weights of its
// inputs ("bar" quantities).  Double precision throughout.
//
// Forward definitions (reduced distributions G, H; K internal degrees of
// freedom; c = xi - U):
//   primitives, Eq. (4):   rho = W0, U = W1/W0, V = W2/W0,
//                          RT = (2 W3/W0 - U^2 - V^2)/(K+2)
//   relaxation time:       tau = mu_ref (RT/RT_ref)^omega / (rho RT)
//   reduced Maxwellian, Eq. (2), (5):  E = rho/(2 pi RT) exp(-c^2/(2 RT)),
//                          G^M = E, H^M = K RT E
//   Shakhov, Eq. (20):     P = (1-Pr)(c.q) / ((K+4) rho RT^2),
//                          G^S = E (1 + P (c^2/RT - 4)), H^S = K RT E (1 + P (c^2/RT - 2))
//   heat flux:             q = 1/2 sum_k w c (c^2 G + H)
//   Euler flux (macroscopic predictor, Eq. 28-31): F.n of the conservative W
//   Venkatakrishnan function, Eq. (17): theta(x) = (x^2 + 2x)/(x^2 + x + 2)
#pragma once

#include <cmath>

#if defined(__CUDACC__)
#define IDG_AD __host__ __device__ __forceinline__
#else
#define IDG_AD inline
#endif

namespace idg {
namespace adj {

struct Prim {
    double rho, U, V, RT;
};

IDG_AD Prim prim_of(const double *W, int K)
{
    Prim p;
    p.rho = W[0];
    p.U = W[1] / W[0];
    p.V = W[2] / W[0];
    p.RT = (2.0 * W[3] / W[0] - p.U * p.U - p.V * p.V) / (K + 2);
    return p;
}

// bW += (d prim / d W)^T (brho, bU, bV, bRT)
IDG_AD void prim_vjp(const double *W, int K, double brho, double bU, double bV, double bRT, double *bW)
{
    const double rho = W[0], U = W[1] / rho, V = W[2] / rho, k2 = 1.0 / (K + 2);
    bW[0] += brho - (U * bU + V * bV) / rho +
             bRT * k2 * (-2.0 * W[3] / (rho * rho) + 2.0 * (U * U + V * V) / rho);
    bW[1] += bU / rho - bRT * k2 * 2.0 * U / rho;
    bW[2] += bV / rho - bRT * k2 * 2.0 * V / rho;
    bW[3] += bRT * k2 * 2.0 / rho;
}

IDG_AD double tau_of(double rho, double RT, double mu_ref, double RT_ref, double omega)
{
    return mu_ref * pow(RT / RT_ref, omega) / (rho * RT);
}

// brho, bRT (and the Kn weight: tau is proportional to Kn) from btau
IDG_AD void tau_vjp(double tau, double rho, double RT, double omega, double btau, double &brho,
                    double &bRT, double &bKn_times_Kn)
{
    brho += -tau / rho * btau;
    bRT += (omega - 1.0) * tau / RT * btau;
    bKn_times_Kn += tau * btau;
}

// Shakhov (or BGK when kappa = 0) equilibrium at one discrete velocity
struct Eq {
    double rho, U, V, RT, qx, qy;
    double kappa;  // (1 - Pr)/(K + 4); 0 for BGK
    int K;
};

IDG_AD void eq_eval(const Eq &e, double ux, double uy, double &G, double &H)
{
    const double cx = ux - e.U, cy = uy - e.V, c2 = cx * cx + cy * cy;
    const double E = e.rho / (2.0 * M_PI * e.RT) * exp(-c2 / (2.0 * e.RT));
    const double P = e.kappa * (cx * e.qx + cy * e.qy) / (e.rho * e.RT * e.RT);
    G = E * (1.0 + P * (c2 / e.RT - 4.0));
    H = e.K * e.RT * E * (1.0 + P * (c2 / e.RT - 2.0));
}

// b[0..5] += (d(G,H)/d(rho, U, V, RT, qx, qy))^T (bG, bH) at one velocity
IDG_AD void eq_vjp(const Eq &e, double ux, double uy, double bG, double bH, double *b)
{
    const double RT = e.RT, rho = e.rho;
    const double cx = ux - e.U, cy = uy - e.V, c2 = cx * cx + cy * cy;
    const double E = rho / (2.0 * M_PI * RT) * exp(-c2 / (2.0 * RT));
    const double r2 = 1.0 / (rho * RT * RT);
    const double P = e.kappa * (cx * e.qx + cy * e.qy) * r2;
    const double sG = c2 / RT - 4.0, sH = c2 / RT - 2.0, kRT = e.K * RT;
    const double bE = bG * (1.0 + P * sG) + bH * kRT * (1.0 + P * sH);
    const double bP = (bG * sG + bH * kRT * sH) * E;
    const double bs = (bG + bH * kRT) * E * P;
    const double bRTd = bH * e.K * E * (1.0 + P * sH);
    b[0] += bE * E / rho - bP * P / rho;
    b[1] += bE * E * cx / RT - bP * e.kappa * e.qx * r2 - bs * 2.0 * cx / RT;
    b[2] += bE * E * cy / RT - bP * e.kappa * e.qy * r2 - bs * 2.0 * cy / RT;
    b[3] += bE * E * (c2 / (2.0 * RT * RT) - 1.0 / RT) - bP * 2.0 * P / RT - bs * c2 / (RT * RT) + bRTd;
    b[4] += bP * e.kappa * cx * r2;
    b[5] += bP * e.kappa * cy * r2;
}

// Maxwellian of a boundary (q = 0): (G, H) and their derivatives with
// respect to (u, v, RT) of the boundary, at one velocity
IDG_AD void bnd_eval(double rho, double u, double v, double RT, int K, double ux, double uy, double &G,
                     double &H)
{
    const double cx = ux - u, cy = uy - v, c2 = cx * cx + cy * cy;
    G = rho / (2.0 * M_PI * RT) * exp(-c2 / (2.0 * RT));
    H = K * RT * G;
}

IDG_AD void bnd_vjp(double rho, double u, double v, double RT, int K, double ux, double uy, double bG,
                    double bH, double &bu, double &bv, double &bRT)
{
    const double cx = ux - u, cy = uy - v, c2 = cx * cx + cy * cy;
    const double G = rho / (2.0 * M_PI * RT) * exp(-c2 / (2.0 * RT));
    const double bE = bG + bH * K * RT;
    bu += bE * G * cx / RT;
    bv += bE * G * cy / RT;
    bRT += bE * G * (c2 / (2.0 * RT * RT) - 1.0 / RT) + bH * K * G;
}

// The heat flux q = 1/2 sum w c (c^2 G + H) depends on U, V through c.  Given
// the sums e1 = sum w (c^2 G + H), sxx = sum w cx^2 G, sxy = sum w cx cy G,
// syy = sum w cy^2 G, this adds (dq/d(U,V))^T (bqx, bqy).
IDG_AD void heat_uv_vjp(double e1, double sxx, double sxy, double syy, double bqx, double bqy, double &bU,
                        double &bV)
{
    bU += -0.5 * e1 * bqx - sxx * bqx - sxy * bqy;
    bV += -0.5 * e1 * bqy - syy * bqy - sxy * bqx;
}

// Venkatakrishnan function and its derivative
IDG_AD double venkat(double x) { return (x * x + 2.0 * x) / (x * x + x + 2.0); }
IDG_AD double venkat_d(double x)
{
    const double d = x * x + x + 2.0;
    return (-x * x + 4.0 * x + 4.0) / (d * d);
}

// The limiter's factor at one face with the smoothing constant e2 = eps^2 >
// 0, phi = N / M with N = P^2 + e2 + 2 D P, M = P^2 + 2 D^2 + P D + e2 (P the
// increment to the neighbourhood's extremum, D the extrapolated one), and its
// partial derivatives in P and D
IDG_AD double venkat_eps(double P, double D, double e2)
{
    return (P * P + e2 + 2.0 * D * P) / (P * P + 2.0 * D * D + P * D + e2);
}
IDG_AD void venkat_eps_d(double P, double D, double e2, double &dP, double &dD)
{
    const double N = P * P + e2 + 2.0 * D * P, M = P * P + 2.0 * D * D + P * D + e2, iM2 = 1.0 / (M * M);
    dP = ((2.0 * P + 2.0 * D) * M - N * (2.0 * P + D)) * iM2;
    dD = (2.0 * P * M - N * (4.0 * D + P)) * iM2;
}

// Euler flux F(W).n and the transposed Jacobian product (dF.n/dW)^T y
IDG_AD void euler_flux(const double *W, double gam, double nx, double ny, double *F)
{
    const double rho = W[0], u = W[1] / rho, v = W[2] / rho;
    const double p = (gam - 1.0) * (W[3] - 0.5 * rho * (u * u + v * v));
    const double vn = u * nx + v * ny;
    F[0] = rho * vn;
    F[1] = W[1] * vn + p * nx;
    F[2] = W[2] * vn + p * ny;
    F[3] = (W[3] + p) * vn;
}

IDG_AD void euler_jacT(const double *W, double gam, double nx, double ny, const double *y, double *out)
{
    const double rho = W[0], u = W[1] / rho, v = W[2] / rho, g1 = gam - 1.0;
    const double q2 = 0.5 * (u * u + v * v);
    const double p = g1 * (W[3] - rho * q2);
    const double Hs = (W[3] + p) / rho, vn = u * nx + v * ny;
    // rows of A = dF/dW
    const double A[4][4] = {
        {0.0, nx, ny, 0.0},
        {-u * vn + g1 * q2 * nx, vn + u * nx - g1 * u * nx, u * ny - g1 * v * nx, g1 * nx},
        {-v * vn + g1 * q2 * ny, v * nx - g1 * u * ny, vn + v * ny - g1 * v * ny, g1 * ny},
        {vn * (g1 * q2 - Hs), Hs * nx - g1 * u * vn, Hs * ny - g1 * v * vn, gam * vn},
    };
    for (int j = 0; j < 4; ++j) out[j] = A[0][j] * y[0] + A[1][j] * y[1] + A[2][j] * y[2] + A[3][j] * y[3];
}

}  // namespace adj
}  // namespace idg
