// Central-difference check of the local chain rules in adjoint_math.h, run on
// the CPU by tests/test_adjoint_math.py.  Prints "name max_relative_error".
#include "adjoint_math.h"

#include <cmath>
#include <algorithm>
#include <cstdio>
#include <random>

using namespace idg::adj;

static std::mt19937_64 rng(1709);
static double U(double a, double b) { return std::uniform_real_distribution<double>(a, b)(rng); }

// relative error, with derivatives below 1e-3 compared in absolute terms
static double rel(double a, double b) { return std::fabs(a - b) / (std::max(std::fabs(a), std::fabs(b)) + 1e-3); }

int main()
{
    const double eps = 1e-6;
    double worst;
    // primitives
    worst = 0;
    for (int t = 0; t < 200; ++t) {
        double W[4] = {U(0.5, 2), U(-0.5, 0.5), U(-0.5, 0.5), U(1, 3)};
        int K = 1 + t % 3;
        double b[4] = {U(-1, 1), U(-1, 1), U(-1, 1), U(-1, 1)}, bW[4] = {0, 0, 0, 0};
        prim_vjp(W, K, b[0], b[1], b[2], b[3], bW);
        for (int j = 0; j < 4; ++j) {
            double Wp[4], Wm[4];
            for (int q = 0; q < 4; ++q) Wp[q] = Wm[q] = W[q];
            Wp[j] += eps; Wm[j] -= eps;
            Prim p = prim_of(Wp, K), m = prim_of(Wm, K);
            double fd = (b[0] * (p.rho - m.rho) + b[1] * (p.U - m.U) + b[2] * (p.V - m.V) + b[3] * (p.RT - m.RT)) / (2 * eps);
            worst = std::max(worst, rel(fd, bW[j]));
        }
    }
    printf("prim_vjp %.3e\n", worst);
    // relaxation time
    worst = 0;
    for (int t = 0; t < 200; ++t) {
        double rho = U(0.5, 2), RT = U(0.2, 1), om = U(0.5, 1), mu = U(0.01, 1), RTr = 0.5, bt = U(-1, 1);
        double tau = tau_of(rho, RT, mu, RTr, om), br = 0, bR = 0, bk = 0;
        tau_vjp(tau, rho, RT, om, bt, br, bR, bk);
        double fr = bt * (tau_of(rho + eps, RT, mu, RTr, om) - tau_of(rho - eps, RT, mu, RTr, om)) / (2 * eps);
        double fR = bt * (tau_of(rho, RT + eps, mu, RTr, om) - tau_of(rho, RT - eps, mu, RTr, om)) / (2 * eps);
        // tau is linear in mu_ref, i.e. in Kn: Kn dtau/dKn = tau
        double fk = bt * mu * (tau_of(rho, RT, mu + eps, RTr, om) - tau_of(rho, RT, mu - eps, RTr, om)) / (2 * eps);
        worst = std::max({worst, rel(fr, br), rel(fR, bR), rel(fk, bk)});
    }
    printf("tau_vjp %.3e\n", worst);
    // Shakhov / BGK equilibrium
    for (int shak = 0; shak < 2; ++shak) {
        worst = 0;
        for (int t = 0; t < 400; ++t) {
            Eq e;
            e.rho = U(0.5, 2); e.U = U(-0.5, 0.5); e.V = U(-0.5, 0.5); e.RT = U(0.2, 1);
            e.qx = U(-0.1, 0.1); e.qy = U(-0.1, 0.1); e.K = 1 + t % 3;
            e.kappa = shak ? (1.0 - 2.0 / 3.0) / (e.K + 4) : 0.0;
            double ux = U(-3, 3), uy = U(-3, 3), bG = U(-1, 1), bH = U(-1, 1), b[6] = {0, 0, 0, 0, 0, 0};
            eq_vjp(e, ux, uy, bG, bH, b);
            for (int j = 0; j < 6; ++j) {
                Eq p = e, m = e;
                double *pp[6] = {&p.rho, &p.U, &p.V, &p.RT, &p.qx, &p.qy};
                double *mm[6] = {&m.rho, &m.U, &m.V, &m.RT, &m.qx, &m.qy};
                *pp[j] += eps; *mm[j] -= eps;
                double Gp, Hp, Gm, Hm;
                eq_eval(p, ux, uy, Gp, Hp);
                eq_eval(m, ux, uy, Gm, Hm);
                double fd = (bG * (Gp - Gm) + bH * (Hp - Hm)) / (2 * eps);
                if (std::fabs(fd) + std::fabs(b[j]) > 1e-10) worst = std::max(worst, rel(fd, b[j]));
            }
        }
        printf(shak ? "eq_vjp_shakhov %.3e\n" : "eq_vjp_bgk %.3e\n", worst);
    }
    // boundary Maxwellian
    worst = 0;
    for (int t = 0; t < 200; ++t) {
        double rho = U(0.5, 2), u = U(-0.5, 0.5), v = U(-0.5, 0.5), RT = U(0.2, 1), ux = U(-3, 3), uy = U(-3, 3);
        int K = 1 + t % 2;
        double bG = U(-1, 1), bH = U(-1, 1), bu = 0, bv = 0, bR = 0;
        bnd_vjp(rho, u, v, RT, K, ux, uy, bG, bH, bu, bv, bR);
        double Gp, Hp, Gm, Hm, fd[3];
        bnd_eval(rho, u + eps, v, RT, K, ux, uy, Gp, Hp); bnd_eval(rho, u - eps, v, RT, K, ux, uy, Gm, Hm);
        fd[0] = (bG * (Gp - Gm) + bH * (Hp - Hm)) / (2 * eps);
        bnd_eval(rho, u, v + eps, RT, K, ux, uy, Gp, Hp); bnd_eval(rho, u, v - eps, RT, K, ux, uy, Gm, Hm);
        fd[1] = (bG * (Gp - Gm) + bH * (Hp - Hm)) / (2 * eps);
        bnd_eval(rho, u, v, RT + eps, K, ux, uy, Gp, Hp); bnd_eval(rho, u, v, RT - eps, K, ux, uy, Gm, Hm);
        fd[2] = (bG * (Gp - Gm) + bH * (Hp - Hm)) / (2 * eps);
        worst = std::max({worst, rel(fd[0], bu), rel(fd[1], bv), rel(fd[2], bR)});
    }
    printf("bnd_vjp %.3e\n", worst);
    // heat flux about (U, V)
    worst = 0;
    for (int t = 0; t < 50; ++t) {
        const int n = 40;
        double x[n], y[n], w[n], G[n], H[n];
        for (int k = 0; k < n; ++k) { x[k] = U(-3, 3); y[k] = U(-3, 3); w[k] = U(0, 1); G[k] = U(0, 1); H[k] = U(0, 1); }
        double Uc = U(-0.5, 0.5), Vc = U(-0.5, 0.5), bqx = U(-1, 1), bqy = U(-1, 1);
        auto q = [&](double u0, double v0, double &qx, double &qy) {
            qx = qy = 0;
            for (int k = 0; k < n; ++k) {
                double cx = x[k] - u0, cy = y[k] - v0, e = (cx * cx + cy * cy) * G[k] + H[k];
                qx += 0.5 * w[k] * cx * e;
                qy += 0.5 * w[k] * cy * e;
            }
        };
        double e1 = 0, sxx = 0, sxy = 0, syy = 0;
        for (int k = 0; k < n; ++k) {
            double cx = x[k] - Uc, cy = y[k] - Vc;
            e1 += w[k] * ((cx * cx + cy * cy) * G[k] + H[k]);
            sxx += w[k] * cx * cx * G[k]; sxy += w[k] * cx * cy * G[k]; syy += w[k] * cy * cy * G[k];
        }
        double bU = 0, bV = 0, a, b, c, d;
        heat_uv_vjp(e1, sxx, sxy, syy, bqx, bqy, bU, bV);
        q(Uc + eps, Vc, a, b); q(Uc - eps, Vc, c, d);
        double fU = (bqx * (a - c) + bqy * (b - d)) / (2 * eps);
        q(Uc, Vc + eps, a, b); q(Uc, Vc - eps, c, d);
        double fV = (bqx * (a - c) + bqy * (b - d)) / (2 * eps);
        worst = std::max({worst, rel(fU, bU), rel(fV, bV)});
    }
    printf("heat_uv_vjp %.3e\n", worst);
    // Venkatakrishnan function
    worst = 0;
    for (int t = 0; t < 200; ++t) {
        double x = U(0, 5);
        worst = std::max(worst, rel((venkat(x + eps) - venkat(x - eps)) / (2 * eps), venkat_d(x)));
    }
    printf("venkat_d %.3e\n", worst);
    // the smoothed factor's partial derivatives
    worst = 0;
    for (int t = 0; t < 200; ++t) {
        double P = U(-2, 2), D = U(0.05, 2) * (t & 1 ? 1 : -1), e2 = U(1e-4, 1), dP, dD;
        venkat_eps_d(P, D, e2, dP, dD);
        worst = std::max({worst, rel((venkat_eps(P + eps, D, e2) - venkat_eps(P - eps, D, e2)) / (2 * eps), dP),
                          rel((venkat_eps(P, D + eps, e2) - venkat_eps(P, D - eps, e2)) / (2 * eps), dD)});
    }
    printf("venkat_eps_d %.3e\n", worst);
    // Euler flux Jacobian, transposed
    worst = 0;
    for (int t = 0; t < 200; ++t) {
        double W[4] = {U(0.5, 2), U(-0.5, 0.5), U(-0.5, 0.5), U(1, 3)}, th = U(0, 6.3);
        double nx = std::cos(th), ny = std::sin(th), gam = 5.0 / 3.0, y[4], out[4];
        for (int q = 0; q < 4; ++q) y[q] = U(-1, 1);
        euler_jacT(W, gam, nx, ny, y, out);
        for (int j = 0; j < 4; ++j) {
            double Wp[4], Wm[4], Fp[4], Fm[4];
            for (int q = 0; q < 4; ++q) Wp[q] = Wm[q] = W[q];
            Wp[j] += eps; Wm[j] -= eps;
            euler_flux(Wp, gam, nx, ny, Fp);
            euler_flux(Wm, gam, nx, ny, Fm);
            double fd = 0;
            for (int q = 0; q < 4; ++q) fd += y[q] * (Fp[q] - Fm[q]) / (2 * eps);
            worst = std::max(worst, rel(fd, out[j]));
        }
    }
    printf("euler_jacT %.3e\n", worst);
    return 0;
}
