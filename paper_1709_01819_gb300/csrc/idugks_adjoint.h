// idugks_adjoint.h -- data shared by the host side and the kernels of the
// discrete adjoint of the steady IDUGKS solve.  Not part of the C ABI.
//
// The adjoint runs in float64 on its own workspace.  It linearises the
// iteration at the state held by the forward context (absolute G, H and W),
// then iterates the transposed fixed-point map
//     lambda <- dJ/du + M^T lambda,   M = d(iteration)/du at the steady state,
// whose fixed point gives dJ/dp = dJ/dp|_u + lambda^T d(iteration)/dp.
#pragma once

#include "idugks_internal.h"

namespace idg {

constexpr int kCP = 16;  // per-cell linearisation record
constexpr int kFP = 24;  // per-face linearisation record
constexpr int kFPar = 4; // per-face parameter partials: u_w, v_w, RT_w, Kn*d/dKn

// per-cell record: rho U V RT tau qtx qty qx qy c1 c2 cq e1 sxx sxy syy
enum { CP_RHO, CP_U, CP_V, CP_RT, CP_TAU, CP_QTX, CP_QTY, CP_QX, CP_QY, CP_C1, CP_C2, CP_CQ, CP_E1,
       CP_SXX, CP_SXY, CP_SYY };
// per-face record
enum { FP_RHO, FP_U, FP_V, FP_RT, FP_TAU, FP_QBX, FP_QBY, FP_QX, FP_QY, FP_A, FP_B, FP_RW, FP_IN,
       FP_OUT, FP_E1, FP_SXX, FP_SXY, FP_SYY, FP_PHI0, FP_PHI1, FP_PHI2, FP_PHI3, FP_ON, FP_LAM };

struct AParams {
    // sizes and model
    int N, Nv, nf, ni, nj, K, shakhov, limiter;
    int lim_frozen;    // 1: the limiter factor is held at its linearisation value (no derivative)
    double venkat_k3;  // cube of the limiter's smoothing constant (0: Eq. 16-17)
    double dt, h, mu_ref, RT_ref, omega, Pr, gam, lusgs_omega, kappa;
    // geometry of the forward context (device, float64 / int)
    const double *area, *dtimp, *fgeo, *ux, *uy, *w;
    const int *cface, *cnb, *csign, *fL, *fR, *fbc, *fside;
    const double *W;   // [N][4] conservative state
    // boundary data (by side): density (1 for walls), velocity, RT
    double b_rho[4], b_u[4], b_v[4], b_RT[4];
    int b_kind[4];
    // objective: x- (axis 0) or y- (axis 1) force on the walls of obj_mask
    int obj_axis, obj_mask;
    // right-hand side of this adjoint solve: 0 the objective J, 1 the total
    // mass sum_c Omega_c W_c[0] (closed domains, see the host)
    int seed;
    // own float64 tables
    double *lsw;       // [N][8] least-squares weight vector per slot (0 if excluded)
    double *crv;       // [N][8] face midpoint minus centroid per slot
    double *G, *H;     // [N][Nv] state
    double *cpar;      // [N][kCP]
    double *fbG, *fbH; // [N][Nv] fb+
    double *sig;       // [2][N][Nv][2] gradients of fb+ (G then H)
    double *lim;       // [2][N][Nv][3] limiter phi, A = theta'/d, B = -x theta'/d
    signed char *lsl;  // [2][N][Nv][2] limiter: binding face slot, extreme-neighbour slot (-1: self)
    double *fpar;      // [nf][kFP]
    double *fbarG, *fbarH;  // [nf][Nv]
    double *DW;        // [N] macroscopic LU-SGS diagonal
    // adjoint iteration
    double *lamG, *lamH, *lamW;  // [N][Nv], [N][Nv], [N][4]
    double *bbG, *bbH;           // [N][Nv] P_f^-T lambda_f
    double *bwp;                 // [N][4]  bar W' (+ lambda_W)
    double *ba;                  // [N][4]  P_W^-T bar W'
    double *bqc;                 // [N][2]  bar q of the cell from the collision term
    double *bfG, *bfH;           // [nf][Nv] bar of the face reconstruction
    double *crec;                // [2][N][Nv][4] bself, bsx, bsy, bext
    double *bfb;                 // [2][N][Nv] bar fb+
    double *fpp;                 // [nf][kFPar]
    double *cpp;                 // [N][2]  Kn partials of the cell (collision, cell prep)
    double *rpart;               // [N] squared increment of lambda_f per cell
    double *res;                 // [kMaxHist] ||increment of lambda_f|| per adjoint iteration
    double *dlamW;               // [N][4] increment of lambda_W of the last iteration
};

// Workspace of the linearisation and of nrhs (1 or 2) adjoint solves that
// share it; out[r] describes solve r.
size_t adjoint_layout(const AParams &shape, int nrhs, char *base, AParams *out);
int launch_adjoint_setup(const AParams &a, void *stream);  // linearisation
int launch_adjoint_zero(const AParams &a, void *stream);   // lambda = 0 of one solve
int launch_adjoint_iteration(const AParams &a, int it, void *stream);
// float64 vectors of the Krylov solve: per-block partials of x.y (vec_dot_blocks()
// of them, summed on the host in order) and y = a x + b y
int launch_vec_dot(const double *x, const double *y, size_t n, double *dpart, void *stream);
int launch_vec_axpby(double a, const double *x, double b, double *y, size_t n, void *stream);
int vec_dot_blocks();

}  // namespace idg
