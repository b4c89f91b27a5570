// idugks_internal.h -- data shared by the host side (idugks_host.cpp) and the
// kernels (idugks_kernels.cu) of libidugks.  Not part of the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>

namespace idg {

constexpr int kMaxVel = 16384;
constexpr int kMaxHist = 1 << 16;  // residual-history ring (iterations)

// Everything one kernel launch needs, passed by value.  Device pointers point
// into the caller's workspace.  "dev" quantities are relative to the global
// reference Maxwellian M_ref (f = M_ref + dev), see storage in DESIGN notes of
// the kernels file.
struct KParams {
    // sizes
    int N, Nv, nf, ni, nj, nvx;
    int K, shakhov, limiter;
    int per_i, per_j;
    // cells
    const double *area;    // [N]
    const double *dtimp;   // [N]
    const int *cface;      // [N][4] faces in slots west, east, south, north
    const int *cnb;        // [N][4] neighbour across the slot (-1 ghost)
    const int *csign;      // [N][4] +1 if the cell is the L side of that face
    const double *cr;      // [N][4][2] face midpoint minus centroid, per slot
    const double *clsg;    // [N][4][2] least-squares weight vector per slot
    // faces
    const int *fL, *fR;    // [nf]
    const double *fgeo;    // [nf][7] nx, ny, S, rLx, rLy, rRx, rRy
    const int *fbc;        // [nf] -1 interior, else boundary kind
    const int *fside;      // [nf] boundary side or -1
    // velocity tables
    const double *ux, *uy, *w;   // [Nv]
    const double *gref;          // [Nv] reduced reference Maxwellian G
    const double *lngref;        // [Nv] log of it
    const float *uxf, *uyf, *wf, *greff, *lngreff;  // float copies
    const double *bndG, *bndH;   // [4][Nv] boundary Maxwellians (wall: unit density)
    // gas and numerics
    double dt, h, mu_ref, RT_ref, omega, Pr, gam, lusgs_omega;
    // reference Maxwellian parameters and its discrete moments
    double rho_r, U_r, V_r, RT_r;
    double mref_raw[11];       // raw moments: G: 1,x,y,xx,xy,yy,x|xi|^2,y|xi|^2; H: 1,x,y
    double mref_flux[4][2];    // sum w psi xi_a M_ref, psi = 1, xi_x, xi_y, energy
    // state and work (T2 = {G, H} deviation pairs of the storage type)
    void *f;        // [N][Nv] T2 state f~ - M_ref
    void *fbp;      // [N][Nv] T2 fb+ - M_ref
    void *F;        // [nf][Nv] T2 flux of (f_face - M_ref)
    void *dst;      // [N][Nv] T2 Delta* then Delta
    double *W;      // [N][4]
    double *cellq;  // [N][2]  heat flux of f at cells (from f~^n)
    double *cellp;  // [N][16] post-predictor cell coefficients
    double *phi;    // [nf][4]
    double *rw;     // [N][4]
    double *dW;     // [N][4]
    double *lam;    // [nf]
    double *Dm;     // [N]
    // macroscopic LU-SGS work (T = storage precision of the sweep)
    void *mbase;    // [N][8] T: rho, m_x, m_y, E, u, v, p, E+p of W^n
    void *moff;     // [N][4][4] T: (S/2) n_out, (omega/2) Lambda, 0 per slot
    void *mD;       // [N] T diagonal
    void *mR;       // [N][4] T residual
    void *mdW;      // [N][4] T increments (Delta W* then Delta W)
    double *mpart;  // [ceil(N/256)] block partial sums of ||R/Omega||^2
    void *cellpT;   // [N][16] T copy of cellp for the sweeps
    double *res;    // [kMaxHist] absolute residual per iteration
    int *iter;      // [1] device iteration counter
    int *status;    // [1] device status word
    // face lists: interior faces, boundary faces
    const int *ilist, *blist;
    int nilist, nblist;
    // launch shape of the sweeps
    int sweep_tv, sweep_pc;
};

// coefficients of the deviation equilibrium (see dev_equilibrium in kernels)
constexpr int kCellP = 16;

// kernel launchers (idugks_kernels.cu)
int configure_kernels(const KParams &p, bool fp64);
int launch_iteration(const KParams &p, bool fp64, void *stream, void **events = nullptr);
int launch_cell_moments(const KParams &p, bool fp64, double *out6_dev, void *stream);
int launch_to_dev(const KParams &p, bool fp64, const double *G, const double *H, void *stream);
int launch_from_dev(const KParams &p, bool fp64, double *G, double *H, void *stream);

}  // namespace idg
