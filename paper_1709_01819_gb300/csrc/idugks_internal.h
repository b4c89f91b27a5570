// idugks_internal.h -- data shared by the host side (idugks_host.cpp) and the
// kernels (idugks_kernels.cu) of libidugks.  Not part of the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>

namespace idg {

constexpr int kMaxVel = 16384;
constexpr int kMaxHist = 1 << 16;  // residual-history ring (iterations)
constexpr int kCellP = 16;         // per-cell / per-face coefficient records
constexpr int kRaw = 11;           // raw velocity moments kept per cell / face
constexpr int kNoAllocMaxCells = 16384;  // cell limit of idg_get_moments_noalloc

// Everything one kernel launch needs, passed by value.  Device pointers point
// into the caller's workspace.  "T" below is the storage precision (float for
// IDG_MIXED, double for IDG_FP64); "acc" entries are 8 bytes: a float-float
// pair (hi, lo) in mixed precision, a double in FP64.  Distributions are kept
// relative to one reference Maxwellian M_ref (f = M_ref + dev).
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
    const void *crT;       // [N][8] T: face midpoint minus centroid, per slot
    const void *clsgT;     // [N][8] T: least-squares weight vector per slot
    const void *cslotT;    // [N][4][2] T: sign*nx*S, sign*ny*S per slot (micro sweeps)
    const int *scode;      // [2][N][4] forward, backward: role of each slot's neighbour in that micro sweep
    // faces
    const int *fL, *fR;    // [nf]
    const double *fgeo;    // [nf][7] nx, ny, S, rLx, rLy, rRx, rRy
    const void *fgeoT;     // [nf][8] T copy of fgeo
    const int *fbc;        // [nf] -1 interior, else boundary kind
    const int *fside;      // [nf] boundary side or -1
    const double *bconst;  // [nf][2] boundary faces: sum_out w (xi.n_out) G_ref, sum_in w |xi.n_out| G_bnd
    // velocity tables
    const double *ux, *uy, *w;   // [Nv]
    const double *gref;          // [Nv] reduced reference Maxwellian G
    const float *uxf, *uyf, *wf, *greff;  // float copies
    const void *bdevG, *bdevH;   // [4][Nv] T: boundary Maxwellian minus M_ref (wall: unit density)
    // gas and numerics
    double dt, h, mu_ref, RT_ref, omega, Pr, gam, lusgs_omega;
    double venkat_k3;  // cube of the limiter's smoothing constant: eps^2 = venkat_k3 * area^(3/2)
    // reference Maxwellian parameters and its discrete moments
    double rho_r, U_r, V_r, RT_r;
    double mref_raw[kRaw];     // raw moments: G: 1,x,y,xx,xy,yy,x|xi|^2,y|xi|^2; H: 1,x,y
    double mref_flux[4][2];    // sum w psi xi_a M_ref, psi = 1, xi_x, xi_y, energy
    // state and work (T2 = {G, H} deviation pairs of the storage type)
    void *f;        // [N][Nv] T2 state f~ - M_ref
    void *fbp;      // [N][Nv] T2 fb+ - M_ref
    void *grad;     // [N][Nv][4] T limited gradients phi sigma of G and H (limiter on; else null)
    void *F;        // [nf][Nv] T2 flux of (f_face - M_ref)
    void *dst;      // [N][Nv] T2 Delta* then Delta
    double *W;      // [N][4]
    void *cellraw;  // [N][kRaw] acc raw moments of f~ - M_ref
    void *cellA;    // [N][16] T: equilibrium at W^n (14), c1, c2 of fb+
    double *cellq;  // [N][2]  heat flux of f at cells (from f~^n)
    double *cellp;  // [N][16] post-predictor cell coefficients (float64)
    void *cellpT;   // [N][16] T copy of cellp for the sweeps
    void *faceraw;  // [nf][12] acc raw moments of fb - M_ref, wall outgoing sum
    double *facerw; // [nf] wall density rho_w (1 elsewhere)
    void *faceA;    // [nf][16] T: face equilibrium (14), a, b of Eq. (18)
    void *phiraw;   // [nf][4] acc moments of the deviation flux
    double *phi;    // [nf][4]
    double *rw;     // [N][4]
    // macroscopic LU-SGS work (T = storage precision of the sweep)
    void *mrec;     // [N][24] T: R, 1/D, own base state, per slot (S/2) n_out, (omega/2) Lambda
    void *mdW;      // [N][4] T increments (Delta W* then Delta W)
    void *mdW2;     // [N][4] T second increment buffer of the point relaxation (else null)
    double *mpart;  // [ceil(N/256)] block partial sums of ||R/Omega||^2
    double *res;    // [kMaxHist] absolute residual per iteration
    int *iter;      // [1] device iteration counter
    int *status;    // [1] device status word
    // launch shape of the wavefront kernels: velocities per CTA and cell
    // slots of the micro sweeps, prefetch depths (hyperplanes; 4 or 8)
    int sweep_tv, sweep_pc, sweep_stages, macro_stages;
    int sweep_vpt;  // consecutive velocities per thread in the micro sweeps (1, 2, 4)
    int macro_kind; // macroscopic LU-SGS on a structured block: 0 hyperplane slots (k_macro_sweep),
                    // 1 one thread per line of cells (k_macro_lines)
    int relax_sweeps;  // macroscopic predictor: 0 LU-SGS, n >= 1 n point-relaxation sweeps
    // unstructured meshes: the sweeps' schedule (null on a structured block,
    // whose sweeps walk the i+j hyperplanes): sched [2][N] cells in processing
    // order for the forward then the backward sweep, sptr the step offsets
    // into each ([nsteps_f + 1] then [nsteps_b + 1]); the cells of one step
    // depend on none of each other
    const int *sched, *sptr;
    int nsteps_f, nsteps_b;
    // linearised diffuse wall of the micro sweeps (Eq. 33-35), implicit_wall
    // = 1: per face, wallS the inner cell's outgoing sum sum_out w (xi.n_out)
    // G~ of the last iteration, walldrg the ghost density increment drho_g
    // (wall faces only; else null); wallok 0 after a restart (no last
    // increment), 1 once an iteration has stored wallS
    int implicit_wall;
    double *wallS, *walldrg;
    int *wallok;
};

// kernels of one iteration, in launch order
enum KType {
    KT_CELL_MOM, KT_CELL_PAR, KT_FBP, KT_FACE_MOM, KT_FACE_PAR, KT_FACE_FLUX, KT_FACE_PHI,
    KT_MACRO_PRE, KT_MACRO_SWEEP, KT_MACRO_POST, KT_MICRO_RES, KT_SWEEP, KT_COUNT
};

// How one iteration is launched over one or many instances: the instances'
// parameters in device memory, per-kernel prefix sums of blocks per instance
// (null for a single instance), activity flags (null: all active), and the
// block shapes common to all instances.
struct Plan {
    const KParams *dparams;
    const int *doff;     // [KT_COUNT][ninst + 1]
    const int *dactive;  // [ninst]
    int ninst;
    int nblocks[KT_COUNT];
    int macro_threads, sweep_threads;
    size_t macro_smem, fwd_smem, bwd_smem;
    int macro_stages, sweep_stages, limiter_any, sweep_vpt;
    int macro_kind;      // KParams::macro_kind of every instance
    int any_seam;        // 1: an instance has a periodic direction (k_macro_lines' seam terms)
    int explicit_dugks;  // 1: launch_iteration runs one explicit DUGKS step (Eq. 21)
    int relax_sweeps;    // macroscopic predictor of every instance (KParams::relax_sweeps)
    int sched;           // 1: the instances are unstructured (scheduled sweeps)
    size_t sched_smem;   // shared memory of the scheduled macroscopic sweep (0: increments in global memory)
};

// kernel launchers (idugks_kernels.cu)
int configure_kernels(bool fp64);
void blocks_per_instance(const KParams &p, int out[KT_COUNT]);
int plan_shapes(const KParams *hp, int n, bool fp64, Plan &plan);
constexpr int kProfiled = 6;  // timed groups in launch_iteration(events)
int launch_iteration(const Plan &plan, bool fp64, void *stream, void **events = nullptr);
int launch_cell_moments(const KParams &p, bool fp64, double *out6_dev, void *stream);
// explicit DUGKS: W and the raw moments of the current f~ before the first step
int launch_explicit_prologue(const Plan &plan, bool fp64, void *stream);
// idg_get_moments_noalloc: raw moments in a static device array (no workspace)
int launch_cell_moments_noalloc(const KParams &p, bool fp64, int device, double *out6_dev, void *stream);
// absolute float64 G, H of [N][nvu] (the first nvu stored velocities of each
// cell) to / from the storage; to_dev sets the ghost velocities beyond nvu to M_ref
// float64 (G, H) [N][nvu] <-> the storage; deviation: the arrays hold f~ - M_ref
int launch_to_dev(const KParams &p, bool fp64, const double *G, const double *H, int nvu, void *stream,
                  bool deviation = false);
int launch_from_dev(const KParams &p, bool fp64, double *G, double *H, int nvu, void *stream,
                    bool deviation = false);

}  // namespace idg
