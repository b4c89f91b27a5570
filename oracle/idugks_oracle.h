/*
 * idugks_oracle.h -- plain FP64 CPU oracle of explicit DUGKS and of the
 * implicit DUGKS (IDUGKS) iteration of Pan, Zhong & Zhuo, "An Implicit
 * Discrete Unified Gas-Kinetic Scheme for Simulations of Steady Flow in All
 * Flow Regimes" (arXiv 1709.01819).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library (include/idugks.h).
 *
 * Conventions (the paper fixes none): reference density 1, reference length 1,
 * velocity unit sqrt(2 R T_ref) = 1, so R T_ref = 1/2 by default.  Temperatures
 * passed in are in units of T_ref (R T = T * RT_ref).
 */
#ifndef IDUGKS_ORACLE_H
#define IDUGKS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_PERIODIC = 0, ORC_BC_WALL = 1, ORC_BC_FARFIELD = 2 };
enum { ORC_NC_TRAP = 0, ORC_NC_SIMPSON = 1, ORC_GAUSS_HERMITE = 2 };
/* sides of the structured block */
enum { ORC_IMIN = 0, ORC_IMAX = 1, ORC_JMIN = 2, ORC_JMAX = 3 };
/* flags */
#define ORC_FLAG_FEQ_MASS_NORMALIZE 1

typedef struct {
    int ni, nj;                 /* cells in i and j                                   */
    const double *nodes_x;      /* (ni+1)*(nj+1) node coordinates, index j*(ni+1)+i  */
    const double *nodes_y;
    int bc_kind[4];             /* per side: ORC_BC_*; PERIODIC on both ends of a dir */
    double bc_rho[4], bc_u[4], bc_v[4], bc_T[4]; /* wall: u,v,T; farfield: all four */
    int vrule, nvx, nvy;        /* velocity quadrature rule and points per axis       */
    double vxmin, vxmax, vymin, vymax; /* NC ranges; GH uses the scale vxmax (>0)     */
    int K;                      /* internal degrees of freedom                        */
    double Pr, omega, Kn, RT_ref;
    int shakhov;                /* 0: BGK, 1: Shakhov                                  */
    double cfl_imp, cfl_phys;
    int limiter;                /* 0: phi = 1; 1: Venkatakrishnan, Eq. (16)-(17)      */
    int flags;
    double lusgs_omega;         /* macro LU-SGS relaxation; 2 is the Eq. (30) form    */
    int relax_sweeps;           /* 0: LU-SGS predictor; n >= 1: point relaxation of   */
                                /* the same equations, n Jacobi sweeps from dW = 0     */
    /* unstructured mesh (used when n_ucells > 0; ni, nj are then ignored):      */
    int n_ucells, n_unodes;     /* cells (triangles or quadrilaterals), nodes         */
    const int *ucell_nodes;     /* [n_ucells][4] node indices counter-clockwise, -1   */
                                /* as the 4th of a triangle; nodes_x/y hold n_unodes  */
    const int *uedge_side;      /* [n_ucells][4] boundary group (0..3, the bc_* slot)  */
                                /* of edge m (node m -> m+1) where it has no neighbour */
    int implicit_wall;          /* 1: the ghost cell of a wall face takes the          */
                                /* linearised diffuse-reflection increment of Eq.     */
                                /* (34)-(35) from the inner cell's last increment;    */
                                /* 0: ghost increments are zero (end of Section 2.3)  */
    double venkat_k;            /* 0: the limiter of Eq. (16)-(17) as printed; K > 0: */
                                /* Venkatakrishnan's smoothing constant, eps^2 =      */
                                /* (K h)^3 with h = sqrt(cell area), in the ratio      */
} orc_problem;

typedef struct orc_state orc_state;

orc_state *orc_create(const orc_problem *p);
void orc_destroy(orc_state *s);
int orc_num_cells(const orc_state *s);
int orc_num_vel(const orc_state *s);
int orc_num_faces(const orc_state *s);
double orc_dt(const orc_state *s);

void orc_init_uniform(orc_state *s, double rho, double u, double v, double T);
void orc_set_state(orc_state *s, const double *G, const double *H, const double *W);
void orc_get_state(const orc_state *s, double *G, double *H, double *W);

/* n IDUGKS iterations; res_abs[n] = ||R_W / Omega||_2 before each update. */
void orc_iterate(orc_state *s, int n, double *res_abs);
/* n explicit DUGKS steps, Eq. (21). */
void orc_explicit_step(orc_state *s, int n);
/* R_W of the current state and the predictor's dW, without advancing it. */
void orc_debug_predictor(orc_state *s, double *rw, double *dW);
/* right-hand side of the micro sweeps (Eq. 23 with the Omega/dt factor, plus
 * the wall ghost term when implicit_wall is set) of the current state, G and
 * H [N][Nv], without advancing it. */
void orc_debug_micro_residual(orc_state *s, double *RG, double *RH);

/* per cell: rho, u, v, T/T_ref, qx, qy (q from the stored state) */
void orc_get_moments(orc_state *s, double *out6);
/* last computed face flux moments Phi[face][4] and cell residual R_W[cell][4] */
void orc_get_face_phi(const orc_state *s, double *phi4);
void orc_get_rw(const orc_state *s, double *rw4);
/* face list: L, R (-1 for a ghost), bc kind, side */
void orc_get_faces(const orc_state *s, int *L, int *R, int *bc, int *side,
                   double *nx, double *ny, double *S);
void orc_get_geometry(const orc_state *s, double *cx, double *cy, double *area);

/* building blocks exposed for the pin tests */
int orc_quadrature(int rule, int n, double a, double b, double *x, double *w);
void orc_velocity_grid(const orc_state *s, double *ux, double *uy, double *w);
void orc_equilibrium(const orc_state *s, double rho, double u, double v, double RT,
                     double qx, double qy, double *G, double *H);
/* least-squares gradient of a scalar cell field, Eq. (14)-(15) */
void orc_ls_gradient(const orc_state *s, const double *phi, double *grad2);
/* Venkatakrishnan limiter value (Eq. 16-17) of a cell scalar field [N]. */
void orc_limiter(const orc_state *s, const double *phi, double *lim);
double orc_venkat_theta(double x);
/* the micro LU-SGS sweeps (Eq. 26) of the current state applied to the
 * right-hand side (RG, RH) [N][Nv]: increments (dG, dH) and the diagonal D
 * [N][Nv] of the state's iteration; the state is not advanced */
void orc_debug_micro_sweeps(orc_state *s, const double *RG, const double *RH, double *dG, double *dH,
                            double *D);
/* runs the cell-prep step (Eq. 10, 12) on the stored state and copies out
 * fb+ [N][Nv] (G and H), the cell heat flux q [N][2] and tau [N] */
void orc_debug_cell_prep(orc_state *s, double *fbG, double *fbH, double *q, double *tau);

#ifdef __cplusplus
}
#endif
#endif
