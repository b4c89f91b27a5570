// idugks_kernels.cu -- sm_103a kernels of one IDUGKS iteration
// (arXiv 1709.01819, Section 2).
//
// Storage.  The distribution f~ (Eq. 10) of every (cell, discrete velocity) is
// kept as a pair {G, H} (Eq. 5) relative to one global reference Maxwellian
// M_ref: dev = f~ - M_ref.  All per-velocity operations of the scheme are
// linear in f~ except the equilibria, which are evaluated directly in deviation
// form (dev_equilibrium), so float32 storage rounds relative to the deviation
// and not to f.  The flux of M_ref through the closed surface of a cell
// vanishes (sum_f n_f S_f = 0), so stored face fluxes are fluxes of
// (f_face - M_ref); the macroscopic face moments add M_ref's float64 moments
// back.  Layouts are velocity-contiguous: [cell][velocity]{G,H}.
//
// Precision.  GB300 runs float64 at 1/64 of the float32 rate (a warp-wide
// float64 instruction occupies an SM for ~16 cycles), so in mixed precision
// every per-velocity operation is float32 and the velocity sums are
// accumulated in float32 over at most 8 terms per lane, then in a compensated
// float-float pair (about 48 significant bits) across lanes; the pair is
// widened to float64 by the lane-parallel per-cell / per-face kernels, which
// do all scalar physics (state from moments, tau, equilibrium coefficients)
// in float64.  In FP64 mode the same code runs in float64 throughout.
//
// One iteration, in launch order on the caller's stream:
//   k_cell_moments   warp per cell: raw moments of f~                     [a1]
//   k_cell_params    thread per cell: heat flux (q of Eq. 20), tau,
//                    equilibrium at W^n, coefficients of fb+ (Eq. 10, 12)
//   k_fbp            per (cell, velocity): fb+ = c1 f~ + c2 f^S
//   k_cell_grad      (limiter on) per (cell, velocity): least-squares gradient
//                    (Eq. 14-15) and limiter (Eq. 16-17), stored as phi sigma
//   k_face_moments   warp per face: characteristic reconstruction of fb at the
//                    half step (Eq. 11, 13) with the gradient (computed in
//                    place when the limiter is off), wall density (Eq. 35),
//                    raw moments of fb; with the linearised wall the ghost
//                    density increment of Eq. (35)                     [a2-a3]
//   k_face_params    thread per face: face state, tau, q, equilibrium, and
//                    the weights of Eq. (18)                              [a4]
//   k_face_flux      warp per face: f at the face (Eq. 18), flux (Eq. 19),
//                    flux moments; with the linearised wall the ghost term
//                    of Eq. (34) on the incoming velocities of wall faces
//   k_face_phi       thread per face: Phi_f = sum_k w psi F_k (Eq. 27)
//   k_macro_pre, k_macro_sweep, k_macro_post: macroscopic LU-SGS          [a5]
//                    (k_macro_sweep_sched on an unstructured mesh; with the
//                    point-relaxation predictor k_record_residual and n
//                    launches of k_macro_relax in place of the sweep)
//   k_micro_residual, k_sweep_fwd, k_sweep_bwd: micro LU-SGS sweeps and
//                    update (hyperplanes on a structured block, level
//                    schedules on an unstructured mesh)              [a6-a7]
// Explicit DUGKS (Eq. 21) runs the cell and face kernels, then
// k_explicit_update, k_cell_moments, k_explicit_w and k_record_residual.
// Data are laid out per cell in four face slots (a triangle's fourth slot is
// unused: sign 0, no neighbour, no geometry).
#include "idugks_internal.h"

#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

namespace idg {

// ---------------------------------------------------------------------------
// precision helpers
// ---------------------------------------------------------------------------
template <class T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
// correctly rounded reciprocals: the same value as 1 / x in IEEE division,
// without the general division routine
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }
// 1/x in the line macroscopic sweep's flux increments: one approximate
// reciprocal in float32 -- the predictor's increments set the convergence
// path, not the fixed point, which the residual alone fixes -- and correctly
// rounded in float64 (FP64 parity with the oracle)
__device__ __forceinline__ float rcp_line(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp_line(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float t_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double t_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float t_exp(float x) { return expf(x); }
__device__ __forceinline__ double t_exp(double x) { return exp(x); }

template <class T> __device__ __forceinline__ T vx(const KParams &p, int k);
template <> __device__ __forceinline__ float vx<float>(const KParams &p, int k) { return p.uxf[k]; }
template <> __device__ __forceinline__ double vx<double>(const KParams &p, int k) { return p.ux[k]; }
template <class T> __device__ __forceinline__ T vy(const KParams &p, int k);
template <> __device__ __forceinline__ float vy<float>(const KParams &p, int k) { return p.uyf[k]; }
template <> __device__ __forceinline__ double vy<double>(const KParams &p, int k) { return p.uy[k]; }
template <class T> __device__ __forceinline__ T vw(const KParams &p, int k);
template <> __device__ __forceinline__ float vw<float>(const KParams &p, int k) { return p.wf[k]; }
template <> __device__ __forceinline__ double vw<double>(const KParams &p, int k) { return p.w[k]; }
template <class T> __device__ __forceinline__ T vgref(const KParams &p, int k);
template <> __device__ __forceinline__ float vgref<float>(const KParams &p, int k) { return p.greff[k]; }
template <> __device__ __forceinline__ double vgref<double>(const KParams &p, int k) { return p.gref[k]; }

// xi . n without contraction, so the sign decision matches a plain
// multiply-add evaluation bit for bit in float64
template <class T> __device__ __forceinline__ T xi_dot_n(T ux, T uy, T nx, T ny)
{
    return add_rn(mul_rn(ux, nx), mul_rn(uy, ny));
}

// ---------------------------------------------------------------------------
// accumulators: float-float pairs in mixed precision, double in FP64
// ---------------------------------------------------------------------------
struct FF {
    float hi, lo;
};
// error-free sum of two floats (Knuth's two-sum)
__device__ __forceinline__ FF two_sum(float a, float b)
{
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    FF s = two_sum(a.hi, b.hi);
    float e = s.lo + (a.lo + b.lo);
    float hi = s.hi + e;
    return {hi, e - (hi - s.hi)};
}

template <class T> struct Acc;
template <> struct Acc<float> {
    FF v;
    __device__ __forceinline__ void zero() { v = {0.f, 0.f}; }
    __device__ __forceinline__ void add(float x) { v = ff_add(v, FF{x, 0.f}); }
    __device__ __forceinline__ void warp_sum()
    {
        for (int o = 16; o > 0; o >>= 1) {
            FF u{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
            v = ff_add(v, u);
        }
    }
    __device__ __forceinline__ void store(void *base, size_t i) const { ((float2 *)base)[i] = make_float2(v.hi, v.lo); }
    __device__ __forceinline__ double value() const { return (double)v.hi + (double)v.lo; }
};
template <> struct Acc<double> {
    double v;
    __device__ __forceinline__ void zero() { v = 0.0; }
    __device__ __forceinline__ void add(double x) { v += x; }
    __device__ __forceinline__ void warp_sum()
    {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __device__ __forceinline__ void store(void *base, size_t i) const { ((double *)base)[i] = v; }
    __device__ __forceinline__ double value() const { return v; }
};

// an accumulator entry widened to float64
template <class T> __device__ __forceinline__ double acc_load(const void *base, size_t i);
template <> __device__ __forceinline__ double acc_load<float>(const void *base, size_t i)
{
    float2 a = ((const float2 *)base)[i];
    return (double)a.x + (double)a.y;
}
template <> __device__ __forceinline__ double acc_load<double>(const void *base, size_t i)
{
    return ((const double *)base)[i];
}

// block sum of float64 values (fixed tree: deterministic); result in thread 0
template <int NV>
__device__ void block_sum(double (&v)[NV], double *sm /* >= 32*NV */)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) sm[wid * NV + q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 0; q < NV; ++q) {
            double a = 0.0;
            for (int u = 0; u < nw; ++u) a += sm[u * NV + q];
            v[q] = a;
        }
    }
}

// ---------------------------------------------------------------------------
// launches over one or many problem instances
// ---------------------------------------------------------------------------
// Every iteration kernel takes a Launch: the instances' parameters in device
// memory, the prefix sums of blocks per instance for this kernel (null for a
// single instance) and per-instance activity flags (converged instances of a
// batch are skipped).  A block finds its instance by binary search.
struct Launch {
    const KParams *params;
    const int *off;     // [ninst + 1] or null
    const int *active;  // [ninst] or null
    int ninst;
};

__device__ __forceinline__ bool locate(const Launch &L, const KParams *&pp, int &blk)
{
    int b = blockIdx.x, inst = 0;
    if (L.off) {
        int lo = 0, hi = L.ninst;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (L.off[mid] <= b) lo = mid;
            else hi = mid;
        }
        inst = lo;
        b -= L.off[lo];
    }
    pp = L.params + inst;
    blk = b;
    return !L.active || L.active[inst];
}

#define IDG_LOCATE()                                   \
    const KParams *pp_;                                \
    int blk;                                           \
    if (!locate(L, pp_, blk)) return;                  \
    const KParams &__restrict__ p = *pp_;

// ---------------------------------------------------------------------------
// kinetic model in float64 (per cell / per face quantities)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double viscosity(const KParams &p, double RT)
{
    return p.mu_ref * pow(RT / p.RT_ref, p.omega);
}

// The power law of the viscosity for tau in the iteration's kernels: with
// float32 storage tau only sets float32 coefficients (fb+ weights, Eq. 18
// weights, the collision rate, the Shakhov factor) and the float32
// preconditioner, so the power is taken in float32; float64 keeps float64.
template <class T> __device__ __forceinline__ double viscosity_t(const KParams &p, double RT);
template <> __device__ __forceinline__ double viscosity_t<double>(const KParams &p, double RT)
{
    return viscosity(p, RT);
}
template <> __device__ __forceinline__ double viscosity_t<float>(const KParams &p, double RT)
{
    return p.mu_ref * (double)powf((float)(RT / p.RT_ref), (float)p.omega);
}

// heat flux q = 1/2 sum w c (c^2 G + H) about (U, V) from raw moments
// (G: 1,x,y,xx,xy,yy,x|xi|^2,y|xi|^2; H: 1,x,y), Eq. (4)-(5)
__device__ __forceinline__ void raw_heat_flux(const double *r, double U, double V, double &qx,
                                              double &qy)
{
    double U2 = U * U + V * V;
    double sx = r[6] - 2.0 * U * r[3] - 2.0 * V * r[4] + U2 * r[1] - U * (r[3] + r[5]) +
                2.0 * U * U * r[1] + 2.0 * U * V * r[2] - U * U2 * r[0];
    double sy = r[7] - 2.0 * U * r[4] - 2.0 * V * r[5] + U2 * r[2] - V * (r[3] + r[5]) +
                2.0 * U * V * r[1] + 2.0 * V * V * r[2] - V * U2 * r[0];
    qx = 0.5 * (sx + r[9] - U * r[8]);
    qy = 0.5 * (sy + r[10] - V * r[8]);
}

__device__ void raw_to_state(const double *r, int K, double &rho, double &U, double &V,
                             double &RT, double &qx, double &qy)
{
    rho = r[0];
    U = r[1] / rho;
    V = r[2] / rho;
    double rhoE = 0.5 * (r[3] + r[5] + r[8]);
    RT = (2.0 * rhoE / rho - U * U - V * V) / (K + 2);
    raw_heat_flux(r, U, V, qx, qy);
}

// Coefficients of the deviation equilibrium at (rho, U, V, RT, q):
// reduced Maxwellian (Eq. 2, 5) with the Shakhov factor (Eq. 20 read for
// D = 2 + K dof: G factor (c^2/RT - 4), H factor (c^2/RT - 2)).
struct EqD {
    double e0, ex, ey, e2, U, V, invRT, pqx, pqy, rr, rrm1, kRT, A, lam;
};

__device__ EqD make_eq(const KParams &p, double rho, double U, double V, double RT, double qx,
                       double qy)
{
    EqD e;
    double lam = 0.5 / RT, lamr = 0.5 / p.RT_r;
    e.e2 = lamr - lam;
    e.ex = 2.0 * (lam * U - lamr * p.U_r);
    e.ey = 2.0 * (lam * V - lamr * p.V_r);
    // a non-positive density (a transient state, e.g. an evacuated wall
    // face after an impulsive start) has no logarithm: e0 then sends every
    // velocity to the direct branch, which takes the signed amplitude A
    e.e0 = rho > 0.0 ? log(rho * lam / (p.rho_r * lamr)) - lam * (U * U + V * V) +
                           lamr * (p.U_r * p.U_r + p.V_r * p.V_r)
                     : 1e30;
    e.U = U;
    e.V = V;
    e.invRT = 1.0 / RT;
    double pc = p.shakhov && rho != 0.0 ? (1.0 - p.Pr) / ((p.K + 4) * rho * RT * RT) : 0.0;
    e.pqx = pc * qx;
    e.pqy = pc * qy;
    e.rr = RT / p.RT_r;
    e.rrm1 = (RT - p.RT_r) / p.RT_r;
    e.kRT = p.K * RT;
    e.A = rho * lam / M_PI;
    e.lam = lam;
    return e;
}

template <class T> struct EqT {
    T e0, ex, ey, e2, U, V, invRT, pqx, pqy, rr, rrm1, kRT, A, lam;
};

template <class T> __device__ __forceinline__ void eq_storeT(T *cp, const EqD &e)
{
    cp[0] = (T)e.e0; cp[1] = (T)e.ex; cp[2] = (T)e.ey; cp[3] = (T)e.e2; cp[4] = (T)e.U;
    cp[5] = (T)e.V; cp[6] = (T)e.invRT; cp[7] = (T)e.pqx; cp[8] = (T)e.pqy; cp[9] = (T)e.rr;
    cp[10] = (T)e.rrm1; cp[11] = (T)e.kRT; cp[12] = (T)e.A; cp[13] = (T)e.lam;
}

__device__ __forceinline__ void eq_store(double *cp, const EqD &e) { eq_storeT<double>(cp, e); }

template <class T> __device__ __forceinline__ EqT<T> eq_loadT(const T *cp)
{
    EqT<T> e;
    e.e0 = cp[0]; e.ex = cp[1]; e.ey = cp[2]; e.e2 = cp[3]; e.U = cp[4]; e.V = cp[5];
    e.invRT = cp[6]; e.pqx = cp[7]; e.pqy = cp[8]; e.rr = cp[9]; e.rrm1 = cp[10]; e.kRT = cp[11];
    e.A = cp[12]; e.lam = cp[13];
    return e;
}

// f^S(k) - M_ref(k) for G and H.  Near M_ref (|E| < 1/2) through expm1 of the
// exponent difference E = ln(f^eq/M_ref), so the result is accurate relative
// to the deviation; far from it directly (no cancellation is possible then).
template <class T>
__device__ __forceinline__ void dev_equilibrium(const EqT<T> &e, T ux, T uy, T gref, T kRTr,
                                                T &dG, T &dH)
{
    T cx = ux - e.U, cy = uy - e.V;
    T q2 = cx * cx + cy * cy;
    T t = q2 * e.invRT;
    T P = e.pqx * cx + e.pqy * cy;
    T PG = P * (t - (T)4), PH = P * (t - (T)2);
    T E = e.e0 + e.ex * ux + e.ey * uy + e.e2 * (ux * ux + uy * uy);
    T href = kRTr * gref;
    if (fabs(E) < (T)0.5) {
        T em = t_expm1(E);
        T s = em + PG * ((T)1 + em);
        dG = gref * s;
        dH = href * (e.rrm1 + e.rr * (em + PH * ((T)1 + em)));
    } else {
        T g = e.A * t_exp(-e.lam * q2);
        dG = g * ((T)1 + PG) - gref;
        dH = e.kRT * g * ((T)1 + PH) - href;
    }
}

// raw-moment partials of one velocity: G: 1,x,y,xx,xy,yy,x|xi|^2,y|xi|^2; H: 1,x,y
template <class T>
__device__ __forceinline__ void raw_terms(T (&a)[kRaw], T w, T ux, T uy, T g, T h)
{
    T wg = w * g, wh = w * h, s2 = ux * ux + uy * uy;
    a[0] += wg; a[1] += wg * ux; a[2] += wg * uy; a[3] += wg * ux * ux; a[4] += wg * ux * uy;
    a[5] += wg * uy * uy; a[6] += wg * ux * s2; a[7] += wg * uy * s2;
    a[8] += wh; a[9] += wh * ux; a[10] += wh * uy;
}

// Warp loop over the discrete velocities: lane l takes k = k0 + 32u + l,
// u < 8, for chunks of 256 velocities; each chunk's per-lane partial sums
// (at most 8 terms, storage precision) are folded into the accumulators.
// Full chunks run unchecked and unrolled so several velocities' loads are in
// flight; the ragged last chunk is bounds-checked.
template <int NA, class T, class Body>
__device__ __forceinline__ void vel_loop(int Nv, int lane, Acc<T> (&acc)[NA], Body body)
{
    int k0 = 0;
    for (; k0 + 256 <= Nv; k0 += 256) {
        T a[NA];
#pragma unroll
        for (int q = 0; q < NA; ++q) a[q] = (T)0;
#pragma unroll 4
        for (int u = 0; u < 8; ++u) body(k0 + 32 * u + lane, a);
#pragma unroll
        for (int q = 0; q < NA; ++q) acc[q].add(a[q]);
    }
    if (k0 < Nv) {
        T a[NA];
#pragma unroll
        for (int q = 0; q < NA; ++q) a[q] = (T)0;
        for (int u = 0; u < 8; ++u) {
            int k = k0 + 32 * u + lane;
            if (k < Nv) body(k, a);
        }
#pragma unroll
        for (int q = 0; q < NA; ++q) acc[q].add(a[q]);
    }
}

template <class T> __device__ __forceinline__ void load_pair(const void *base, size_t i, T (&g)[2], T (&h)[2]);

// Pair loop over the discrete velocities: lane l takes the two velocities
// k, k + 1 with k = k0 + 64u + 2l, u < 4, for chunks of 256 velocities (the
// stored velocity count is a multiple of 4, so pairs are whole and start on
// 16-byte boundaries); each chunk's per-lane partial sums (at most 8 terms)
// are folded into the accumulators as in vel_loop.
template <int NA, class T, class Body>
__device__ __forceinline__ void vel_loop2(int Nv, int lane, Acc<T> (&acc)[NA], Body body)
{
    int k0 = 0;
    for (; k0 + 256 <= Nv; k0 += 256) {
        T a[NA];
#pragma unroll
        for (int q = 0; q < NA; ++q) a[q] = (T)0;
#pragma unroll 2
        for (int u = 0; u < 4; ++u) body(k0 + 64 * u + 2 * lane, a);
#pragma unroll
        for (int q = 0; q < NA; ++q) acc[q].add(a[q]);
    }
    if (k0 < Nv) {
        T a[NA];
#pragma unroll
        for (int q = 0; q < NA; ++q) a[q] = (T)0;
        for (int u = 0; u < 4; ++u) {
            int k = k0 + 64 * u + 2 * lane;
            if (k < Nv) body(k, a);
        }
#pragma unroll
        for (int q = 0; q < NA; ++q) acc[q].add(a[q]);
    }
}

// store of two consecutive velocities' {G, H} (see load_pair)
template <class T> __device__ __forceinline__ void store_pair(void *base, size_t i, const T (&g)[2], const T (&h)[2]);
template <> __device__ __forceinline__ void store_pair<float>(void *base, size_t i, const float (&g)[2], const float (&h)[2])
{
    ((float4 *)base)[i >> 1] = make_float4(g[0], h[0], g[1], h[1]);
}
template <> __device__ __forceinline__ void store_pair<double>(void *base, size_t i, const double (&g)[2], const double (&h)[2])
{
    ((double2 *)base)[i] = make_double2(g[0], h[0]);
    ((double2 *)base)[i + 1] = make_double2(g[1], h[1]);
}

// velocity table entries k, k + 1 (k even)
template <class T> __device__ __forceinline__ void vtab2(const float *tf, const double *td, int k, T (&o)[2]);
template <> __device__ __forceinline__ void vtab2<float>(const float *tf, const double *, int k, float (&o)[2])
{
    const float2 v = ((const float2 *)tf)[k >> 1];
    o[0] = v.x; o[1] = v.y;
}
template <> __device__ __forceinline__ void vtab2<double>(const float *, const double *td, int k, double (&o)[2])
{
    const double2 v = ((const double2 *)td)[k >> 1];
    o[0] = v.x; o[1] = v.y;
}

// The same loop with each thread's float-float accumulators held in shared
// memory (sacc[q * blockDim.x + threadIdx.x]) between chunks: the arithmetic is
// that of vel_loop, while the registers of a 64-register thread stay free for
// the loads in flight.  Float storage only; the float64 path keeps vel_loop.
template <int NA, class Body>
__device__ __forceinline__ void vel_loop_sm(int Nv, int lane, FF *sacc, Body body)
{
    const int t = threadIdx.x, nt = blockDim.x;
#pragma unroll
    for (int q = 0; q < NA; ++q) sacc[q * nt + t] = FF{0.f, 0.f};
    auto fold = [&](const float(&a)[NA]) {
#pragma unroll
        for (int q = 0; q < NA; ++q) sacc[q * nt + t] = ff_add(sacc[q * nt + t], FF{a[q], 0.f});
    };
    int k0 = 0;
    for (; k0 + 256 <= Nv; k0 += 256) {
        float a[NA];
#pragma unroll
        for (int q = 0; q < NA; ++q) a[q] = 0.f;
#pragma unroll 4
        for (int u = 0; u < 8; ++u) body(k0 + 32 * u + lane, a);
        fold(a);
    }
    if (k0 < Nv) {
        float a[NA];
#pragma unroll
        for (int q = 0; q < NA; ++q) a[q] = 0.f;
        for (int u = 0; u < 8; ++u) {
            int k = k0 + 32 * u + lane;
            if (k < Nv) body(k, a);
        }
        fold(a);
    }
}

// vel_loop2 with the accumulators of vel_loop_sm
template <int NA, class Body>
__device__ __forceinline__ void vel_loop2_sm(int Nv, int lane, FF *sacc, Body body)
{
    const int t = threadIdx.x, nt = blockDim.x;
#pragma unroll
    for (int q = 0; q < NA; ++q) sacc[q * nt + t] = FF{0.f, 0.f};
    auto fold = [&](const float(&a)[NA]) {
#pragma unroll
        for (int q = 0; q < NA; ++q) sacc[q * nt + t] = ff_add(sacc[q * nt + t], FF{a[q], 0.f});
    };
    int k0 = 0;
    for (; k0 + 256 <= Nv; k0 += 256) {
        float a[NA];
#pragma unroll
        for (int q = 0; q < NA; ++q) a[q] = 0.f;
#pragma unroll 2
        for (int u = 0; u < 4; ++u) body(k0 + 64 * u + 2 * lane, a);
        fold(a);
    }
    if (k0 < Nv) {
        float a[NA];
#pragma unroll
        for (int q = 0; q < NA; ++q) a[q] = 0.f;
        for (int u = 0; u < 4; ++u) {
            int k = k0 + 64 * u + 2 * lane;
            if (k < Nv) body(k, a);
        }
        fold(a);
    }
}

// ---------------------------------------------------------------------------
// cell moments and cell prep (Eq. 10, 12)                                [a1]
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void cell_moments_body(const KParams &__restrict__ p, int blk)
{
    using T2 = typename V2<T>::t;
    const int lane = threadIdx.x & 31;
    const int c = blk * 8 + (threadIdx.x >> 5);
    if (c >= p.N) return;  // whole warp
    const T2 *f = (const T2 *)p.f + (size_t)c * p.Nv;
    Acc<T> acc[kRaw];
#pragma unroll
    for (int q = 0; q < kRaw; ++q) acc[q].zero();
    vel_loop2<kRaw, T>(p.Nv, lane, acc, [&](int k, T(&a)[kRaw]) {
        T ux[2], uy[2], w[2], g[2], h[2];
        vtab2<T>(p.uxf, p.ux, k, ux);
        vtab2<T>(p.uyf, p.uy, k, uy);
        vtab2<T>(p.wf, p.w, k, w);
        load_pair<T>(f, k, g, h);
        raw_terms<T>(a, w[0], ux[0], uy[0], g[0], h[0]);
        raw_terms<T>(a, w[1], ux[1], uy[1], g[1], h[1]);
    });
#pragma unroll
    for (int q = 0; q < kRaw; ++q) acc[q].warp_sum();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < kRaw; ++q) acc[q].store(p.cellraw, (size_t)c * kRaw + q);
}

template <class T>
__global__ void __launch_bounds__(256) k_cell_moments(Launch L)
{
    IDG_LOCATE();
    cell_moments_body<T>(p, blk);
}

// the same with the parameters passed by value (moment queries)
template <class T>
__global__ void __launch_bounds__(256) k_cell_moments_v(KParams p)
{
    cell_moments_body<T>(p, blockIdx.x);
}

// per cell: heat flux of f from f~ (about U of W), tau, equilibrium at W^n,
// and the two coefficients of fb+ = (2tau-h)/(2tau+dt) f~ + 3h/(2tau+dt) f^S
template <class T>
__global__ void __launch_bounds__(32) k_cell_params(Launch L)
{
    IDG_LOCATE();
    const int c = blk * blockDim.x + threadIdx.x;
    if (c >= p.N) return;
    double r[kRaw];
    for (int q = 0; q < kRaw; ++q) r[q] = acc_load<T>(p.cellraw, (size_t)c * kRaw + q) + p.mref_raw[q];
    const double *W = p.W + 4 * c;
    double rho = W[0], U = W[1] / rho, V = W[2] / rho;
    double RT = (2.0 * W[3] / rho - U * U - V * V) / (p.K + 2);
    double tau = viscosity_t<T>(p, RT) / (rho * RT);
    double qtx, qty;
    raw_heat_flux(r, U, V, qtx, qty);
    double Pr = p.shakhov ? p.Pr : 1.0;
    double qx = 2.0 * tau * qtx / (2.0 * tau + p.dt * Pr);
    double qy = 2.0 * tau * qty / (2.0 * tau + p.dt * Pr);
    p.cellq[2 * c] = qx;
    p.cellq[2 * c + 1] = qy;
    T *cA = (T *)p.cellA + kCellP * c;
    eq_storeT<T>(cA, make_eq(p, rho, U, V, RT, qx, qy));
    cA[14] = (T)((2.0 * tau - p.h) / (2.0 * tau + p.dt));
    cA[15] = (T)(3.0 * p.h / (2.0 * tau + p.dt));
}

// per (cell, pair of velocities): fb+ = c1 f~ + c2 f^S; 128-thread blocks,
// each over 256 velocities of one cell
template <class T>
__global__ void __launch_bounds__(128) k_fbp(Launch L)
{
    IDG_LOCATE();
    const int nvb = (p.Nv + 255) / 256;
    const int c = blk / nvb;
    const int k = 2 * ((blk - c * nvb) * 128 + threadIdx.x);
    if (k >= p.Nv) return;
    const T *cA = (const T *)p.cellA + kCellP * c;
    const EqT<T> e = eq_loadT<T>(cA);
    const T c1 = cA[14], c2 = cA[15], kRTr = (T)(p.K * p.RT_r);
    const size_t ck = (size_t)c * p.Nv + k;
    T ux[2], uy[2], gr[2], g[2], h[2];
    vtab2<T>(p.uxf, p.ux, k, ux);
    vtab2<T>(p.uyf, p.uy, k, uy);
    vtab2<T>(p.greff, p.gref, k, gr);
    load_pair<T>(p.f, ck, g, h);
#pragma unroll
    for (int v = 0; v < 2; ++v) {
        T dG, dH;
        dev_equilibrium<T>(e, ux[v], uy[v], gr[v], kRTr, dG, dH);
        g[v] = c1 * g[v] + c2 * dG;
        h[v] = c1 * h[v] + c2 * dH;
    }
    store_pair<T>(p.fbp, ck, g, h);
}

// ---------------------------------------------------------------------------
// faces: reconstruction from one cell along the characteristic (Eq. 11,
// 13-17), moments, face equilibrium and flux (Eq. 18-19)            [a2-a4]
// ---------------------------------------------------------------------------
template <class T> struct SideRec {
    int c;
    int nb[4];
    T gx[4], gy[4];    // least-squares weights: sigma = sum_m g_m (phi_nb - phi_c)
    T rx, ry;          // face midpoint minus centroid for the face being built
    T frx[4], fry[4];  // all four face offsets of the cell (limiter)
};

template <class T>
__device__ __forceinline__ void load_side(const KParams &p, int c, T rx, T ry, SideRec<T> &r)
{
    const T *g = (const T *)p.clsgT + 8 * c;
    const T *o = (const T *)p.crT + 8 * c;
    r.c = c;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        r.nb[m] = p.cnb[4 * c + m];
        r.gx[m] = g[2 * m];
        r.gy[m] = g[2 * m + 1];
        r.frx[m] = o[2 * m];
        r.fry[m] = o[2 * m + 1];
    }
    r.rx = rx;
    r.ry = ry;
}

// Divisions of the limiter: exact in float64 (the oracle's rounding up to
// order); in float32 storage the approximate quotient (2 ulp) of the fast
// reciprocal path, the limiter being a smooth function of its ratios
__device__ __forceinline__ float lim_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double lim_div(double a, double b) { return a / b; }

template <class T> __device__ __forceinline__ T venkat(T x) { return lim_div(x * x + (T)2 * x, x * x + x + (T)2); }

// G and H of two consecutive velocities k, k + 1 (k even: 16-byte aligned
// because the stored velocity count is a multiple of 4)
template <class T> __device__ __forceinline__ void load_pair(const void *base, size_t i, T (&g)[2], T (&h)[2]);
template <> __device__ __forceinline__ void load_pair<float>(const void *base, size_t i, float (&g)[2], float (&h)[2])
{
    const float4 a = ((const float4 *)base)[i >> 1];
    g[0] = a.x; h[0] = a.y; g[1] = a.z; h[1] = a.w;
}
template <> __device__ __forceinline__ void load_pair<double>(const void *base, size_t i, double (&g)[2], double (&h)[2])
{
    const double2 a = ((const double2 *)base)[i], b = ((const double2 *)base)[i + 1];
    g[0] = a.x; h[0] = a.y; g[1] = b.x; h[1] = b.y;
}

// four storage scalars (one velocity's limited gradients), 16- or 32-byte aligned
template <class T> __device__ __forceinline__ void store4(T *d, T a, T b, T c, T e);
template <> __device__ __forceinline__ void store4<float>(float *d, float a, float b, float c, float e)
{
    *(float4 *)d = make_float4(a, b, c, e);
}
template <> __device__ __forceinline__ void store4<double>(double *d, double a, double b, double c, double e)
{
    ((double2 *)d)[0] = make_double2(a, b);
    ((double2 *)d)[1] = make_double2(c, e);
}
template <class T> __device__ __forceinline__ void load4(const T *s, T &a, T &b, T &c, T &e);
template <> __device__ __forceinline__ void load4<float>(const float *s, float &a, float &b, float &c, float &e)
{
    const float4 v = *(const float4 *)s;
    a = v.x; b = v.y; c = v.z; e = v.w;
}
template <> __device__ __forceinline__ void load4<double>(const double *s, double &a, double &b, double &c, double &e)
{
    const double2 v = ((const double2 *)s)[0], w = ((const double2 *)s)[1];
    a = v.x; b = v.y; c = w.x; e = w.y;
}

// limiter of one scalar (Eq. 16-17): phi = min over the faces of
// theta(x_m), x_m = (v_max - v0)/d_m where the extrapolated increment d_m to
// the face is positive, (v_min - v0)/d_m where it is negative (faces with
// d_m = 0 impose nothing), capped at 1.  Every x_m is >= 0, and theta rises
// monotonically from theta(0) = 0 to theta(2) = 1 and stays >= 1 beyond, so
// phi = theta(min(2, min_m x_m)): one evaluation of theta instead of four.
// Selects instead of branches: the sign of d differs between neighbouring
// velocities.
// With the smoothing constant (e2 = eps^2 > 0) each face's factor is
// (P^2 + e2 + 2 D P) / (P^2 + 2 D^2 + P D + e2), P the increment to the
// neighbourhood's max or min, D the extrapolated one, and the minimum is
// taken over the four faces (the factor is no function of P / D alone).
template <class T>
__device__ __forceinline__ T limit_scalar_sel(const T (&frx)[4], const T (&fry)[4], T v0, T vmax, T vmin, T sx, T sy,
                                              T e2)
{
    if (e2 > (T)0) {
        T phi = (T)1;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const T d = sx * frx[m] + sy * fry[m];
            const T P = (d > (T)0 ? vmax : vmin) - v0;
            const T t = lim_div(P * P + e2 + (T)2 * d * P, P * P + (T)2 * d * d + P * d + e2);
            phi = (d != (T)0 && t < phi) ? t : phi;
        }
        return phi;
    }
    T xm = (T)2;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const T d = sx * frx[m] + sy * fry[m];
        const T x = lim_div((d > (T)0 ? vmax : vmin) - v0, d);
        xm = (d != (T)0 && x < xm) ? x : xm;
    }
    return venkat<T>(xm);
}

// per (cell, pair of velocities), limiter on: least-squares gradients of fb+
// (Eq. 14-15) and the Venkatakrishnan limiter (Eq. 16-17) of G and H, stored
// as the limited gradients phi sigma for the reconstructions at the cell's
// faces.  128-thread blocks, each over 256 velocities of one cell; the cell's
// stencil record is read by every thread (one broadcast per load).
template <class T>
__global__ void __launch_bounds__(128) k_cell_grad(Launch L)
{
    IDG_LOCATE();
    if (!p.limiter) return;
    const int nvb = (p.Nv + 255) / 256;
    const int c = blk / nvb;
    const int k = 2 * ((blk - c * nvb) * 128 + threadIdx.x);
    if (k >= p.Nv) return;
    int nb[4];
    T gx[4], gy[4], frx[4], fry[4];
    {
        const int4 n4 = *(const int4 *)(p.cnb + 4 * c);
        nb[0] = n4.x; nb[1] = n4.y; nb[2] = n4.z; nb[3] = n4.w;
        const T *g = (const T *)p.clsgT + 8 * c;
        const T *o = (const T *)p.crT + 8 * c;
        load4<T>(g, gx[0], gy[0], gx[1], gy[1]);
        load4<T>(g + 4, gx[2], gy[2], gx[3], gy[3]);
        load4<T>(o, frx[0], fry[0], frx[1], fry[1]);
        load4<T>(o + 4, frx[2], fry[2], frx[3], fry[3]);
    }
    T g0[2], h0[2];
    load_pair<T>(p.fbp, (size_t)c * p.Nv + k, g0, h0);
    T sgx[2] = {0, 0}, sgy[2] = {0, 0}, shx[2] = {0, 0}, shy[2] = {0, 0};
    T gmax[2] = {g0[0], g0[1]}, gmin[2] = {g0[0], g0[1]}, hmax[2] = {h0[0], h0[1]}, hmin[2] = {h0[0], h0[1]};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (nb[m] < 0) continue;
        T gn[2], hn[2];
        load_pair<T>(p.fbp, (size_t)nb[m] * p.Nv + k, gn, hn);
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const T dg = gn[v] - g0[v], dh = hn[v] - h0[v];
            sgx[v] += gx[m] * dg; sgy[v] += gy[m] * dg;
            shx[v] += gx[m] * dh; shy[v] += gy[m] * dh;
            gmax[v] = gn[v] > gmax[v] ? gn[v] : gmax[v]; gmin[v] = gn[v] < gmin[v] ? gn[v] : gmin[v];
            hmax[v] = hn[v] > hmax[v] ? hn[v] : hmax[v]; hmin[v] = hn[v] < hmin[v] ? hn[v] : hmin[v];
        }
    }
    T *gout = (T *)p.grad + 4 * ((size_t)c * p.Nv + k);
    // the smoothing constant's eps^2 = (K h)^3, h = sqrt(area) (0: Eq. 16-17)
    T e2 = (T)0;
    if (p.venkat_k3 > 0.0) {
        const double a = p.area[c];
        e2 = (T)(p.venkat_k3 * a * sqrt(a));
    }
#pragma unroll
    for (int v = 0; v < 2; ++v) {
        const T pg = limit_scalar_sel<T>(frx, fry, g0[v], gmax[v], gmin[v], sgx[v], sgy[v], e2);
        const T ph = limit_scalar_sel<T>(frx, fry, h0[v], hmax[v], hmin[v], shx[v], shy[v], e2);
        store4<T>(gout + 4 * v, pg * sgx[v], pg * sgy[v], ph * shx[v], ph * shy[v]);
    }
}

// fb at the face from side r: fb+_c + phi sigma_c . (x_f - xi h - x_c).  The
// limiter ratios only involve differences of fb+ between cells at one
// velocity, so the M_ref offset cancels and deviations serve as is.
template <class T, bool LIM>
__device__ __forceinline__ typename V2<T>::t reconstruct(const KParams &p, const SideRec<T> &r,
                                                         int k, T ux, T uy, T h)
{
    using T2 = typename V2<T>::t;
    const T2 *fb = (const T2 *)p.fbp;
    T2 f0 = fb[(size_t)r.c * p.Nv + k];
    if (LIM && p.limiter) {
        // limited gradients phi sigma of G and H, stored once per (cell,
        // velocity) by k_cell_grad
        T g0, g1, g2, g3;
        load4<T>((const T *)p.grad + 4 * ((size_t)r.c * p.Nv + k), g0, g1, g2, g3);
        const T ax = r.rx - ux * h, ay = r.ry - uy * h;
        T2 o;
        o.x = f0.x + (g0 * ax + g1 * ay);
        o.y = f0.y + (g2 * ax + g3 * ay);
        return o;
    }
    // limiter off: the unlimited least-squares gradient in place
    T sgx = 0, sgy = 0, shx = 0, shy = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (r.nb[m] < 0) continue;
        T2 fn = fb[(size_t)r.nb[m] * p.Nv + k];
        T dg = fn.x - f0.x, dh = fn.y - f0.y;
        sgx += r.gx[m] * dg; sgy += r.gy[m] * dg;
        shx += r.gx[m] * dh; shy += r.gy[m] * dh;
    }
    T ax = r.rx - ux * h, ay = r.ry - uy * h;
    T2 o;
    o.x = f0.x + (sgx * ax + sgy * ay);
    o.y = f0.y + (shx * ax + shy * ay);
    return o;
}

// reconstruct for the velocity pair k, k + 1 from one side
template <class T, bool LIM>
__device__ __forceinline__ void reconstruct2(const KParams &p, const SideRec<T> &r, int k, const T (&ux)[2],
                                             const T (&uy)[2], T h, T (&og)[2], T (&oh)[2])
{
    T g0[2], h0[2];
    load_pair<T>(p.fbp, (size_t)r.c * p.Nv + k, g0, h0);
    if (LIM) {
        const T *gp = (const T *)p.grad + 4 * ((size_t)r.c * p.Nv + k);
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            T a0, a1, a2, a3;
            load4<T>(gp + 4 * v, a0, a1, a2, a3);
            const T ax = r.rx - ux[v] * h, ay = r.ry - uy[v] * h;
            og[v] = g0[v] + (a0 * ax + a1 * ay);
            oh[v] = h0[v] + (a2 * ax + a3 * ay);
        }
        return;
    }
    T sgx[2] = {0, 0}, sgy[2] = {0, 0}, shx[2] = {0, 0}, shy[2] = {0, 0};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (r.nb[m] < 0) continue;
        T gn[2], hn[2];
        load_pair<T>(p.fbp, (size_t)r.nb[m] * p.Nv + k, gn, hn);
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const T dg = gn[v] - g0[v], dh = hn[v] - h0[v];
            sgx[v] += r.gx[m] * dg; sgy[v] += r.gy[m] * dg;
            shx[v] += r.gx[m] * dh; shy[v] += r.gy[m] * dh;
        }
    }
#pragma unroll
    for (int v = 0; v < 2; ++v) {
        const T ax = r.rx - ux[v] * h, ay = r.ry - uy[v] * h;
        og[v] = g0[v] + (sgx[v] * ax + sgy[v] * ay);
        oh[v] = h0[v] + (shx[v] * ax + shy[v] * ay);
    }
}

// The two side records live in shared memory (one pair per warp) so the
// per-lane choice of the upwind side is an indexed shared-memory read.
template <class T> struct FaceCtx {
    int kind;          // -1 interior, 1 wall, 2 far field
    int side;
    T nx, ny, S, on;   // normal L->R, length; boundary: +1 if the interior cell is L
    const SideRec<T> *rec;  // [2]: L, R (boundary faces: [0] is the interior cell)
};

template <class T>
__device__ __forceinline__ void load_face(const KParams &p, int f, SideRec<T> *srec, FaceCtx<T> &fc)
{
    const int lane = threadIdx.x & 31;
    const T *g = (const T *)p.fgeoT + 8 * f;
    fc.nx = g[0];
    fc.ny = g[1];
    fc.S = g[2];
    fc.kind = p.fbc[f];
    fc.side = p.fside[f];
    const int L = p.fL[f], R = p.fR[f];
    fc.on = (fc.kind < 0 || L >= 0) ? (T)1 : (T)-1;
    if (lane == 0) {
        if (L >= 0) load_side<T>(p, L, g[3], g[4], srec[0]);
        else load_side<T>(p, R, g[5], g[6], srec[0]);
    } else if (lane == 1 && fc.kind < 0) {
        load_side<T>(p, R, g[5], g[6], srec[1]);
    }
    __syncwarp();
    fc.rec = srec;
}

// fb - M_ref at velocity k.  Interior: upwind side by sign(xi.n), average at
// a tie.  Boundary: outgoing from the interior cell; incoming from the wall
// Maxwellian rho_w M_w (rho_w - 1 passed as rwm1) or the far-field state.
template <class T, bool LIM>
__device__ __forceinline__ typename V2<T>::t face_fbar(const KParams &p, const FaceCtx<T> &fc, int k,
                                                       T ux, T uy, T s, T rhow, T rwm1)
{
    using T2 = typename V2<T>::t;
    const T h = (T)p.h;
    if (fc.kind < 0) {
        T2 fb = reconstruct<T, LIM>(p, fc.rec[s > (T)0 ? 0 : 1], k, ux, uy, h);
        if (s == (T)0) {
            T2 o = reconstruct<T, LIM>(p, fc.rec[0], k, ux, uy, h);
            fb.x = (T)0.5 * (o.x + fb.x);
            fb.y = (T)0.5 * (o.y + fb.y);
        }
        return fb;
    }
    T so = fc.on * s;
    T2 in;
    if (so <= (T)0) {
        const T *bG = (const T *)p.bdevG + (size_t)fc.side * p.Nv;
        const T *bH = (const T *)p.bdevH + (size_t)fc.side * p.Nv;
        T gref = vgref<T>(p, k);
        in.x = rhow * bG[k] + rwm1 * gref;
        in.y = rhow * bH[k] + rwm1 * (T)(p.K * p.RT_r) * gref;
        if (so < (T)0) return in;
    }
    T2 fb = reconstruct<T, LIM>(p, fc.rec[0], k, ux, uy, h);
    if (so == (T)0) {
        fb.x = (T)0.5 * (fb.x + in.x);
        fb.y = (T)0.5 * (fb.y + in.y);
    }
    return fb;
}

// Linearised wall (Eq. 33-35), at a wall face f: the outgoing sum
// S = sum_out w (xi.n_out) G~ of the inner cell's stored state (products in
// the storage type, compensated sum across lanes: float64 stays exact to
// round-off, float32 rounds each product as the fluxes themselves are
// rounded) and the ghost density increment of Eq. (35),
//   drho_g = (S^n - S^{n-1}) / sum_in w |xi.n_out| G_w,
// zero in the first iteration after a restart.  The M_ref part of f~
// cancels in the difference.  Out of line: the wall faces' extra work keeps
// out of the register allocation of the kernel's hot path.
template <class T>
__device__ __noinline__ void wall_ghost_density(const KParams &p, int f, int lane, int c, T on, T nx, T ny,
                                                double in_sum)
{
    using T2 = typename V2<T>::t;
    const T2 *fc0 = (const T2 *)p.f + (size_t)c * p.Nv;
    Acc<T> a[1];
    a[0].zero();
    vel_loop<1, T>(p.Nv, lane, a, [&](int k, T(&q)[1]) {
        const T so = on * xi_dot_n<T>(vx<T>(p, k), vy<T>(p, k), nx, ny);
        if (so > (T)0) q[0] += vw<T>(p, k) * so * fc0[k].x;
    });
    a[0].warp_sum();
    const double sn = __shfl_sync(0xffffffffu, a[0].value(), 0);
    if (lane == 0) {
        p.walldrg[f] = *p.wallok ? (sn - p.wallS[f]) / in_sum : 0.0;
        p.wallS[f] = sn;
    }
}

// raw moments of fb - M_ref at every face (plus the wall density, Eq. 35).
// float32: the kernel is bound by the latency of its stencil loads, so
// occupancy decides: four 256-thread blocks per SM (64 registers, the lanes'
// float-float accumulators in shared memory, two velocities per lane); three
// or two blocks without spills, or five, six and eight with more, were slower
template <class T, bool LIM>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 1) k_face_moments(Launch L)
{
    IDG_LOCATE();
    using T2 = typename V2<T>::t;
    __shared__ SideRec<T> srec[8][2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int f = blk * 8 + wid;
    if (f >= p.nf) return;  // whole warp
    FaceCtx<T> fc;
    load_face<T>(p, f, srec[wid], fc);
    const T h = (T)p.h;
    T rhow = (T)1, rwm1 = (T)0;
    double rw = 1.0;
    Acc<T> outsum[1];
    outsum[0].zero();
    if (fc.kind == 1) {
        // zero net mass flux: rho_w sum_in w |xi.n| G_w = sum_out w (xi.n) fb
        vel_loop<1, T>(p.Nv, lane, outsum, [&](int k, T(&a)[1]) {
            T ux = vx<T>(p, k), uy = vy<T>(p, k);
            T so = fc.on * xi_dot_n<T>(ux, uy, fc.nx, fc.ny);
            if (so > (T)0) {
                T2 fb = reconstruct<T, LIM>(p, fc.rec[0], k, ux, uy, h);
                a[0] += vw<T>(p, k) * so * fb.x;
            }
        });
        outsum[0].warp_sum();
        double o = __shfl_sync(0xffffffffu, outsum[0].value(), 0);
        const double *bc = p.bconst + 2 * f;
        rw = (bc[0] + o) / bc[1];
        rhow = (T)rw;
        rwm1 = (T)((bc[0] - bc[1] + o) / bc[1]);
        if (p.implicit_wall) wall_ghost_density<T>(p, f, lane, fc.rec[0].c, fc.on, fc.nx, fc.ny, bc[1]);
    }
    // fb - M_ref is kept in the face-flux buffer for k_face_flux
    T2 *Fo = (T2 *)p.F + (size_t)f * p.Nv;
    Acc<T> acc[kRaw];
    auto body = [&](int k, T(&a)[kRaw]) {
        T ux = vx<T>(p, k), uy = vy<T>(p, k);
        T s = xi_dot_n<T>(ux, uy, fc.nx, fc.ny);
        T2 fb = face_fbar<T, LIM>(p, fc, k, ux, uy, s, rhow, rwm1);
        Fo[k] = fb;
        raw_terms<T>(a, vw<T>(p, k), ux, uy, fb.x, fb.y);
    };
    // velocity pairs: at an interior face whose two velocities are upwind
    // from the same side (no tie) one pair reconstruction; else per velocity
    auto body2 = [&](int k, T(&a)[kRaw]) {
        T ux[2], uy[2], w[2], s[2], g[2], hh[2];
        vtab2<T>(p.uxf, p.ux, k, ux);
        vtab2<T>(p.uyf, p.uy, k, uy);
        vtab2<T>(p.wf, p.w, k, w);
        s[0] = xi_dot_n<T>(ux[0], uy[0], fc.nx, fc.ny);
        s[1] = xi_dot_n<T>(ux[1], uy[1], fc.nx, fc.ny);
        const bool up0 = s[0] > (T)0, up1 = s[1] > (T)0;
        if (fc.kind < 0 && up0 == up1 && s[0] != (T)0 && s[1] != (T)0) {
            reconstruct2<T, LIM>(p, fc.rec[up0 ? 0 : 1], k, ux, uy, h, g, hh);
        } else {
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const T2 fb = face_fbar<T, LIM>(p, fc, k + v, ux[v], uy[v], s[v], rhow, rwm1);
                g[v] = fb.x;
                hh[v] = fb.y;
            }
        }
        store_pair<T>(Fo, k, g, hh);
        raw_terms<T>(a, w[0], ux[0], uy[0], g[0], hh[0]);
        raw_terms<T>(a, w[1], ux[1], uy[1], g[1], hh[1]);
    };
    if constexpr (sizeof(T) == 4) {
        __shared__ FF sacc[kRaw * 256];
        vel_loop2_sm<kRaw>(p.Nv, lane, sacc, body2);
#pragma unroll
        for (int q = 0; q < kRaw; ++q) acc[q].v = sacc[q * blockDim.x + threadIdx.x];
    } else {
#pragma unroll
        for (int q = 0; q < kRaw; ++q) acc[q].zero();
        vel_loop<kRaw, T>(p.Nv, lane, acc, body);
    }
#pragma unroll
    for (int q = 0; q < kRaw; ++q) acc[q].warp_sum();
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < kRaw; ++q) acc[q].store(p.faceraw, (size_t)f * 12 + q);
        outsum[0].store(p.faceraw, (size_t)f * 12 + 11);
        p.facerw[f] = rw;
    }
}

// per face: state from the moments of fb, tau, q = 2 tau qbar/(2 tau + h Pr),
// equilibrium, and the weights a, b of f = a fb + b f^S (Eq. 18)
template <class T>
__global__ void __launch_bounds__(32) k_face_params(Launch L)
{
    IDG_LOCATE();
    const int f = blk * blockDim.x + threadIdx.x;
    if (f >= p.nf) return;
    double r[kRaw];
    for (int q = 0; q < kRaw; ++q) r[q] = acc_load<T>(p.faceraw, (size_t)f * 12 + q) + p.mref_raw[q];
    double rho, U, V, RT, qbx, qby;
    raw_to_state(r, p.K, rho, U, V, RT, qbx, qby);
    T *fA = (T *)p.faceA + kCellP * f;
    // float32 storage keeps fb relative to the reference Maxwellian, so a
    // face that an impulsive start evacuates (density ~1e-18 of the reference
    // at the lee of a hypersonic body) is not resolved: its moments are
    // rounding noise of the reference's.  Below 1e-6 of the reference density
    // or temperature such a face takes the vacuum limit of Eq. (18):
    // tau -> infinity, f = fb (free transport), no equilibrium part.
    if (sizeof(T) == 4 && !(rho > 1e-6 * p.rho_r && RT > 1e-6 * p.RT_r)) {
        eq_storeT<T>(fA, make_eq(p, 0.0, p.U_r, p.V_r, p.RT_r, 0.0, 0.0));
        fA[14] = (T)1;
        fA[15] = (T)0;
        return;
    }
    double tau = viscosity_t<T>(p, RT) / (rho * RT);
    double Pr = p.shakhov ? p.Pr : 1.0;
    double qx = 2.0 * tau * qbx / (2.0 * tau + p.h * Pr);
    double qy = 2.0 * tau * qby / (2.0 * tau + p.h * Pr);
    eq_storeT<T>(fA, make_eq(p, rho, U, V, RT, qx, qy));
    fA[14] = (T)(2.0 * tau / (2.0 * tau + p.h));
    fA[15] = (T)(p.h / (2.0 * tau + p.h));
}

// face flux of (f_face - M_ref), Eq. (18)-(19), and its moments; fb - M_ref
// comes from k_face_moments through the same buffer and is overwritten
template <class T>
__global__ void __launch_bounds__(256) k_face_flux(Launch L)
{
    IDG_LOCATE();
    using T2 = typename V2<T>::t;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int f = blk * 8 + wid;
    if (f >= p.nf) return;  // whole warp
    const T *g = (const T *)p.fgeoT + 8 * f;
    const T nx = g[0], ny = g[1], S = g[2];
    const T *fA = (const T *)p.faceA + kCellP * f;
    const EqT<T> e = eq_loadT<T>(fA);
    const T wa = fA[14], wb = fA[15], kRTr = (T)(p.K * p.RT_r);
    T2 *Fo = (T2 *)p.F + (size_t)f * p.Nv;
    Acc<T> acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q].zero();
    vel_loop2<4, T>(p.Nv, lane, acc, [&](int k, T(&a)[4]) {
        T ux[2], uy[2], w[2], gr[2], fg[2], fh[2];
        vtab2<T>(p.uxf, p.ux, k, ux);
        vtab2<T>(p.uyf, p.uy, k, uy);
        vtab2<T>(p.wf, p.w, k, w);
        vtab2<T>(p.greff, p.gref, k, gr);
        load_pair<T>(Fo, k, fg, fh);
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            T s = xi_dot_n<T>(ux[v], uy[v], nx, ny);
            T dG, dH;
            dev_equilibrium<T>(e, ux[v], uy[v], gr[v], kRTr, dG, dH);
            T sS = s * S;
            fg[v] = sS * (wa * fg[v] + wb * dG);
            fh[v] = sS * (wa * fh[v] + wb * dH);
            T wg = w[v] * fg[v];
            a[0] += wg;
            a[1] += wg * ux[v];
            a[2] += wg * uy[v];
            a[3] += (T)0.5 * w[v] * ((ux[v] * ux[v] + uy[v] * uy[v]) * fg[v] + fh[v]);
        }
        store_pair<T>(Fo, k, fg, fh);
    });
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q].warp_sum();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q].store(p.phiraw, (size_t)f * 4 + q);
    if (p.implicit_wall && p.fbc[f] == 1) {
        // linearised wall (Eq. 33-35): the ghost increment drho_g M_w of the
        // incoming velocities enters the micro sweeps as the upwind term
        // |xi.n| S Delta_ghost, i.e. as an extra flux s S drho_g M_w on the
        // stored F (after Phi is summed: R_W and Phi exclude it)
        __syncwarp();
        const double drg = p.walldrg[f];
        if (drg != 0.0) {
            const T on = p.fL[f] >= 0 ? (T)1 : (T)-1, SD = S * (T)drg;
            const T *bG = (const T *)p.bdevG + (size_t)p.fside[f] * p.Nv;
            const T *bH = (const T *)p.bdevH + (size_t)p.fside[f] * p.Nv;
            for (int k = lane; k < p.Nv; k += 32) {
                const T sn = xi_dot_n<T>(vx<T>(p, k), vy<T>(p, k), nx, ny);
                if (on * sn < (T)0) {
                    const T a = sn * SD, gr = vgref<T>(p, k);
                    T2 v = Fo[k];
                    v.x += a * (bG[k] + gr);
                    v.y += a * (bH[k] + kRTr * gr);
                    Fo[k] = v;
                }
            }
        }
    }
}

// Phi_f = sum_k w psi F_k (Eq. 27): deviation part plus the flux of M_ref;
// the mass flux through an impermeable wall is exactly zero
template <class T>
__global__ void __launch_bounds__(256) k_face_phi(Launch L)
{
    IDG_LOCATE();
    const int f = blk * blockDim.x + threadIdx.x;
    if (f >= p.nf) return;
    const double *g = p.fgeo + 7 * f;
    for (int q = 0; q < 4; ++q)
        p.phi[4 * f + q] = acc_load<T>(p.phiraw, (size_t)f * 4 + q) +
                           g[2] * (g[0] * p.mref_flux[q][0] + g[1] * p.mref_flux[q][1]);
    if (p.fbc[f] == 1) p.phi[4 * f] = 0.0;
    // the wall sums of this iteration are stored: the next one has a last increment
    if (f == 0 && p.implicit_wall) *p.wallok = 1;
}

// ---------------------------------------------------------------------------
// macroscopic predictor (Eq. 27-31)                                     [a5]
//   k_macro_pre    (all cells, many CTAs): residual R_W = -sum Phi, partial
//                  norms, spectral radii (Eq. 31 at the face average), the
//                  LU-SGS diagonal D (Eq. 30) and per-neighbour coefficients
//   k_macro_sweep  (one CTA): forward and backward sweeps on i+j hyperplanes,
//                  the lexicographic dependency order, with the matrix-free
//                  off-diagonal term 1/2 (dF S - omega Lambda dW) of Eq. (30)
//   k_macro_post   (all cells): W^{n+1} = W + dW (Eq. 32) in float64 and the
//                  micro coefficients at the predicted state
// ---------------------------------------------------------------------------
__device__ __forceinline__ void prim_uvc(const KParams &p, const double *W, double &u, double &v,
                                         double &cs)
{
    double rho = W[0];
    u = W[1] / rho;
    v = W[2] / rho;
    double RT = (2.0 * W[3] / rho - u * u - v * v) / (p.K + 2);
    cs = sqrt(p.gam * RT);
}

__device__ __forceinline__ double face_lambda(const KParams &p, int fi)
{
    int L = p.fL[fi], R = p.fR[fi];
    const double *g = p.fgeo + 7 * fi;
    double u, v, cs;
    if (L >= 0 && R >= 0) {
        double u1, v1, c1, u2, v2, c2;
        prim_uvc(p, p.W + 4 * L, u1, v1, c1);
        prim_uvc(p, p.W + 4 * R, u2, v2, c2);
        u = 0.5 * (u1 + u2); v = 0.5 * (v1 + v2); cs = 0.5 * (c1 + c2);
    } else {
        prim_uvc(p, p.W + 4 * (L >= 0 ? L : R), u, v, cs);
    }
    return (fabs(u * g[0] + v * g[1]) + cs) * g[2];
}

// Preconditioner coefficients of the macroscopic LU-SGS: in float32 storage
// the spectral radius and the neighbours' base states only enter the float32
// wavefront (R_W, the diagonal's sum and W^{n+1} stay float64), so they are
// evaluated in float32; float64 storage evaluates them in float64.
template <class T> __device__ __forceinline__ double face_lambda_t(const KParams &p, int fi);
template <> __device__ __forceinline__ double face_lambda_t<double>(const KParams &p, int fi)
{
    return face_lambda(p, fi);
}
template <> __device__ __forceinline__ double face_lambda_t<float>(const KParams &p, int fi)
{
    const int L = p.fL[fi], R = p.fR[fi];
    const double *g = p.fgeo + 7 * fi;
    const float gam = (float)p.gam, k2 = 1.0f / (float)(p.K + 2);
    float u = 0.f, v = 0.f, cs = 0.f;
    int nc = 0;
    for (int side = 0; side < 2; ++side) {
        const int c = side ? R : L;
        if (c < 0) continue;
        const double *W = p.W + 4 * c;
        const float rho = (float)W[0], ir = 1.0f / rho, uc = (float)W[1] * ir, vc = (float)W[2] * ir;
        const float RT = (2.0f * (float)W[3] * ir - uc * uc - vc * vc) * k2;
        u += uc; v += vc; cs += sqrtf(gam * RT);
        ++nc;
    }
    if (nc == 2) { u *= 0.5f; v *= 0.5f; cs *= 0.5f; }
    return (double)((fabsf(u * (float)g[0] + v * (float)g[1]) + cs) * (float)g[2]);
}

// base state (rho, m_x, m_y, u, v, E + p) of a neighbour for the flux increments
template <class T> __device__ __forceinline__ void base_state(const KParams &p, const double *W, T *o);
template <> __device__ __forceinline__ void base_state<double>(const KParams &p, const double *W, double *o)
{
    double rho = W[0], u = W[1] / rho, v = W[2] / rho;
    double pr = (p.gam - 1.0) * (W[3] - 0.5 * rho * (u * u + v * v));
    o[0] = rho; o[1] = W[1]; o[2] = W[2];
    o[3] = u; o[4] = v; o[5] = W[3] + pr;
}
template <> __device__ __forceinline__ void base_state<float>(const KParams &p, const double *W, float *o)
{
    const float rho = (float)W[0], mx = (float)W[1], my = (float)W[2], E = (float)W[3];
    const float ir = 1.0f / rho, u = mx * ir, v = my * ir;
    const float pr = (float)(p.gam - 1.0) * (E - 0.5f * rho * (u * u + v * v));
    o[0] = rho; o[1] = mx; o[2] = my;
    o[3] = u; o[4] = v; o[5] = E + pr;
}

// cp.async helpers: asynchronous global -> shared copies used to prefetch
// the next hyperplanes of a wavefront while the current one is computed
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(void *s, const void *g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async8(void *s, const void *g)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async4(void *s, const void *g)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
template <int B> __device__ __forceinline__ void cp_async_b(void *s, const void *g);
template <> __device__ __forceinline__ void cp_async_b<4>(void *s, const void *g) { cp_async4(s, g); }
template <> __device__ __forceinline__ void cp_async_b<8>(void *s, const void *g) { cp_async8(s, g); }
template <> __device__ __forceinline__ void cp_async_b<16>(void *s, const void *g) { cp_async16(s, g); }
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

constexpr int kMRec = 24;  // macroscopic sweep record: R[4], 1/D, pad, own base[6], 4 x (n S/2 [2], omega Lambda/2)
constexpr int kMRing = 12; // ring entry per cell: increment[4], base state[6], pad[2]

// per cell: R_W, ||R_W/Omega||^2 partials, and the record of the macroscopic
// sweep (inverse diagonal, the cell's own base state for its neighbours'
// flux increments, per-slot face coefficients)
template <class T>
__global__ void __launch_bounds__(32) k_macro_pre(Launch L)
{
    IDG_LOCATE();
    __shared__ double sm[32];
    const int c = blk * blockDim.x + threadIdx.x;
    double part[1] = {0.0};
    if (c < p.N) {
        T *rec = (T *)p.mrec + (size_t)kMRec * c;
        double acc[4] = {0, 0, 0, 0};
        for (int m = 0; m < 4; ++m) {
            double s = p.csign[4 * c + m];
            const double *ph = p.phi + 4 * p.cface[4 * c + m];
            for (int q = 0; q < 4; ++q) acc[q] -= s * ph[q];
        }
        for (int q = 0; q < 4; ++q) {
            p.rw[4 * c + q] = acc[q];
            rec[q] = (T)acc[q];
            double rr = acc[q] / p.area[c];
            part[0] += rr * rr;
        }
        double d = p.area[c] / p.dtimp[c];
        for (int m = 0; m < 4; ++m) {
            int fi = p.cface[4 * c + m];
            double lam = face_lambda_t<T>(p, fi);
            double s = p.csign[4 * c + m];  // 0: a triangle's unused slot
            if (s != 0.0 && p.fL[fi] != p.fR[fi]) d += 0.5 * p.lusgs_omega * lam;
            const double *g = p.fgeo + 7 * fi;
            T *o = rec + 12 + 3 * m;
            o[0] = (T)(0.5 * g[2] * s * g[0]);
            o[1] = (T)(0.5 * g[2] * s * g[1]);
            o[2] = (T)(0.5 * p.lusgs_omega * lam);
        }
        rec[4] = (T)(1.0 / d);
        rec[5] = (T)0;
        base_state<T>(p, p.W + 4 * c, rec + 6);
    }
    block_sum<1>(part, sm);
    if (threadIdx.x == 0) p.mpart[blk] = part[0];
}

// ||R_W/Omega||_2 of this iteration from k_macro_pre's partials (fixed
// order) into the residual ring; a non-finite value raises the status word
__device__ __forceinline__ void record_residual(const KParams &p)
{
    double s = 0.0;
    const int nb = (p.N + 31) / 32;
    for (int q = 0; q < nb; ++q) s += p.mpart[q];
    const int it = *p.iter;
    const double r = sqrt(s);
    p.res[it & (kMaxHist - 1)] = r;
    if (!isfinite(r)) *p.status = 5;
}

// Exact increment F_n(W + dW) - F_n(W) of the Euler flux, written so that no
// two O(1) quantities are subtracted (every term is an increment times a
// base quantity); n is pre-scaled by S/2.  b = rho, m_x, m_y, u, v, E+p.
template <class T>
__device__ __forceinline__ void euler_dflux(T gm1, const T *b, const T *dW, T nx, T ny, T *dF)
{
    T rho = b[0], mx = b[1], my = b[2], u = b[3], v = b[4], H = b[5];
    T ir1 = rcp_rn(rho + dW[0]);
    T du = (dW[1] - u * dW[0]) * ir1, dv = (dW[2] - v * dW[0]) * ir1;
    T vn = u * nx + v * ny, dvn = du * nx + dv * ny, vn1 = vn + dvn;
    T dmu = dW[1] * (u + du) + dW[2] * (v + dv) + mx * du + my * dv;
    T dp = gm1 * (dW[3] - (T)0.5 * dmu);
    dF[0] = dW[0] * vn1 + rho * dvn;
    dF[1] = dW[1] * vn1 + mx * dvn + dp * nx;
    dF[2] = dW[2] * vn1 + my * dvn + dp * ny;
    dF[3] = (dW[3] + dp) * vn1 + H * dvn;
}

// One CTA: forward then backward sweep over the i+j hyperplanes (the
// lexicographic dependency order).  Two threads own one cell of the
// hyperplane: thread h handles the slot pair (west, east) for h = 0 and
// (south, north) for h = 1 -- of each pair at most one neighbour is on the
// already-swept side away from a periodic seam, so each thread usually
// evaluates one flux increment 1/2 (dF S - omega Lambda dW_nb).  The two
// partial sums meet in one pair shuffle and thread h writes components 2h and
// 2h+1 of the increment.  Neighbours are found from the cell's (i, j) and the
// periodic flags.  Records and (backward) the cell's own dW* are prefetched
// kStages-1 hyperplanes ahead with cp.async; the previous hyperplane's
// increments and base states sit in a shared-memory ring indexed by the slot
// in the hyperplane; neighbours across a periodic seam (earlier hyperplanes)
// come from global memory.
template <class T, int kStages>
__global__ void __launch_bounds__(512) k_macro_sweep(Launch L)
{
    IDG_LOCATE();
    extern __shared__ __align__(16) unsigned char smraw[];
    const int tid = threadIdx.x, ncs = blockDim.x >> 1;  // cell slots
    const int cs = tid >> 1, h = tid & 1;
    const int ni = p.ni, nj = p.nj, nh = ni + nj - 1;
    const bool per_i = p.per_i, per_j = p.per_j;
    T *srec = (T *)smraw;                               // [kStages][ncs][kMRec]
    T *sdw = srec + (size_t)kStages * ncs * kMRec;      // [kStages][ncs][4] own dW* (backward)
    T *ring = sdw + (size_t)kStages * ncs * 4;          // [2][ncs][kMRing]
    if (tid == 0) record_residual(p);
    const T gm1 = (T)(p.gam - 1.0);
    T *dWg = (T *)p.mdW;
    const T *mrec = (const T *)p.mrec;
    constexpr int RC = kMRec * sizeof(T) / 16;  // 16-byte chunks of one record
    constexpr int DC = 4 * sizeof(T) / 16;      // chunks of one dW
    for (int dir = 1; dir >= -1; dir -= 2) {
        auto step_d = [&](int s) { return dir > 0 ? s : nh - 1 - s; };
        auto issue = [&](int s) {
            if (s < nh) {
                const int d = step_d(s);
                const int i = max(0, d - (nj - 1)) + cs;
                if (i <= min(ni - 1, d)) {
                    const int c = (d - i) * ni + i;
                    const size_t e = (size_t)(s & (kStages - 1)) * ncs + cs;
                    const int nch = RC + (dir < 0 ? DC : 0);
                    for (int q = h; q < nch; q += 2) {
                        if (q < RC) cp_async16((char *)(srec + e * kMRec) + 16 * q, (const char *)(mrec + (size_t)kMRec * c) + 16 * q);
                        else cp_async16((char *)(sdw + e * 4) + 16 * (q - RC), (const char *)(dWg + 4 * (size_t)c) + 16 * (q - RC));
                    }
                }
            }
            cp_commit();
        };
        for (int s = 0; s < kStages - 1; ++s) issue(s);
        for (int s = 0; s < nh; ++s) {
            cp_wait<kStages - 2>();
            __syncthreads();
            issue(s + kStages - 1);
            const int d = step_d(s);
            const int ilo = max(0, d - (nj - 1)), ihi = min(ni - 1, d);
            const int i = ilo + cs, j = d - i;
            const bool valid = i <= ihi;
            const int c = j * ni + i;
            const size_t e = (size_t)(s & (kStages - 1)) * ncs + cs;
            const T *rec = srec + e * kMRec;
            T acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
            if (valid) {
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    // slot m = 2h + u: west, east (h = 0); south, north (h = 1)
                    const int m = 2 * h + u;
                    int nbi = i, nbj = j;
                    bool ex = true;
                    if (h == 0) {
                        nbi = u ? i + 1 : i - 1;
                        if (u ? i == ni - 1 : i == 0) { ex = per_i; nbi = u ? 0 : ni - 1; }
                    } else {
                        nbj = u ? j + 1 : j - 1;
                        if (u ? j == nj - 1 : j == 0) { ex = per_j; nbj = u ? 0 : nj - 1; }
                    }
                    const int nb = nbj * ni + nbi;
                    if (!ex || !(dir > 0 ? nb < c : nb > c)) continue;
                    T dn[4];
                    const T *base;
                    if (nbi + nbj == d - dir) {
                        const int ts = nbi - max(0, d - dir - (nj - 1));
                        const T *x = ring + ((size_t)((s + 1) & 1) * ncs + ts) * kMRing;
                        dn[0] = x[0]; dn[1] = x[1]; dn[2] = x[2]; dn[3] = x[3];
                        base = x + 4;
                    } else {
                        const T *x = dWg + 4 * (size_t)nb;
                        dn[0] = x[0]; dn[1] = x[1]; dn[2] = x[2]; dn[3] = x[3];
                        base = mrec + (size_t)kMRec * nb + 6;
                    }
                    const T *cf = rec + 12 + 3 * m;
                    T dF[4];
                    euler_dflux<T>(gm1, base, dn, cf[0], cf[1], dF);
                    acc0 += dF[0] - cf[2] * dn[0];
                    acc1 += dF[1] - cf[2] * dn[1];
                    acc2 += dF[2] - cf[2] * dn[2];
                    acc3 += dF[3] - cf[2] * dn[3];
                }
            }
            // sum over the two slot pairs of the cell
            acc0 += __shfl_xor_sync(0xffffffffu, acc0, 1);
            acc1 += __shfl_xor_sync(0xffffffffu, acc1, 1);
            acc2 += __shfl_xor_sync(0xffffffffu, acc2, 1);
            acc3 += __shfl_xor_sync(0xffffffffu, acc3, 1);
            if (valid) {
                // forward: dW*_c = (R_c - sum_lower) / D_c;  backward: dW_c = dW*_c - sum_upper / D_c
                const T iD = rec[4];
                const T a0 = h ? acc2 : acc0, a1 = h ? acc3 : acc1;
                const int q0 = 2 * h;
                T x0, x1;
                if (dir > 0) {
                    x0 = (rec[q0] - a0) * iD;
                    x1 = (rec[q0 + 1] - a1) * iD;
                } else {
                    x0 = sdw[e * 4 + q0] - a0 * iD;
                    x1 = sdw[e * 4 + q0 + 1] - a1 * iD;
                }
                T *r = ring + ((size_t)(s & 1) * ncs + cs) * kMRing;
                r[q0] = x0;
                r[q0 + 1] = x1;
                r[4 + 3 * h] = rec[6 + 3 * h];
                r[5 + 3 * h] = rec[7 + 3 * h];
                r[6 + 3 * h] = rec[8 + 3 * h];
                dWg[4 * (size_t)c + q0] = x0;
                dWg[4 * (size_t)c + q0 + 1] = x1;
            }
        }
        cp_wait<0>();
        __syncthreads();
    }
    if (tid == 0) *p.iter += 1;
}

// The same sweeps with one thread per line of cells.  The lines run along
// the longer axis (w), one thread per line of the shorter axis (t: columns,
// t = i, when ni <= nj, else rows, t = j), so at step d thread t owns cell
// (t, w = d - t) of the i+j hyperplane d -- the lexicographic dependency order
// as above.  Of a cell's lower neighbours (forward; upper ones backward) the
// one on the same line is the thread's own result of the previous step, kept
// in registers; the one on the adjacent line is the neighbouring lane's result
// of the previous step, taken by a warp shuffle (across a warp boundary from a
// two-slot shared-memory exchange behind the step's barrier).  Across a
// periodic seam along the lines the neighbour is the thread's own first cell
// (registers); across a seam between the last and the first line it is kept
// in shared memory by the line that computed it.  Each thread prefetches its
// cell records (and, backward, its dW*) kStages-1 steps ahead with cp.async
// into its own stage slots.  One thread owns all four components of its
// cell: no pair shuffle, no hyperplane ring.
constexpr int kLRec = kMRec + 4;  // stage entry: the record, then dW* (backward)

template <class T> struct LineNb {
    T dw[4], b[6];
};

template <class T> static size_t macro_lines_smem_bytes(int nlines, int stages, int nw, bool seam)
{
    return ((size_t)stages * nlines * kLRec + 2 * 32 * 12 + (seam ? (size_t)nw * 10 : 0)) * sizeof(T);
}

// what every step of k_macro_lines reads that does not change
template <class T> struct LineCtx {
    T *stage, *xb, *seam, *dWg;
    const T *mrec;
    T gm1;
    int ni, nt, nw, nh, nthr, t, lane, wid, nwarp, s_tm, s_tp, s_wm, s_wp;
    bool cols, line, per_t, per_w;
    __device__ __forceinline__ int cell_of(int w) const { return cols ? w * ni + t : t * ni + w; }
};

// 16-byte cp.async that copies nothing and zero-fills its destination when
// !valid (the source must still be a valid address)
__device__ __forceinline__ void cp_async16_zfill(void *s, const void *g, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(s)), "l"(g), "r"(valid ? 16 : 0)
                 : "memory");
}

// the record's first 12 entries (R[4], 1/D, pad, base state[6]) by 16-byte
// shared-memory loads (the stage slots are 16-byte aligned)
__device__ __forceinline__ void ld_rec12(const float *rec, float (&o)[12])
{
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float4 v = reinterpret_cast<const float4 *>(rec)[q];
        o[4 * q] = v.x, o[4 * q + 1] = v.y, o[4 * q + 2] = v.z, o[4 * q + 3] = v.w;
    }
}
__device__ __forceinline__ void ld_rec12(const double *rec, double (&o)[12])
{
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const double2 v = reinterpret_cast<const double2 *>(rec)[q];
        o[2 * q] = v.x, o[2 * q + 1] = v.y;
    }
}


// acc += 1/2 (dF S - omega Lambda dW_nb) of one neighbour through the slot
// whose coefficients start at cf (euler_dflux with rcp_line)
template <class T>
__device__ __forceinline__ void line_term2(T gm1, const T *cf, const LineNb<T> &nb, T (&acc)[4])
{
    const T nx = cf[0], ny = cf[1], ol = cf[2];
    const T *b = nb.b, *dW = nb.dw;
    T rho = b[0], mx = b[1], my = b[2], u = b[3], v = b[4], H = b[5];
    T ir1 = rcp_line(rho + dW[0]);
    T du = (dW[1] - u * dW[0]) * ir1, dv = (dW[2] - v * dW[0]) * ir1;
    T vn = u * nx + v * ny, dvn = du * nx + dv * ny, vn1 = vn + dvn;
    T dmu = dW[1] * (u + du) + dW[2] * (v + dv) + mx * du + my * dv;
    T dp = gm1 * (dW[3] - (T)0.5 * dmu);
    acc[0] += dW[0] * vn1 + rho * dvn - ol * dW[0];
    acc[1] += dW[1] * vn1 + mx * dvn + dp * nx - ol * dW[1];
    acc[2] += dW[2] * vn1 + my * dvn + dp * ny - ol * dW[2];
    acc[3] += (dW[3] + dp) * vn1 + H * dvn - ol * dW[3];
}

// one direction of k_macro_lines (the direction a template parameter: one
// shuffle direction, one set of slots; SEAM: the block has a periodic seam).
// The step is written without branches on the common path so that the
// compiler can interleave the prefetch, the record loads and the stores with
// the dependent flux arithmetic: every thread issues its copies each step
// (zero-filling the slot where its line has no cell at that step), evaluates
// the step on whatever the slot holds, and keeps the result only where the
// line has a cell.  A neighbour that does not exist enters with a zero
// increment on a unit-density base state: its flux increment is exactly
// zero, so no term needs a branch.
template <class T, int kStages, bool FWD, bool SEAM> __device__ __forceinline__ void line_sweep(const LineCtx<T> &x)
{
    constexpr int RC = kMRec * sizeof(T) / 16, DC = 4 * sizeof(T) / 16;
    auto step_d = [&](int s) { return FWD ? s : x.nh - 1 - s; };
    auto issue = [&](int s) {
        const int w = step_d(s) - x.t;
        const bool valid = s < x.nh && x.line && (unsigned)w < (unsigned)x.nw;
        const int c = valid ? x.cell_of(w) : 0;
        T *dst = x.stage + ((size_t)(s & (kStages - 1)) * x.nthr + x.t) * kLRec;
#pragma unroll
        for (int q = 0; q < RC; ++q)
            cp_async16_zfill((char *)dst + 16 * q, (const char *)(x.mrec + (size_t)kMRec * c) + 16 * q, valid);
        if (!FWD)
#pragma unroll
            for (int q = 0; q < DC; ++q)
                cp_async16_zfill((char *)(dst + kMRec) + 16 * q, (const char *)(x.dWg + 4 * (size_t)c) + 16 * q, valid);
        cp_commit();
    };
    for (int s = 0; s < kStages - 1; ++s) issue(s);
    LineNb<T> prev, first;  // this line's result of the previous step / of its first cell
#pragma unroll
    for (int q = 0; q < 4; ++q) prev.dw[q] = first.dw[q] = (T)0;
#pragma unroll
    for (int q = 0; q < 6; ++q) prev.b[q] = first.b[q] = q == 0 ? (T)1 : (T)0;
    const int s_adj = FWD ? x.s_tm : x.s_tp, s_own = FWD ? x.s_wm : x.s_wp;
    const int s_seam_t = FWD ? x.s_tp : x.s_tm, s_seam_w = FWD ? x.s_wp : x.s_wm;
    const bool has_adj = FWD ? x.t >= 1 : x.t + 1 < x.nt;
    const bool seam_t_reader = SEAM && x.per_t && x.t == (FWD ? x.nt - 1 : 0);
    const bool seam_t_writer = SEAM && x.per_t && x.t == (FWD ? 0 : x.nt - 1);
    const bool edge_reader = FWD ? (x.lane == 0 && x.wid > 0) : (x.lane == 31 && x.wid + 1 < x.nwarp);
    const bool edge_writer = FWD ? x.lane == 31 : x.lane == 0;
    // the exchange entry this thread may read (a valid one for every thread)
    const int edge_src = edge_reader ? (FWD ? x.wid - 1 : x.wid + 1) : 0;
    for (int s = 0; s < x.nh; ++s) {
        cp_wait<kStages - 2>();
        __syncthreads();  // the step's records and the exchange entries of the previous step are written
        issue(s + kStages - 1);
        const int w = step_d(s) - x.t;
        const bool on = x.line && (unsigned)w < (unsigned)x.nw;
        const T *rec = x.stage + ((size_t)(s & (kStages - 1)) * x.nthr + x.t) * kLRec;
        T r12[12];
        ld_rec12(rec, r12);
        // the adjacent line's result of the previous step, at this thread's w
        T ev[12];
        ld_rec12(x.xb + ((size_t)((s + 1) & 1) * 32 + edge_src) * 12, ev);
        LineNb<T> adj;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const T sh = FWD ? __shfl_up_sync(0xffffffffu, prev.dw[q], 1) : __shfl_down_sync(0xffffffffu, prev.dw[q], 1);
            adj.dw[q] = has_adj ? (edge_reader ? ev[q] : sh) : (T)0;
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const T sh = FWD ? __shfl_up_sync(0xffffffffu, prev.b[q], 1) : __shfl_down_sync(0xffffffffu, prev.b[q], 1);
            adj.b[q] = edge_reader ? ev[4 + q] : sh;
        }
        T acc[4] = {0, 0, 0, 0};
        line_term2<T>(x.gm1, rec + 12 + 3 * s_adj, adj, acc);
        // prev is the zero-increment initial state at the line's first cell
        line_term2<T>(x.gm1, rec + 12 + 3 * s_own, prev, acc);
        if (SEAM && on) {
            if (seam_t_reader) {
                LineNb<T> sn;
                const T *e = x.seam + (size_t)w * 10;
#pragma unroll
                for (int q = 0; q < 4; ++q) sn.dw[q] = e[q];
#pragma unroll
                for (int q = 0; q < 6; ++q) sn.b[q] = e[4 + q];
                line_term2<T>(x.gm1, rec + 12 + 3 * s_seam_t, sn, acc);
            }
            if (x.per_w && w == (FWD ? x.nw - 1 : 0)) line_term2<T>(x.gm1, rec + 12 + 3 * s_seam_w, first, acc);
        }
        // forward: dW*_c = (R_c - sum_lower) / D_c;  backward: dW_c = dW*_c - sum_upper / D_c
        const T iD = r12[4];
        LineNb<T> out;
        if (FWD) {
#pragma unroll
            for (int q = 0; q < 4; ++q) out.dw[q] = (r12[q] - acc[q]) * iD;
        } else {
            T ds[4];
            if (sizeof(T) == 4) {
                const float4 v = *reinterpret_cast<const float4 *>(rec + kMRec);
                ds[0] = v.x, ds[1] = v.y, ds[2] = v.z, ds[3] = v.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) ds[q] = rec[kMRec + q];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) out.dw[q] = ds[q] - acc[q] * iD;
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) out.b[q] = r12[6 + q];
#pragma unroll
        for (int q = 0; q < 4; ++q) prev.dw[q] = on ? out.dw[q] : prev.dw[q];
#pragma unroll
        for (int q = 0; q < 6; ++q) prev.b[q] = on ? out.b[q] : prev.b[q];
        if (on) {
            T *g = x.dWg + 4 * (size_t)x.cell_of(w);
            if (sizeof(T) == 4) {
                *reinterpret_cast<float4 *>(g) = make_float4(out.dw[0], out.dw[1], out.dw[2], out.dw[3]);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) g[q] = out.dw[q];
            }
        }
        if (SEAM && on) {
            // the cell a later cell of this line meets across the seam along the line
            if (x.per_w && w == (FWD ? 0 : x.nw - 1)) first = out;
            // the seam line's cells for the line across the seam between lines
            if (seam_t_writer) {
                T *e = x.seam + (size_t)w * 10;
#pragma unroll
                for (int q = 0; q < 4; ++q) e[q] = out.dw[q];
#pragma unroll
                for (int q = 0; q < 6; ++q) e[4 + q] = out.b[q];
            }
        }
        // the warp-boundary lane's result for the next warp's edge lane
        // (its line's current state; a line without a cell leaves it as it was)
        if (edge_writer) {
            T *e = x.xb + ((size_t)(s & 1) * 32 + x.wid) * 12;
#pragma unroll
            for (int q = 0; q < 4; ++q) e[q] = prev.dw[q];
#pragma unroll
            for (int q = 0; q < 6; ++q) e[4 + q] = prev.b[q];
        }
    }
    cp_wait<0>();
    __syncthreads();
}

template <class T, int kStages, bool SEAM>
__global__ void __launch_bounds__(256, 1) k_macro_lines(Launch L)
{
    IDG_LOCATE();
    (void)blk;
    extern __shared__ __align__(16) unsigned char smraw[];
    LineCtx<T> x;
    x.ni = p.ni;
    x.cols = p.ni <= p.nj;
    x.nt = x.cols ? p.ni : p.nj;
    x.nw = x.cols ? p.nj : p.ni;
    x.nh = x.nt + x.nw - 1;
    x.nthr = blockDim.x;
    x.t = threadIdx.x;
    x.lane = x.t & 31;
    x.wid = x.t >> 5;
    x.nwarp = blockDim.x >> 5;
    x.line = x.t < x.nt;
    // periodic between the last and the first line / along the lines; a
    // direction one cell wide wraps onto the cell itself (no term)
    x.per_t = (x.cols ? p.per_i : p.per_j) && x.nt > 1;
    x.per_w = (x.cols ? p.per_j : p.per_i) && x.nw > 1;
    // slots (west 0, east 1, south 2, north 3) towards line t-1 / t+1 and
    // towards w-1 / w+1
    x.s_tm = x.cols ? 0 : 2;
    x.s_tp = x.cols ? 1 : 3;
    x.s_wm = x.cols ? 2 : 0;
    x.s_wp = x.cols ? 3 : 1;
    x.stage = (T *)smraw;                                     // [kStages][nthr][kLRec]
    x.xb = x.stage + (size_t)kStages * x.nthr * kLRec;        // [2][32 warps][12] warp-boundary exchange
    x.seam = x.xb + 2 * 32 * 12;                              // [nw][10] the seam line's cells (per_t)
    x.dWg = (T *)p.mdW;
    x.mrec = (const T *)p.mrec;
    x.gm1 = (T)(p.gam - 1.0);
    // exchange entries never written read as benign neighbours (zero
    // increment, unit density)
    for (int q = x.t; q < 2 * 32 * 12; q += x.nthr) x.xb[q] = (q % 12 == 4) ? (T)1 : (T)0;
    if (x.t == 0) record_residual(p);
    __syncthreads();
    line_sweep<T, kStages, true, SEAM>(x);
    line_sweep<T, kStages, false, SEAM>(x);
    if (x.t == 0) *p.iter += 1;
}

// The macroscopic LU-SGS sweeps on an unstructured mesh: one CTA walks the
// steps of the forward, then the backward schedule (the lower- and
// upper-neighbour levels of the cell numbering), a thread per cell of a step
// (a step holds at most blockDim.x cells); the same equations and cell order
// as k_macro_sweep.  Everything of a step that the sweep does not change --
// the cell, its neighbours, its record, their base states -- is loaded into
// registers before the barrier that opens the step, so after it only the
// neighbours' increments are read.  SMEM: the increments of all cells live in
// shared memory for the two sweeps and go to global memory at the end;
// otherwise they are read from global memory.
template <class T> struct MacroCell {
    int c, nb[4];
    T r[4], iD, cf[12], base[4][6];
};

template <class T>
__device__ __forceinline__ void macro_cell_load(const KParams &p, const int *sc, const int *sp, int st, int ns,
                                                int dir, MacroCell<T> &x)
{
    x.c = -1;
    if (st >= ns || (int)threadIdx.x >= sp[st + 1] - sp[st]) return;
    const int c = sc[sp[st] + threadIdx.x];
    const T *mrec = (const T *)p.mrec;
    const T *rec = mrec + (size_t)kMRec * c;
    x.c = c;
#pragma unroll
    for (int q = 0; q < 4; ++q) x.r[q] = rec[q];
    x.iD = rec[4];
#pragma unroll
    for (int q = 0; q < 12; ++q) x.cf[q] = rec[12 + q];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        int nb = p.cnb[4 * c + m];
        if (nb < 0 || nb == c || !(dir > 0 ? nb < c : nb > c)) nb = -1;
        x.nb[m] = nb;
        if (nb >= 0)
#pragma unroll
            for (int q = 0; q < 6; ++q) x.base[m][q] = mrec[(size_t)kMRec * nb + 6 + q];
    }
}

template <class T, bool SMEM>
__global__ void __launch_bounds__(256) k_macro_sweep_sched(Launch L)
{
    IDG_LOCATE();
    (void)blk;
    extern __shared__ __align__(16) unsigned char smraw[];
    if (threadIdx.x == 0) record_residual(p);
    const T gm1 = (T)(p.gam - 1.0);
    T *dWg = (T *)p.mdW;
    T *dw = SMEM ? (T *)smraw : dWg;  // [N][4]
    for (int dir = 1; dir >= -1; dir -= 2) {
        const int *sc = p.sched + (dir > 0 ? 0 : (size_t)p.N);
        const int *sp = p.sptr + (dir > 0 ? 0 : p.nsteps_f + 1);
        const int ns = dir > 0 ? p.nsteps_f : p.nsteps_b;
        MacroCell<T> cur;
        macro_cell_load<T>(p, sc, sp, 0, ns, dir, cur);
        for (int st = 0; st < ns; ++st) {
            MacroCell<T> nxt;
            macro_cell_load<T>(p, sc, sp, st + 1, ns, dir, nxt);
            __syncthreads();
            if (cur.c >= 0) {
                T acc[4] = {0, 0, 0, 0};
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    if (cur.nb[m] < 0) continue;
                    const T *x4 = dw + 4 * (size_t)cur.nb[m];
                    const T dn[4] = {x4[0], x4[1], x4[2], x4[3]};
                    T dF[4];
                    euler_dflux<T>(gm1, cur.base[m], dn, cur.cf[3 * m], cur.cf[3 * m + 1], dF);
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[q] += dF[q] - cur.cf[3 * m + 2] * dn[q];
                }
                // forward: dW*_c = (R_c - sum_lower) / D_c;  backward: dW_c = dW*_c - sum_upper / D_c
                T *o = dw + 4 * (size_t)cur.c;
#pragma unroll
                for (int q = 0; q < 4; ++q) o[q] = dir > 0 ? (cur.r[q] - acc[q]) * cur.iD : o[q] - acc[q] * cur.iD;
            }
            cur = nxt;
        }
        __syncthreads();
    }
    if (SMEM)
        for (int q = threadIdx.x; q < 4 * p.N; q += blockDim.x) dWg[q] = dw[q];
    if (threadIdx.x == 0) *p.iter += 1;
}

template <class T>
__global__ void __launch_bounds__(32) k_macro_post(Launch L)
{
    IDG_LOCATE();
    const int c = blk * blockDim.x + threadIdx.x;
    if (c >= p.N) return;
    double *W = p.W + 4 * c;
    const T *dW = (const T *)p.mdW + 4 * c;
    for (int q = 0; q < 4; ++q) W[q] += (double)dW[q];
    double rho = W[0], U = W[1] / rho, V = W[2] / rho;
    double RT = (2.0 * W[3] / rho - U * U - V * V) / (p.K + 2);
    double taup = viscosity_t<T>(p, RT) / (rho * RT);
    EqD e = make_eq(p, rho, U, V, RT, p.cellq[2 * c], p.cellq[2 * c + 1]);
    double *cp = p.cellp + kCellP * c;
    eq_store(cp, e);
    double cq = 2.0 * p.area[c] / (2.0 * taup + p.dt);
    cp[14] = cq;
    cp[15] = p.area[c] / p.dtimp[c] + cq;
    T *ct = (T *)p.cellpT + kCellP * c;
    for (int q = 0; q < kCellP; ++q) ct[q] = (T)cp[q];
}

// Point relaxation of the predictor equations (the alternative to LU-SGS the
// conclusions name): D dW_c + sum_nb 1/2 (dF_nb S - omega Lambda dW_nb) = R_c
// solved by Jacobi sweeps from dW = 0, every cell at once from the previous
// sweep's increments of all its neighbours -- no wavefront, every SM busy.
// Sweep k of n (1-based) writes mdW when n - k is even, mdW2 when odd, so the
// last one leaves dW in mdW for k_macro_post; sweep 1 gives dW = R / D.  The
// record of k_macro_pre holds R, 1/D, the cell's base state and per slot
// (S/2) n_out and (omega/2) Lambda, as for the sweeps.
template <class T>
__global__ void __launch_bounds__(32) k_macro_relax(Launch L, int sweep, int nsweeps)
{
    IDG_LOCATE();
    const int c = blk * blockDim.x + threadIdx.x;
    if (c >= p.N) return;
    const bool odd = (nsweeps - sweep) & 1;
    T *dst = (T *)(odd ? p.mdW2 : p.mdW);
    const T *src = (const T *)(odd ? p.mdW : p.mdW2);
    const T *mrec = (const T *)p.mrec;
    const T *rec = mrec + (size_t)kMRec * c;
    const T gm1 = (T)(p.gam - 1.0);
    T acc[4] = {0, 0, 0, 0};
    if (sweep > 1) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int nb = p.cnb[4 * c + m];
            if (nb < 0 || nb == c) continue;  // ghost, or a cell wrapped onto itself
            const T *x = src + 4 * (size_t)nb;
            const T dn[4] = {x[0], x[1], x[2], x[3]};
            const T *cf = rec + 12 + 3 * m;
            T dF[4];
            euler_dflux<T>(gm1, mrec + (size_t)kMRec * nb + 6, dn, cf[0], cf[1], dF);
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += dF[q] - cf[2] * dn[q];
        }
    }
    const T iD = rec[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[4 * (size_t)c + q] = (rec[q] - acc[q]) * iD;
}

// ---------------------------------------------------------------------------
// explicit DUGKS (Eq. 10, 21): the cell and face kernels of the implicit
// iteration build the face fluxes with the physical step dt, then
//   k_explicit_update  per (cell, velocity):
//                      f~ <- (2tau-dt)/(2tau+dt) f~ + 2dt/(2tau+dt) f^S - dt/Omega sum F
//   k_cell_moments, k_explicit_w: W = moments of the new f~ (the collision
//                      conserves them, so f~ and f share them), which the
//                      next step's cell prep reads, and partial sums of
//                      ||(W^{n+1} - W^n)/dt||^2
//   k_record_residual  the step's residual ||(W^{n+1} - W^n)/dt||_2.
// At the fixed point of the march R_W = -sum Phi does not vanish: it balances
// the moments of the discrete collision term (the quadrature error of the
// discrete equilibrium), so the march is measured by its rate of change.
// ---------------------------------------------------------------------------

// one thread per instance: the residual of this iteration from the block
// partials of the kernel before it into the ring, and the iteration count
template <class T>
__global__ void __launch_bounds__(32) k_record_residual(Launch L)
{
    IDG_LOCATE();
    (void)blk;
    if (threadIdx.x == 0) {
        record_residual(p);
        *p.iter += 1;
    }
}

template <class T>
__global__ void __launch_bounds__(128) k_explicit_update(Launch L)
{
    IDG_LOCATE();
    const int nvb = (p.Nv + 255) / 256;
    const int c = blk / nvb;
    const int k = 2 * ((blk - c * nvb) * 128 + threadIdx.x);
    if (k >= p.Nv) return;
    const T *cA = (const T *)p.cellA + kCellP * c;
    const EqT<T> e = eq_loadT<T>(cA);
    // k_cell_params stores c2 = 3h/(2tau+dt) = (3/4) 2dt/(2tau+dt) (h = dt/2)
    const T b = cA[15] * (T)(4.0 / 3.0), a = (T)1 - b;
    const T dto = (T)(p.dt / p.area[c]), kRTr = (T)(p.K * p.RT_r);
    T ux[2], uy[2], gr[2];
    vtab2<T>(p.uxf, p.ux, k, ux);
    vtab2<T>(p.uyf, p.uy, k, uy);
    vtab2<T>(p.greff, p.gref, k, gr);
    T sg_[2] = {0, 0}, sh_[2] = {0, 0};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        T fg[2], fh[2];
        load_pair<T>(p.F, (size_t)p.cface[4 * c + m] * p.Nv + k, fg, fh);
        const T sg = (T)p.csign[4 * c + m];
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            sg_[v] += sg * fg[v];
            sh_[v] += sg * fh[v];
        }
    }
    const size_t ck = (size_t)c * p.Nv + k;
    T g[2], h[2];
    load_pair<T>(p.f, ck, g, h);
#pragma unroll
    for (int v = 0; v < 2; ++v) {
        T dG, dH;
        dev_equilibrium<T>(e, ux[v], uy[v], gr[v], kRTr, dG, dH);
        g[v] = a * g[v] + b * dG - dto * sg_[v];
        h[v] = a * h[v] + b * dH - dto * sh_[v];
    }
    store_pair<T>(p.f, ck, g, h);
}

// W = (rho, rho U, rho V, rho E) of f~ from its raw moments (Eq. 4), and
// block partials of ||(W_new - W_old)/dt||^2 (fixed order)
template <class T>
__global__ void __launch_bounds__(32) k_explicit_w(Launch L)
{
    IDG_LOCATE();
    __shared__ double sm[32];
    const int c = blk * blockDim.x + threadIdx.x;
    double part[1] = {0.0};
    if (c < p.N) {
        auto r = [&](int q) { return acc_load<T>(p.cellraw, (size_t)c * kRaw + q) + p.mref_raw[q]; };
        double *W = p.W + 4 * c;
        const double Wn[4] = {r(0), r(1), r(2), 0.5 * (r(3) + r(5) + r(8))};
        for (int q = 0; q < 4; ++q) {
            const double d = (Wn[q] - W[q]) / p.dt;
            part[0] += d * d;
            W[q] = Wn[q];
        }
    }
    block_sum<1>(part, sm);
    if (threadIdx.x == 0) p.mpart[blk] = part[0];
}

// ---------------------------------------------------------------------------
// micro LU-SGS (Eq. 22-26)                                            [a6-a7]
//   k_micro_residual  per (cell, velocity), fully parallel:
//                     R = -sum_faces F - (2 Omega/(2 tau' + dt)) (f~ - f^S(W^{n+1})),
//                     written into the increment buffer
//   k_sweep_fwd       Delta*_c = (R_c + sum_{lower inflow nb} |xi.n| S Delta*_nb) / D_c
//   k_sweep_bwd       Delta_c = Delta*_c + sum_{upper inflow nb} |xi.n| S Delta_nb / D_c,
//                     f~ += Delta (Eq. 32)
// with D = Omega/dt_imp + sum_{outflow} xi.n S + 2 Omega/(2 tau' + dt).
// The sweeps run one CTA per tile of sweep_tv velocities over the i+j
// hyperplanes; thread (slot, t) owns cell (ilo + slot) of each hyperplane at
// velocity t.  Everything a step reads except the neighbours' increments is
// prefetched kStages-1 hyperplanes ahead with cp.async; the previous
// hyperplane's increments sit in a shared-memory ring, and neighbours across
// a periodic seam (earlier hyperplanes) are read back from global memory.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(128) k_micro_residual(Launch L)
{
    IDG_LOCATE();
    const int nvb = (p.Nv + 255) / 256;
    const int c = blk / nvb;
    const int k = 2 * ((blk - c * nvb) * 128 + threadIdx.x);
    if (k >= p.Nv) return;
    const T *cp = (const T *)p.cellpT + kCellP * c;
    const EqT<T> e = eq_loadT<T>(cp);
    const T cq = cp[14], kRTr = (T)(p.K * p.RT_r);
    T ux[2], uy[2], gr[2];
    vtab2<T>(p.uxf, p.ux, k, ux);
    vtab2<T>(p.uyf, p.uy, k, uy);
    vtab2<T>(p.greff, p.gref, k, gr);
    const size_t ck = (size_t)c * p.Nv + k;
    T rg[2], rh[2];
    load_pair<T>(p.f, ck, rg, rh);
#pragma unroll
    for (int v = 0; v < 2; ++v) {
        T dG, dH;
        dev_equilibrium<T>(e, ux[v], uy[v], gr[v], kRTr, dG, dH);
        rg[v] = -cq * (rg[v] - dG);
        rh[v] = -cq * (rh[v] - dH);
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        T fg[2], fh[2];
        load_pair<T>(p.F, (size_t)p.cface[4 * c + m] * p.Nv + k, fg, fh);
        const T sg = (T)p.csign[4 * c + m];
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            rg[v] -= sg * fg[v];
            rh[v] -= sg * fh[v];
        }
    }
    store_pair<T>(p.dst, ck, rg, rh);
}

// 16 storage scalars from 16-byte-aligned shared memory
template <class T> __device__ __forceinline__ void load16(T (&r)[16], const T *s);
template <> __device__ __forceinline__ void load16<float>(float (&r)[16], const float *s)
{
    const float4 *q = (const float4 *)s;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        float4 a = q[u];
        r[4 * u] = a.x; r[4 * u + 1] = a.y; r[4 * u + 2] = a.z; r[4 * u + 3] = a.w;
    }
}
template <> __device__ __forceinline__ void load16<double>(double (&r)[16], const double *s)
{
    const double2 *q = (const double2 *)s;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        double2 a = q[u];
        r[2 * u] = a.x; r[2 * u + 1] = a.y;
    }
}

// Role of the neighbour across each slot of a cell in one micro sweep
// (computed on the host): >= 0 its slot in the previous hyperplane's ring;
// kOther a ghost or a neighbour not yet swept (outflow only adds to D); kSelf
// the cell itself across a periodic direction one cell wide (no term at all);
// <= kSeam the neighbour kSeam - code across a periodic seam (already swept,
// read from global memory).
constexpr int kOther = -2, kSelf = -3, kSeam = -4;

// 8 storage scalars from 16-byte-aligned shared memory
template <class T> __device__ __forceinline__ void load8(T (&r)[8], const T *s);
template <> __device__ __forceinline__ void load8<float>(float (&r)[8], const float *s)
{
    const float4 a = ((const float4 *)s)[0], b = ((const float4 *)s)[1];
    r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w; r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
}
template <> __device__ __forceinline__ void load8<double>(double (&r)[8], const double *s)
{
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const double2 a = ((const double2 *)s)[u];
        r[2 * u] = a.x; r[2 * u + 1] = a.y;
    }
}

// shared-memory layout of the micro sweeps (VPT consecutive velocities per thread)
template <class T, int kStages, int VPT> struct SweepSmem {
    using T2 = typename V2<T>::t;
    T2 *R;      // [kStages][pc][tv*VPT]  R (forward) / Delta* (backward)
    T2 *F;      // [kStages][pc][tv*VPT]  f~ (backward only)
    T *geo;     // [kStages][pc][8]  per slot: sign*nx*S, sign*ny*S
    int *code;  // [kStages][pc][4]  per slot: the neighbour's role in this sweep (sweep_codes)
    T2 *ring;   // [2][pc][tv*VPT]  increments of the previous hyperplane, by slot
    T *D0;      // [kStages][pc]
    __device__ SweepSmem(unsigned char *base, int pc, int tv, bool withF)
    {
        size_t o = 0;
        const size_t w = (size_t)tv * VPT;
        R = (T2 *)(base + o); o += (size_t)kStages * pc * w * sizeof(T2);
        F = (T2 *)(base + o); if (withF) o += (size_t)kStages * pc * w * sizeof(T2);
        geo = (T *)(base + o); o += (size_t)kStages * pc * 8 * sizeof(T);
        code = (int *)(base + o); o += (size_t)kStages * pc * 4 * sizeof(int);
        ring = (T2 *)(base + o); o += (size_t)2 * pc * w * sizeof(T2);
        D0 = (T *)(base + o);
    }
};

template <class T, int kStages, int VPT> static size_t sweep_smem_bytes(int pc, int tv, bool withF)
{
    using T2 = typename V2<T>::t;
    const size_t w = (size_t)tv * VPT;
    size_t o = (size_t)kStages * pc * w * sizeof(T2) * (withF ? 2 : 1);
    o += (size_t)kStages * pc * (8 * sizeof(T) + 4 * sizeof(int));
    o += (size_t)2 * pc * w * sizeof(T2) + (size_t)kStages * pc * sizeof(T);
    return o;
}

// the parameters a sweep touches every step, held in registers
struct SweepArgs {
    int Nv, ni, nj, tv, pc;
    void *dst, *f;
    const void *cslotT, *cellpT;
    const int *codes;  // this sweep's [N][4] slot codes
    const int *sched, *sptr;  // this sweep's schedule (unstructured) or null
    int nsteps;               // steps of the sweep
};

// the cell of slot `slot` at step d (a hyperplane i + j = d on a structured
// block, with its (i, j); the d-th step of the schedule otherwise), -1 past
// the step's end
template <bool SCHED> __device__ __forceinline__ int sweep_cell(const SweepArgs &p, int d, int slot, int &i, int &j)
{
    if (SCHED) {
        const int b = p.sptr[d];
        i = j = 0;
        return slot < p.sptr[d + 1] - b ? p.sched[b + slot] : -1;
    }
    const int ilo = max(0, d - (p.nj - 1)), ihi = min(p.ni - 1, d);
    i = ilo + slot;
    j = d - i;
    return i <= ihi ? j * p.ni + i : -1;
}

// asynchronous copy of one step's data for the thread's cell: its VPT
// consecutive velocities of R (or Delta*, f~), and the cell's slot geometry
// and diagonal base spread over the cell's tv threads
template <class T, int kStages, int VPT, bool SCHED>
__device__ __forceinline__ void sweep_issue(const SweepArgs &p, const SweepSmem<T, kStages, VPT> &sm, int s, int d,
                                            int slot, int t, int k0, bool act, bool withF)
{
    using T2 = typename V2<T>::t;
    const int tv = p.tv, pc = p.pc;
    if (s < p.nsteps) {
        int ci, cj;
        const int c = sweep_cell<SCHED>(p, d, slot, ci, cj);
        if (c >= 0) {
            int st = s & (kStages - 1);
            size_t e = ((size_t)st * pc + slot);
            if (act) {
                constexpr int B = VPT * sizeof(T2);
                constexpr int CH = B < 16 ? B : 16;
                size_t ck = (size_t)c * p.Nv + k0;
                char *sr = (char *)(sm.R + e * tv * VPT + (size_t)t * VPT);
                const char *gr = (const char *)((const T2 *)p.dst + ck);
#pragma unroll
                for (int b = 0; b < B; b += CH) cp_async_b<CH>(sr + b, gr + b);
                if (withF) {
                    char *sf = (char *)(sm.F + e * tv * VPT + (size_t)t * VPT);
                    const char *gf = (const char *)((const T2 *)p.f + ck);
#pragma unroll
                    for (int b = 0; b < B; b += CH) cp_async_b<CH>(sf + b, gf + b);
                }
            }
            constexpr int ng = 8 * sizeof(T) / 16;  // 16-byte chunks of the slot geometry
            for (int q = t; q < ng + 2; q += tv) {
                if (q < ng) cp_async16((char *)(sm.geo + e * 8) + 16 * q, (const char *)((const T *)p.cslotT + 8 * (size_t)c) + 16 * q);
                else if (q == ng) cp_async16(sm.code + e * 4, p.codes + 4 * (size_t)c);
                else cp_async_b<sizeof(T)>(sm.D0 + e, (const T *)p.cellpT + kCellP * (size_t)c + 15);
            }
        }
    }
    cp_commit();
}

template <class T, bool FWD, int kStages, int VPT, bool SCHED = false>
__global__ void __launch_bounds__(512) k_sweep(Launch L)
{
    IDG_LOCATE();
    using T2 = typename V2<T>::t;
    extern __shared__ __align__(16) unsigned char smraw[];
    // SCHED (unstructured mesh): the steps of the schedule; otherwise the i+j
    // hyperplanes, compiled without any schedule state
    const SweepArgs a{p.Nv, p.ni, p.nj, p.sweep_tv, p.sweep_pc, p.dst, p.f, p.cslotT, p.cellpT,
                      p.scode + (FWD ? 0 : 4 * (size_t)p.N),
                      SCHED ? p.sched + (FWD ? 0 : (size_t)p.N) : nullptr,
                      SCHED ? p.sptr + (FWD ? 0 : p.nsteps_f + 1) : nullptr,
                      SCHED ? (FWD ? p.nsteps_f : p.nsteps_b) : p.ni + p.nj - 1};
    const int tv = a.tv, pc = a.pc, ni = a.ni, nj = a.nj, Nv = a.Nv;
    const bool per_i = p.per_i, per_j = p.per_j;
    const SweepSmem<T, kStages, VPT> sm(smraw, pc, tv, !FWD);
    const int t = threadIdx.x % tv, slot = threadIdx.x / tv;
    const int k0 = (blk * tv + t) * VPT;  // Nv is a multiple of VPT
    const bool act = k0 < Nv;
    T ux[VPT], uy[VPT];
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        const int kk = act ? k0 + v : 0;
        ux[v] = vx<T>(p, kk);
        uy[v] = vy<T>(p, kk);
    }
    T2 *ds = (T2 *)a.dst;
    T2 *f = (T2 *)a.f;
    const int nh = a.nsteps;
    const size_t w = (size_t)tv * VPT;
    // a schedule lists the backward sweep's steps in processing order
    auto step_d = [&](int s) { return (FWD || SCHED) ? s : nh - 1 - s; };
    for (int s = 0; s < kStages - 1; ++s) sweep_issue<T, kStages, VPT, SCHED>(a, sm, s, step_d(s), slot, t, k0, act, !FWD);
    for (int s = 0; s < nh; ++s) {
        cp_wait<kStages - 2>();
        __syncthreads();
        sweep_issue<T, kStages, VPT, SCHED>(a, sm, s + kStages - 1, step_d(s + kStages - 1), slot, t, k0, act, !FWD);
        int i, j;
        const int c = sweep_cell<SCHED>(a, step_d(s), slot, i, j);
        if (c < 0 || !act) continue;
        const size_t e = (size_t)(s & (kStages - 1)) * pc + slot;
        T g[8];
        load8<T>(g, sm.geo + e * 8);
        const int4 cd = *(const int4 *)(sm.code + e * 4);
        const int code[4] = {cd.x, cd.y, cd.z, cd.w};
        const T D0 = sm.D0[e];
        const size_t ck = (size_t)c * Nv + k0;
        const size_t rbase = e * w + (size_t)t * VPT;
        const size_t rprev = (size_t)((s + 1) & 1) * pc * w + (size_t)t * VPT;
        // the backward sweep's increments are read back from global memory
        // only across a periodic seam (the first and last cells of a periodic
        // direction); elsewhere only f and the ring take them
        const bool keep = FWD || SCHED || (per_i && (i == 0 || i == ni - 1)) || (per_j && (j == 0 || j == nj - 1));
        // the step of one cell; SEAM: some neighbour lies across a periodic
        // seam (read from global memory), otherwise every inflow comes from
        // the ring
        auto cell_step = [&](auto seam_tag) {
            constexpr bool SEAM = decltype(seam_tag)::value;
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                // slot terms, branch-free: outflow adds (xi.n) S to D, inflow
                // from the already-swept side adds |xi.n| S Delta_nb
                T D = D0;
                T aS[4];
                bool in[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    aS[m] = add_rn(mul_rn(ux[v], g[2 * m]), mul_rn(uy[v], g[2 * m + 1]));
                    D += (aS[m] > (T)0 && code[m] != kSelf) ? aS[m] : (T)0;
                    in[m] = aS[m] < (T)0 && (code[m] >= 0 || (SEAM && code[m] <= kSeam));
                }
                T2 dn[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    dn[m].x = (T)0;
                    dn[m].y = (T)0;
                    if (in[m]) {
                        if (!SEAM || code[m] >= 0) dn[m] = sm.ring[rprev + (size_t)code[m] * w + v];
                        else dn[m] = ds[(size_t)(kSeam - code[m]) * Nv + k0 + v];
                    }
                }
                T ag = 0, ah = 0;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    ag -= aS[m] * dn[m].x;
                    ah -= aS[m] * dn[m].y;
                }
                const T2 r = sm.R[rbase + v];
                const T iD = rcp_rn(D);
                T2 o;
                if (FWD) {
                    o.x = (r.x + ag) * iD;
                    o.y = (r.y + ah) * iD;
                } else {
                    o.x = r.x + ag * iD;
                    o.y = r.y + ah * iD;
                    T2 fv = sm.F[rbase + v];
                    fv.x += o.x;
                    fv.y += o.y;
                    f[ck + v] = fv;
                }
                if (keep) ds[ck + v] = o;
                sm.ring[((size_t)(s & 1) * pc + slot) * w + (size_t)t * VPT + v] = o;
            }
        };
        if (code[0] <= kSeam || code[1] <= kSeam || code[2] <= kSeam || code[3] <= kSeam)
            cell_step(std::true_type{});
        else
            cell_step(std::false_type{});
    }
    cp_wait<0>();
}

// ---------------------------------------------------------------------------
// state conversion and diagnostics
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_to_dev(KParams p, const double *G, const double *H, int nvu, int deviation)
{
    using T2 = typename V2<T>::t;
    size_t n = (size_t)p.N * p.Nv;
    // deviation: G, H already hold f~ - M_ref (a checkpoint's stored form)
    const double ref = deviation ? 0.0 : 1.0;
    double kRTr = p.K * p.RT_r;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t c = i / p.Nv;
        const int k = (int)(i - c * p.Nv);
        T2 o;
        o.x = (T)0;
        o.y = (T)0;
        if (k < nvu) {
            const size_t j = c * nvu + k;
            o.x = (T)(G[j] - ref * p.gref[k]);
            o.y = (T)(H[j] - ref * kRTr * p.gref[k]);
        }
        ((T2 *)p.f)[i] = o;
    }
}

template <class T>
__global__ void k_from_dev(KParams p, double *G, double *H, int nvu, int deviation)
{
    using T2 = typename V2<T>::t;
    size_t n = (size_t)p.N * p.Nv;
    const double ref = deviation ? 0.0 : 1.0;
    double kRTr = p.K * p.RT_r;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t c = i / p.Nv;
        const int k = (int)(i - c * p.Nv);
        if (k >= nvu) continue;
        const size_t j = c * nvu + k;
        T2 v = ((const T2 *)p.f)[i];
        G[j] = ref * p.gref[k] + (double)v.x;
        H[j] = ref * kRTr * p.gref[k] + (double)v.y;
    }
}

// per cell: rho, u, v, T/T_ref from W; heat flux of f from f~ (cellraw)
template <class T>
__global__ void __launch_bounds__(256) k_moments_out(KParams p, double *out6)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p.N) return;
    double r[kRaw];
    for (int q = 0; q < kRaw; ++q) r[q] = acc_load<T>(p.cellraw, (size_t)c * kRaw + q) + p.mref_raw[q];
    const double *W = p.W + 4 * c;
    double rho = W[0], U = W[1] / rho, V = W[2] / rho;
    double RT = (2.0 * W[3] / rho - U * U - V * V) / (p.K + 2);
    double tau = viscosity_t<T>(p, RT) / (rho * RT);
    double qtx, qty;
    raw_heat_flux(r, U, V, qtx, qty);
    double Pr = p.shakhov ? p.Pr : 1.0;
    out6[6 * c + 0] = rho;
    out6[6 * c + 1] = U;
    out6[6 * c + 2] = V;
    out6[6 * c + 3] = RT / p.RT_ref;
    out6[6 * c + 4] = 2.0 * tau * qtx / (2.0 * tau + p.dt * Pr);
    out6[6 * c + 5] = 2.0 * tau * qty / (2.0 * tau + p.dt * Pr);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline int nblk(int n, int per) { return (n + per - 1) / per; }

static int macro_threads(const KParams &p) { return std::min(512, ((2 * std::min(p.ni, p.nj) + 31) / 32) * 32); }

template <class T> static size_t macro_smem_bytes(const KParams &p, int nt, int stages)
{
    return (size_t)stages * (nt / 2) * (kMRec + 4) * sizeof(T) + (size_t)2 * (nt / 2) * kMRing * sizeof(T);
}

template <class T, int S> static size_t sweep_bytes_s(const KParams &p, bool withF)
{
    switch (p.sweep_vpt) {
    case 4: return sweep_smem_bytes<T, S, 4>(p.sweep_pc, p.sweep_tv, withF);
    case 2: return sweep_smem_bytes<T, S, 2>(p.sweep_pc, p.sweep_tv, withF);
    default: return sweep_smem_bytes<T, S, 1>(p.sweep_pc, p.sweep_tv, withF);
    }
}

template <class T> static size_t sweep_bytes(const KParams &p, bool withF, int stages)
{
    return stages == 8 ? sweep_bytes_s<T, 8>(p, withF)
         : stages == 2 ? sweep_bytes_s<T, 2>(p, withF) : sweep_bytes_s<T, 4>(p, withF);
}

void blocks_per_instance(const KParams &p, int out[KT_COUNT])
{
    const int nvb = nblk(p.Nv, 256);
    out[KT_CELL_MOM] = nblk(p.N, 8);
    out[KT_CELL_PAR] = nblk(p.N, 32);
    out[KT_FBP] = p.N * nvb;
    out[KT_FACE_MOM] = nblk(p.nf, 8);
    out[KT_FACE_PAR] = nblk(p.nf, 32);
    out[KT_FACE_FLUX] = nblk(p.nf, 8);
    out[KT_FACE_PHI] = nblk(p.nf, 64);
    out[KT_MACRO_PRE] = nblk(p.N, 32);
    out[KT_MACRO_SWEEP] = 1;
    out[KT_MACRO_POST] = nblk(p.N, 32);
    out[KT_MICRO_RES] = p.N * nvb;
    out[KT_SWEEP] = nblk(p.Nv, p.sweep_tv * p.sweep_vpt);
}

// block shape, shared memory and prefetch depth common to all instances of
// a plan (the maxima of the instances; the deepest pipeline that fits all)
int plan_shapes(const KParams *hp, int n, bool fp64, Plan &pl)
{
    const size_t lim = 227 * 1024;
    pl.macro_threads = pl.sweep_threads = 0;
    pl.limiter_any = 0;
    pl.sweep_vpt = hp[0].sweep_vpt;
    pl.relax_sweeps = hp[0].relax_sweeps;
    pl.sched = hp[0].sched != nullptr;
    pl.sched_smem = 0;
    for (int i = 0; i < n; ++i) {
        if ((hp[i].sched != nullptr) != (pl.sched != 0)) return (int)cudaErrorInvalidValue;
        pl.sched_smem = std::max(pl.sched_smem, (size_t)hp[i].N * 4 * (fp64 ? 8 : 4));
        if (hp[i].relax_sweeps != pl.relax_sweeps) return (int)cudaErrorInvalidValue;
        pl.macro_threads = std::max(pl.macro_threads, macro_threads(hp[i]));
        pl.sweep_threads = std::max(pl.sweep_threads, hp[i].sweep_tv * hp[i].sweep_pc);
        pl.limiter_any |= hp[i].limiter;
        if (hp[i].sweep_vpt != pl.sweep_vpt) return (int)cudaErrorInvalidValue;
    }
    if (!pl.sched || pl.sched_smem > 200 * 1024) pl.sched_smem = 0;
    pl.any_seam = 0;
    for (int i = 0; i < n; ++i) pl.any_seam |= hp[i].per_i | hp[i].per_j;
    pl.macro_kind = hp[0].macro_kind;
    for (int i = 0; i < n; ++i)
        if (hp[i].macro_kind != pl.macro_kind) return (int)cudaErrorInvalidValue;
    if (pl.macro_kind == 1 && !pl.sched) {
        // one thread per line of the shorter axis; the seam array holds the
        // walk axis' cells when the lines wrap around (a periodic shorter axis)
        int ntmax = 0;
        for (int i = 0; i < n; ++i) ntmax = std::max(ntmax, std::min(hp[i].ni, hp[i].nj));
        pl.macro_threads = ((ntmax + 31) / 32) * 32;
        const int nlines = pl.macro_threads;
        for (int stages : {std::min(hp[0].macro_stages, 8), 4, 2}) {
            size_t m = 0;
            for (int i = 0; i < n; ++i) {
                const bool cols = hp[i].ni <= hp[i].nj;
                const bool seam = cols ? hp[i].per_i : hp[i].per_j;
                const int nw = std::max(hp[i].ni, hp[i].nj);
                m = std::max(m, fp64 ? macro_lines_smem_bytes<double>(nlines, stages, nw, seam)
                                     : macro_lines_smem_bytes<float>(nlines, stages, nw, seam));
            }
            pl.macro_stages = stages;
            pl.macro_smem = m;
            if (m <= lim) break;
        }
    } else {
    // a 2-stage prefetch is the fallback that fits a 256-cell hyperplane of
    // float64 records
    for (int stages : {std::min(hp[0].macro_stages, 8), 4, 2}) {
        size_t m = 0;
        for (int i = 0; i < n; ++i)
            m = std::max(m, fp64 ? macro_smem_bytes<double>(hp[i], pl.macro_threads, stages)
                                 : macro_smem_bytes<float>(hp[i], pl.macro_threads, stages));
        pl.macro_stages = stages;
        pl.macro_smem = m;
        if (m <= lim) break;
    }
    }
    for (int stages : {pl.sched ? 4 : std::min(hp[0].sweep_stages, 8), 4}) {
        size_t f = 0, b = 0;
        for (int i = 0; i < n; ++i) {
            f = std::max(f, fp64 ? sweep_bytes<double>(hp[i], false, stages) : sweep_bytes<float>(hp[i], false, stages));
            b = std::max(b, fp64 ? sweep_bytes<double>(hp[i], true, stages) : sweep_bytes<float>(hp[i], true, stages));
        }
        pl.sweep_stages = stages;
        pl.fwd_smem = f;
        pl.bwd_smem = b;
        if (b <= lim) break;
    }
    if (pl.macro_smem > lim || pl.bwd_smem > lim) return (int)cudaErrorInvalidValue;
    return 0;
}

template <class T, bool FWD, int S>
static void launch_sweep_s(const Plan &pl, cudaStream_t st, const Launch &L)
{
    const size_t sm = FWD ? pl.fwd_smem : pl.bwd_smem;
    const int nb = pl.nblocks[KT_SWEEP], nt = pl.sweep_threads;
    switch (pl.sweep_vpt) {
    case 4: k_sweep<T, FWD, S, 4><<<nb, nt, sm, st>>>(L); break;
    case 2: k_sweep<T, FWD, S, 2><<<nb, nt, sm, st>>>(L); break;
    default: k_sweep<T, FWD, S, 1><<<nb, nt, sm, st>>>(L); break;
    }
}

// unstructured meshes: the scheduled sweeps (always a 4-step prefetch)
template <class T, bool FWD>
static void launch_sweep_sched(const Plan &pl, cudaStream_t st, const Launch &L)
{
    const size_t sm = FWD ? pl.fwd_smem : pl.bwd_smem;
    const int nb = pl.nblocks[KT_SWEEP], nt = pl.sweep_threads;
    switch (pl.sweep_vpt) {
    case 4: k_sweep<T, FWD, 4, 4, true><<<nb, nt, sm, st>>>(L); break;
    case 2: k_sweep<T, FWD, 4, 2, true><<<nb, nt, sm, st>>>(L); break;
    default: k_sweep<T, FWD, 4, 1, true><<<nb, nt, sm, st>>>(L); break;
    }
}

template <class T, bool FWD> static void launch_sweep(const Plan &pl, cudaStream_t st, const Launch &L)
{
    if (pl.sched) launch_sweep_sched<T, FWD>(pl, st, L);
    else if (pl.sweep_stages == 8) launch_sweep_s<T, FWD, 8>(pl, st, L);
    else if (pl.sweep_stages == 2) launch_sweep_s<T, FWD, 2>(pl, st, L);
    else launch_sweep_s<T, FWD, 4>(pl, st, L);
}

template <class T> static Launch launch_of(const Plan &pl, int kt)
{
    Launch L;
    L.params = pl.dparams;
    L.off = pl.doff ? pl.doff + (size_t)kt * (pl.ninst + 1) : nullptr;
    L.active = pl.dactive;
    L.ninst = pl.ninst;
    return L;
}

// events (optional): kProfiled+1 cudaEvent_t recorded between the six groups
// cell prep | face moments+params | face flux+phi | macro | residual+fwd | bwd
template <class T>
static int iteration_t(const Plan &pl, cudaStream_t st, void **events)
{
    auto mark = [&](int q) {
        if (events) cudaEventRecord((cudaEvent_t)events[q], st);
    };
    auto L = [&](int kt) { return launch_of<T>(pl, kt); };
    const int *nb = pl.nblocks;
    if (pl.explicit_dugks) {
        // W^n and the raw moments of f~^n are left by the previous step (or
        // by launch_explicit_prologue)
        mark(0);
        k_cell_params<T><<<nb[KT_CELL_PAR], 32, 0, st>>>(L(KT_CELL_PAR));
        k_fbp<T><<<nb[KT_FBP], 128, 0, st>>>(L(KT_FBP));
        mark(1);
        if (pl.limiter_any) k_cell_grad<T><<<nb[KT_FBP], 128, 0, st>>>(L(KT_FBP));
        if (pl.limiter_any) k_face_moments<T, true><<<nb[KT_FACE_MOM], 256, 0, st>>>(L(KT_FACE_MOM));
        else k_face_moments<T, false><<<nb[KT_FACE_MOM], 256, 0, st>>>(L(KT_FACE_MOM));
        k_face_params<T><<<nb[KT_FACE_PAR], 32, 0, st>>>(L(KT_FACE_PAR));
        mark(2);
        k_face_flux<T><<<nb[KT_FACE_FLUX], 256, 0, st>>>(L(KT_FACE_FLUX));
        k_face_phi<T><<<nb[KT_FACE_PHI], 64, 0, st>>>(L(KT_FACE_PHI));
        mark(3);
        mark(4);
        k_explicit_update<T><<<nb[KT_MICRO_RES], 128, 0, st>>>(L(KT_MICRO_RES));
        k_cell_moments<T><<<nb[KT_CELL_MOM], 256, 0, st>>>(L(KT_CELL_MOM));
        k_explicit_w<T><<<nb[KT_CELL_PAR], 32, 0, st>>>(L(KT_CELL_PAR));
        k_record_residual<T><<<nb[KT_MACRO_SWEEP], 32, 0, st>>>(L(KT_MACRO_SWEEP));
        mark(5);
        mark(6);
        return (int)cudaGetLastError();
    }
    mark(0);
    k_cell_moments<T><<<nb[KT_CELL_MOM], 256, 0, st>>>(L(KT_CELL_MOM));
    k_cell_params<T><<<nb[KT_CELL_PAR], 32, 0, st>>>(L(KT_CELL_PAR));
    k_fbp<T><<<nb[KT_FBP], 128, 0, st>>>(L(KT_FBP));
    mark(1);
    if (pl.limiter_any) k_cell_grad<T><<<nb[KT_FBP], 128, 0, st>>>(L(KT_FBP));
    if (pl.limiter_any) k_face_moments<T, true><<<nb[KT_FACE_MOM], 256, 0, st>>>(L(KT_FACE_MOM));
    else k_face_moments<T, false><<<nb[KT_FACE_MOM], 256, 0, st>>>(L(KT_FACE_MOM));
    k_face_params<T><<<nb[KT_FACE_PAR], 32, 0, st>>>(L(KT_FACE_PAR));
    mark(2);
    k_face_flux<T><<<nb[KT_FACE_FLUX], 256, 0, st>>>(L(KT_FACE_FLUX));
    k_face_phi<T><<<nb[KT_FACE_PHI], 64, 0, st>>>(L(KT_FACE_PHI));
    mark(3);
    k_macro_pre<T><<<nb[KT_MACRO_PRE], 32, 0, st>>>(L(KT_MACRO_PRE));
    if (pl.relax_sweeps > 0) {
        k_record_residual<T><<<nb[KT_MACRO_SWEEP], 32, 0, st>>>(L(KT_MACRO_SWEEP));
        for (int k = 1; k <= pl.relax_sweeps; ++k)
            k_macro_relax<T><<<nb[KT_MACRO_PRE], 32, 0, st>>>(L(KT_MACRO_PRE), k, pl.relax_sweeps);
    } else if (pl.sched) {
        if (pl.sched_smem)
            k_macro_sweep_sched<T, true><<<nb[KT_MACRO_SWEEP], 256, pl.sched_smem, st>>>(L(KT_MACRO_SWEEP));
        else
            k_macro_sweep_sched<T, false><<<nb[KT_MACRO_SWEEP], 256, 0, st>>>(L(KT_MACRO_SWEEP));
    } else if (pl.macro_kind == 1) {
        const int nb1 = nb[KT_MACRO_SWEEP], nt1 = pl.macro_threads;
        const size_t sm1 = pl.macro_smem;
        const Launch L1 = L(KT_MACRO_SWEEP);
        if (pl.any_seam) {
            if (pl.macro_stages == 8) k_macro_lines<T, 8, true><<<nb1, nt1, sm1, st>>>(L1);
            else if (pl.macro_stages == 4) k_macro_lines<T, 4, true><<<nb1, nt1, sm1, st>>>(L1);
            else k_macro_lines<T, 2, true><<<nb1, nt1, sm1, st>>>(L1);
        } else {
            if (pl.macro_stages == 8) k_macro_lines<T, 8, false><<<nb1, nt1, sm1, st>>>(L1);
            else if (pl.macro_stages == 4) k_macro_lines<T, 4, false><<<nb1, nt1, sm1, st>>>(L1);
            else k_macro_lines<T, 2, false><<<nb1, nt1, sm1, st>>>(L1);
        }
    } else if (pl.macro_stages == 8)
        k_macro_sweep<T, 8><<<nb[KT_MACRO_SWEEP], pl.macro_threads, pl.macro_smem, st>>>(L(KT_MACRO_SWEEP));
    else if (pl.macro_stages == 4)
        k_macro_sweep<T, 4><<<nb[KT_MACRO_SWEEP], pl.macro_threads, pl.macro_smem, st>>>(L(KT_MACRO_SWEEP));
    else
        k_macro_sweep<T, 2><<<nb[KT_MACRO_SWEEP], pl.macro_threads, pl.macro_smem, st>>>(L(KT_MACRO_SWEEP));
    k_macro_post<T><<<nb[KT_MACRO_POST], 32, 0, st>>>(L(KT_MACRO_POST));
    mark(4);
    k_micro_residual<T><<<nb[KT_MICRO_RES], 128, 0, st>>>(L(KT_MICRO_RES));
    launch_sweep<T, true>(pl, st, L(KT_SWEEP));
    mark(5);
    launch_sweep<T, false>(pl, st, L(KT_SWEEP));
    mark(6);
    return (int)cudaGetLastError();
}

// opt the wavefront kernels in to the largest dynamic shared memory once
template <class T> static int configure_t()
{
    const int lim = 227 * 1024;
    cudaError_t e = cudaSuccess;
    auto opt = [&](const void *fn) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    };
    opt((const void *)k_macro_sweep_sched<T, true>);
    opt((const void *)k_macro_lines<T, 8, false>);
    opt((const void *)k_macro_lines<T, 4, false>);
    opt((const void *)k_macro_lines<T, 2, false>);
    opt((const void *)k_macro_lines<T, 8, true>);
    opt((const void *)k_macro_lines<T, 4, true>);
    opt((const void *)k_macro_lines<T, 2, true>);
    opt((const void *)k_macro_sweep<T, 8>);
    opt((const void *)k_macro_sweep<T, 4>);
    opt((const void *)k_macro_sweep<T, 2>);
    opt((const void *)k_sweep<T, true, 4, 1, true>);
    opt((const void *)k_sweep<T, false, 4, 1, true>);
    opt((const void *)k_sweep<T, true, 4, 2, true>);
    opt((const void *)k_sweep<T, false, 4, 2, true>);
    opt((const void *)k_sweep<T, true, 4, 4, true>);
    opt((const void *)k_sweep<T, false, 4, 4, true>);
    opt((const void *)k_sweep<T, true, 2, 1>);
    opt((const void *)k_sweep<T, false, 2, 1>);
    opt((const void *)k_sweep<T, true, 2, 2>);
    opt((const void *)k_sweep<T, false, 2, 2>);
    opt((const void *)k_sweep<T, true, 2, 4>);
    opt((const void *)k_sweep<T, false, 2, 4>);
    opt((const void *)k_sweep<T, true, 8, 1>);
    opt((const void *)k_sweep<T, false, 8, 1>);
    opt((const void *)k_sweep<T, true, 4, 1>);
    opt((const void *)k_sweep<T, false, 4, 1>);
    opt((const void *)k_sweep<T, true, 8, 2>);
    opt((const void *)k_sweep<T, false, 8, 2>);
    opt((const void *)k_sweep<T, true, 4, 2>);
    opt((const void *)k_sweep<T, false, 4, 2>);
    opt((const void *)k_sweep<T, true, 8, 4>);
    opt((const void *)k_sweep<T, false, 8, 4>);
    opt((const void *)k_sweep<T, true, 4, 4>);
    opt((const void *)k_sweep<T, false, 4, 4>);
    return (int)e;
}

int configure_kernels(bool fp64) { return fp64 ? configure_t<double>() : configure_t<float>(); }

int launch_iteration(const Plan &pl, bool fp64, void *stream, void **events)
{
    cudaStream_t st = (cudaStream_t)stream;
    return fp64 ? iteration_t<double>(pl, st, events) : iteration_t<float>(pl, st, events);
}

template <class T> static int explicit_prologue_t(const Plan &pl, cudaStream_t st)
{
    auto L = [&](int kt) { return launch_of<T>(pl, kt); };
    k_cell_moments<T><<<pl.nblocks[KT_CELL_MOM], 256, 0, st>>>(L(KT_CELL_MOM));
    k_explicit_w<T><<<pl.nblocks[KT_CELL_PAR], 32, 0, st>>>(L(KT_CELL_PAR));
    return (int)cudaGetLastError();
}

int launch_explicit_prologue(const Plan &pl, bool fp64, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    return fp64 ? explicit_prologue_t<double>(pl, st) : explicit_prologue_t<float>(pl, st);
}

int launch_cell_moments(const KParams &p, bool fp64, double *out6_dev, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    if (fp64) {
        k_cell_moments_v<double><<<nblk(p.N, 8), 256, 0, st>>>(p);
        k_moments_out<double><<<nblk(p.N, 256), 256, 0, st>>>(p, out6_dev);
    } else {
        k_cell_moments_v<float><<<nblk(p.N, 8), 256, 0, st>>>(p);
        k_moments_out<float><<<nblk(p.N, 256), 256, 0, st>>>(p, out6_dev);
    }
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// moments without a workspace scratch region
// ---------------------------------------------------------------------------
// Raw-moment scratch of idg_get_moments_noalloc: kNoAllocMaxCells cells x
// kRaw accumulators of 8 bytes (1.375 MiB), held by every GPU that loads the
// library until the process exits.  Every call overwrites all entries it
// reads, so nothing needs clearing; calls that overlap on the GPU race on it.
static __device__ __align__(256) unsigned char g_noalloc_raw[(size_t)kNoAllocMaxCells * kRaw * 8];

// Device address of the scratch, resolved once per device with that device
// current (a host-side use of the symbol's name is not a device address).
// The cache is guarded by a mutex: first calls from several host threads at
// once resolve it once.  It is keyed by device ordinal, so a cudaDeviceReset
// of that device (which unloads the module) leaves a stale address behind.
static void *noalloc_scratch(int device, int *err)
{
    static std::mutex mu;
    static void *addr[64] = {nullptr};
    *err = 0;
    if (device < 0 || device >= 64) {
        *err = (int)cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_raw);
        if (e != cudaSuccess) {
            *err = (int)e;
            return nullptr;
        }
        addr[device] = ptr;
    }
    return addr[device];
}

int launch_cell_moments_noalloc(const KParams &p0, bool fp64, int device, double *out6_dev, void *stream)
{
    if (p0.N > kNoAllocMaxCells) return (int)cudaErrorInvalidValue;
    int err = 0;
    void *scratch = noalloc_scratch(device, &err);
    if (!scratch) return err;
    KParams p = p0;
    p.cellraw = scratch;
    cudaStream_t st = (cudaStream_t)stream;
    if (fp64) {
        k_cell_moments_v<double><<<nblk(p.N, 8), 256, 0, st>>>(p);
        k_moments_out<double><<<nblk(p.N, 256), 256, 0, st>>>(p, out6_dev);
    } else {
        k_cell_moments_v<float><<<nblk(p.N, 8), 256, 0, st>>>(p);
        k_moments_out<float><<<nblk(p.N, 256), 256, 0, st>>>(p, out6_dev);
    }
    return (int)cudaGetLastError();
}

// residuals of the last `last` iterations and the status word of every
// instance of a batch (inactive instances repeat their last values)
__global__ void k_batch_gather(const KParams *ps, int n, int last, double *res, int *status)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const KParams &p = ps[i];
    const int it = *p.iter;
    for (int q = 0; q < last; ++q) res[(size_t)i * 16 + q] = p.res[(it - last + q) & (kMaxHist - 1)];
    status[i] = *p.status;
}

int launch_batch_gather(const KParams *dparams, int n, int last, double *dres, int *dstatus, void *stream)
{
    if (last > 16) return (int)cudaErrorInvalidValue;
    k_batch_gather<<<nblk(n, 64), 64, 0, (cudaStream_t)stream>>>(dparams, n, last, dres, dstatus);
    return (int)cudaGetLastError();
}

int launch_to_dev(const KParams &p, bool fp64, const double *G, const double *H, int nvu, void *stream,
                  bool deviation)
{
    cudaStream_t st = (cudaStream_t)stream;
    if (fp64) k_to_dev<double><<<1024, 256, 0, st>>>(p, G, H, nvu, deviation ? 1 : 0);
    else k_to_dev<float><<<1024, 256, 0, st>>>(p, G, H, nvu, deviation ? 1 : 0);
    return (int)cudaGetLastError();
}

int launch_from_dev(const KParams &p, bool fp64, double *G, double *H, int nvu, void *stream, bool deviation)
{
    cudaStream_t st = (cudaStream_t)stream;
    if (fp64) k_from_dev<double><<<1024, 256, 0, st>>>(p, G, H, nvu, deviation ? 1 : 0);
    else k_from_dev<float><<<1024, 256, 0, st>>>(p, G, H, nvu, deviation ? 1 : 0);
    return (int)cudaGetLastError();
}

}  // namespace idg
