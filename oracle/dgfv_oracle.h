/*
 * Plain FP64 CPU oracle of the hp-adaptive hybrid DG/FV right-hand side
 * U_t = R(U) for the multi-component compressible Navier-Stokes equations
 * (Mossier, Kopper, Keim, Beck, Munz; arXiv 2502.19342).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package's smoke check
 * and the benchmark's CPU-baseline leg may load this library.  It shares no
 * code with the CUDA path and is written for readability, not speed.
 *
 * Conventions (shared with the CUDA path by specification, not by code):
 *   - State ordering per point: rho_1..rho_Nk, rho*v_x, rho*v_y, rho*v_z, rho*E
 *     (V = Nk + 4 conserved variables; rho = sum_k rho_k).
 *   - Elements are ordered domain by domain, x fastest:
 *     e = first_element(domain) + ix + nx*(iy + ny*iz).
 *   - Element-contiguous state: U[off_e + v*n^3 + i + n*(j + n*k)] with
 *     n = N_e + 1 for DG elements and n = N_FV for FV elements; off_e is the
 *     exclusive prefix sum of V*n_e^3.
 *   - Domains are Cartesian boxes, periodic each on its own or glued along x
 *     into one periodic chain with conforming and mortar interfaces (chain_x).
 */
#ifndef DGFV_ORACLE_H
#define DGFV_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int n_domains;
    const int32_t* dims;   /* 3 per domain: nx, ny, nz                   */
    const double* lo;      /* 3 per domain: lower corner                 */
    const double* hi;      /* 3 per domain: upper corner                 */
    int n_fv;              /* FV sub-cells per direction (global)        */
    int n_species;         /* Nk, 1..3                                   */
    const double* gamma;   /* per species ratio of heat capacities       */
    const double* Rgas;    /* per species specific gas constant          */
    const double* mu;      /* per species dynamic viscosity              */
    const double* Pr;      /* per species Prandtl number                 */
    const double* Dk;      /* per species diffusion coefficient          */
    int riemann;           /* 0 = local Lax-Friedrichs, 1 = Roe + Harten-Hyman, 2 = Roe + Harten-Hyman
                              between DG elements and local Lax-Friedrichs on every face touching FV data */
    const int8_t* N;       /* per element DG degree (kept while FV)      */
    const uint8_t* fv;     /* per element: 1 = FV sub-cell element       */
    int nodes;             /* 0 = Legendre-Gauss, 1 = Legendre-Gauss-Lobatto */
    int split;             /* 1 = split-form volume integral, kinetic-energy-preserving
                              two-point flux (needs nodes = 1), Sec. 3.5     */
    int sutherland;        /* 1 = viscosity mu_mix (T/T_ref)^{3/2} (T_ref+S)/(T+S) (Sec. 4.3) */
    double T_ref;          /* Sutherland reference temperature (> 0)         */
    double S_sutherland;   /* Sutherland constant S (>= 0)                   */
    int indicator_vars;    /* 0: p-adaptation on rho, FV on min(p, Y_k);
                              1: p-adaptation on p, FV on rho (Sec. 4.3)     */
    int pp_limiter;        /* 1 = Zhang-Shu positivity limiter after every RK stage (Sec. 3.5) */
    double pp_eps;         /* its floor for partial densities and internal energy (> 0) */
    int chain_x;           /* 0: every domain a periodic box of its own.  1: the domains are
                              glued in order along x (the +x side of domain i meets the -x side
                              of domain i+1, the last wraps to the first), each periodic in y and
                              z; all share the y and z extents, and neighbouring domains have
                              equal ny, nz (conforming) or twice as many in one or both of them
                              (non-conforming mortar interfaces of types 1-3, Sec. 3.2.3) */
    int fv_own_n;          /* 0: every FV element has n_fv sub-cells per direction.  1: the
                              per-element variant (Sec. 1, the common-DOF scheme of Sonntag and
                              Munz): an FV element of degree N has N+1 sub-cells per direction,
                              so switching between DG and FV keeps its DOF count; n_fv is then
                              unused.  Not with chain_x.                    */
} oracle_problem;

/* 0 on success, negative on a malformed problem. */
int64_t oracle_state_size(const oracle_problem* p);
int oracle_elem_offsets(const oracle_problem* p, int64_t* off);

/* Semi-discrete right-hand side R(U), Sec. 3.1-3.2. */
int oracle_eval_rhs(const oracle_problem* p, const double* U, double* R);

/* The same R(U) evaluated in long double (the reference-element operators
 * stay the double ones): measures the double evaluation's own rounding error. */
int oracle_eval_rhs_extended(const oracle_problem* p, const double* U, double* R);

/* Forward-mode directional derivative dR = R'(U) dU (dual numbers). */
int oracle_eval_rhs_jvp(const oracle_problem* p, const double* U, const double* dU,
                        double* R, double* dR);

/* The same directional derivative with value and derivative carried in long
   double, rounded to double at the end: the rounding-error reference of the
   FP64 tangent (and of adjoints checked against it). */
int oracle_eval_rhs_jvp_extended(const oracle_problem* p, const double* U, const double* dU,
                                 double* R, double* dR);

/* The whole adjoint U_bar = R'(U)^T R_bar, one entry per tangent along a unit
   vector (n evaluations: tiny meshes only).  extended = 0: tangent and sum in
   double; extended = 1: both in long double (the rounding reference). */
int oracle_adjoint_columns(const oracle_problem* p, const double* U, const double* Rbar,
                           int extended, double* Ubar);

/* Floating-point operation count of one evaluation of R(U), counted on the
 * oracle's own arithmetic (abs and comparisons are not counted):
 * out[0] add/sub, out[1] mul, out[2] div, out[3] sqrt, out[4] unused, and per
 * step s = 1..6 of the evaluation (face values, FV sub-cells, lifting value,
 * DG lifting and volume integral, face fluxes, surface integral)
 * out[8 + 4*s + {0,1,2,3}].  out must hold 40 doubles. */
int oracle_count_flops(const oracle_problem* p, const double* U, double* out);

/* Time step of Sec. 3.3 (out: dt, min dt_c, min dt_v). */
int oracle_dt(const oracle_problem* p, const double* U, double cfl_c, double cfl_v,
              double* out3);

/* n_steps SSP-RK3 steps in place; dt_fixed > 0 uses that step, otherwise the
 * CFL step of Sec. 3.3 recomputed from U at the start of every step.
 * dts (optional, n_steps entries) receives the steps taken. */
int oracle_rk3(const oracle_problem* p, double* U, int n_steps, double dt_fixed,
               double cfl_c, double cfl_v, double* dts);

/* One SSP-RK3 step of the scalar ODE u' = lambda*u, through the same stage
 * combination routine as oracle_rk3 (test hook for the stage coefficients). */
double oracle_rk3_scalar_linear(double lambda, double dt, double u0);

/* n_steps steps of the five-stage fourth-order low-storage Runge-Kutta scheme
 * (Sec. 3.3), otherwise as oracle_rk3. */
int oracle_lsrk4(const oracle_problem* p, double* U, int n_steps, double dt_fixed,
                 double cfl_c, double cfl_v, double* dts);

/* Host threads of the oracle's parallel loops (n > 0 sets them); returns the
 * number in use. */
int oracle_set_threads(int n);

/* Positivity limiter of Sec. 3.5 applied once to U in place (floor eps);
 * returns the number of DG elements it changed, or -1. */
int64_t oracle_pp_limit(const oracle_problem* p, double* U, double eps);

/* One low-storage RK4 step of u' = lambda u (kind 0) or u' = -u^2 (kind 1),
 * through the same stage routine as oracle_lsrk4 (test hook). */
double oracle_lsrk4_scalar(int kind, double lambda, double dt, double u0);

/* Modal indicator of Sec. 3.4 per element: Ip = I(rho), Ih = min(I(p), I(Y_k))
 * (indicator_vars 1: Ip = I(p), Ih = I(rho)). */
int oracle_indicator(const oracle_problem* p, const double* U, double* Ip, double* Ih);

/* Adaptation decision per element from Ip, Ih and thresholds
 * thr = {T_fv_on, T_fv_off, T_ref, T_crs}; writes the new N and FV flags. */
int oracle_adapt_decide(const oracle_problem* p, const double* Ip, const double* Ih,
                        const double* thr, int N_min, int N_max,
                        int8_t* N_new, uint8_t* fv_new);

/* State re-layout for new degrees / FV flags (Sec. 3.2 mappings). */
int oracle_remap(const oracle_problem* p_old, const int8_t* N_new, const uint8_t* fv_new,
                 const double* U_old, double* U_new);

/* Reference-element operators (for pins). Matrices are row-major; nodes:
 * 0 = Legendre-Gauss, 1 = Legendre-Gauss-Lobatto. */
int oracle_basis(int N, double* x, double* w, double* D, double* Dhat,
                 double* l_minus, double* l_plus, int nodes);
int oracle_vmap(int N_from, int N_to, double* M, int nodes);   /* (N_to+1) x (N_from+1) */
int oracle_dg2fv(int N, int n_fv, double* M, int nodes);       /* n_fv x (N+1)          */
int oracle_fv2dg(int N, int n_fv, double* M, int nodes);       /* (N+1) x n_fv: pseudo-inverse of
                                                                   V^{DG->FV} (n_fv >= N+1), else the
                                                                   L2 projection of the sub-cell values */
int oracle_fv_overlap(int n_from, int n_to, double* M);         /* n_to x n_from: sub-cell overlaps */
int oracle_leg_vandermonde(int N, double* V, int nodes);       /* V[i][m] = Lhat_m(x_i) */
/* Mortar operators of Sec. 3.2.3 for half s (0: [-1,0], 1: [0,1]): proj = 0 the
 * interpolation to the virtual small side, 1 the L2 projection back; fv = 0 on
 * the nodes of degree N ((N+1) x (N+1)), fv = 1 on N sub-cells (N x N). */
int oracle_mortar(int N, int s, int proj, int fv, double* M, int nodes);

/* Pointwise physics (for pins): convective and viscous flux in direction
 * dir of state u (V) and conservative gradient g (3*V, g[d*V+v] = du_v/dx_d). */
int oracle_flux(const oracle_problem* p, const double* u, const double* g, int dir,
                double* Fc, double* Fv);
int oracle_riemann(const oracle_problem* p, const double* uL, const double* uR, int dir,
                   double* F);
int oracle_primitives(const oracle_problem* p, const double* u, double* out);
/* out: rho, p, T, c, kappa, cv, cp, mu, lambda, Y_1..Y_Nk */

#ifdef __cplusplus
}
#endif
#endif
