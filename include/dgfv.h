/*
 * dgfv -- FP64 CUDA implementation (sm_103a) of the per-stage right-hand side
 * U_t = R(U) of the hp-adaptive hybrid discontinuous-Galerkin / finite-volume
 * operator for the compressible multi-component Navier-Stokes equations
 * (Mossier, Kopper, Keim, Beck, Munz: "Tackling Compressible Turbulent
 * Multi-Component Flows with Dynamic hp-Adaptation", arXiv 2502.19342).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Mesh      One or more independent periodic Cartesian boxes ("domains").
 *           Elements are numbered domain by domain, x fastest:
 *           e = first_element(domain) + ix + nx*(iy + ny*iz).
 * Degrees   Each element has a DG degree N_e in [N_min, N_max] (1..7) and a
 *           flag is_fv_e; an FV element keeps N_e for its return to DG.
 * State     Conserved variables per point, V = Nk + 4:
 *           (rho_1..rho_Nk, rho v_x, rho v_y, rho v_z, rho E).
 *           Element-contiguous structure of arrays, FP64:
 *               U[off_e + v*n^3 + i + n*(j + n*k)]
 *           with n = N_e + 1 Legendre-Gauss nodes (DG) or n = N_FV sub-cell
 *           means (FV) per direction and off_e the exclusive prefix sum of
 *           V*n_e^3 (dgfv_state_layout).
 * Memory    Arguments named d_* are device pointers owned by the caller; the
 *           library never frees them.  The library owns only its scratch
 *           (face buffers, stage buffers, tables), allocated in
 *           dgfv_init_mesh at the capacity of the worst case (every element at
 *           N_max or FV), so no later call allocates device memory.
 * Streams   Every call that takes `stream` (a cudaStream_t, NULL = legacy
 *           default stream) enqueues its work on it and returns without
 *           synchronising, except where a host result is requested.
 * Errors    Every call returns dgfv_status.  Kernels never trap: a detected
 *           problem sets a device status word (the first one wins) with the
 *           element it was found in, which the next synchronising call (or
 *           dgfv_sync_status) reports.  Every Runge-Kutta stage checks the
 *           new state at every node: NaN or Inf gives DGFV_ERR_NONFINITE,
 *           rho <= 0 or rho E - |rho v|^2/(2 rho) <= 0 (p <= 0)
 *           DGFV_ERR_NONPHYSICAL.  The state is left as computed; set a
 *           valid state to go on.  dgfv_last_error gives the message.
 * Devices   A context belongs to the device that was current in
 *           dgfv_init_mesh; every call that touches device memory returns
 *           DGFV_ERR_ARG, before any CUDA work, when another device is current.
 * Threads   One context is used by one host thread and one stream at a time.
 * Tracing   The calls that enqueue work (set_degrees, eval_rhs, compute_dt,
 *           rk_step, rk_steps, rk_step_save, adapt, autotune and the VJPs)
 *           open an NVTX range named after the call on the host timeline of
 *           a profiler that attaches through NVTX; per-kernel device times
 *           come from dgfv_profile_enable / dgfv_profile_read.
 */
#ifndef DGFV_H
#define DGFV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dgfv_ctx dgfv_ctx;

typedef enum {
    DGFV_OK = 0,
    DGFV_ERR_ARG = -1,          /* invalid argument (null, out of range, size mismatch) */
    DGFV_ERR_CUDA = -2,         /* a CUDA runtime call failed                            */
    DGFV_ERR_OOM = -3,          /* device allocation failed                              */
    DGFV_ERR_NONPHYSICAL = -4,  /* density or pressure <= 0 detected                      */
    DGFV_ERR_NONFINITE = -5,    /* NaN or Inf detected in an updated state               */
    DGFV_ERR_TIMEOUT = -6,      /* a bounded device wait gave up                          */
    DGFV_ERR_STATE = -7         /* call order (e.g. rk_step before set_state)             */
} dgfv_status;

/* Convective flux: local Lax-Friedrichs, Roe with the Harten-Hyman entropy fix
 * (Sec. 3.1.1), or Roe-HH between DG elements and LLF on every face that
 * touches FV data (FV sub-cell faces, FV/FV and DG/FV faces), the choice of the
 * jet computation (Sec. 5.1). */
typedef enum { DGFV_RIEMANN_LLF = 0, DGFV_RIEMANN_ROE_HH = 1, DGFV_RIEMANN_HYBRID = 2 } dgfv_riemann;

/* Time integrator of dgfv_rk_step / dgfv_rk_steps: the three-stage SSP-RK3 of
 * Shu and Osher, or the explicit fourth-order low-storage scheme of Sec. 3.3
 * (five stages, 2N storage, Carpenter and Kennedy's coefficients).
 * dgfv_rk_step_vjp supports both; dgfv_rk_step_save and
 * dgfv_rk_step_vjp_stages support SSP-RK3 only. */
typedef enum { DGFV_INTEGRATOR_SSPRK3 = 0, DGFV_INTEGRATOR_LSRK4 = 1 } dgfv_integrator;

/* Mesh: n_domains Cartesian boxes; arrays have 3 entries per domain.
 * chain_x = 0: every domain is a periodic box of its own (batched domains).
 * chain_x = 1: the domains are glued in order along x into one periodic
 *   chain: the +x side of domain i meets the -x side of domain i+1, the last
 *   wraps to the first; each domain stays periodic in y and z.  All domains
 *   share the y and z extents; neighbouring domains have equal ny and nz
 *   (conforming interface) or one has twice as many in one of them (mortar
 *   types 1 and 2) or in both (type 3), Sec. 3.2.3.  The coarser side holds
 *   the big mortar sides.  Other ratios: DGFV_ERR_ARG.
 * Element order: domain by domain, x fastest within a domain. */
typedef struct {
    int n_domains;
    const int32_t* dims;  /* nx, ny, nz per domain (>= 1)               */
    const double* lo;     /* lower corner per domain                    */
    const double* hi;     /* upper corner per domain (hi > lo)          */
    int N_min, N_max;     /* degree bounds, 1 <= N_min <= N_max <= 7    */
    int N_fv;             /* FV sub-cells per direction, N_max+1 <= N_fv <= 9; the
                             sub-cells of one FV element must fit in one CTA's
                             shared memory (N_fv = 9: at most 2 species).
                             N_fv = 0: per-element counts, an FV element of degree
                             N has N+1 sub-cells per direction, so switching between
                             DG and FV keeps its DOFs (the common-DOF scheme the
                             paper contrasts with its own in Sec. 1).  A DG/FV face
                             then couples on the FV side's grid (V^{FV->DG}: the L2
                             projection where that grid has fewer than N+1
                             sub-cells); FV/FV faces of unequal counts on the finer
                             grid, by sub-cell overlaps.  Not with chain_x = 1
                             (DGFV_ERR_ARG). */
    int chain_x;          /* 0 or 1, see above                          */
} dgfv_mesh_desc;

/* Species (Sec. 2): constant properties, ideal-gas mixture, 1 <= n_species <= 3. */
typedef struct {
    int n_species;
    double gamma[3];  /* ratio of heat capacities                   */
    double Rgas[3];   /* specific gas constant                      */
    double mu[3];     /* dynamic viscosity                          */
    double Pr[3];     /* Prandtl number                             */
    double D[3];      /* Fickian diffusion coefficient              */
    int sutherland;   /* 1: mixture viscosity scaled by Sutherland's law
                         (T/T_ref)^{3/2} (T_ref + S)/(T + S) (Sec. 4.3)  */
    double T_ref;     /* Sutherland reference temperature (> 0)     */
    double S;         /* Sutherland constant (>= 0)                 */
} dgfv_phys;

typedef struct {
    int riemann;        /* dgfv_riemann                                        */
    double cfl_c;       /* convective CFL number (Sec. 3.3)                    */
    double cfl_v;       /* viscous CFL number (Sec. 3.3)                       */
    double T_fv_on;     /* DG -> FV when I_h < T_fv_on (Sec. 3.4)              */
    double T_fv_off;    /* FV -> DG when I_h > T_fv_off                        */
    double T_ref;       /* N -> N+1 when I_p < T_ref                           */
    double T_crs;       /* N -> N-1 when I_p > T_crs                           */
    int nodes;          /* DG nodes: 0 Legendre-Gauss, 1 Legendre-Gauss-Lobatto  */
    int split_form;     /* 1: split-form volume integral with the kinetic-energy-
                           preserving two-point flux of Pirozzoli (Sec. 3.5);
                           needs nodes = 1                                    */
    int integrator;     /* dgfv_integrator                                      */
    int indicator_vars; /* 0: p-adaptation on I(rho), FV on min(I(p), I(Y_k));
                           1: p-adaptation on I(p), FV on I(rho) (the TGV of
                           Sec. 4.3)                                          */
    int pp_limiter;     /* 1: Zhang-Shu positivity limiter on every DG element
                           after every Runge-Kutta stage (Sec. 3.5)           */
    double pp_eps;      /* its floor for partial densities and internal energy
                           (> 0 when pp_limiter = 1)                          */
} dgfv_opts;

typedef struct {
    int64_t n_fv;           /* FV elements after the call                      */
    int64_t hist[8];        /* DG elements per degree N (index N) after        */
    int64_t n_changed;      /* elements whose degree or type changed           */
    int64_t n_near;         /* elements whose indicator lies within 1e-10 of a
                               threshold that decided them                     */
    double mean_dofs;       /* mean DOFs (nodes or sub-cells) per element      */
} dgfv_adapt_stats;

/* Creates a context for the mesh, species and options.  All elements start at
 * degree N_min, DG.  Allocates every device buffer the context will need.
 * Errors: DGFV_ERR_ARG, DGFV_ERR_OOM, DGFV_ERR_CUDA. */
int dgfv_init_mesh(dgfv_ctx** ctx, const dgfv_mesh_desc* mesh, const dgfv_phys* phys,
                   const dgfv_opts* opts);

/* Number of elements of the mesh. */
int64_t dgfv_num_elements(const dgfv_ctx* ctx);

/* Sets the degree N[e] and FV flag is_fv[e] of every element (host arrays of
 * dgfv_num_elements entries).  With remap_state != 0 the context's state is
 * mapped to the new pattern (V^{N->M}, V^{DG->FV}, V^{FV->DG}, Sec. 3.2);
 * otherwise the state becomes undefined until dgfv_set_state.  Synchronises.
 * Errors: DGFV_ERR_ARG (degree out of [N_min, N_max]). */
int dgfv_set_degrees(dgfv_ctx* ctx, const int8_t* N, const uint8_t* is_fv, int remap_state);

/* Current degrees and FV flags (host arrays, may be NULL). Synchronises. */
int dgfv_get_degrees(dgfv_ctx* ctx, int8_t* N, uint8_t* is_fv);

/* Size of one state in doubles and the device array of the n_elem element
 * offsets (owned by the context; valid until the pattern changes). */
int dgfv_state_layout(dgfv_ctx* ctx, int64_t* n_doubles, const int64_t** d_elem_offsets);

/* Copies n doubles (must equal the layout size) into / out of the context's
 * state.  d_U is device memory, or host memory for the *_host variants
 * (which synchronise the stream).  Page-locked host memory (cudaHostAlloc,
 * cudaHostRegister, a pinned torch tensor) is copied by a kernel on every SM
 * through its device mapping (full C2C bandwidth also on the first copy after
 * heavy GPU work, when the copy engines first refill the address translations
 * of the buffer's pages); pageable host memory by cudaMemcpyAsync. */
int dgfv_set_state(dgfv_ctx* ctx, const double* d_U, int64_t n, void* stream);
int dgfv_get_state(dgfv_ctx* ctx, double* d_U, int64_t n, void* stream);
int dgfv_set_state_host(dgfv_ctx* ctx, const double* h_U, int64_t n, void* stream);
int dgfv_get_state_host(dgfv_ctx* ctx, double* h_U, int64_t n, void* stream);

/* R = R(U), Eqs. 22 (DG, semidiscrete), 23 (lifting), 26 (FV,
 * semidiscrete_fv), with the interface coupling of Sec. 3.2.1-3.2.2.
 * d_U, d_R: caller-owned device arrays in the current layout; they must not
 * alias.  Allocates nothing. */
int dgfv_eval_rhs(dgfv_ctx* ctx, const double* d_U, double* d_R, void* stream);

/* Time step of Sec. 3.3 for the state d_U: out3 (host) = {dt, min dt_c,
 * min dt_v}.  Synchronises the stream. */
int dgfv_compute_dt(dgfv_ctx* ctx, const double* d_U, double* out3, void* stream);

/* Allocation-free variant of dgfv_compute_dt, for callers that may not
 * allocate device memory when they need a time step: code in a
 * latency-critical loop, where cudaMalloc/cudaFree would synchronise the
 * device, and hosts that own all device memory and forbid allocations after
 * start-up.  The paper has no counterpart; it is an interface of this
 * library.  Same result as dgfv_compute_dt, written to d_out3, a device array
 * of 3 doubles the caller owns ({dt, min dt_c, min dt_v}); nothing is copied
 * to the host and the stream is not synchronised.  The reduction's per-block
 * maxima of the convective and viscous factors (turned into the minimum step
 * by the final pass) live in one fixed device array of 65536 block pairs
 * (1 MiB) that
 * every GPU loading the library holds until the process exits; contexts
 * whose time-step launch needs more blocks get DGFV_ERR_ARG.  The first call
 * on a device looks the array's device address up; make that first call
 * before any stream capture.  All calls share the array: calls that may run
 * at the same time on the GPU (different streams, different contexts) race
 * and must be ordered by the caller.  Allocates nothing. */
int dgfv_compute_dt_noalloc(dgfv_ctx* ctx, const double* d_U, double* d_out3, void* stream);

/* One SSP-RK3 step (Shu-Osher) of the context's state.  dt > 0 uses that
 * step; dt <= 0 uses the CFL step of Sec. 3.3 computed on the device from
 * the state at the start of the step.  dt_used (host, may be NULL) receives
 * the step taken, which synchronises the stream; with NULL the call does not
 * synchronise.  Errors: DGFV_ERR_STATE before the first set_state. */
int dgfv_rk_step(dgfv_ctx* ctx, double dt, double* dt_used, void* stream);

/* n_steps SSP-RK3 steps captured once as a CUDA graph per degree pattern and
 * replayed; same dt semantics as dgfv_rk_step (dt_used = last step). */
int dgfv_rk_steps(dgfv_ctx* ctx, int n_steps, double dt, double* dt_used, void* stream);

/* Adjoint (vector-Jacobian product) of the right-hand side:
 * d_Ubar = (dR/dU)^T d_Rbar at the state d_U, with the degree pattern frozen.
 * The hp/FV pattern is frozen: DG and FV sub-cell elements (the minmod
 * limiter differentiated along the branch the forward evaluation takes), LG
 * or LGL nodes, the standard or the split-form volume integral, every flux
 * choice, constant or Sutherland viscosity, conforming and mortar meshes.
 * Device arrays in the current layout;
 * d_Ubar must not alias d_U or d_Rbar.  Uses the context's forward face
 * buffers (a later eval_rhs recomputes them).  The first adjoint call
 * allocates the adjoint scratch (four face-adjoint buffers and sixteen
 * state-sized buffers: stage states and adjoints, nodal gradient and flux
 * adjoints, FV scratch). */
int dgfv_rhs_vjp(dgfv_ctx* ctx, const double* d_U, const double* d_Rbar, double* d_Ubar, void* stream);

/* Adjoint of one step of size dt of the context's integrator from the state
 * d_U0: d_Ubar = (dU1/dU0)^T d_Ubar_next.  The intermediate stage states are
 * recomputed from d_U0 (stage checkpointing: a caller stores only the state
 * at the start of every step): two for SSP-RK3, four for the low-storage RK4
 * (whose reverse runs the 2N-storage recursion backwards).  Same
 * restrictions as dgfv_rhs_vjp, and no positivity limiter; d_Ubar must not
 * alias the inputs. */
int dgfv_rk_step_vjp(dgfv_ctx* ctx, const double* d_U0, double dt, const double* d_Ubar_next, double* d_Ubar,
                     void* stream);

/* One SSP-RK3 step of size dt > 0 of the context's state that also copies the
 * two intermediate stage states U1, U2 into caller-owned device arrays (for
 * dgfv_rk_step_vjp_stages). */
int dgfv_rk_step_save(dgfv_ctx* ctx, double dt, double* d_stage1, double* d_stage2, void* stream);

/* Adjoint of one SSP-RK3 step from stored stage states: d_stages = {U0, U1,
 * U2} (device arrays), otherwise as dgfv_rk_step_vjp without recomputing the
 * stages. */
int dgfv_rk_step_vjp_stages(dgfv_ctx* ctx, const double* const* d_stages, double dt, const double* d_Ubar_next,
                            double* d_Ubar, void* stream);

/* Positivity limiter of Sec. 3.5 (Zhang and Shu) applied once, in place, to
 * the caller's device state d_U (the context's layout): every DG element's
 * partial densities and internal energy are pulled towards the element mean
 * until they are >= min(pp_eps, mean value) at the nodes and face points; the
 * means are unchanged.  *changed (host, may be NULL) receives the number of
 * elements changed (synchronises when non-NULL).  With pp_limiter = 1 the same
 * kernel runs after every stage of dgfv_rk_step / dgfv_rk_steps. */
int dgfv_pp_limit(dgfv_ctx* ctx, double* d_U, int64_t* changed, void* stream);

/* Number of element limitings by the stage limiter since the last reset
 * (reset != 0 clears the counter after reading).  Synchronises. */
int dgfv_pp_count(dgfv_ctx* ctx, int64_t* count, int reset, void* stream);

/* Modal indicator of Sec. 3.4 on the state d_U: per element I_p = I(rho),
 * I_h = min(I(p), I(Y_k)) (device arrays of n_elem doubles, may be NULL) and
 * the decision code (device array of n_elem bytes, may be NULL):
 * 0 keep, 1 DG->FV, 2 FV->DG, 3 N+1, 4 N-1. */
int dgfv_indicator(dgfv_ctx* ctx, const double* d_U, double* d_Ip, double* d_Ih,
                   uint8_t* d_decision, void* stream);

/* Indicator on the context's state, decisions, remap of the state to the new
 * pattern (Sec. 3.2 mappings).  Synchronises.  stats may be NULL. */
int dgfv_adapt(dgfv_ctx* ctx, dgfv_adapt_stats* stats, void* stream);

/* Kernel timing for measurements.  With on != 0 every launch of the
 * library's kernels is bracketed by CUDA events on its stream, and
 * dgfv_rk_steps launches the stages directly instead of replaying its graph.
 * dgfv_profile_read synchronises and returns, per kernel in the order
 *   0 prolong, 1 fv, 2 face_lift, 3 dg_volume, 4 face_flux, 5 surface,
 *   6 dt, 7 indicator, 8 remap,
 * the summed milliseconds and the number of launches since the last
 * dgfv_profile_enable, and the number of kernels written (at most cap). */
int dgfv_profile_enable(dgfv_ctx* ctx, int on);
int dgfv_profile_read(dgfv_ctx* ctx, double* ms, int64_t* launches, int cap);

/* Launch organisation of the element and conforming-face kernels: mode 0 (the
 * default) issues one launch per kernel covering every degree (tiles of
 * elements of one degree, the degree read per tile); mode 1 issues one launch
 * per degree bin, the loop a per-degree implementation would run; mode 2 is
 * mode 0 with the volume kernel persistent: as many CTAs as are resident at
 * once take the tiles of every degree from a work queue, costliest degrees
 * first (standard volume integral; the split form keeps mode 0).  Modes 0 and
 * 1 give identical results; mode 2 agrees with them to rounding (the same
 * element body compiled into another kernel). */
int dgfv_set_launch_mode(dgfv_ctx* ctx, int mode);

/* Shared-memory layout of the FV sub-cell kernel (Sec. 3.1.2, Eq. 26):
 * variant 0 (the default) chooses by the shared memory one element needs
 * (3 where it fits, else 2, else 1); 1 recomputes the central-difference
 * gradient of a sub-cell at each of its faces; 2 keeps every sub-cell's
 * gradient in shared memory (one CTA of 512 threads per SM; falls back to 1
 * where that layout does not fit); 3 keeps them and runs the z faces in a
 * second pass, so that two CTAs of 256 threads fit per SM (N_FV != 8 only;
 * falls back to the automatic choice elsewhere).  2 and 3 give identical
 * results, 1 agrees with them to rounding.  Errors: DGFV_ERR_ARG for another
 * value. */
int dgfv_set_fv_variant(dgfv_ctx* ctx, int variant);

/* Chooses the launch variant of the volume kernel (bit 0: 128 instead of 256
 * threads per CTA; bit 1: a register budget for three instead of two 256-thread
 * CTAs per SM) and then, for every degree present, the number of elements per
 * tile (64 to 2048 nodes per tile), by timing candidates on the context's state;
 * keeps the fastest.  per_tile_out (host, 9 entries, may be NULL) receives the
 * variant in entry 0 and the tile size per point count n = N+1 in entry n.
 * Synchronises. */
int dgfv_autotune(dgfv_ctx* ctx, int* per_tile_out, void* stream);

/* Device status word: DGFV_OK or the first error a kernel recorded (the
 * message names the element); clears it.  Synchronises. */
int dgfv_sync_status(dgfv_ctx* ctx, void* stream);

const char* dgfv_status_string(int status);
const char* dgfv_last_error(const dgfv_ctx* ctx);
void dgfv_destroy(dgfv_ctx* ctx);

/* Operator bank entries, for checks against an independent computation:
 * which = 0 nodes, 1 weights, 2 Dhat (n x n), 3 l(-1), 4 l(+1),
 * 5 V^{N->M} ((M+1) x (N+1)), 6 V^{DG->FV} (N_fv x (N+1); M >= 1: to M
 * sub-cells), 7 V^{FV->DG} ((N+1) x N_fv; M >= 1: from M sub-cells, the L2
 * projection where M < N+1), 8 inverse Legendre Vandermonde, 9 D (n x n),
 * 10 / 11 mortar interpolation to / L2 projection from the virtual small side
 * of half M (0 or 1) ((N+1) x (N+1), Sec. 3.2.3), 12 / 13 the same on the
 * N_fv sub-cells (N_fv x N_fv), 14 the sub-cell overlaps from N+1 to M
 * sub-cells per direction (M x (N+1)), all on the context's node family.
 * Copies the row-major matrix to host memory `out` of `cap` doubles and
 * returns the number of entries, or a negative status. */
int64_t dgfv_bank_entry(dgfv_ctx* ctx, int which, int N, int M, double* out, int64_t cap);

/* Peak FP64 throughput probe: a kernel of independent DFMA chains; returns
 * achieved FMA-flops per second (2 per DFMA) over `iters` iterations.
 * Synchronises. */
double dgfv_probe_dfma(int iters, void* stream);

/* FP64 tensor-core probe: independent mma.sync m8n8k4 f64 chains; returns
 * achieved flops per second (2 per multiply-add) over `iters` iterations.
 * Decides whether the small tensor-product contractions of the volume kernel
 * would gain from FP64 MMA on this GPU.  Synchronises. */
double dgfv_probe_dmma(int iters, void* stream);

#ifdef __cplusplus
}
#endif
#endif
