/*
 * pf.h -- C ABI of the GB300 phase-field two-phase flow step.
 *
 * One library call advances a one-fluid, variable-density, incompressible
 * two-phase flow on a uniform periodic staggered grid by one fractional time
 * step. The interface is captured by a second-order conservative phase field
 * phi in [0, 1] (phi = 1 inside the drop) evolved by one of the three models
 * of Table 1 of Mirjalili, Khanwale & Mani (arXiv 2205.05835):
 *   CDI   g = Gamma div[eps grad phi - phi (1 - phi) n]            (Table 1)
 *   SB    g = Gamma [eps lap phi - psi'/eps + eps |grad phi| kappa] (Table 1)
 *   ISODI g = Gamma [eps lap phi - psi'/eps + phi (1 - phi) kappa]  (Table 1)
 * Surface tension enters the momentum equation as one of
 *   EB    F = mu grad phi, mu = (6 sigma/eps) psi' - 6 sigma eps lap phi
 *         (Eq. eb_st with Eq. ac_mu and sigma_hat = 6 sigma, Section 2)
 *   CSF   F = sigma kappa grad phi                                  (Section 2)
 *   LCSF  F = 6 sigma kappa phi (1 - phi) grad phi                  (Eq. equivalence)
 * and the velocity is projected onto divergence-free fields by solving the
 * variable-coefficient Poisson equation div(grad p / rho) = div(u*) / tau
 * with a multigrid-preconditioned conjugate-gradient method.
 * The time integrator is projected RK4 (Section 3) or forward Euler.
 *
 * Conventions (all entry points):
 *  - Every call returns a pf_status; PF_OK is 0. Errors found on the GPU
 *    (non-convergence, non-finite values) are latched in a device status word
 *    and returned by the next call that synchronises (pf_step, pf_project,
 *    pf_diagnostics, pf_get_field, pf_sync).
 *  - Arrays are structure-of-arrays with x the fastest index:
 *    idx = (k * ny + j) * nx + i. Velocity component d lives on the d-faces;
 *    face i - 1/2 along d is stored at the index of cell i. Field arrays passed
 *    across the ABI are float64 with nx*ny*nz entries, in host or device
 *    memory (the library uses unified addressing to tell them apart).
 *  - Memory ownership: the caller allocates the device workspace (size from
 *    pf_workspace_size) and keeps it alive until pf_destroy; the library never
 *    allocates or frees device memory itself and never frees caller memory.
 *    The pf_ctx object is host memory owned by the library (freed by
 *    pf_destroy). A small pinned host buffer is allocated per context.
 *  - Streams: all GPU work of a context is issued on the stream given to
 *    pf_init (a cudaStream_t passed as void*; NULL is the legacy default
 *    stream). Calls on one context are not thread safe.
 */
#ifndef PF_H
#define PF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PF_OK = 0,
    PF_ERR_INVALID = 1,        /* bad parameter, size or pointer */
    PF_ERR_CUDA = 2,           /* a CUDA runtime call failed; see pf_last_error */
    PF_ERR_NOT_CONVERGED = 3,  /* Poisson solve hit poisson_maxit before poisson_rtol */
    PF_ERR_NONFINITE = 4,      /* NaN or Inf found in the state */
    PF_ERR_UNBOUNDED = 5,      /* phi left [-bound_tol, 1 + bound_tol] (when checked) */
    PF_ERR_TIMEOUT = 6,        /* a bounded device wait gave up (TMA-staged sweeps) */
    PF_ERR_WORKSPACE = 7       /* workspace pointer misaligned or too small */
} pf_status;

enum { PF_CDI = 0, PF_SB = 1, PF_ISODI = 2,                /* phase-field model (Table 1) */
       PF_ACDI = 3 };  /* accurate conservative diffuse interface (Jain, J. Comput. Phys. 469,
                          2022; not in the paper): the CDI flux with the sharpening term
                          (1/4)[1 - tanh^2(psi_f / (2 eps))] n_f, psi = eps ln((phi + e0) /
                          (1 - phi + e0)) of clip(phi, 0, 1), e0 = 1e-20, n the normals of psi */
enum { PF_FORCE_EB = 0, PF_FORCE_CSF = 1, PF_FORCE_LCSF = 2 }; /* surface tension force */
enum { PF_FP64 = 0, PF_MIXED = 1 };                         /* precision of stencils and V-cycles */
enum { PF_RK4_PROJ = 0, PF_FE = 1 };                        /* time integrator */
enum { PF_MOMENTUM_ADVECTIVE = 0, PF_MOMENTUM_CONSISTENT = 1 }; /* momentum transport */
enum { PF_SHAPE_DROP = 0, PF_SHAPE_WAVE = 1 };              /* initial phi (pf_params.shape) */
enum { PF_FIELD_PHI = 0, PF_FIELD_U = 1, PF_FIELD_V = 2, PF_FIELD_W = 3, PF_FIELD_P = 4 };

typedef struct {
    int dim;              /* 2 or 3 */
    int n[3];             /* cells per axis (n[2] = 1 in 2D); each >= 4; the box is n[d]*L/n[0] long */
    double L;             /* box length along x; dx = L / n[0] (uniform spacing) */
    int model;            /* PF_CDI, PF_SB, PF_ISODI or PF_ACDI */
    int force;            /* PF_FORCE_EB, PF_FORCE_CSF or PF_FORCE_LCSF */
    int precision;        /* PF_FP64: everything in float64.
                             PF_MIXED: phi, u and the stencils in float32, the double-well
                             psi'(phi) in float64, the Poisson solve as float64 CG with a
                             float32 multigrid preconditioner, reductions in float64 */
    int scheme;           /* PF_RK4_PROJ or PF_FE */
    double sigma;         /* surface tension coefficient */
    double eps;           /* interface thickness parameter epsilon */
    double rho_in, rho_out;  /* densities for phi = 1 and phi = 0; rho linear in clip(phi,0,1) */
    double mu_in, mu_out;    /* dynamic viscosities, linear in clip(phi,0,1) */
    double gamma_fixed;   /* > 0: Gamma fixed; else Gamma = max(gamma_min, max|u^n|) per step */
    double gamma_min;
    double dt;            /* time step */
    double delta_n;       /* regulariser of the normal grad phi / (|grad phi| + delta_n) */
    double poisson_rtol;  /* stop when ||r|| <= rtol * ||rhs|| (float64 residual) */
    int poisson_maxit;    /* iteration cap of each Poisson solve */
    double R;             /* initial drop radius (box centre) */
    int pert_mode;        /* surface perturbation mode n (0: none) */
    double pert_amp;      /* relative amplitude a: R(theta) = R (1 + a cos n theta) [2D],
                             R (1 + a P_n(cos theta)) [3D] */
    int mg_pre, mg_post;  /* red-black Gauss-Seidel sweeps before/after coarse correction, 0..16 (0: 1) */
    double bound_tol;     /* > 0: flag PF_ERR_UNBOUNDED when phi leaves [-tol, 1 + tol] */
    double inner_tol;     /* mixed precision: relative residual reduction of each float32
                             inner solve between float64 refinements (0: 1e-6) */
    int use_graph;        /* 1: pf_step replays one CUDA graph per step (captured at the first
                             pf_step), the pressure solves' CG and refinement loops as
                             device-driven WHILE nodes; no host round trips inside a step.
                             Same results as 0 (host-driven loops). */
    int momentum;         /* PF_MOMENTUM_ADVECTIVE: du/dt = -(u.grad)u + (div tau + F) / rho_f.
                             PF_MOMENTUM_CONSISTENT (CDI model only): rho_f u advanced in
                             conservative form, d(rho_f u)/dt = -div(m u) + div tau + F, with
                             the mass flux m = rho_out u + (rho_in - rho_out) F_CDI consistent
                             with the phase-field flux (the transport the paper's Section 3
                             takes from its reference Mirjalili 2021; the discrete form is this
                             library's). Stage velocities are the new momentum over rho_f. */
    int wall_y;           /* 0: periodic in y. 1 (2D, advective momentum): free-slip walls at
                             y = 0 and y = n[1] dx (Section 3.2 standing wave): zero normal
                             velocity, no flux of phi and a homogeneous Neumann condition on p
                             at the walls; phi, the x-velocity and every other cell-centred
                             quantity mirror across them (zero normal gradient). The y-face of
                             index 0 is the wall (face n[1] wraps to it); it holds v = 0. */
    int shape;            /* initial phi when pf_init gets no phi0: PF_SHAPE_DROP, or
                             PF_SHAPE_WAVE (needs wall_y = 1): phi = 1 below the interface
                             y = R (1 - pert_amp cos(k (x - dx/2))), k = 2 pi pert_mode / (n[0] dx)
                             (R: mean height, pert_amp: amplitude over R) */
    int mg_coarse_cells;  /* multigrid levels of at most this many cells are solved together by
                             one single-CTA V-cycle kernel (0: 4096; else 16 .. 2^20). A
                             tuning knob: it changes the preconditioner, not the converged
                             solution (see the package's autotune module) */
    int sweep_staging;    /* finest-level red-black sweeps of the 3D mixed path: 0 (default)
                             planes staged into shared memory by the Tensor Memory Accelerator
                             (tensor and bulk copies completing on mbarriers) where the grid
                             allows (n[0] % 4 == 0, n[0] >= 40); 1: by per-thread cp.async
                             chunks. Same arithmetic, same results. */
    int stage_kernel;     /* 3D mixed path, CDI or ACDI with the EB force and advective transport:
                             0 (default) one fused kernel per stage forms the normals, mu and
                             psi in shared memory and evaluates the right-hand sides (no HBM
                             round trip of the derived fields; n[0] % 4 == 0, n[0] >= 40,
                             n[1] >= 12); 1: a cell-pass kernel writes them to the workspace
                             and the stage kernel reads them back. Same arithmetic. */
    int sweep_tile;       /* TMA-staged finest sweeps, the CTA's column tile and the cells per
                             thread of zero-start / other sweeps: 0 (default) 32 x 8, two /
                             one; 1: 32 x 8, two; 2: 32 x 16, two; 3: 32 x 16, one; 4: 32 x 8,
                             one (32 x 16 needs n[1] >= 20, else 32 x 8). A tuning knob: every
                             cell gets the same update; only the fused dot products' partial
                             sums are grouped differently. */
    int reserved[1];      /* must be zero */
} pf_params;

typedef struct {
    double mass;          /* sum phi dV */
    double ke;            /* 1/2 sum_faces rho_f u_d^2 dV */
    double se;            /* sum [(6 sigma/eps) psi + 3 sigma eps |grad phi|^2] dV */
    double umax;          /* max |u_d| over all faces */
    double ca_inf;        /* umax * mu_in / sigma (Section 3.1) */
    double dp_laplace;    /* mean(p | phi >= 0.999) - mean(p | phi <= 0.001) */
    double phi_min, phi_max;
    double poisson_relres;/* relative residual of the last Poisson solve */
    double gamma;         /* Gamma used by the last step */
    int poisson_iters;    /* CG iterations of the last Poisson solve */
    int poisson_iters_max;/* largest iteration count since the last pf_diagnostics */
    long long step;
    double t;
} pf_diag;

typedef struct pf_ctx pf_ctx;

/* Bytes of device workspace a context with these parameters needs (256-byte
 * aligned base required). Returns PF_ERR_INVALID for unsupported parameters. */
pf_status pf_workspace_size(const pf_params* prm, size_t* bytes);

/* Create a context on the current CUDA device. workspace: device memory of at
 * least pf_workspace_size bytes, 256-byte aligned, owned by the caller.
 * phi0: optional float64 initial phase field (host or device, nx*ny*nz);
 * NULL computes phi0 = [1 + tanh((R(theta) - r) / (2 eps))] / 2 on the GPU
 * (equilibrium profile, footnote to Eq. ac_mu). Velocity and pressure start at 0.
 * stream: cudaStream_t as void* (NULL: default stream). */
pf_status pf_init(const pf_params* prm, void* workspace, size_t workspace_bytes,
                  const double* phi0, void* stream, pf_ctx** out);

/* Advance nsteps time steps (Gamma from max|u^n| at each step start unless
 * fixed). Synchronises at the end and returns the latched device status. */
pf_status pf_step(pf_ctx* ctx, int nsteps);

/* Project the current velocity onto divergence-free fields with rho(phi) and
 * tau = dt; stores the resulting pressure. */
pf_status pf_project(pf_ctx* ctx);

/* Reductions over the current state (Section 3.1 Ca_inf, Section 3.2 energies);
 * synchronises the stream. */
pf_status pf_diagnostics(pf_ctx* ctx, pf_diag* out);

/* Copy one field out as float64 (PF_FIELD_*; pressure returned with zero mean).
 * dst: host or device memory of nx*ny*nz doubles. Synchronises. */
pf_status pf_get_field(pf_ctx* ctx, int field, double* dst);

/* Overwrite one field from float64 host or device memory (rounded to the
 * storage precision). */
pf_status pf_set_field(pf_ctx* ctx, int field, const double* src);

/* Raw state (phi, u, p, step, t) in storage precision, for checkpoint/restart
 * and host round trips: pf_state_bytes gives the size; dst/src host or device. */
size_t pf_state_bytes(const pf_ctx* ctx);
pf_status pf_get_state(pf_ctx* ctx, void* dst);
pf_status pf_set_state(pf_ctx* ctx, const void* src);

/* Operator-level entry points (used by parity tests).
 * pf_eval_rhs: the phase-field right-hand side (Eq. 1 with Table 1) and the
 * momentum right-hand side without pressure (viscous + advective + F/rho_f) at
 * the current state for a given Gamma; outputs are float64 arrays (host or
 * device) of nx*ny*nz (kphi) and dim*nx*ny*nz (ku, components back to back). */
pf_status pf_eval_rhs(pf_ctx* ctx, double gamma, double* kphi, double* ku);

/* pf_poisson_solve: solve -div(grad x / rho(phi)) = rhs for the current phi
 * (rhs projected to zero mean; x returned with zero mean). rhs, x: float64,
 * host or device. x is also the initial guess. Reports iterations and the
 * final relative residual. */
pf_status pf_poisson_solve(pf_ctx* ctx, const double* rhs, double* x,
                           int* iters, double* relres);

/* Tracing: per kernel class, the number of launches and (when timing is
 * enabled) the summed CUDA-event duration on the context's stream. Launch
 * counts are always kept; timing records an event pair around each launch
 * and is off by default. pf_profile_read fills up to max_entries entries
 * (names are static strings), returns the number of classes, synchronises the
 * stream, and clears the counters when reset != 0. */
typedef struct {
    const char* name;
    long long launches;
    double ms;
} pf_profile_entry;
pf_status pf_profile_enable(pf_ctx* ctx, int enable);
int pf_profile_read(pf_ctx* ctx, pf_profile_entry* out, int max_entries, int reset);

/* Allocation-free pressure solve, for callers that cannot allocate device
 * memory: a host framework whose memory pool owns all device memory (a
 * cudaMalloc of its own would fail or fragment that pool), or a real-time
 * loop that must not allocate after start-up (an allocation may synchronise
 * the device and take unbounded time). It solves the same system as
 * pf_poisson_solve, -div(grad x / rho(phi)) = rhs with the mean of rhs
 * removed and x returned with zero mean, without a context or workspace: all
 * scratch lives in one fixed array inside the library of
 * PF_STATIC_SCRATCH_BYTES (64 MiB), which every GPU that loads the library
 * holds until the process exits. Capacity: about 100 bytes per cell in
 * float64 (about 650k cells, e.g. 80^3 or 512^2) and about 47 bytes per cell
 * in mixed precision (about 1.4M cells, e.g. 112^3); larger grids return
 * PF_ERR_INVALID with the sizes in pf_last_error(NULL).
 * prm: as for pf_init (the fields of the pressure solve are used: dim, n, L,
 * rho_in, rho_out, precision, poisson_rtol, poisson_maxit, mg_pre, mg_post).
 * phi, rhs: float64 device arrays of nx*ny*nz (inputs); x: float64 device
 * array, initial guess on entry and solution on exit. stream: cudaStream_t as
 * void*. Synchronises the stream before returning. iters, relres: optional.
 * Returns PF_ERR_NOT_CONVERGED (x still written) when poisson_maxit is hit.
 * The first call on a device looks up the array's device address (with that
 * device current), so make it before any stream capture. The array keeps the
 * last call's contents and every call clears what must start at zero; calls
 * that overlap on the GPU (two streams or threads at once) share the array and
 * race. The paper has no counterpart: this is a deployment variant of the
 * projection's Poisson solve. */
#define PF_STATIC_SCRATCH_BYTES (64u << 20)
pf_status pf_poisson_solve_static(const pf_params* prm, const double* phi, const double* rhs,
                                  double* x, void* stream, int* iters, double* relres);

/* Batched execution of many independent instances (uneven grid sizes and
 * physical parameters, e.g. a set of drops for a convergence or parameter
 * study). Each instance is a context on its own CUDA stream, carved from one
 * caller-owned workspace (256-byte aligned, pf_batch_workspace_size bytes);
 * pf_batch_step advances every instance by nsteps with a pool of nthreads
 * host threads (0: 16) that hand out instances largest first and sleep in
 * blocking waits, so the kernels of different instances overlap on the GPU.
 * Each instance computes exactly what pf_step computes on its own context.
 * The library creates (and pf_batch_destroy destroys) one stream per instance;
 * it allocates no device memory. When every instance has use_graph = 1, one
 * host thread instead enqueues the captured step graphs of all instances on
 * their streams and then waits for them (no host work inside a step).
 * pf_batch_context gives the context of
 * instance i for pf_get_field / pf_diagnostics (do not pf_destroy it). Returns
 * the first failing instance's status; the text is in pf_batch_last_error. */
typedef struct pf_batch pf_batch;
pf_status pf_batch_workspace_size(const pf_params* prms, int count, size_t* bytes);
pf_status pf_batch_init(const pf_params* prms, int count, void* workspace, size_t workspace_bytes,
                        int nthreads, pf_batch** out);
pf_status pf_batch_step(pf_batch* b, int nsteps);
/* Instance i advances nsteps[i] steps (0: left as is); same execution model. */
pf_status pf_batch_step_each(pf_batch* b, const int* nsteps);
int pf_batch_size(const pf_batch* b);
pf_ctx* pf_batch_context(pf_batch* b, int i);
void pf_batch_destroy(pf_batch* b);
const char* pf_batch_last_error(const pf_batch* b);

/* Reverse mode (discrete adjoint of pf_step), float64 contexts with the CDI
 * model (Table 1) and the EB force (Eq. eb_st with Eq. ac_mu). It gives the
 * gradient of an objective of the state after many steps with respect to the
 * initial phase field, sigma, the densities and the viscosities; the
 * checkpoint schedule (which states to keep) is the caller's.
 *
 * pf_adjoint_workspace_size: bytes of the adjoint workspace (device memory,
 * 256-byte aligned, caller-owned) that pf_step_adjoint needs for these
 * parameters (54 doubles per cell in 2D, 74 in 3D). PF_ERR_INVALID for
 * unsupported parameters (mixed precision, SB / ISODI, CSF / LCSF, consistent
 * momentum transport, walls in y).
 *
 * pf_step_adjoint: transposed Jacobian of one step applied to a cotangent.
 *  state_n: the state at the start of the step in the pf_get_state layout
 *    (host or device), e.g. a checkpoint; the step is recomputed from it, and
 *    on return the context holds the state after the step.
 *  lam: device float64 array of (1 + dim) * nx*ny*nz entries, components back
 *    to back (phi, u, v[, w]); on entry the cotangent dJ/d(state after the
 *    step), on return dJ/d(state at the start of the step).
 *  gparam: device float64[5] or NULL; dJ/d(sigma, rho_in, rho_out, mu_in,
 *    mu_out) of this step is ADDED to it.
 *  The transpose follows the forward arithmetic: the stage right-hand sides
 *  (normals, CDI flux, chemical potential, EB force, advection, viscous
 *  stress, face densities) and each projection u = u* - tau beta G p with
 *  A p = -D u* / tau, whose transpose is mu = lam + G A^+ D(beta lam) (one
 *  Poisson solve with the same operator) plus the density term
 *  (tau/2) sum_f mu_f beta_f^2 (G p)_f through rho(phi). Gamma: fixed when
 *  gamma_fixed > 0; otherwise max(gamma_min, max|u^n|) is differentiated at
 *  the first face (lowest index, x faces first) that attains the maximum.
 *  clip(phi, 0, 1) has derivative 1 strictly inside (0, 1) and 0 elsewhere.
 *  The Poisson solves use poisson_rtol. Synchronises the stream.
 *
 * pf_objective: J = w_ke KE + (w_shape / 2) sum (phi - phi_target)^2 dV of the
 *  current state (KE as in pf_diagnostics; phi_target a device float64 array
 *  or NULL for no misfit term). J is written to host memory; grad (device,
 *  (1 + dim) * nx*ny*nz doubles, layout of lam) receives dJ/d(phi, u); gparam
 *  (device float64[5] or NULL) receives dJ/d(rho_in, rho_out) added to its
 *  entries 1 and 2. Synchronises the stream. */
pf_status pf_adjoint_workspace_size(const pf_params* prm, size_t* bytes);
pf_status pf_step_adjoint(pf_ctx* ctx, void* adj_workspace, size_t adj_bytes, const void* state_n,
                          double* lam, double* gparam);
pf_status pf_objective(pf_ctx* ctx, const double* phi_target, double w_ke, double w_shape,
                       double* J, double* grad, double* gparam);

/* Wait for all work of the context and return the latched device status. */
pf_status pf_sync(pf_ctx* ctx);

void pf_destroy(pf_ctx* ctx);

/* Text of the last error of a context (or of the last failed pf_init when
 * ctx is NULL). Valid until the next call on the context. */
const char* pf_last_error(const pf_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PF_H */
