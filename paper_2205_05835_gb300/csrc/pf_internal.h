// Internal declarations shared by the CUDA translation units of libpf.
// Nothing here is part of the public ABI (include/pf.h).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace pf {

constexpr int kMaxLevels = 16;
constexpr int kRedBlocks = 152 * 8;   // fixed grid of every reduction kernel (deterministic sums)
constexpr int kThreads = 256;

// Geometry of one grid level (periodic, uniform spacing h). The inverse
// spacings are formed once on the host (a float64 division per cell would run
// on GB300's narrow float64 pipe).
struct Dims {
    int nx, ny, nz;
    int ncell;
    int wall_y;               // 1: free-slip walls at y = 0 and y = ny h (2D), else periodic
    double h;
    double ih, i2h, ih2;      // 1/h, 1/(2h), 1/h^2
    float ihf, i2hf, ih2f;
};
inline Dims make_dims(int nx, int ny, int nz, double h) {
    Dims g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.ncell = nx * ny * nz;
    g.wall_y = 0;
    g.h = h;
    g.ih = 1.0 / h;
    g.i2h = 0.5 / h;
    g.ih2 = 1.0 / (h * h);
    g.ihf = float(g.ih);
    g.i2hf = float(g.i2h);
    g.ih2f = float(g.ih2);
    return g;
}
// the inverse spacings in the arithmetic type of a kernel
__host__ __device__ inline float ih_of(const Dims& g, float) { return g.ihf; }
__host__ __device__ inline double ih_of(const Dims& g, double) { return g.ih; }
__host__ __device__ inline float i2h_of(const Dims& g, float) { return g.i2hf; }
__host__ __device__ inline double i2h_of(const Dims& g, double) { return g.i2h; }
__host__ __device__ inline float ih2_of(const Dims& g, float) { return g.ih2f; }
__host__ __device__ inline double ih2_of(const Dims& g, double) { return g.ih2; }

// Physical and model constants of a context, passed by value to kernels. The
// float copies and differences are formed once on the host so that no kernel
// converts a double per cell (conversions run on GB300's narrow float64 pipe).
struct Phys {
    int dim, model, force;
    int momentum;                         // 0 advective, 1 consistent (conservative) transport
    int fused_stage;                      // 1: 3D float32 stage with the cell pass fused in
    double sigma, eps, rho_in, rho_out, mu_in, mu_out, delta_n;
    double drho, dmu;                     // rho_in - rho_out, mu_in - mu_out
    float sigma_f, eps_f, rho_out_f, drho_f, mu_out_f, dmu_f, delta_n_f;
};

// The constants in the arithmetic type T of a kernel.
template <typename T>
struct PC {
    T sigma, eps, rho_out, drho, mu_out, dmu, delta_n;
};
__host__ __device__ inline PC<float> pc_of(const Phys& p, float) {
    return PC<float>{p.sigma_f, p.eps_f, p.rho_out_f, p.drho_f, p.mu_out_f, p.dmu_f, p.delta_n_f};
}
__host__ __device__ inline PC<double> pc_of(const Phys& p, double) {
    return PC<double>{p.sigma, p.eps, p.rho_out, p.drho, p.mu_out, p.dmu, p.delta_n};
}

// Pointers of the state a stage kernel reads and writes. T is the storage type.
template <typename T>
struct StageIO {
    const T* phi_s;      // stage phase field (read with halo)
    const T* u_s[3];     // stage velocity (read with halo)
    const T* phi_n;      // phi at the step start (own cell)
    const T* u_n[3];
    T* acc_phi;          // RK accumulators
    T* acc_u[3];
    T* phi_out;          // next stage / new phi
    T* u_out[3];         // u* (unprojected)
    const T* nrm[3];     // cell normals of phi_s (scratch)
    const T* aux;        // mu (EB) or kappa (CSF/LCSF/SB/ISODI) of phi_s (scratch)
    const double* gamma; // device scalar
    T* rhs_phi;          // right-hand sides (operator evaluation only)
    T* rhs_u[3];
};

// Scalars of one pressure solve kept on the device. The solve is iterative
// refinement: a float64 outer residual r = f - A x and inner preconditioned CG
// in the storage precision T on A e = r (T = double: the inner CG is the whole
// solve). Reductions write these from the last block of each kernel; the host
// only polls `done` / `idone`.
struct CGScalars {
    double ff;        // ||f||^2 of the right-hand side
    double rr;        // ||f - A x||^2 (float64, true residual)
    double rr0_in;    // ||r_in||^2 at the start of the inner solve
    double rr_in;     // ||r_in||^2 (recursive inner residual)
    double rz, zq, pq, alpha, beta;
    double mean_b;    // mean of the right-hand side (removed)
    double rtol2;     // squared relative tolerance of the solve (set at init)
    double eta2_min;  // squared floor of the inner relative tolerance
    double eta2;      // squared inner relative tolerance of the current outer step
    int maxit;        // cap on inner iterations per solve (set at init)
    int done;         // 1 once converged or stopped (all kernels early-exit)
    int idone;        // 1 once the inner solve stopped (inner kernels early-exit)
    int iters;        // inner iterations of the current / last solve
    int outer;        // outer residual evaluations of the current / last solve
    int status;       // latched device error (pf_status value), 0 if none
    int capped;       // inner iteration cap reached
    int it_in;        // iterations of the current inner solve (device-driven loops)
};

// One multigrid level of the preconditioner.
template <typename T>
struct MGLevel {
    Dims g;
    T* x;          // correction
    T* f;          // right-hand side
    T* beta[3];    // face coefficients 1/rho_f (nullptr on level 0: computed from phi)
    T* x2;         // second correction buffer for out-of-place sweeps (nullptr: in place)
};



// TMA-staged finest-level sweep (pf_sweep_tma.cu): tensor maps of the level-0
// arrays of one context.
struct SweepTMA;

// Coarse levels whose operator is rediscretised from cell densities (the mean
// of the 8 children's) instead of face coefficients averaged from the level
// above (3D float32 path).
constexpr int kDensityLevels = 1;

template <typename T>
struct MGHier {
    const float* rho0 = nullptr;   // float32 cell densities of level 0 (3D mixed path), formed
                                   // once per solve; the finest sweep reads them instead of phi
    float* rhoc[kMaxLevels] = {};  // densities of the tiled levels 1 .. kDensityLevels (mean of the 8
                                   // children's), from which their face coefficients are
                                   // formed (3D mixed path; nullptr elsewhere)
    const SweepTMA* tma = nullptr; // level 0 sweeps staged by the TMA (nullptr: cp.async)
    const SweepTMA* tmac[kMaxLevels] = {};   // the same for the levels l >= 1 with densities
    int nlev;
    int first_coarse;   // levels >= first_coarse are handled by one single-CTA kernel
    int pre, post;
    int coarse_sweeps;
    MGLevel<T> lev[kMaxLevels];
};

// Reduction scratch: partial sums per block and a completion counter.
struct RedBuf {
    double* part;          // kRedPart doubles (partials of up to kRedPart/2 blocks x 2 values)
    unsigned int* counter; // one counter, reset by the last block
};
constexpr int kRedPart = 1 << 17;

// One-pass red-black Gauss-Seidel sweep of a 3D float32 level (pf_mg3d.cu).
bool sweep3d_ok(const Dims& g);
// Sets the sweep kernels' launch attributes (done by the first launch
// otherwise); called before a stream capture.
void sweep3d_prepare();
// Same for the shared-memory coarse-grid kernels.
void coarse_prepare();
long long sweep3d_blocks(const Dims& g);   // CTAs of a tiled sweep / direction kernel
// dots: also form r.z (r = the level's f, z = x_out) and z.q and set the CG
// beta / rz scalars (the work of the CG dot kernel), first: no previous q.
struct SweepDots {
    const float* q;
    RedBuf rb;
    CGScalars* sc;
    int first;
};
// The finest-level sweep staged by the TMA: eligible grids, tensor maps of
// the cell densities rho, the right-hand side f and the two correction buffers
// of level 0 (host object, nullptr when not eligible or the driver lacks the
// encoder), and the launch (false: not launched, use launch_sweep3d). A
// bounded wait that gives up latches PF_ERR_TIMEOUT in the solve's scalars.
// tile: the tile shape of pf_params.sweep_tile (0 .. 4).
bool sweep_tma_ok(const Dims& g);
SweepTMA* sweep_tma_create(const Dims& g, const float* rho, const float* f, const float* xa,
                           const float* xb, int tile);
void sweep_tma_destroy(SweepTMA* t);
void sweep_tma_prepare();
bool launch_sweep_tma(const SweepTMA* t, const MGLevel<float>& L, const float* xin, float* xout,
                      const SweepDots* dots, int first_color, const CGScalars* sc,
                      cudaStream_t s);
// CG direction update and operator product (3D float32, face arrays).
bool dir3d_ok(const Dims& g);
// rho != nullptr: coefficients 2 / (rho_c + rho_q) from the cell densities
// (hardware reciprocal) instead of the face arrays.
void launch_dir3d_reg(const Dims& g, const float* z, const float* p_old, float* p_new, float* q,
                      const float* const* beta, const float* rho, int first, RedBuf rb,
                      CGScalars* sc, cudaStream_t s);
// Float64-accurate outer residual r = sign (b - mean b) - A x of the mixed 3D
// path (x, b double-floats: n hi parts then n lo parts; r float32), one thread
// per column marching in z; also ||f||^2 (first) and ||r||^2 and the solve's
// scalars.
bool ir3d_ok(const Dims& g);
void launch_ir_residual3d(const Dims& g, const float* x, const float* b, const float* const* beta,
                          double sign, float* r, int first, RedBuf rb, CGScalars* sc,
                          cudaStream_t s);
// Restriction (mean of the children's residual) from a 3D float32 level with
// face arrays and even sizes to the next coarser level.
bool restrict3d_ok(const Dims& fine);
// rho != nullptr (finest level): weights 2 / (rho_c + rho_q) from the cell
// densities instead of the level's face arrays.
void launch_restrict3d(const MGLevel<float>& F, const MGLevel<float>& C, const float* rho,
                       const CGScalars* sc, cudaStream_t s);
// The fused stage of the 3D float32 path (pf_stage_fused.cu): cell pass and
// stage in one kernel for CDI / ACDI with the EB force and advective transport.
bool stage_fused_ok(const Dims& g, const Phys& ph);
void stage_fused_prepare();
void launch_stage_fused(const Dims& g, const Phys& ph, const StageIO<float>& io, int stage,
                        int scheme, double wdt, double cdt, int write_rhs, cudaStream_t s);
// Column-marching per-stage kernels for 3D float32 grids (pf_stage3d.cu).
// psi != nullptr (ACDI): normals of psi = acdi_psi(phi), and psi written
void launch_cell_pass_mu3d(const Dims& g, const Phys& ph, const float* phi, float* n0, float* n1,
                           float* n2, float* mu, float* psi, cudaStream_t s);
bool divergence3d_ok(const Dims& g);
void launch_divergence3d(const Dims& g, const float* const* u, double inv_tau, double* b,
                         RedBuf rb, CGScalars* sc, cudaStream_t s);
void launch_correct3d(const Dims& g, const float* const* beta32, const float* const* ustar,
                      const double* p, double tau, float* const* uout, cudaStream_t s);
// phi != nullptr: finest level, smoother weights from rho(phi) (rho_ready: the
// array already holds rho); else the level's face coefficient arrays
void launch_sweep3d(const MGLevel<float>& L, const float* phi, int rho_ready, const Phys& ph,
                    const float* xin,
                    float* xout, const SweepDots* dots, int first_color, const CGScalars* sc,
                    cudaStream_t s);

struct DiagOut {
    double mass, ke, se, umax, phi_min, phi_max;
    double p_in_sum, p_out_sum, n_in, n_out, p_sum;
    double nonfinite;
};

// Kernel classes timed by the optional profiler.
enum KernelClass {
    KC_CELL = 0, KC_STAGE, KC_GAMMA, KC_DIV, KC_CORRECT, KC_COARSEN, KC_GS0, KC_GS,
    KC_RESTRICT, KC_PROLONG, KC_COARSE, KC_IR_RESIDUAL, KC_CG_DOTS, KC_CG_DIR, KC_CG_UPDATE,
    KC_DIAG, KC_MISC, KC_IR_ADDCORR, KC_BETA0, KC_COUNT
};

// Launch counter and optional CUDA-event timer per kernel class. Event pairs
// are harvested at host synchronisation points.
struct Prof {
    bool timing = false;
    long long launches[KC_COUNT] = {};
    double ms[KC_COUNT] = {};
    static constexpr int kPool = 4096;
    cudaEvent_t ev[kPool][2];
    int cls[kPool];
    int used = 0;
    bool created = false;
    cudaStream_t st = nullptr;
    void begin(int k);
    void end();
    void harvest();   // requires the stream to be idle (or synchronises it)
    void destroy();
};

// ---- launch wrappers (defined in the .cu files) ----
template <typename T, int DIM>
void launch_init_phi(const Dims& g, const Phys& ph, double R, int mode, double amp, int shape, T* phi,
                     cudaStream_t s);
template <typename T>
void launch_convert_in(const double* src, T* dst, int n, cudaStream_t s);
template <typename T>
void launch_convert_out(const T* src, double* dst, int n, double shift_from_sum,
                        const double* sum_ptr, double inv_n, cudaStream_t s);

template <typename T, int DIM>
void launch_cell_pass(const Dims& g, const Phys& ph, const T* phi, T* nrm0, T* nrm1, T* nrm2,
                      T* aux, cudaStream_t s);
template <typename T, int DIM>
void launch_stage(const Dims& g, const Phys& ph, const StageIO<T>& io, int stage, int scheme,
                  double wdt, double cdt, int write_rhs, cudaStream_t s);
template <typename T, int DIM>
void launch_gamma(const Dims& g, const T* const* u, double gamma_fixed, double gamma_min,
                  double* gamma, RedBuf rb, cudaStream_t s);
template <typename T, int DIM>
void launch_correct(const Dims& g, const Phys& ph, const T* phi, const double* const* beta64,
                    const float* const* beta32, const T* const* ustar, const double* p,
                    double tau, T* const* uout, cudaStream_t s);
// b = D u / tau; with mom_phi != nullptr, u holds momenta rho_f u and is
// divided by the face densities of mom_phi first (consistent transport).
template <typename T, int DIM>
void launch_divergence(const Dims& g, const T* const* u, double inv_tau, double* b, RedBuf rb,
                       CGScalars* sc, cudaStream_t s, const T* mom_phi = nullptr,
                       const Phys* ph = nullptr);
template <typename T, int DIM>
void launch_diagnostics(const Dims& g, const Phys& ph, const T* phi, const T* const* u,
                        const double* p, RedBuf rb, DiagOut* out, cudaStream_t s);

// Poisson: float64 iterative refinement around multigrid-preconditioned
// flexible CG in precision T.
template <typename T, int DIM>
struct SolveIO {
    const T* phi;          // phase field defining rho
    const double* beta64[3];  // float64 face coefficients (T = double), else nullptr
    const float* beta32[3];   // float32 face coefficients (T = float), else nullptr
    // right-hand side (mean removed on the fly, times sign) and solution (warm
    // start): float64 arrays (T = double) or double-floats in the same 8 n
    // bytes, n hi parts then n lo parts (T = float)
    const double* b;
    double sign;
    double* x;
    T* r;                  // inner residual (= level-0 f of the V-cycle)
    T* z;                  // preconditioned residual (= level-0 x)
    T* p[2];               // search directions (double buffered)
    T* q;                  // A p
    T* e;                  // inner solution (correction of x)
};

template <typename T, int DIM>
void launch_beta0(const Dims& g, const Phys& ph, const T* phi, double* const* beta,
                  cudaStream_t s);
template <int DIM>
void launch_beta0_32(const Dims& g, const Phys& ph, const float* phi, float* const* beta,
                     float* rho, cudaStream_t s);
template <typename T, int DIM>
void launch_mg_setup(const Dims& g0, const Phys& ph, const T* phi, MGHier<T>& H, cudaStream_t s);
// Runs one V-cycle; returns the level-0 buffer that holds the result. With
// dots != nullptr the last level-0 sweep may also perform the CG dot products
// (then *dots_done is set).
template <typename T, int DIM>
T* launch_vcycle(const Phys& ph, const T* phi, MGHier<T>& H, const CGScalars* sc,
                 cudaStream_t s, Prof* pr, const SweepDots* dots = nullptr,
                 bool* dots_done = nullptr);
template <typename T, int DIM>
void launch_ir_residual(const Dims& g, const Phys& ph, const SolveIO<T, DIM>& io, int first,
                        RedBuf rb, CGScalars* sc, cudaStream_t s);
template <typename T, int DIM>
void launch_ir_addcorr(const Dims& g, const SolveIO<T, DIM>& io, CGScalars* sc, cudaStream_t s);
template <typename T, int DIM>
void launch_in_dots(const Dims& g, const SolveIO<T, DIM>& io, int first, RedBuf rb,
                    CGScalars* sc, cudaStream_t s);
template <typename T, int DIM>
void launch_in_dir(const Dims& g, const Phys& ph, const SolveIO<T, DIM>& io, int cur, int first,
                   RedBuf rb, CGScalars* sc, cudaStream_t s);
template <typename T, int DIM>
void launch_in_update(const Dims& g, const SolveIO<T, DIM>& io, int cur, int first, RedBuf rb,
                      CGScalars* sc, cudaStream_t s);
void launch_sum(int n, const double* x, RedBuf rb, double* out, cudaStream_t s);
// Sets the condition of a WHILE node of a captured solve (which = 0: inner CG
// loop, 1: outer refinement loop) from the solve's device scalars.
void launch_set_cond(cudaGraphConditionalHandle h, const CGScalars* sc, int which, cudaStream_t s);
// The mixed path keeps the pressure and the projection's right-hand side as
// double-floats: n float hi parts followed by n float lo parts, in the 8 n
// bytes of a float64 array of n entries.
void launch_double_to_df(const double* src, float* hi, float* lo, int n, cudaStream_t s);
void launch_df_to_double(const float* hi, const float* lo, double* dst, int n, cudaStream_t s);
void launch_sub_mean(double* x, int n, const double* sum_ptr, double inv_n, cudaStream_t s);
// out = 2 a - b elementwise (float64, or double-float planes when df); out may be b
void launch_extrapolate(int n, bool df, const double* a, const double* b, double* out,
                        cudaStream_t s);

// ---- reverse mode (float64; pf_adjoint.cu) ----
// Arrays of the transposed right-hand side of one stage (CDI + EB force).
struct AdjRhsIO {
    const double* phi;        // stage phase field
    const double* u[3];       // stage velocity
    const double* nrm[3];     // cell normals of phi (forward cell pass)
    const double* mu;         // chemical potential of phi (forward cell pass)
    const double* gamma;      // device scalar Gamma of the step
    const double* kbar_phi;   // cotangent of the phase-field rhs (cells)
    const double* kbar_u[3];  // cotangent of the momentum rhs (faces)
    double* lo[3];            // phi cotangent a d-face sends to its high cell
    double* hi[3];            // ... and to its low cell
    double* nfb[3];           // face-normal cotangents
    double* mufb[3];          // face chemical-potential cotangents
    double* rhofb[3];         // face-density cotangents
    double* W[3];             // b_d beta_d (cotangent of visc + force)
    double* te[3];            // edge stress cotangents, pairs (0,1), (0,2), (1,2)
    double* gbar[3];          // cotangent of the central gradient (cells)
    double* mubar;            // cotangent of mu (cells)
    double* phibar_tmp;       // partial phi cotangent
    double* phibar;           // out: phi cotangent (written)
    double* ubar[3];          // out: u cotangent (written)
    double* acc;              // [6] sums: sigma, rho_in, rho_out, mu_in, mu_out, Gamma
};
// Arrays of the transposed projection u = u* - tau beta G p.
struct AdjProjIO {
    const double* phi;        // phase field of the projection's density
    const double* p;          // its pressure
    const double* lam[3];     // cotangent of the projected velocity (faces)
    double* v[3];             // scratch: beta lam
    const double* w;          // A^+ D(beta lam)
    double tau;
    double* mu[3];            // out: cotangent of u* (faces), written
    double* phibar;           // phi cotangent (density part added)
    double* acc;              // [6] parameter sums
};
template <int DIM>
void launch_adj_rhs(const Dims& g, const Phys& ph, const AdjRhsIO& io, RedBuf rb, cudaStream_t s);
template <int DIM>
void launch_adj_beta_lam(const Dims& g, const Phys& ph, const AdjProjIO& io, cudaStream_t s);
template <int DIM>
void launch_adj_proj_post(const Dims& g, const Phys& ph, const AdjProjIO& io, RedBuf rb,
                          cudaStream_t s);
template <int DIM>
void launch_objective(const Dims& g, const Phys& ph, const double* phi, const double* const* u,
                      const double* target, double w_ke, double w_shape, double* gphi,
                      double* const* gu, RedBuf rb, double* J, double* acc, cudaStream_t s);
template <int DIM>
void launch_adj_gamma(const Dims& g, const double* const* u, const double* gamma, double gamma_min,
                      const double* acc, double* const* lam_u, RedBuf rb, cudaStream_t s);
void launch_axpby(int n, double alpha, const double* x, double beta, const double* y, double* out,
                  cudaStream_t s);
void launch_addto(int n, const double* x, double* y, cudaStream_t s);
void launch_add_small(int k, const double* src, double* dst, cudaStream_t s);

}  // namespace pf

struct pf_ctx;
namespace pf {
// Make the context's host waits sleep on a blocking-sync event (pf_capi.cu).
int ctx_set_blocking(pf_ctx* ctx, int on);
// Graph mode: enqueue nsteps captured steps without waiting / wait for them and
// return the latched status (host-driven contexts: step_begin runs the steps).
int ctx_step_begin(pf_ctx* ctx, int nsteps);
int ctx_step_end(pf_ctx* ctx);
}  // namespace pf
