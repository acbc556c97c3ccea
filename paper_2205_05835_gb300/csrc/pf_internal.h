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

// Geometry of one grid level (periodic, uniform spacing h).
struct Dims {
    int nx, ny, nz;
    int ncell;
    double h;
};

// Physical and model constants of a context, passed by value to kernels.
struct Phys {
    int dim, model, force;
    double sigma, eps, rho_in, rho_out, mu_in, mu_out, delta_n;
};

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
    int pad;
};

// One multigrid level of the preconditioner.
template <typename T>
struct MGLevel {
    Dims g;
    T* x;          // correction
    T* f;          // right-hand side
    T* beta[3];    // face coefficients 1/rho_f (nullptr on level 0: computed from phi)
};

template <typename T>
struct MGHier {
    int nlev;
    int first_coarse;   // levels >= first_coarse are handled by one single-CTA kernel
    int pre, post;
    int coarse_sweeps;
    MGLevel<T> lev[kMaxLevels];
};

// Reduction scratch: partial sums per block and a completion counter.
struct RedBuf {
    double* part;          // kRedBlocks * 8 doubles
    unsigned int* counter; // one counter, reset by the last block
};

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
void launch_init_phi(const Dims& g, const Phys& ph, double R, int mode, double amp, T* phi,
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
                    const T* const* ustar, const double* p, double tau, T* const* uout,
                    cudaStream_t s);
template <typename T, int DIM>
void launch_divergence(const Dims& g, const T* const* u, double inv_tau, double* b, RedBuf rb,
                       CGScalars* sc, cudaStream_t s);
template <typename T, int DIM>
void launch_diagnostics(const Dims& g, const Phys& ph, const T* phi, const T* const* u,
                        const double* p, RedBuf rb, DiagOut* out, cudaStream_t s);

// Poisson: float64 iterative refinement around multigrid-preconditioned
// flexible CG in precision T.
template <typename T, int DIM>
struct SolveIO {
    const T* phi;          // phase field defining rho
    const double* beta64[3];  // float64 face coefficients (T = double), else nullptr
    const double* b;       // right-hand side (mean removed on the fly, times sign)
    double sign;
    double* x;             // float64 solution (warm start)
    T* r;                  // inner residual (= level-0 f of the V-cycle)
    T* z;                  // preconditioned residual (= level-0 x)
    T* p[2];               // search directions (double buffered)
    T* q;                  // A p
    T* e;                  // inner solution (correction of x)
};

template <typename T, int DIM>
void launch_beta0(const Dims& g, const Phys& ph, const T* phi, double* const* beta,
                  cudaStream_t s);
template <typename T, int DIM>
void launch_mg_setup(const Dims& g0, const Phys& ph, const T* phi, MGHier<T>& H, cudaStream_t s);
template <typename T, int DIM>
void launch_vcycle(const Phys& ph, const T* phi, MGHier<T>& H, const CGScalars* sc,
                   cudaStream_t s, Prof* pr);
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

}  // namespace pf
