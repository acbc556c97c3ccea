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
    double* rhs_phi;     // float64 right-hand sides (operator evaluation only)
    double* rhs_u[3];
};

// Scalars of one conjugate-gradient solve kept on the device. Reductions
// write them from the last block of each kernel; no host round trip.
struct CGScalars {
    double ff;        // ||f||^2 of the right-hand side
    double rr;        // ||r||^2
    double rz;        // r.z (current)
    double rz_old;
    double zq;        // z.q (flexible beta)
    double pq;        // p.q
    double alpha, beta;
    double mean_b;    // mean of the divergence (removed)
    double sum_x;
    double rtol2;     // squared relative tolerance (set at init)
    int maxit;        // iteration cap (set at init)
    int done;         // 1 once converged or stopped (kernels early-exit)
    int iters;        // iterations of the current / last solve
    int status;       // latched device error (pf_status value), 0 if none
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
    KC_RESTRICT, KC_PROLONG, KC_COARSE, KC_CG_START, KC_CG_DOTS, KC_CG_DIR, KC_CG_UPDATE,
    KC_DIAG, KC_MISC, KC_COUNT
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
void launch_correct(const Dims& g, const Phys& ph, const T* phi, const T* const* ustar,
                    const double* p, double tau, T* const* uout, cudaStream_t s);
template <typename T, int DIM>
void launch_divergence(const Dims& g, const T* const* u, double inv_tau, double* b, RedBuf rb,
                       CGScalars* sc, cudaStream_t s);
template <typename T, int DIM>
void launch_diagnostics(const Dims& g, const Phys& ph, const T* phi, const T* const* u,
                        const double* p, RedBuf rb, DiagOut* out, cudaStream_t s);

// Poisson (MG-preconditioned flexible CG, float64 outer iteration)
template <typename T, int DIM>
void launch_mg_setup(const Dims& g0, const Phys& ph, const T* phi, MGHier<T>& H, cudaStream_t s);
template <typename T, int DIM>
void launch_vcycle(const Phys& ph, const T* phi, MGHier<T>& H, const CGScalars* sc,
                   cudaStream_t s, Prof* pr);
template <typename T, int DIM>
void launch_cg_start(const Dims& g, const Phys& ph, const T* phi, const double* b, double sign,
                     double* x, double* r, T* rT, RedBuf rb, CGScalars* sc, cudaStream_t s);
template <typename T, int DIM>
void launch_cg_dots(const Dims& g, const T* z, const double* r, const double* q, int first,
                    RedBuf rb, CGScalars* sc, cudaStream_t s);
template <typename T, int DIM>
void launch_cg_dir(const Dims& g, const Phys& ph, const T* phi, const T* z, const double* p_old,
                   double* p_new, double* q, int first, RedBuf rb, CGScalars* sc,
                   cudaStream_t s);
template <typename T, int DIM>
void launch_cg_update(const Dims& g, const double* p, const double* q, double* x, double* r,
                      T* rT, RedBuf rb, CGScalars* sc, cudaStream_t s);
void launch_sum(int n, const double* x, RedBuf rb, double* out, cudaStream_t s);

}  // namespace pf
