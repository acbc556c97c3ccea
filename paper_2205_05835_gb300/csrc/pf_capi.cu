// C ABI (include/pf.h) and the host-side orchestration of one fractional step:
// workspace layout, projected RK4 / forward Euler stage sequence, the
// multigrid-preconditioned CG loop, diagnostics and state transfer.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/pf.h"
#include "pf_internal.h"

using namespace pf;

namespace {

thread_local std::string g_init_error;

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

// Sequential carving of the caller's workspace (also used with base == nullptr
// to compute the size).
struct Carver {
    char* base;
    size_t off = 0;
    template <typename T>
    T* take(size_t count) {
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off = align_up(off + count * sizeof(T));
        return p;
    }
};

// A CUDA graph assembled from stream-capture segments and conditional nodes:
// `tail` holds the nodes the next segment or node depends on.
struct GraphBuilder {
    cudaGraph_t g = nullptr;
    std::vector<cudaGraphNode_t> tail;
    cudaError_t begin(cudaStream_t s) {
        return cudaStreamBeginCaptureToGraph(s, g, tail.empty() ? nullptr : tail.data(), nullptr,
                                             tail.size(), cudaStreamCaptureModeRelaxed);
    }
    cudaError_t end(cudaStream_t s) {
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, nullptr, &nd);
        std::vector<cudaGraphNode_t> t;
        if (e == cudaSuccess && deps) t.assign(deps, deps + nd);
        cudaGraph_t out = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(s, &out);
        if (e == cudaSuccess && e2 == cudaSuccess) tail.swap(t);
        return e != cudaSuccess ? e : e2;
    }
};

const char* kClassNames[KC_COUNT] = {
    "cell_pass", "stage", "gamma", "divergence", "correct", "mg_coarsen_beta", "mg_gs_level0",
    "mg_gs_coarse_levels", "mg_restrict", "mg_prolong", "mg_coarse_vcycle", "ir_residual_f64",
    "cg_dots", "cg_dir_spmv", "cg_update", "diagnostics", "misc", "ir_addcorr", "beta0_f64"};

const double kRK4C[4] = {0.0, 0.5, 0.5, 1.0};
const double kRK4W[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};

struct Impl {
    virtual ~Impl() {}
    virtual pf_status set_blocking(bool on) = 0;
    virtual void carve(Carver& cv) = 0;
    virtual void init_phi(const double* phi0) = 0;
    virtual void zero_state() = 0;
    virtual pf_status step(int nsteps) = 0;
    virtual pf_status step_begin(int nsteps) = 0;   // graph mode: enqueue only
    virtual pf_status step_end() = 0;               // graph mode: wait and check
    virtual pf_status project() = 0;
    virtual pf_status diagnostics(pf_diag* out) = 0;
    virtual pf_status get_field(int f, double* dst) = 0;
    virtual pf_status set_field(int f, const double* src) = 0;
    virtual size_t state_bytes() const = 0;
    virtual pf_status get_state(void* dst) = 0;
    virtual pf_status set_state(const void* src) = 0;
    virtual pf_status eval_rhs(double gamma, double* kphi, double* ku) = 0;
    virtual pf_status poisson_solve(const double* rhs, double* x, int* iters, double* relres) = 0;
    virtual pf_status sync() = 0;
    virtual size_t adjoint_bytes() = 0;
    virtual pf_status step_adjoint(void* aws, size_t abytes, const void* state_n, double* lam,
                                   double* gparam) = 0;
    virtual pf_status objective(const double* target, double w_ke, double w_shape, double* J,
                                double* grad, double* gparam) = 0;
    Prof prof;
};

}  // namespace

namespace pf {
void Prof::begin(int k) {
    ++launches[k];
    if (!timing) return;
    if (!created) {
        for (int i = 0; i < kPool; ++i) {
            cudaEventCreate(&ev[i][0]);
            cudaEventCreate(&ev[i][1]);
        }
        created = true;
    }
    if (used == kPool) harvest();
    cls[used] = k;
    cudaEventRecord(ev[used][0], st);
}
void Prof::end() {
    if (!timing) return;
    cudaEventRecord(ev[used][1], st);
    ++used;
}
void Prof::harvest() {
    if (!used) return;
    cudaEventSynchronize(ev[used - 1][1]);
    for (int i = 0; i < used; ++i) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, ev[i][0], ev[i][1]) == cudaSuccess) ms[cls[i]] += t;
    }
    used = 0;
}
void Prof::destroy() {
    if (!created) return;
    for (int i = 0; i < kPool; ++i) {
        cudaEventDestroy(ev[i][0]);
        cudaEventDestroy(ev[i][1]);
    }
    created = false;
}
}  // namespace pf

struct pf_ctx {
    pf_params prm;
    Impl* impl = nullptr;
    std::string err;
};

namespace {

pf_status validate(const pf_params* p, std::string& why) {
    if (!p) { why = "params is NULL"; return PF_ERR_INVALID; }
    if (p->dim != 2 && p->dim != 3) { why = "dim must be 2 or 3"; return PF_ERR_INVALID; }
    long long nc = 1;
    for (int d = 0; d < p->dim; ++d) {
        if (p->n[d] < 4) { why = "each n[d] must be >= 4"; return PF_ERR_INVALID; }
        nc *= p->n[d];
    }
    if (p->dim == 2 && p->n[2] != 1) { why = "n[2] must be 1 in 2D"; return PF_ERR_INVALID; }
    if (nc > (1LL << 30)) { why = "grid too large (more than 2^30 cells)"; return PF_ERR_INVALID; }
    if (p->model < 0 || p->model > 3) { why = "bad model"; return PF_ERR_INVALID; }
    if (p->force < 0 || p->force > 2) { why = "bad force"; return PF_ERR_INVALID; }
    if (p->precision < 0 || p->precision > 1) { why = "bad precision"; return PF_ERR_INVALID; }
    if (p->scheme < 0 || p->scheme > 1) { why = "bad scheme"; return PF_ERR_INVALID; }
    if (!(p->L > 0) || !(p->eps > 0) || !(p->dt > 0) || !(p->rho_in > 0) || !(p->rho_out > 0)) {
        why = "L, eps, dt and densities must be positive";
        return PF_ERR_INVALID;
    }
    if (p->mu_in < 0 || p->mu_out < 0 || p->sigma < 0 || p->delta_n < 0) {
        why = "viscosities, sigma and delta_n must be non-negative";
        return PF_ERR_INVALID;
    }
    if (p->mg_pre < 0 || p->mg_pre > 16 || p->mg_post < 0 || p->mg_post > 16) {
        why = "mg_pre and mg_post must be in [0, 16] (0: one sweep)";
        return PF_ERR_INVALID;
    }
    if (p->inner_tol < 0 || p->inner_tol >= 1) {
        why = "inner_tol must be in [0, 1)";
        return PF_ERR_INVALID;
    }
    if (!(p->poisson_rtol > 0) || p->poisson_maxit < 1) {
        why = "poisson_rtol must be > 0 and poisson_maxit >= 1";
        return PF_ERR_INVALID;
    }
    if (p->use_graph != 0 && p->use_graph != 1) { why = "use_graph must be 0 or 1"; return PF_ERR_INVALID; }
    if (p->momentum != PF_MOMENTUM_ADVECTIVE && p->momentum != PF_MOMENTUM_CONSISTENT) {
        why = "bad momentum transport";
        return PF_ERR_INVALID;
    }
    if (p->momentum == PF_MOMENTUM_CONSISTENT && p->model != PF_CDI) {
        why = "consistent momentum transport needs the CDI model";
        return PF_ERR_INVALID;
    }
    if (p->wall_y != 0 && p->wall_y != 1) { why = "wall_y must be 0 or 1"; return PF_ERR_INVALID; }
    if (p->wall_y == 1 && (p->dim != 2 || p->momentum != PF_MOMENTUM_ADVECTIVE)) {
        why = "walls in y need dim 2 and advective momentum transport";
        return PF_ERR_INVALID;
    }
    if (p->shape != PF_SHAPE_DROP && p->shape != PF_SHAPE_WAVE) {
        why = "bad initial shape";
        return PF_ERR_INVALID;
    }
    if (p->shape == PF_SHAPE_WAVE && p->wall_y != 1) {
        why = "the standing-wave shape needs walls in y";
        return PF_ERR_INVALID;
    }
    if (p->mg_coarse_cells != 0 && (p->mg_coarse_cells < 16 || p->mg_coarse_cells > (1 << 20))) {
        why = "mg_coarse_cells must be 0 or in 16 .. 2^20";
        return PF_ERR_INVALID;
    }
    if (p->sweep_staging != 0 && p->sweep_staging != 1) {
        why = "sweep_staging must be 0 or 1";
        return PF_ERR_INVALID;
    }
    if (p->stage_kernel != 0 && p->stage_kernel != 1) {
        why = "stage_kernel must be 0 or 1";
        return PF_ERR_INVALID;
    }
    if (p->sweep_tile < 0 || p->sweep_tile > 4) {
        why = "sweep_tile must be 0 .. 4";
        return PF_ERR_INVALID;
    }
    for (int i = 0; i < 1; ++i)
        if (p->reserved[i] != 0) { why = "reserved fields must be zero"; return PF_ERR_INVALID; }
    return PF_OK;
}

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            err = std::string(#call) + ": " + cudaGetErrorString(e_);                    \
            return PF_ERR_CUDA;                                                          \
        }                                                                                \
    } while (0)

template <typename T, int DIM>
struct ImplT final : Impl {
    pf_params prm;
    Dims g;
    Phys ph;
    cudaStream_t st;
    std::string& err;
    // fields
    T *phiN, *phiA, *phiB, *accphi;
    T *uN[3], *uS[3], *uStar[3], *accu[3];
    T *nrm[3], *aux;
    double *p, *b;
    double* beta64[3];   // float64 face coefficients (float64 path only)
    float* beta32[3] = {nullptr, nullptr, nullptr};  // float32 face coefficients (mixed path)
    float* rho0 = nullptr;                            // float32 cell densities (3D mixed path)
    T *rT, *z, *pd[2], *qT, *eT;
    MGHier<T> H;
    RedBuf rb;
    CGScalars* sc;
    double* gamma;
    DiagOut* dout;
    double* dsum;
    // pinned host mirrors
    CGScalars* h_sc = nullptr;
    DiagOut* h_dout = nullptr;
    double* h_scalar = nullptr;
    long long nstep = 0;
    double time = 0.0;
    // reverse mode: stage record of one step (phi_0..phi_3, phi^{n+1}; u_0..u_3;
    // the pressures of the four projections) and an explicit solve target
    struct Tape {
        T* phi[5];
        T* u[4][3];
        double* p[4];
    };
    Tape* tape = nullptr;
    double* xsolve = nullptr;
    // Pressure of the first projection of an RK4 step (its solve target); the
    // state's pressure p holds the other three in turn (see one_step).
    double* pw = nullptr;
    // graph mode: the captured step and the builder while capturing
    cudaGraphExec_t gexec = nullptr;
    GraphBuilder* gb = nullptr;
    int pending = 0;          // graph launches enqueued by step_begin
    int last_iters = 0, max_iters = 0;
    double last_relres = 0.0, last_gamma = 0.0;
    int host_status = 0;

    ImplT(const pf_params& p_, cudaStream_t s_, std::string& e_) : prm(p_), st(s_), err(e_) {
        prof.st = s_;
        g = make_dims(prm.n[0], prm.n[1], DIM == 3 ? prm.n[2] : 1, prm.L / prm.n[0]);
        g.wall_y = prm.wall_y;
        ph.dim = DIM;
        ph.model = prm.model;
        ph.force = prm.force;
        ph.momentum = prm.momentum;
        ph.sigma = prm.sigma;
        ph.eps = prm.eps;
        ph.rho_in = prm.rho_in;
        ph.rho_out = prm.rho_out;
        ph.mu_in = prm.mu_in;
        ph.mu_out = prm.mu_out;
        ph.delta_n = prm.delta_n;
        ph.drho = prm.rho_in - prm.rho_out;
        ph.dmu = prm.mu_in - prm.mu_out;
        ph.sigma_f = float(prm.sigma);
        ph.eps_f = float(prm.eps);
        ph.rho_out_f = float(prm.rho_out);
        ph.drho_f = float(prm.rho_in) - float(prm.rho_out);
        ph.mu_out_f = float(prm.mu_out);
        ph.dmu_f = float(prm.mu_in) - float(prm.mu_out);
        ph.delta_n_f = float(prm.delta_n);
        ph.fused_stage = 0;
        if (DIM == 3 && sizeof(T) == sizeof(float) && prm.stage_kernel == 0)
            ph.fused_stage = stage_fused_ok(g, ph) ? 1 : 0;
        for (int d = 0; d < 3; ++d) uN[d] = uS[d] = uStar[d] = accu[d] = nrm[d] = nullptr;
        // multigrid hierarchy geometry
        H.nlev = 1;
        H.lev[0].g = g;
        while (H.nlev < kMaxLevels) {
            const Dims& f = H.lev[H.nlev - 1].g;
            bool ok = (f.nx % 2 == 0) && (f.ny % 2 == 0) && (DIM == 2 || f.nz % 2 == 0) &&
                      f.nx >= 4 && f.ny >= 4 && (DIM == 2 || f.nz >= 4);
            if (!ok) break;
            H.lev[H.nlev].g = make_dims(f.nx / 2, f.ny / 2, DIM == 3 ? f.nz / 2 : 1, f.h * 2.0);
            H.lev[H.nlev].g.wall_y = f.wall_y;
            ++H.nlev;
        }
        for (int l = 0; l < kMaxLevels; ++l) H.lev[l].x2 = nullptr;
        H.first_coarse = H.nlev - 1;
        const int coarse_cells = prm.mg_coarse_cells > 0 ? prm.mg_coarse_cells : 4096;
        for (int l = 0; l < H.nlev; ++l)
            if (H.lev[l].g.ncell <= coarse_cells) { H.first_coarse = l; break; }
        H.pre = prm.mg_pre > 0 ? prm.mg_pre : 1;
        H.post = prm.mg_post > 0 ? prm.mg_post : 1;
        const Dims& cg = H.lev[H.nlev - 1].g;
        int nmax = cg.nx > cg.ny ? cg.nx : cg.ny;
        if (cg.nz > nmax) nmax = cg.nz;
        int sweeps = 4 * nmax * nmax;
        H.coarse_sweeps = sweeps < 8 ? 8 : (sweeps > 2000 ? 2000 : sweeps);
    }

    bool owns_host = false;
    cudaEvent_t sleep_ev = nullptr;   // blocking-sync event (batched execution)

    SweepTMA* tma = nullptr;   // tensor maps of the TMA-staged finest sweep (host object)
    SweepTMA* tmac[kMaxLevels] = {};   // the same for the coarser tiled levels

    ~ImplT() override {
        if (tma) sweep_tma_destroy(tma);
        for (int l = 0; l < kMaxLevels; ++l)
            if (tmac[l]) sweep_tma_destroy(tmac[l]);
        if (gexec) cudaGraphExecDestroy(gexec);
        prof.destroy();
        if (sleep_ev) cudaEventDestroy(sleep_ev);
        if (!owns_host) return;
        if (h_sc) cudaFreeHost(h_sc);
        if (h_dout) cudaFreeHost(h_dout);
        if (h_scalar) cudaFreeHost(h_scalar);
    }

    // The mixed path keeps the pressure p and the projection's right-hand side
    // b as double-floats: n float hi parts, then n float lo parts, in the 8 n
    // bytes of each array (the float64 path keeps them float64).
    static constexpr bool kDF = sizeof(T) == sizeof(float);
    float* df_hi(double* a) { return reinterpret_cast<float*>(a); }
    float* df_lo(double* a) { return reinterpret_cast<float*>(a) + g.ncell; }
    // float64 array src (device) -> double-float planes of dst, through the CG
    // direction buffers (free outside a solve); src and dst may be the same array
    void to_df(const double* src, double* dst) {
        float* t0 = reinterpret_cast<float*>(pd[0]);
        float* t1 = reinterpret_cast<float*>(pd[1]);
        launch_double_to_df(src, t0, t1, g.ncell, st);
        const size_t nb = (size_t)g.ncell * sizeof(float);
        cudaMemcpyAsync(df_hi(dst), t0, nb, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(df_lo(dst), t1, nb, cudaMemcpyDeviceToDevice, st);
    }
    // p with zero mean as float64 into dst (device), through b
    void pressure_out(double* dst) {
        const int n = g.ncell;
        if (kDF) {
            launch_df_to_double(df_hi(p), df_lo(p), b, n, st);
            launch_sum(n, b, rb, dsum, st);
            launch_sub_mean(b, n, dsum, 1.0 / (double)n, st);
        } else {
            launch_sum(n, p, rb, dsum, st);
            launch_convert_out<double>(p, b, n, 0.0, dsum, 1.0 / (double)n, st);
        }
        cudaMemcpyAsync(dst, b, (size_t)n * sizeof(double), cudaMemcpyDefault, st);
    }

    void carve(Carver& cv) override {
        const size_t n = g.ncell;
        phiN = cv.take<T>(n);
        phiA = cv.take<T>(n);
        phiB = cv.take<T>(n);
        accphi = cv.take<T>(n);
        for (int d = 0; d < DIM; ++d) {
            uN[d] = cv.take<T>(n);
            uS[d] = cv.take<T>(n);
            uStar[d] = cv.take<T>(n);
            accu[d] = cv.take<T>(n);
            nrm[d] = cv.take<T>(n);
        }
        aux = cv.take<T>(2 * n);
        p = cv.take<double>(n);
        b = cv.take<double>(n);
        pw = prm.scheme == PF_FE ? nullptr : cv.take<double>(n);
        rT = cv.take<T>(n);
        z = cv.take<T>(n);
        pd[0] = cv.take<T>(n);
        pd[1] = cv.take<T>(n);
        qT = cv.take<T>(n);
        eT = cv.take<T>(n);
        for (int d = 0; d < 3; ++d)
            beta64[d] = (sizeof(T) == sizeof(double) && d < DIM) ? cv.take<double>(n) : nullptr;
        for (int d = 0; d < 3; ++d)
            beta32[d] = (sizeof(T) == sizeof(float) && d < DIM) ? cv.take<float>(n) : nullptr;
        if (DIM == 3 && sizeof(T) == sizeof(float)) {
            rho0 = cv.take<float>(n);
            H.rho0 = rho0;
        }
        H.lev[0].x = z;
        H.lev[0].f = rT;
        for (int d = 0; d < 3; ++d)
            H.lev[0].beta[d] = sizeof(T) == sizeof(double) ? reinterpret_cast<T*>(beta64[d])
                                                           : reinterpret_cast<T*>(beta32[d]);
        for (int l = 1; l < H.nlev; ++l) {
            const size_t m = H.lev[l].g.ncell;
            H.lev[l].x = cv.take<T>(m);
            H.lev[l].f = cv.take<T>(m);
            for (int d = 0; d < 3; ++d) H.lev[l].beta[d] = d < DIM ? cv.take<T>(m) : nullptr;
        }
        // second buffers for the one-pass out-of-place sweeps (3D float32 levels
        // below the single-CTA levels)
        if (DIM == 3 && sizeof(T) == sizeof(float))
            for (int l = 0; l < H.first_coarse; ++l)
                H.lev[l].x2 = sweep3d_ok(H.lev[l].g) ? cv.take<T>(H.lev[l].g.ncell) : nullptr;
        // densities of level 1 (3D float32): its operator is rediscretised from
        // them, so its sweeps run the TMA-staged density kernel. Rediscretising
        // levels 2 and 3 as well was measured to cost CG iterations at 384^3
        // (35.6 against 33.2 V-cycles per step), so they keep face arrays
        // coarsened from the level above. (Decided on the level's geometry, not
        // on a pointer: the sizing pass carves from a null base.)
        if (DIM == 3 && sizeof(T) == sizeof(float))
            for (int l = 1; l < H.first_coarse && l <= kDensityLevels; ++l)
                H.rhoc[l] = sweep3d_ok(H.lev[l].g) ? cv.take<float>(H.lev[l].g.ncell) : nullptr;
        rb.part = cv.take<double>(kRedPart);
        rb.counter = cv.take<unsigned int>(4);
        sc = cv.take<CGScalars>(1);
        gamma = cv.take<double>(1);
        dout = cv.take<DiagOut>(1);
        dsum = cv.take<double>(4);
    }

    // Layout of a pressure solve alone (phi plus the solver's vectors), used by
    // the allocation-free entry point; the stage fields stay unset.
    void carve_solver_only(Carver& cv) {
        const size_t n = g.ncell;
        phiN = cv.take<T>(n);
        p = cv.take<double>(n);
        b = cv.take<double>(n);
        rT = cv.take<T>(n);
        z = cv.take<T>(n);
        pd[0] = cv.take<T>(n);
        pd[1] = cv.take<T>(n);
        qT = cv.take<T>(n);
        eT = cv.take<T>(n);
        for (int d = 0; d < 3; ++d)
            beta64[d] = (sizeof(T) == sizeof(double) && d < DIM) ? cv.take<double>(n) : nullptr;
        H.lev[0].x = z;
        H.lev[0].f = rT;
        for (int d = 0; d < 3; ++d)
            H.lev[0].beta[d] = sizeof(T) == sizeof(double) ? reinterpret_cast<T*>(beta64[d]) : nullptr;
        for (int l = 1; l < H.nlev; ++l) {
            const size_t m = H.lev[l].g.ncell;
            H.lev[l].x = cv.take<T>(m);
            H.lev[l].f = cv.take<T>(m);
            for (int d = 0; d < 3; ++d) H.lev[l].beta[d] = d < DIM ? cv.take<T>(m) : nullptr;
        }
        rb.part = cv.take<double>(kRedPart);
        rb.counter = cv.take<unsigned int>(4);
        sc = cv.take<CGScalars>(1);
        dsum = cv.take<double>(4);
    }

    // One pressure solve on the solver-only layout without any allocation:
    // phi, rhs and x are float64 device arrays; host mirrors are caller-provided
    // pageable memory. Everything that must start at zero is cleared here.
    pf_status solve_static(const double* phi_in, const double* rhs, double* x, CGScalars* hsc,
                           int* iters, double* relres) {
        h_sc = hsc;
        const size_t n = g.ncell;
        CK(cudaMemsetAsync(rb.counter, 0, 4 * sizeof(unsigned int), st));
        CGScalars s0;
        memset(&s0, 0, sizeof(s0));
        s0.rtol2 = prm.poisson_rtol * prm.poisson_rtol;
        s0.maxit = prm.poisson_maxit;
        s0.eta2_min = sizeof(T) == sizeof(double) ? 0.0 : inner_eta2();
        CK(cudaMemcpyAsync(sc, &s0, sizeof(CGScalars), cudaMemcpyHostToDevice, st));
        launch_convert_in<T>(phi_in, phiN, (int)n, st);
        CK(cudaMemcpyAsync(b, rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        if (kDF) {
            launch_double_to_df(x, df_hi(p), df_lo(p), (int)n, st);
        } else {
            CK(cudaMemcpyAsync(p, x, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        }
        launch_sum((int)n, b, rb, dsum, st);
        if (kDF) to_df(b, b);
        double sum_b = 0.0;
        CK(cudaMemcpyAsync(&sum_b, dsum, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const double mean_b = sum_b / (double)n;
        CK(cudaMemcpyAsync(&sc->mean_b, &mean_b, sizeof(double), cudaMemcpyHostToDevice, st));
        pf_status s = solve(phiN, 1.0);
        if (iters) *iters = last_iters;
        if (relres) *relres = last_relres;
        if (s != PF_OK && s != PF_ERR_NOT_CONVERGED) {
            h_sc = nullptr;
            return s;
        }
        pressure_out(x);
        CK(cudaStreamSynchronize(st));
        CK(cudaGetLastError());
        h_sc = nullptr;
        return s;
    }

    // squared floor of the inner relative tolerance (mixed path)
    double inner_eta2() const {
        const double t = prm.inner_tol > 0 ? prm.inner_tol : 1e-6;
        return t * t;
    }

    pf_status alloc_host() {
        owns_host = true;
        CK(cudaHostAlloc((void**)&h_sc, sizeof(CGScalars), cudaHostAllocDefault));
        CK(cudaHostAlloc((void**)&h_dout, sizeof(DiagOut), cudaHostAllocDefault));
        CK(cudaHostAlloc((void**)&h_scalar, 8 * sizeof(double), cudaHostAllocDefault));
        return PF_OK;
    }

    pf_status init_device() {
        const size_t n = g.ncell;
        // zero everything that must start at zero
        for (int d = 0; d < DIM; ++d) {
            CK(cudaMemsetAsync(uN[d], 0, n * sizeof(T), st));
            CK(cudaMemsetAsync(uS[d], 0, n * sizeof(T), st));
            CK(cudaMemsetAsync(uStar[d], 0, n * sizeof(T), st));
            CK(cudaMemsetAsync(accu[d], 0, n * sizeof(T), st));
        }
        CK(cudaMemsetAsync(p, 0, n * sizeof(double), st));
        CK(cudaMemsetAsync(qT, 0, n * sizeof(T), st));
        CK(cudaMemsetAsync(pd[0], 0, n * sizeof(T), st));
        CK(cudaMemsetAsync(pd[1], 0, n * sizeof(T), st));
        CK(cudaMemsetAsync(eT, 0, n * sizeof(T), st));
        CK(cudaMemsetAsync(aux, 0, 2 * n * sizeof(T), st));
        CK(cudaMemsetAsync(rb.counter, 0, 4 * sizeof(unsigned int), st));
        CGScalars s0;
        memset(&s0, 0, sizeof(s0));
        s0.rtol2 = prm.poisson_rtol * prm.poisson_rtol;
        s0.maxit = prm.poisson_maxit;
        // inner relative tolerance floor: float32 inner solves gain ~4 digits per
        // outer step; float64 inner solves go straight to the final tolerance
        s0.eta2_min = sizeof(T) == sizeof(double) ? 0.0 : inner_eta2();
        *h_sc = s0;
        CK(cudaMemcpyAsync(sc, h_sc, sizeof(CGScalars), cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(gamma, 0, sizeof(double), st));
        CK(cudaStreamSynchronize(st));
        // finest-level sweeps staged by the TMA (3D mixed path; the rest of the
        // hierarchy keeps the cp.async sweeps)
        if (DIM == 3 && sizeof(T) == sizeof(float) && rho0 != nullptr && H.lev[0].x2 != nullptr &&
            prm.sweep_staging == 0 && H.first_coarse > 0) {
            tma = sweep_tma_create(g, rho0, reinterpret_cast<const float*>(H.lev[0].f),
                                   reinterpret_cast<const float*>(H.lev[0].x),
                                   reinterpret_cast<const float*>(H.lev[0].x2),
                                   prm.sweep_tile);
            H.tma = tma;
            // the coarser tiled levels with densities too
            for (int l = 1; l < H.first_coarse; ++l) {
                if (H.rhoc[l] == nullptr) continue;
                tmac[l] = sweep_tma_create(H.lev[l].g, H.rhoc[l],
                                           reinterpret_cast<const float*>(H.lev[l].f),
                                           reinterpret_cast<const float*>(H.lev[l].x),
                                           reinterpret_cast<const float*>(H.lev[l].x2),
                                           prm.sweep_tile);
                H.tmac[l] = tmac[l];
            }
        }
        return PF_OK;
    }

    void init_phi(const double* phi0) override {
        if (phi0) {
            // stage through b (float64 device buffer) so host or device sources work
            cudaMemcpyAsync(b, phi0, g.ncell * sizeof(double), cudaMemcpyDefault, st);
            launch_convert_in<T>(b, phiN, g.ncell, st);
        } else {
            launch_init_phi<T, DIM>(g, ph, prm.R, prm.pert_mode, prm.pert_amp, prm.shape, phiN,
                                    st);
        }
    }

    void zero_state() override {}

    // ---------------- projection ----------------
    // u_out = u_in - tau beta G p with D(beta G p) = D u_in / tau (phi -> rho)
    // mom: uin holds the momentum rho_f u* of consistent transport (the RK
    // stages), divided by rho_f(phi) on the fly; else a velocity
    pf_status do_project(const T* phi, T* const* uin, double tau, T* const* uout,
                         bool mom = false) {
        const T* uin_c[3] = {uin[0], uin[1], DIM == 3 ? uin[2] : uin[0]};
        Phys phc = ph;
        phc.momentum = mom ? 1 : 0;
        prof.begin(KC_DIV);
        launch_divergence<T, DIM>(g, uin_c, 1.0 / tau, b, rb, sc, st, mom ? phi : nullptr, &phc);
        prof.end();
        pf_status s = solve(phi, -1.0);
        if (s != PF_OK) return s;
        prof.begin(KC_CORRECT);
        launch_correct<T, DIM>(g, phc, phi, sizeof(T) == sizeof(double) ? beta64 : nullptr,
                               beta32[0] ? beta32 : nullptr, uin_c, xsolve ? xsolve : p, tau,
                               uout, st);
        prof.end();
        return PF_OK;
    }

    SolveIO<T, DIM> solve_io(const T* phi, double sign) {
        SolveIO<T, DIM> io;
        io.phi = phi;
        for (int d = 0; d < 3; ++d) io.beta64[d] = sizeof(T) == sizeof(double) ? beta64[d] : nullptr;
        for (int d = 0; d < 3; ++d) io.beta32[d] = sizeof(T) == sizeof(float) ? beta32[d] : nullptr;
        io.b = b;
        io.sign = sign;
        io.x = xsolve ? xsolve : p;
        io.r = rT;
        io.z = z;
        io.p[0] = pd[0];
        io.p[1] = pd[1];
        io.q = qT;
        io.e = eT;
        return io;
    }

    pf_status poll() {
        CK(cudaMemcpyAsync(h_sc, sc, sizeof(CGScalars), cudaMemcpyDeviceToHost, st));
        if (sleep_ev) {
            // the calling thread sleeps instead of spinning (many contexts per thread pool)
            CK(cudaEventRecord(sleep_ev, st));
            CK(cudaEventSynchronize(sleep_ev));
        } else {
            CK(cudaStreamSynchronize(st));
        }
        prof.harvest();
        return PF_OK;
    }

    // A x = sign (b - mean b): float64 iterative refinement around inner
    // MG-preconditioned CG in T, warm start from x = p
    // one inner CG iteration: V-cycle (with the CG dot products fused into its
    // last sweep where possible), direction and operator product, update.
    // first < 0: the kernels read "first iteration" from the device counter.
    void cg_iter(SolveIO<T, DIM>& io, const T* phi, int cur, int first) {
        SweepDots sd;
        sd.q = reinterpret_cast<const float*>(qT);
        sd.rb = rb;
        sd.sc = sc;
        sd.first = first;
        bool dots_done = false;
        io.z = launch_vcycle<T, DIM>(ph, phi, H, sc, st, &prof, &sd, &dots_done);
        if (!dots_done) {
            prof.begin(KC_CG_DOTS);
            launch_in_dots<T, DIM>(g, io, first, rb, sc, st);
            prof.end();
        }
        prof.begin(KC_CG_DIR);
        if (DIM == 3 && sizeof(T) == sizeof(float) && beta32[0] != nullptr && dir3d_ok(g)) {
            const float* bl[3] = {beta32[0], beta32[1], beta32[2]};
            launch_dir3d_reg(g, reinterpret_cast<const float*>(io.z),
                             reinterpret_cast<const float*>(cur ? pd[1] : pd[0]),
                             reinterpret_cast<float*>(cur ? pd[0] : pd[1]),
                             reinterpret_cast<float*>(qT), bl, rho0, first, rb, sc, st);
        } else {
            launch_in_dir<T, DIM>(g, ph, io, cur, first, rb, sc, st);
        }
        prof.end();
        prof.begin(KC_CG_UPDATE);
        launch_in_update<T, DIM>(g, io, cur, first, rb, sc, st);
        prof.end();
    }

    // operator setup and the first outer residual of a solve
    void solve_prologue(SolveIO<T, DIM>& io, const T* phi) {
        if (sizeof(T) == sizeof(double)) {
            prof.begin(KC_BETA0);
            launch_beta0<T, DIM>(g, ph, phi, beta64, st);
            prof.end();
        } else if (beta32[0] != nullptr) {
            prof.begin(KC_BETA0);
            launch_beta0_32<DIM>(g, ph, reinterpret_cast<const float*>(phi), beta32, rho0, st);
            prof.end();
        }
        prof.begin(KC_COARSEN);
        launch_mg_setup<T, DIM>(g, ph, phi, H, st);
        prof.end();
        prof.begin(KC_IR_RESIDUAL);
        launch_ir_residual<T, DIM>(g, ph, io, 1, rb, sc, st);
        prof.end();
    }
    // x += e and the next outer residual
    void solve_refine(SolveIO<T, DIM>& io) {
        prof.begin(KC_IR_ADDCORR);
        launch_ir_addcorr<T, DIM>(g, io, sc, st);
        prof.end();
        prof.begin(KC_IR_RESIDUAL);
        launch_ir_residual<T, DIM>(g, ph, io, 0, rb, sc, st);
        prof.end();
    }

    // A x = sign (b - mean b): float64 iterative refinement around inner
    // MG-preconditioned CG in T, warm start from x = p
    pf_status solve(const T* phi, double sign) {
        if (gb) return solve_captured(phi, sign);
        SolveIO<T, DIM> io = solve_io(phi, sign);
        solve_prologue(io, phi);
        pf_status ps = poll();
        if (ps != PF_OK) return ps;
        const int poll_every = 2;
        int outer = 0;
        while (!h_sc->done && outer < 64) {
            int cur = 0;
            for (int it = 0; it <= prm.poisson_maxit + poll_every; ++it) {
                cg_iter(io, phi, cur, it == 0 ? 1 : 0);
                cur = 1 - cur;
                if ((it + 1) % poll_every == 0) {
                    ps = poll();
                    if (ps != PF_OK) return ps;
                    if (h_sc->idone || h_sc->done) break;
                }
            }
            solve_refine(io);
            ps = poll();
            if (ps != PF_OK) return ps;
            ++outer;
        }
        CK(cudaGetLastError());
        return solve_status();
    }

    // iteration counts and the latched status of the last solve (h_sc current)
    pf_status solve_status() {
        last_iters = h_sc->iters;
        if (last_iters > max_iters) max_iters = last_iters;
        last_relres = h_sc->ff > 0 ? sqrt(h_sc->rr / h_sc->ff) : 0.0;
        if (!h_sc->done && h_sc->status == 0) h_sc->status = PF_ERR_NOT_CONVERGED;
        if (h_sc->status) {
            int stt = h_sc->status;
            h_sc->status = 0;
            CK(cudaMemsetAsync(&sc->status, 0, sizeof(int), st));
            // a timed-out sweep stopped the solve in the middle of a launch: blocks
            // that started after it may have skipped a grid reduction, so its
            // completion counter is cleared for the next solve
            if (stt == PF_ERR_TIMEOUT)
                CK(cudaMemsetAsync(rb.counter, 0, 4 * sizeof(unsigned int), st));
            err = stt == PF_ERR_NOT_CONVERGED ? "Poisson solve reached poisson_maxit"
                  : stt == PF_ERR_TIMEOUT
                      ? "a bounded wait of the TMA-staged sweep gave up (copies did not land)"
                      : "non-finite value in the Poisson solve";
            return (pf_status)stt;
        }
        return PF_OK;
    }

    // ---------------- graph capture ----------------
    // WHILE node in the graph being built: its condition is set by a kernel
    // just before the node and at the end of every pass of its body (which = 0
    // inner CG loop, 1 outer refinement loop, see launch_set_cond).
    template <typename F>
    pf_status add_while(int which, F body_fn) {
        cudaGraphConditionalHandle h;
        CK(cudaGraphConditionalHandleCreate(&h, gb->g, 0, 0));
        launch_set_cond(h, sc, which, st);
        CK(gb->end(st));
        // (the parameter union has no default constructor: zeroed raw storage)
        alignas(cudaGraphNodeParams) unsigned char np_raw[sizeof(cudaGraphNodeParams)];
        memset(np_raw, 0, sizeof(np_raw));
        cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(np_raw);
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        CK(cudaGraphAddNode(&node, gb->g, gb->tail.empty() ? nullptr : gb->tail.data(), nullptr,
                            gb->tail.size(), &np));
        GraphBuilder body;
        body.g = np.conditional.phGraph_out[0];
        GraphBuilder* outer = gb;
        gb = &body;
        CK(body.begin(st));
        pf_status s = body_fn();
        launch_set_cond(h, sc, which, st);
        cudaError_t e = body.end(st);
        gb = outer;
        if (s != PF_OK) return s;
        CK(e);
        gb->tail.assign(1, node);
        CK(gb->begin(st));
        return PF_OK;
    }

    // the solve inside a graph: refinement loop around the inner CG loop
    // (unrolled by two: the direction buffers alternate), both device-driven
    pf_status solve_captured(const T* phi, double sign) {
        SolveIO<T, DIM> io = solve_io(phi, sign);
        solve_prologue(io, phi);
        return add_while(1, [&]() -> pf_status {
            pf_status s = add_while(0, [&]() -> pf_status {
                cg_iter(io, phi, 0, -1);
                cg_iter(io, phi, 1, -1);
                return PF_OK;
            });
            if (s != PF_OK) return s;
            solve_refine(io);
            return PF_OK;
        });
    }

    // Capture one step into gexec (kernel attributes are set beforehand: no
    // such call runs inside the capture).
    pf_status capture_step() {
        sweep3d_prepare();
        sweep_tma_prepare();
        stage_fused_prepare();
        coarse_prepare();
        // the legacy default stream cannot be captured: record on a private
        // stream (recording runs nothing); the graph replays on the context's
        cudaStream_t own = st, rec = nullptr;
        if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread) {
            CK(cudaStreamSynchronize(st));
            CK(cudaStreamCreateWithFlags(&rec, cudaStreamNonBlocking));
            st = rec;
        }
        GraphBuilder top;
        cudaError_t e = cudaGraphCreate(&top.g, 0);
        const bool timing = prof.timing;
        prof.timing = false;
        gb = &top;
        if (e == cudaSuccess) e = top.begin(st);
        pf_status s = e == cudaSuccess ? one_step() : PF_ERR_CUDA;
        if (gb != &top) s = PF_ERR_CUDA;
        gb = nullptr;
        cudaError_t e2 = top.g ? top.end(st) : cudaErrorInvalidValue;
        prof.timing = timing;
        st = own;
        if (rec) cudaStreamDestroy(rec);
        if (s == PF_OK && e == cudaSuccess && e2 == cudaSuccess)
            e = cudaGraphInstantiate(&gexec, top.g, 0);
        cudaGraphDestroy(top.g);
        if (s != PF_OK || e != cudaSuccess || e2 != cudaSuccess) {
            gexec = nullptr;
            cudaGetLastError();
            if (err.empty()) err = std::string("graph capture failed: ") +
                                   cudaGetErrorString(e != cudaSuccess ? e : e2);
            return s != PF_OK ? s : PF_ERR_CUDA;
        }
        return PF_OK;
    }

    // ---------------- one step ----------------
    pf_status one_step() {
        const double dt = prm.dt;
        const T* uNc[3] = {uN[0], uN[1], DIM == 3 ? uN[2] : uN[0]};
        prof.begin(KC_GAMMA);
        launch_gamma<T, DIM>(g, uNc, prm.gamma_fixed, prm.gamma_min, gamma, rb, st);
        prof.end();
        StageIO<T> io;
        memset(&io, 0, sizeof(io));
        io.phi_n = phiN;
        io.acc_phi = accphi;
        io.gamma = gamma;
        io.aux = aux;
        for (int d = 0; d < 3; ++d) {
            io.u_n[d] = uN[d];
            io.acc_u[d] = accu[d];
            io.u_out[d] = uStar[d];
            io.nrm[d] = nrm[d];
        }
        if (tape) {
            tape_copy(tape->phi[0], phiN);
            for (int d = 0; d < DIM; ++d) tape_copy(tape->u[0][d], uN[d]);
        }
        if (prm.scheme == PF_FE) {
            io.phi_s = phiN;
            for (int d = 0; d < 3; ++d) io.u_s[d] = uN[d];
            io.phi_out = phiA;
            if (!ph.fused_stage) {
                prof.begin(KC_CELL);
                launch_cell_pass<T, DIM>(g, ph, phiN, nrm[0], nrm[1], nrm[2], aux, st);
                prof.end();
            }
            prof.begin(KC_STAGE);
            launch_stage<T, DIM>(g, ph, io, 0, 1, dt, dt, 0, st);
            prof.end();
            pf_status s = do_project(phiA, uStar, dt, uN, prm.momentum == PF_MOMENTUM_CONSISTENT);
            if (tape) {
                tape_copy(tape->phi[1], phiA);
                tape_copy(tape->p[0], p);
            }
            if (gb) {
                // a captured step keeps its buffers: the new phi is copied back
                tape_copy(phiN, static_cast<const T*>(phiA));
            } else {
                T* t = phiN;
                phiN = phiA;
                phiA = t;
            }
            return s;
        }
        T* phin_s[4] = {phiN, phiA, phiB, phiA};
        T* phout[4] = {phiA, phiB, phiA, phiN};
        for (int s = 0; s < 4; ++s) {
            io.phi_s = phin_s[s];
            for (int d = 0; d < 3; ++d) io.u_s[d] = s == 0 ? uN[d] : uS[d];
            io.phi_out = phout[s];
            if (!ph.fused_stage) {
                prof.begin(KC_CELL);
                launch_cell_pass<T, DIM>(g, ph, phin_s[s], nrm[0], nrm[1], nrm[2], aux, st);
                prof.end();
            }
            const double wdt = kRK4W[s] * dt;
            const double cdt = s < 3 ? kRK4C[s + 1] * dt : dt;
            prof.begin(KC_STAGE);
            launch_stage<T, DIM>(g, ph, io, s, 0, wdt, cdt, 0, st);
            prof.end();
            // Initial guesses of the four pressure solves. Projection s carries
            // the pressure of k_s, whose time level is t^n, t^n + dt/2,
            // t^n + dt/2 and (Simpson's mean of the four) t^n + dt/2 + O(dt^2);
            // the state's pressure p is the last projection of the previous
            // step (t^n - dt/2). So projection 0 starts from p, projection 1
            // from the linear extrapolation 2 p_0 - p (second order in dt),
            // projections 2 and 3 from their predecessor. Only the state and
            // this step enter the guess, so a restart from a saved state
            // reproduces the run bit for bit.
            if (s == 0) {
                cudaMemcpyAsync(pw, p, (size_t)g.ncell * sizeof(double), cudaMemcpyDeviceToDevice,
                                st);
                xsolve = pw;
            } else if (s == 1) {
                launch_extrapolate(g.ncell, sizeof(T) == sizeof(float), pw, p, p, st);
            }
            double* xs = xsolve ? xsolve : p;
            pf_status ps = do_project(phout[s], uStar, cdt, s < 3 ? uS : uN,
                                      prm.momentum == PF_MOMENTUM_CONSISTENT);
            xsolve = nullptr;
            if (ps != PF_OK) return ps;
            if (tape) {
                tape_copy(tape->phi[s + 1], phout[s]);
                if (s < 3)
                    for (int d = 0; d < DIM; ++d) tape_copy(tape->u[s + 1][d], uS[d]);
                tape_copy(tape->p[s], xs);
            }
        }
        return PF_OK;
    }


    template <typename Q>
    void tape_copy(Q* dst, const Q* src) {
        cudaMemcpyAsync(dst, src, (size_t)g.ncell * sizeof(Q), cudaMemcpyDeviceToDevice, st);
    }

    pf_status step(int nsteps) override {
        if (prm.use_graph) {
            pf_status s = step_begin(nsteps);
            if (s != PF_OK) return s;
            return step_end();
        }
        for (int k = 0; k < nsteps; ++k) {
            pf_status s = one_step();
            if (s != PF_OK) return s;
            ++nstep;
            time += prm.dt;
        }
        CK(cudaMemcpyAsync(h_scalar, gamma, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        last_gamma = h_scalar[0];
        CK(cudaGetLastError());
        return PF_OK;
    }

    // Graph mode: enqueue nsteps replays of the captured step (captured at the
    // first call); host-driven mode: the steps.
    pf_status step_begin(int nsteps) override {
        if (!prm.use_graph) return step(nsteps);
        if (nsteps <= 0) return PF_OK;
        if (!gexec) {
            pf_status s = capture_step();
            if (s != PF_OK) return s;
        }
        for (int k = 0; k < nsteps; ++k) {
            CK(cudaGraphLaunch(gexec, st));
            ++nstep;
            time += prm.dt;
        }
        pending += nsteps;
        return PF_OK;
    }

    // Waits for the enqueued replays and returns the first latched error of
    // their solves (non-finite values, iteration cap).
    pf_status step_end() override {
        if (!prm.use_graph) return PF_OK;
        CK(cudaMemcpyAsync(h_sc, sc, sizeof(CGScalars), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(h_scalar, gamma, sizeof(double), cudaMemcpyDeviceToHost, st));
        if (sleep_ev) {
            CK(cudaEventRecord(sleep_ev, st));
            CK(cudaEventSynchronize(sleep_ev));
        } else {
            CK(cudaStreamSynchronize(st));
        }
        CK(cudaGetLastError());
        last_gamma = h_scalar[0];
        pending = 0;
        return solve_status();
    }

    pf_status project() override {
        pf_status s = do_project(phiN, uN, prm.dt, uN);
        if (s != PF_OK) return s;
        CK(cudaStreamSynchronize(st));
        return PF_OK;
    }

    pf_status diagnostics(pf_diag* out) override {
        const T* uNc[3] = {uN[0], uN[1], DIM == 3 ? uN[2] : uN[0]};
        prof.begin(KC_DIAG);
        launch_diagnostics<T, DIM>(g, ph, phiN, uNc, p, rb, dout, st);
        prof.end();
        CK(cudaMemcpyAsync(h_dout, dout, sizeof(DiagOut), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        CK(cudaGetLastError());
        const DiagOut& d = *h_dout;
        memset(out, 0, sizeof(*out));
        out->mass = d.mass;
        out->ke = d.ke;
        out->se = d.se;
        out->umax = d.umax;
        out->ca_inf = prm.sigma > 0 ? d.umax * prm.mu_in / prm.sigma : 0.0;
        out->dp_laplace = (d.n_in > 0 && d.n_out > 0) ? d.p_in_sum / d.n_in - d.p_out_sum / d.n_out
                                                      : 0.0;
        out->phi_min = d.phi_min;
        out->phi_max = d.phi_max;
        out->poisson_relres = last_relres;
        out->poisson_iters = last_iters;
        out->poisson_iters_max = max_iters;
        out->gamma = last_gamma;
        out->step = nstep;
        out->t = time;
        max_iters = 0;
        if (d.nonfinite > 0) {
            err = "non-finite value in the state";
            return PF_ERR_NONFINITE;
        }
        if (prm.bound_tol > 0 && (d.phi_min < -prm.bound_tol || d.phi_max > 1.0 + prm.bound_tol)) {
            err = "phi left [-bound_tol, 1 + bound_tol]";
            return PF_ERR_UNBOUNDED;
        }
        return PF_OK;
    }

    T* field_ptr(int f) {
        switch (f) {
            case PF_FIELD_PHI: return phiN;
            case PF_FIELD_U: return uN[0];
            case PF_FIELD_V: return uN[1];
            case PF_FIELD_W: return DIM == 3 ? uN[2] : nullptr;
            default: return nullptr;
        }
    }

    pf_status get_field(int f, double* dst) override {
        if (!dst) { err = "dst is NULL"; return PF_ERR_INVALID; }
        const size_t bytes = (size_t)g.ncell * sizeof(double);
        if (f == PF_FIELD_P) {
            pressure_out(dst);
        } else {
            T* src = field_ptr(f);
            if (!src) { err = "bad field id"; return PF_ERR_INVALID; }
            launch_convert_out<T>(src, b, g.ncell, 0.0, nullptr, 0.0, st);
            CK(cudaMemcpyAsync(dst, b, bytes, cudaMemcpyDefault, st));
        }
        CK(cudaStreamSynchronize(st));
        CK(cudaGetLastError());
        return PF_OK;
    }

    pf_status set_field(int f, const double* src) override {
        if (!src) { err = "src is NULL"; return PF_ERR_INVALID; }
        const size_t bytes = (size_t)g.ncell * sizeof(double);
        CK(cudaMemcpyAsync(b, src, bytes, cudaMemcpyDefault, st));
        if (f == PF_FIELD_P) {
            if (kDF)
                launch_double_to_df(b, df_hi(p), df_lo(p), g.ncell, st);
            else
                CK(cudaMemcpyAsync(p, b, bytes, cudaMemcpyDeviceToDevice, st));
        } else {
            T* dstp = field_ptr(f);
            if (!dstp) { err = "bad field id"; return PF_ERR_INVALID; }
            launch_convert_in<T>(b, dstp, g.ncell, st);
        }
        CK(cudaStreamSynchronize(st));
        CK(cudaGetLastError());
        return PF_OK;
    }

    size_t state_bytes() const override {
        return (size_t)g.ncell * ((1 + DIM) * sizeof(T) + sizeof(double)) + 2 * sizeof(double);
    }

    pf_status get_state(void* dst) override {
        if (!dst) { err = "dst is NULL"; return PF_ERR_INVALID; }
        char* o = static_cast<char*>(dst);
        const size_t nT = (size_t)g.ncell * sizeof(T);
        CK(cudaMemcpyAsync(o, phiN, nT, cudaMemcpyDefault, st));
        o += nT;
        for (int d = 0; d < DIM; ++d) {
            CK(cudaMemcpyAsync(o, uN[d], nT, cudaMemcpyDefault, st));
            o += nT;
        }
        CK(cudaMemcpyAsync(o, p, (size_t)g.ncell * sizeof(double), cudaMemcpyDefault, st));
        o += (size_t)g.ncell * sizeof(double);
        h_scalar[0] = (double)nstep;
        h_scalar[1] = time;
        CK(cudaMemcpyAsync(o, h_scalar, 2 * sizeof(double), cudaMemcpyDefault, st));
        CK(cudaStreamSynchronize(st));
        return PF_OK;
    }

    pf_status set_state(const void* src) override {
        if (!src) { err = "src is NULL"; return PF_ERR_INVALID; }
        const char* o = static_cast<const char*>(src);
        const size_t nT = (size_t)g.ncell * sizeof(T);
        CK(cudaMemcpyAsync(phiN, o, nT, cudaMemcpyDefault, st));
        o += nT;
        for (int d = 0; d < DIM; ++d) {
            CK(cudaMemcpyAsync(uN[d], o, nT, cudaMemcpyDefault, st));
            o += nT;
        }
        CK(cudaMemcpyAsync(p, o, (size_t)g.ncell * sizeof(double), cudaMemcpyDefault, st));
        o += (size_t)g.ncell * sizeof(double);
        CK(cudaMemcpyAsync(h_scalar, o, 2 * sizeof(double), cudaMemcpyDefault, st));
        CK(cudaStreamSynchronize(st));
        nstep = (long long)h_scalar[0];
        time = h_scalar[1];
        return PF_OK;
    }

    pf_status eval_rhs(double gam, double* kphi, double* ku) override {
        if (!kphi || !ku) { err = "NULL output"; return PF_ERR_INVALID; }
        h_scalar[2] = gam;
        CK(cudaMemcpyAsync(gamma, h_scalar + 2, sizeof(double), cudaMemcpyHostToDevice, st));
        StageIO<T> io;
        memset(&io, 0, sizeof(io));
        io.phi_s = phiN;
        io.phi_n = phiN;
        io.acc_phi = accphi;
        io.gamma = gamma;
        io.aux = aux;
        io.phi_out = phiA;
        for (int d = 0; d < 3; ++d) {
            io.u_s[d] = uN[d];
            io.u_n[d] = uN[d];
            io.acc_u[d] = accu[d];
            io.u_out[d] = uStar[d];
            io.nrm[d] = nrm[d];
        }
        // outputs in scratch arrays of the storage type (phiA, u*), then
        // converted to float64 one field at a time through b
        io.rhs_phi = phiA;
        for (int d = 0; d < 3; ++d) io.rhs_u[d] = uStar[d];
        launch_cell_pass<T, DIM>(g, ph, phiN, nrm[0], nrm[1], nrm[2], aux, st);
        launch_stage<T, DIM>(g, ph, io, 0, 0, 0.0, 0.0, 1, st);
        const size_t bytes = (size_t)g.ncell * sizeof(double);
        launch_convert_out<T>(phiA, b, g.ncell, 0.0, nullptr, 0.0, st);
        CK(cudaMemcpyAsync(kphi, b, bytes, cudaMemcpyDefault, st));
        for (int d = 0; d < DIM; ++d) {
            launch_convert_out<T>(uStar[d], b, g.ncell, 0.0, nullptr, 0.0, st);
            CK(cudaMemcpyAsync(ku + (size_t)d * g.ncell, b, bytes, cudaMemcpyDefault, st));
        }
        CK(cudaStreamSynchronize(st));
        CK(cudaGetLastError());
        return PF_OK;
    }

    pf_status poisson_solve(const double* rhs, double* x, int* iters, double* relres) override {
        if (!rhs || !x) { err = "NULL pointer"; return PF_ERR_INVALID; }
        const size_t bytes = (size_t)g.ncell * sizeof(double);
        if (kDF) {
            CK(cudaMemcpyAsync(b, x, bytes, cudaMemcpyDefault, st));
            launch_double_to_df(b, df_hi(p), df_lo(p), g.ncell, st);
        } else {
            CK(cudaMemcpyAsync(p, x, bytes, cudaMemcpyDefault, st));
        }
        CK(cudaMemcpyAsync(b, rhs, bytes, cudaMemcpyDefault, st));
        launch_sum(g.ncell, b, rb, dsum, st);
        // mean_b = sum / n, written into the scalars
        CK(cudaMemcpyAsync(h_scalar + 3, dsum, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        h_scalar[4] = h_scalar[3] / g.ncell;
        CK(cudaMemcpyAsync(&sc->mean_b, h_scalar + 4, sizeof(double), cudaMemcpyHostToDevice, st));
        if (kDF) to_df(b, b);
        pf_status s = solve(phiN, 1.0);
        if (iters) *iters = last_iters;
        if (relres) *relres = last_relres;
        if (s != PF_OK && s != PF_ERR_NOT_CONVERGED) return s;
        pressure_out(x);
        CK(cudaStreamSynchronize(st));
        return s;
    }

    // ---------------- reverse mode (float64, CDI + EB) ----------------
    // Adjoint workspace: the stage record of one step and the cotangent arrays.
    struct AdjWS {
        Tape tp;
        double *Lphi, *Lu[3];        // cotangent of the step's initial state (accumulated)
        double *P4phi, *P4u[3];      // cotangent of phi^{n+1} and of the last u* (kept)
        double *prevPhi, *prevU[3];  // cotangent of phi_{s+1}, u*_{s+1} of the stage above
        double *kphi, *ku[3];        // cotangent of the stage right-hand sides
        double *sphi, *su[3];        // transposed right-hand side outputs
        double *mus[3];              // projection transpose output
        double *v[3], *w;            // beta lam and A^+ D(beta lam)
        AdjRhsIO rio;
        double* acc;                 // [8] parameter and Gamma sums of the step
    };

    bool adjoint_supported(std::string& why) const {
        if (sizeof(T) != sizeof(double)) { why = "the adjoint needs precision PF_FP64"; return false; }
        if (prm.model != PF_CDI || prm.force != PF_FORCE_EB ||
            prm.momentum != PF_MOMENTUM_ADVECTIVE || prm.wall_y != 0) {
            why = "the adjoint supports the periodic CDI model with the EB force and advective "
                  "momentum";
            return false;
        }
        return true;
    }

    void carve_adj(Carver& cv, AdjWS& a) {
        const size_t n = g.ncell;
        memset(&a, 0, sizeof(a));
        for (int s = 0; s < 5; ++s) a.tp.phi[s] = cv.take<T>(n);
        for (int s = 0; s < 4; ++s)
            for (int d = 0; d < DIM; ++d) a.tp.u[s][d] = cv.take<T>(n);
        for (int s = 0; s < 4; ++s) a.tp.p[s] = cv.take<double>(n);
        a.Lphi = cv.take<double>(n);
        a.P4phi = cv.take<double>(n);
        a.prevPhi = cv.take<double>(n);
        a.kphi = cv.take<double>(n);
        a.sphi = cv.take<double>(n);
        a.w = cv.take<double>(n);
        for (int d = 0; d < DIM; ++d) {
            a.Lu[d] = cv.take<double>(n);
            a.P4u[d] = cv.take<double>(n);
            a.prevU[d] = cv.take<double>(n);
            a.ku[d] = cv.take<double>(n);
            a.su[d] = cv.take<double>(n);
            a.mus[d] = cv.take<double>(n);
            a.v[d] = cv.take<double>(n);
            a.rio.lo[d] = cv.take<double>(n);
            a.rio.hi[d] = cv.take<double>(n);
            a.rio.nfb[d] = cv.take<double>(n);
            a.rio.mufb[d] = cv.take<double>(n);
            a.rio.rhofb[d] = cv.take<double>(n);
            a.rio.W[d] = cv.take<double>(n);
            a.rio.gbar[d] = cv.take<double>(n);
        }
        const int npair = DIM == 3 ? 3 : 1;
        for (int q = 0; q < npair; ++q) a.rio.te[q] = cv.take<double>(n);
        a.rio.mubar = cv.take<double>(n);
        a.rio.phibar_tmp = cv.take<double>(n);
        a.acc = cv.take<double>(8);
    }

    size_t adjoint_bytes() override {
        AdjWS a;
        Carver cv{nullptr};
        carve_adj(cv, a);
        return cv.off;
    }

    // transposed right-hand side of stage (phi_s, u_s) applied to (kphi, ku):
    // sphi, su written; parameter and Gamma sums added to acc
    void adj_rhs(AdjWS& a, const double* phis, double* const* us) {
        launch_cell_pass<T, DIM>(g, ph, reinterpret_cast<const T*>(phis), nrm[0], nrm[1], nrm[2],
                                 aux, st);
        AdjRhsIO io = a.rio;
        io.phi = phis;
        for (int d = 0; d < 3; ++d) {
            io.u[d] = d < DIM ? us[d] : nullptr;
            io.nrm[d] = d < DIM ? reinterpret_cast<const double*>(nrm[d]) : nullptr;
            io.kbar_u[d] = d < DIM ? a.ku[d] : nullptr;
            io.ubar[d] = d < DIM ? a.su[d] : nullptr;
        }
        io.mu = reinterpret_cast<const double*>(aux);
        io.gamma = gamma;
        io.kbar_phi = a.kphi;
        io.phibar = a.sphi;
        io.acc = a.acc;
        launch_adj_rhs<DIM>(g, ph, io, rb, st);
    }

    // transposed projection u = P(phi) u* (pressure p, time factor tau) applied
    // to lam: mu = P^T lam written, the density part added to phibar
    pf_status adj_project(AdjWS& a, const double* phis, const double* pr, double tau,
                          double* const* lam, double* const* mu, double* phibar) {
        AdjProjIO io;
        memset(&io, 0, sizeof(io));
        io.phi = phis;
        io.p = pr;
        for (int d = 0; d < DIM; ++d) {
            io.lam[d] = lam[d];
            io.v[d] = a.v[d];
            io.mu[d] = mu[d];
        }
        io.w = a.w;
        io.tau = tau;
        io.phibar = phibar;
        io.acc = a.acc;
        launch_adj_beta_lam<DIM>(g, ph, io, st);
        const T* vc[3] = {reinterpret_cast<const T*>(a.v[0]), reinterpret_cast<const T*>(a.v[1]),
                          reinterpret_cast<const T*>(DIM == 3 ? a.v[2] : a.v[0])};
        launch_divergence<T, DIM>(g, vc, 1.0, b, rb, sc, st);
        // A w = D(beta lam) - mean, from a zero start (a zero right-hand side
        // then ends the solve at once)
        CK(cudaMemsetAsync(a.w, 0, (size_t)g.ncell * sizeof(double), st));
        xsolve = a.w;
        pf_status s = solve(reinterpret_cast<const T*>(phis), 1.0);
        xsolve = nullptr;
        if (s != PF_OK) return s;
        launch_adj_proj_post<DIM>(g, ph, io, rb, st);
        return PF_OK;
    }

    pf_status step_adjoint(void* aws, size_t abytes, const void* state_n, double* lam,
                           double* gparam) override {
        std::string why;
        if (!adjoint_supported(why)) { err = why; return PF_ERR_INVALID; }
        if (!aws || !state_n || !lam) { err = "NULL pointer"; return PF_ERR_INVALID; }
        if ((reinterpret_cast<uintptr_t>(aws) % kAlign) != 0 || abytes < adjoint_bytes()) {
            err = "adjoint workspace NULL, not 256-byte aligned or smaller than pf_adjoint_workspace_size";
            return PF_ERR_WORKSPACE;
        }
        AdjWS a;
        Carver cv{static_cast<char*>(aws)};
        carve_adj(cv, a);
        const size_t n = g.ncell;
        const size_t nb = n * sizeof(double);
        double* lam_phi = lam;
        double* lam_u[3] = {lam + n, lam + 2 * n, DIM == 3 ? lam + 3 * n : nullptr};
        // forward recomputation of the step with its stage record
        pf_status s = set_state(state_n);
        if (s != PF_OK) return s;
        tape = &a.tp;
        s = one_step();
        tape = nullptr;
        if (s != PF_OK) return s;
        ++nstep;
        time += prm.dt;
        CK(cudaMemsetAsync(a.acc, 0, 8 * sizeof(double), st));
        const double dt = prm.dt;
        double* tphi[5];
        double* tu[4][3];
        for (int q = 0; q < 5; ++q) tphi[q] = reinterpret_cast<double*>(a.tp.phi[q]);
        for (int q = 0; q < 4; ++q)
            for (int d = 0; d < 3; ++d)
                tu[q][d] = d < DIM ? reinterpret_cast<double*>(a.tp.u[q][d]) : nullptr;
        // last projection: u^{n+1} = P(phi^{n+1}) u*
        const int last = prm.scheme == PF_FE ? 1 : 4;
        CK(cudaMemcpyAsync(a.P4phi, lam_phi, nb, cudaMemcpyDeviceToDevice, st));
        s = adj_project(a, tphi[last], a.tp.p[last - 1], dt, lam_u, a.P4u, a.P4phi);
        if (s != PF_OK) return s;
        if (prm.scheme == PF_FE) {
            launch_axpby((int)n, dt, a.P4phi, 0.0, nullptr, a.kphi, st);
            for (int d = 0; d < DIM; ++d) launch_axpby((int)n, dt, a.P4u[d], 0.0, nullptr, a.ku[d], st);
            adj_rhs(a, tphi[0], tu[0]);
            launch_axpby((int)n, 1.0, a.P4phi, 1.0, a.sphi, a.Lphi, st);
            for (int d = 0; d < DIM; ++d) launch_axpby((int)n, 1.0, a.P4u[d], 1.0, a.su[d], a.Lu[d], st);
        } else {
            CK(cudaMemcpyAsync(a.Lphi, a.P4phi, nb, cudaMemcpyDeviceToDevice, st));
            for (int d = 0; d < DIM; ++d)
                CK(cudaMemcpyAsync(a.Lu[d], a.P4u[d], nb, cudaMemcpyDeviceToDevice, st));
            for (int sg = 3; sg >= 0; --sg) {
                // cotangent of k_s: from phi^{n+1} / u^{n+1} (weight w_s) and from
                // stage s + 1 (phi_{s+1} = phi^n + c_{s+1} dt k_s)
                const double wdt = kRK4W[sg] * dt;
                const double cdt_up = sg < 3 ? kRK4C[sg + 1] * dt : 0.0;
                launch_axpby((int)n, wdt, a.P4phi, cdt_up, sg < 3 ? a.prevPhi : nullptr, a.kphi, st);
                for (int d = 0; d < DIM; ++d)
                    launch_axpby((int)n, wdt, a.P4u[d], cdt_up, sg < 3 ? a.prevU[d] : nullptr,
                                 a.ku[d], st);
                adj_rhs(a, tphi[sg], tu[sg]);
                if (sg >= 1) {
                    // u_s = P(phi_s) u*_s with tau = c_s dt
                    s = adj_project(a, tphi[sg], a.tp.p[sg - 1], kRK4C[sg] * dt, a.su, a.mus,
                                    a.sphi);
                    if (s != PF_OK) return s;
                    launch_addto((int)n, a.sphi, a.Lphi, st);
                    CK(cudaMemcpyAsync(a.prevPhi, a.sphi, nb, cudaMemcpyDeviceToDevice, st));
                    for (int d = 0; d < DIM; ++d) {
                        launch_addto((int)n, a.mus[d], a.Lu[d], st);
                        CK(cudaMemcpyAsync(a.prevU[d], a.mus[d], nb, cudaMemcpyDeviceToDevice, st));
                    }
                } else {
                    launch_addto((int)n, a.sphi, a.Lphi, st);
                    for (int d = 0; d < DIM; ++d) launch_addto((int)n, a.su[d], a.Lu[d], st);
                }
            }
        }
        // Gamma = max(gamma_min, max |u^n|) (unless fixed)
        if (!(prm.gamma_fixed > 0.0)) {
            const double* u0c[3] = {tu[0][0], tu[0][1], DIM == 3 ? tu[0][2] : tu[0][0]};
            launch_adj_gamma<DIM>(g, u0c, gamma, prm.gamma_min, a.acc, a.Lu, rb, st);
        }
        CK(cudaMemcpyAsync(lam_phi, a.Lphi, nb, cudaMemcpyDeviceToDevice, st));
        for (int d = 0; d < DIM; ++d)
            CK(cudaMemcpyAsync(lam_u[d], a.Lu[d], nb, cudaMemcpyDeviceToDevice, st));
        if (gparam) launch_add_small(5, a.acc, gparam, st);
        CK(cudaStreamSynchronize(st));
        CK(cudaGetLastError());
        return PF_OK;
    }

    pf_status objective(const double* target, double w_ke, double w_shape, double* J,
                        double* grad, double* gparam) override {
        if (sizeof(T) != sizeof(double)) {
            err = "the objective gradient needs precision PF_FP64";
            return PF_ERR_INVALID;
        }
        if (!J || !grad) { err = "NULL pointer"; return PF_ERR_INVALID; }
        const size_t n = g.ncell;
        const double* uc[3] = {reinterpret_cast<const double*>(uN[0]),
                               reinterpret_cast<const double*>(uN[1]),
                               DIM == 3 ? reinterpret_cast<const double*>(uN[2]) : nullptr};
        double* gu[3] = {grad + n, grad + 2 * n, DIM == 3 ? grad + 3 * n : nullptr};
        // parameter sums go to dsum[1..2] when gparam is NULL
        CK(cudaMemsetAsync(dsum, 0, 4 * sizeof(double), st));
        double* acc = gparam ? gparam : dsum;
        launch_objective<DIM>(g, ph, reinterpret_cast<const double*>(phiN), uc, target, w_ke,
                              w_shape, grad, gu, rb, dsum + 3, acc, st);
        CK(cudaMemcpyAsync(h_scalar + 5, dsum + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        CK(cudaGetLastError());
        *J = h_scalar[5];
        return PF_OK;
    }

    pf_status sync() override {
        CK(cudaStreamSynchronize(st));
        CK(cudaGetLastError());
        return PF_OK;
    }

    pf_status set_blocking(bool on) override {
        if (on && !sleep_ev)
            CK(cudaEventCreateWithFlags(&sleep_ev, cudaEventBlockingSync | cudaEventDisableTiming));
        if (!on && sleep_ev) {
            CK(cudaEventDestroy(sleep_ev));
            sleep_ev = nullptr;
        }
        return PF_OK;
    }
};

Impl* make_impl(const pf_params& p, cudaStream_t s, std::string& err) {
    const bool mixed = p.precision == PF_MIXED;
    if (p.dim == 2) {
        if (mixed) return new (std::nothrow) ImplT<float, 2>(p, s, err);
        return new (std::nothrow) ImplT<double, 2>(p, s, err);
    }
    if (mixed) return new (std::nothrow) ImplT<float, 3>(p, s, err);
    return new (std::nothrow) ImplT<double, 3>(p, s, err);
}

// ---------------------------------------------------------------------------
// Allocation-free pressure solve: scratch in a fixed device array
// ---------------------------------------------------------------------------
// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_pf_static_scratch[PF_STATIC_SCRATCH_BYTES];

// Device address of the array per device, looked up once per device with that
// device current (the host-side symbol is only a stand-in for it). Host
// threads making their first calls at once may each look it up; they store
// the same address, and the atomics keep those stores well defined.
std::atomic<void*> g_static_scratch_addr[64] = {};

template <typename T, int DIM>
pf_status run_static_solve(const pf_params& prm, cudaStream_t st, void* scratch,
                           const double* phi, const double* rhs, double* x, int* iters,
                           double* relres, std::string& err) {
    ImplT<T, DIM> im(prm, st, err);
    if (!err.empty()) return PF_ERR_INVALID;
    Carver size_cv{nullptr};
    im.carve_solver_only(size_cv);
    if (size_cv.off > (size_t)PF_STATIC_SCRATCH_BYTES) {
        err = "grid too large for the static scratch of pf_poisson_solve_static (" +
              std::to_string(size_cv.off) + " bytes needed, " +
              std::to_string((size_t)PF_STATIC_SCRATCH_BYTES) + " available)";
        return PF_ERR_INVALID;
    }
    Carver cv{static_cast<char*>(scratch)};
    im.carve_solver_only(cv);
    CGScalars host_sc;
    return im.solve_static(phi, rhs, x, &host_sc, iters, relres);
}

}  // namespace

namespace pf {
int ctx_step_begin(pf_ctx* ctx, int nsteps) {
    if (!ctx || nsteps < 0) return PF_ERR_INVALID;
    return (int)ctx->impl->step_begin(nsteps);
}
int ctx_step_end(pf_ctx* ctx) {
    if (!ctx) return PF_ERR_INVALID;
    return (int)ctx->impl->step_end();
}
int ctx_set_blocking(pf_ctx* ctx, int on) {
    if (!ctx) return PF_ERR_INVALID;
    return (int)ctx->impl->set_blocking(on != 0);
}
}  // namespace pf

extern "C" {

pf_status pf_poisson_solve_static(const pf_params* prm, const double* phi, const double* rhs,
                                  double* x, void* stream, int* iters, double* relres) {
    std::string why;
    pf_status s = validate(prm, why);
    if (s != PF_OK) { g_init_error = why; return s; }
    if (!phi || !rhs || !x) { g_init_error = "phi, rhs and x must be device pointers"; return PF_ERR_INVALID; }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        g_init_error = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return PF_ERR_CUDA;
    }
    void* scratch = g_static_scratch_addr[dev].load(std::memory_order_acquire);
    if (!scratch) {
        e = cudaGetSymbolAddress(&scratch, g_pf_static_scratch);
        if (e != cudaSuccess || !scratch) {
            g_init_error = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return PF_ERR_CUDA;
        }
        g_static_scratch_addr[dev].store(scratch, std::memory_order_release);
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::string err;
    const bool mixed = prm->precision == PF_MIXED;
    if (prm->dim == 2)
        s = mixed ? run_static_solve<float, 2>(*prm, st, scratch, phi, rhs, x, iters, relres, err)
                  : run_static_solve<double, 2>(*prm, st, scratch, phi, rhs, x, iters, relres, err);
    else
        s = mixed ? run_static_solve<float, 3>(*prm, st, scratch, phi, rhs, x, iters, relres, err)
                  : run_static_solve<double, 3>(*prm, st, scratch, phi, rhs, x, iters, relres, err);
    if (s != PF_OK) g_init_error = err;
    return s;
}


pf_status pf_workspace_size(const pf_params* prm, size_t* bytes) {
    std::string why;
    pf_status s = validate(prm, why);
    if (s != PF_OK) { g_init_error = why; return s; }
    if (!bytes) { g_init_error = "bytes is NULL"; return PF_ERR_INVALID; }
    std::string err;
    Impl* im = make_impl(*prm, nullptr, err);
    if (!im) return PF_ERR_INVALID;
    Carver cv{nullptr};
    im->carve(cv);
    *bytes = cv.off;
    delete im;
    return PF_OK;
}

pf_status pf_init(const pf_params* prm, void* workspace, size_t workspace_bytes, const double* phi0,
                  void* stream, pf_ctx** out) {
    std::string why;
    if (!out) { g_init_error = "out is NULL"; return PF_ERR_INVALID; }
    *out = nullptr;
    pf_status s = validate(prm, why);
    if (s != PF_OK) { g_init_error = why; return s; }
    size_t need = 0;
    pf_workspace_size(prm, &need);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0 ||
        workspace_bytes < need) {
        g_init_error = "workspace NULL, not 256-byte aligned or smaller than pf_workspace_size";
        return PF_ERR_WORKSPACE;
    }
    pf_ctx* ctx = new (std::nothrow) pf_ctx();
    if (!ctx) { g_init_error = "out of host memory"; return PF_ERR_INVALID; }
    ctx->prm = *prm;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Impl* im = make_impl(*prm, st, ctx->err);
    if (!im) { delete ctx; g_init_error = "out of host memory"; return PF_ERR_INVALID; }
    ctx->impl = im;
    Carver cv{static_cast<char*>(workspace)};
    im->carve(cv);
    pf_status hs;
    if (prm->dim == 2) {
        hs = prm->precision == PF_MIXED ? static_cast<ImplT<float, 2>*>(im)->alloc_host()
                                        : static_cast<ImplT<double, 2>*>(im)->alloc_host();
        if (hs == PF_OK)
            hs = prm->precision == PF_MIXED ? static_cast<ImplT<float, 2>*>(im)->init_device()
                                            : static_cast<ImplT<double, 2>*>(im)->init_device();
    } else {
        hs = prm->precision == PF_MIXED ? static_cast<ImplT<float, 3>*>(im)->alloc_host()
                                        : static_cast<ImplT<double, 3>*>(im)->alloc_host();
        if (hs == PF_OK)
            hs = prm->precision == PF_MIXED ? static_cast<ImplT<float, 3>*>(im)->init_device()
                                            : static_cast<ImplT<double, 3>*>(im)->init_device();
    }
    if (hs != PF_OK) {
        g_init_error = ctx->err;
        delete im;
        delete ctx;
        return hs;
    }
    im->init_phi(phi0);
    s = im->sync();
    if (s != PF_OK) {
        g_init_error = ctx->err;
        delete im;
        delete ctx;
        return s;
    }
    *out = ctx;
    return PF_OK;
}

pf_status pf_step(pf_ctx* ctx, int nsteps) {
    if (!ctx || nsteps < 0) return PF_ERR_INVALID;
    return ctx->impl->step(nsteps);
}

pf_status pf_project(pf_ctx* ctx) {
    if (!ctx) return PF_ERR_INVALID;
    return ctx->impl->project();
}

pf_status pf_diagnostics(pf_ctx* ctx, pf_diag* out) {
    if (!ctx || !out) return PF_ERR_INVALID;
    return ctx->impl->diagnostics(out);
}

pf_status pf_get_field(pf_ctx* ctx, int field, double* dst) {
    if (!ctx) return PF_ERR_INVALID;
    return ctx->impl->get_field(field, dst);
}

pf_status pf_set_field(pf_ctx* ctx, int field, const double* src) {
    if (!ctx) return PF_ERR_INVALID;
    return ctx->impl->set_field(field, src);
}

size_t pf_state_bytes(const pf_ctx* ctx) { return ctx ? ctx->impl->state_bytes() : 0; }

pf_status pf_get_state(pf_ctx* ctx, void* dst) {
    if (!ctx) return PF_ERR_INVALID;
    return ctx->impl->get_state(dst);
}

pf_status pf_set_state(pf_ctx* ctx, const void* src) {
    if (!ctx) return PF_ERR_INVALID;
    return ctx->impl->set_state(src);
}

pf_status pf_eval_rhs(pf_ctx* ctx, double gamma, double* kphi, double* ku) {
    if (!ctx) return PF_ERR_INVALID;
    return ctx->impl->eval_rhs(gamma, kphi, ku);
}

pf_status pf_poisson_solve(pf_ctx* ctx, const double* rhs, double* x, int* iters,
                           double* relres) {
    if (!ctx) return PF_ERR_INVALID;
    return ctx->impl->poisson_solve(rhs, x, iters, relres);
}

pf_status pf_adjoint_workspace_size(const pf_params* prm, size_t* bytes) {
    std::string why;
    pf_status s = validate(prm, why);
    if (s != PF_OK) { g_init_error = why; return s; }
    if (!bytes) { g_init_error = "bytes is NULL"; return PF_ERR_INVALID; }
    if (prm->precision != PF_FP64 || prm->model != PF_CDI || prm->force != PF_FORCE_EB ||
        prm->momentum != PF_MOMENTUM_ADVECTIVE || prm->wall_y != 0) {
        g_init_error = "the adjoint supports precision PF_FP64 with the CDI model, the EB force, "
                       "advective momentum and a periodic box";
        return PF_ERR_INVALID;
    }
    std::string err;
    Impl* im = make_impl(*prm, nullptr, err);
    if (!im) return PF_ERR_INVALID;
    *bytes = im->adjoint_bytes();
    delete im;
    return PF_OK;
}

pf_status pf_step_adjoint(pf_ctx* ctx, void* adj_workspace, size_t adj_bytes, const void* state_n,
                          double* lam, double* gparam) {
    if (!ctx) return PF_ERR_INVALID;
    return ctx->impl->step_adjoint(adj_workspace, adj_bytes, state_n, lam, gparam);
}

pf_status pf_objective(pf_ctx* ctx, const double* phi_target, double w_ke, double w_shape,
                       double* J, double* grad, double* gparam) {
    if (!ctx) return PF_ERR_INVALID;
    return ctx->impl->objective(phi_target, w_ke, w_shape, J, grad, gparam);
}

pf_status pf_profile_enable(pf_ctx* ctx, int enable) {
    if (!ctx) return PF_ERR_INVALID;
    ctx->impl->sync();
    ctx->impl->prof.harvest();
    ctx->impl->prof.timing = enable != 0;
    return PF_OK;
}

int pf_profile_read(pf_ctx* ctx, pf_profile_entry* out, int max_entries, int reset) {
    if (!ctx) return -1;
    Prof& pr = ctx->impl->prof;
    ctx->impl->sync();
    pr.harvest();
    int n = 0;
    for (int k = 0; k < KC_COUNT; ++k) {
        if (out && n < max_entries) {
            out[n].name = kClassNames[k];
            out[n].launches = pr.launches[k];
            out[n].ms = pr.ms[k];
        }
        ++n;
    }
    if (reset) {
        for (int k = 0; k < KC_COUNT; ++k) {
            pr.launches[k] = 0;
            pr.ms[k] = 0.0;
        }
    }
    return n;
}

pf_status pf_sync(pf_ctx* ctx) {
    if (!ctx) return PF_ERR_INVALID;
    return ctx->impl->sync();
}

void pf_destroy(pf_ctx* ctx) {
    if (!ctx) return;
    if (ctx->impl) {
        ctx->impl->sync();
        delete ctx->impl;
    }
    delete ctx;
}

const char* pf_last_error(const pf_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

}  // extern "C"
