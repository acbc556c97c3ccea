// Variable-coefficient pressure Poisson solve: -div(beta grad p) = f with
// beta = 1/rho_f on the periodic cell-centred grid (rho_f the two-cell mean
// of rho(phi)), by flexible (Polak-Ribiere) conjugate gradients in float64
// preconditioned with one geometric multigrid V-cycle in precision T:
//   red-black Gauss-Seidel smoothing, residual restriction by the mean of the
//   2^d children, (bi/tri)linear prolongation, coarse face coefficients the
//   mean of the fine faces they cover; the coarse levels run in one
//   single-CTA kernel. The singular periodic system is handled by removing
//   the mean of the right-hand side; the solution is defined up to a constant.
#include "pf_device.cuh"

namespace pf {

template <typename T>
__device__ __forceinline__ T rho_of_p(T phi, const Phys& ph) {
    T c = phi < T(0) ? T(0) : (phi > T(1) ? T(1) : phi);
    return T(ph.rho_out) + (T(ph.rho_in) - T(ph.rho_out)) * c;
}

// neighbour indices (-x, +x, -y, +y, -z, +z) of a cell on a periodic level
template <int DIM>
__device__ __forceinline__ void nbrs(int idx, const Dims& g, int (&nb)[6], Cell& c) {
    c = decode(idx, g);
    const int sxy = g.nx * g.ny;
    nb[0] = c.i == 0 ? idx + g.nx - 1 : idx - 1;
    nb[1] = c.i == g.nx - 1 ? idx - (g.nx - 1) : idx + 1;
    nb[2] = c.j == 0 ? idx + (g.ny - 1) * g.nx : idx - g.nx;
    nb[3] = c.j == g.ny - 1 ? idx - (g.ny - 1) * g.nx : idx + g.nx;
    if (DIM == 3) {
        nb[4] = c.k == 0 ? idx + (g.nz - 1) * sxy : idx - sxy;
        nb[5] = c.k == g.nz - 1 ? idx - (g.nz - 1) * sxy : idx + sxy;
    }
}

// Face weights beta/h^2 of the 2*DIM faces of a cell at level L (level 0:
// computed from phi).
template <typename T, int DIM>
__device__ __forceinline__ void face_w(const MGLevel<T>& L, const T* __restrict__ phi,
                                       const Phys& ph, int idx, const int (&nb)[6], T (&w)[6]) {
    const T ih2 = T(1.0 / (L.g.h * L.g.h));
    if (L.beta[0] == nullptr) {
        const T rc = rho_of_p(__ldg(phi + idx), ph);
#pragma unroll
        for (int q = 0; q < 2 * DIM; ++q)
            w[q] = ih2 / (T(0.5) * (rc + rho_of_p(__ldg(phi + nb[q]), ph)));
    } else {
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            w[2 * d] = L.beta[d][idx] * ih2;
            w[2 * d + 1] = L.beta[d][nb[2 * d + 1]] * ih2;
        }
    }
}

template <typename T, int DIM>
__device__ __forceinline__ T residual_at(const MGLevel<T>& L, const T* __restrict__ phi,
                                         const Phys& ph, int idx) {
    int nb[6];
    Cell c;
    nbrs<DIM>(idx, L.g, nb, c);
    T w[6];
    face_w<T, DIM>(L, phi, ph, idx, nb, w);
    const T xc = L.x[idx];
    T ax = T(0);
#pragma unroll
    for (int q = 0; q < 2 * DIM; ++q) ax += w[q] * (xc - L.x[nb[q]]);
    return L.f[idx] - ax;
}

// One red (color 0) or black (color 1) Gauss-Seidel update of a cell;
// zero_start: the level's x is taken as 0 and both colors are written.
template <typename T, int DIM>
__device__ __forceinline__ void gs_cell(const MGLevel<T>& L, const T* __restrict__ phi,
                                        const Phys& ph, int idx, int color, bool zero_start) {
    int nb[6];
    Cell c;
    nbrs<DIM>(idx, L.g, nb, c);
    const int col = (c.i + c.j + c.k) & 1;
    if (zero_start) {
        if (col != color) {
            L.x[idx] = T(0);
            return;
        }
        T w[6];
        face_w<T, DIM>(L, phi, ph, idx, nb, w);
        T diag = T(0);
#pragma unroll
        for (int q = 0; q < 2 * DIM; ++q) diag += w[q];
        L.x[idx] = L.f[idx] / diag;
        return;
    }
    if (col != color) return;
    T w[6];
    face_w<T, DIM>(L, phi, ph, idx, nb, w);
    T diag = T(0), off = T(0);
#pragma unroll
    for (int q = 0; q < 2 * DIM; ++q) {
        diag += w[q];
        off += w[q] * L.x[nb[q]];
    }
    L.x[idx] = (L.f[idx] + off) / diag;
}

// f_{l+1}(I) = mean of the residual of the 2^d children of coarse cell I
template <typename T, int DIM>
__device__ __forceinline__ void restrict_cell(const MGLevel<T>& F, const MGLevel<T>& C,
                                              const T* __restrict__ phi, const Phys& ph, int I) {
    Cell cc = decode(I, C.g);
    T s = T(0);
#pragma unroll
    for (int a = 0; a < (DIM == 3 ? 2 : 1); ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                int fi = 2 * cc.i + e, fj = 2 * cc.j + b, fk = DIM == 3 ? 2 * cc.k + a : 0;
                s += residual_at<T, DIM>(F, phi, ph, (fk * F.g.ny + fj) * F.g.nx + fi);
            }
    C.f[I] = s * T(DIM == 3 ? 0.125 : 0.25);
}

// x_l(i) += linear interpolation of x_{l+1} (weights 3/4, 1/4 per axis)
template <typename T, int DIM>
__device__ __forceinline__ void prolong_cell(const MGLevel<T>& F, const MGLevel<T>& C, int idx) {
    Cell c = decode(idx, F.g);
    int I0 = c.i >> 1, J0 = c.j >> 1, K0 = DIM == 3 ? c.k >> 1 : 0;
    int I1 = wrapi(I0 + ((c.i & 1) ? 1 : -1), C.g.nx);
    int J1 = wrapi(J0 + ((c.j & 1) ? 1 : -1), C.g.ny);
    int K1 = DIM == 3 ? wrapi(K0 + ((c.k & 1) ? 1 : -1), C.g.nz) : 0;
    const T* xc = C.x;
    auto at = [&](int i, int j, int k) { return xc[(k * C.g.ny + j) * C.g.nx + i]; };
    T v = T(0.5625) * at(I0, J0, K0) + T(0.1875) * (at(I1, J0, K0) + at(I0, J1, K0)) +
          T(0.0625) * at(I1, J1, K0);
    if (DIM == 3) {
        T v1 = T(0.5625) * at(I0, J0, K1) + T(0.1875) * (at(I1, J0, K1) + at(I0, J1, K1)) +
               T(0.0625) * at(I1, J1, K1);
        v = T(0.75) * v + T(0.25) * v1;
    }
    F.x[idx] += v;
}

// ---------------------------------------------------------------------------
// grid kernels for the large levels
// ---------------------------------------------------------------------------
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_gs(MGLevel<T> L, const T* __restrict__ phi, Phys ph, int color, int zero_start,
     const CGScalars* sc) {
    if (sc && sc->done) return;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= L.g.ncell) return;
    gs_cell<T, DIM>(L, phi, ph, idx, color, zero_start != 0);
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_restrict(MGLevel<T> F, MGLevel<T> C, const T* __restrict__ phi, Phys ph, const CGScalars* sc) {
    if (sc && sc->done) return;
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= C.g.ncell) return;
    restrict_cell<T, DIM>(F, C, phi, ph, I);
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_prolong(MGLevel<T> F, MGLevel<T> C, const CGScalars* sc) {
    if (sc && sc->done) return;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= F.g.ncell) return;
    prolong_cell<T, DIM>(F, C, idx);
}

// coarse face coefficients: mean of the 2^(d-1) fine faces on each coarse face
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_coarsen_beta(MGLevel<T> F, MGLevel<T> C, const T* __restrict__ phi, Phys ph) {
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= C.g.ncell) return;
    Cell cc = decode(I, C.g);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        T s = T(0);
        int cnt = 0;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < (DIM == 3 ? 2 : 1); ++b) {
                int o[3] = {0, 0, 0};
                // the two transverse axes of d get offsets a, b
                int e1 = (d + 1) % DIM, e2 = (d + 2) % 3;
                o[e1] = a;
                if (DIM == 3) o[e2] = b;
                int fi = 2 * cc.i + o[0], fj = 2 * cc.j + o[1], fk = DIM == 3 ? 2 * cc.k + o[2] : 0;
                int fidx = (fk * F.g.ny + fj) * F.g.nx + fi;
                T bf;
                if (F.beta[0] == nullptr) {
                    int nb[6];
                    Cell c;
                    nbrs<DIM>(fidx, F.g, nb, c);
                    bf = T(1) / (T(0.5) * (rho_of_p(__ldg(phi + fidx), ph) +
                                           rho_of_p(__ldg(phi + nb[2 * d]), ph)));
                } else {
                    bf = F.beta[d][fidx];
                }
                s += bf;
                ++cnt;
            }
        C.beta[d][I] = s / T(cnt);
    }
}

// ---------------------------------------------------------------------------
// single-CTA kernel for all levels >= first_coarse
// ---------------------------------------------------------------------------
constexpr int kCoarseThreads = 1024;

template <typename T, int DIM>
__global__ void __launch_bounds__(kCoarseThreads)
k_coarse_vcycle(MGHier<T> H, const T* __restrict__ phi, Phys ph, const CGScalars* sc) {
    if (sc && sc->done) return;
    __shared__ double red[32];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int l0 = H.first_coarse, lb = H.nlev - 1;
    // down
    for (int l = l0; l < lb; ++l) {
        const MGLevel<T>& L = H.lev[l];
        for (int s = 0; s < H.pre; ++s) {
            for (int i = tid; i < L.g.ncell; i += nt) gs_cell<T, DIM>(L, phi, ph, i, 0, s == 0);
            __syncthreads();
            for (int i = tid; i < L.g.ncell; i += nt) gs_cell<T, DIM>(L, phi, ph, i, 1, false);
            __syncthreads();
        }
        for (int I = tid; I < H.lev[l + 1].g.ncell; I += nt)
            restrict_cell<T, DIM>(L, H.lev[l + 1], phi, ph, I);
        __syncthreads();
    }
    // bottom: remove the mean of f (compatibility), then many sweeps
    {
        const MGLevel<T>& L = H.lev[lb];
        double s = 0.0;
        for (int i = tid; i < L.g.ncell; i += nt) s += double(L.f[i]);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if ((tid & 31) == 0) red[tid >> 5] = s;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < nt / 32; ++w) t += red[w];
            red[0] = t / L.g.ncell;
        }
        __syncthreads();
        const T mean = T(red[0]);
        for (int i = tid; i < L.g.ncell; i += nt) L.f[i] -= mean;
        __syncthreads();
        for (int s2 = 0; s2 < H.coarse_sweeps; ++s2) {
            for (int i = tid; i < L.g.ncell; i += nt) gs_cell<T, DIM>(L, phi, ph, i, 0, s2 == 0);
            __syncthreads();
            for (int i = tid; i < L.g.ncell; i += nt) gs_cell<T, DIM>(L, phi, ph, i, 1, false);
            __syncthreads();
        }
    }
    // up
    for (int l = lb - 1; l >= l0; --l) {
        const MGLevel<T>& L = H.lev[l];
        for (int i = tid; i < L.g.ncell; i += nt) prolong_cell<T, DIM>(L, H.lev[l + 1], i);
        __syncthreads();
        for (int s = 0; s < H.post; ++s) {
            for (int i = tid; i < L.g.ncell; i += nt) gs_cell<T, DIM>(L, phi, ph, i, 1, false);
            __syncthreads();
            for (int i = tid; i < L.g.ncell; i += nt) gs_cell<T, DIM>(L, phi, ph, i, 0, false);
            __syncthreads();
        }
    }
}

template <typename T, int DIM>
void launch_mg_setup(const Dims&, const Phys& ph, const T* phi, MGHier<T>& H, cudaStream_t s) {
    for (int l = 0; l + 1 < H.nlev; ++l)
        k_coarsen_beta<T, DIM><<<lin_grid(H.lev[l + 1].g.ncell), kThreads, 0, s>>>(
            H.lev[l], H.lev[l + 1], phi, ph);
}

template <typename T, int DIM>
void launch_vcycle(const Phys& ph, const T* phi, MGHier<T>& H, const CGScalars* sc,
                   cudaStream_t s, Prof* pr) {
    const int l0 = H.first_coarse;
    auto gs = [&](int l, int color, int zero) {
        const MGLevel<T>& L = H.lev[l];
        pr->begin(l == 0 ? KC_GS0 : KC_GS);
        k_gs<T, DIM><<<lin_grid(L.g.ncell), kThreads, 0, s>>>(L, phi, ph, color, zero, sc);
        pr->end();
    };
    for (int l = 0; l < l0; ++l) {
        for (int p = 0; p < H.pre; ++p) {
            gs(l, 0, p == 0);
            gs(l, 1, 0);
        }
        pr->begin(KC_RESTRICT);
        k_restrict<T, DIM><<<lin_grid(H.lev[l + 1].g.ncell), kThreads, 0, s>>>(H.lev[l], H.lev[l + 1],
                                                                                phi, ph, sc);
        pr->end();
    }
    pr->begin(KC_COARSE);
    k_coarse_vcycle<T, DIM><<<1, kCoarseThreads, 0, s>>>(H, phi, ph, sc);
    pr->end();
    for (int l = l0 - 1; l >= 0; --l) {
        pr->begin(KC_PROLONG);
        k_prolong<T, DIM><<<lin_grid(H.lev[l].g.ncell), kThreads, 0, s>>>(H.lev[l], H.lev[l + 1], sc);
        pr->end();
        for (int p = 0; p < H.post; ++p) {
            gs(l, 1, 0);
            gs(l, 0, 0);
        }
    }
}

// ---------------------------------------------------------------------------
// float64 CG kernels (operator from phi in float64)
// ---------------------------------------------------------------------------
template <typename T, int DIM>
__device__ __forceinline__ double apply_A64(const Dims& g, const Phys& ph,
                                            const T* __restrict__ phi, const double* __restrict__ x,
                                            int idx) {
    int nb[6];
    Cell c;
    nbrs<DIM>(idx, g, nb, c);
    const double ih2 = 1.0 / (g.h * g.h);
    const double rc = double(rho_of_p(double(__ldg(phi + idx)), ph));
    const double xc = x[idx];
    double ax = 0.0;
#pragma unroll
    for (int q = 0; q < 2 * DIM; ++q) {
        double rf = 0.5 * (rc + rho_of_p(double(__ldg(phi + nb[q])), ph));
        ax += (1.0 / rf) * (xc - x[nb[q]]);
    }
    return ax * ih2;
}

// r = sign (b - mean b) - A x ; ff = ||f||^2, rr = ||r||^2
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_cg_start(Dims g, Phys ph, const T* __restrict__ phi, const double* __restrict__ b, double sign,
           const double* __restrict__ x, double* __restrict__ r, T* __restrict__ rT, RedBuf rb,
           CGScalars* sc) {
    const double mb = sc->mean_b;
    double ff = 0.0, rr = 0.0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.ncell;
         idx += gridDim.x * blockDim.x) {
        double f = sign * (b[idx] - mb);
        double rv = f - apply_A64<T, DIM>(g, ph, phi, x, idx);
        r[idx] = rv;
        if ((void*)rT != (void*)r) rT[idx] = T(rv);
        ff += f * f;
        rr += rv * rv;
    }
    double v[2] = {ff, rr}, tot[2];
    const int mode[2] = {0, 0};
    if (grid_reduce<2>(v, mode, rb, tot) && threadIdx.x == 0) {
        sc->ff = tot[0];
        sc->rr = tot[1];
        sc->iters = 0;
        // nothing to do when the residual already meets the tolerance (incl. f = 0, r = 0)
        sc->done = (tot[1] <= sc->rtol2 * tot[0]) ? 1 : 0;
        if (!(tot[1] == tot[1])) {
            sc->done = 1;
            sc->status = 4;
        }
    }
}

// rz = r.z ; zq = z.q (previous q) ; beta (Polak-Ribiere)
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_cg_dots(Dims g, const T* __restrict__ z, const double* __restrict__ r,
          const double* __restrict__ q, int first, RedBuf rb, CGScalars* sc) {
    if (sc->done) return;
    double rz = 0.0, zq = 0.0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.ncell;
         idx += gridDim.x * blockDim.x) {
        double zv = double(z[idx]);
        rz += r[idx] * zv;
        if (!first) zq += zv * q[idx];
    }
    double v[2] = {rz, zq}, tot[2];
    const int mode[2] = {0, 0};
    if (grid_reduce<2>(v, mode, rb, tot) && threadIdx.x == 0) {
        if (first) {
            sc->beta = 0.0;
        } else {
            sc->beta = -sc->alpha * tot[1] / sc->rz;
        }
        sc->rz = tot[0];
    }
}

// p_new = z + beta p_old ; q = A p_new ; pq = p_new . q ; alpha = rz / pq
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_cg_dir(Dims g, Phys ph, const T* __restrict__ phi, const T* __restrict__ z,
         const double* __restrict__ p_old, double* __restrict__ p_new, double* __restrict__ q,
         int first, RedBuf rb, CGScalars* sc) {
    if (sc->done) return;
    const double beta = first ? 0.0 : sc->beta;
    const double ih2 = 1.0 / (g.h * g.h);
    double pq = 0.0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.ncell;
         idx += gridDim.x * blockDim.x) {
        int nb[6];
        Cell c;
        nbrs<DIM>(idx, g, nb, c);
        const double pc = double(z[idx]) + (first ? 0.0 : beta * p_old[idx]);
        const double rc = rho_of_p(double(__ldg(phi + idx)), ph);
        double ax = 0.0;
#pragma unroll
        for (int k = 0; k < 2 * DIM; ++k) {
            const double pn = double(z[nb[k]]) + (first ? 0.0 : beta * p_old[nb[k]]);
            const double rf = 0.5 * (rc + rho_of_p(double(__ldg(phi + nb[k])), ph));
            ax += (1.0 / rf) * (pc - pn);
        }
        ax *= ih2;
        p_new[idx] = pc;
        q[idx] = ax;
        pq += pc * ax;
    }
    double v[1] = {pq}, tot[1];
    const int mode[1] = {0};
    if (grid_reduce<1>(v, mode, rb, tot) && threadIdx.x == 0) {
        sc->pq = tot[0];
        sc->alpha = tot[0] != 0.0 ? sc->rz / tot[0] : 0.0;
    }
}

// x += alpha p ; r -= alpha q ; rr = r.r ; convergence flag
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_cg_update(Dims g, const double* __restrict__ p, const double* __restrict__ q,
            double* __restrict__ x, double* __restrict__ r, T* __restrict__ rT, RedBuf rb,
            CGScalars* sc) {
    if (sc->done) return;
    const double alpha = sc->alpha;
    double rr = 0.0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.ncell;
         idx += gridDim.x * blockDim.x) {
        x[idx] += alpha * p[idx];
        double rv = r[idx] - alpha * q[idx];
        r[idx] = rv;
        if ((void*)rT != (void*)r) rT[idx] = T(rv);
        rr += rv * rv;
    }
    double v[1] = {rr}, tot[1];
    const int mode[1] = {0};
    if (grid_reduce<1>(v, mode, rb, tot) && threadIdx.x == 0) {
        sc->rr = tot[0];
        sc->iters += 1;
        if (!(tot[0] == tot[0])) {
            sc->done = 1;
            sc->status = 4;   // PF_ERR_NONFINITE
        } else if (tot[0] <= sc->rtol2 * sc->ff) {
            sc->done = 1;
        } else if (sc->iters >= sc->maxit) {
            sc->done = 1;
            if (sc->status == 0) sc->status = 3;   // PF_ERR_NOT_CONVERGED
        }
    }
}

template <typename T, int DIM>
void launch_cg_start(const Dims& g, const Phys& ph, const T* phi, const double* b, double sign,
                     double* x, double* r, T* rT, RedBuf rb, CGScalars* sc, cudaStream_t s) {
    k_cg_start<T, DIM><<<red_grid(g.ncell), kThreads, 0, s>>>(g, ph, phi, b, sign, x, r, rT, rb,
                                                               sc);
}
template <typename T, int DIM>
void launch_cg_dots(const Dims& g, const T* z, const double* r, const double* q, int first,
                    RedBuf rb, CGScalars* sc, cudaStream_t s) {
    k_cg_dots<T, DIM><<<red_grid(g.ncell), kThreads, 0, s>>>(g, z, r, q, first, rb, sc);
}
template <typename T, int DIM>
void launch_cg_dir(const Dims& g, const Phys& ph, const T* phi, const T* z, const double* p_old,
                   double* p_new, double* q, int first, RedBuf rb, CGScalars* sc,
                   cudaStream_t s) {
    k_cg_dir<T, DIM><<<red_grid(g.ncell), kThreads, 0, s>>>(g, ph, phi, z, p_old, p_new, q, first,
                                                             rb, sc);
}
template <typename T, int DIM>
void launch_cg_update(const Dims& g, const double* p, const double* q, double* x, double* r,
                      T* rT, RedBuf rb, CGScalars* sc, cudaStream_t s) {
    k_cg_update<T, DIM><<<red_grid(g.ncell), kThreads, 0, s>>>(g, p, q, x, r, rT, rb, sc);
}

__global__ void __launch_bounds__(kThreads)
k_sum(int n, const double* __restrict__ x, RedBuf rb, double* out) {
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += x[i];
    double v[1] = {s}, tot[1];
    const int mode[1] = {0};
    if (grid_reduce<1>(v, mode, rb, tot) && threadIdx.x == 0) *out = tot[0];
}

void launch_sum(int n, const double* x, RedBuf rb, double* out, cudaStream_t s) {
    k_sum<<<red_grid(n), kThreads, 0, s>>>(n, x, rb, out);
}

#define PF_INST_P(T, D)                                                                         \
    template void launch_mg_setup<T, D>(const Dims&, const Phys&, const T*, MGHier<T>&,         \
                                        cudaStream_t);                                          \
    template void launch_vcycle<T, D>(const Phys&, const T*, MGHier<T>&, const CGScalars*,      \
                                      cudaStream_t, Prof*);                                     \
    template void launch_cg_start<T, D>(const Dims&, const Phys&, const T*, const double*,      \
                                        double, double*, double*, T*, RedBuf, CGScalars*,        \
                                        cudaStream_t);                                          \
    template void launch_cg_dots<T, D>(const Dims&, const T*, const double*, const double*, int, \
                                       RedBuf, CGScalars*, cudaStream_t);                       \
    template void launch_cg_dir<T, D>(const Dims&, const Phys&, const T*, const T*,             \
                                      const double*, double*, double*, int, RedBuf, CGScalars*, \
                                      cudaStream_t);                                            \
    template void launch_cg_update<T, D>(const Dims&, const double*, const double*, double*,    \
                                         double*, T*, RedBuf, CGScalars*, cudaStream_t);

PF_INST_P(double, 2)
PF_INST_P(double, 3)
PF_INST_P(float, 2)
PF_INST_P(float, 3)

}  // namespace pf
