// Variable-coefficient pressure Poisson solve  A x = f,  A = -D beta G,
// beta = 1/rho_f on the periodic cell-centred grid (rho_f the two-cell mean of
// rho(phi)); the singular periodic system is handled by removing the mean of
// the right-hand side, and x is defined up to a constant.
//
// Structure (GB300: the float64 pipe is a small fraction of float32, so float64
// arithmetic is kept out of every inner pass):
//   outer  float64 iterative refinement: r = f - A x evaluated in float64,
//          x += e; stops at ||r|| <= rtol ||f||;
//   inner  flexible (Polak-Ribiere) CG in the storage precision T on A e = r,
//          preconditioned by one multigrid V-cycle: red-black Gauss-Seidel,
//          restriction by the mean of the 2^d children, (bi/tri)linear
//          prolongation, coarse face coefficients the mean of the fine faces
//          they cover, and every level of <= 4096 cells inside one
//          single-CTA kernel.
// T = double: beta comes from precomputed float64 arrays and the inner CG is
// run to the final tolerance (one outer step); T = float: beta = a correctly
// rounded float32 reciprocal of rho_f, identical in every kernel (operator,
// smoother, correction), and each inner solve reduces its residual by eta.
#include <type_traits>

#include <mutex>

#include "pf_device.cuh"

namespace pf {

// Face weights beta/h^2 of the 2*DIM faces of a cell on level L.
template <typename T, int DIM>
__device__ __forceinline__ void face_w(const MGLevel<T>& L, const T* __restrict__ phi,
                                       const Phys& ph, int idx, const Nb6& nb, T (&w)[6]) {
    const T ih2 = ih2_of(L.g, T());
    if (L.beta[0] == nullptr) {
        // level 0, float path: from phi
        const float pc = float(__ldg(phi + idx));
#pragma unroll
        for (int q = 0; q < 2 * DIM; ++q)
            w[q] = T(beta_face32(pc, float(__ldg(phi + nb.m[q])), ph)) * ih2;
        if (L.g.wall_y) {
            const int j = (idx / L.g.nx) % L.g.ny;
            if (wall_face(L.g, j, 2)) w[2] = T(0);
            if (wall_face(L.g, j, 3)) w[3] = T(0);
        }
    } else {
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            w[2 * d] = L.beta[d][idx] * ih2;
            w[2 * d + 1] = L.beta[d][nb.m[2 * d + 1]] * ih2;
        }
    }
}

template <typename T, int DIM>
__device__ __forceinline__ T residual_at(const MGLevel<T>& L, const T* __restrict__ phi,
                                         const Phys& ph, int i, int j, int k, int idx) {
    const Nb6 nb = nb6<DIM>(L.g, i, j, k, idx);
    T w[6];
    face_w<T, DIM>(L, phi, ph, idx, nb, w);
    const T xc = L.x[idx];
    T ax = T(0);
#pragma unroll
    for (int q = 0; q < 2 * DIM; ++q) ax += w[q] * (xc - L.x[nb.m[q]]);
    return L.f[idx] - ax;
}

// Gauss-Seidel update of one cell; zero_start: x is taken as 0 (the cell's
// neighbours are all of the other colour and still 0), so x = f / diag.
template <typename T, int DIM>
__device__ __forceinline__ void gs_cell(const MGLevel<T>& L, const T* __restrict__ phi,
                                        const Phys& ph, int i, int j, int k, int idx,
                                        bool zero_start) {
    const Nb6 nb = nb6<DIM>(L.g, i, j, k, idx);
    T w[6];
    face_w<T, DIM>(L, phi, ph, idx, nb, w);
    T diag = T(0), off = T(0);
#pragma unroll
    for (int q = 0; q < 2 * DIM; ++q) {
        diag += w[q];
        if (!zero_start) off += w[q] * L.x[nb.m[q]];
    }
    L.x[idx] = divq(L.f[idx] + off, diag);
}

// f_{l+1}(I) = mean of the residual of the 2^d children of coarse cell I
template <typename T, int DIM>
__device__ __forceinline__ void restrict_cell(const MGLevel<T>& F, const MGLevel<T>& C,
                                              const T* __restrict__ phi, const Phys& ph, int ci,
                                              int cj, int ck, int I) {
    T s = T(0);
#pragma unroll
    for (int a = 0; a < (DIM == 3 ? 2 : 1); ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int fi = 2 * ci + e, fj = 2 * cj + b, fk = DIM == 3 ? 2 * ck + a : 0;
                s += residual_at<T, DIM>(F, phi, ph, fi, fj, fk, (fk * F.g.ny + fj) * F.g.nx + fi);
            }
    C.f[I] = s * T(DIM == 3 ? 0.125 : 0.25);
}

// x_l(i) += linear interpolation of x_{l+1} (weights 3/4, 1/4 per axis)
template <typename T, int DIM>
__device__ __forceinline__ void prolong_cell(const MGLevel<T>& F, const MGLevel<T>& C, int i, int j,
                                             int k, int idx) {
    const int I0 = i >> 1, J0 = j >> 1, K0 = DIM == 3 ? k >> 1 : 0;
    const int I1 = wrapi(I0 + ((i & 1) ? 1 : -1), C.g.nx);
    const int J1 = wrapi(J0 + ((j & 1) ? 1 : -1), C.g.ny);
    const int K1 = DIM == 3 ? wrapi(K0 + ((k & 1) ? 1 : -1), C.g.nz) : 0;
    const T* xc = C.x;
    auto at = [&](int a, int b, int c) { return xc[(c * C.g.ny + b) * C.g.nx + a]; };
    T v = T(0.5625) * at(I0, J0, K0) + T(0.1875) * (at(I1, J0, K0) + at(I0, J1, K0)) +
          T(0.0625) * at(I1, J1, K0);
    if (DIM == 3) {
        T v1 = T(0.5625) * at(I0, J0, K1) + T(0.1875) * (at(I1, J0, K1) + at(I0, J1, K1)) +
               T(0.0625) * at(I1, J1, K1);
        v = T(0.75) * v + T(0.25) * v1;
    }
    F.x[idx] += v;
}

__device__ __forceinline__ bool inner_stopped(const CGScalars* sc) { return sc->done || sc->idone; }

// ---------------------------------------------------------------------------
// grid kernels for the large levels
// ---------------------------------------------------------------------------
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_gs(MGLevel<T> L, const T* __restrict__ phi, Phys ph, int color, int zero_start,
     const CGScalars* sc) {
    if (inner_stopped(sc)) return;
    if (zero_start) {
        // both colours: active colour x = f/diag, the other 0
        for_cells(L.g, [&](int i, int j, int k, int idx) {
            if (((i + j + k) & 1) == color) gs_cell<T, DIM>(L, phi, ph, i, j, k, idx, true);
            else L.x[idx] = T(0);
        });
    } else {
        for_color_cells(L.g, color, [&](int i, int j, int k, int idx) {
            gs_cell<T, DIM>(L, phi, ph, i, j, k, idx, false);
        });
    }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_restrict(MGLevel<T> F, MGLevel<T> C, const T* __restrict__ phi, Phys ph, const CGScalars* sc) {
    if (inner_stopped(sc)) return;
    for_cells(C.g, [&](int i, int j, int k, int I) {
        restrict_cell<T, DIM>(F, C, phi, ph, i, j, k, I);
    });
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_prolong(MGLevel<T> F, MGLevel<T> C, const CGScalars* sc) {
    if (inner_stopped(sc)) return;
    for_cells(F.g, [&](int i, int j, int k, int idx) { prolong_cell<T, DIM>(F, C, i, j, k, idx); });
}

// 3D, even nx: one thread per pair of fine cells (2I, 2I+1) of a row, which
// share the coarse column I; the fine pair is read and written as a vector.
// The launch is a 3D grid over (pair, row, plane), so no thread decodes its
// cell from a linear index (integer divisions by the level's sizes).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_prolong_pairs(MGLevel<T> F, MGLevel<T> C, const CGScalars* sc) {
    if (inner_stopped(sc)) return;
    using V2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    const int npair = F.g.nx >> 1;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (I >= npair || j >= F.g.ny) return;
    const int cx = C.g.nx, cy = C.g.ny, cz = C.g.nz;
    const int J0 = j >> 1, K0 = k >> 1;
    const int J1 = wrapi(J0 + ((j & 1) ? 1 : -1), cy);
    const int K1 = wrapi(K0 + ((k & 1) ? 1 : -1), cz);
    const int Im = wrapi(I - 1, cx), Ip = wrapi(I + 1, cx);
    const T* xc = C.x;
    auto row3 = [&](int J, int K, T& m, T& c, T& p) {
        const int base = (K * cy + J) * cx;
        m = __ldg(xc + base + Im);
        c = __ldg(xc + base + I);
        p = __ldg(xc + base + Ip);
    };
    T m00, c00, p00, m10, c10, p10, m01, c01, p01, m11, c11, p11;
    row3(J0, K0, m00, c00, p00);
    row3(J1, K0, m10, c10, p10);
    row3(J0, K1, m01, c01, p01);
    row3(J1, K1, m11, c11, p11);
    // even fine cell uses the -x coarse neighbour, odd the +x one
    auto interp = [&](T nb00, T nb10, T nb01, T nb11) {
        T v = T(0.5625) * c00 + T(0.1875) * (nb00 + c10) + T(0.0625) * nb10;
        T v1 = T(0.5625) * c01 + T(0.1875) * (nb01 + c11) + T(0.0625) * nb11;
        return T(0.75) * v + T(0.25) * v1;
    };
    const T ve = interp(m00, m10, m01, m11);
    const T vo = interp(p00, p10, p01, p11);
    V2* xf = reinterpret_cast<V2*>(F.x + ((size_t)k * F.g.ny + j) * F.g.nx + 2 * I);
    V2 cur = *xf;
    cur.x += ve;
    cur.y += vo;
    *xf = cur;
}

// 3D float32: one thread per coarse column (I, J) of a 32 x 8 tile, marching
// over a chunk of kc coarse planes K. The 3 x 3 coarse neighbourhood of the
// planes K - 1, K and K + 1 is carried in registers, so a coarse value is
// loaded once per thread and plane: 9 loads per coarse plane for its 8 fine
// children (fine planes 2K and 2K + 1, rows 2J and 2J + 1, each an x pair read
// and written as a vector), against 12 per fine pair in k_prolong_pairs. Same
// interpolation formula and evaluation order per fine cell.
__global__ void __launch_bounds__(256)
k_prolong_zm(MGLevel<float> F, MGLevel<float> C, int kc, const CGScalars* sc) {
    if (inner_stopped(sc)) return;
    const int cx = C.g.nx, cy = C.g.ny, cz = C.g.nz;
    const int I = blockIdx.x * 32 + threadIdx.x % 32;
    const int J = blockIdx.y * 8 + threadIdx.x / 32;
    if (I >= cx || J >= cy) return;
    const int K0 = blockIdx.z * kc;
    const int K1 = min(K0 + kc, cz);
    const int Im = wrapi(I - 1, cx), Ip = wrapi(I + 1, cx);
    const int rows[3] = {wrapi(J - 1, cy) * cx, J * cx, wrapi(J + 1, cy) * cx};
    const int cols[3] = {Im, I, Ip};
    const float* __restrict__ xc = C.x;
    const size_t cplane = (size_t)cx * cy;
    // v[y][x]: coarse rows J - 1, J, J + 1 and columns I - 1, I, I + 1
    auto load = [&](int K, float (&v)[3][3]) {
        const float* b = xc + (size_t)K * cplane;
#pragma unroll
        for (int y = 0; y < 3; ++y)
#pragma unroll
            for (int x = 0; x < 3; ++x) v[y][x] = __ldg(b + rows[y] + cols[x]);
    };
    float a[3][3], b[3][3], c[3][3];
    load(wrapi(K0 - 1, cz), a);
    load(K0, b);
    const int fnx = F.g.nx, fny = F.g.ny;
    for (int K = K0; K < K1; ++K) {
        load(K + 1 == cz ? 0 : K + 1, c);
#pragma unroll
        for (int zp = 0; zp < 2; ++zp) {
            const float (&zn)[3][3] = zp ? c : a;   // coarse plane K - 1 or K + 1
#pragma unroll
            for (int yp = 0; yp < 2; ++yp) {
                const int yn = yp ? 2 : 0;           // coarse row J - 1 or J + 1
                // even fine cell uses the -x coarse neighbour, odd the +x one
                auto interp = [&](int xn) {
                    const float v = 0.5625f * b[1][1] + 0.1875f * (b[1][xn] + b[yn][1]) +
                                    0.0625f * b[yn][xn];
                    const float v1 = 0.5625f * zn[1][1] + 0.1875f * (zn[1][xn] + zn[yn][1]) +
                                     0.0625f * zn[yn][xn];
                    return 0.75f * v + 0.25f * v1;
                };
                const float ve = interp(0), vo = interp(2);
                float2* xf = reinterpret_cast<float2*>(
                    F.x + ((size_t)(2 * K + zp) * fny + (2 * J + yp)) * fnx + 2 * I);
                float2 cur = *xf;
                cur.x += ve;
                cur.y += vo;
                *xf = cur;
            }
        }
#pragma unroll
        for (int y = 0; y < 3; ++y)
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                a[y][x] = b[y][x];
                b[y][x] = c[y][x];
            }
    }
}

// coarse face coefficients: mean of the 2^(d-1) fine faces on each coarse face
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_coarsen_beta(MGLevel<T> F, MGLevel<T> C, const T* __restrict__ phi, Phys ph) {
    for_cells(C.g, [&](int ci, int cj, int ck, int I) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            T s = T(0);
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < (DIM == 3 ? 2 : 1); ++b) {
                    int o[3] = {0, 0, 0};
                    const int e1 = (d + 1) % DIM, e2 = (d + 2) % 3;
                    o[e1] = a;
                    if (DIM == 3) o[e2] = b;
                    const int fi = 2 * ci + o[0], fj = 2 * cj + o[1],
                              fk = DIM == 3 ? 2 * ck + o[2] : 0;
                    const int fidx = (fk * F.g.ny + fj) * F.g.nx + fi;
                    T bf;
                    if (F.beta[0] == nullptr) {
                        const Nb6 nb = nb6<DIM>(F.g, fi, fj, fk, fidx);
                        bf = wall_face(F.g, fj, 2 * d)
                                 ? T(0)
                                 : T(beta_face32(float(__ldg(phi + fidx)),
                                                 float(__ldg(phi + nb.m[2 * d])), ph));
                    } else {
                        bf = F.beta[d][fidx];
                    }
                    s += bf;
                }
            C.beta[d][I] = s * T(DIM == 3 ? 0.25 : 0.5);
        }
    });
}

// 3D float32, a tiled coarse level from the cell densities of the level above:
// the coarse density of a cell is the mean of its 8 children's (stored in
// rhoc), and the face coefficient is 1 / rho_f of the two coarse densities (a
// rediscretised coarse operator, which the level's TMA-staged sweep and
// restriction form from rhoc the way level 0's do from its densities)
__global__ void __launch_bounds__(kThreads)
k_beta_rho(MGLevel<float> C, const float* __restrict__ rhof, Dims fg, float* __restrict__ rhoc) {
    for_cells(C.g, [&](int ci, int cj, int ck, int I) {
        auto mean8 = [&](int a, int b, int c) {
            float s = 0.f;
#pragma unroll
            for (int dz = 0; dz < 2; ++dz)
#pragma unroll
                for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 2; ++dx)
                        s += __ldg(rhof + ((size_t)(2 * c + dz) * fg.ny + 2 * b + dy) * fg.nx +
                                   2 * a + dx);
            return 0.125f * s;
        };
        const float rc = mean8(ci, cj, ck);
        rhoc[I] = rc;
        const float rx = mean8(wrapi(ci - 1, C.g.nx), cj, ck);
        const float ry = mean8(ci, wrapi(cj - 1, C.g.ny), ck);
        const float rz = mean8(ci, cj, wrapi(ck - 1, C.g.nz));
        C.beta[0][I] = __frcp_rn(0.5f * (rc + rx));
        C.beta[1][I] = __frcp_rn(0.5f * (rc + ry));
        C.beta[2][I] = __frcp_rn(0.5f * (rc + rz));
    });
}

// float64 face coefficients 1 / rho_f (float64 path)
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_beta0(Dims g, Phys ph, const T* __restrict__ phi, double* __restrict__ b0,
        double* __restrict__ b1, double* __restrict__ b2) {
    const PC<double> pc = pc_of(ph, double());
    for_cells(g, [&](int i, int j, int k, int idx) {
        const Nb6 nb = nb6<DIM>(g, i, j, k, idx);
        const double rc = rho_of_p(double(__ldg(phi + idx)), pc);
        double* bb[3] = {b0, b1, b2};
#pragma unroll
        for (int d = 0; d < DIM; ++d)
            bb[d][idx] = wall_face(g, j, 2 * d)
                             ? 0.0
                             : 1.0 / (0.5 * (rc + rho_of_p(double(__ldg(phi + nb.m[2 * d])), pc)));
    });
}

// float32 face coefficients of the mixed path (the same beta_face32 as every
// kernel that evaluates them from phi) and, optionally, the cell densities
// rho32(phi) that the finest smoother reads
template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_beta0_32(Dims g, Phys ph, const float* __restrict__ phi, float* __restrict__ b0,
           float* __restrict__ b1, float* __restrict__ b2, float* __restrict__ rho) {
    for_cells(g, [&](int i, int j, int k, int idx) {
        const Nb6 nb = nb6<DIM>(g, i, j, k, idx);
        const float pc = __ldg(phi + idx);
        if (rho) rho[idx] = rho32(pc, ph);
        b0[idx] = beta_face32(pc, __ldg(phi + nb.m[0]), ph);
        b1[idx] = wall_face(g, j, 2) ? 0.f : beta_face32(pc, __ldg(phi + nb.m[2]), ph);
        if (DIM == 3) b2[idx] = beta_face32(pc, __ldg(phi + nb.m[4]), ph);
    });
}

template <int DIM>
void launch_beta0_32(const Dims& g, const Phys& ph, const float* phi, float* const* beta,
                     float* rho, cudaStream_t s) {
    k_beta0_32<DIM><<<row_grid(g, kThreads, 1 << 30), kThreads, 0, s>>>(
        g, ph, phi, beta[0], beta[1], DIM == 3 ? beta[2] : beta[1], rho);
}
template void launch_beta0_32<2>(const Dims&, const Phys&, const float*, float* const*, float*,
                                 cudaStream_t);
template void launch_beta0_32<3>(const Dims&, const Phys&, const float*, float* const*, float*,
                                 cudaStream_t);

// ---------------------------------------------------------------------------
// single-CTA kernel for all levels >= first_coarse
// ---------------------------------------------------------------------------
constexpr int kCoarseThreads = 1024;
constexpr size_t kCoarseSmemMax = 200 * 1024;   // staged coarse hierarchy, bytes

// One colour of a red-black sweep over a (small) level by threads t0, t0 + nt,
// ...: item q = (row, m) with cell i = 2 m + parity(row) of the colour; all:
// the other colour's cell of the pair is zeroed. Rows and positions come from
// float reciprocals: (q + 1/2) / n lies at least 1/(2n) from an integer and
// the two roundings move it by at most (q + 1/2) 2^-23 / n, so the quotient
// truncates exactly for q < 2^22 (levels up to 2^20 cells run here).
template <typename T, int DIM>
__device__ __forceinline__ void cta_cells(const Dims& g, int color, bool all, const MGLevel<T>& L,
                                          const T* phi, const Phys& ph, bool zero_start,
                                          int t0, int nt) {
    const int nhx = (g.nx + 1) >> 1;
    const int rows = g.ny * g.nz;
    const int items = rows * nhx;
    const float inv_nhx = 1.0f / float(nhx), inv_ny = 1.0f / float(g.ny);
    for (int q = t0; q < items; q += nt) {
        const int r = int((float(q) + 0.5f) * inv_nhx);
        const int m = q - r * nhx;
        const int k = int((float(r) + 0.5f) * inv_ny);
        const int j = r - k * g.ny;
        const int par = (j + k + color) & 1;
        const int i = 2 * m + par;
        const int base = r * g.nx;
        if (i < g.nx) gs_cell<T, DIM>(L, phi, ph, i, j, k, base + i, zero_start);
        if (all) {
            const int io = 2 * m + (1 - par);
            if (io < g.nx) L.x[base + io] = T(0);
        }
    }
}

// Cell coordinates of a linear index on a small level by float reciprocals
// (exact for idx < 2^22, by the argument given for the sweep items above).
__device__ __forceinline__ Cell decode_small(int idx, const Dims& g, float inv_nx, float inv_ny) {
    Cell c;
    const int r = int((float(idx) + 0.5f) * inv_nx);
    c.i = idx - r * g.nx;
    c.k = int((float(r) + 0.5f) * inv_ny);
    c.j = r - c.k * g.ny;
    return c;
}

// V-cycle over levels l0..lb of L (one CTA): pre-sweeps and restriction on the
// way down, many sweeps on the coarsest level (after removing the mean of its
// right-hand side), prolongation and post-sweeps on the way up.
template <typename T, int DIM>
__device__ __forceinline__ void coarse_vcycle_body(MGLevel<T>* L_, int l0, int lb, int pre,
                                                   int post, int coarse_sweeps,
                                                   const T* __restrict__ phi, const Phys& ph,
                                                   double* red) {
    const int tid = threadIdx.x, nt = blockDim.x;
    // down
    for (int l = l0; l < lb; ++l) {
        const MGLevel<T>& L = L_[l];
        for (int s = 0; s < pre; ++s) {
            cta_cells<T, DIM>(L.g, 0, s == 0, L, phi, ph, s == 0, tid, nt);
            __syncthreads();
            cta_cells<T, DIM>(L.g, 1, false, L, phi, ph, false, tid, nt);
            __syncthreads();
        }
        const MGLevel<T>& C = L_[l + 1];
        const float cix = 1.0f / float(C.g.nx), ciy = 1.0f / float(C.g.ny);
        for (int I = tid; I < C.g.ncell; I += nt) {
            Cell c = decode_small(I, C.g, cix, ciy);
            restrict_cell<T, DIM>(L, C, phi, ph, c.i, c.j, c.k, I);
        }
        __syncthreads();
    }
    // bottom: remove the mean of f (compatibility), then many sweeps
    {
        const MGLevel<T>& L = L_[lb];
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
        for (int s2 = 0; s2 < coarse_sweeps; ++s2) {
            cta_cells<T, DIM>(L.g, 0, s2 == 0, L, phi, ph, s2 == 0, tid, nt);
            __syncthreads();
            cta_cells<T, DIM>(L.g, 1, false, L, phi, ph, false, tid, nt);
            __syncthreads();
        }
    }
    // up
    for (int l = lb - 1; l >= l0; --l) {
        const MGLevel<T>& L = L_[l];
        const float fix = 1.0f / float(L.g.nx), fiy = 1.0f / float(L.g.ny);
        for (int i = tid; i < L.g.ncell; i += nt) {
            Cell c = decode_small(i, L.g, fix, fiy);
            prolong_cell<T, DIM>(L, L_[l + 1], c.i, c.j, c.k, i);
        }
        __syncthreads();
        for (int s = 0; s < post; ++s) {
            cta_cells<T, DIM>(L.g, 1, false, L, phi, ph, false, tid, nt);
            __syncthreads();
            cta_cells<T, DIM>(L.g, 0, false, L, phi, ph, false, tid, nt);
            __syncthreads();
        }
    }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kCoarseThreads)
k_coarse_vcycle(MGHier<T> H, const T* __restrict__ phi, Phys ph, const CGScalars* sc) {
    if (inner_stopped(sc)) return;
    __shared__ double red[32];
    __shared__ MGLevel<T> Ls[kMaxLevels];   // one copy of the level descriptors
    if (threadIdx.x == 0)
        for (int l = 0; l < H.nlev; ++l) Ls[l] = H.lev[l];
    __syncthreads();
    coarse_vcycle_body<T, DIM>(Ls, H.first_coarse, H.nlev - 1, H.pre, H.post, H.coarse_sweeps,
                               phi, ph, red);
}

// The same V-cycle on copies in shared memory: every coarse level's
// correction, right-hand side and face coefficients (about 85 KB for a 2D
// float32 hierarchy below 64^2) are staged in once, so the ~70 dependent
// half-sweeps and transfers of one call run at shared-memory latency instead
// of L2 latency. Only the first coarse level's right-hand side (written by
// the restriction) comes in and only its correction goes out.
template <typename T, int DIM>
__global__ void __launch_bounds__(kCoarseThreads)
k_coarse_vcycle_smem(MGHier<T> H, const T* __restrict__ phi, Phys ph, const CGScalars* sc) {
    if (inner_stopped(sc)) return;
    __shared__ double red[32];
    extern __shared__ __align__(16) unsigned char craw[];
    T* sm = reinterpret_cast<T*>(craw);
    const int l0 = H.first_coarse, lb = H.nlev - 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    __shared__ MGLevel<T> S[kMaxLevels];   // level descriptors viewing the staged copies
    if (tid == 0) {
        int off = 0;
        for (int l = l0; l <= lb; ++l) {
            S[l] = H.lev[l];
            const int n = S[l].g.ncell;
            S[l].x = sm + off;
            off += n;
            S[l].f = sm + off;
            off += n;
            for (int d = 0; d < 3; ++d) {
                S[l].beta[d] = d < DIM ? sm + off : nullptr;
                if (d < DIM) off += n;
            }
        }
    }
    __syncthreads();
    for (int l = l0; l <= lb; ++l)
        for (int d = 0; d < DIM; ++d)
            for (int i = tid; i < S[l].g.ncell; i += nt) S[l].beta[d][i] = H.lev[l].beta[d][i];
    for (int i = tid; i < S[l0].g.ncell; i += nt) S[l0].f[i] = H.lev[l0].f[i];
    __syncthreads();
    coarse_vcycle_body<T, DIM>(S, l0, lb, H.pre, H.post, H.coarse_sweeps, phi, ph, red);
    for (int i = tid; i < S[l0].g.ncell; i += nt) H.lev[l0].x[i] = S[l0].x[i];
}

// shared-memory bytes of the staged coarse hierarchy, or 0 when it does not
// fit (or a level computes its coefficients from phi)
template <typename T, int DIM>
size_t coarse_smem_bytes(const MGHier<T>& H) {
    size_t n = 0;
    for (int l = H.first_coarse; l < H.nlev; ++l) {
        for (int d = 0; d < DIM; ++d)
            if (H.lev[l].beta[d] == nullptr) return 0;
        n += (size_t)H.lev[l].g.ncell * (2 + DIM);
    }
    const size_t bytes = n * sizeof(T);
    return bytes <= kCoarseSmemMax ? bytes : 0;
}

template <typename T, int DIM>
void coarse_smem_attribute() {
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_coarse_vcycle_smem<T, DIM>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCoarseSmemMax);
    });
}

template <typename T, int DIM>
void launch_mg_setup(const Dims&, const Phys& ph, const T* phi, MGHier<T>& H, cudaStream_t s) {
    for (int l = 0; l + 1 < H.nlev; ++l) {
        if constexpr (DIM == 3 && sizeof(T) == sizeof(float)) {
            const float* rf = l == 0 ? H.rho0 : H.rhoc[l];
            if (rf != nullptr && H.rhoc[l + 1] != nullptr) {
                k_beta_rho<<<row_grid(H.lev[l + 1].g, kThreads, 1 << 30), kThreads, 0, s>>>(
                    reinterpret_cast<const MGLevel<float>&>(H.lev[l + 1]), rf, H.lev[l].g,
                    H.rhoc[l + 1]);
                continue;
            }
        }
        k_coarsen_beta<T, DIM><<<row_grid(H.lev[l + 1].g, kThreads, 1 << 30), kThreads, 0, s>>>(
            H.lev[l], H.lev[l + 1], phi, ph);
    }
}

template <typename T, int DIM>
void launch_beta0(const Dims& g, const Phys& ph, const T* phi, double* const* beta,
                  cudaStream_t s) {
    k_beta0<T, DIM><<<row_grid(g, kThreads, 1 << 30), kThreads, 0, s>>>(
        g, ph, phi, beta[0], beta[1], DIM == 3 ? beta[2] : beta[1]);
}

// Tiled one-pass sweeps apply to 3D float32 levels with even sizes and an
// out-of-place buffer; every other level uses the half-sweep kernels.
template <typename T, int DIM>
static bool tiled_level(const MGLevel<T>& L) {
    if constexpr (DIM == 3 && sizeof(T) == sizeof(float)) {
        return L.x2 != nullptr && sweep3d_ok(L.g);
    } else {
        return false;
    }
}

template <typename T, int DIM>
T* launch_vcycle(const Phys& ph, const T* phi, MGHier<T>& H, const CGScalars* sc,
                 cudaStream_t s, Prof* pr, const SweepDots* dots, bool* dots_done) {
    if (dots_done) *dots_done = false;
    const int l0 = H.first_coarse;
    // finest tiled sweep: the precomputed cell densities when present, else phi
    const float* phi0 = H.rho0 != nullptr ? H.rho0 : reinterpret_cast<const float*>(phi);
    const int rho_ready = H.rho0 != nullptr ? 1 : 0;
    // coefficient source of a tiled level's sweep: the level's densities (phi
    // on level 0 without them), else its face arrays
    auto dens = [&](int l) -> const float* {
        return l == 0 ? phi0 : (H.rho0 != nullptr ? H.rhoc[l] : nullptr);
    };
    auto rho_ready_of = [&](int l) { return l == 0 ? rho_ready : 1; };
    T* fin[kMaxLevels];   // buffer holding each level's result
    for (int l = l0; l < H.nlev; ++l) fin[l] = H.lev[l].x;
    auto gs = [&](const MGLevel<T>& L, int lvl, int color, int zero) {
        pr->begin(lvl == 0 ? KC_GS0 : KC_GS);
        k_gs<T, DIM><<<row_grid(L.g, kThreads, 1 << 30), kThreads, 0, s>>>(L, phi, ph, color,
                                                                          zero, sc);
        pr->end();
    };
    T* pre_buf[kMaxLevels];
    for (int l = 0; l < l0; ++l) {
        MGLevel<T> L = H.lev[l];
        if (tiled_level<T, DIM>(L)) {
            if constexpr (DIM == 3 && sizeof(T) == sizeof(float)) {
                // the zero-start sweep writes x; each further sweep reads the
                // current buffer and writes the other
                T* cur = L.x;
                T* oth = L.x2;
                for (int p = 0; p < H.pre; ++p) {
                    pr->begin(l == 0 ? KC_GS0 : KC_GS);
                    const float* xin = p == 0 ? nullptr : reinterpret_cast<const float*>(cur);
                    float* xout = reinterpret_cast<float*>(p == 0 ? cur : oth);
                    if (!(launch_sweep_tma(l == 0 ? H.tma : H.tmac[l],
                                                     reinterpret_cast<const MGLevel<float>&>(L),
                                                     xin, xout, nullptr, 0, sc, s)))
                        launch_sweep3d(reinterpret_cast<const MGLevel<float>&>(L), dens(l),
                                       rho_ready_of(l), ph, xin, xout, nullptr, 0, sc, s);
                    pr->end();
                    if (p > 0) { T* t = cur; cur = oth; oth = t; }
                }
                pre_buf[l] = cur;
            }
        } else {
            for (int p = 0; p < H.pre; ++p) {
                gs(L, l, 0, p == 0);
                gs(L, l, 1, 0);
            }
            pre_buf[l] = L.x;
        }
        L.x = pre_buf[l];
        pr->begin(KC_RESTRICT);
        bool done_r = false;
        if constexpr (DIM == 3 && sizeof(T) == sizeof(float)) {
            if (L.beta[0] != nullptr && restrict3d_ok(L.g)) {
                launch_restrict3d(reinterpret_cast<const MGLevel<float>&>(L),
                                  reinterpret_cast<const MGLevel<float>&>(H.lev[l + 1]),
                                  l == 0 ? H.rho0 : H.rhoc[l], sc, s);
                done_r = true;
            }
        }
        if (!done_r)
            k_restrict<T, DIM><<<row_grid(H.lev[l + 1].g, kThreads, 1 << 30), kThreads, 0, s>>>(
                L, H.lev[l + 1], phi, ph, sc);
        pr->end();
    }
    pr->begin(KC_COARSE);
    const size_t cbytes = coarse_smem_bytes<T, DIM>(H);
    if (cbytes > 0) {
        coarse_smem_attribute<T, DIM>();
        k_coarse_vcycle_smem<T, DIM><<<1, kCoarseThreads, cbytes, s>>>(H, phi, ph, sc);
    } else {
        k_coarse_vcycle<T, DIM><<<1, kCoarseThreads, 0, s>>>(H, phi, ph, sc);
    }
    pr->end();
    for (int l = l0 - 1; l >= 0; --l) {
        MGLevel<T> L = H.lev[l];
        MGLevel<T> C = H.lev[l + 1];
        C.x = fin[l + 1];
        if (tiled_level<T, DIM>(L)) {
            if constexpr (DIM == 3 && sizeof(T) == sizeof(float)) {
                T* cur = pre_buf[l];
                T* oth = cur == L.x ? L.x2 : L.x;
                MGLevel<T> Lp = L;
                Lp.x = cur;
                pr->begin(KC_PROLONG);
                if (2 * C.g.nx == L.g.nx && 2 * C.g.ny == L.g.ny && 2 * C.g.nz == L.g.nz) {
                    // coarse-column z-march; chunks of kc planes, at least
                    // about eight CTAs per SM in all
                    const int bx = (C.g.nx + 31) / 32, by = (C.g.ny + 7) / 8;
                    int kc = 16;
                    while (kc > 1 && (long long)bx * by * ((C.g.nz + kc - 1) / kc) < 8 * 152)
                        kc >>= 1;
                    const dim3 grd(bx, by, (C.g.nz + kc - 1) / kc);
                    k_prolong_zm<<<grd, 256, 0, s>>>(reinterpret_cast<const MGLevel<float>&>(Lp),
                                                     reinterpret_cast<const MGLevel<float>&>(C),
                                                     kc, sc);
                } else {
                    const int npair = L.g.nx >> 1;
                    const dim3 blk(npair >= 64 ? 64 : 32, npair >= 64 ? 4 : 8);
                    const dim3 grd((npair + blk.x - 1) / blk.x, (L.g.ny + blk.y - 1) / blk.y,
                                   L.g.nz);
                    k_prolong_pairs<T><<<grd, blk, 0, s>>>(Lp, C, sc);
                }
                pr->end();
                for (int p = 0; p < H.post; ++p) {
                    // the last level-0 sweep also forms the CG dot products
                    const bool fuse = dots && l == 0 && p == H.post - 1 &&
                                      2 * sweep3d_blocks(L.g) <= kRedPart;
                    pr->begin(l == 0 ? KC_GS0 : KC_GS);
                    const float* xin = reinterpret_cast<const float*>(cur);
                    float* xout = reinterpret_cast<float*>(oth);
                    if (!(launch_sweep_tma(l == 0 ? H.tma : H.tmac[l],
                                                     reinterpret_cast<const MGLevel<float>&>(L),
                                                     xin, xout, fuse ? dots : nullptr, 1, sc, s)))
                        launch_sweep3d(reinterpret_cast<const MGLevel<float>&>(L), dens(l),
                                       rho_ready_of(l), ph, xin, xout, fuse ? dots : nullptr, 1,
                                       sc, s);
                    pr->end();
                    if (fuse && dots_done) *dots_done = true;
                    T* t = cur; cur = oth; oth = t;
                }
                fin[l] = cur;
            }
        } else {
            L.x = pre_buf[l];
            pr->begin(KC_PROLONG);
            k_prolong<T, DIM><<<row_grid(L.g, kThreads, 1 << 30), kThreads, 0, s>>>(L, C, sc);
            pr->end();
            for (int p = 0; p < H.post; ++p) {
                gs(L, l, 1, 0);
                gs(L, l, 0, 0);
            }
            fin[l] = L.x;
        }
    }
    return fin[0];
}

// ---------------------------------------------------------------------------
// float64 outer kernels
// ---------------------------------------------------------------------------
// (A x)_c in float64 with the same face coefficients as the inner operator
template <typename T, int DIM>
__device__ __forceinline__ double apply_A64(const Dims& g, const Phys& ph,
                                            const SolveIO<T, DIM>& io, const double* __restrict__ x,
                                            int i, int j, int k, int idx) {
    const Nb6 nb = nb6<DIM>(g, i, j, k, idx);
    const double ih2 = g.ih2;
    const double xc = x[idx];
    double ax = 0.0;
    if (io.beta64[0] != nullptr) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            ax += io.beta64[d][idx] * (xc - x[nb.m[2 * d]]);
            ax += io.beta64[d][nb.m[2 * d + 1]] * (xc - x[nb.m[2 * d + 1]]);
        }
    } else if (io.beta32[0] != nullptr) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            ax += double(__ldg(io.beta32[d] + idx)) * (xc - x[nb.m[2 * d]]);
            ax += double(__ldg(io.beta32[d] + nb.m[2 * d + 1])) * (xc - x[nb.m[2 * d + 1]]);
        }
    } else {
        const float pc = float(__ldg(io.phi + idx));
#pragma unroll
        for (int q = 0; q < 2 * DIM; ++q)
            if (!wall_face(g, j, q))
                ax += double(beta_face32(pc, float(__ldg(io.phi + nb.m[q])), ph)) *
                      (xc - x[nb.m[q]]);
    }
    return ax * ih2;
}

// r = f - A x with f = sign (b - mean b); r stored in T for the inner solve.
// first: also ||f||^2 and the solve's counters.
// Float64 path: x, b float64. Mixed path: x and b are double-floats (hi plane,
// lo plane) and the residual is formed with error-free transformations on the
// float32 pipe (GB300's float64 pipe is narrow): each x_c - x_q as an exact
// TwoSum of the hi parts plus the lo difference, each product with the float32
// face coefficient as an exact TwoProduct, the six products summed with
// TwoSum and every rounding error carried in a second float (a compensated
// dot product, as accurate as evaluation in twice the working precision). Its
// rounding floor is about 2^-48 |x| |sum beta| per cell, i.e. a relative
// residual near 1e-16 N^2 for a smooth solution on an N-cell axis.
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_ir_residual(Dims g, Phys ph, SolveIO<T, DIM> io, int first, RedBuf rb, CGScalars* sc) {
    if (!first && sc->done) return;
    const double mb = sc->mean_b;
    const bool pos = io.sign > 0.0;
    // norms accumulate the rounded values per thread in T (a stopping test
    // needs a few digits); the residual itself is formed to float64 accuracy
    T ff = T(0), rr = T(0);
    if constexpr (sizeof(T) == sizeof(float)) {
        const int n = g.ncell;
        const float* __restrict__ xh = reinterpret_cast<const float*>(io.x);
        const float* __restrict__ xl = xh + n;
        const float* __restrict__ bh = reinterpret_cast<const float*>(io.b);
        const float* __restrict__ bl = bh + n;
        const f2 mdf = df_neg(df_of(mb));
        const f2 ih2 = df_of(g.ih2);
        for_cells(g, [&](int i, int j, int k, int idx) {
            f2 f = df_add(f2{bh[idx], bl[idx]}, mdf);
            if (!pos) f = df_neg(f);
            const Nb6 nb = nb6<DIM>(g, i, j, k, idx);
            const float xch = xh[idx], xcl = xl[idx];
            const float pc = io.beta32[0] != nullptr ? 0.f : float(__ldg(io.phi + idx));
            float S = 0.f, c = 0.f;
#pragma unroll
            for (int q = 0; q < 2 * DIM; ++q) {
                const int m = nb.m[q];
                // face q of the cell: the minus face is stored at the cell, the
                // plus face at the neighbour
                float beta;
                if (io.beta32[0] != nullptr)
                    beta = __ldg(io.beta32[q >> 1] + ((q & 1) ? m : idx));
                else
                    beta = wall_face(g, j, q) ? 0.f : beta_face32(pc, float(__ldg(io.phi + m)), ph);
                df_face_term(beta, xch, xcl, xh[m], xl[m], S, c);
            }
            const f2 ax = f2_mul(two_sum(S, c), ih2);
            const f2 r = df_add(f, df_neg(ax));
            const float rt = __fadd_rn(r.hi, r.lo);
            io.r[idx] = rt;
            if (first) {
                const float ft = __fadd_rn(f.hi, f.lo);
                ff += ft * ft;
            }
            rr += rt * rt;
        });
    } else {
        for_cells(g, [&](int i, int j, int k, int idx) {
            const double f = pos ? io.b[idx] - mb : mb - io.b[idx];
            const double rv = f - apply_A64<T, DIM>(g, ph, io, io.x, i, j, k, idx);
            const T rt = T(rv);
            io.r[idx] = rt;
            if (first) {
                const T ft = T(f);
                ff += ft * ft;
            }
            rr += rt * rt;
        });
    }
    double v[3] = {double(ff), double(rr), double(rr)}, tot[3];
    const int mode[3] = {0, 0, 0};
    if (grid_reduce<3>(v, mode, rb, tot) && threadIdx.x == 0) ir_finish(tot, first, sc);
}

// x += e (mixed path: x a double-float, hi plane and lo plane)
__device__ __forceinline__ void df_acc(float& h, float& l, float e) {
    const f2 s = two_sum(h, e);
    const f2 r = two_sum(s.hi, __fadd_rn(s.lo, l));
    h = r.hi;
    l = r.lo;
}
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_ir_addcorr(Dims g, SolveIO<T, DIM> io, const CGScalars* sc) {
    if (sc->done) return;
    if constexpr (sizeof(T) == sizeof(float)) {
        float* __restrict__ xh = reinterpret_cast<float*>(io.x);
        float* __restrict__ xl = xh + g.ncell;
        const int stride = gridDim.x * blockDim.x;
        if ((g.ncell & 3) == 0) {
            const int n4 = g.ncell >> 2;
            const float4* __restrict__ e4 = reinterpret_cast<const float4*>(io.e);
            float4* __restrict__ h4 = reinterpret_cast<float4*>(xh);
            float4* __restrict__ l4 = reinterpret_cast<float4*>(xl);
            for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += stride) {
                const float4 ev = e4[t];
                float4 h = h4[t], l = l4[t];
                df_acc(h.x, l.x, ev.x);
                df_acc(h.y, l.y, ev.y);
                df_acc(h.z, l.z, ev.z);
                df_acc(h.w, l.w, ev.w);
                h4[t] = h;
                l4[t] = l;
            }
            return;
        }
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.ncell; t += stride)
            df_acc(xh[t], xl[t], io.e[t]);
        return;
    }
    for_cells(g, [&](int, int, int, int idx) { io.x[idx] += double(io.e[idx]); });
}

// ---------------------------------------------------------------------------
// inner flexible CG in precision T (float64 scalars)
// ---------------------------------------------------------------------------
// rz = r.z ; zq = z.q (previous q) ; beta = -alpha zq / rz_old
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_in_dots(Dims g, SolveIO<T, DIM> io, int first_arg, RedBuf rb, CGScalars* sc) {
    if (inner_stopped(sc)) return;
    const int first = first_of(first_arg, sc);
    double rz = 0.0, zq = 0.0;
    for_cells(g, [&](int, int, int, int idx) {
        const double zv = double(io.z[idx]);
        rz += double(io.r[idx]) * zv;
        if (!first) zq += zv * double(io.q[idx]);
    });
    double v[2] = {rz, zq}, tot[2];
    const int mode[2] = {0, 0};
    if (grid_reduce<2>(v, mode, rb, tot) && threadIdx.x == 0) {
        sc->beta = first ? 0.0 : -sc->alpha * tot[1] / sc->rz;
        sc->rz = tot[0];
    }
}

// p_new = z + beta p_old ; q = A p_new ; alpha = rz / (p.q)
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_in_dir(Dims g, Phys ph, SolveIO<T, DIM> io, int cur, int first_arg, RedBuf rb,
         CGScalars* sc) {
    if (inner_stopped(sc)) return;
    const int first = first_of(first_arg, sc);
    const T beta = first ? T(0) : T(sc->beta);
    const T* __restrict__ po = cur ? io.p[1] : io.p[0];
    T* __restrict__ pn = cur ? io.p[0] : io.p[1];
    const T ih2 = ih2_of(g, T());
    double pq = 0.0;
    for_cells(g, [&](int i, int j, int k, int idx) {
        const Nb6 nb = nb6<DIM>(g, i, j, k, idx);
        const T pc = first ? io.z[idx] : io.z[idx] + beta * po[idx];
        T ax = T(0);
        if (io.beta64[0] != nullptr) {
#pragma unroll
            for (int q = 0; q < 2 * DIM; ++q) {
                const int m = nb.m[q];
                const T pm = first ? io.z[m] : io.z[m] + beta * po[m];
                const int d = q >> 1;
                const T bf = T((q & 1) ? io.beta64[d][m] : io.beta64[d][idx]);
                ax += bf * (pc - pm);
            }
        } else if (io.beta32[0] != nullptr) {
#pragma unroll
            for (int q = 0; q < 2 * DIM; ++q) {
                const int m = nb.m[q];
                const T pm = first ? io.z[m] : io.z[m] + beta * po[m];
                const int d = q >> 1;
                const T bf = T(__ldg(io.beta32[d] + ((q & 1) ? m : idx)));
                ax += bf * (pc - pm);
            }
        } else {
            const float phc = float(__ldg(io.phi + idx));
#pragma unroll
            for (int q = 0; q < 2 * DIM; ++q) {
                const int m = nb.m[q];
                const T pm = first ? io.z[m] : io.z[m] + beta * po[m];
                if (!wall_face(g, j, q))
                    ax += T(beta_face32(phc, float(__ldg(io.phi + m)), ph)) * (pc - pm);
            }
        }
        ax *= ih2;
        pn[idx] = pc;
        io.q[idx] = ax;
        pq += double(pc) * double(ax);
    });
    double v[1] = {pq}, tot[1];
    const int mode[1] = {0};
    if (grid_reduce<1>(v, mode, rb, tot) && threadIdx.x == 0) {
        sc->pq = tot[0];
        sc->alpha = tot[0] != 0.0 ? sc->rz / tot[0] : 0.0;
    }
}

// e += alpha p ; r -= alpha q ; ||r||^2 ; inner stopping test
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_in_update(Dims g, SolveIO<T, DIM> io, int cur, int first_arg, RedBuf rb, CGScalars* sc) {
    if (inner_stopped(sc)) return;
    const int first = first_of(first_arg, sc);
    const T alpha = T(sc->alpha);
    const T* __restrict__ pn = cur ? io.p[0] : io.p[1];
    T rr = T(0);   // per-thread partial in T, float64 across threads
    bool done = false;
    if constexpr (sizeof(T) == sizeof(float)) {
        // float32 vectors in 16-byte pieces (sub-buffers are 256-byte aligned):
        // four times the bytes in flight per load
        if ((g.ncell & 3) == 0) {
            const int n4 = g.ncell >> 2;
            const float4* __restrict__ p4 = reinterpret_cast<const float4*>(pn);
            const float4* __restrict__ q4 = reinterpret_cast<const float4*>(io.q);
            float4* __restrict__ e4 = reinterpret_cast<float4*>(io.e);
            float4* __restrict__ r4 = reinterpret_cast<float4*>(io.r);
            const int stride = gridDim.x * blockDim.x;
#pragma unroll 2
            for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += stride) {
                const float4 pv = p4[t], qv = q4[t];
                float4 rv = r4[t];
                float4 ev = first ? make_float4(0.f, 0.f, 0.f, 0.f) : e4[t];
                ev.x += alpha * pv.x;
                ev.y += alpha * pv.y;
                ev.z += alpha * pv.z;
                ev.w += alpha * pv.w;
                rv.x -= alpha * qv.x;
                rv.y -= alpha * qv.y;
                rv.z -= alpha * qv.z;
                rv.w -= alpha * qv.w;
                e4[t] = ev;
                r4[t] = rv;
                rr += (rv.x * rv.x + rv.y * rv.y) + (rv.z * rv.z + rv.w * rv.w);
            }
            done = true;
        }
    }
    if (!done) {
        for_cells(g, [&](int, int, int, int idx) {
            const T pv = pn[idx];
            io.e[idx] = first ? alpha * pv : io.e[idx] + alpha * pv;
            const T rv = io.r[idx] - alpha * io.q[idx];
            io.r[idx] = rv;
            rr += rv * rv;
        });
    }
    double v[1] = {double(rr)}, tot[1];
    const int mode[1] = {0};
    if (grid_reduce<1>(v, mode, rb, tot) && threadIdx.x == 0) {
        sc->rr_in = tot[0];
        sc->iters += 1;
        sc->it_in += 1;
        if (!(tot[0] == tot[0])) {
            sc->idone = 1;
        } else if (tot[0] <= sc->eta2 * sc->rr0_in) {
            sc->idone = 1;
        } else if (sc->iters >= sc->maxit) {
            sc->idone = 1;
            sc->capped = 1;
        }
    }
}

void coarse_prepare() {
    coarse_smem_attribute<float, 2>();
    coarse_smem_attribute<float, 3>();
    coarse_smem_attribute<double, 2>();
    coarse_smem_attribute<double, 3>();
}

// Condition of a WHILE node of a solve captured in a CUDA graph: which = 0
// inner CG loop (runs while the inner solve has not stopped), which = 1 outer
// refinement loop (runs while the solve has not converged or stopped; at most
// 64 outer residuals, as in the host-driven loop).
__global__ void k_set_cond(cudaGraphConditionalHandle h, const CGScalars* sc, int which) {
    unsigned v;
    if (which == 0) v = (sc->done || sc->idone) ? 0u : 1u;
    else v = (!sc->done && sc->outer < 64) ? 1u : 0u;
    cudaGraphSetConditional(h, v);
}
void launch_set_cond(cudaGraphConditionalHandle h, const CGScalars* sc, int which, cudaStream_t s) {
    k_set_cond<<<1, 1, 0, s>>>(h, sc, which);
}

template <typename T, int DIM>
void launch_ir_residual(const Dims& g, const Phys& ph, const SolveIO<T, DIM>& io, int first,
                        RedBuf rb, CGScalars* sc, cudaStream_t s) {
    if constexpr (DIM == 3 && sizeof(T) == sizeof(float)) {
        if (io.beta32[0] != nullptr && ir3d_ok(g)) {
            launch_ir_residual3d(g, reinterpret_cast<const float*>(io.x),
                                 reinterpret_cast<const float*>(io.b), io.beta32, io.sign,
                                 reinterpret_cast<float*>(io.r), first, rb, sc, s);
            return;
        }
    }
    k_ir_residual<T, DIM><<<row_grid(g, kThreads, kRedBlocks), kThreads, 0, s>>>(g, ph, io, first,
                                                                                  rb, sc);
}
template <typename T, int DIM>
void launch_ir_addcorr(const Dims& g, const SolveIO<T, DIM>& io, CGScalars* sc, cudaStream_t s) {
    k_ir_addcorr<T, DIM><<<row_grid(g, kThreads, 1 << 30), kThreads, 0, s>>>(g, io, sc);
}
template <typename T, int DIM>
void launch_in_dots(const Dims& g, const SolveIO<T, DIM>& io, int first, RedBuf rb,
                    CGScalars* sc, cudaStream_t s) {
    k_in_dots<T, DIM><<<row_grid(g, kThreads, kRedBlocks), kThreads, 0, s>>>(g, io, first, rb, sc);
}
template <typename T, int DIM>
void launch_in_dir(const Dims& g, const Phys& ph, const SolveIO<T, DIM>& io, int cur, int first,
                   RedBuf rb, CGScalars* sc, cudaStream_t s) {
    k_in_dir<T, DIM><<<row_grid(g, kThreads, kRedBlocks), kThreads, 0, s>>>(g, ph, io, cur, first,
                                                                             rb, sc);
}
template <typename T, int DIM>
void launch_in_update(const Dims& g, const SolveIO<T, DIM>& io, int cur, int first, RedBuf rb,
                      CGScalars* sc, cudaStream_t s) {
    k_in_update<T, DIM><<<row_grid(g, kThreads, kRedBlocks), kThreads, 0, s>>>(g, io, cur, first,
                                                                                rb, sc);
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

#define PF_INST_P(T, D)                                                                          \
    template void launch_mg_setup<T, D>(const Dims&, const Phys&, const T*, MGHier<T>&,          \
                                        cudaStream_t);                                           \
    template void launch_beta0<T, D>(const Dims&, const Phys&, const T*, double* const*,         \
                                     cudaStream_t);                                              \
    template T* launch_vcycle<T, D>(const Phys&, const T*, MGHier<T>&, const CGScalars*,         \
                                    cudaStream_t, Prof*, const SweepDots*, bool*);               \
    template void launch_ir_residual<T, D>(const Dims&, const Phys&, const SolveIO<T, D>&, int,  \
                                           RedBuf, CGScalars*, cudaStream_t);                    \
    template void launch_ir_addcorr<T, D>(const Dims&, const SolveIO<T, D>&, CGScalars*,         \
                                          cudaStream_t);                                         \
    template void launch_in_dots<T, D>(const Dims&, const SolveIO<T, D>&, int, RedBuf,           \
                                       CGScalars*, cudaStream_t);                                \
    template void launch_in_dir<T, D>(const Dims&, const Phys&, const SolveIO<T, D>&, int, int,  \
                                      RedBuf, CGScalars*, cudaStream_t);                         \
    template void launch_in_update<T, D>(const Dims&, const SolveIO<T, D>&, int, int, RedBuf,    \
                                         CGScalars*, cudaStream_t);

PF_INST_P(double, 2)
PF_INST_P(double, 3)
PF_INST_P(float, 2)
PF_INST_P(float, 3)

}  // namespace pf
