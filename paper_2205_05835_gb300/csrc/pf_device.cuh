// Device helpers shared by the kernels: periodic indexing and deterministic
// block reductions finished by the last block of a fixed-size grid.
#pragma once

#include "pf_internal.h"

namespace pf {

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }
// mirror image of cell i across the walls at 0 and n (|i| < n): -1-i, 2n-1-i
__device__ __forceinline__ int mirrori(int i, int n) {
    return i < 0 ? -1 - i : (i >= n ? 2 * n - 1 - i : i);
}

// Free-slip walls at y = 0 and y = ny h (Dims::wall_y): face q (0..5 = -x, +x,
// -y, +y, -z, +z) of a cell in row j lies on a wall. The y-face of index 0 is
// both walls (face ny wraps to it); the normal velocity there is zero, and so
// are the flux of phi, the pressure operator's face coefficient (a homogeneous
// Neumann condition) and the face gradient of phi.
__device__ __forceinline__ bool wall_face(const Dims& g, int j, int q) {
    return g.wall_y && ((q == 2 && j == 0) || (q == 3 && j == g.ny - 1));
}

// Cell coordinates of a linear index (x fastest).
struct Cell {
    int i, j, k;
};

__device__ __forceinline__ Cell decode(int idx, const Dims& g) {
    Cell c;
    c.i = idx % g.nx;
    int t = idx / g.nx;
    c.j = t % g.ny;
    c.k = t / g.ny;
    return c;
}

// Wrapped neighbour index for offsets |o| <= 3 along each axis (n >= 4). Cells
// at least 3 away from every periodic seam use plain offsets. With walls in y
// (Dims::wall_y) a cell-centred quantity mirrors across them (its image cell:
// zero normal gradient, free slip of the tangential velocity), while the
// y-velocity, which lives on the y-faces, is read through atv: the wrapped
// face index, so face ny is the wall face 0 (zero normal velocity).
template <int DIM>
struct Nbr {
    int nx, ny, nz;
    int idx, sz, cj;
    bool inner;
    int im[7], jm[7], km[7];   // wrapped (mirrored) coordinates for offsets -3..3
    __device__ __forceinline__ Nbr(const Cell& c, const Dims& g) : nx(g.nx), ny(g.ny), nz(g.nz) {
        sz = g.nx * g.ny;
        cj = c.j;
        idx = (c.k * g.ny + c.j) * g.nx + c.i;
        inner = c.i >= 3 && c.i < g.nx - 3 && c.j >= 3 && c.j < g.ny - 3 &&
                (DIM == 2 || (c.k >= 3 && c.k < g.nz - 3));
        if (!inner) {
#pragma unroll
            for (int o = -3; o <= 3; ++o) {
                im[o + 3] = wrapi(c.i + o, g.nx);
                jm[o + 3] = g.wall_y ? mirrori(c.j + o, g.ny) : wrapi(c.j + o, g.ny);
                km[o + 3] = (DIM == 3) ? wrapi(c.k + o, g.nz) : 0;
            }
        }
    }
    __device__ __forceinline__ int at(int di, int dj, int dk) const {
        if (inner) return idx + di + dj * nx + (DIM == 3 ? dk * sz : 0);
        return (km[dk + 3] * ny + jm[dj + 3]) * nx + im[di + 3];
    }
    // neighbour of a y-face quantity (periodic wrap in y also with walls)
    __device__ __forceinline__ int atv(int di, int dj, int dk) const {
        if (inner) return at(di, dj, dk);
        return (km[dk + 3] * ny + wrapi(cj + dj, ny)) * nx + im[di + 3];
    }
    // neighbour for a load of velocity component comp
    __device__ __forceinline__ int atc(int comp, int di, int dj, int dk) const {
        return comp == 1 ? atv(di, dj, dk) : at(di, dj, dk);
    }
    __device__ __forceinline__ int axc(int comp, int d, int o) const {
        return d == 0 ? atc(comp, o, 0, 0) : (d == 1 ? atc(comp, 0, o, 0) : atc(comp, 0, 0, o));
    }
    __device__ __forceinline__ int ax2c(int comp, int d1, int o1, int d2, int o2) const {
        int di = (d1 == 0 ? o1 : 0) + (d2 == 0 ? o2 : 0);
        int dj = (d1 == 1 ? o1 : 0) + (d2 == 1 ? o2 : 0);
        int dk = (d1 == 2 ? o1 : 0) + (d2 == 2 ? o2 : 0);
        return atc(comp, di, dj, dk);
    }
    // offset o along axis d
    __device__ __forceinline__ int ax(int d, int o) const {
        return d == 0 ? at(o, 0, 0) : (d == 1 ? at(0, o, 0) : at(0, 0, o));
    }
    // offsets o1 along d1 and o2 along d2 (d1 != d2)
    __device__ __forceinline__ int ax2(int d1, int o1, int d2, int o2) const {
        int di = (d1 == 0 ? o1 : 0) + (d2 == 0 ? o2 : 0);
        int dj = (d1 == 1 ? o1 : 0) + (d2 == 1 ? o2 : 0);
        int dk = (d1 == 2 ? o1 : 0) + (d2 == 2 ? o2 : 0);
        return at(di, dj, dk);
    }
};

template <typename T>
__device__ __forceinline__ T ldg(const T* p, int i) { return __ldg(p + i); }

// Density (linear in clip(phi, 0, 1), phi = 1 the drop).
template <typename T>
__device__ __forceinline__ T rho_of_p(T phi, const PC<T>& c) {
    const T s = phi < T(0) ? T(0) : (phi > T(1) ? T(1) : phi);
    return c.rho_out + c.drho * s;
}

// 1 / rho_f of the face between two cells in float32: a correctly rounded
// reciprocal, used identically by the pressure operator, the smoother and the
// velocity correction of the mixed-precision path.
// Written with explicitly rounded operations (no contraction into FMA) so the
// operator is reproducible bit for bit by any IEEE float32 evaluation.
__device__ __forceinline__ float rho32(float phi, const Phys& ph) {
    const float c = phi < 0.f ? 0.f : (phi > 1.f ? 1.f : phi);
    return __fadd_rn(ph.rho_out_f, __fmul_rn(ph.drho_f, c));
}
__device__ __forceinline__ float beta_face32(float pa, float pb, const Phys& ph) {
    return __frcp_rn(__fmul_rn(0.5f, __fadd_rn(rho32(pa, ph), rho32(pb, ph))));
}

// Double-float arithmetic (a value is an unevaluated sum hi + lo of two floats):
// Knuth's TwoSum and the FMA form of Dekker's TwoProduct, both error free.
struct f2 {
    float hi, lo;
};
__device__ __forceinline__ f2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return f2{s, e};
}
__device__ __forceinline__ f2 two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return f2{p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ f2 quick_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return f2{s, __fsub_rn(b, __fsub_rn(s, a))};
}
// (a.hi + a.lo) * (b.hi + b.lo), relative error about 2^-44
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    f2 p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return quick_two_sum(p.hi, p.lo);
}

// a + b for double-floats (relative error about 2^-47)
__device__ __forceinline__ f2 df_add(f2 a, f2 b) {
    f2 s = two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return two_sum(s.hi, s.lo);
}
__device__ __forceinline__ f2 df_neg(f2 a) { return f2{-a.hi, -a.lo}; }
// a float64 value as a double-float (float64 operations: per-thread constants only)
__device__ __forceinline__ f2 df_of(double v) {
    const float h = __double2float_rn(v);
    return f2{h, __double2float_rn(v - double(h))};
}

// Double-well term c psi'(phi) = c phi (1 - phi) (1 - 2 phi) for a float32 phi:
// 1 - phi and 1 - 2 phi are formed exactly as double-floats and multiplied with
// error-free products, so the float32 result is the float64 evaluation rounded
// to float32 (up to a rounding tie), without the float64 pipe. c is given as a
// double-float (ch + cl).
__device__ __forceinline__ float dwell32(float phi, float ch, float cl) {
    const f2 a{phi, 0.f};
    const f2 b = two_sum(1.f, -phi);
    const f2 c = two_sum(1.f, -2.f * phi);   // 2 phi is exact
    const f2 p = f2_mul(f2_mul(a, b), c);
    const f2 q = f2_mul(p, f2{ch, cl});
    return __fadd_rn(q.hi, q.lo);
}

// ACDI phase field (the accurate conservative diffuse-interface model of Jain,
// J. Comput. Phys. 469, 2022): psi = eps ln((phi + e0) / (1 - phi + e0)) of
// clip(phi, 0, 1) with e0 = 1e-20 (finite where phi is 0 or 1), and the
// sharpening coefficient (1/4) [1 - tanh^2(psi_f / (2 eps))] of a face value
// psi_f. Float64: the library's log and tanh. Float32 (mixed path): the fast
// logarithm of the ratio, and the coefficient in the equivalent form
// e / (1 + e)^2 with e = exp(-|psi_f| / eps) (1 - tanh^2(y) = 4 e^{-2|y|} /
// (1 + e^{-2|y|})^2), through the fast exponential: a few ulp of float32.
constexpr double kAcdiE0 = 1e-20;
__device__ __forceinline__ double acdi_psi(double p, double eps) {
    p = p < 0.0 ? 0.0 : (p > 1.0 ? 1.0 : p);
    return eps * log((p + kAcdiE0) / (1.0 - p + kAcdiE0));
}
__device__ __forceinline__ float acdi_psi(float p, float eps) {
    p = p < 0.f ? 0.f : (p > 1.f ? 1.f : p);
    return eps * __logf(__fdividef(p + float(kAcdiE0), 1.f - p + float(kAcdiE0)));
}
__device__ __forceinline__ double acdi_sharp(double psif, double eps) {
    const double t = tanh(psif / (2.0 * eps));
    return 0.25 * (1.0 - t * t);
}
__device__ __forceinline__ float acdi_sharp(float psif, float eps) {
    const float e = __expf(-fabsf(psif) * __frcp_rn(eps));
    const float q = 1.f + e;
    return __fdividef(e, q * q);
}

// a / b: IEEE division in float64, multiplication by the correctly rounded
// reciprocal in float32.
__device__ __forceinline__ double divq(double a, double b) { return a / b; }
__device__ __forceinline__ float divq(float a, float b) { return a * __frcp_rn(b); }

// Row-wise cell loop: a block covers whole rows of nx cells (x fastest), so
// (i, j, k) need no per-cell division; rows are strided by the grid. Threads
// beyond the last full row of the block do nothing (but still reach any
// reduction that follows).
template <typename F>
__device__ __forceinline__ void for_cells(const Dims& g, F f) {
    const int nxe = g.nx < (int)blockDim.x ? g.nx : (int)blockDim.x;
    const int rpb = blockDim.x / nxe;
    const int rsub = threadIdx.x / nxe;
    if (rsub >= rpb) return;
    const int i0 = threadIdx.x - rsub * nxe;
    const int nrows = g.ny * g.nz;
    for (int row = blockIdx.x * rpb + rsub; row < nrows; row += gridDim.x * rpb) {
        const int k = row / g.ny, j = row - k * g.ny;
        const int base = row * g.nx;
        for (int i = i0; i < g.nx; i += nxe) f(i, j, k, base + i);
    }
}

// Same, over the cells of one colour ((i + j + k) % 2 == color).
template <typename F>
__device__ __forceinline__ void for_color_cells(const Dims& g, int color, F f) {
    const int nh = (g.nx + 1) >> 1;
    const int nxe = nh < (int)blockDim.x ? nh : (int)blockDim.x;
    const int rpb = blockDim.x / nxe;
    const int rsub = threadIdx.x / nxe;
    if (rsub >= rpb) return;
    const int m0 = threadIdx.x - rsub * nxe;
    const int nrows = g.ny * g.nz;
    for (int row = blockIdx.x * rpb + rsub; row < nrows; row += gridDim.x * rpb) {
        const int k = row / g.ny, j = row - k * g.ny;
        const int base = row * g.nx;
        const int s = (j + k + color) & 1;
        for (int i = 2 * m0 + s; i < g.nx; i += 2 * nxe) f(i, j, k, base + i);
    }
}

// Periodic neighbour indices (-x, +x, -y, +y, -z, +z) of cell (i, j, k).
struct Nb6 {
    int m[6];
};
template <int DIM>
__device__ __forceinline__ Nb6 nb6(const Dims& g, int i, int j, int k, int idx) {
    Nb6 n;
    const int sxy = g.nx * g.ny;
    n.m[0] = i == 0 ? idx + g.nx - 1 : idx - 1;
    n.m[1] = i == g.nx - 1 ? idx - (g.nx - 1) : idx + 1;
    n.m[2] = j == 0 ? idx + (g.ny - 1) * g.nx : idx - g.nx;
    n.m[3] = j == g.ny - 1 ? idx - (g.ny - 1) * g.nx : idx + g.nx;
    if (DIM == 3) {
        n.m[4] = k == 0 ? idx + (g.nz - 1) * sxy : idx - sxy;
        n.m[5] = k == g.nz - 1 ? idx - (g.nz - 1) * sxy : idx + sxy;
    } else {
        n.m[4] = n.m[5] = idx;
    }
    return n;
}

// Grid size of a row-wise kernel (cap: fixed grid of reduction kernels).
inline int row_grid(const Dims& g, int threads, int cap) {
    int nxe = g.nx < threads ? g.nx : threads;
    int rpb = threads / nxe;
    long long rows = (long long)g.ny * g.nz;
    long long b = (rows + rpb - 1) / rpb;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

// Sum of K values over the block (deterministic order). Result valid in thread 0.
template <int K>
__device__ __forceinline__ void block_reduce_sum(double (&v)[K], double* smem /* K*32 */) {
#pragma unroll
    for (int q = 0; q < K; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < K; ++q) smem[q * 32 + warp] = v[q];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            double t = lane < nw ? smem[q * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            v[q] = t;
        }
    }
    __syncthreads();
}

template <int K>
__device__ __forceinline__ void block_reduce_max(double (&v)[K], double* smem) {
#pragma unroll
    for (int q = 0; q < K; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] = fmax(v[q], __shfl_down_sync(0xffffffffu, v[q], o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < K; ++q) smem[q * 32 + warp] = v[q];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            double t = lane < nw ? smem[q * 32 + lane] : -1.0e308;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_down_sync(0xffffffffu, t, o));
            v[q] = t;
        }
    }
    __syncthreads();
}

// Stores the block's K partials; returns true in every thread of the last
// block to finish, after which `tot` holds the grid totals (fixed order).
// Mode per value: 0 sum, 1 max. bid / nblocks: linear block index and count.
template <int K>
__device__ __forceinline__ bool grid_reduce_lin(double (&v)[K], const int (&mode)[K], RedBuf rb,
                                                double (&tot)[K], int bid, int nblocks) {
    __shared__ double smem[K * 32];
    __shared__ bool last;
    double s[K], m[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        s[q] = mode[q] == 0 ? v[q] : 0.0;
        m[q] = mode[q] == 1 ? v[q] : -1.0e308;
    }
    block_reduce_sum<K>(s, smem);
    block_reduce_max<K>(m, smem);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) rb.part[bid * K + q] = mode[q] == 0 ? s[q] : m[q];
        __threadfence();
        unsigned t = atomicAdd(rb.counter, 1u);
        last = (t == (unsigned)nblocks - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int q = 0; q < K; ++q) {
        s[q] = 0.0;
        m[q] = -1.0e308;
    }
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            double t = __ldcg(rb.part + b * K + q);
            if (mode[q] == 0) s[q] += t; else m[q] = fmax(m[q], t);
        }
    }
    block_reduce_sum<K>(s, smem);
    block_reduce_max<K>(m, smem);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) tot[q] = mode[q] == 0 ? s[q] : m[q];
        *rb.counter = 0u;
    }
    return true;
}

template <int K>
__device__ __forceinline__ bool grid_reduce(double (&v)[K], const int (&mode)[K], RedBuf rb,
                                            double (&tot)[K]) {
    return grid_reduce_lin<K>(v, mode, rb, tot, blockIdx.x, gridDim.x);
}

// Scalars of the solve after an outer residual (totals: ||f||^2 when first,
// ||f - A x||^2 twice): convergence, non-finite values, iteration cap, and
// the inner tolerance of the next inner solve. Called by the last block.
__device__ __forceinline__ void ir_finish(const double (&tot)[3], int first, CGScalars* sc) {
    if (first) {
        sc->ff = tot[0];
        sc->iters = 0;
        sc->outer = 0;
        sc->capped = 0;
        sc->done = 0;
    }
    const double ffv = sc->ff;
    sc->rr = tot[1];
    sc->rr0_in = tot[2];
    sc->outer += 1;
    sc->idone = 0;
    sc->it_in = 0;
    if (!(tot[1] == tot[1])) {
        sc->done = 1;
        sc->status = 4;  // PF_ERR_NONFINITE
    } else if (tot[1] <= sc->rtol2 * ffv) {
        sc->done = 1;
    } else if (sc->capped) {
        sc->done = 1;
        if (sc->status == 0) sc->status = 3;  // PF_ERR_NOT_CONVERGED
    } else {
        double e2 = sc->rtol2 * ffv / tot[1];
        sc->eta2 = e2 > sc->eta2_min ? e2 : sc->eta2_min;
    }
}

// First inner CG iteration: given by the launch (f >= 0, host-driven loops) or
// read from the device counter (f < 0, loops inside a CUDA graph). Every
// kernel of an iteration reads the counter before that iteration's update
// kernel advances it.
__device__ __forceinline__ int first_of(int f, const CGScalars* sc) {
    return f >= 0 ? f : (sc->it_in == 0 ? 1 : 0);
}

// One face term of a compensated double-float operator sum: adds
// beta (x_c - x_q) with x_c = (ch, cl), x_q = (qh, ql) to the running sum S
// and its error accumulator c (TwoSum of the hi parts, TwoProduct with beta,
// TwoSum into S; every rounding error carried in c).
__device__ __forceinline__ void df_face_term(float beta, float ch, float cl, float qh, float ql,
                                             float& S, float& c) {
    const f2 d = two_sum(ch, -qh);
    const float t = __fadd_rn(d.lo, __fsub_rn(cl, ql));
    const f2 pr = two_prod(beta, d.hi);
    const f2 sm = two_sum(S, pr.hi);
    S = sm.hi;
    c = __fadd_rn(c, __fadd_rn(sm.lo, __fmaf_rn(beta, t, pr.lo)));
}

inline int red_grid(int n) {
    int b = (n + kThreads - 1) / kThreads;
    return b < kRedBlocks ? (b < 1 ? 1 : b) : kRedBlocks;
}

inline int lin_grid(int n) {
    int b = (n + kThreads - 1) / kThreads;
    return b < 1 ? 1 : b;
}

}  // namespace pf
