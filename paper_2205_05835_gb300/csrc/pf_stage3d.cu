// Column-marching versions of the per-stage cell kernels for 3D float32
// grids: one thread per (i, j) column of a 32 x 8 tile marching along z, the
// column's values of the planes k - 1, k, k + 1 carried in registers and the
// in-plane neighbours read through L1 (their lines are the neighbouring
// threads' own loads). The arithmetic is that of the generic kernels in
// pf_stage.cu, cell by cell.
//   * cell pass for the energy-based force with the CDI model: normals
//     n = grad_c phi / (|grad_c phi| + delta_n) and the chemical potential
//     mu = (6 sigma / eps) psi'(phi) - 6 sigma eps lap(phi) (Eq. ac_mu); with
//     the ACDI model the normals are those of psi (acdi_psi), also written;
//   * divergence b = D u* / tau of the face velocities and its mean;
//   * correction u = u* - tau beta G p with the float32 face coefficients.
#include "pf_device.cuh"

namespace pf {
namespace {

constexpr int ZX = 32, ZY = 8, ZT = ZX * ZY;

struct Col {
    int col, ox_m, ox_p, oy_m, oy_p;
    bool own;
};

__device__ __forceinline__ Col column(const Dims& g) {
    Col c;
    const int i = blockIdx.x * ZX + threadIdx.x % ZX;
    const int j = blockIdx.y * ZY + threadIdx.x / ZX;
    c.own = i < g.nx && j < g.ny;
    const int ii = c.own ? i : 0, jj = c.own ? j : 0;
    const int im = ii == 0 ? g.nx - 1 : ii - 1, ip = ii == g.nx - 1 ? 0 : ii + 1;
    const int jm = jj == 0 ? g.ny - 1 : jj - 1, jp = jj == g.ny - 1 ? 0 : jj + 1;
    c.col = jj * g.nx + ii;
    c.ox_m = im - ii;
    c.ox_p = ip - ii;
    c.oy_m = (jm - jj) * g.nx;
    c.oy_p = (jp - jj) * g.nx;
    return c;
}

struct CellPassArgs {
    Dims g;
    const float* phi;
    float* n0;
    float* n1;
    float* n2;
    float* mu;
    float* psi;        // ACDI: psi of phi (written), normals of psi; nullptr: normals of phi
    float dn, c_dw_hi, c_dw_lo, c_lap, eps;
    int zc;
};

__global__ void __launch_bounds__(ZT) k_cell_pass_mu3d(CellPassArgs A) {
    const Dims& g = A.g;
    const Col c = column(g);
    if (!c.own) return;
    const int sz = g.nx * g.ny;
    const int z0 = blockIdx.z * A.zc, z1 = min(z0 + A.zc, g.nz);
    const float inv2h = g.i2hf, inv_h2 = g.ih2f;
    const float* __restrict__ phi = A.phi;
    float* __restrict__ n0 = A.n0;
    float* __restrict__ n1 = A.n1;
    float* __restrict__ n2 = A.n2;
    float* __restrict__ mu = A.mu;
    float* __restrict__ psi = A.psi;
    const float eps = A.eps;
    float pm = __ldg(phi + (z0 == 0 ? g.nz - 1 : z0 - 1) * sz + c.col);
    float pc = __ldg(phi + z0 * sz + c.col);
    // ACDI: psi of the column's planes k - 1, k
    float sm = psi ? acdi_psi(pm, eps) : 0.f, sc_ = psi ? acdi_psi(pc, eps) : 0.f;
#pragma unroll 2
    for (int k = z0; k < z1; ++k) {
        const int idx = k * sz + c.col;
        const float pp = __ldg(phi + (k + 1 == g.nz ? 0 : k + 1) * sz + c.col);
        const float xm = __ldg(phi + idx + c.ox_m), xp = __ldg(phi + idx + c.ox_p);
        const float ym = __ldg(phi + idx + c.oy_m), yp = __ldg(phi + idx + c.oy_p);
        // normal (central gradient of phi, or of psi for ACDI)
        float g0, g1, g2, sp = 0.f;
        if (psi) {
            sp = acdi_psi(pp, eps);
            g0 = (acdi_psi(xp, eps) - acdi_psi(xm, eps)) * inv2h;
            g1 = (acdi_psi(yp, eps) - acdi_psi(ym, eps)) * inv2h;
            g2 = (sp - sm) * inv2h;
            psi[idx] = sc_;
        } else {
            g0 = (xp - xm) * inv2h;
            g1 = (yp - ym) * inv2h;
            g2 = (pp - pm) * inv2h;
        }
        float s = g0 * g0 + g1 * g1;
        s += g2 * g2;
        const float den = sqrtf(s) + A.dn;
        n0[idx] = divq(g0, den);
        n1[idx] = divq(g1, den);
        n2[idx] = divq(g2, den);
        // mu: double-well term in double-float, Laplacian in float32
        float lap = 0.f;
        lap = lap + (xp - 2.f * pc + xm) * inv_h2;
        lap = lap + (yp - 2.f * pc + ym) * inv_h2;
        lap = lap + (pp - 2.f * pc + pm) * inv_h2;
        mu[idx] = dwell32(pc, A.c_dw_hi, A.c_dw_lo) - A.c_lap * lap;
        pm = pc;
        pc = pp;
        sm = sc_;
        sc_ = sp;
    }
}

struct DivArgs {
    Dims g;
    const float* u0;
    const float* u1;
    const float* u2;
    double scale;   // 1 / (h tau)
    double* b;
    RedBuf rb;
    CGScalars* sc;
    int zc;
};

__global__ void __launch_bounds__(ZT) k_divergence3d(DivArgs A) {
    const Dims& g = A.g;
    const Col c = column(g);
    const int sz = g.nx * g.ny;
    const int z0 = blockIdx.z * A.zc, z1 = min(z0 + A.zc, g.nz);
    f2 acc{0.f, 0.f};
    if (c.own) {
        const float* __restrict__ u0 = A.u0;
        const float* __restrict__ u1 = A.u1;
        const float* __restrict__ u2 = A.u2;
        float* __restrict__ bh = reinterpret_cast<float*>(A.b);
        float* __restrict__ bl = bh + g.ncell;
        const f2 scale = df_of(A.scale);
        float wc = __ldg(u2 + z0 * sz + c.col);
#pragma unroll 2
        for (int k = z0; k < z1; ++k) {
            const int idx = k * sz + c.col;
            const float wp = __ldg(u2 + (k + 1 == g.nz ? 0 : k + 1) * sz + c.col);
            // exact differences (TwoSum) summed as a double-float
            const f2 a = two_sum(__ldg(u0 + idx + c.ox_p), -__ldg(u0 + idx));
            const f2 b1 = two_sum(__ldg(u1 + idx + c.oy_p), -__ldg(u1 + idx));
            f2 t = two_sum(a.hi, b1.hi);
            t.lo = __fadd_rn(t.lo, __fadd_rn(a.lo, b1.lo));
            const f2 c1 = two_sum(wp, -wc);
            f2 t2 = two_sum(t.hi, c1.hi);
            t2.lo = __fadd_rn(t2.lo, __fadd_rn(t.lo, c1.lo));
            // b as a double-float (hi plane, lo plane), scaled by 1 / (h tau)
            const f2 dv = f2_mul(t2, scale);
            bh[idx] = dv.hi;
            bl[idx] = dv.lo;
            acc = df_add(acc, dv);
            wc = wp;
        }
    }
    double v[1] = {double(acc.hi) + double(acc.lo)}, tot[1];
    const int mode[1] = {0};
    const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    if (grid_reduce_lin<1>(v, mode, A.rb, tot, bid, nb) && threadIdx.x == 0)
        A.sc->mean_b = tot[0] / g.ncell;
}

struct CorrArgs {
    Dims g;
    const float* s0;
    const float* s1;
    const float* s2;
    const float* f0;
    const float* f1;
    const float* f2;
    const double* p;
    float tau_h;
    float* o0;
    float* o1;
    float* o2;
    int zc;
};

__global__ void __launch_bounds__(ZT) k_correct3d(CorrArgs A) {
    const Dims& g = A.g;
    const Col c = column(g);
    if (!c.own) return;
    const int sz = g.nx * g.ny;
    const int z0 = blockIdx.z * A.zc, z1 = min(z0 + A.zc, g.nz);
    // the pressure is a double-float: hi plane, then lo plane
    const float* __restrict__ ph = reinterpret_cast<const float*>(A.p);
    const float* __restrict__ pl = ph + g.ncell;
    const float tau_h = A.tau_h;
    const int i0 = (z0 == 0 ? g.nz - 1 : z0 - 1) * sz + c.col;
    float pmh = ph[i0], pml = pl[i0];
#pragma unroll 2
    for (int k = z0; k < z1; ++k) {
        const int idx = k * sz + c.col;
        const float pch = ph[idx], pcl = pl[idx];
        // the pressure difference from both parts, scaled and applied in float32
        const int ix = idx + c.ox_m, iy = idx + c.oy_m;
        const float gx = __fadd_rn(__fsub_rn(pch, ph[ix]), __fsub_rn(pcl, pl[ix])) * tau_h;
        const float gy = __fadd_rn(__fsub_rn(pch, ph[iy]), __fsub_rn(pcl, pl[iy])) * tau_h;
        const float gz = __fadd_rn(__fsub_rn(pch, pmh), __fsub_rn(pcl, pml)) * tau_h;
        A.o0[idx] = __ldg(A.s0 + idx) - __ldg(A.f0 + idx) * gx;
        A.o1[idx] = __ldg(A.s1 + idx) - __ldg(A.f1 + idx) * gy;
        A.o2[idx] = __ldg(A.s2 + idx) - __ldg(A.f2 + idx) * gz;
        pmh = pch;
        pml = pcl;
    }
}

// planes per CTA: enough CTAs for about 8 per SM
int zchunk(const Dims& g) {
    const long long cols = (long long)((g.nx + ZX - 1) / ZX) * ((g.ny + ZY - 1) / ZY);
    int zc = 64;
    while (zc > 1 && cols * ((g.nz + zc - 1) / zc) < 8 * 152) zc >>= 1;
    return zc;
}

dim3 zgrid(const Dims& g, int zc) {
    return dim3((g.nx + ZX - 1) / ZX, (g.ny + ZY - 1) / ZY, (g.nz + zc - 1) / zc);
}

}  // namespace

void launch_cell_pass_mu3d(const Dims& g, const Phys& ph, const float* phi, float* n0, float* n1,
                           float* n2, float* mu, float* psi, cudaStream_t s) {
    CellPassArgs a;
    a.g = g;
    a.phi = phi;
    a.n0 = n0;
    a.n1 = n1;
    a.n2 = n2;
    a.mu = mu;
    a.psi = psi;
    a.eps = ph.eps_f;
    const double sh = 6.0 * ph.sigma;
    const double c_dw = sh / ph.eps;
    a.dn = float(ph.delta_n);
    a.c_dw_hi = float(c_dw);
    a.c_dw_lo = float(c_dw - double(float(c_dw)));
    a.c_lap = float(sh * ph.eps);
    a.zc = zchunk(g);
    k_cell_pass_mu3d<<<zgrid(g, a.zc), ZT, 0, s>>>(a);
}

bool divergence3d_ok(const Dims& g) {
    const int zc = zchunk(g);
    const dim3 gr = zgrid(g, zc);
    return g.nz > 1 && (long long)gr.x * gr.y * gr.z <= kRedPart;
}

void launch_divergence3d(const Dims& g, const float* const* u, double inv_tau, double* b,
                         RedBuf rb, CGScalars* sc, cudaStream_t s) {
    DivArgs a;
    a.g = g;
    a.u0 = u[0];
    a.u1 = u[1];
    a.u2 = u[2];
    a.scale = g.ih * inv_tau;
    a.b = b;
    a.rb = rb;
    a.sc = sc;
    a.zc = zchunk(g);
    k_divergence3d<<<zgrid(g, a.zc), ZT, 0, s>>>(a);
}

void launch_correct3d(const Dims& g, const float* const* beta32, const float* const* ustar,
                      const double* p, double tau, float* const* uout, cudaStream_t s) {
    CorrArgs a;
    a.g = g;
    a.s0 = ustar[0];
    a.s1 = ustar[1];
    a.s2 = ustar[2];
    a.f0 = beta32[0];
    a.f1 = beta32[1];
    a.f2 = beta32[2];
    a.p = p;
    a.tau_h = float(tau * g.ih);
    a.o0 = uout[0];
    a.o1 = uout[1];
    a.o2 = uout[2];
    a.zc = zchunk(g);
    k_correct3d<<<zgrid(g, a.zc), ZT, 0, s>>>(a);
}

}  // namespace pf
