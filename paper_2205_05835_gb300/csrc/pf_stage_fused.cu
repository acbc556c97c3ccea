// The fused stage of the 3D float32 path for the CDI / ACDI phase field with
// the energy-based force and advective momentum transport: the cell pass
// (normals, chemical potential mu (Eq. ac_mu), the ACDI variable psi) and the
// stage (phase-field flux divergence, momentum right-hand side with the EB
// force (Eq. eb_st), RK update) in one kernel, with the derived fields living
// in shared memory only (no HBM round trip for n, mu, psi).
//
// A CTA owns a 32 x 8 column tile and marches along z. The planes of phi
// (halo 2) and of the three face velocities (halo 1) are copied into
// shared-memory rings by cp.async, one step ahead of their use. The step for
// plane k
//   (1) forms n (of phi, or of psi for ACDI), mu and psi of plane k + 1 on
//       the tile plus a one-cell ring (they need phi of planes k .. k + 2;
//       ACDI: psi of plane k + 2 is formed here on the tile plus a two-cell
//       ring, once per cell, into a ring of four psi planes that the
//       normals of the next steps and the face sharpening read);
//   (2) evaluates the phase-field and momentum right-hand sides of plane k
//       from the staged phi, u and the derived fields of planes k - 1 .. k + 1
//       and applies the RK stage update.
// The arithmetic is that of k_cell_pass_mu3d and k_stage3d (pf_stage.cu),
// term by term; only where the operands come from differs.
#include <cstddef>
#include <mutex>

#include "pf_device.cuh"

namespace pf {
namespace {

constexpr int TX = 32, TY = 8, NTH = TX * TY;
constexpr int OX = 4, OY = 2;                 // staged plane origin (i0 - 4, j0 - 2)
constexpr int HX = TX + 2 * OX;               // 40 columns
constexpr int HY = TY + 2 * OY;               // 12 rows
constexpr int PL = HX * HY;                   // 480 floats per plane
constexpr int CPR = HX / 4, NCH = CPR * HY;   // 16-byte chunks per row / plane
constexpr int RP = 5, RU = 4, RD = 3;         // ring planes: phi, each u, each derived field
constexpr int RQ = 4;                         // ring planes of the ACDI psi
constexpr int RXC = TX + 2;                   // derived-field row (tile + one-cell ring): 34
constexpr int NR = RXC * (TY + 2);            // derived-field cells: 340
constexpr int NR2 = (TX + 4) * (TY + 4);      // psi cells (tile + two-cell ring): 432

// the normals and mu are stored on the tile plus a one-cell ring only (34 x
// 10), which keeps the CTA within a quarter of the SM's shared memory (four
// resident CTAs); phi, u and psi keep the staged plane's layout
struct Smem {
    float phi[RP][PL];
    float u[3][RU][PL];
    float n[3][RD][NR];
    float mu[RD][NR];
    float psi[RQ][PL];
};

struct FusedArgs {
    Dims g;
    Phys ph;
    StageIO<float> io;
    int stage, scheme, write_rhs, zc, acdi;
    float wdt, cdt;
    float dn, c_dw_hi, c_dw_lo, c_lap;
};

__device__ __forceinline__ int modp(int a, int m) { int r = a % m; return r < 0 ? r + m : r; }
__device__ __forceinline__ void cp16(float* dst, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__global__ void __launch_bounds__(NTH, 4) k_stage3d_fused(FusedArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& S = *reinterpret_cast<Smem*>(smem_raw);
    const Dims& g = A.g;
    const StageIO<float>& io = A.io;
    const PC<float> pcs = pc_of(A.ph, float());
    const float gam = float(*io.gamma);
    const float inv_h = g.ihf, inv2h = g.i2hf, inv_h2 = g.ih2f;
    const float eps = pcs.eps;
    const bool acdi = A.acdi != 0;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * A.zc, z1 = min(z0 + A.zc, g.nz);
    const int sz = g.nx * g.ny;
    const bool own = i0 + tx < g.nx && j0 + ty < g.ny;
    const int gidx_col = (j0 + ty) * g.nx + i0 + tx;       // own column (when own)

    // this thread's 16-byte copy chunks of a staged plane (wrapped addresses:
    // nx and the tile origin are multiples of 4, so a chunk never straddles
    // the periodic seam), fixed across planes
    int c_off[2], c_so[2];
    bool c_has[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int c = tid + q * NTH;
        c_has[q] = c < NCH;
        const int r = c / CPR, a = 4 * (c - r * CPR);
        c_off[q] = modp(j0 - OY + r, g.ny) * g.nx + modp(i0 - OX + a, g.nx);
        c_so[q] = r * HX + a;
    }
    auto stage_plane = [&](const float* src, float* dst, int k) {
        const float* pl = src + (size_t)modp(k, g.nz) * sz;
#pragma unroll
        for (int q = 0; q < 2; ++q)
            if (c_has[q]) cp16(dst + c_so[q], pl + c_off[q]);
    };
    // ring slot offsets
    auto sp = [&](int k) { return modp(k - z0, RP); };
    auto su = [&](int k) { return modp(k - z0, RU); };
    auto sd = [&](int k) { return modp(k - z0, RD); };
    auto sq = [&](int k) { return modp(k - z0, RQ); };
    // ACDI: psi of plane k on the tile plus a two-cell ring, once per cell
    // (the normals of plane k - 1 read it at in-plane neighbours, those of
    // k - 2 and k at the own column)
    auto psi_plane = [&](int k) {
        const float* P = S.phi[sp(k)];
        float* Q = S.psi[sq(k)];
        for (int c = tid; c < NR2; c += NTH) {
            const int ry = c / (TX + 4), rx = c - ry * (TX + 4);
            const int o = (ry + OY - 2) * HX + rx + OX - 2;
            Q[o] = acdi_psi(P[o], eps);
        }
    };

    // prologue: phi of planes z0 - 2 .. z0, u of plane z0 - 1
    stage_plane(io.phi_s, S.phi[sp(z0 - 2)], z0 - 2);
    stage_plane(io.phi_s, S.phi[sp(z0 - 1)], z0 - 1);
    stage_plane(io.phi_s, S.phi[sp(z0)], z0);
#pragma unroll
    for (int d = 0; d < 3; ++d) stage_plane(io.u_s[d], S.u[d][su(z0 - 1)], z0 - 1);
    cp_commit();

    // the thread's own cell in a staged plane
    const int cs = (ty + OY) * HX + tx + OX;
    if (acdi) {
        // psi of planes z0 - 2 and z0 - 1 (the first step forms z0)
        cp_wait_all();
        __syncthreads();
        psi_plane(z0 - 2);
        psi_plane(z0 - 1);
    }

    for (int k = z0 - 2; k < z1; ++k) {
        cp_wait_all();
        __syncthreads();   // planes of this step landed; the previous step is done
        // next planes: phi k + 3, u k + 2 (one step ahead)
        if (k + 3 <= z1 + 1) stage_plane(io.phi_s, S.phi[sp(k + 3)], k + 3);
        if (k + 2 <= z1) {
#pragma unroll
            for (int d = 0; d < 3; ++d) stage_plane(io.u_s[d], S.u[d][su(k + 2)], k + 2);
        }
        cp_commit();

        // (1) derived fields of plane k + 1 on the tile plus a one-cell ring
        // (ACDI: with psi of plane k + 2 on the tile plus a two-cell ring; psi
        // of the planes k and k + 1 was formed by the two steps before)
        if (k + 1 <= z1) {
            const float* P0 = S.phi[sp(k)];
            const float* P1 = S.phi[sp(k + 1)];
            const float* P2 = S.phi[sp(k + 2)];
            float* N0 = S.n[0][sd(k + 1)];
            float* N1 = S.n[1][sd(k + 1)];
            float* N2 = S.n[2][sd(k + 1)];
            float* MU = S.mu[sd(k + 1)];
            const float* Q0 = S.psi[sq(k)];
            const float* Q1 = S.psi[sq(k + 1)];
            float* Q2 = S.psi[sq(k + 2)];
            for (int c = tid; c < (acdi ? NR2 : NR); c += NTH) {
                int o, oc;   // staged-plane and derived-field index of the cell
                if (acdi) {
                    const int ry = c / (TX + 4), rx = c - ry * (TX + 4);
                    o = (ry + OY - 2) * HX + rx + OX - 2;
                    Q2[o] = acdi_psi(P2[o], eps);
                    if (ry < 1 || ry > TY + 2 || rx < 1 || rx > TX + 2) continue;   // outer ring
                    oc = (ry - 1) * RXC + rx - 1;
                } else {
                    const int ry = c / RXC, rx = c - ry * RXC;
                    o = (ry + OY - 1) * HX + rx + OX - 1;
                    oc = c;
                }
                const float pc = P1[o];
                const float xm = P1[o - 1], xp = P1[o + 1], ym = P1[o - HX], yp = P1[o + HX];
                const float zm = P0[o], zp = P2[o];
                float g0, g1, g2;
                if (acdi) {
                    g0 = (Q1[o + 1] - Q1[o - 1]) * inv2h;
                    g1 = (Q1[o + HX] - Q1[o - HX]) * inv2h;
                    g2 = (Q2[o] - Q0[o]) * inv2h;
                } else {
                    g0 = (xp - xm) * inv2h;
                    g1 = (yp - ym) * inv2h;
                    g2 = (zp - zm) * inv2h;
                }
                float s = g0 * g0 + g1 * g1;
                s += g2 * g2;
                const float den = sqrtf(s) + A.dn;
                N0[oc] = divq(g0, den);
                N1[oc] = divq(g1, den);
                N2[oc] = divq(g2, den);
                float lap = 0.f;
                lap = lap + (xp - 2.f * pc + xm) * inv_h2;
                lap = lap + (yp - 2.f * pc + ym) * inv_h2;
                lap = lap + (zp - 2.f * pc + zm) * inv_h2;
                MU[oc] = dwell32(pc, A.c_dw_hi, A.c_dw_lo) - A.c_lap * lap;
            }
        }
        __syncthreads();   // derived fields of plane k + 1 visible
        if (k < z0 || !own) continue;

        // (2) right-hand sides of plane k at the thread's cell
        // plane pointers of planes k - 1, k, k + 1 (index 0, 1, 2)
        const float* Pp[3] = {S.phi[sp(k - 1)], S.phi[sp(k)], S.phi[sp(k + 1)]};
        const float* Up[3][3];
        const float* Np[3][3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
#pragma unroll
            for (int z = 0; z < 3; ++z) {
                Up[d][z] = S.u[d][su(k - 1 + z)];
                Np[d][z] = S.n[d][sd(k - 1 + z)];
            }
        }
        const float* Mp[3] = {S.mu[sd(k - 1)], S.mu[sd(k)], S.mu[sd(k + 1)]};
        const float* Qp[3] = {S.psi[sq(k - 1)], S.psi[sq(k)], S.psi[sq(k + 1)]};
        // value of a plane set at the offset (dx, dy, dz) from the own cell
        auto at = [&](const float* const* pl, int dx, int dy, int dz) {
            return pl[1 + dz][cs + dx + dy * HX];
        };
        // the same for the derived fields (n, mu) on the tile plus ring
        const int csd = (ty + 1) * RXC + tx + 1;
        auto atd = [&](const float* const* pl, int dx, int dy, int dz) {
            return pl[1 + dz][csd + dx + dy * RXC];
        };
        // offset vectors of +/- e_d
        auto ax = [](int d, int o, int (&v)[3]) { v[0] = v[1] = v[2] = 0; v[d] = o; };
        const float pc = Pp[1][cs];

        // ---------------- phase field (CDI / ACDI flux) ----------------
        float kphi = 0.f;
        {
            const float psc = acdi ? Qp[1][cs] : 0.f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                int m[3], p[3];
                ax(d, -1, m);
                ax(d, 1, p);
                const float pm = at(Pp, m[0], m[1], m[2]);
                const float pf = 0.5f * (pc + pm);
                const float nf = 0.5f * (Np[d][1][csd] + atd(Np[d], m[0], m[1], m[2]));
                const float shlo = acdi ? acdi_sharp(0.5f * (psc + at(Qp, m[0], m[1], m[2])), eps)
                                        : pf * (1.f - pf);
                const float Flo = Up[d][1][cs] * pf - gam * (eps * ((pc - pm) * inv_h) - shlo * nf);
                const float pp = at(Pp, p[0], p[1], p[2]);
                const float pf2 = 0.5f * (pp + pc);
                const float nf2 = 0.5f * (atd(Np[d], p[0], p[1], p[2]) + Np[d][1][csd]);
                const float shhi = acdi ? acdi_sharp(0.5f * (at(Qp, p[0], p[1], p[2]) + psc), eps)
                                        : pf2 * (1.f - pf2);
                const float Fhi = at(Up[d], p[0], p[1], p[2]) * pf2 -
                                  gam * (eps * ((pp - pc) * inv_h) - shhi * nf2);
                kphi = kphi - (Fhi - Flo) * inv_h;
            }
        }

        // ---------------- momentum at the low faces ----------------
        float ku[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            int m[3];
            ax(d, -1, m);
            const float pm = at(Pp, m[0], m[1], m[2]);
            const float udc = Up[d][1][cs];
            // advection -(u.grad) u_d, central, transverse components from 4 faces
            float adv = 0.f;
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                int pe[3], me[3];
                ax(e, 1, pe);
                ax(e, -1, me);
                float vel;
                if (e == d) {
                    vel = udc;
                } else {
                    vel = 0.25f * (Up[e][1][cs] + at(Up[e], pe[0], pe[1], pe[2]) +
                                   at(Up[e], m[0], m[1], m[2]) +
                                   at(Up[e], m[0] + pe[0], m[1] + pe[1], m[2] + pe[2]));
                }
                adv = adv + vel * ((at(Up[d], pe[0], pe[1], pe[2]) - at(Up[d], me[0], me[1], me[2])) *
                                   inv2h);
            }
            // viscous stress divergence
            float visc = 0.f;
            const float etac = pcs.mu_out + pcs.dmu * fminf(fmaxf(pc, 0.f), 1.f);
            const float etam = pcs.mu_out + pcs.dmu * fminf(fmaxf(pm, 0.f), 1.f);
            auto eta = [&](float p) { return pcs.mu_out + pcs.dmu * fminf(fmaxf(p, 0.f), 1.f); };
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                int pe[3], me[3];
                ax(e, 1, pe);
                ax(e, -1, me);
                if (e == d) {
                    const float thi = 2.f * etac * ((at(Up[d], pe[0], pe[1], pe[2]) - udc) * inv_h);
                    const float tlo = 2.f * etam * ((udc - at(Up[d], m[0], m[1], m[2])) * inv_h);
                    visc = visc + (thi - tlo) * inv_h;
                } else {
                    // edge at (c - e_d/2 - e_e/2): cells c, c-e_d, c-e_e, c-e_d-e_e
                    const float eta_lo =
                        0.25f * (etac + etam + eta(at(Pp, me[0], me[1], me[2])) +
                                 eta(at(Pp, m[0] + me[0], m[1] + me[1], m[2] + me[2])));
                    const float tlo = eta_lo * ((udc - at(Up[d], me[0], me[1], me[2])) * inv_h +
                                                (Up[e][1][cs] - at(Up[e], m[0], m[1], m[2])) * inv_h);
                    // edge at (c - e_d/2 + e_e/2): cells c+e_e, c+e_e-e_d, c, c-e_d
                    const float eta_hi =
                        0.25f * (eta(at(Pp, pe[0], pe[1], pe[2])) +
                                 eta(at(Pp, m[0] + pe[0], m[1] + pe[1], m[2] + pe[2])) + etac + etam);
                    const float thi =
                        eta_hi * ((at(Up[d], pe[0], pe[1], pe[2]) - udc) * inv_h +
                                  (at(Up[e], pe[0], pe[1], pe[2]) -
                                   at(Up[e], m[0] + pe[0], m[1] + pe[1], m[2] + pe[2])) *
                                      inv_h);
                    visc = visc + (thi - tlo) * inv_h;
                }
            }
            // energy-based surface tension force at the face (Eq. eb_st)
            const float dphi = (pc - pm) * inv_h;
            const float F = 0.5f * (Mp[1][csd] + atd(Mp, m[0], m[1], m[2])) * dphi;
            const float beta = divq(1.f, 0.5f * (rho_of_p(pc, pcs) + rho_of_p(pm, pcs)));
            ku[d] = -adv + beta * visc + beta * F;
        }

        const int idx = k * sz + gidx_col;
        if (A.write_rhs) {
            io.rhs_phi[idx] = kphi;
#pragma unroll
            for (int d = 0; d < 3; ++d) io.rhs_u[d][idx] = ku[d];
            continue;
        }
        // ---------------- RK stage update ----------------
        const float phin = __ldg(io.phi_n + idx);
        const float wdt = A.wdt, cdt = A.cdt;
        if (A.scheme == 1) {   // forward Euler
            io.phi_out[idx] = phin + cdt * kphi;
#pragma unroll
            for (int d = 0; d < 3; ++d) io.u_out[d][idx] = __ldg(io.u_n[d] + idx) + cdt * ku[d];
            continue;
        }
        if (A.stage < 3) {
            const float a = A.stage == 0 ? wdt * kphi : io.acc_phi[idx] + wdt * kphi;
            io.acc_phi[idx] = a;
            io.phi_out[idx] = phin + cdt * kphi;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float au = A.stage == 0 ? wdt * ku[d] : io.acc_u[d][idx] + wdt * ku[d];
                io.acc_u[d][idx] = au;
                io.u_out[d][idx] = __ldg(io.u_n[d] + idx) + cdt * ku[d];
            }
        } else {
            io.phi_out[idx] = phin + (io.acc_phi[idx] + wdt * kphi);
#pragma unroll
            for (int d = 0; d < 3; ++d)
                io.u_out[d][idx] = __ldg(io.u_n[d] + idx) + (io.acc_u[d][idx] + wdt * ku[d]);
        }
    }
    cp_wait_all();
}

void fused_attributes() {
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_stage3d_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(Smem));
        cudaFuncSetAttribute(k_stage3d_fused, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    });
}

}  // namespace

// Eligible: 3D float32, advective momentum, CDI or ACDI with the EB force,
// rows of whole 16-byte chunks (nx % 4 == 0), halos that wrap at most once.
bool stage_fused_ok(const Dims& g, const Phys& ph) {
    return g.nz >= 4 && g.nx % 4 == 0 && g.nx >= HX && g.ny >= HY && ph.momentum == 0 &&
           ph.force == 0 && (ph.model == 0 || ph.model == 3) && g.wall_y == 0;
}

void stage_fused_prepare() { fused_attributes(); }

void launch_stage_fused(const Dims& g, const Phys& ph, const StageIO<float>& io, int stage,
                        int scheme, double wdt, double cdt, int write_rhs, cudaStream_t s) {
    FusedArgs a;
    a.g = g;
    a.ph = ph;
    a.io = io;
    a.stage = stage;
    a.scheme = scheme;
    a.write_rhs = write_rhs;
    a.acdi = ph.model == 3 ? 1 : 0;
    a.wdt = float(wdt);
    a.cdt = float(cdt);
    const double sh = 6.0 * ph.sigma;
    const double c_dw = sh / ph.eps;
    a.dn = float(ph.delta_n);
    a.c_dw_hi = float(c_dw);
    a.c_dw_lo = float(c_dw - double(float(c_dw)));
    a.c_lap = float(sh * ph.eps);
    const long long cols = (long long)((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    int zc = 64;
    while (zc > 4 && cols * ((g.nz + zc - 1) / zc) < 4 * 152) zc >>= 1;
    a.zc = zc;
    fused_attributes();
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + zc - 1) / zc);
    k_stage3d_fused<<<grid, NTH, sizeof(Smem), s>>>(a);
}

}  // namespace pf
