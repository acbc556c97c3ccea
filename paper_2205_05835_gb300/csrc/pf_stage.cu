// Stage kernels of the fractional step: initial profile, the cell pass
// (normals, curvature, chemical potential), the fused phase-field +
// momentum right-hand side with the RK stage update, Gamma, divergence,
// velocity correction and diagnostics.
//
// Discretization (uniform periodic staggered grid, face i-1/2 stored at i):
//   phase field   d phi/dt + div(u phi) = g(phi), g from Table 1 (CDI, SB, ISODI)
//   chemical pot. mu = (6 sigma/eps) psi'(phi) - 6 sigma eps lap(phi)      (Eq. ac_mu)
//   EB force      F = mu_f (phi_i - phi_{i-1}) / h                         (Eq. eb_st)
//   CSF / LCSF    F = sigma kappa_f dphi, 6 sigma kappa_f phi_f(1-phi_f) dphi (Section 2)
//   momentum      du/dt = -(u.grad)u + div(eta (grad u + grad u^T))/rho_f + F/rho_f
#include "pf_device.cuh"

namespace pf {

template <typename T>
__device__ __forceinline__ T clamp01(T v) { return v < T(0) ? T(0) : (v > T(1) ? T(1) : v); }

template <typename T>
__device__ __forceinline__ T rho_of(T phi, const PC<T>& c) {
    return rho_of_p(phi, c);
}

template <typename T>
__device__ __forceinline__ T eta_of(T phi, const PC<T>& c) {
    return c.mu_out + c.dmu * clamp01(phi);
}

// velocity from the momentum rho_f u on the face between cells a and b
// (consistent transport): rho_f from clip(phi) as everywhere, IEEE division
// in float64, the correctly rounded reciprocal in float32
template <typename T>
__device__ __forceinline__ T mom_to_vel(T mom, T pa, T pb, const Phys& ph) {
    const PC<T> c = pc_of(ph, T());
    return divq(mom, T(0.5) * (rho_of(pa, c) + rho_of(pb, c)));
}

// psi'(phi) = phi (1 - phi) (1 - 2 phi), always evaluated in float64.
__device__ __forceinline__ double dpsi64(double p) { return p * (1.0 - p) * (1.0 - 2.0 * p); }

// ---------------------------------------------------------------------------
// initial profile phi0 = [1 + tanh(s / (2 eps))] / 2, s the signed distance:
// drop, s = R(theta) - r; wave (2D), s = y_i(x) - y with the interface height
// y_i = R (1 - a cos(k (x - h/2))), k = 2 pi mode / (nx h), phi = 1 below it
// ---------------------------------------------------------------------------
template <typename T, int DIM>
__global__ void k_init_phi(Dims g, Phys ph, double R, int mode, double amp, int shape,
                           T* __restrict__ phi) {
    for_cells(g, [&](int ci, int cj, int ck, int idx) {
    Cell c{ci, cj, ck};
    if (shape == 1) {
        const double kx = 2.0 * 3.14159265358979323846 * mode / (g.nx * g.h);
        const double yi = R * (1.0 - amp * cos(kx * (c.i * g.h)));
        phi[idx] = T(0.5 * (1.0 + tanh((yi - (c.j + 0.5) * g.h) / (2.0 * ph.eps))));
        return;
    }
    double cx = 0.5 * g.nx * g.h, cy = 0.5 * g.ny * g.h, cz = 0.5 * g.nz * g.h;
    double x = (c.i + 0.5) * g.h - cx, y = (c.j + 0.5) * g.h - cy;
    double z = DIM == 3 ? (c.k + 0.5) * g.h - cz : 0.0;
    double r = sqrt(x * x + y * y + z * z);
    double Rt = R;
    if (mode > 0 && amp != 0.0) {
        if (DIM == 2) {
            Rt = R * (1.0 + amp * cos(mode * atan2(y, x)));
        } else {
            double ct = r > 0.0 ? z / r : 1.0;
            // Legendre P_mode(ct) by the three-term (Bonnet) recurrence
            double p0 = 1.0, p1 = ct;
            for (int l = 1; l < mode; ++l) {
                double p2 = ((2 * l + 1) * ct * p1 - l * p0) / (l + 1);
                p0 = p1;
                p1 = p2;
            }
            Rt = R * (1.0 + amp * (mode == 0 ? 1.0 : p1));
        }
    }
    phi[idx] = T(0.5 * (1.0 + tanh((Rt - r) / (2.0 * ph.eps))));
    });
}

template <typename T, int DIM>
void launch_init_phi(const Dims& g, const Phys& ph, double R, int mode, double amp, int shape,
                     T* phi, cudaStream_t s) {
    k_init_phi<T, DIM><<<row_grid(g, kThreads, 1 << 30), kThreads, 0, s>>>(g, ph, R, mode, amp,
                                                                            shape, phi);
}

template <typename T>
__global__ void k_convert_in(const double* __restrict__ src, T* __restrict__ dst, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = T(src[i]);
}

template <typename T>
__global__ void k_convert_out(const T* __restrict__ src, double* __restrict__ dst, int n,
                              const double* sum_ptr, double inv_n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double m = sum_ptr ? (*sum_ptr) * inv_n : 0.0;
    if (i < n) dst[i] = double(src[i]) - m;
}

template <typename T>
void launch_convert_in(const double* src, T* dst, int n, cudaStream_t s) {
    k_convert_in<T><<<lin_grid(n), kThreads, 0, s>>>(src, dst, n);
}

template <typename T>
void launch_convert_out(const T* src, double* dst, int n, double, const double* sum_ptr,
                        double inv_n, cudaStream_t s) {
    k_convert_out<T><<<lin_grid(n), kThreads, 0, s>>>(src, dst, n, sum_ptr, inv_n);
}

// ---------------------------------------------------------------------------
// cell pass: normals n = grad_c phi / (|grad_c phi| + delta_n), and mu (EB
// force) and/or kappa = -div_c n (CSF, LCSF, SB, ISODI)
// ---------------------------------------------------------------------------
template <typename T, int DIM>
__device__ __forceinline__ void normal_at(const T* __restrict__ phi, const Nbr<DIM>& nb, int oi,
                                          int oj, int ok, T inv2h, T dn, T (&n)[3], T& mag) {
    T gr[3];
    gr[0] = (ldg(phi, nb.at(oi + 1, oj, ok)) - ldg(phi, nb.at(oi - 1, oj, ok))) * inv2h;
    gr[1] = (ldg(phi, nb.at(oi, oj + 1, ok)) - ldg(phi, nb.at(oi, oj - 1, ok))) * inv2h;
    gr[2] = DIM == 3 ? (ldg(phi, nb.at(oi, oj, ok + 1)) - ldg(phi, nb.at(oi, oj, ok - 1))) * inv2h
                     : T(0);
    T s = gr[0] * gr[0] + gr[1] * gr[1];
    if (DIM == 3) s += gr[2] * gr[2];
    mag = sqrt(s);
    T den = mag + dn;
#pragma unroll
    for (int d = 0; d < DIM; ++d) n[d] = divq(gr[d], den);
}

// ACDI: the normal of psi (central gradient of psi of the neighbours' phi)
template <typename T, int DIM>
__device__ __forceinline__ void normal_psi(const T* __restrict__ phi, const Nbr<DIM>& nb, T eps,
                                           T inv2h, T dn, T (&n)[3]) {
    auto ps = [&](int oi, int oj, int ok) { return acdi_psi(ldg(phi, nb.at(oi, oj, ok)), eps); };
    T gr[3];
    gr[0] = (ps(1, 0, 0) - ps(-1, 0, 0)) * inv2h;
    gr[1] = (ps(0, 1, 0) - ps(0, -1, 0)) * inv2h;
    gr[2] = DIM == 3 ? (ps(0, 0, 1) - ps(0, 0, -1)) * inv2h : T(0);
    T s = gr[0] * gr[0] + gr[1] * gr[1];
    if (DIM == 3) s += gr[2] * gr[2];
    const T den = sqrt(s) + dn;
#pragma unroll
    for (int d = 0; d < DIM; ++d) n[d] = divq(gr[d], den);
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_cell_pass(Dims g, Phys ph, const T* __restrict__ phi, T* __restrict__ n0, T* __restrict__ n1,
            T* __restrict__ n2, T* __restrict__ mu_out, T* __restrict__ kap_out,
            T* __restrict__ psi_out) {
    const PC<T> pcn = pc_of(ph, T());
    const double sh = 6.0 * ph.sigma;
    const double c_dw = sh / ph.eps;         // (6 sigma / eps), float64 double-well factor
    const float c_dw_hi = float(c_dw), c_dw_lo = float(c_dw - double(float(c_dw)));
    const T c_lap = T(sh * ph.eps);          // 6 sigma eps
    for_cells(g, [&](int ci, int cj, int ck, int idx) {
    Cell c{ci, cj, ck};
    Nbr<DIM> nb(c, g);
    const T inv_h = ih_of(g, T()), inv2h = i2h_of(g, T()), inv_h2 = ih2_of(g, T());
    const T dn = pcn.delta_n;
    T n[3], mag;
    const T pc = ldg(phi, idx);
    if (psi_out) {
        // ACDI: normals of psi, and psi itself for the face sharpening terms
        normal_psi<T, DIM>(phi, nb, pcn.eps, inv2h, dn, n);
        psi_out[idx] = acdi_psi(pc, pcn.eps);
    } else {
        normal_at<T, DIM>(phi, nb, 0, 0, 0, inv2h, dn, n, mag);
    }
    n0[idx] = n[0];
    n1[idx] = n[1];
    if (DIM == 3) n2[idx] = n[2];
    if (mu_out) {
        T lap = T(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d)
            lap = lap + (ldg(phi, nb.ax(d, 1)) - T(2) * pc + ldg(phi, nb.ax(d, -1))) * inv_h2;
        // double-well term psi'(phi) in float64 precision (cancellation near
        // phi = 0, 1): float64 arithmetic for the float64 path, error-free
        // double-float products for the float32 path
        T dw;
        if constexpr (sizeof(T) == sizeof(double)) {
            dw = T(c_dw * dpsi64(double(pc)));
        } else {
            dw = dwell32(float(pc), c_dw_hi, c_dw_lo);
        }
        mu_out[idx] = dw - c_lap * lap;
    }
    if (kap_out) {
        T div = T(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            T np_[3], nm_[3], mg;
            int oi = d == 0, oj = d == 1, ok = d == 2;
            normal_at<T, DIM>(phi, nb, oi, oj, ok, inv2h, dn, np_, mg);
            normal_at<T, DIM>(phi, nb, -oi, -oj, -ok, inv2h, dn, nm_, mg);
            div = div + (np_[d] - nm_[d]) * inv2h;
        }
        kap_out[idx] = -div;
    }
    (void)inv_h;
    });
}

template <typename T, int DIM>
void launch_cell_pass(const Dims& g, const Phys& ph, const T* phi, T* nrm0, T* nrm1, T* nrm2,
                      T* aux, cudaStream_t s) {
    // aux holds mu for the EB force, kappa otherwise; kappa for SB/ISODI with the
    // EB force, or psi for ACDI, is stored after it (aux + ncell).
    T* mu = nullptr;
    T* kap = nullptr;
    T* psi = ph.model == 3 ? aux + g.ncell : nullptr;
    if (ph.force == 0) {
        mu = aux;
        if (ph.model == 1 || ph.model == 2) kap = aux + g.ncell;
    } else {
        kap = aux;
    }
    if constexpr (DIM == 3 && sizeof(T) == sizeof(float)) {
        if (ph.fused_stage) return;   // the fused stage kernel forms them itself
        if (mu != nullptr && kap == nullptr) {
            launch_cell_pass_mu3d(g, ph, phi, nrm0, nrm1, nrm2, mu, psi, s);
            return;
        }
    }
    k_cell_pass<T, DIM><<<row_grid(g, kThreads, 1 << 30), kThreads, 0, s>>>(g, ph, phi, nrm0, nrm1,
                                                                              nrm2, mu, kap, psi);
}

// ---------------------------------------------------------------------------
// fused stage kernel: phase-field rhs at the cell, momentum rhs at the cell's
// low faces, and the RK stage update of both
// ---------------------------------------------------------------------------
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_stage(Dims g, Phys ph, StageIO<T> io, int stage, int scheme, T wdt, T cdt, int write_rhs) {
    const PC<T> pcs = pc_of(ph, T());
    const T gam_k = T(*io.gamma);
    for_cells(g, [&](int ci, int cj, int ck, int idx) {
    Cell c{ci, cj, ck};
    Nbr<DIM> nb(c, g);
    const T h = T(0), inv_h = ih_of(g, T()), inv2h = i2h_of(g, T()), inv_h2 = ih2_of(g, T());
    const T eps = pcs.eps;
    const T gam = gam_k;
    const T* __restrict__ phi = io.phi_s;
    const T pc = ldg(phi, idx);

    // ---------------- phase field (Eq. 1, Table 1) ----------------
    T kphi = T(0);
    if (ph.model == 0 || ph.model == 3) {
        // CDI flux; ACDI: the sharpening coefficient from psi at the face
        const bool acdi = ph.model == 3;
        const T* __restrict__ psi = io.aux + g.ncell;
        const T psc = acdi ? ldg(psi, idx) : T(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const T* __restrict__ nd = io.nrm[d];
            const T* __restrict__ ud = io.u_s[d];
            // low face (between c - e_d and c)
            T pm = ldg(phi, nb.ax(d, -1));
            T pf = T(0.5) * (pc + pm);
            T nf = T(0.5) * (ldg(nd, idx) + ldg(nd, nb.ax(d, -1)));
            const T shlo = acdi ? acdi_sharp(T(0.5) * (psc + ldg(psi, nb.ax(d, -1))), eps)
                                : pf * (T(1) - pf);
            T Flo = ldg(ud, idx) * pf - gam * (eps * ((pc - pm) * inv_h) - shlo * nf);
            // high face (between c and c + e_d)
            int ip = nb.ax(d, 1);
            T pp = ldg(phi, ip);
            T pf2 = T(0.5) * (pp + pc);
            T nf2 = T(0.5) * (ldg(nd, ip) + ldg(nd, idx));
            const T shhi = acdi ? acdi_sharp(T(0.5) * (ldg(psi, ip) + psc), eps)
                                : pf2 * (T(1) - pf2);
            T Fhi = ldg(ud, nb.axc(d, d, 1)) * pf2 -
                    gam * (eps * ((pp - pc) * inv_h) - shhi * nf2);
            // no flux through a wall
            if (wall_face(g, c.j, 2 * d)) Flo = T(0);
            if (wall_face(g, c.j, 2 * d + 1)) Fhi = T(0);
            kphi = kphi - (Fhi - Flo) * inv_h;
        }
    } else {
        T lap = T(0), g2 = T(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const T* __restrict__ ud = io.u_s[d];
            T pm = ldg(phi, nb.ax(d, -1));
            int ip = nb.ax(d, 1);
            T pp = ldg(phi, ip);
            T Flo = ldg(ud, idx) * (T(0.5) * (pc + pm));
            T Fhi = ldg(ud, nb.axc(d, d, 1)) * (T(0.5) * (pp + pc));
            if (wall_face(g, c.j, 2 * d)) Flo = T(0);
            if (wall_face(g, c.j, 2 * d + 1)) Fhi = T(0);
            kphi = kphi - (Fhi - Flo) * inv_h;
            lap = lap + (pp - T(2) * pc + pm) * inv_h2;
            T gd = (pp - pm) * inv2h;
            g2 = g2 + gd * gd;
        }
        const T* kap = (ph.force == 0) ? io.aux + g.ncell : io.aux;
        T kc = ldg(kap, idx);
        T third = (ph.model == 1) ? eps * sqrt(g2) * kc : pc * (T(1) - pc) * kc;
        T dp;
        if constexpr (sizeof(T) == sizeof(double)) dp = T(dpsi64(double(pc)));
        else dp = dwell32(float(pc), 1.f, 0.f);
        kphi = kphi + gam * (eps * lap - divq(dp, eps) + third);
    }

    // ---------------- momentum at the low faces ----------------
    T ku[3];
    const T sigma = pcs.sigma;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const T* __restrict__ ud = io.u_s[d];
        const int im = nb.ax(d, -1);
        const T pm = ldg(phi, im);
        const T udc = ldg(ud, idx);
        T adv = T(0);
        if (ph.momentum == 0) {
            // advection -(u.grad) u_d, central, transverse components from 4 faces
#pragma unroll
            for (int e = 0; e < DIM; ++e) {
                T vel;
                if (e == d) {
                    vel = udc;
                } else {
                    const T* __restrict__ ue = io.u_s[e];
                    vel = T(0.25) * (ldg(ue, idx) + ldg(ue, nb.axc(e, e, 1)) + ldg(ue, im) +
                                     ldg(ue, nb.ax2c(e, d, -1, e, 1)));
                }
                adv = adv + vel * ((ldg(ud, nb.axc(d, e, 1)) - ldg(ud, nb.axc(d, e, -1))) * inv2h);
            }
        } else {
            // consistent transport: div(m u_d) in flux form, m the mass flux
            // rho_out u + (rho_in - rho_out) F of the CDI phase-field flux F
            // through the face of cell j along dd (cells j and jm = j - e_dd)
            auto mfl = [&](int dd, int j, int jm) -> T {
                const T pj = ldg(phi, j), pjm = ldg(phi, jm);
                const T pf = T(0.5) * (pj + pjm);
                const T nf = T(0.5) * (ldg(io.nrm[dd], j) + ldg(io.nrm[dd], jm));
                const T uj = ldg(io.u_s[dd], j);
                const T F = uj * pf - gam * (eps * ((pj - pjm) * inv_h) - pf * (T(1) - pf) * nf);
                return pcs.rho_out * uj + pcs.drho * F;
            };
            auto cell = [&](int o1, int e1, int o2, int e2) {   // c + o1 e_e1 + o2 e_e2
                int o[3] = {0, 0, 0};
                o[e1] += o1;
                o[e2] += o2;
                return nb.at(o[0], o[1], o[2]);
            };
#pragma unroll
            for (int e = 0; e < DIM; ++e) {
                if (e == d) {
                    // along d: flux at the cells c - e_d and c (their two d-faces)
                    const int ip = nb.ax(d, 1), im2 = nb.ax(d, -2);
                    const T m_lo = mfl(d, im, im2), m_c = mfl(d, idx, im), m_hi = mfl(d, ip, idx);
                    const T u_lo = ldg(ud, im), u_hi = ldg(ud, ip);
                    const T c_hi = T(0.5) * (m_c + m_hi) * (T(0.5) * (udc + u_hi));
                    const T c_lo = T(0.5) * (m_lo + m_c) * (T(0.5) * (u_lo + udc));
                    adv = adv + (c_hi - c_lo) * inv_h;
                } else {
                    // along e: flux at the edges below and above the face (cells
                    // j, j - e_d, j - e_e, j - e_d - e_e for edge j = c, c + e_e)
                    const int jme = nb.ax(e, -1), jmde = cell(-1, d, -1, e);
                    const int jpe = nb.ax(e, 1), jpemd = cell(1, e, -1, d);
                    const T me_lo = T(0.5) * (mfl(e, idx, jme) + mfl(e, im, jmde));
                    const T me_hi = T(0.5) * (mfl(e, jpe, idx) + mfl(e, jpemd, im));
                    const T e_lo = me_lo * (T(0.5) * (udc + ldg(ud, jme)));
                    const T e_hi = me_hi * (T(0.5) * (ldg(ud, jpe) + udc));
                    adv = adv + (e_hi - e_lo) * inv_h;
                }
            }
        }
        // viscous stress divergence
        T visc = T(0);
        const T etac = eta_of(pc, pcs), etam = eta_of(pm, pcs);
#pragma unroll
        for (int e = 0; e < DIM; ++e) {
            if (e == d) {
                T thi = T(2) * etac * ((ldg(ud, nb.axc(d, d, 1)) - udc) * inv_h);
                T tlo = T(2) * etam * ((udc - ldg(ud, im)) * inv_h);
                visc = visc + (thi - tlo) * inv_h;
            } else {
                const T* __restrict__ ue = io.u_s[e];
                // edge at (c - e_d/2 - e_e/2): cells c, c-e_d, c-e_e, c-e_d-e_e
                T eta_lo = T(0.25) * (etac + etam + eta_of(ldg(phi, nb.ax(e, -1)), pcs) +
                                      eta_of(ldg(phi, nb.ax2(d, -1, e, -1)), pcs));
                T tlo = eta_lo * ((udc - ldg(ud, nb.axc(d, e, -1))) * inv_h +
                                  (ldg(ue, idx) - ldg(ue, im)) * inv_h);
                // edge at (c - e_d/2 + e_e/2): cells c+e_e, c+e_e-e_d, c, c-e_d
                const int iep = nb.ax(e, 1), iepm = nb.ax2(d, -1, e, 1);
                T eta_hi = T(0.25) * (eta_of(ldg(phi, iep), pcs) + eta_of(ldg(phi, iepm), pcs) +
                                      etac + etam);
                T thi = eta_hi * ((ldg(ud, nb.axc(d, e, 1)) - udc) * inv_h +
                                  (ldg(ue, nb.axc(e, e, 1)) - ldg(ue, nb.ax2c(e, d, -1, e, 1))) *
                                      inv_h);
                visc = visc + (thi - tlo) * inv_h;
            }
        }
        // surface tension force at the face
        const T dphi = (pc - pm) * inv_h;
        T F;
        if (ph.force == 0) {
            F = T(0.5) * (ldg(io.aux, idx) + ldg(io.aux, im)) * dphi;
        } else {
            T kf = T(0.5) * (ldg(io.aux, idx) + ldg(io.aux, im));
            if (ph.force == 1) {
                F = sigma * kf * dphi;
            } else {
                T pf = T(0.5) * (pc + pm);
                F = T(6) * sigma * kf * pf * (T(1) - pf) * dphi;
            }
        }
        if (ph.momentum == 0) {
            const T beta = divq(T(1), T(0.5) * (rho_of(pc, pcs) + rho_of(pm, pcs)));
            ku[d] = -adv + beta * visc + beta * F;
        } else {
            ku[d] = -adv + visc + F;   // d(rho_f u_d)/dt
        }
        if (wall_face(g, c.j, 2 * d)) ku[d] = T(0);   // the wall's normal velocity stays 0
    }
    (void)h;

    if (write_rhs) {
        io.rhs_phi[idx] = kphi;
#pragma unroll
        for (int d = 0; d < DIM; ++d) io.rhs_u[d][idx] = ku[d];
        return;
    }
    // ---------------- RK stage update ----------------
    const T phin = ldg(io.phi_n, idx);
    // advective: the stages advance u from u^n; consistent: they advance
    // rho_f u from rho_f(phi^n) u^n, which needs phi^n of the neighbour. The
    // last RK4 stage writes phi^{n+1} over phi^n in place, so there the
    // momentum of the step start is not re-formed: the consistent
    // accumulator carries it from stage 0 on.
    const bool cons = ph.momentum == 1;
    T vn[3];
    if (scheme == 1 || stage < 3) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            vn[d] = ldg(io.u_n[d], idx);
            if (cons)
                vn[d] = T(0.5) * (rho_of(phin, pcs) + rho_of(ldg(io.phi_n, nb.ax(d, -1)), pcs)) *
                        vn[d];
        }
    }
    if (scheme == 1) {  // forward Euler
        io.phi_out[idx] = phin + cdt * kphi;
#pragma unroll
        for (int d = 0; d < DIM; ++d) io.u_out[d][idx] = vn[d] + cdt * ku[d];
        return;
    }
    if (stage < 3) {
        T a = stage == 0 ? wdt * kphi : io.acc_phi[idx] + wdt * kphi;
        io.acc_phi[idx] = a;
        io.phi_out[idx] = phin + cdt * kphi;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            T au = stage == 0 ? (cons ? vn[d] + wdt * ku[d] : wdt * ku[d])
                              : io.acc_u[d][idx] + wdt * ku[d];
            io.acc_u[d][idx] = au;
            io.u_out[d][idx] = vn[d] + cdt * ku[d];
        }
    } else {
        io.phi_out[idx] = phin + (io.acc_phi[idx] + wdt * kphi);
#pragma unroll
        for (int d = 0; d < DIM; ++d)
            io.u_out[d][idx] = cons ? io.acc_u[d][idx] + wdt * ku[d]
                                    : ldg(io.u_n[d], idx) + (io.acc_u[d][idx] + wdt * ku[d]);
    }
    });
}

// The same stage on 3D float32 grids, one thread per (i, j) column of a
// 32 x 8 tile marching along z: the periodic neighbour offsets of the column
// are formed once (x, y) or once per plane (z), so every neighbour is one
// address add; the arithmetic is that of k_stage, term by term.
__global__ void __launch_bounds__(256)
k_stage3d(Dims g, Phys ph, StageIO<float> io, int stage, int scheme, float wdt, float cdt,
          int write_rhs, int zc) {
    const int i = blockIdx.x * 32 + threadIdx.x % 32;
    const int j = blockIdx.y * 8 + threadIdx.x / 32;
    if (i >= g.nx || j >= g.ny) return;
    const PC<float> pcs = pc_of(ph, float());
    const float gam = float(*io.gamma);
    const float inv_h = g.ihf, inv2h = g.i2hf, inv_h2 = g.ih2f;
    const float eps = pcs.eps, sigma = pcs.sigma;
    const int sz = g.nx * g.ny;
    const int col = j * g.nx + i;
    int om[3], op[3];   // offsets of the -1 / +1 neighbour along x, y, z
    om[0] = (i == 0 ? g.nx - 1 : i - 1) - i;
    op[0] = (i == g.nx - 1 ? 0 : i + 1) - i;
    om[1] = ((j == 0 ? g.ny - 1 : j - 1) - j) * g.nx;
    op[1] = ((j == g.ny - 1 ? 0 : j + 1) - j) * g.nx;
    const float* __restrict__ phi = io.phi_s;
    const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, g.nz);
    for (int k = z0; k < z1; ++k) {
        om[2] = ((k == 0 ? g.nz - 1 : k - 1) - k) * sz;
        op[2] = ((k == g.nz - 1 ? 0 : k + 1) - k) * sz;
        const int idx = k * sz + col;
        auto at = [&](const float* a, int o) { return __ldg(a + idx + o); };
        const float pc = at(phi, 0);

        // ---------------- phase field (Eq. 1, Table 1) ----------------
        float kphi = 0.f;
        if (ph.model == 0 || ph.model == 3) {
            // CDI flux; ACDI: the sharpening coefficient from psi at the face
            const bool acdi = ph.model == 3;
            const float* __restrict__ psi = io.aux + g.ncell;
            const float psc = acdi ? at(psi, 0) : 0.f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float* __restrict__ nd = io.nrm[d];
                const float* __restrict__ ud = io.u_s[d];
                const float pm = at(phi, om[d]);
                const float pf = 0.5f * (pc + pm);
                const float nf = 0.5f * (at(nd, 0) + at(nd, om[d]));
                const float shlo =
                    acdi ? acdi_sharp(0.5f * (psc + at(psi, om[d])), eps) : pf * (1.f - pf);
                const float Flo = at(ud, 0) * pf - gam * (eps * ((pc - pm) * inv_h) - shlo * nf);
                const float pp = at(phi, op[d]);
                const float pf2 = 0.5f * (pp + pc);
                const float nf2 = 0.5f * (at(nd, op[d]) + at(nd, 0));
                const float shhi =
                    acdi ? acdi_sharp(0.5f * (at(psi, op[d]) + psc), eps) : pf2 * (1.f - pf2);
                const float Fhi = at(ud, op[d]) * pf2 - gam * (eps * ((pp - pc) * inv_h) - shhi * nf2);
                kphi = kphi - (Fhi - Flo) * inv_h;
            }
        } else {
            float lap = 0.f, g2 = 0.f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float* __restrict__ ud = io.u_s[d];
                const float pm = at(phi, om[d]);
                const float pp = at(phi, op[d]);
                const float Flo = at(ud, 0) * (0.5f * (pc + pm));
                const float Fhi = at(ud, op[d]) * (0.5f * (pp + pc));
                kphi = kphi - (Fhi - Flo) * inv_h;
                lap = lap + (pp - 2.f * pc + pm) * inv_h2;
                const float gd = (pp - pm) * inv2h;
                g2 = g2 + gd * gd;
            }
            const float* kap = (ph.force == 0) ? io.aux + g.ncell : io.aux;
            const float kc = at(kap, 0);
            const float third = (ph.model == 1) ? eps * sqrtf(g2) * kc : pc * (1.f - pc) * kc;
            const float dp = dwell32(pc, 1.f, 0.f);
            kphi = kphi + gam * (eps * lap - divq(dp, eps) + third);
        }

        // ---------------- momentum at the low faces ----------------
        float ku[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float* __restrict__ ud = io.u_s[d];
            const int im = om[d];
            const float pm = at(phi, im);
            const float udc = at(ud, 0);
            // advection -(u.grad) u_d, central, transverse components from 4 faces
            float adv = 0.f;
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                float vel;
                if (e == d) {
                    vel = udc;
                } else {
                    const float* __restrict__ ue = io.u_s[e];
                    vel = 0.25f * (at(ue, 0) + at(ue, op[e]) + at(ue, im) + at(ue, im + op[e]));
                }
                adv = adv + vel * ((at(ud, op[e]) - at(ud, om[e])) * inv2h);
            }
            // viscous stress divergence
            float visc = 0.f;
            const float etac = eta_of(pc, pcs), etam = eta_of(pm, pcs);
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                if (e == d) {
                    const float thi = 2.f * etac * ((at(ud, op[d]) - udc) * inv_h);
                    const float tlo = 2.f * etam * ((udc - at(ud, im)) * inv_h);
                    visc = visc + (thi - tlo) * inv_h;
                } else {
                    const float* __restrict__ ue = io.u_s[e];
                    // edge at (c - e_d/2 - e_e/2): cells c, c-e_d, c-e_e, c-e_d-e_e
                    const float eta_lo = 0.25f * (etac + etam + eta_of(at(phi, om[e]), pcs) +
                                                  eta_of(at(phi, im + om[e]), pcs));
                    const float tlo = eta_lo * ((udc - at(ud, om[e])) * inv_h +
                                                (at(ue, 0) - at(ue, im)) * inv_h);
                    // edge at (c - e_d/2 + e_e/2): cells c+e_e, c+e_e-e_d, c, c-e_d
                    const int iep = op[e], iepm = im + op[e];
                    const float eta_hi = 0.25f * (eta_of(at(phi, iep), pcs) +
                                                  eta_of(at(phi, iepm), pcs) + etac + etam);
                    const float thi = eta_hi * ((at(ud, iep) - udc) * inv_h +
                                                (at(ue, iep) - at(ue, iepm)) * inv_h);
                    visc = visc + (thi - tlo) * inv_h;
                }
            }
            // surface tension force at the face
            const float dphi = (pc - pm) * inv_h;
            float F;
            if (ph.force == 0) {
                F = 0.5f * (at(io.aux, 0) + at(io.aux, im)) * dphi;
            } else {
                const float kf = 0.5f * (at(io.aux, 0) + at(io.aux, im));
                if (ph.force == 1) {
                    F = sigma * kf * dphi;
                } else {
                    const float pf = 0.5f * (pc + pm);
                    F = 6.f * sigma * kf * pf * (1.f - pf) * dphi;
                }
            }
            const float beta = divq(1.f, 0.5f * (rho_of(pc, pcs) + rho_of(pm, pcs)));
            ku[d] = -adv + beta * visc + beta * F;
        }

        if (write_rhs) {
            io.rhs_phi[idx] = kphi;
#pragma unroll
            for (int d = 0; d < 3; ++d) io.rhs_u[d][idx] = ku[d];
            continue;
        }
        // ---------------- RK stage update ----------------
        const float phin = __ldg(io.phi_n + idx);
        if (scheme == 1) {  // forward Euler
            io.phi_out[idx] = phin + cdt * kphi;
#pragma unroll
            for (int d = 0; d < 3; ++d) io.u_out[d][idx] = __ldg(io.u_n[d] + idx) + cdt * ku[d];
            continue;
        }
        if (stage < 3) {
            const float a = stage == 0 ? wdt * kphi : io.acc_phi[idx] + wdt * kphi;
            io.acc_phi[idx] = a;
            io.phi_out[idx] = phin + cdt * kphi;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float au = stage == 0 ? wdt * ku[d] : io.acc_u[d][idx] + wdt * ku[d];
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
}

template <typename T, int DIM>
void launch_stage(const Dims& g, const Phys& ph, const StageIO<T>& io, int stage, int scheme,
                  double wdt, double cdt, int write_rhs, cudaStream_t s) {
    if constexpr (DIM == 3 && sizeof(T) == sizeof(float)) {
        if (ph.fused_stage) {
            launch_stage_fused(g, ph, io, stage, scheme, wdt, cdt, write_rhs, s);
            return;
        }
        if (ph.momentum == 1) {
            k_stage<T, DIM><<<row_grid(g, kThreads, 1 << 30), kThreads, 0, s>>>(
                g, ph, io, stage, scheme, T(wdt), T(cdt), write_rhs);
            return;
        }
        const long long cols = (long long)((g.nx + 31) / 32) * ((g.ny + 7) / 8);
        int zc = 64;
        while (zc > 1 && cols * ((g.nz + zc - 1) / zc) < 8 * 152) zc >>= 1;
        dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, (g.nz + zc - 1) / zc);
        k_stage3d<<<grid, 256, 0, s>>>(g, ph, io, stage, scheme, float(wdt), float(cdt),
                                       write_rhs, zc);
        return;
    }
    k_stage<T, DIM><<<row_grid(g, kThreads, 1 << 30), kThreads, 0, s>>>(g, ph, io, stage, scheme,
                                                                          T(wdt), T(cdt), write_rhs);
}

// ---------------------------------------------------------------------------
// Gamma = gamma_fixed, or max(gamma_min, max |u|)
// ---------------------------------------------------------------------------
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_gamma(Dims g, const T* __restrict__ u0, const T* __restrict__ u1, const T* __restrict__ u2,
        double gamma_fixed, double gamma_min, double* gamma, RedBuf rb) {
    // the maximum of |u| is exact in the storage precision: float32 values
    // are compared on the float32 pipe and widened once per thread
    T m = T(0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.ncell; i += gridDim.x * blockDim.x) {
        m = max(m, abs(u0[i]));
        m = max(m, abs(u1[i]));
        if (DIM == 3) m = max(m, abs(u2[i]));
    }
    double v[1] = {double(m)}, tot[1];
    const int mode[1] = {1};
    if (grid_reduce<1>(v, mode, rb, tot) && threadIdx.x == 0)
        *gamma = gamma_fixed > 0.0 ? gamma_fixed : fmax(gamma_min, tot[0]);
}

template <typename T, int DIM>
void launch_gamma(const Dims& g, const T* const* u, double gamma_fixed, double gamma_min,
                  double* gamma, RedBuf rb, cudaStream_t s) {
    k_gamma<T, DIM><<<red_grid(g.ncell), kThreads, 0, s>>>(g, u[0], u[1], DIM == 3 ? u[2] : u[0],
                                                            gamma_fixed, gamma_min, gamma, rb);
}

// ---------------------------------------------------------------------------
// b = D u* / tau and its sum (the mean is removed by the solver). Float64
// path: b float64. Mixed path: b a double-float (hi plane, then lo plane in
// the same 8 n bytes), formed without the float64 pipe.
// ---------------------------------------------------------------------------
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_divergence(Dims g, const T* __restrict__ u0, const T* __restrict__ u1, const T* __restrict__ u2,
             double inv_tau, double* __restrict__ b, RedBuf rb, CGScalars* sc,
             const T* __restrict__ mphi, Phys ph) {
    double s = 0.0;
    const double inv_h = g.ih;
    f2 acc{0.f, 0.f};
    const f2 scale = sizeof(T) == sizeof(float) ? df_of(inv_h * inv_tau) : f2{0.f, 0.f};
    for_cells(g, [&](int i, int j, int k, int idx) {
        const Nb6 nb = nb6<DIM>(g, i, j, k, idx);
        if (mphi != nullptr) {
            // consistent transport: u* = (rho_f u*) / rho_f, formed as in k_correct
            const T* uu[3] = {u0, u1, u2};
            T v[3][2];
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                v[d][0] = mom_to_vel<T>(uu[d][idx], mphi[idx], mphi[nb.m[2 * d]], ph);
                v[d][1] = mom_to_vel<T>(uu[d][nb.m[2 * d + 1]], mphi[nb.m[2 * d + 1]], mphi[idx], ph);
            }
            if constexpr (sizeof(T) == sizeof(double)) {
                double dv = (double(v[0][1]) - double(v[0][0])) * inv_h;
                dv += (double(v[1][1]) - double(v[1][0])) * inv_h;
                if (DIM == 3) dv += (double(v[2][1]) - double(v[2][0])) * inv_h;
                dv *= inv_tau;
                b[idx] = dv;
                s += dv;
            } else {
                f2 t = two_sum(float(v[0][1]), -float(v[0][0]));
#pragma unroll
                for (int d = 1; d < DIM; ++d) {
                    const f2 c1 = two_sum(float(v[d][1]), -float(v[d][0]));
                    f2 t2 = two_sum(t.hi, c1.hi);
                    t2.lo = __fadd_rn(t2.lo, __fadd_rn(t.lo, c1.lo));
                    t = t2;
                }
                const f2 r = f2_mul(t, scale);
                float* bf = reinterpret_cast<float*>(b);
                bf[idx] = r.hi;
                bf[idx + g.ncell] = r.lo;
                acc = df_add(acc, r);
            }
            return;
        }
        if (sizeof(T) == sizeof(double)) {
            double dv = (double(u0[nb.m[1]]) - double(u0[idx])) * inv_h;
            dv += (double(u1[nb.m[3]]) - double(u1[idx])) * inv_h;
            if (DIM == 3) dv += (double(u2[nb.m[5]]) - double(u2[idx])) * inv_h;
            dv *= inv_tau;
            b[idx] = dv;
            s += dv;
        } else {
            // float32 velocities: exact differences (TwoSum) summed as a
            // double-float and scaled by 1 / (h tau) as a double-float
            const float* uf0 = reinterpret_cast<const float*>(u0);
            const float* uf1 = reinterpret_cast<const float*>(u1);
            const float* uf2 = reinterpret_cast<const float*>(u2);
            f2 a = two_sum(uf0[nb.m[1]], -uf0[idx]);
            const f2 b1 = two_sum(uf1[nb.m[3]], -uf1[idx]);
            f2 t = two_sum(a.hi, b1.hi);
            t.lo = __fadd_rn(t.lo, __fadd_rn(a.lo, b1.lo));
            if (DIM == 3) {
                const f2 c1 = two_sum(uf2[nb.m[5]], -uf2[idx]);
                f2 t2 = two_sum(t.hi, c1.hi);
                t2.lo = __fadd_rn(t2.lo, __fadd_rn(t.lo, c1.lo));
                t = t2;
            }
            const f2 r = f2_mul(t, scale);
            float* bf = reinterpret_cast<float*>(b);
            bf[idx] = r.hi;
            bf[idx + g.ncell] = r.lo;
            acc = df_add(acc, r);
        }
    });
    if (sizeof(T) == sizeof(float)) s = double(acc.hi) + double(acc.lo);
    double v[1] = {s}, tot[1];
    const int mode[1] = {0};
    if (grid_reduce<1>(v, mode, rb, tot) && threadIdx.x == 0) sc->mean_b = tot[0] / g.ncell;
}

template <typename T, int DIM>
void launch_divergence(const Dims& g, const T* const* u, double inv_tau, double* b, RedBuf rb,
                       CGScalars* sc, cudaStream_t s, const T* mom_phi, const Phys* ph) {
    if constexpr (DIM == 3 && sizeof(T) == sizeof(float)) {
        if (mom_phi == nullptr && divergence3d_ok(g)) {
            launch_divergence3d(g, u, inv_tau, b, rb, sc, s);
            return;
        }
    }
    Phys pz;
    memset(&pz, 0, sizeof(pz));
    k_divergence<T, DIM><<<row_grid(g, kThreads, kRedBlocks), kThreads, 0, s>>>(
        g, u[0], u[1], DIM == 3 ? u[2] : u[0], inv_tau, b, rb, sc, mom_phi, ph ? *ph : pz);
}

// ---------------------------------------------------------------------------
// correction u = u* - tau G p / rho_f
// ---------------------------------------------------------------------------
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_correct(Dims g, Phys ph, const T* __restrict__ phi, const double* __restrict__ b0,
          const double* __restrict__ b1, const double* __restrict__ b2,
          const float* __restrict__ f0, const float* __restrict__ f1, const float* __restrict__ f2,
          const T* __restrict__ s0,
          const T* __restrict__ s1, const T* __restrict__ s2, const double* __restrict__ p,
          double tau, T* __restrict__ o0, T* __restrict__ o1, T* __restrict__ o2) {
    const double inv_h = g.ih;
    const float tau_h = float(tau * g.ih);
    for_cells(g, [&](int i, int j, int k, int idx) {
        const Nb6 nb = nb6<DIM>(g, i, j, k, idx);
        const double pp = b0 != nullptr ? p[idx] : 0.0;
        const T* sv[3] = {s0, s1, s2};
        T* ov[3] = {o0, o1, o2};
        const double* bv[3] = {b0, b1, b2};
        const float* fv[3] = {f0, f1, f2};
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const int m = nb.m[2 * d];
            // consistent transport: s holds rho_f u*, formed into u* as in k_divergence
            const T us = ph.momentum == 1 ? mom_to_vel<T>(sv[d][idx], phi[idx], phi[m], ph)
                                          : sv[d][idx];
            if (b0 != nullptr) {
                // float64 path: the solver's float64 face coefficients
                const double gp = (pp - p[m]) * inv_h;
                ov[d][idx] = T(double(us) - tau * bv[d][idx] * gp);
            } else {
                // float32 path: same beta as the pressure operator; the pressure
                // is a double-float (hi plane, lo plane), its difference formed
                // from both parts, scaled and applied in float32
                const float beta = f0 != nullptr        ? __ldg(fv[d] + idx)
                                   : wall_face(g, j, 2 * d) ? 0.f
                                                            : beta_face32(float(phi[idx]), float(phi[m]), ph);
                const float* ph_ = reinterpret_cast<const float*>(p);
                const float* pl_ = ph_ + g.ncell;
                const float gp =
                    __fadd_rn(__fsub_rn(ph_[idx], ph_[m]), __fsub_rn(pl_[idx], pl_[m])) * tau_h;
                ov[d][idx] = T(float(us) - beta * gp);
            }
        }
    });
}

template <typename T, int DIM>
void launch_correct(const Dims& g, const Phys& ph, const T* phi, const double* const* beta64,
                    const float* const* beta32, const T* const* ustar, const double* p,
                    double tau, T* const* uout, cudaStream_t s) {
    const double* b0 = beta64 ? beta64[0] : nullptr;
    const double* b1 = beta64 ? beta64[1] : nullptr;
    const double* b2 = beta64 ? beta64[DIM == 3 ? 2 : 1] : nullptr;
    const float* f0 = beta32 ? beta32[0] : nullptr;
    const float* f1 = beta32 ? beta32[1] : nullptr;
    const float* f2 = beta32 ? beta32[DIM == 3 ? 2 : 1] : nullptr;
    if constexpr (DIM == 3 && sizeof(T) == sizeof(float)) {
        if (f0 != nullptr && ph.momentum == 0) {
            launch_correct3d(g, beta32, ustar, p, tau, uout, s);
            return;
        }
    }
    k_correct<T, DIM><<<row_grid(g, kThreads, 1 << 30), kThreads, 0, s>>>(
        g, ph, phi, b0, b1, b2, f0, f1, f2, ustar[0], ustar[1], DIM == 3 ? ustar[2] : ustar[0], p,
        tau, uout[0], uout[1], DIM == 3 ? uout[2] : uout[0]);
}

// ---------------------------------------------------------------------------
// diagnostics (Section 3.1 Ca_inf, Section 3.2 energies)
// ---------------------------------------------------------------------------
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_diag(Dims g, Phys ph, const T* __restrict__ phi, const T* __restrict__ u0,
       const T* __restrict__ u1, const T* __restrict__ u2, const double* __restrict__ p, RedBuf rb,
       DiagOut* out) {
    const PC<double> pcd = pc_of(ph, double());
    double mass = 0, ke = 0, se = 0, umax = 0, pmin = 1e308, pmax = -1e308;
    double pin = 0, pout = 0, nin = 0, nout = 0, psum = 0, bad = 0;
    const double inv_h = g.ih, sh = 6.0 * ph.sigma;
    for_cells(g, [&](int ci, int cj, int ck, int idx) {
        const Nb6 nb = nb6<DIM>(g, ci, cj, ck, idx);
        double pc = double(phi[idx]);
        int im[3] = {nb.m[0], nb.m[2], nb.m[4]};
        const T* uv[3] = {u0, u1, u2};
        double rc = rho_of(pc, pcd);
        double grad2 = 0.0;
        for (int d = 0; d < DIM; ++d) {
            double pm = double(phi[im[d]]);
            double rf = 0.5 * (rc + rho_of(pm, pcd));
            double ud = double(uv[d][idx]);
            ke += 0.5 * rf * ud * ud;
            umax = fmax(umax, fabs(ud));
            // no gradient across a wall (the image cell mirrors phi)
            double df = wall_face(g, cj, 2 * d) ? 0.0 : (pc - pm) * inv_h;
            grad2 += df * df;
            if (!isfinite(ud)) bad += 1.0;
        }
        double w = pc * (1.0 - pc);
        se += (sh / ph.eps) * 0.5 * w * w + 0.5 * sh * ph.eps * grad2;
        mass += pc;
        pmin = fmin(pmin, pc);
        pmax = fmax(pmax, pc);
        double pp;
        if constexpr (sizeof(T) == sizeof(float)) {
            // mixed path: the pressure is a double-float (hi plane, lo plane)
            const float* pf = reinterpret_cast<const float*>(p);
            pp = double(pf[idx]) + double(pf[idx + g.ncell]);
        } else {
            pp = p[idx];
        }
        psum += pp;
        if (pc >= 0.999) { pin += pp; nin += 1.0; }
        if (pc <= 0.001) { pout += pp; nout += 1.0; }
        if (!isfinite(pc) || !isfinite(pp)) bad += 1.0;
    });
    double v[12] = {mass, ke, se, umax, -pmin, pmax, pin, pout, nin, nout, psum, bad};
    const int mode[12] = {0, 0, 0, 1, 1, 1, 0, 0, 0, 0, 0, 0};
    double tot[12];
    if (grid_reduce<12>(v, mode, rb, tot) && threadIdx.x == 0) {
        double dV = 1.0;
        for (int d = 0; d < DIM; ++d) dV *= g.h;
        out->mass = tot[0] * dV;
        out->ke = tot[1] * dV;
        out->se = tot[2] * dV;
        out->umax = tot[3];
        out->phi_min = -tot[4];
        out->phi_max = tot[5];
        out->p_in_sum = tot[6];
        out->p_out_sum = tot[7];
        out->n_in = tot[8];
        out->n_out = tot[9];
        out->p_sum = tot[10];
        out->nonfinite = tot[11];
    }
}

template <typename T, int DIM>
void launch_diagnostics(const Dims& g, const Phys& ph, const T* phi, const T* const* u,
                        const double* p, RedBuf rb, DiagOut* out, cudaStream_t s) {
    k_diag<T, DIM><<<row_grid(g, kThreads, kRedBlocks), kThreads, 0, s>>>(g, ph, phi, u[0], u[1],
                                                           DIM == 3 ? u[2] : u[0], p, rb, out);
}

// ---------------------------------------------------------------------------
// double-float planes <-> float64 (API transfers of the mixed path's pressure
// and right-hand side)
// ---------------------------------------------------------------------------
__global__ void k_double_to_df(const double* __restrict__ src, float* __restrict__ hi,
                               float* __restrict__ lo, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const f2 v = df_of(src[i]);
        hi[i] = v.hi;
        lo[i] = v.lo;
    }
}
__global__ void k_df_to_double(const float* __restrict__ hi, const float* __restrict__ lo,
                               double* __restrict__ dst, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = double(hi[i]) + double(lo[i]);
}
__global__ void k_sub_mean(double* x, int n, const double* sum_ptr, double inv_n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double m = (*sum_ptr) * inv_n;
    if (i < n) x[i] -= m;
}
// out = 2 a - b (float64 arrays, or double-float planes when df); out may be b
__global__ void k_extrapolate(int n, int df, const double* a, const double* b, double* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (df) {
        const float* ah = reinterpret_cast<const float*>(a);
        const float* bh = reinterpret_cast<const float*>(b);
        float* oh = reinterpret_cast<float*>(out);
        const f2 v = df_add(f2{2.f * ah[i], 2.f * ah[i + n]}, f2{-bh[i], -bh[i + n]});
        oh[i] = v.hi;
        oh[i + n] = v.lo;
    } else {
        out[i] = 2.0 * a[i] - b[i];
    }
}
void launch_extrapolate(int n, bool df, const double* a, const double* b, double* out,
                        cudaStream_t s) {
    k_extrapolate<<<lin_grid(n), kThreads, 0, s>>>(n, df ? 1 : 0, a, b, out);
}
void launch_double_to_df(const double* src, float* hi, float* lo, int n, cudaStream_t s) {
    k_double_to_df<<<lin_grid(n), kThreads, 0, s>>>(src, hi, lo, n);
}
void launch_df_to_double(const float* hi, const float* lo, double* dst, int n, cudaStream_t s) {
    k_df_to_double<<<lin_grid(n), kThreads, 0, s>>>(hi, lo, dst, n);
}
void launch_sub_mean(double* x, int n, const double* sum_ptr, double inv_n, cudaStream_t s) {
    k_sub_mean<<<lin_grid(n), kThreads, 0, s>>>(x, n, sum_ptr, inv_n);
}

// ---------------------------------------------------------------------------
// explicit instantiations
// ---------------------------------------------------------------------------
#define PF_INST_TD(T, D)                                                                        \
    template void launch_init_phi<T, D>(const Dims&, const Phys&, double, int, double, int, T*, \
                                        cudaStream_t);                                          \
    template void launch_cell_pass<T, D>(const Dims&, const Phys&, const T*, T*, T*, T*, T*,    \
                                         cudaStream_t);                                         \
    template void launch_stage<T, D>(const Dims&, const Phys&, const StageIO<T>&, int, int,     \
                                     double, double, int, cudaStream_t);                        \
    template void launch_gamma<T, D>(const Dims&, const T* const*, double, double, double*,     \
                                     RedBuf, cudaStream_t);                                     \
    template void launch_divergence<T, D>(const Dims&, const T* const*, double, double*,        \
                                          RedBuf, CGScalars*, cudaStream_t, const T*,           \
                                          const Phys*);                                         \
    template void launch_correct<T, D>(const Dims&, const Phys&, const T*, const double* const*, \
                                       const float* const*, const T* const*, const double*,     \
                                       double, T* const*, cudaStream_t);                        \
    template void launch_diagnostics<T, D>(const Dims&, const Phys&, const T*, const T* const*, \
                                           const double*, RedBuf, DiagOut*, cudaStream_t);

PF_INST_TD(double, 2)
PF_INST_TD(double, 3)
PF_INST_TD(float, 2)
PF_INST_TD(float, 3)

template void launch_convert_in<double>(const double*, double*, int, cudaStream_t);
template void launch_convert_in<float>(const double*, float*, int, cudaStream_t);
template void launch_convert_out<double>(const double*, double*, int, double, const double*,
                                         double, cudaStream_t);
template void launch_convert_out<float>(const float*, double*, int, double, const double*, double,
                                        cudaStream_t);

}  // namespace pf
