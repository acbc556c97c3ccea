// Reverse-mode (adjoint) kernels of the float64 fractional step: the
// transposed Jacobian of the phase-field right-hand side (CDI, Table 1), of the
// momentum right-hand side with the energy-based force (Eq. eb_st, Eq. ac_mu),
// and of the variable-density projection, applied to given cotangents; plus
// the objective (kinetic energy and interface misfit) with its gradient.
//
// Notation: a = cotangent of the phase-field rhs (cells), b_d = cotangent of
// the momentum rhs on the d-faces. Every forward quantity the transposes need
// (face averages, normals, viscous stress, face coefficients) is recomputed
// from the stage state exactly as the forward kernels form it. Each transpose
// is written as a gather (one thread per output entry), so there are no
// atomics and every sum has a fixed order.
#include "pf_device.cuh"

namespace pf {

namespace {

__device__ __forceinline__ double clip01(double v) { return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v); }
// d clip(phi) / d phi: 1 strictly inside (0, 1), 0 elsewhere
__device__ __forceinline__ double dclip(double v) { return (v > 0.0 && v < 1.0) ? 1.0 : 0.0; }
__device__ __forceinline__ double rho_c(double phi, const Phys& ph) {
    return ph.rho_out + ph.drho * clip01(phi);
}
__device__ __forceinline__ double eta_c(double phi, const Phys& ph) {
    return ph.mu_out + ph.dmu * clip01(phi);
}
__device__ __forceinline__ double beta_f(double pa, double pb, const Phys& ph) {
    return 1.0 / (0.5 * (rho_c(pa, ph) + rho_c(pb, ph)));
}
__device__ __forceinline__ double dpsi(double p) { return p * (1.0 - p) * (1.0 - 2.0 * p); }
__device__ __forceinline__ double d2psi(double p) { return 1.0 - 6.0 * p + 6.0 * p * p; }

// index of pair (d, e), d != e: (0,1) -> 0, (0,2) -> 1, (1,2) -> 2
__device__ __forceinline__ int pidx(int d, int e) { return d + e - 1; }

template <int DIM>
__device__ __forceinline__ int off(const Nbr<DIM>& nb, int d1, int o1, int d2, int o2) {
    int o[3] = {0, 0, 0};
    o[d1] += o1;
    o[d2] += o2;
    return nb.at(o[0], o[1], o[2]);
}
template <int DIM>
__device__ __forceinline__ int off3(const Nbr<DIM>& nb, int d1, int o1, int d2, int o2, int d3,
                                    int o3) {
    int o[3] = {0, 0, 0};
    o[d1] += o1;
    o[d2] += o2;
    o[d3] += o3;
    return nb.at(o[0], o[1], o[2]);
}

// Viscous term visc_d at the d-face of cell c (face c - e_d/2), formed as the
// forward stage kernel forms it.
template <int DIM>
__device__ double visc_at(const Nbr<DIM>& nb, int idx, int d, const double* phi,
                          const double* const* u, const Phys& ph, double inv_h) {
    const double* ud = u[d];
    const int im = nb.ax(d, -1);
    const double pc = phi[idx], pm = phi[im];
    const double udc = ud[idx];
    const double etac = eta_c(pc, ph), etam = eta_c(pm, ph);
    double visc = 0.0;
    for (int e = 0; e < DIM; ++e) {
        if (e == d) {
            const double thi = 2.0 * etac * ((ud[nb.ax(d, 1)] - udc) * inv_h);
            const double tlo = 2.0 * etam * ((udc - ud[im]) * inv_h);
            visc += (thi - tlo) * inv_h;
        } else {
            const double* ue = u[e];
            const double eta_lo = 0.25 * (etac + etam + eta_c(phi[nb.ax(e, -1)], ph) +
                                          eta_c(phi[off(nb, d, -1, e, -1)], ph));
            const double tlo = eta_lo * ((udc - ud[nb.ax(e, -1)]) * inv_h + (ue[idx] - ue[im]) * inv_h);
            const int iep = nb.ax(e, 1), iepm = off(nb, d, -1, e, 1);
            const double eta_hi =
                0.25 * (eta_c(phi[iep], ph) + eta_c(phi[iepm], ph) + etac + etam);
            const double thi = eta_hi * ((ud[iep] - udc) * inv_h + (ue[iep] - ue[iepm]) * inv_h);
            visc += (thi - tlo) * inv_h;
        }
    }
    return visc;
}

// Accumulate K block sums into acc[slot..slot+K) from the last block (fixed order).
template <int K>
__device__ __forceinline__ void reduce_into(double (&v)[K], RedBuf rb, double* acc) {
    int mode[K];
#pragma unroll
    for (int q = 0; q < K; ++q) mode[q] = 0;
    double tot[K];
    if (grid_reduce<K>(v, mode, rb, tot) && threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) acc[q] += tot[q];
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// face pass: per d-face of cell c, the face-local parts of the transposes
//   phase field (CDI flux F = u phi_f - Gamma[eps dphi - phi_f (1 - phi_f) n_f]):
//     Fbar = (a_c - a_{c-d}) / h, ubar_d = Fbar phi_f,
//     phi_f-bar = Fbar (u + Gamma (1 - 2 phi_f) n_f), dphi-bar = -Gamma eps Fbar,
//     n_f-bar = Gamma phi_f (1 - phi_f) Fbar, Gamma-bar += -Fbar (eps dphi - phi_f(1-phi_f) n_f)
//   momentum (ku = -adv + beta (visc + F), F = mu_f dphi):
//     W = b beta, rho_f-bar = -beta^2 b (visc + F), mu_f-bar = W dphi, dphi-bar += W mu_f
// lo / hi: the phi cotangent this face sends to cell c / cell c - d.
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_adj_faces(Dims g, Phys ph, AdjRhsIO io, RedBuf rb) {
    const double inv_h = g.ih;
    const double gam = *io.gamma;
    const double eps = ph.eps;
    double gsum = 0.0;
    for_cells(g, [&](int ci, int cj, int ck, int idx) {
        Cell c{ci, cj, ck};
        Nbr<DIM> nb(c, g);
        const double pc = io.phi[idx];
        const double ac = io.kbar_phi[idx];
        const double muc = io.mu[idx];
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const int im = nb.ax(d, -1);
            const double pm = io.phi[im];
            const double pf = 0.5 * (pc + pm);
            const double dphi = (pc - pm) * inv_h;
            const double nf = 0.5 * (io.nrm[d][idx] + io.nrm[d][im]);
            const double ud = io.u[d][idx];
            const double Fb = (ac - io.kbar_phi[im]) * inv_h;
            const double pfb = Fb * (ud + gam * (1.0 - 2.0 * pf) * nf);
            double dpb = -gam * eps * Fb;
            const double nfb = gam * pf * (1.0 - pf) * Fb;
            gsum += -Fb * (eps * dphi - pf * (1.0 - pf) * nf);
            // momentum
            const double bd = io.kbar_u[d][idx];
            const double beta = beta_f(pc, pm, ph);
            const double visc = visc_at<DIM>(nb, idx, d, io.phi, io.u, ph, inv_h);
            const double muf = 0.5 * (muc + io.mu[im]);
            const double F = muf * dphi;
            const double W = bd * beta;
            io.rhofb[d][idx] = -beta * beta * bd * (visc + F);
            io.mufb[d][idx] = W * dphi;
            dpb += W * muf;
            io.W[d][idx] = W;
            io.nfb[d][idx] = nfb;
            io.lo[d][idx] = 0.5 * pfb + dpb * inv_h;
            io.hi[d][idx] = 0.5 * pfb - dpb * inv_h;
            io.ubar[d][idx] = Fb * pf;
        }
    });
    double v[1] = {gsum};
    reduce_into<1>(v, rb, io.acc + 5);
}

// edge cotangent of the symmetric viscous stress tau_de at the edge of index j
// (cells j, j-d, j-e, j-d-e): (W_d(j-e) - W_d(j)) / h + (W_e(j-d) - W_e(j)) / h
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_adj_edges(Dims g, AdjRhsIO io) {
    const double inv_h = g.ih;
    for_cells(g, [&](int ci, int cj, int ck, int idx) {
        Cell c{ci, cj, ck};
        Nbr<DIM> nb(c, g);
#pragma unroll
        for (int d = 0; d < DIM; ++d)
#pragma unroll
            for (int e = d + 1; e < DIM; ++e)
                io.te[pidx(d, e)][idx] = (io.W[d][nb.ax(e, -1)] - io.W[d][idx]) * inv_h +
                                         (io.W[e][nb.ax(d, -1)] - io.W[e][idx]) * inv_h;
    });
}

// cell pass: gathers the face contributions of cell c and forms
//   n-bar = mean of the two n_f-bars, g-bar = (dn/dg)^T n-bar (n = g / (|g| + delta_n)),
//   mu-bar = mean of the mu_f-bars, phi-bar += (6 sigma/eps) psi'' mu-bar,
//   rho-bar, eta-bar (diagonal and edge stresses) -> phi-bar through clip(phi),
//   parameter sums: sigma, rho_in, rho_out, mu_in, mu_out
template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_adj_cells(Dims g, Phys ph, AdjRhsIO io, RedBuf rb) {
    const double inv_h = g.ih, inv2h = g.i2h, inv_h2 = g.ih2;
    const double sh = 6.0 * ph.sigma;
    double s_sig = 0.0, s_rin = 0.0, s_rout = 0.0, s_min = 0.0, s_mout = 0.0;
    for_cells(g, [&](int ci, int cj, int ck, int idx) {
        Cell c{ci, cj, ck};
        Nbr<DIM> nb(c, g);
        const double pc = io.phi[idx];
        double phib = 0.0, mub = 0.0, rhob = 0.0, etab = 0.0, lap = 0.0;
        double gr[3] = {0.0, 0.0, 0.0}, nb_[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const int ip = nb.ax(d, 1), im = nb.ax(d, -1);
            phib += io.lo[d][idx] + io.hi[d][ip];
            nb_[d] = 0.5 * (io.nfb[d][idx] + io.nfb[d][ip]);
            mub += 0.5 * (io.mufb[d][idx] + io.mufb[d][ip]);
            rhob += 0.5 * (io.rhofb[d][idx] + io.rhofb[d][ip]);
            gr[d] = (io.phi[ip] - io.phi[im]) * inv2h;
            lap += (io.phi[ip] - 2.0 * pc + io.phi[im]) * inv_h2;
            // diagonal stress tau_dd at the cell: 2 eta (u_d(c+d) - u_d(c)) / h
            const double tb = (io.W[d][idx] - io.W[d][ip]) * inv_h;
            etab += tb * 2.0 * (io.u[d][ip] - io.u[d][idx]) * inv_h;
        }
        // edge stresses around the cell: edges c, c+d, c+e, c+d+e of each pair
#pragma unroll
        for (int d = 0; d < DIM; ++d)
#pragma unroll
            for (int e = d + 1; e < DIM; ++e) {
                const double* te = io.te[pidx(d, e)];
                const double* ud = io.u[d];
                const double* ue = io.u[e];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int od = q & 1, oe = q >> 1;   // edge j = c + od e_d + oe e_e
                    const int j = off(nb, d, od, e, oe);
                    const int jme = off(nb, d, od, e, oe - 1);
                    const int jmd = off(nb, d, od - 1, e, oe);
                    const double S = (ud[j] - ud[jme]) * inv_h + (ue[j] - ue[jmd]) * inv_h;
                    etab += 0.25 * te[j] * S;
                }
            }
        // normals n = g / (|g| + delta_n)
        double m2 = 0.0, ng = 0.0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            m2 += gr[d] * gr[d];
            ng += nb_[d] * gr[d];
        }
        const double m = sqrt(m2);
        const double den = m + ph.delta_n;
        const double corr = m > 0.0 ? ng / (m * den * den) : 0.0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) io.gbar[d][idx] = nb_[d] / den - gr[d] * corr;
        // chemical potential mu = (6 sigma/eps) psi'(phi) - 6 sigma eps lap(phi)
        phib += (sh / ph.eps) * d2psi(pc) * mub;
        s_sig += mub * ((6.0 / ph.eps) * dpsi(pc) - 6.0 * ph.eps * lap);
        io.mubar[idx] = mub;
        // density and viscosity through clip(phi)
        const double dc = dclip(pc), cl = clip01(pc);
        phib += dc * (ph.drho * rhob + ph.dmu * etab);
        s_rin += cl * rhob;
        s_rout += (1.0 - cl) * rhob;
        s_min += cl * etab;
        s_mout += (1.0 - cl) * etab;
        io.phibar_tmp[idx] = phib;
    });
    double v[5] = {s_sig, s_rin, s_rout, s_min, s_mout};
    reduce_into<5>(v, rb, io.acc);
}

// phi-bar = partial + (central gradient)^T g-bar - 6 sigma eps lap(mu-bar)
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_adj_cells2(Dims g, Phys ph, AdjRhsIO io) {
    const double inv2h = g.i2h, inv_h2 = g.ih2;
    const double c_lap = 6.0 * ph.sigma * ph.eps;
    for_cells(g, [&](int ci, int cj, int ck, int idx) {
        Cell c{ci, cj, ck};
        Nbr<DIM> nb(c, g);
        double v = io.phibar_tmp[idx];
        const double mc = io.mubar[idx];
        double lapm = 0.0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const int ip = nb.ax(d, 1), im = nb.ax(d, -1);
            v += (io.gbar[d][im] - io.gbar[d][ip]) * inv2h;
            lapm += (io.mubar[ip] - 2.0 * mc + io.mubar[im]) * inv_h2;
        }
        io.phibar[idx] = v - c_lap * lapm;
    });
}

// velocity cotangent on the d-face of cell c: advection (central, transverse
// velocity from four faces) and viscous stress transposes, added to the
// phase-field part already in ubar
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_adj_vel(Dims g, Phys ph, AdjRhsIO io) {
    const double inv_h = g.ih, inv2h = g.i2h;
    for_cells(g, [&](int ci, int cj, int ck, int idx) {
        Cell c{ci, cj, ck};
        Nbr<DIM> nb(c, g);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const double* ud = io.u[d];
            const double* bd = io.kbar_u[d];
            const int ip = nb.ax(d, 1), im = nb.ax(d, -1);
            // A = -b is the cotangent of adv
            double r = 0.0;
            // own equation, e = d: adv_d = u_d (u_d(+d) - u_d(-d)) / 2h
            r += -bd[idx] * (ud[ip] - ud[im]) * inv2h;
            r += (-bd[im] * ud[im] + bd[ip] * ud[ip]) * inv2h;
            // viscous diagonal: tau_dd(c) = 2 eta_c (u_d(c+d) - u_d(c)) / h
            const double tb_c = (io.W[d][idx] - io.W[d][ip]) * inv_h;
            const double tb_m = (io.W[d][im] - io.W[d][idx]) * inv_h;
            r += 2.0 * (tb_m * eta_c(io.phi[im], ph) - tb_c * eta_c(io.phi[idx], ph)) * inv_h;
#pragma unroll
            for (int e = 0; e < DIM; ++e) {
                if (e == d) continue;
                const double* ue = io.u[e];
                const double* be = io.kbar_u[e];
                // own equation, transverse e: u_d(c) enters the central difference
                // along e at faces c - e and c + e, with vel_de = mean of 4 e-faces
                {
                    const int jm = nb.ax(e, -1), jp = nb.ax(e, 1);
                    // vel_de(j) = (u_e(j) + u_e(j+e) + u_e(j-d) + u_e(j-d+e)) / 4
                    const double velm = 0.25 * (ue[jm] + ue[idx] + ue[off(nb, e, -1, d, -1)] +
                                                ue[nb.ax(d, -1)]);
                    const double velp = 0.25 * (ue[jp] + ue[off(nb, e, 2, d, 0)] +
                                                ue[off(nb, e, 1, d, -1)] + ue[off(nb, e, 2, d, -1)]);
                    r += (-bd[jm] * velm + bd[jp] * velp) * inv2h;
                }
                // equation e, transverse d: vel_ed(j) = (u_d(j) + u_d(j+d) + u_d(j-e)
                // + u_d(j-e+d)) / 4 at e-faces j = c, c - d, c + e, c + e - d, times
                // the central difference of u_e along d
                {
                    auto vbar = [&](int j_e, int j_d) {
                        const int j = off(nb, e, j_e, d, j_d);
                        const int jp_ = off(nb, e, j_e, d, j_d + 1);
                        const int jm_ = off(nb, e, j_e, d, j_d - 1);
                        return -be[j] * (ue[jp_] - ue[jm_]) * inv2h;
                    };
                    r += 0.25 * (vbar(0, 0) + vbar(0, -1) + vbar(1, 0) + vbar(1, -1));
                }
                // viscous edges: u_d(c) enters the strain of edges c and c + e
                {
                    const double* te = io.te[pidx(d, e)];
                    auto eta_edge = [&](int j_e) {   // edge c + j_e e_e: cells j, j-d, j-e, j-d-e
                        return 0.25 * (eta_c(io.phi[off(nb, e, j_e, d, 0)], ph) +
                                       eta_c(io.phi[off(nb, e, j_e, d, -1)], ph) +
                                       eta_c(io.phi[off(nb, e, j_e - 1, d, 0)], ph) +
                                       eta_c(io.phi[off(nb, e, j_e - 1, d, -1)], ph));
                    };
                    r += (te[idx] * eta_edge(0) - te[nb.ax(e, 1)] * eta_edge(1)) * inv_h;
                }
            }
            io.ubar[d][idx] += r;
        }
    });
}

// ---------------------------------------------------------------------------
// projection transpose, second half: mu = lam + G w (w = A^+ D(beta lam)) on
// the faces, and the density part of the transpose,
//   rho-bar_c = (tau / 2) sum over the faces f of c of mu_f beta_f^2 (G p)_f,
// added to phi-bar through clip(phi) and to the rho_in / rho_out sums.
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_adj_proj_post(Dims g, Phys ph, AdjProjIO io, RedBuf rb) {
    const double inv_h = g.ih;
    double s_rin = 0.0, s_rout = 0.0;
    for_cells(g, [&](int ci, int cj, int ck, int idx) {
        Cell c{ci, cj, ck};
        Nbr<DIM> nb(c, g);
        const double pc = io.phi[idx];
        const double wc = io.w[idx], prc = io.p[idx];
        double rb_ = 0.0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const int im = nb.ax(d, -1), ip = nb.ax(d, 1);
            const double mu_lo = io.lam[d][idx] + (wc - io.w[im]) * inv_h;
            const double mu_hi = io.lam[d][ip] + (io.w[ip] - wc) * inv_h;
            io.mu[d][idx] = mu_lo;
            const double b_lo = beta_f(pc, io.phi[im], ph);
            const double b_hi = beta_f(io.phi[ip], pc, ph);
            rb_ += mu_lo * b_lo * b_lo * (prc - io.p[im]) * inv_h;
            rb_ += mu_hi * b_hi * b_hi * (io.p[ip] - prc) * inv_h;
        }
        rb_ *= 0.5 * io.tau;
        io.phibar[idx] += dclip(pc) * ph.drho * rb_;
        const double cl = clip01(pc);
        s_rin += cl * rb_;
        s_rout += (1.0 - cl) * rb_;
    });
    double v[2] = {s_rin, s_rout};
    reduce_into<2>(v, rb, io.acc + 1);
}

// v_d = beta_d lam_d on the faces (the right-hand side of the transposed solve
// is D v)
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_adj_beta_lam(Dims g, Phys ph, AdjProjIO io) {
    for_cells(g, [&](int ci, int cj, int ck, int idx) {
        Cell c{ci, cj, ck};
        Nbr<DIM> nb(c, g);
        const double pc = io.phi[idx];
#pragma unroll
        for (int d = 0; d < DIM; ++d)
            io.v[d][idx] = beta_f(pc, io.phi[nb.ax(d, -1)], ph) * io.lam[d][idx];
    });
}

// ---------------------------------------------------------------------------
// objective J = w_ke KE + (w_shape / 2) sum (phi - phi_target)^2 dV with
// KE = sum over faces of rho_f u^2 / 2 dV, its gradient with respect to
// (phi, u), and its rho_in / rho_out derivatives (added to acc[1], acc[2])
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_objective(Dims g, Phys ph, const double* __restrict__ phi, const double* const* u,
            const double* __restrict__ target, double w_ke, double w_shape, double dV,
            double* __restrict__ gphi, double* const* gu, RedBuf rb, double* J, double* acc) {
    double s_ke = 0.0, s_m = 0.0, s_rin = 0.0, s_rout = 0.0;
    for_cells(g, [&](int ci, int cj, int ck, int idx) {
        Cell c{ci, cj, ck};
        Nbr<DIM> nb(c, g);
        const double pc = phi[idx];
        double q = 0.0;   // sum over the faces of c of u^2 / 4 (d rho_f / d rho_c = 1/2)
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const int im = nb.ax(d, -1), ip = nb.ax(d, 1);
            const double ul = u[d][idx], uh = u[d][ip];
            const double rf = 0.5 * (rho_c(pc, ph) + rho_c(phi[im], ph));
            s_ke += 0.5 * rf * ul * ul;
            gu[d][idx] = w_ke * rf * ul * dV;
            q += 0.25 * (ul * ul + uh * uh);
        }
        const double diff = target ? pc - target[idx] : 0.0;
        s_m += 0.5 * diff * diff;
        gphi[idx] = (w_ke * dclip(pc) * ph.drho * q + w_shape * diff) * dV;
        const double cl = clip01(pc);
        s_rin += w_ke * cl * q * dV;
        s_rout += w_ke * (1.0 - cl) * q * dV;
    });
    double v[4] = {s_ke, s_m, s_rin, s_rout}, tot[4];
    const int mode[4] = {0, 0, 0, 0};
    if (grid_reduce<4>(v, mode, rb, tot) && threadIdx.x == 0) {
        *J = (w_ke * tot[0] + w_shape * tot[1]) * dV;
        acc[1] += tot[2];
        acc[2] += tot[3];
    }
}

// Gamma = max(gamma_min, max |u^n|): the Gamma cotangent acc[5] goes to the
// first face (lowest linear index over d, then cells) that attains the max,
// with the sign of u there, when the max exceeds gamma_min.
template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_adj_gamma(Dims g, const double* const* u, const double* gamma, double gamma_min,
            const double* acc, double* const* lam_u, RedBuf rb) {
    const double gm = *gamma;
    double best = -1.0e308;   // max of -(linear index)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.ncell; i += gridDim.x * blockDim.x) {
#pragma unroll
        for (int d = 0; d < DIM; ++d)
            if (fabs(u[d][i]) == gm) best = fmax(best, -(double)((long long)d * g.ncell + i));
    }
    double v[1] = {best}, tot[1];
    const int mode[1] = {1};
    if (grid_reduce<1>(v, mode, rb, tot) && threadIdx.x == 0) {
        if (gm > gamma_min && tot[0] > -1.0e307) {
            const long long lin = (long long)(-tot[0]);
            const int d = (int)(lin / g.ncell), i = (int)(lin - (long long)d * g.ncell);
            const double s = u[d][i] > 0.0 ? 1.0 : (u[d][i] < 0.0 ? -1.0 : 0.0);
            lam_u[d][i] += s * acc[5];
        }
    }
}

// out = alpha x + beta y (y may be null)
__global__ void k_axpby(int n, double alpha, const double* __restrict__ x, double beta,
                        const double* __restrict__ y, double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = alpha * x[i] + (y ? beta * y[i] : 0.0);
}

// y += x
__global__ void k_addto(int n, const double* __restrict__ x, double* __restrict__ y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] += x[i];
}

// dst[0..k) += src[0..k)
__global__ void k_add_small(int k, const double* __restrict__ src, double* __restrict__ dst) {
    if (threadIdx.x < k) dst[threadIdx.x] += src[threadIdx.x];
}

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------
template <int DIM>
void launch_adj_rhs(const Dims& g, const Phys& ph, const AdjRhsIO& io, RedBuf rb, cudaStream_t s) {
    const int gr = row_grid(g, kThreads, kRedBlocks);
    const int gl = row_grid(g, kThreads, 1 << 30);
    k_adj_faces<DIM><<<gr, kThreads, 0, s>>>(g, ph, io, rb);
    if (DIM > 1) k_adj_edges<DIM><<<gl, kThreads, 0, s>>>(g, io);
    k_adj_cells<DIM><<<gr, kThreads, 0, s>>>(g, ph, io, rb);
    k_adj_cells2<DIM><<<gl, kThreads, 0, s>>>(g, ph, io);
    k_adj_vel<DIM><<<gl, kThreads, 0, s>>>(g, ph, io);
}

template <int DIM>
void launch_adj_beta_lam(const Dims& g, const Phys& ph, const AdjProjIO& io, cudaStream_t s) {
    k_adj_beta_lam<DIM><<<row_grid(g, kThreads, 1 << 30), kThreads, 0, s>>>(g, ph, io);
}

template <int DIM>
void launch_adj_proj_post(const Dims& g, const Phys& ph, const AdjProjIO& io, RedBuf rb,
                          cudaStream_t s) {
    k_adj_proj_post<DIM><<<row_grid(g, kThreads, kRedBlocks), kThreads, 0, s>>>(g, ph, io, rb);
}

template <int DIM>
void launch_objective(const Dims& g, const Phys& ph, const double* phi, const double* const* u,
                      const double* target, double w_ke, double w_shape, double* gphi,
                      double* const* gu, RedBuf rb, double* J, double* acc, cudaStream_t s) {
    double dV = 1.0;
    for (int d = 0; d < DIM; ++d) dV *= g.h;
    k_objective<DIM><<<row_grid(g, kThreads, kRedBlocks), kThreads, 0, s>>>(
        g, ph, phi, u, target, w_ke, w_shape, dV, gphi, gu, rb, J, acc);
}

template <int DIM>
void launch_adj_gamma(const Dims& g, const double* const* u, const double* gamma, double gamma_min,
                      const double* acc, double* const* lam_u, RedBuf rb, cudaStream_t s) {
    k_adj_gamma<DIM><<<red_grid(g.ncell), kThreads, 0, s>>>(g, u, gamma, gamma_min, acc, lam_u, rb);
}

void launch_axpby(int n, double alpha, const double* x, double beta, const double* y, double* out,
                  cudaStream_t s) {
    k_axpby<<<red_grid(n), kThreads, 0, s>>>(n, alpha, x, beta, y, out);
}
void launch_addto(int n, const double* x, double* y, cudaStream_t s) {
    k_addto<<<red_grid(n), kThreads, 0, s>>>(n, x, y);
}
void launch_add_small(int k, const double* src, double* dst, cudaStream_t s) {
    k_add_small<<<1, 32, 0, s>>>(k, src, dst);
}

#define PF_INST_ADJ(D)                                                                           \
    template void launch_adj_rhs<D>(const Dims&, const Phys&, const AdjRhsIO&, RedBuf,           \
                                    cudaStream_t);                                               \
    template void launch_adj_beta_lam<D>(const Dims&, const Phys&, const AdjProjIO&,             \
                                         cudaStream_t);                                          \
    template void launch_adj_proj_post<D>(const Dims&, const Phys&, const AdjProjIO&, RedBuf,    \
                                          cudaStream_t);                                         \
    template void launch_objective<D>(const Dims&, const Phys&, const double*,                   \
                                      const double* const*, const double*, double, double,       \
                                      double*, double* const*, RedBuf, double*, double*,         \
                                      cudaStream_t);                                             \
    template void launch_adj_gamma<D>(const Dims&, const double* const*, const double*, double,  \
                                      const double*, double* const*, RedBuf, cudaStream_t);

PF_INST_ADJ(2)
PF_INST_ADJ(3)

}  // namespace pf
