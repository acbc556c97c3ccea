// One full red-black Gauss-Seidel sweep of a 3D float32 multigrid level in a
// single pass over memory (out of place: x_in -> x_out).
//
// A CTA owns a 32 x 8 column tile and marches along z. Each plane of x_in, f
// and the coefficient source (rho(phi) on the finest level, the three face
// coefficient arrays on coarser ones) is copied with a two-cell halo into
// shared-memory rings by cp.async two planes ahead of its use, so global
// latency overlaps the arithmetic. In the step for plane k the first three
// warps update the first colour on plane k over the tile plus a one-cell ring
// (its x_in neighbours are all of the other colour) and the last two warps
// update the second colour of plane k - 2 from the new first-colour values of
// planes k - 3 .. k - 1 and write both colours of plane k - 2, two cells per
// thread: one barrier per plane. The halo ring is recomputed by both
// neighbouring CTAs, so no CTA reads another's output. Zero start (x_in = 0)
// skips the x_in copies.
//
// The smoother solves each cell's row of sum_q w_q (x_c - x_q) = f h^2 / s
// with unscaled weights (w_q = 1 / (rho_c + rho_q), s = 2, on the finest
// level; the level's face coefficients, s = 1, below) and approximate
// reciprocals: it is a preconditioner inside flexible CG, and the operator
// itself (CG product, float64 residual) uses the exact coefficients.
// Requires even nx, ny, nz (consistent periodic colouring); tiles may be
// ragged (sizes need not be multiples of 32 x 8) since every index wraps.
// Rows of the finest level are copied in 16-byte chunks when nx is a multiple
// of 4, else (and on coarser levels) in 8-byte chunks.
#include <cstddef>
#include <mutex>

#include "pf_device.cuh"

namespace pf {

namespace {

constexpr int TX = 32, TY = 8;              // tile (columns per CTA)
constexpr int HY = TY + 4;                  // rows j0-2 .. j0+TY+1 of a halo-2 plane
constexpr int RXS = TX + 2, RYS = TY + 2;   // halo-1 plane (first-colour values)
constexpr int N1 = (RXS / 2) * RYS;         // first-colour cells per plane (170)
constexpr int N2 = (TX / 2) * TY;           // second-colour cells per plane (128)
constexpr int W1 = 96;                      // first-colour threads (3 warps, 2 cells each)
constexpr int W2 = N2 / 2;                  // second-colour threads (2 warps, 2 cells each)
constexpr int NT = W1 + W2;                 // 160 threads

// halo-2 plane geometry for copy chunks of V floats: shared-memory column a
// holds global column i0 - OX + a
template <int V>
struct Geo {
    static constexpr int OX = V == 4 ? 4 : 2;
    static constexpr int HX = TX + 2 * OX;  // 40 or 36
    static constexpr int CPR = HX / V;      // chunks per row
    static constexpr int NCH = CPR * HY;    // chunks per plane (120 or 216)
};

__device__ __forceinline__ int mod(int a, int m) { int r = a % m; return r < 0 ? r + m : r; }

template <int B>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(B)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
// ring slot of plane kp (kp >= -8)
template <int R>
__device__ __forceinline__ int slot(int kp) { return (int)((unsigned)(kp + 8 * R) % (unsigned)R); }
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct SweepArgs {
    Dims g;
    const float* xin;     // nullptr: zero start
    const float* f;
    float* xout;
    const float* phi;     // finest level: coefficients from rho(phi)
    const float* bx;      // coarser levels: face coefficient arrays
    const float* by;
    const float* bz;
    Phys ph;
    int rho_ready;        // phi already holds rho32(phi)
    float fs;             // f scale: h^2 / 2 (from phi) or h^2 (face arrays)
    int first_color;
    int zc;
    int dots;             // also r.z and z.q (see SweepDots)
    int first;
    const float* q;
    RedBuf rb;
    CGScalars* scw;
};

// Copies run PD planes ahead. Rings (planes): x_in 3 + PD, f 4 + PD, rho 5 + PD
// or 4 + PD per face array, new first-colour values 4.
constexpr int PD = 2;
constexpr int RX_ = 3 + PD, RF_ = 4 + PD, RR_ = 5 + PD, RB_ = 4 + PD, RN_ = 4;
template <bool FROM_PHI, int V>
struct Smem {
    static constexpr int HX = Geo<V>::HX;
    float f[RF_][HY][HX];
    float c[FROM_PHI ? RR_ : 3 * RB_][HY][HX];
    float n[RN_][RYS][RXS / 2];   // first-colour values only, (a1 >> 1) per row
    float x[RX_][HY][HX];         // last: a zero-start launch leaves it out
};

// plane offset o (floats) of a ring of R planes of P floats, moved by d planes
template <int R, int P>
__device__ __forceinline__ int ring(int o, int d) {
    o += d * P;
    o += o < 0 ? R * P : 0;
    return o >= R * P ? o - R * P : o;
}
template <bool FROM_PHI, int V>
__device__ __forceinline__ void sweep3d_body(const SweepArgs& A, unsigned char* smem_raw) {
    using G = Geo<V>;
    constexpr int HX = G::HX, OX = G::OX;
    constexpr int PLANE = HY * HX;   // floats per halo-2 plane
    constexpr int RXH = RXS / 2;     // first-colour cells per halo-1 row
    constexpr int NPL = RYS * RXH;   // floats per first-colour plane
    constexpr int RC = FROM_PHI ? RR_ : RB_;
    constexpr int CH = (G::NCH + NT - 1) / NT;   // copy chunks per thread
    Smem<FROM_PHI, V>& S = *reinterpret_cast<Smem<FROM_PHI, V>*>(smem_raw);
    float* const Xs = &S.x[0][0][0];
    float* const Fs = &S.f[0][0][0];
    float* const Cs = &S.c[0][0][0];
    float* const Ns = &S.n[0][0][0];
    float rz = 0.f, zq = 0.f;   // per-thread partial dots (A.dots)
    const int first_it = A.dots ? first_of(A.first, A.scw) : 1;

    const Dims& g = A.g;
    const int tid = threadIdx.x;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * A.zc;
    const int z1 = min(z0 + A.zc, g.nz);
    const int sy = g.nx, sz = g.nx * g.ny;
    const int c0 = A.first_color;
    const bool zero = A.xin == nullptr;
    const float ro = A.ph.rho_out_f, dr = A.ph.drho_f;
    const float fs = A.fs;

    // this thread's copy chunks of a halo-2 plane (fixed across planes)
    int so[CH], poff[CH];
    bool has[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        const int lid = tid + c * NT;
        has[c] = lid < G::NCH;
        const int pb = lid / G::CPR, pa = V * (lid - pb * G::CPR);
        poff[c] = mod(j0 - 2 + pb, g.ny) * sy + mod(i0 - OX + pa, g.nx);
        so[c] = pb * HX + pa;
    }
    // next plane to copy: index, global plane base and ring plane offsets
    int kiss = z0 - 2;
    int gz = mod(kiss, g.nz) * sz;
    int ix = slot<RX_>(kiss) * PLANE, iff = slot<RF_>(kiss) * PLANE, ic = slot<RC>(kiss) * PLANE;

    auto issue = [&]() {
        if (kiss <= z1 + 1) {
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                if (!has[c]) continue;
                const int gidx = gz + poff[c];
                if (!zero) cp_async<4 * V>(Xs + ix + so[c], A.xin + gidx);
                cp_async<4 * V>(Fs + iff + so[c], A.f + gidx);
                if (FROM_PHI) {
                    cp_async<4 * V>(Cs + ic + so[c], A.phi + gidx);
                } else {
                    cp_async<4 * V>(Cs + ic + so[c], A.bx + gidx);
                    cp_async<4 * V>(Cs + RB_ * PLANE + ic + so[c], A.by + gidx);
                    cp_async<4 * V>(Cs + 2 * RB_ * PLANE + ic + so[c], A.bz + gidx);
                }
            }
        }
        cp_commit();
        ++kiss;
        gz += sz;
        if (gz >= g.ncell) gz -= g.ncell;
        ix = ring<RX_, PLANE>(ix, 1);
        iff = ring<RF_, PLANE>(iff, 1);
        ic = ring<RC, PLANE>(ic, 1);
    };
    // rho(phi) in place for this thread's own chunks of the plane at ring
    // offset o (after their copies landed)
    auto transform = [&](int o, bool used) {
        if (FROM_PHI && used && !A.rho_ready) {
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                if (!has[c]) continue;
                float* cp = Cs + o + so[c];
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    const float v = fminf(fmaxf(cp[e], 0.f), 1.f);
                    cp[e] = __fadd_rn(ro, __fmul_rn(dr, v));
                }
            }
        }
    };
    // weights -x, +x, -y, +y, -z, +z of the cell at offset co of the plane at
    // coefficient ring offset o (om, op: the planes below and above)
    auto weights = [&](int co, int o, int om, int op, float (&w)[6]) {
        if (FROM_PHI) {
            const float* cc = Cs + o + co;
            const float rc = cc[0];
            w[0] = rcp_approx(rc + cc[-1]);
            w[1] = rcp_approx(rc + cc[1]);
            w[2] = rcp_approx(rc + cc[-HX]);
            w[3] = rcp_approx(rc + cc[HX]);
            w[4] = rcp_approx(rc + Cs[om + co]);
            w[5] = rcp_approx(rc + Cs[op + co]);
        } else {
            const float* cx = Cs + o + co;
            const float* cy = cx + RB_ * PLANE;
            w[0] = cx[0];
            w[1] = cx[1];
            w[2] = cy[0];
            w[3] = cy[HX];
            w[4] = cx[2 * RB_ * PLANE];
            w[5] = Cs[2 * RB_ * PLANE + op + co];
        }
    };

    // fixed per-thread cell offsets (two cells per thread): first colour on
    // halo-1 cells u = tid, tid + W1 (row u / 17, pair u % 17); second colour on
    // tile cells t, t + W2 (row t / 16, pair t % 16); each cell's colour parity
    // flips from plane to plane
    const bool first_grp = tid < W1;
    int co[2], cn[2], par[2], g2[2];
    bool act[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (first_grp) {
            const int u = tid + h * W1;
            act[h] = u < N1;
            const int b1 = u / RXH, m = u - b1 * RXH;
            co[h] = (b1 + 1) * HX + 2 * m + OX - 1;
            cn[h] = b1 * RXH + m;
            par[h] = (c0 + b1 + z0 - 1) & 1;
            g2[h] = 0;
        } else {
            const int t = tid - W1 + h * W2;
            const int tb = t >> 4, m = t & 15;
            act[h] = (j0 + tb < g.ny) && (i0 + 2 * m < g.nx);
            co[h] = (tb + 2) * HX + 2 * m + OX;
            cn[h] = (tb + 1) * RXH + m;
            par[h] = (c0 + 1 + tb + z0 - 3) & 1;
            g2[h] = (z0 - 3) * sz + (j0 + tb) * sy + i0 + 2 * m;   // output of plane kb
        }
    }
    // q of the second-colour cells (fused dots), loaded one plane ahead
    const bool want_q = A.dots && !first_it && !first_grp;
    float2 qv[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    if (want_q && z0 < z1) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (act[h]) qv[h] = __ldg(reinterpret_cast<const float2*>(A.q + g2[h] + 3 * sz));
    }

    // prologue: planes z0-2, z0-1 landed; z0 .. z0+PD-1 in flight
    const int c_lo = slot<RC>(z0 - 2) * PLANE;
    issue();
    issue();
    cp_wait_all();
    transform(c_lo, true);
    transform(ring<RC, PLANE>(c_lo, 1), true);
    for (int q = 0; q < PD; ++q) issue();
    // ring plane offsets of plane kr
    int ox = slot<RX_>(z0 - 1) * PLANE, of = slot<RF_>(z0 - 1) * PLANE;
    int oc = slot<RC>(z0 - 1) * PLANE, on = slot<RN_>(z0 - 1) * NPL;
    // step kr: first colour on plane kr (kr <= z1), second colour on kb = kr - 2
    for (int kr = z0 - 1; kr <= z1 + 1; ++kr) {
        cp_wait<PD - 1>();      // own copies of plane kr + 1 have landed
        const int ocp = ring<RC, PLANE>(oc, 1);
        transform(ocp, kr + 1 <= z1 + 1);
        __syncthreads();        // every copy of plane kr + 1 visible; step kr - 1 done
        issue();                // plane kr + 1 + PD; overlaps with the next PD steps
        if (first_grp) {
            if (kr <= z1) {
                const int ocm = ring<RC, PLANE>(oc, -1);
                const int oxm = ring<RX_, PLANE>(ox, -1), oxp = ring<RX_, PLANE>(ox, 1);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (!act[h]) continue;
                    const int c = co[h] + par[h];
                    float w[6];
                    weights(c, oc, ocm, ocp, w);
                    const float diag = w[0] + w[1] + w[2] + w[3] + w[4] + w[5];
                    float num = Fs[of + c] * fs;
                    if (!zero) {
                        const float* xc = Xs + ox + c;
                        num += w[0] * xc[-1] + w[1] * xc[1] + w[2] * xc[-HX] + w[3] * xc[HX] +
                               w[4] * Xs[oxm + c] + w[5] * Xs[oxp + c];
                    }
                    Ns[on + cn[h]] = num * rcp_approx(diag);
                }
            }
        } else {
            const int kb = kr - 2;
            if (kb >= z0 && kb < z1) {
                const int onb = ring<RN_, NPL>(on, -2), onm = ring<RN_, NPL>(on, -3),
                          onp = ring<RN_, NPL>(on, -1);
                const int ofb = ring<RF_, PLANE>(of, -2);
                const int ocb = ring<RC, PLANE>(oc, -2), ocbm = ring<RC, PLANE>(oc, -3),
                          ocbp = ring<RC, PLANE>(oc, -1);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int s2 = par[h];
                    const int c = co[h] + s2;
                    float w[6];
                    weights(c, ocb, ocbm, ocbp, w);
                    const float diag = w[0] + w[1] + w[2] + w[3] + w[4] + w[5];
                    // first-colour neighbours: x at (a1 -+ 1) >> 1, the rest at a1 >> 1
                    const float* nc = Ns + onb + cn[h];
                    const float num = Fs[ofb + c] * fs + w[0] * nc[0] + w[1] * nc[1] +
                                      w[2] * nc[s2 - RXH] + w[3] * nc[s2 + RXH] +
                                      w[4] * Ns[onm + cn[h] + s2] + w[5] * Ns[onp + cn[h] + s2];
                    const float v2 = num * rcp_approx(diag);
                    // the pair (2 m, 2 m + 1) of this row holds one cell of each colour
                    const float other = nc[1 - s2];
                    const float v_even = s2 == 0 ? v2 : other;
                    const float v_odd = s2 == 1 ? v2 : other;
                    if (act[h]) {
                        *reinterpret_cast<float2*>(A.xout + g2[h]) = make_float2(v_even, v_odd);
                        if (A.dots) {
                            rz += Fs[ofb + co[h]] * v_even + Fs[ofb + co[h] + 1] * v_odd;
                            if (want_q) {
                                zq += v_even * qv[h].x + v_odd * qv[h].y;
                                if (kb + 1 < z1)
                                    qv[h] = __ldg(
                                        reinterpret_cast<const float2*>(A.q + g2[h] + sz));
                            }
                        }
                    }
                }
            }
        }
        ox = ring<RX_, PLANE>(ox, 1);
        of = ring<RF_, PLANE>(of, 1);
        oc = ocp;
        on = ring<RN_, NPL>(on, 1);
        par[0] ^= 1;
        par[1] ^= 1;
        g2[0] += sz;
        g2[1] += sz;
    }
    cp_wait_all();
    if (A.dots) {
        double v[2] = {double(rz), double(zq)}, tot[2];
        const int mode[2] = {0, 0};
        const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        const int nb = gridDim.x * gridDim.y * gridDim.z;
        if (grid_reduce_lin<2>(v, mode, A.rb, tot, bid, nb) && threadIdx.x == 0) {
            CGScalars* sc = A.scw;
            sc->beta = first_it ? 0.0 : -sc->alpha * tot[1] / sc->rz;
            sc->rz = tot[0];
        }
    }
}

// finest level (coefficients from phi) and coarser levels (face arrays), in
// 16-byte (V = 4) or 8-byte (V = 2) copy chunks
template <bool FROM_PHI, int V>
__global__ void __launch_bounds__(NT, FROM_PHI ? 6 : 4) k_sweep3d(SweepArgs A, const CGScalars* sc) {
    if (sc && (sc->done || sc->idone)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    sweep3d_body<FROM_PHI, V>(A, smem_raw);
}

// dynamic shared memory beyond 48 KB, and a shared-memory carveout that lets
// several CTAs share an SM (once per process)
template <bool FROM_PHI, int V>
void sweep3d_attributes() {
    static std::once_flag attr_once;
    std::call_once(attr_once, [] {
        cudaFuncSetAttribute(k_sweep3d<FROM_PHI, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(Smem<FROM_PHI, V>));
        cudaFuncSetAttribute(k_sweep3d<FROM_PHI, V>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    });
}

template <bool FROM_PHI, int V>
void launch_sweep3d_t(const SweepArgs& a, dim3 grid, const CGScalars* sc, cudaStream_t s) {
    // a zero-start sweep copies no x_in: its launch leaves out the x ring
    using SM = Smem<FROM_PHI, V>;
    const size_t bytes = a.xin == nullptr ? offsetof(SM, x) : sizeof(SM);
    sweep3d_attributes<FROM_PHI, V>();
    k_sweep3d<FROM_PHI, V><<<grid, NT, bytes, s>>>(a, sc);
}

}  // namespace

// z chunk of the tiled kernels: enough CTAs to fill the GPU (about 8 per SM),
// 2..32 planes each
int tiled_zc(const Dims& g) {
    const int cols = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    int zc = 32;
    while (zc > 2 && (long long)cols * ((g.nz + zc - 1) / zc) < 8 * 152) zc >>= 1;
    return zc;
}

long long sweep3d_blocks(const Dims& g) {
    const int zc = tiled_zc(g);
    return (long long)((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY) * ((g.nz + zc - 1) / zc);
}

void sweep3d_prepare() {
    sweep3d_attributes<true, 4>();
    sweep3d_attributes<true, 2>();
    sweep3d_attributes<false, 2>();
}

// Eligible: 3D float level with even sizes.
bool sweep3d_ok(const Dims& g) {
    return g.nz > 1 && (g.nx % 2 == 0) && (g.ny % 2 == 0) && (g.nz % 2 == 0) && g.nx >= 4 &&
           g.ny >= 4 && g.nz >= 4;
}

void launch_sweep3d(const MGLevel<float>& L, const float* phi, int rho_ready, const Phys& ph,
                    const float* xin, float* xout, const SweepDots* dots, int first_color,
                    const CGScalars* sc, cudaStream_t s) {
    SweepArgs a;
    a.g = L.g;
    a.rho_ready = rho_ready;
    a.xin = xin;
    a.f = L.f;
    a.xout = xout;
    a.phi = phi;
    a.bx = L.beta[0];
    a.by = L.beta[1];
    a.bz = L.beta[2];
    a.ph = ph;
    const bool from_phi = phi != nullptr;
    a.fs = float(from_phi ? 0.5 * L.g.h * L.g.h : L.g.h * L.g.h);
    a.first_color = first_color;
    a.dots = dots != nullptr;
    a.first = dots ? dots->first : 0;
    a.q = dots ? dots->q : nullptr;
    if (dots) {
        a.rb = dots->rb;
        a.scw = dots->sc;
    } else {
        a.rb = RedBuf{nullptr, nullptr};
        a.scw = nullptr;
    }
    // 64-plane chunks where that still gives 8 CTAs per SM (the z halo and
    // the pipeline start are paid once per chunk), else the shared choice
    int zc = tiled_zc(L.g);
    {
        const long long cols = (long long)((L.g.nx + TX - 1) / TX) * ((L.g.ny + TY - 1) / TY);
        if (zc == 32 && cols * ((L.g.nz + 63) / 64) >= 8 * 152) zc = 64;
    }
    a.zc = zc;
    dim3 grid((L.g.nx + TX - 1) / TX, (L.g.ny + TY - 1) / TY, (L.g.nz + zc - 1) / zc);
    if (dots && 2LL * grid.x * grid.y * grid.z > (long long)kRedPart) {
        // more CTAs than reduction slots: the caller runs the dot kernel instead
        a.dots = 0;
    }
    // coarser levels keep 8-byte chunks: their three coefficient rings in
    // 16-byte rows would leave room for only three CTAs per SM
    if (from_phi && L.g.nx % 4 == 0)
        launch_sweep3d_t<true, 4>(a, grid, sc, s);
    else if (from_phi)
        launch_sweep3d_t<true, 2>(a, grid, sc, s);
    else
        launch_sweep3d_t<false, 2>(a, grid, sc, s);
}

bool dir3d_ok(const Dims& g) {
    return g.nz > 1 && (g.nx % 2 == 0) && (g.ny % 2 == 0) && g.nx >= 4 && g.ny >= 4 &&
           g.nz >= 4 && sweep3d_blocks(g) <= kRedPart;
}

}  // namespace pf

// ---------------------------------------------------------------------------
// CG search direction and operator product on 3D float32 grids:
//   p_new = z + beta p_old ; q = A' p_new ; alpha = rz / (p_new . q)
// Register z-march: one thread per column of a 32 x 8 tile; p_new of the
// column at k-1, k, k+1 and the z-face coefficient above are carried in
// registers, the in-plane neighbours come through L1. No shared memory and no
// barriers.
//
// The face coefficients come either from the three face arrays (A' = A, the
// float32 operator of the outer residual) or from the cell densities as
// 2 / (rho_c + rho_q) with the hardware reciprocal (RHO): one array instead of
// three, 8 fewer bytes per cell. The inner CG then solves with A' = A up to
// the reciprocal's rounding (about 2^-22 relative per coefficient); the
// float64 refinement around it forms every residual with A, so the converged
// pressure is that of A all the same.
// ---------------------------------------------------------------------------
namespace pf {
namespace {

struct DirRegArgs {
    Dims g;
    const float* z;
    const float* p_old;
    float* p_new;
    float* q;
    const float* bx;
    const float* by;
    const float* bz;
    const float* rho;
    float ih2;
    int first;
    int zc;
    RedBuf rb;
    CGScalars* sc;
};

__device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Fetch the 128-byte line holding p into L2 without waiting for it.
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
constexpr int kColumnAhead = 4;   // planes between an L2 prefetch and its use (column marches)

template <bool RHO>
__global__ void __launch_bounds__(256, 4) k_dir3d_reg(DirRegArgs A) {
    CGScalars* sc = A.sc;
    if (sc->done || sc->idone) return;
    const Dims& g = A.g;
    const int first_it = first_of(A.first, sc);
    const float bcg = first_it ? 0.f : float(sc->beta);
    const int i = blockIdx.x * 32 + threadIdx.x % 32;
    const int j = blockIdx.y * 8 + threadIdx.x / 32;
    const int z0 = blockIdx.z * A.zc;
    const int z1 = min(z0 + A.zc, g.nz);
    float pq = 0.f;
    if (i < g.nx && j < g.ny) {
        const int sy = g.nx, sz = g.nx * g.ny;
        const int im = i == 0 ? g.nx - 1 : i - 1, ip = i == g.nx - 1 ? 0 : i + 1;
        const int jm = j == 0 ? g.ny - 1 : j - 1, jp = j == g.ny - 1 ? 0 : j + 1;
        const int col = j * sy + i;
        const int ox_m = im - i, ox_p = ip - i, oy_m = (jm - j) * sy, oy_p = (jp - j) * sy;
        const float* __restrict__ zp = A.z;
        const float* __restrict__ po = A.p_old;
        const float* __restrict__ bxp = A.bx;
        const float* __restrict__ byp = A.by;
        const float* __restrict__ bzp = A.bz;
        const float* __restrict__ rp = A.rho;
        float* __restrict__ pnew = A.p_new;
        float* __restrict__ qo = A.q;
        const bool first = first_it != 0;
        auto pn = [&](int idx) {
            const float zv = __ldg(zp + idx);
            return first ? zv : zv + bcg * __ldg(po + idx);
        };
        const int km1 = z0 == 0 ? g.nz - 1 : z0 - 1;
        float p_m = pn(km1 * sz + col);
        float p_c = pn(z0 * sz + col);
        // z-face coefficient below plane k; RHO: also rho of plane k
        float r_c = 0.f, bz_c;
        if (RHO) {
            r_c = __ldg(rp + z0 * sz + col);
            bz_c = rcp_fast(r_c + __ldg(rp + km1 * sz + col));
        } else {
            bz_c = __ldg(bzp + z0 * sz + col);
        }
        // the loads of plane k: in-plane neighbours of p_new (as z, p_old), the
        // x / y face coefficients (RHO: the neighbours' densities), and the
        // centre of plane k + 1 with its z face (RHO: its density)
        struct Ld {
            float z[4], p[4], c[4], zn, pnx, bzn;
        };
        auto load = [&](int k, Ld& L) {
            const int idx = k * sz + col;
            const int idxp = (k + 1 == g.nz ? 0 : k + 1) * sz + col;
            const int o[4] = {idx + ox_m, idx + ox_p, idx + oy_m, idx + oy_p};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                L.z[q] = __ldg(zp + o[q]);
                L.p[q] = first ? 0.f : __ldg(po + o[q]);
            }
            if (RHO) {
#pragma unroll
                for (int q = 0; q < 4; ++q) L.c[q] = __ldg(rp + o[q]);
                L.bzn = __ldg(rp + idxp);
            } else {
                L.c[0] = __ldg(bxp + idx);
                L.c[1] = __ldg(bxp + idx + ox_p);
                L.c[2] = __ldg(byp + idx);
                L.c[3] = __ldg(byp + idx + oy_p);
                L.bzn = __ldg(bzp + idxp);
            }
            L.zn = __ldg(zp + idxp);
            L.pnx = first ? 0.f : __ldg(po + idxp);
        };
        auto apply = [&](int k, const Ld& L) {
            const int idx = k * sz + col;
            const float p_p = L.zn + bcg * L.pnx;
            float nb[4], w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) nb[q] = L.z[q] + bcg * L.p[q];
            float bz_n;
            if (RHO) {
#pragma unroll
                for (int q = 0; q < 4; ++q) w[q] = rcp_fast(r_c + L.c[q]);
                bz_n = rcp_fast(r_c + L.bzn);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) w[q] = L.c[q];
                bz_n = L.bzn;
            }
            const float ax = w[0] * (p_c - nb[0]) + w[1] * (p_c - nb[1]) + w[2] * (p_c - nb[2]) +
                             w[3] * (p_c - nb[3]) + bz_c * (p_c - p_m) + bz_n * (p_c - p_p);
            const float qv = ax * A.ih2;
            pnew[idx] = p_c;
            qo[idx] = qv;
            pq += p_c * qv;
            p_m = p_c;
            p_c = p_p;
            bz_c = bz_n;
            if (RHO) r_c = L.bzn;
        };
        // L2 prefetch of the warp's row (32 columns) of z, p_old and rho (RHO)
        // or z, p_old and the z faces, kColumnAhead planes ahead: lane l < 6
        // takes array l % 3 of plane (l / 3) of the round
        const int lane = threadIdx.x % 32;
        const int pf_arr = lane % 3, pf_dz = lane / 3;
        const float* pf_ptr = (pf_arr == 0 ? zp : pf_arr == 1 ? po : (RHO ? rp : bzp)) +
                              (j * sy + blockIdx.x * 32);
        const bool pf_on = lane < 6 && !(pf_arr == 1 && first);
        // two planes per round: all loads of both before the arithmetic
        int k = z0;
        for (; k + 1 < z1; k += 2) {
            const int kq = k + kColumnAhead + pf_dz;
            if (pf_on && kq <= z1) prefetch_l2(pf_ptr + (size_t)(kq >= g.nz ? kq - g.nz : kq) * sz);
            Ld a, b;
            load(k, a);
            load(k + 1, b);
            apply(k, a);
            apply(k + 1, b);
        }
        if (k < z1) {
            Ld a;
            load(k, a);
            apply(k, a);
        }
    }
    double v[1] = {double(pq)}, tot[1];
    const int mode[1] = {0};
    const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    if (grid_reduce_lin<1>(v, mode, A.rb, tot, bid, nb) && threadIdx.x == 0) {
        sc->pq = tot[0];
        sc->alpha = tot[0] != 0.0 ? sc->rz / tot[0] : 0.0;
    }
}

}  // namespace

void launch_dir3d_reg(const Dims& g, const float* z, const float* p_old, float* p_new, float* q,
                      const float* const* beta, const float* rho, int first, RedBuf rb,
                      CGScalars* sc, cudaStream_t s) {
    DirRegArgs a;
    a.g = g;
    a.z = z;
    a.p_old = p_old;
    a.p_new = p_new;
    a.q = q;
    a.bx = beta[0];
    a.by = beta[1];
    a.bz = beta[2];
    a.rho = rho;
    // 1/rho_f = 2 / (rho_c + rho_q): the factor 2 goes with 1/h^2
    a.ih2 = rho ? 2.f * g.ih2f : g.ih2f;
    a.first = first;
    a.rb = rb;
    a.sc = sc;
    const int zc = tiled_zc(g);
    a.zc = zc;
    dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, (g.nz + zc - 1) / zc);
    if (rho)
        k_dir3d_reg<true><<<grid, 256, 0, s>>>(a);
    else
        k_dir3d_reg<false><<<grid, 256, 0, s>>>(a);
}

}  // namespace pf

// ---------------------------------------------------------------------------
// Outer residual of the mixed 3D path, r = sign (b - mean b) - A x, with x and
// b double-floats (n hi parts, then n lo parts) and A formed from the float32
// face coefficients by a compensated double-float sum on the float32 pipe
// (df_face_term). One thread per column of a 32 x 8 tile marching in z: x of
// the column at k-1, k, k+1 and the z-face coefficient above are carried in
// registers, the in-plane neighbours come through L1.
// ---------------------------------------------------------------------------
namespace pf {
namespace {

struct IRArgs {
    Dims g;
    const float* xh;
    const float* xl;
    const float* bh;
    const float* bl;
    const float* bx;
    const float* by;
    const float* bz;
    float* r;
    double sign;
    int first;
    int zc;
    RedBuf rb;
    CGScalars* sc;
};

__global__ void __launch_bounds__(256, 6) k_ir_residual3d(IRArgs A) {
    CGScalars* sc = A.sc;
    if (!A.first && sc->done) return;
    const Dims& g = A.g;
    const int i = blockIdx.x * 32 + threadIdx.x % 32;
    const int j = blockIdx.y * 8 + threadIdx.x / 32;
    const int z0 = blockIdx.z * A.zc;
    const int z1 = min(z0 + A.zc, g.nz);
    float ff = 0.f, rr = 0.f;
    if (i < g.nx && j < g.ny) {
        const int sy = g.nx, sz = g.nx * g.ny;
        const int im = i == 0 ? g.nx - 1 : i - 1, ip = i == g.nx - 1 ? 0 : i + 1;
        const int jm = j == 0 ? g.ny - 1 : j - 1, jp = j == g.ny - 1 ? 0 : j + 1;
        const int col = j * sy + i;
        const int o[4] = {im - i, ip - i, (jm - j) * sy, (jp - j) * sy};
        const float* __restrict__ xh = A.xh;
        const float* __restrict__ xl = A.xl;
        const f2 mdf = df_neg(df_of(sc->mean_b));
        const f2 ih2 = df_of(g.ih2);
        const bool pos = A.sign > 0.0;
        const int km1 = z0 == 0 ? g.nz - 1 : z0 - 1;
        float mh = __ldg(xh + km1 * sz + col), ml = __ldg(xl + km1 * sz + col);
        float ch = __ldg(xh + z0 * sz + col), cl = __ldg(xl + z0 * sz + col);
        float bz_c = __ldg(A.bz + z0 * sz + col);
        // the loads of plane k: in-plane neighbours, face coefficients, the
        // column's next plane and the right-hand side
        struct Ld {
            float nh[4], nl[4], w[4], ph, pl, bzn, bh, bl;
        };
        auto load = [&](int k, Ld& L) {
            const int idx = k * sz + col;
            const int idxp = (k + 1 == g.nz ? 0 : k + 1) * sz + col;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                L.nh[q] = __ldg(xh + idx + o[q]);
                L.nl[q] = __ldg(xl + idx + o[q]);
            }
            L.w[0] = __ldg(A.bx + idx);
            L.w[1] = __ldg(A.bx + idx + o[1]);
            L.w[2] = __ldg(A.by + idx);
            L.w[3] = __ldg(A.by + idx + o[3]);
            L.ph = __ldg(xh + idxp);
            L.pl = __ldg(xl + idxp);
            L.bzn = __ldg(A.bz + idxp);
            L.bh = __ldg(A.bh + idx);
            L.bl = __ldg(A.bl + idx);
        };
        auto apply = [&](int k, const Ld& L) {
            const int idx = k * sz + col;
            f2 f = df_add(f2{L.bh, L.bl}, mdf);
            if (!pos) f = df_neg(f);
            float S = 0.f, c = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) df_face_term(L.w[q], ch, cl, L.nh[q], L.nl[q], S, c);
            df_face_term(bz_c, ch, cl, mh, ml, S, c);
            df_face_term(L.bzn, ch, cl, L.ph, L.pl, S, c);
            const f2 ax = f2_mul(two_sum(S, c), ih2);
            const f2 rv = df_add(f, df_neg(ax));
            const float rt = __fadd_rn(rv.hi, rv.lo);
            A.r[idx] = rt;
            if (A.first) {
                const float ft = __fadd_rn(f.hi, f.lo);
                ff += ft * ft;
            }
            rr += rt * rt;
            mh = ch;
            ml = cl;
            ch = L.ph;
            cl = L.pl;
            bz_c = L.bzn;
        };
        // two planes per round: all loads of both before the arithmetic (an L2
        // prefetch of later planes, as in the direction kernel, measured
        // slower here: the registers it takes cost resident CTAs)
        int k = z0;
        for (; k + 1 < z1; k += 2) {
            Ld a, b;
            load(k, a);
            load(k + 1, b);
            apply(k, a);
            apply(k + 1, b);
        }
        if (k < z1) {
            Ld a;
            load(k, a);
            apply(k, a);
        }
    }
    double v[3] = {double(ff), double(rr), double(rr)}, tot[3];
    const int mode[3] = {0, 0, 0};
    const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    if (grid_reduce_lin<3>(v, mode, A.rb, tot, bid, nb) && threadIdx.x == 0)
        ir_finish(tot, A.first, sc);
}

}  // namespace

bool ir3d_ok(const Dims& g) {
    return g.nz > 1 && 3LL * sweep3d_blocks(g) <= kRedPart;
}

void launch_ir_residual3d(const Dims& g, const float* x, const float* b, const float* const* beta,
                          double sign, float* r, int first, RedBuf rb, CGScalars* sc,
                          cudaStream_t s) {
    IRArgs a;
    a.g = g;
    a.xh = x;
    a.xl = x + g.ncell;
    a.bh = b;
    a.bl = b + g.ncell;
    a.bx = beta[0];
    a.by = beta[1];
    a.bz = beta[2];
    a.r = r;
    a.sign = sign;
    a.first = first;
    a.rb = rb;
    a.sc = sc;
    const int zc = tiled_zc(g);
    a.zc = zc;
    dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, (g.nz + zc - 1) / zc);
    k_ir_residual3d<<<grid, 256, 0, s>>>(a);
}

}  // namespace pf

// ---------------------------------------------------------------------------
// Restriction on 3D float32 levels: f_C(I) = mean over the 8 children of the
// fine residual f - A x. One thread per coarse column (I, J) marching in z;
// the 2 x 2 fine block of the planes k - 1, k, k + 1 and the z-face
// coefficients are carried in registers, the in-plane neighbours and
// coefficients come through L1 as pairs. The coefficients come from the
// level's face arrays, or on the finest level from the cell densities as
// 2 / (rho_c + rho_q) with the hardware reciprocal (RHO), the weights the
// finest smoother uses: one array instead of three.
// ---------------------------------------------------------------------------
namespace pf {
namespace {

struct RestrictArgs {
    Dims fg, cg;
    const float* x;
    const float* f;
    const float* bx;
    const float* by;
    const float* bz;
    const float* rho;
    float* cf;
    int zc;   // coarse planes per CTA
};

__device__ __forceinline__ float2 rcp2(float2 a, float2 b) {
    return make_float2(rcp_fast(a.x + b.x), rcp_fast(a.y + b.y));
}

constexpr int kRestrictAhead = 3;   // fine planes between an L2 prefetch and its use

template <bool RHO>
__global__ void __launch_bounds__(256, 5) k_restrict3d_reg(RestrictArgs A, const CGScalars* sc) {
    if (sc->done || sc->idone) return;
    const int I = blockIdx.x * 32 + threadIdx.x % 32;
    const int J = blockIdx.y * 8 + threadIdx.x / 32;
    const Dims& g = A.fg;
    if (I >= A.cg.nx || J >= A.cg.ny) return;
    const int nx = g.nx, ny = g.ny, nz = g.nz, sz = nx * ny;
    const int i = 2 * I, j = 2 * J;
    const int im = i == 0 ? nx - 1 : i - 1, ip2 = i + 2 == nx ? 0 : i + 2;
    const int r0 = j * nx, r1 = r0 + nx;
    const int rs = (j == 0 ? ny - 1 : j - 1) * nx, rn = (j + 2 == ny ? 0 : j + 2) * nx;
    // 1/rho_f = 2 / (rho_c + rho_q): the factor 2 goes with 1/h^2
    const float ih2 = RHO ? 2.f * g.ih2f : g.ih2f;
    const float* __restrict__ x = A.x;
    const float* __restrict__ f = A.f;
    const float* __restrict__ bx = A.bx;
    const float* __restrict__ by = A.by;
    const float* __restrict__ bz = A.bz;
    const float* __restrict__ rho = A.rho;
    auto pair = [](const float* a, int o) { return __ldg(reinterpret_cast<const float2*>(a + o)); };
    float* __restrict__ cf = A.cf;
    const int K0 = blockIdx.z * A.zc;
    const int K1 = min(K0 + A.zc, A.cg.nz);
    // 2 x 2 blocks (rows j, j + 1 as pairs) of planes k - 1 (m), k (c), k + 1 (p)
    int k = 2 * K0;
    int kb = k * sz;
    const int kbm = (k == 0 ? nz - 1 : k - 1) * sz;
    float2 m0 = pair(x, kbm + r0 + i), m1 = pair(x, kbm + r1 + i);
    float2 c0 = pair(x, kb + r0 + i), c1 = pair(x, kb + r1 + i);
    float2 zc0, zc1;
    float2 rc0 = make_float2(0.f, 0.f), rc1 = rc0;   // RHO: densities of the block in plane k
    if (RHO) {
        rc0 = pair(rho, kb + r0 + i);
        rc1 = pair(rho, kb + r1 + i);
        zc0 = rcp2(rc0, pair(rho, kbm + r0 + i));
        zc1 = rcp2(rc1, pair(rho, kbm + r1 + i));
    } else {
        zc0 = pair(bz, kb + r0 + i);
        zc1 = pair(bz, kb + r1 + i);
    }
    // L2 prefetch of the warp's two fine rows of x, f (and rho) kRestrictAhead
    // planes ahead: lane l < 12 takes array l / 4, row (l / 2) % 2 and the
    // 128-byte half l % 2 of the warp's 256-byte row segment
    const int lane = threadIdx.x % 32;
    const int i_w = 2 * (blockIdx.x * 32);           // first fine column of the warp
    const int pf_arr = lane >> 2, pf_row = (lane >> 1) & 1, pf_half = lane & 1;
    const float* pf_base = pf_arr == 0 ? x : pf_arr == 1 ? f : rho;
    const int pf_col = i_w + 32 * pf_half;
    const bool pf_on = lane < (RHO ? 12 : 8) && pf_col < nx;
    const int pf_off = (pf_row ? r1 : r0) + pf_col;
    const int k_last = 2 * K1;                        // one past the last fine plane read
    for (int K = K0; K < K1; ++K) {
        float s = 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h, ++k) {
            if (pf_on && k + kRestrictAhead <= k_last) {
                const int kq = k + kRestrictAhead;
                prefetch_l2(pf_base + (size_t)(kq >= nz ? kq - nz : kq) * sz + pf_off);
            }
            const int kp = k + 1 == nz ? 0 : k + 1;
            const int kpb = kp * sz;
            const float2 p0 = pair(x, kpb + r0 + i), p1 = pair(x, kpb + r1 + i);
            // in-plane neighbours of plane k
            const float xl0 = __ldg(x + kb + r0 + im), xl1 = __ldg(x + kb + r1 + im);
            const float xr0 = __ldg(x + kb + r0 + ip2), xr1 = __ldg(x + kb + r1 + ip2);
            const float2 xs = pair(x, kb + rs + i), xn = pair(x, kb + rn + i);
            const float2 f0 = pair(f, kb + r0 + i), f1 = pair(f, kb + r1 + i);
            // face coefficients of plane k: x faces at i, i + 1 (pairs) and
            // i + 2, y faces at j, j + 1, j + 2 (pairs), z faces above
            float2 bx0, bx1, by0, by1, by2, zp0, zp1, rp0, rp1;
            float bxr0, bxr1;
            if (RHO) {
                rp0 = pair(rho, kpb + r0 + i);
                rp1 = pair(rho, kpb + r1 + i);
                const float rl0 = __ldg(rho + kb + r0 + im), rl1 = __ldg(rho + kb + r1 + im);
                const float rr0 = __ldg(rho + kb + r0 + ip2), rr1 = __ldg(rho + kb + r1 + ip2);
                const float2 rsv = pair(rho, kb + rs + i), rnv = pair(rho, kb + rn + i);
                bx0 = make_float2(rcp_fast(rl0 + rc0.x), rcp_fast(rc0.x + rc0.y));
                bx1 = make_float2(rcp_fast(rl1 + rc1.x), rcp_fast(rc1.x + rc1.y));
                bxr0 = rcp_fast(rc0.y + rr0);
                bxr1 = rcp_fast(rc1.y + rr1);
                by0 = rcp2(rsv, rc0);
                by1 = rcp2(rc0, rc1);
                by2 = rcp2(rc1, rnv);
                zp0 = rcp2(rc0, rp0);
                zp1 = rcp2(rc1, rp1);
            } else {
                zp0 = pair(bz, kpb + r0 + i);
                zp1 = pair(bz, kpb + r1 + i);
                bx0 = pair(bx, kb + r0 + i);
                bx1 = pair(bx, kb + r1 + i);
                bxr0 = __ldg(bx + kb + r0 + ip2);
                bxr1 = __ldg(bx + kb + r1 + ip2);
                by0 = pair(by, kb + r0 + i);
                by1 = pair(by, kb + r1 + i);
                by2 = pair(by, kb + rn + i);
            }
            // children in the order (x fastest, then y) of the plane
            const float a00 = bx0.x * (c0.x - xl0) + bx0.y * (c0.x - c0.y) +
                              by0.x * (c0.x - xs.x) + by1.x * (c0.x - c1.x) +
                              zc0.x * (c0.x - m0.x) + zp0.x * (c0.x - p0.x);
            const float a10 = bx0.y * (c0.y - c0.x) + bxr0 * (c0.y - xr0) +
                              by0.y * (c0.y - xs.y) + by1.y * (c0.y - c1.y) +
                              zc0.y * (c0.y - m0.y) + zp0.y * (c0.y - p0.y);
            const float a01 = bx1.x * (c1.x - xl1) + bx1.y * (c1.x - c1.y) +
                              by1.x * (c1.x - c0.x) + by2.x * (c1.x - xn.x) +
                              zc1.x * (c1.x - m1.x) + zp1.x * (c1.x - p1.x);
            const float a11 = bx1.y * (c1.y - c1.x) + bxr1 * (c1.y - xr1) +
                              by1.y * (c1.y - c0.y) + by2.y * (c1.y - xn.y) +
                              zc1.y * (c1.y - m1.y) + zp1.y * (c1.y - p1.y);
            s += ((f0.x - ih2 * a00) + (f0.y - ih2 * a10)) + ((f1.x - ih2 * a01) + (f1.y - ih2 * a11));
            m0 = c0;
            m1 = c1;
            c0 = p0;
            c1 = p1;
            zc0 = zp0;
            zc1 = zp1;
            if (RHO) {
                rc0 = rp0;
                rc1 = rp1;
            }
            kb = kpb;
        }
        cf[(K * A.cg.ny + J) * A.cg.nx + I] = 0.125f * s;
    }
}

}  // namespace

bool restrict3d_ok(const Dims& fine) {
    return fine.nz > 1 && fine.nx % 2 == 0 && fine.ny % 2 == 0 && fine.nz % 2 == 0 &&
           fine.nx >= 4 && fine.ny >= 4 && fine.nz >= 4;
}

void launch_restrict3d(const MGLevel<float>& F, const MGLevel<float>& C, const float* rho,
                       const CGScalars* sc, cudaStream_t s) {
    RestrictArgs a;
    a.rho = rho;
    a.fg = F.g;
    a.cg = C.g;
    a.x = F.x;
    a.f = F.f;
    a.bx = F.beta[0];
    a.by = F.beta[1];
    a.bz = F.beta[2];
    a.cf = C.f;
    const int cols = ((C.g.nx + 31) / 32) * ((C.g.ny + 7) / 8);
    int zc = 32;
    while (zc > 1 && (long long)cols * ((C.g.nz + zc - 1) / zc) < 8 * 152) zc >>= 1;
    a.zc = zc;
    dim3 grid((C.g.nx + 31) / 32, (C.g.ny + 7) / 8, (C.g.nz + zc - 1) / zc);
    if (rho)
        k_restrict3d_reg<true><<<grid, 256, 0, s>>>(a, sc);
    else
        k_restrict3d_reg<false><<<grid, 256, 0, s>>>(a, sc);
}

}  // namespace pf
