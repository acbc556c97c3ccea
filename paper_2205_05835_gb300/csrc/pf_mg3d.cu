// One full red-black Gauss-Seidel sweep of a 3D float32 multigrid level in a
// single pass over memory (out of place: x_in -> x_out).
//
// A CTA owns a 32 x 8 column tile and marches along z. Each plane of x_in, f
// and the coefficient source (rho(phi) on the finest level, the three face
// coefficient arrays on coarser ones) is copied with a two-cell halo into
// shared-memory rings by cp.async one plane ahead of its use, so global
// latency overlaps the arithmetic. In the step for plane k the CTA updates the
// first colour on plane k over the tile plus a one-cell ring (its x_in
// neighbours are all of the other colour) and, concurrently on other warps,
// the second colour of plane k - 2 from the new first-colour values of planes
// k - 3 .. k - 1, then writes both colours of plane k - 2: one barrier per
// plane. The halo ring is recomputed by both neighbouring CTAs, so no CTA
// reads another's output. Zero start (x_in = 0) skips the x_in copies.
// Requires even nx, ny, nz (consistent periodic colouring); tiles may be
// ragged (sizes need not be multiples of 32 x 8) since every index wraps.
#include <mutex>

#include "pf_device.cuh"

namespace pf {

namespace {

constexpr int TX = 32, TY = 8;              // tile (columns per CTA)
constexpr int HX = TX + 4, HY = TY + 4;     // halo-2 plane in shared memory
constexpr int NPAIR = (HX / 2) * HY;        // 8-byte pairs per halo-2 plane (216)
constexpr int RXS = TX + 2, RYS = TY + 2;   // halo-1 plane (first-colour values)
constexpr int N1 = (RXS / 2) * RYS;         // first-colour cells per plane (170)
constexpr int N2 = (TX / 2) * TY;           // second-colour cells per plane (128)
constexpr int NT = 320;                     // threads: N1 + N2 rounded up to warps

__device__ __forceinline__ int mod(int a, int m) { int r = a % m; return r < 0 ? r + m : r; }

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
// ring slot of plane kp (kp >= -8)
template <int R>
__device__ __forceinline__ int slot(int kp) { return (int)((unsigned)(kp + 8 * R) % (unsigned)R); }

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
    float ih2;            // 1 / h^2
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
template <bool FROM_PHI>
struct Smem {
    float x[RX_][HY][HX];
    float f[RF_][HY][HX];
    float c[FROM_PHI ? RR_ : 3 * RB_][HY][HX];
    float n[RN_][RYS][RXS];
};

template <bool FROM_PHI>
__device__ __forceinline__ void sweep3d_body(const SweepArgs& A, unsigned char* smem_raw) {
    Smem<FROM_PHI>& S = *reinterpret_cast<Smem<FROM_PHI>*>(smem_raw);
    float rz = 0.f, zq = 0.f;   // per-thread partial dots (A.dots)

    const Dims& g = A.g;
    const int tid = threadIdx.x;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * A.zc;
    const int z1 = min(z0 + A.zc, g.nz);
    const int sy = g.nx, sz = g.nx * g.ny;
    const float ih2 = A.ih2;
    const int c0 = A.first_color;
    const bool zero = A.xin == nullptr;
    const float ro = A.ph.rho_out_f, dr = A.ph.drho_f;

    // this thread's 8-byte pair of the halo-2 plane (fixed across planes)
    const bool has_pair = tid < NPAIR;
    const int pb = tid / (HX / 2), pa = 2 * (tid - pb * (HX / 2));
    const int pgi = mod(i0 - 2 + pa, g.nx), pgj = mod(j0 - 2 + pb, g.ny);
    const int poff = pgj * sy + pgi;

    // copies of plane kp (x_in, f, coefficient source) as one commit group;
    // nothing past the last plane needed
    auto issue = [&](int kp) {
        if (has_pair && kp <= z1 + 1) {
            const int gidx = mod(kp, g.nz) * sz + poff;
            if (!zero) cp_async8(&S.x[slot<RX_>(kp)][pb][pa], A.xin + gidx);
            cp_async8(&S.f[slot<RF_>(kp)][pb][pa], A.f + gidx);
            if (FROM_PHI) {
                cp_async8(&S.c[slot<RR_>(kp)][pb][pa], A.phi + gidx);
            } else {
                const int s = slot<RB_>(kp);
                cp_async8(&S.c[s][pb][pa], A.bx + gidx);
                cp_async8(&S.c[RB_ + s][pb][pa], A.by + gidx);
                cp_async8(&S.c[2 * RB_ + s][pb][pa], A.bz + gidx);
            }
        }
        cp_commit();
    };
    // rho(phi) in place for this thread's own pair of plane kp (after it landed)
    auto transform = [&](int kp) {
        if (FROM_PHI && has_pair && kp <= z1 + 1) {
            float* c = &S.c[slot<RR_>(kp)][pb][pa];
            const float s0 = fminf(fmaxf(c[0], 0.f), 1.f), s1 = fminf(fmaxf(c[1], 0.f), 1.f);
            c[0] = __fadd_rn(ro, __fmul_rn(dr, s0));
            c[1] = __fadd_rn(ro, __fmul_rn(dr, s1));
        }
    };
    auto inv2 = [&](float ra, float rb) { return __frcp_rn(__fmul_rn(0.5f, __fadd_rn(ra, rb))) * ih2; };
    // face weights -x, +x, -y, +y, -z, +z of the cell at (a, b) in plane kp
    auto weights = [&](int a, int b, int kp, float (&w)[6]) {
        if (FROM_PHI) {
            const int s0 = slot<RR_>(kp), sm = slot<RR_>(kp - 1), sp = slot<RR_>(kp + 1);
            const float rc = S.c[s0][b][a];
            w[0] = inv2(rc, S.c[s0][b][a - 1]);
            w[1] = inv2(rc, S.c[s0][b][a + 1]);
            w[2] = inv2(rc, S.c[s0][b - 1][a]);
            w[3] = inv2(rc, S.c[s0][b + 1][a]);
            w[4] = inv2(rc, S.c[sm][b][a]);
            w[5] = inv2(rc, S.c[sp][b][a]);
        } else {
            const int s0 = slot<RB_>(kp), sp = slot<RB_>(kp + 1);
            w[0] = S.c[s0][b][a] * ih2;
            w[1] = S.c[s0][b][a + 1] * ih2;
            w[2] = S.c[RB_ + s0][b][a] * ih2;
            w[3] = S.c[RB_ + s0][b + 1][a] * ih2;
            w[4] = S.c[2 * RB_ + s0][b][a] * ih2;
            w[5] = S.c[2 * RB_ + sp][b][a] * ih2;
        }
    };

    // prologue: planes z0-2, z0-1 landed; z0 .. z0+PD-1 in flight
    issue(z0 - 2);
    issue(z0 - 1);
    cp_wait_all();
    transform(z0 - 2);
    transform(z0 - 1);
    for (int q = 0; q < PD; ++q) issue(z0 + q);
    // step kr: first colour on plane kr (kr <= z1), second colour on kb = kr - 2
    for (int kr = z0 - 1; kr <= z1 + 1; ++kr) {
        cp_wait<PD - 1>();      // own copies of plane kr + 1 have landed
        transform(kr + 1);
        __syncthreads();        // every copy of plane kr + 1 visible; step kr - 1 done
        issue(kr + 1 + PD);     // overlaps with the next PD steps
        if (tid < N1) {
            if (kr <= z1) {
                const int kk = kr < 0 ? kr + g.nz : (kr >= g.nz ? kr - g.nz : kr);
                const int sx0 = slot<RX_>(kr), sxm = slot<RX_>(kr - 1), sxp = slot<RX_>(kr + 1);
                const int per_row = RXS / 2;
                const int b1 = tid / per_row, m = tid - b1 * per_row;
                // halo-1 (a1, b1) has the colour (a1 + b1 + k) & 1 (i0, j0 even, n even)
                const int a1 = 2 * m + ((c0 + b1 + kk) & 1);
                const int a = a1 + 1, b = b1 + 1;
                float w[6];
                weights(a, b, kr, w);
                const float diag = w[0] + w[1] + w[2] + w[3] + w[4] + w[5];
                float off = 0.f;
                if (!zero)
                    off = w[0] * S.x[sx0][b][a - 1] + w[1] * S.x[sx0][b][a + 1] +
                          w[2] * S.x[sx0][b - 1][a] + w[3] * S.x[sx0][b + 1][a] +
                          w[4] * S.x[sxm][b][a] + w[5] * S.x[sxp][b][a];
                S.n[slot<RN_>(kr)][b1][a1] = (S.f[slot<RF_>(kr)][b][a] + off) * __frcp_rn(diag);
            }
        } else if (tid < N1 + N2) {
            const int kb = kr - 2;
            if (kb >= z0 && kb < z1) {
                const int t = tid - N1;
                const int kk = kb < 0 ? kb + g.nz : (kb >= g.nz ? kb - g.nz : kb);
                const int snb = slot<RN_>(kb), snm = slot<RN_>(kb - 1), snp = slot<RN_>(kb + 1);
                const int tb = t / (TX / 2), m = t - tb * (TX / 2);
                const int b = tb + 2, b1 = tb + 1;
                // interior (ta, tb) has the colour (ta + tb + k) & 1; second colour 1 - c0
                const int s2 = (c0 + 1 + tb + kk) & 1;
                const int ta = 2 * m + s2;
                const int a = ta + 2, a1 = ta + 1;
                float w[6];
                weights(a, b, kb, w);
                const float diag = w[0] + w[1] + w[2] + w[3] + w[4] + w[5];
                const float off = w[0] * S.n[snb][b1][a1 - 1] + w[1] * S.n[snb][b1][a1 + 1] +
                                  w[2] * S.n[snb][b1 - 1][a1] + w[3] * S.n[snb][b1 + 1][a1] +
                                  w[4] * S.n[snm][b1][a1] + w[5] * S.n[snp][b1][a1];
                const float v2 = (S.f[slot<RF_>(kb)][b][a] + off) * __frcp_rn(diag);
                // the pair (2m, 2m + 1) of this row holds one cell of each colour
                const int ea = 2 * m;
                const float v_even = s2 == 0 ? v2 : S.n[snb][b1][ea + 1];
                const float v_odd = s2 == 1 ? v2 : S.n[snb][b1][ea + 2];
                const int gi = i0 + ea, gj = j0 + tb;
                if (gj < g.ny && gi < g.nx) {
                    float* out = A.xout + kk * sz + gj * sy + gi;
                    *reinterpret_cast<float2*>(out) = make_float2(v_even, v_odd);
                    if (A.dots) {
                        const int sfb = slot<RF_>(kb);
                        rz += S.f[sfb][b][ea + 2] * v_even + S.f[sfb][b][ea + 3] * v_odd;
                        if (!A.first) {
                            const float2 qq = __ldg(reinterpret_cast<const float2*>(
                                A.q + (kk * sz + gj * sy + gi)));
                            zq += v_even * qq.x + v_odd * qq.y;
                        }
                    }
                }
            }
        }
    }
    cp_wait_all();
    if (A.dots) {
        double v[2] = {double(rz), double(zq)}, tot[2];
        const int mode[2] = {0, 0};
        const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        const int nb = gridDim.x * gridDim.y * gridDim.z;
        if (grid_reduce_lin<2>(v, mode, A.rb, tot, bid, nb) && threadIdx.x == 0) {
            CGScalars* sc = A.scw;
            sc->beta = A.first ? 0.0 : -sc->alpha * tot[1] / sc->rz;
            sc->rz = tot[0];
        }
    }
}

// finest level (coefficients from phi) and coarser levels (face arrays)
__global__ void __launch_bounds__(NT) k_sweep3d_fine(SweepArgs A, const CGScalars* sc) {
    if (sc && (sc->done || sc->idone)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    sweep3d_body<true>(A, smem_raw);
}
__global__ void __launch_bounds__(NT) k_sweep3d_coarse(SweepArgs A, const CGScalars* sc) {
    if (sc && (sc->done || sc->idone)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    sweep3d_body<false>(A, smem_raw);
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

// Eligible: 3D float level with even sizes.
bool sweep3d_ok(const Dims& g) {
    return g.nz > 1 && (g.nx % 2 == 0) && (g.ny % 2 == 0) && (g.nz % 2 == 0) && g.nx >= 4 &&
           g.ny >= 4 && g.nz >= 4;
}

void launch_sweep3d(const MGLevel<float>& L, const float* phi, const Phys& ph, const float* xin,
                    float* xout, const SweepDots* dots, int first_color, const CGScalars* sc,
                    cudaStream_t s) {
    static std::once_flag attr_once;
    std::call_once(attr_once, [] {
        // dynamic shared memory beyond 48 KB, and a shared-memory carveout that
        // lets several CTAs share an SM
        cudaFuncSetAttribute(k_sweep3d_fine, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(Smem<true>));
        cudaFuncSetAttribute(k_sweep3d_coarse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(Smem<false>));
        cudaFuncSetAttribute(k_sweep3d_fine, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaFuncSetAttribute(k_sweep3d_coarse, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    });
    SweepArgs a;
    a.g = L.g;
    a.xin = xin;
    a.f = L.f;
    a.xout = xout;
    a.phi = phi;
    a.bx = L.beta[0];
    a.by = L.beta[1];
    a.bz = L.beta[2];
    a.ph = ph;
    a.ih2 = L.g.ih2f;
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
    const int zc = tiled_zc(L.g);
    a.zc = zc;
    dim3 grid((L.g.nx + TX - 1) / TX, (L.g.ny + TY - 1) / TY, (L.g.nz + zc - 1) / zc);
    if (dots && 2LL * grid.x * grid.y * grid.z > (long long)kRedPart) {
        // more CTAs than reduction slots: the caller runs the dot kernel instead
        a.dots = 0;
    }
    if (L.beta[0] == nullptr)
        k_sweep3d_fine<<<grid, NT, sizeof(Smem<true>), s>>>(a, sc);
    else
        k_sweep3d_coarse<<<grid, NT, sizeof(Smem<false>), s>>>(a, sc);
}

}  // namespace pf

// ---------------------------------------------------------------------------
// CG search direction and operator product on 3D float32 grids, tiled:
//   p_new = z + beta p_old ; q = A p_new ; alpha = rz / (p_new . q)
// A CTA owns a 32 x 8 column tile and marches along z; z, p_old and the face
// coefficients are copied into shared-memory rings by cp.async two planes
// ahead, p_new of the neighbours is formed on the fly from them.
// ---------------------------------------------------------------------------
namespace pf {
namespace {

constexpr int DR = 5;     // ring planes (3 in use + 2 in flight)
constexpr int DNT = 256;  // threads: one per tile column

struct DirSmem {
    float z[DR][HY][HX];
    float p[DR][HY][HX];
    float b[3][DR][HY][HX];
};

struct DirArgs {
    Dims g;
    const float* z;
    const float* p_old;
    float* p_new;
    float* q;
    const float* bx;
    const float* by;
    const float* bz;
    float ih2;
    int first;
    int zc;
    RedBuf rb;
    CGScalars* sc;
};

__global__ void __launch_bounds__(DNT) k_dir3d(DirArgs A) {
    CGScalars* sc = A.sc;
    if (sc->done || sc->idone) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DirSmem& S = *reinterpret_cast<DirSmem*>(smem_raw);
    const Dims& g = A.g;
    const int tid = threadIdx.x;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * A.zc;
    const int z1 = min(z0 + A.zc, g.nz);
    const int sy = g.nx, sz = g.nx * g.ny;
    const float bcg = A.first ? 0.f : float(sc->beta);
    const bool has_pair = tid < NPAIR;
    const int pb = tid / (HX / 2), pa = 2 * (tid - pb * (HX / 2));
    const int poff = mod(j0 - 2 + pb, g.ny) * sy + mod(i0 - 2 + pa, g.nx);

    auto issue = [&](int kp) {
        if (has_pair && kp <= z1) {
            const int gidx = mod(kp, g.nz) * sz + poff;
            const int s = slot<DR>(kp);
            cp_async8(&S.z[s][pb][pa], A.z + gidx);
            if (!A.first) cp_async8(&S.p[s][pb][pa], A.p_old + gidx);
            cp_async8(&S.b[0][s][pb][pa], A.bx + gidx);
            cp_async8(&S.b[1][s][pb][pa], A.by + gidx);
            cp_async8(&S.b[2][s][pb][pa], A.bz + gidx);
        }
        cp_commit();
    };
    auto pn = [&](int s, int b, int a) {
        return A.first ? S.z[s][b][a] : S.z[s][b][a] + bcg * S.p[s][b][a];
    };

    // prologue: planes z0-1 .. z0+2; each step waits for plane k + 1 and keeps
    // two planes in flight
    issue(z0 - 1);
    issue(z0);
    issue(z0 + 1);
    issue(z0 + 2);
    float pq = 0.f;
    const int ta = tid % TX, tb = tid / TX;
    const int a = ta + 2, b = tb + 2;
    const int gi = i0 + ta, gj = j0 + tb;
    const bool own = gi < g.nx && gj < g.ny;
    for (int k = z0; k < z1; ++k) {
        cp_wait<1>();           // own copies up to plane k + 1 landed
        __syncthreads();        // all copies of plane k + 1 visible; step k - 1 done
        issue(k + 3);
        const int s0 = slot<DR>(k), sm = slot<DR>(k - 1), sp = slot<DR>(k + 1);
        const float pc = pn(s0, b, a);
        float ax = S.b[0][s0][b][a] * (pc - pn(s0, b, a - 1)) +
                   S.b[0][s0][b][a + 1] * (pc - pn(s0, b, a + 1)) +
                   S.b[1][s0][b][a] * (pc - pn(s0, b - 1, a)) +
                   S.b[1][s0][b + 1][a] * (pc - pn(s0, b + 1, a)) +
                   S.b[2][s0][b][a] * (pc - pn(sm, b, a)) +
                   S.b[2][sp][b][a] * (pc - pn(sp, b, a));
        ax *= A.ih2;
        if (own) {
            const int idx = k * sz + gj * sy + gi;
            A.p_new[idx] = pc;
            A.q[idx] = ax;
            pq += pc * ax;
        }
    }
    cp_wait<0>();
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

bool dir3d_ok(const Dims& g) {
    return g.nz > 1 && (g.nx % 2 == 0) && (g.ny % 2 == 0) && g.nx >= 4 && g.ny >= 4 &&
           g.nz >= 4 && sweep3d_blocks(g) <= kRedPart;
}

void launch_dir3d(const Dims& g, const float* z, const float* p_old, float* p_new, float* q,
                  const float* const* beta, int first, RedBuf rb, CGScalars* sc, cudaStream_t s) {
    static std::once_flag attr_once;
    std::call_once(attr_once, [] {
        cudaFuncSetAttribute(k_dir3d, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(DirSmem));
        cudaFuncSetAttribute(k_dir3d, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    });
    DirArgs a;
    a.g = g;
    a.z = z;
    a.p_old = p_old;
    a.p_new = p_new;
    a.q = q;
    a.bx = beta[0];
    a.by = beta[1];
    a.bz = beta[2];
    a.ih2 = g.ih2f;
    a.first = first;
    a.rb = rb;
    a.sc = sc;
    const int zc = tiled_zc(g);
    a.zc = zc;
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + zc - 1) / zc);
    k_dir3d<<<grid, DNT, sizeof(DirSmem), s>>>(a);
}

}  // namespace pf

// ---------------------------------------------------------------------------
// Register z-marching variant of the CG direction kernel: one thread per
// column of a 32 x 8 tile; p_new of the column at k-1, k, k+1 and the z-face
// coefficient above are carried in registers, the in-plane neighbours come
// through L1. No shared memory and no barriers.
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
    float ih2;
    int first;
    int zc;
    RedBuf rb;
    CGScalars* sc;
};

__global__ void __launch_bounds__(256) k_dir3d_reg(DirRegArgs A) {
    CGScalars* sc = A.sc;
    if (sc->done || sc->idone) return;
    const Dims& g = A.g;
    const float bcg = A.first ? 0.f : float(sc->beta);
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
        auto pn = [&](int idx) {
            const float zv = __ldg(A.z + idx);
            return A.first ? zv : zv + bcg * __ldg(A.p_old + idx);
        };
        const int km1 = z0 == 0 ? g.nz - 1 : z0 - 1;
        float p_m = pn(km1 * sz + col);
        float p_c = pn(z0 * sz + col);
        float bz_c = __ldg(A.bz + z0 * sz + col);
#pragma unroll 2
        for (int k = z0; k < z1; ++k) {
            const int kp = k + 1 == g.nz ? 0 : k + 1;
            const int idx = k * sz + col;
            const int idxp = kp * sz + col;
            const float p_p = pn(idxp);
            const float bz_p = __ldg(A.bz + idxp);
            const float ax = __ldg(A.bx + idx) * (p_c - pn(idx + ox_m)) +
                             __ldg(A.bx + idx + ox_p) * (p_c - pn(idx + ox_p)) +
                             __ldg(A.by + idx) * (p_c - pn(idx + oy_m)) +
                             __ldg(A.by + idx + oy_p) * (p_c - pn(idx + oy_p)) +
                             bz_c * (p_c - p_m) + bz_p * (p_c - p_p);
            const float qv = ax * A.ih2;
            A.p_new[idx] = p_c;
            A.q[idx] = qv;
            pq += p_c * qv;
            p_m = p_c;
            p_c = p_p;
            bz_c = bz_p;
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
                      const float* const* beta, int first, RedBuf rb, CGScalars* sc,
                      cudaStream_t s) {
    DirRegArgs a;
    a.g = g;
    a.z = z;
    a.p_old = p_old;
    a.p_new = p_new;
    a.q = q;
    a.bx = beta[0];
    a.by = beta[1];
    a.bz = beta[2];
    a.ih2 = g.ih2f;
    a.first = first;
    a.rb = rb;
    a.sc = sc;
    const int zc = tiled_zc(g);
    a.zc = zc;
    dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, (g.nz + zc - 1) / zc);
    k_dir3d_reg<<<grid, 256, 0, s>>>(a);
}

}  // namespace pf
