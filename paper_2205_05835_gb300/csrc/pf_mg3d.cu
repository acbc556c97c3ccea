// One full red-black Gauss-Seidel sweep of a 3D float32 multigrid level in a
// single pass over memory (out of place: x_in -> x_out).
//
// A CTA owns a 32 x 8 column tile and marches along z. Each plane of x_in, f
// and the coefficient source (rho(phi) on the finest level, the three face
// coefficient arrays on coarser ones) is copied with a two-cell halo into
// shared-memory rings by cp.async two planes ahead of its use, so global
// latency overlaps the arithmetic. In the step for plane k the first six warps
// update the first colour on plane k over the tile plus a one-cell ring (its
// x_in neighbours are all of the other colour) and the last four warps update
// the second colour of plane k - 2 from the new first-colour values of planes
// k - 3 .. k - 1 and write both colours of plane k - 2: one barrier per plane.
// The halo ring is recomputed by both neighbouring CTAs, so no CTA reads
// another's output. Zero start (x_in = 0) skips the x_in copies.
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
#include <mutex>

#include "pf_device.cuh"

namespace pf {

namespace {

constexpr int TX = 32, TY = 8;              // tile (columns per CTA)
constexpr int HY = TY + 4;                  // rows j0-2 .. j0+TY+1 of a halo-2 plane
constexpr int RXS = TX + 2, RYS = TY + 2;   // halo-1 plane (first-colour values)
constexpr int N1 = (RXS / 2) * RYS;         // first-colour cells per plane (170)
constexpr int N2 = (TX / 2) * TY;           // second-colour cells per plane (128)
constexpr int W1 = 192;                     // first-colour threads: six whole warps
constexpr int NT = W1 + N2;                 // 320 threads

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
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) { cp_async<8>(smem, gmem); }
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
// ring slot of plane kp (kp >= -8)
template <int R>
__device__ __forceinline__ int slot(int kp) { return (int)((unsigned)(kp + 8 * R) % (unsigned)R); }
// slot s of a ring of R moved by d in [-R, R]
template <int R>
__device__ __forceinline__ int rmove(int s, int d) {
    s += d;
    s += s < 0 ? R : 0;
    return s >= R ? s - R : s;
}
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
    float x[RX_][HY][HX];
    float f[RF_][HY][HX];
    float c[FROM_PHI ? RR_ : 3 * RB_][HY][HX];
    float n[RN_][RYS][RXS];
};

template <bool FROM_PHI, int V>
__device__ __forceinline__ void sweep3d_body(const SweepArgs& A, unsigned char* smem_raw) {
    using G = Geo<V>;
    constexpr int HX = G::HX, OX = G::OX;
    constexpr int PLANE = HY * HX;   // floats per halo-2 plane
    Smem<FROM_PHI, V>& S = *reinterpret_cast<Smem<FROM_PHI, V>*>(smem_raw);
    float rz = 0.f, zq = 0.f;   // per-thread partial dots (A.dots)

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

    // this thread's copy chunk of a halo-2 plane (fixed across planes); the
    // second-colour warps take the first chunks
    const int lid = tid >= W1 ? tid - W1 : tid + N2;
    const bool has_chunk = lid < G::NCH;
    const int pb = lid / G::CPR, pa = V * (lid - pb * G::CPR);
    const int poff = mod(j0 - 2 + pb, g.ny) * sy + mod(i0 - OX + pa, g.nx);
    const int so = pb * HX + pa;     // chunk offset within a plane
    // next plane to copy: index, global plane base and ring slots
    int kiss = z0 - 2;
    int gz = mod(kiss, g.nz) * sz;
    int ix = slot<RX_>(kiss), iff = slot<RF_>(kiss), ic = slot<FROM_PHI ? RR_ : RB_>(kiss);

    auto issue = [&]() {
        if (has_chunk && kiss <= z1 + 1) {
            const int gidx = gz + poff;
            if (!zero) cp_async<4 * V>(&S.x[0][0][0] + ix * PLANE + so, A.xin + gidx);
            cp_async<4 * V>(&S.f[0][0][0] + iff * PLANE + so, A.f + gidx);
            if (FROM_PHI) {
                cp_async<4 * V>(&S.c[0][0][0] + ic * PLANE + so, A.phi + gidx);
            } else {
                cp_async<4 * V>(&S.c[0][0][0] + ic * PLANE + so, A.bx + gidx);
                cp_async<4 * V>(&S.c[0][0][0] + (RB_ + ic) * PLANE + so, A.by + gidx);
                cp_async<4 * V>(&S.c[0][0][0] + (2 * RB_ + ic) * PLANE + so, A.bz + gidx);
            }
        }
        cp_commit();
        ++kiss;
        gz += sz;
        if (gz >= g.ncell) gz -= g.ncell;
        ix = rmove<RX_>(ix, 1);
        iff = rmove<RF_>(iff, 1);
        ic = rmove<FROM_PHI ? RR_ : RB_>(ic, 1);
    };
    // rho(phi) in place for this thread's own chunk of the ring slot s (after
    // its copy landed)
    auto transform = [&](int s, bool used) {
        if (FROM_PHI && has_chunk && used) {
            float* c = &S.c[0][0][0] + s * PLANE + so;
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const float v = fminf(fmaxf(c[e], 0.f), 1.f);
                c[e] = __fadd_rn(ro, __fmul_rn(dr, v));
            }
        }
    };
    // weights -x, +x, -y, +y, -z, +z of the cell at (a, b); sc: coefficient
    // ring slot of its plane
    auto weights = [&](int a, int b, int sc, float (&w)[6]) {
        if (FROM_PHI) {
            const float* c0p = &S.c[sc][b][a];
            const float* cm = &S.c[rmove<RR_>(sc, -1)][b][a];
            const float* cp = &S.c[rmove<RR_>(sc, 1)][b][a];
            const float rc = c0p[0];
            w[0] = rcp_approx(rc + c0p[-1]);
            w[1] = rcp_approx(rc + c0p[1]);
            w[2] = rcp_approx(rc + c0p[-HX]);
            w[3] = rcp_approx(rc + c0p[HX]);
            w[4] = rcp_approx(rc + cm[0]);
            w[5] = rcp_approx(rc + cp[0]);
        } else {
            const int sp = rmove<RB_>(sc, 1);
            w[0] = S.c[sc][b][a];
            w[1] = S.c[sc][b][a + 1];
            w[2] = S.c[RB_ + sc][b][a];
            w[3] = S.c[RB_ + sc][b + 1][a];
            w[4] = S.c[2 * RB_ + sc][b][a];
            w[5] = S.c[2 * RB_ + sp][b][a];
        }
    };

    // fixed per-thread cell coordinates: first colour (halo-1 row b1, pair m1),
    // second colour (tile row tb, pair m2)
    const int b1f = tid / (RXS / 2), m1 = tid - b1f * (RXS / 2);
    const int t2 = tid - W1;
    const int tb = t2 >> 4, m2 = t2 & 15;

    // prologue: planes z0-2, z0-1 landed; z0 .. z0+PD-1 in flight
    constexpr int RC = FROM_PHI ? RR_ : RB_;
    const int c_lo = slot<RC>(z0 - 2);
    issue();
    issue();
    cp_wait_all();
    transform(c_lo, true);
    transform(rmove<RC>(c_lo, 1), true);
    for (int q = 0; q < PD; ++q) issue();
    // ring slots of plane kr (x, f, coefficients, first-colour values)
    int sx = slot<RX_>(z0 - 1), sf = slot<RF_>(z0 - 1), scr = slot<RC>(z0 - 1),
        sn = slot<RN_>(z0 - 1);
    // step kr: first colour on plane kr (kr <= z1), second colour on kb = kr - 2
    for (int kr = z0 - 1; kr <= z1 + 1; ++kr) {
        cp_wait<PD - 1>();      // own copies of plane kr + 1 have landed
        transform(rmove<RC>(scr, 1), kr + 1 <= z1 + 1);
        __syncthreads();        // every copy of plane kr + 1 visible; step kr - 1 done
        issue();                // plane kr + 1 + PD; overlaps with the next PD steps
        if (tid < W1) {
            if (tid < N1 && kr <= z1) {
                // halo-1 (a1, b1) has the colour (a1 + b1 + k) & 1 (i0, j0, n even)
                const int a1 = 2 * m1 + ((c0 + b1f + kr) & 1);
                const int a = a1 - 1 + OX, b = b1f + 1;
                float w[6];
                weights(a, b, scr, w);
                const float diag = w[0] + w[1] + w[2] + w[3] + w[4] + w[5];
                float num = S.f[sf][b][a] * fs;
                if (!zero) {
                    const float* xc = &S.x[sx][b][a];
                    num += w[0] * xc[-1] + w[1] * xc[1] + w[2] * xc[-HX] + w[3] * xc[HX] +
                           w[4] * S.x[rmove<RX_>(sx, -1)][b][a] +
                           w[5] * S.x[rmove<RX_>(sx, 1)][b][a];
                }
                S.n[sn][b1f][a1] = num * rcp_approx(diag);
            }
        } else {
            const int kb = kr - 2;
            if (kb >= z0 && kb < z1) {
                const int snb = rmove<RN_>(sn, -2), snm = rmove<RN_>(sn, -3),
                          snp = rmove<RN_>(sn, -1);
                const int sfb = rmove<RF_>(sf, -2);
                // interior (ta, tb) has the colour (ta + tb + k) & 1; second colour 1 - c0
                const int s2 = (c0 + 1 + tb + kb) & 1;
                const int ta = 2 * m2 + s2;
                const int a = ta + OX, b = tb + 2;
                const int a1 = ta + 1, b1 = tb + 1;
                float w[6];
                weights(a, b, rmove<RC>(scr, -2), w);
                const float diag = w[0] + w[1] + w[2] + w[3] + w[4] + w[5];
                const float* nc = &S.n[snb][b1][a1];
                const float num = S.f[sfb][b][a] * fs + w[0] * nc[-1] + w[1] * nc[1] +
                                  w[2] * nc[-RXS] + w[3] * nc[RXS] +
                                  w[4] * S.n[snm][b1][a1] + w[5] * S.n[snp][b1][a1];
                const float v2 = num * rcp_approx(diag);
                // the pair (2 m2, 2 m2 + 1) of this row holds one cell of each colour
                const int ea = 2 * m2;
                const float v_even = s2 == 0 ? v2 : S.n[snb][b1][ea + 1];
                const float v_odd = s2 == 1 ? v2 : S.n[snb][b1][ea + 2];
                const int gi = i0 + ea, gj = j0 + tb;
                if (gj < g.ny && gi < g.nx) {
                    const int kk = kb < 0 ? kb + g.nz : (kb >= g.nz ? kb - g.nz : kb);
                    float* out = A.xout + kk * sz + gj * sy + gi;
                    *reinterpret_cast<float2*>(out) = make_float2(v_even, v_odd);
                    if (A.dots) {
                        rz += S.f[sfb][b][ea + OX] * v_even + S.f[sfb][b][ea + OX + 1] * v_odd;
                        if (!A.first) {
                            const float2 qq = __ldg(reinterpret_cast<const float2*>(
                                A.q + (kk * sz + gj * sy + gi)));
                            zq += v_even * qq.x + v_odd * qq.y;
                        }
                    }
                }
            }
        }
        sx = rmove<RX_>(sx, 1);
        sf = rmove<RF_>(sf, 1);
        scr = rmove<RC>(scr, 1);
        sn = rmove<RN_>(sn, 1);
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

// finest level (coefficients from phi) and coarser levels (face arrays), in
// 16-byte (V = 4) or 8-byte (V = 2) copy chunks
template <bool FROM_PHI, int V>
__global__ void __launch_bounds__(NT, FROM_PHI ? 5 : 4) k_sweep3d(SweepArgs A, const CGScalars* sc) {
    if (sc && (sc->done || sc->idone)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    sweep3d_body<FROM_PHI, V>(A, smem_raw);
}

template <bool FROM_PHI, int V>
void launch_sweep3d_t(const SweepArgs& a, dim3 grid, const CGScalars* sc, cudaStream_t s) {
    static std::once_flag attr_once;
    std::call_once(attr_once, [] {
        // dynamic shared memory beyond 48 KB, and a shared-memory carveout that
        // lets several CTAs share an SM
        cudaFuncSetAttribute(k_sweep3d<FROM_PHI, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(Smem<FROM_PHI, V>));
        cudaFuncSetAttribute(k_sweep3d<FROM_PHI, V>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    });
    k_sweep3d<FROM_PHI, V><<<grid, NT, sizeof(Smem<FROM_PHI, V>), s>>>(a, sc);
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
    const int zc = tiled_zc(L.g);
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
//   p_new = z + beta p_old ; q = A p_new ; alpha = rz / (p_new . q)
// Register z-march: one thread per column of a 32 x 8 tile; p_new of the column at k-1, k, k+1 and the z-face
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
