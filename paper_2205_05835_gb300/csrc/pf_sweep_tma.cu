// One full red-black Gauss-Seidel sweep of the finest 3D float32 multigrid
// level (smoother weights from the cell densities rho), with every plane
// staged into shared memory by the Tensor Memory Accelerator.
//
// Same per-cell arithmetic as the cp.async-staged sweep of pf_mg3d.cu, bit for
// bit: a CTA owns a 32 x TY column tile (TY 8 or 16) and marches along z; in
// the step for plane k one group of warps updates the first colour of plane k
// over the tile plus a one-cell ring, and a second group updates the second
// colour of plane k - 2 from the new first-colour values of planes k - 3 ..
// k - 1 and writes both colours of plane k - 2; each thread takes one or two
// cells of its colour per plane. What differs is the staging:
//
//  * a producer warp stages the planes, four steps ahead of their use, into
//    rings of eight planes per array: for tiles whose halo does not cross a
//    periodic seam one tiled tensor copy (cp.async.bulk.tensor, box
//    40 x (TY + 4) x 1) per array, completing on the ring slot's mbarrier with the
//    plane's bytes; for the others 16-byte cp.async chunks with wrapped
//    addresses, which the mbarrier tracks through cp.async.mbarrier.arrive;
//  * the compute warps wait on those mbarriers, synchronise among themselves
//    with a named barrier once per plane, and release a ring slot through an
//    "empty" mbarrier when the last step that reads its plane is done.
//
// Every wait on an mbarrier is bounded (about one second of the global
// timer). A wait that gives up latches PF_ERR_TIMEOUT and `done` in the
// solve's scalars, the CTA leaves its z loop after the next block barrier,
// thread 0 waits (bounded again) for the copies still in flight, and the CTA
// still joins the grid reduction so the reduction buffers stay consistent.
#include <cuda.h>

#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "../../include/pf.h"
#include "pf_device.cuh"
#include "pf_tma.cuh"

namespace pf {

namespace {

using namespace tma;

constexpr int TX = 32, OX = 4;                // tile width, staged columns left of it
constexpr int HX = TX + 2 * OX;               // 40 columns of a staged plane
constexpr int RXS = TX + 2;                   // one-cell ring around the tile, x
constexpr int RXH = RXS / 2;                  // first-colour cells per ring row (17)
constexpr int RING = 8;                       // ring planes of rho, f and x_in
constexpr int RN = 4;                         // ring planes of the new first colour
constexpr int CPR = HX / 4;                   // 16-byte chunks per staged row

// Tile shapes: 32 x TY columns per CTA, each thread updating CPT cells of its
// colour per plane. The staged plane and the shared-memory layout depend on
// TY; the thread groups on both (more cells per thread: fewer warps, the
// per-plane waits, barrier and loop control spread over more cells).
template <int TY_, int CPT_>
struct TileCfg {
    static constexpr int TY = TY_;
    static constexpr int CPT = CPT_;                     // cells per thread and plane
    static constexpr int HY = TY + 4;                    // rows (two-cell halo in y)
    static constexpr int PLANE = HX * HY;                // floats per staged plane
    static constexpr unsigned PLANE_BYTES = PLANE * 4u;
    static constexpr int RYS = TY + 2;                   // one-cell ring, y
    static constexpr int NPL = RYS * RXH;                // first-colour cells per plane
    static constexpr int W1 = ((NPL + 32 * CPT - 1) / (32 * CPT)) * 32;   // first-colour threads
    static constexpr int W2 = (TX / 2) * TY / CPT;       // second-colour threads
    static constexpr int NC = W1 + W2;                   // compute threads
    static constexpr int NT = NC + 32;                   // + one producer warp
    static constexpr int NCH = CPR * HY;                 // 16-byte chunks per staged plane
    static constexpr int F_OFF = RING * PLANE;           // floats from the rho ring to the f ring
    static_assert(PLANE * 4 % 128 == 0, "staged planes must start on 128-byte boundaries");
};

// Shared memory: rings of rho, f (and x_in unless the sweep starts from zero,
// last so that a zero-start launch leaves it out), each RING planes of PLANE
// floats; the new first-colour values; per ring slot a "full" mbarrier for
// rho, one for f / x_in (completed by the copies' bytes) and an "empty" one
// (the compute warps' release of the slot's plane, one arrival per warp).
template <int TY>
struct __align__(128) SmemT {
    float rho[RING][TileCfg<TY, 1>::PLANE];
    float f[RING][TileCfg<TY, 1>::PLANE];
    float n[RN][TileCfg<TY, 1>::NPL];
    unsigned long long bar_r[RING];
    unsigned long long bar_xf[RING];
    unsigned long long bar_empty[RING];
    int abort;
    int issued;                       // last plane the producer issued
    float pad[14];
    alignas(128) float x[RING][TileCfg<TY, 1>::PLANE];
};
template <int TY>
constexpr int x_off() { return (int)(offsetof(SmemT<TY>, x) / sizeof(float)); }   // rho -> x
template <int TY>
constexpr size_t smem_zero() { return offsetof(SmemT<TY>, x) + 128; }   // + alignment slack
template <int TY>
constexpr size_t smem_full() { return sizeof(SmemT<TY>) + 128; }

struct TmaArgs {
    Dims g;
    const float* rho;     // finest-level cell densities (global, for row copies)
    const float* f;       // right-hand side (global, for row copies)
    const float* xin;     // nullptr: zero start
    float* xout;
    float fs;             // h^2 / 2
    int first_color;
    int zc;
    int dots;             // also r.z and z.q (see SweepDots)
    int first;
    const float* q;
    RedBuf rb;
    CGScalars* scw;       // dots: CG scalars written by the last block
    CGScalars* st;        // status and done of the solve (timeout)
    int stall;            // test of the bounded wait: one interior CTA expects bytes that never come
};

// CTAs per SM that shared memory (228 KB, 1 KB reserved per CTA) and the
// 2048 threads allow
template <bool ZERO, int TY, int CPT>
constexpr int tile_min_blocks() {
    constexpr int by_smem = 233472 / (int)((ZERO ? smem_zero<TY>() : smem_full<TY>()) + 1024);
    constexpr int by_threads = 2048 / TileCfg<TY, CPT>::NT;
    return by_smem < by_threads ? by_smem : by_threads;
}

// The last warp is the producer: it issues the copies of every staged plane q (rho,
// f and x_in together) as soon as the compute warps have released the ring
// slot's previous plane q - RING. The compute warps release plane q at the
// end of step q + 3 (the last step that reads it: the second colour on plane
// q + 1 reads rho of q), so a plane is issued four steps before it is needed.
template <bool ZERO, int TY, int CPT_>
__global__ void __launch_bounds__(TileCfg<TY, CPT_>::NT, (tile_min_blocks<ZERO, TY, CPT_>()))
k_sweep3d_tma(const __grid_constant__ CUtensorMap tm_rho, const __grid_constant__ CUtensorMap tm_f,
              const __grid_constant__ CUtensorMap tm_x, TmaArgs A, const CGScalars* sc) {
    using C = TileCfg<TY, CPT_>;
    constexpr int PLANE = C::PLANE, NPL = C::NPL, W1 = C::W1, W2 = C::W2, NC = C::NC;
    constexpr int CPT = CPT_;
    constexpr int F_OFF = C::F_OFF, X_OFF = x_off<TY>();
    constexpr unsigned PLANE_BYTES = C::PLANE_BYTES;
    if (sc && (sc->done || sc->idone)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // 128-byte aligned base (the launch reserves 128 bytes for this)
    SmemT<TY>& S = *reinterpret_cast<SmemT<TY>*>(
        smem_raw + ((128u - (su32(smem_raw) & 127u)) & 127u));
    float* const B = &S.rho[0][0];    // rho ring; f at B + F_OFF, x_in at B + X_OFF
    const Dims& g = A.g;
    const int tid = threadIdx.x, lane = tid & 31;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * A.zc;
    const int z1 = min(z0 + A.zc, g.nz);
    const int P0 = z0 - 2;               // a staged plane's index q is k - P0
    const int QMAX = z1 + 1 - P0;        // staged planes q = 0 .. QMAX
    const int SMAX = QMAX;               // steps s = 1 .. SMAX
    const int sz = g.nx * g.ny;
    const int c0 = A.first_color;
    const float fs = A.fs;
    const bool interior = i0 - OX >= 0 && i0 + TX + OX <= g.nx && j0 - 2 >= 0 && j0 + TY + 2 <= g.ny;
    float rz = 0.f, zq = 0.f;
    const int first_it = A.dots ? first_of(A.first, A.scw) : 1;
    volatile int* abort = &S.abort;

    if (tid == 0) {
        // full barriers: one arrival with the expected bytes of the tensor
        // copies (interior tiles), or one cp.async-tracking arrival per
        // producer lane (tiles across a seam)
        const unsigned nfull = interior ? 1u : (unsigned)NC;
        for (int s = 0; s < RING; ++s) {
            mbar_init(&S.bar_r[s], nfull);
            mbar_init(&S.bar_xf[s], nfull);
            mbar_init(&S.bar_empty[s], NC / 32);
        }
        S.abort = 0;
        S.issued = -1;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    const bool tma = interior;
    if (tid >= NC) {
        // ---------------- producer warp (tiles away from the seams) ----------------
        for (int q = 0; q <= (tma ? QMAX : -1); ++q) {
            const int slot = q & (RING - 1);
            if (q >= RING &&
                !mbar_wait_or_abort(&S.bar_empty[slot], (unsigned)((q >> 3) - 1) & 1u, abort)) {
                if (lane == 0) *abort = 1;
                break;
            }
            const int z = modp(P0 + q, g.nz);
            // one tensor box (40 x (TY + 4) x 1) per array
            if (lane == 0) {
                // the wait test: CTA (1, 1, 0) expects 16 bytes more than plane 2
                // brings, so that phase never completes and its waits run out
                const bool stall = A.stall && q == 2 && blockIdx.x == 1 && blockIdx.y == 1 &&
                                   blockIdx.z == 0;
                mbar_expect_tx(&S.bar_r[slot], PLANE_BYTES + (stall ? 16u : 0u));
                tma_box(S.rho[slot], &tm_rho, i0 - OX, j0 - 2, z, &S.bar_r[slot]);
                mbar_expect_tx(&S.bar_xf[slot], ZERO ? PLANE_BYTES : 2u * PLANE_BYTES);
                tma_box(S.f[slot], &tm_f, i0 - OX, j0 - 2, z, &S.bar_xf[slot]);
                if (!ZERO) tma_box(S.x[slot], &tm_x, i0 - OX, j0 - 2, z, &S.bar_xf[slot]);
                S.issued = q;
            }
            __syncwarp();
        }
    } else {
        // ---------------- compute warps ----------------
        // fixed per-thread cells (CPT per thread). First colour: ring cells
        // u = tid + h W1 (ring row u / 17, pair u % 17), at column offset e0
        // in its pair on even steps and 1 - e0 on odd ones. Second colour: tile
        // cells t = tid - W1 + h W2 (row t / 16, pair t % 16) likewise, on the
        // plane two behind.
        const bool grp1 = tid < W1;
        int ce[CPT], cn[CPT], g2[CPT], e0[CPT];
        bool act[CPT];
#pragma unroll
        for (int h = 0; h < CPT; ++h) {
            if (grp1) {
                const int u = tid + h * W1;
                act[h] = u < NPL;
                const int b1 = u / RXH, m = u - b1 * RXH;
                ce[h] = (b1 + 1) * HX + 2 * m + OX - 1;
                cn[h] = b1 * RXH + m;
                e0[h] = (c0 + b1 + z0) & 1;
                g2[h] = 0;
            } else {
                const int t = tid - W1 + h * W2;
                const int tb = t >> 4, m = t & 15;
                act[h] = (j0 + tb < g.ny) && (i0 + 2 * m < g.nx);
                ce[h] = (tb + 2) * HX + 2 * m + OX;
                cn[h] = (tb + 1) * RXH + m;
                e0[h] = (1 + c0 + tb + z0) & 1;
                g2[h] = (z0 - 3) * sz + (j0 + tb) * g.nx + i0 + 2 * m;   // plane of step 1
            }
        }
        // q of the second-colour cells (fused dots), one plane ahead
        const bool want_q = A.dots && !first_it && !grp1;
        float2 qv[CPT];
#pragma unroll
        for (int h = 0; h < CPT; ++h) qv[h] = make_float2(0.f, 0.f);
        if (want_q && z0 < z1) {
#pragma unroll
            for (int h = 0; h < CPT; ++h)
                if (act[h]) qv[h] = __ldg(reinterpret_cast<const float2*>(A.q + g2[h] + 3 * sz));
        }
        // tiles across a seam: the compute threads copy chunks tid, tid + NC,
        // ... of each staged plane (16 bytes, wrapped address; a chunk never
        // straddles the seam: nx and the tile origin are multiples of 4), PD_E
        // planes ahead, and the slot's full mbarriers track those copies
        constexpr int PD_E = 4;
        constexpr int CH = (C::NCH + NC - 1) / NC;   // chunks per thread and array
        bool has_chunk[CH];
        int c_off[CH], c_so[CH];
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const int ch = tid + k * NC;
            has_chunk[k] = !tma && ch < C::NCH;
            const int r = ch / CPR, a = 4 * (ch - r * CPR);
            c_off[k] = has_chunk[k] ? modp(j0 - 2 + r, g.ny) * g.nx + modp(i0 - OX + a, g.nx) : 0;
            c_so[k] = has_chunk[k] ? r * HX + a : 0;
        }
        auto copy_plane = [&](int q) {
            if (q > QMAX) return;
            const int slot = q & (RING - 1);
            const size_t gz = (size_t)modp(P0 + q, g.nz) * sz;
#pragma unroll
            for (int k = 0; k < CH; ++k)
                if (has_chunk[k])
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(
                                     su32(S.rho[slot] + c_so[k])),
                                 "l"(A.rho + gz + c_off[k])
                                 : "memory");
            cp_async_arrive(&S.bar_r[slot]);
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                if (!has_chunk[k]) continue;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(
                                 su32(S.f[slot] + c_so[k])),
                             "l"(A.f + gz + c_off[k])
                             : "memory");
                if (!ZERO)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(
                                     su32(S.x[slot] + c_so[k])),
                                 "l"(A.xin + gz + c_off[k])
                                 : "memory");
            }
            cp_async_arrive(&S.bar_xf[slot]);
            if (tid == 0) S.issued = q;
        };
        if (!tma)
            for (int q = 0; q <= PD_E; ++q) copy_plane(q);
        // planes 0 and 1 landed
        if (!(mbar_wait(&S.bar_xf[0], 0) && mbar_wait(&S.bar_xf[1], 0) &&
              mbar_wait(&S.bar_r[0], 0) && mbar_wait(&S.bar_r[1], 0)))
            *abort = 1;

#pragma unroll 2
        for (int s = 1; s <= SMAX; ++s) {
            // plane s + 1 landed (the first colour on plane s reads s - 1 .. s + 1)
            if (s + 1 <= QMAX) {
                const unsigned par = (unsigned)((s + 1) >> 3) & 1u;
                const bool w1 = mbar_wait(&S.bar_r[(s + 1) & (RING - 1)], par);
                const bool w2 = mbar_wait(&S.bar_xf[(s + 1) & (RING - 1)], par);
                if (!(w1 && w2)) *abort = 1;
            }
            compute_sync<NC>();   // step s - 1 done by every compute warp
            if (*abort) break;
            if (!tma) copy_plane(s + PD_E);   // slot of plane s - 4, last read in step s - 1
            const int odd = s & 1;
            if (grp1) {
                if (s + 1 <= QMAX) {   // first colour on plane s (k = P0 + s <= z1)
                    const int oc = (s & (RING - 1)) * PLANE;
                    const int om = ((s - 1) & (RING - 1)) * PLANE;
                    const int op = ((s + 1) & (RING - 1)) * PLANE;
                    float* Nn = S.n[s & (RN - 1)];
#pragma unroll
                    for (int h = 0; h < CPT; ++h) {
                        if (!act[h]) continue;
                        const int c = ce[h] + (e0[h] ^ odd);
                        const float* cc = B + oc + c;
                        const float* cm = B + om + c;
                        const float* cp = B + op + c;
                        const float rc = cc[0];
                        float w[6];
                        w[0] = rcp_approx(rc + cc[-1]);
                        w[1] = rcp_approx(rc + cc[1]);
                        w[2] = rcp_approx(rc + cc[-HX]);
                        w[3] = rcp_approx(rc + cc[HX]);
                        w[4] = rcp_approx(rc + cm[0]);
                        w[5] = rcp_approx(rc + cp[0]);
                        const float diag = w[0] + w[1] + w[2] + w[3] + w[4] + w[5];
                        float num = cc[F_OFF] * fs;
                        if (!ZERO) {
                            const float* xc = cc + X_OFF;
                            num += w[0] * xc[-1] + w[1] * xc[1] + w[2] * xc[-HX] + w[3] * xc[HX] +
                                   w[4] * cm[X_OFF] + w[5] * cp[X_OFF];
                        }
                        Nn[cn[h]] = num * rcp_approx(diag);
                    }
                }
            } else if (s >= 4) {   // second colour on plane s - 2 (k = P0 + s - 2 >= z0)
                const int ob = ((s - 2) & (RING - 1)) * PLANE;
                const int obm = ((s - 3) & (RING - 1)) * PLANE;
                const int obp = ((s - 1) & (RING - 1)) * PLANE;
                const float* Nb = S.n[(s - 2) & (RN - 1)];
                const float* Nbm = S.n[(s - 3) & (RN - 1)];
                const float* Nbp = S.n[(s - 1) & (RN - 1)];
                const bool more = s + 1 <= SMAX;   // another second-colour plane follows
#pragma unroll
                for (int h = 0; h < CPT; ++h) {
                    const int s2 = e0[h] ^ odd;    // column offset of the cell in its pair
                    const int c = ce[h] + s2;
                    const float* cc = B + ob + c;
                    const float rc = cc[0];
                    float w[6];
                    w[0] = rcp_approx(rc + cc[-1]);
                    w[1] = rcp_approx(rc + cc[1]);
                    w[2] = rcp_approx(rc + cc[-HX]);
                    w[3] = rcp_approx(rc + cc[HX]);
                    w[4] = rcp_approx(rc + B[obm + c]);
                    w[5] = rcp_approx(rc + B[obp + c]);
                    const float diag = w[0] + w[1] + w[2] + w[3] + w[4] + w[5];
                    const float* nc = Nb + cn[h];
                    const float num = cc[F_OFF] * fs + w[0] * nc[0] + w[1] * nc[1] +
                                      w[2] * nc[s2 - RXH] + w[3] * nc[s2 + RXH] +
                                      w[4] * Nbm[cn[h] + s2] + w[5] * Nbp[cn[h] + s2];
                    const float v2 = num * rcp_approx(diag);
                    const float other = nc[1 - s2];
                    const float v_even = s2 == 0 ? v2 : other;
                    const float v_odd = s2 == 1 ? v2 : other;
                    if (act[h]) {
                        *reinterpret_cast<float2*>(A.xout + g2[h]) = make_float2(v_even, v_odd);
                        if (A.dots) {
                            const float* fp = B + F_OFF + ob + ce[h];
                            rz += fp[0] * v_even + fp[1] * v_odd;
                            if (want_q) {
                                zq += v_even * qv[h].x + v_odd * qv[h].y;
                                if (more)
                                    qv[h] = __ldg(reinterpret_cast<const float2*>(A.q + g2[h] + sz));
                            }
                        }
                    }
                }
            }
            if (!grp1) {
#pragma unroll
                for (int h = 0; h < CPT; ++h) g2[h] += sz;
            }
            // this warp is done with plane s - 3: release its ring slot
            __syncwarp();
            if (lane == 0 && s >= 3) mbar_arrive(&S.bar_empty[(s - 3) & (RING - 1)]);
        }
    }
    __syncthreads();   // producer and compute warps

    if (S.abort) {
        // a wait gave up: latch the timeout, then let the copies still in
        // flight land (bounded) before the shared memory is released; the
        // last plane issued into each ring slot is one of the last RING issued
        if (tid == 0) {
            A.st->status = PF_ERR_TIMEOUT;
            A.st->done = 1;
            const int last = S.issued;
            for (int q = max(0, last - (RING - 1)); q <= last; ++q) {
                const unsigned par = (unsigned)(q >> 3) & 1u;
                mbar_wait(&S.bar_xf[q & (RING - 1)], par, kWaitNs / 10);
                mbar_wait(&S.bar_r[q & (RING - 1)], par, kWaitNs / 10);
            }
        }
    }
    if (A.dots) {
        double v[2] = {double(rz), double(zq)}, tot[2];
        const int mode[2] = {0, 0};
        const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        const int nb = gridDim.x * gridDim.y * gridDim.z;
        if (grid_reduce_lin<2>(v, mode, A.rb, tot, bid, nb) && threadIdx.x == 0) {
            CGScalars* scw = A.scw;
            scw->beta = first_it ? 0.0 : -scw->alpha * tot[1] / scw->rz;
            scw->rz = tot[0];
        }
    }
}

template <bool ZERO, int TY, int CPT>
void tma_attributes() {
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_sweep3d_tma<ZERO, TY, CPT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(ZERO ? smem_zero<TY>() : smem_full<TY>()));
        cudaFuncSetAttribute(k_sweep3d_tma<ZERO, TY, CPT>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    });
}

}  // namespace

struct SweepTMA {
    int stall;            // PF_TEST_SWEEP_STALL was set at creation (test of the bounded wait)
    int ty;               // tile height, 8 or 16
    int cpt_zero;         // cells per thread and plane of zero-start sweeps, 1 or 2
    int cpt_full;         // the same for sweeps from a given x_in
    Dims g;
    CUtensorMap rho, f, xa, xb;
    const float* rho_p;
    const float* f_p;
    const float* xa_p;
    const float* xb_p;
};

// Eligible: 3D, even sizes (consistent colouring), rows of whole 16-byte
// chunks (nx % 4 == 0) and a staged row that wraps at most once (nx >= 40).
bool sweep_tma_ok(const Dims& g) {
    return g.nz >= 4 && g.nx % 4 == 0 && g.nx >= HX && g.ny % 2 == 0 && g.ny >= 4 &&
           g.nz % 2 == 0 && (long long)g.ncell < (1LL << 31);
}

SweepTMA* sweep_tma_create(const Dims& g, const float* rho, const float* f, const float* xa,
                           const float* xb, int tile) {
    if (!sweep_tma_ok(g)) return nullptr;
    SweepTMA* t = new (std::nothrow) SweepTMA;
    if (!t) return nullptr;
    t->g = g;
    t->rho_p = rho;
    t->f_p = f;
    t->xa_p = xa;
    t->xb_p = xb;
    // tile shapes (pf_params.sweep_tile), cells per thread of zero-start /
    // other sweeps: 0 32 x 8, two / one; 1 32 x 8, two; 2 32 x 16, two;
    // 3 32 x 16, one; 4 32 x 8, one. 32 x 16 tiles need a staged plane's 20
    // rows within the grid (else 32 x 8).
    const bool tall = (tile == 2 || tile == 3) && g.ny >= TileCfg<16, 1>::HY;
    t->ty = tall ? 16 : 8;
    t->cpt_zero = (tile == 3 || tile == 4) ? 1 : 2;
    t->cpt_full = (tile == 1 || tile == 2) ? 2 : 1;
    t->stall = std::getenv("PF_TEST_SWEEP_STALL") != nullptr ? 1 : 0;
    const int hy = t->ty + 4;
    if (!encode_plane_map(&t->rho, g, rho, hy) || !encode_plane_map(&t->f, g, f, hy) ||
        !encode_plane_map(&t->xa, g, xa, hy) || !encode_plane_map(&t->xb, g, xb, hy)) {
        delete t;
        return nullptr;
    }
    return t;
}

void sweep_tma_destroy(SweepTMA* t) { delete t; }


void sweep_tma_prepare() {
    tma_attributes<true, 8, 2>();
    tma_attributes<false, 8, 2>();
    tma_attributes<true, 8, 1>();
    tma_attributes<false, 8, 1>();
    tma_attributes<true, 16, 2>();
    tma_attributes<false, 16, 2>();
    tma_attributes<true, 16, 1>();
    tma_attributes<false, 16, 1>();
}

namespace {
template <int TY, int CPT>
void launch_tiles(const SweepTMA* t, const CUtensorMap* tx, TmaArgs& a, bool zero,
                  const SweepDots* dots, bool* ok, const CGScalars* sc, cudaStream_t s) {
    const Dims& g = t->g;
    int zc = 32;
    const long long cols = (long long)((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    while (zc > 2 && cols * ((g.nz + zc - 1) / zc) < 8 * 152) zc >>= 1;
    if (zc == 32 && cols * ((g.nz + 63) / 64) >= 8 * 152) zc = 64;
    a.zc = zc;
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + zc - 1) / zc);
    *ok = !(dots && 2LL * grid.x * grid.y * grid.z > (long long)kRedPart);
    if (!*ok) return;
    if (zero) {
        tma_attributes<true, TY, CPT>();
        k_sweep3d_tma<true, TY, CPT>
            <<<grid, TileCfg<TY, CPT>::NT, smem_zero<TY>(), s>>>(t->rho, t->f, *tx, a, sc);
    } else {
        tma_attributes<false, TY, CPT>();
        k_sweep3d_tma<false, TY, CPT>
            <<<grid, TileCfg<TY, CPT>::NT, smem_full<TY>(), s>>>(t->rho, t->f, *tx, a, sc);
    }
}
}  // namespace

bool launch_sweep_tma(const SweepTMA* t, const MGLevel<float>& L, const float* xin, float* xout,
                      const SweepDots* dots, int first_color, const CGScalars* sc,
                      cudaStream_t s) {
    if (!t || L.f != t->f_p) return false;
    if (sc == nullptr) return false;   // the timeout status needs the solve's scalars
    const CUtensorMap* tx = &t->xa;   // unused for a zero start
    if (xin != nullptr) {
        if (xin == t->xa_p) tx = &t->xa;
        else if (xin == t->xb_p) tx = &t->xb;
        else return false;
    }
    TmaArgs a;
    a.g = t->g;
    a.rho = t->rho_p;
    a.f = t->f_p;
    a.xin = xin;
    a.xout = xout;
    a.fs = float(0.5 * t->g.h * t->g.h);
    a.first_color = first_color;
    a.dots = dots != nullptr;
    a.first = dots ? dots->first : 0;
    a.q = dots ? dots->q : nullptr;
    a.rb = dots ? dots->rb : RedBuf{nullptr, nullptr};
    a.scw = dots ? dots->sc : nullptr;
    a.st = const_cast<CGScalars*>(sc);
    a.stall = t->stall;
    bool ok = false;
    const bool zero = xin == nullptr;
    const int cpt = zero ? t->cpt_zero : t->cpt_full;
    if (t->ty == 16 && cpt == 2)
        launch_tiles<16, 2>(t, tx, a, zero, dots, &ok, sc, s);
    else if (t->ty == 16)
        launch_tiles<16, 1>(t, tx, a, zero, dots, &ok, sc, s);
    else if (cpt == 2)
        launch_tiles<8, 2>(t, tx, a, zero, dots, &ok, sc, s);
    else
        launch_tiles<8, 1>(t, tx, a, zero, dots, &ok, sc, s);
    return ok;
}

}  // namespace pf
