// Device helpers for kernels that stage planes into shared memory with the
// Tensor Memory Accelerator (tiled cp.async.bulk.tensor copies completing on
// mbarriers) and wait on mbarriers with a time bound, and the host-side
// encoding of a tensor map of one float32 array of a 3D grid.
#pragma once

#include <cuda.h>

#include <mutex>

#include "pf_device.cuh"

namespace pf {
namespace tma {

constexpr long long kWaitNs = 1000000000LL;   // bound of one mbarrier wait

__device__ __forceinline__ int modp(int a, int m) { int r = a % m; return r < 0 ? r + m : r; }
__device__ __forceinline__ unsigned su32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Same test, but a thread whose phase is not complete is suspended until it
// completes or about `hint_ns` nanoseconds pass (no busy polling meanwhile).
__device__ __forceinline__ bool mbar_try_wait_sleep(unsigned long long* b, unsigned parity,
                                                    unsigned hint_ns) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}
constexpr unsigned kSuspendNs = 20000;   // one suspended test: 20 us at most
__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits for the phase of parity `parity` of b to complete; false after about
// `limit` nanoseconds without completion.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity,
                                          long long limit = kWaitNs) {
    if (mbar_try_wait(b, parity)) return true;
    const long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait_sleep(b, parity, kSuspendNs)) return true;
        if (global_ns() - t0 > limit) return false;
    }
}
__device__ __forceinline__ void tma_box(float* dst, const CUtensorMap* tm, int x, int y, int z,
                                        unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(su32(dst)),
        "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(z), "r"(su32(bar))
        : "memory");
}
// the barrier's pending count drops when this thread's earlier cp.async land
__device__ __forceinline__ void cp_async_arrive(unsigned long long* b) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(su32(b)) : "memory");
}

// Bounded wait for the phase of parity `parity` of b that also gives up when
// the CTA aborted (the producer warp waits on slots the compute warps release).
__device__ __forceinline__ bool mbar_wait_or_abort(unsigned long long* b, unsigned parity,
                                                   const volatile int* abort) {
    if (mbar_try_wait(b, parity)) return true;
    const long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait_sleep(b, parity, kSuspendNs)) return true;
        if (*abort || global_ns() - t0 > kWaitNs) return false;
    }
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
// barrier of the compute warps (the producer warp runs on its own)
template <int NC>
__device__ __forceinline__ void compute_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(NC) : "memory");
}

}  // namespace tma

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

// tensor map of one float32 array of the grid, box bx x hy x 1 (a staged plane)
inline bool encode_plane_map(CUtensorMap* m, const Dims& g, const float* base, int hy,
                             int bx = 40) {
    EncodeTiled fn = encoder();
    if (!fn || !base) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nx * 4u, (cuuint64_t)g.nx * g.ny * 4u};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)hy, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace
}  // namespace pf
