// grlb_check.cu -- the registry of live regions behind the checked build's access tests
// (grlb_check.cuh).  Empty in the plain build.
#include "grlb_check.cuh"

#include <memory>

#ifdef GRLB_CHECKED
namespace grlb {

__device__ ChkState g_chk;
__device__ __align__(64) unsigned long long g_chk_zero[8];
__device__ __align__(64) unsigned long long g_chk_sink[8];

__device__ bool chk_access(const void* p, unsigned bytes) {
    const unsigned long long a = reinterpret_cast<unsigned long long>(p);
    const int top = *static_cast<volatile int*>(&g_chk.top);
    const volatile unsigned long long* lo = g_chk.lo;
    const volatile unsigned long long* hi = g_chk.hi;
    for (int i = 0; i < top; ++i) {
        const unsigned long long h = hi[i];
        if (h > 1 && a >= lo[i] && a + bytes <= h) return true;
    }
    if (atomicAdd(&g_chk.violations, 1ull) == 0ull) atomicExch(&g_chk.first, a);
    return false;
}

// One thread: claim a free slot (hi 0 -> 1), write lo, then publish hi.
__global__ void chk_register_kernel(unsigned long long lo, unsigned long long hi) {
    for (int i = 0; i < kChkRegions; ++i) {
        if (atomicCAS(&g_chk.hi[i], 0ull, 1ull) == 0ull) {
            g_chk.lo[i] = lo;
            __threadfence();
            atomicMax(&g_chk.top, i + 1);
            __threadfence();
            atomicExch(&g_chk.hi[i], hi);
            return;
        }
    }
    atomicAdd(&g_chk.overflow, 1ull);
}

__global__ void chk_release_kernel(unsigned long long lo) {
    const int top = *static_cast<volatile int*>(&g_chk.top);
    for (int i = 0; i < top; ++i) {
        const unsigned long long h = *static_cast<volatile unsigned long long*>(&g_chk.hi[i]);
        if (h > 1 && *static_cast<volatile unsigned long long*>(&g_chk.lo[i]) == lo) {
            atomicExch(&g_chk.hi[i], 0ull);
            return;
        }
    }
    atomicAdd(&g_chk.unmatched, 1ull);
}

__global__ void chk_probe_kernel(const void* p, unsigned bytes) { chk_access(p, bytes); }

cudaError_t chk_register(const void* p, size_t bytes, cudaStream_t st) {
    if (!p || bytes == 0) return cudaSuccess;
    const unsigned long long lo = reinterpret_cast<unsigned long long>(p);
    chk_register_kernel<<<1, 1, 0, st>>>(lo, lo + bytes);
    return cudaGetLastError();
}

cudaError_t chk_release(const void* p, cudaStream_t st) {
    if (!p) return cudaSuccess;
    chk_release_kernel<<<1, 1, 0, st>>>(reinterpret_cast<unsigned long long>(p));
    return cudaGetLastError();
}

cudaError_t chk_probe(const void* p, size_t bytes, cudaStream_t st) {
    chk_probe_kernel<<<1, 1, 0, st>>>(p, (unsigned)bytes);
    return cudaGetLastError();
}

cudaError_t chk_read(ChkCounts* out, bool reset) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    std::unique_ptr<ChkState> hp(new ChkState);  // 64 KB: kept off the host stack
    ChkState& h = *hp;
    e = cudaMemcpyFromSymbol(&h, g_chk, sizeof h);
    if (e != cudaSuccess) return e;
    out->violations = h.violations;
    out->first = h.first;
    out->unmatched = h.unmatched;
    out->overflow = h.overflow;
    out->live = 0;
    for (int i = 0; i < h.top && i < kChkRegions; ++i) out->live += h.hi[i] > 1 ? 1 : 0;
    if (reset) {
        const unsigned long long zero[4] = {0ull, 0ull, 0ull, 0ull};
        e = cudaMemcpyToSymbol(g_chk, zero, sizeof zero);  // the four counters lead the record
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    return e;
}

}  // namespace grlb
#endif
