// grlb_check.cuh -- bounds checking of every global-memory access (the checked build).
//
// Compiled with -DGRLB_CHECKED (libgrlb_checked.so, relocatable device code so that all
// translation units share one registry), every load and store a kernel makes through the
// helpers below first tests its address range against a device-side registry of live regions:
// the library's own allocations (registered on the allocating stream right after
// cudaMallocAsync, released on the freeing stream right before cudaFreeAsync, so the
// registration brackets every stream-ordered use) and the caller's buffers lent to one call
// (registered and released around that call's kernels on its stream).  An access that lies in
// no live region is counted, its address kept (the first one), and not made: a load returns
// zero, a store goes to a sink.  The host reads the counters with grlb_check_read.
//
// In the plain build the helpers are the bare access and the registration calls are empty
// inline functions, so the product kernels compile exactly as without them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace grlb {

#ifdef GRLB_CHECKED
constexpr bool kChecked = true;
constexpr int kChkRegions = 4096;
struct ChkState {
    unsigned long long violations;  // accesses outside every live region (not made)
    unsigned long long first;       // address of the first such access
    unsigned long long unmatched;   // releases of a region that was not live
    unsigned long long overflow;    // registrations that found the table full
    int top;                        // slots [0, top) have been used
    int pad;
    // region i covers bytes [lo[i], hi[i]); hi[i] == 0: free slot, 1: being filled
    unsigned long long lo[kChkRegions];
    unsigned long long hi[kChkRegions];
};
extern __device__ ChkState g_chk;
// true if [p, p + bytes) lies inside one live region; otherwise counts a violation
__device__ bool chk_access(const void* p, unsigned bytes);
#else
constexpr bool kChecked = false;
#endif

// ---- checked access helpers --------------------------------------------------------------
// An access outside every live region is redirected, without a branch, to a pad: loads read the
// zero pad (never written), stores write the sink pad.  The range test itself is a call, which
// can keep the compiler from fusing a multiply with an add across it, so in-bounds results agree
// with the plain build to rounding (bit for bit where the same multiply-adds are fused).  In the
// plain build the macros are the bare access.
#ifdef GRLB_CHECKED
extern __device__ __align__(64) unsigned long long g_chk_zero[8];
extern __device__ __align__(64) unsigned long long g_chk_sink[8];
template <typename T>
__device__ __forceinline__ const T* chk_src(const T* p) {
    return chk_access(p, sizeof(T)) ? p : reinterpret_cast<const T*>(g_chk_zero);
}
template <typename T>
__device__ __forceinline__ T* chk_dst(T* p) {
    return chk_access(p, sizeof(T)) ? p : reinterpret_cast<T*>(g_chk_sink);
}
#define GRLB_CHK_SRC(p) (::grlb::chk_src(p))
#define GRLB_CHK_DST(p) (::grlb::chk_dst(p))
#else
#define GRLB_CHK_SRC(p) (p)
#define GRLB_CHK_DST(p) (p)
#endif
#define GRLB_LD(p) (*GRLB_CHK_SRC(p))
#define GRLB_LDG(p) (__ldg(GRLB_CHK_SRC(p)))
#define GRLB_ST(p, v) (*GRLB_CHK_DST(p) = (v))
#define GRLB_ATOMIC_ADD(p, v) (atomicAdd(GRLB_CHK_DST(p), (v)))

// ---- host side ------------------------------------------------------------------------------
struct ChkCounts {
    unsigned long long violations, first, unmatched, overflow;
    long long live;
};
#ifdef GRLB_CHECKED
// Stream-ordered: the region becomes live / stops being live when the stream reaches the call.
cudaError_t chk_register(const void* p, size_t bytes, cudaStream_t st);
cudaError_t chk_release(const void* p, cudaStream_t st);
// Synchronises the device, reads the counters (live: regions registered and not released) and
// optionally zeroes violations, first, unmatched and overflow.
cudaError_t chk_read(ChkCounts* out, bool reset);
// Tests [p, p + bytes) against the registry in a one-thread kernel on st, counting a violation
// if it lies outside every live region; the address is compared, never accessed.
cudaError_t chk_probe(const void* p, size_t bytes, cudaStream_t st);
#else
inline cudaError_t chk_register(const void*, size_t, cudaStream_t) { return cudaSuccess; }
inline cudaError_t chk_release(const void*, cudaStream_t) { return cudaSuccess; }
#endif

// Allocation and release with the registration beside them (plain cudaMallocAsync /
// cudaFreeAsync in the plain build).
inline cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t st) {
    cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e == cudaSuccess) e = chk_register(*p, bytes, st);
    return e;
}
template <typename T>
inline cudaError_t dev_alloc(T** p, size_t bytes, cudaStream_t st) {
    return dev_alloc(reinterpret_cast<void**>(p), bytes, st);
}
inline cudaError_t dev_free(void* p, cudaStream_t st) {
    if (!p) return cudaSuccess;
    cudaError_t e = chk_release(p, st);
    cudaError_t e2 = cudaFreeAsync(p, st);
    return e != cudaSuccess ? e : e2;
}

// A caller's buffer lent to the kernels of one call: live from construction to destruction,
// in the order of the stream (nothing in the plain build).
class Lent {
public:
    Lent(const void* p, size_t bytes, cudaStream_t st) : p_(kChecked && p && bytes ? p : nullptr), st_(st) {
        if (p_) err_ = chk_register(p_, bytes, st_);
    }
    ~Lent() {
        if (p_) chk_release(p_, st_);
    }
    Lent(const Lent&) = delete;
    Lent& operator=(const Lent&) = delete;
    cudaError_t error() const { return err_; }

private:
    const void* p_;
    cudaStream_t st_;
    cudaError_t err_ = cudaSuccess;
};

}  // namespace grlb
