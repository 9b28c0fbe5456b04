// grlb_halo.cu -- ghost-plane exchange of z-slabs (one domain split along z).
//
// A slab of nz interior planes lives in an ordinary periodic domain of nz + 2 planes: ghost
// plane 0 below, nz + 1 above.  In a pull sweep an interior cell reads from a ghost plane only
// the population travelling into the slab: f_{k,+z} from plane 0 (into plane 1) and f_{k,-z}
// from plane nz + 1 (into plane nz).  So the exchange copies, for the five fields k, the +z
// population of the lower slab's top interior plane into the upper slab's plane 0, and the -z
// population of the upper slab's bottom interior plane into the lower slab's top ghost plane;
// the interior cells then compute exactly what the undivided domain computes.  One launch per
// pair: 10 slices of nx ny elements (2 x 5 fields).
#include <cuda_runtime.h>

#include "grlb_device.cuh"
#include "grlb_kernels.h"

namespace grlb {

template <typename T>
__global__ void __launch_bounds__(256) halo_z_kernel(T* __restrict__ lower, T* __restrict__ upper, int nzl,
                                                     int64_t nxy) {
    // slices: s < 5: +z of field s, lower top interior (z = nzl - 2) -> upper ghost (z = 0);
    //         s >= 5: -z of field s - 5, upper bottom interior (z = 1) -> lower ghost (z = nzl - 1)
    // (cell bricks: population q of cell c at brick_at(c) + q kBrick)
    const int s = blockIdx.y;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nxy; c += (int64_t)gridDim.x * blockDim.x) {
        if (s < 5) {
            const int64_t q = (7 * s + 5) * kBrick;
            GRLB_ST(upper + brick_at(c) + q, GRLB_LD(lower + brick_at((int64_t)(nzl - 2) * nxy + c) + q));
        } else {
            const int64_t q = (7 * (s - 5) + 6) * kBrick;
            GRLB_ST(lower + brick_at((int64_t)(nzl - 1) * nxy + c) + q, GRLB_LD(upper + brick_at(nxy + c) + q));
        }
    }
}

cudaError_t launch_halo_z(void* lower, void* upper, int nzl, int64_t nxy, size_t elem, cudaStream_t st) {
    int64_t blocks = (nxy + 255) / 256;
    if (blocks > 148 * 4) blocks = 148 * 4;
    const dim3 grid((unsigned)blocks, 10);
    if (elem == 4)
        halo_z_kernel<float><<<grid, 256, 0, st>>>(static_cast<float*>(lower), static_cast<float*>(upper), nzl, nxy);
    else
        halo_z_kernel<unsigned short><<<grid, 256, 0, st>>>(static_cast<unsigned short*>(lower),
                                                            static_cast<unsigned short*>(upper), nzl, nxy);
    return cudaGetLastError();
}

// Ghost exchange between slabs on different devices: the sender packs its two outgoing slices
// into contiguous buffers (5 fields x nx ny, field-major), the buffers travel between ranks, and
// the receiver unpacks them into its ghost planes.  Same slices as halo_z_kernel.
template <typename T>
__global__ void __launch_bounds__(256) halo_pack_kernel(const T* __restrict__ f, T* __restrict__ to_upper,
                                                        T* __restrict__ to_lower, int nz, int64_t nxy) {
    const int s = blockIdx.y;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nxy; c += (int64_t)gridDim.x * blockDim.x) {
        if (s < 5) GRLB_ST(to_upper + s * nxy + c, GRLB_LD(f + brick_at((int64_t)(nz - 2) * nxy + c) + (7 * s + 5) * kBrick));
        else GRLB_ST(to_lower + (s - 5) * nxy + c, GRLB_LD(f + brick_at(nxy + c) + (7 * (s - 5) + 6) * kBrick));
    }
}

template <typename T>
__global__ void __launch_bounds__(256) halo_unpack_kernel(T* __restrict__ f, const T* __restrict__ from_lower,
                                                          const T* __restrict__ from_upper, int nz, int64_t nxy) {
    const int s = blockIdx.y;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nxy; c += (int64_t)gridDim.x * blockDim.x) {
        if (s < 5) GRLB_ST(f + brick_at(c) + (7 * s + 5) * kBrick, GRLB_LD(from_lower + s * nxy + c));
        else GRLB_ST(f + brick_at((int64_t)(nz - 1) * nxy + c) + (7 * (s - 5) + 6) * kBrick, GRLB_LD(from_upper + (s - 5) * nxy + c));
    }
}

cudaError_t launch_halo_pack_z(const void* f, void* to_upper, void* to_lower, int nz, int64_t nxy, size_t elem,
                               cudaStream_t st) {
    int64_t blocks = (nxy + 255) / 256;
    if (blocks > 148 * 4) blocks = 148 * 4;
    const dim3 grid((unsigned)blocks, 10);
    if (elem == 4)
        halo_pack_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(f), static_cast<float*>(to_upper),
                                                      static_cast<float*>(to_lower), nz, nxy);
    else
        halo_pack_kernel<unsigned short><<<grid, 256, 0, st>>>(static_cast<const unsigned short*>(f),
                                                               static_cast<unsigned short*>(to_upper),
                                                               static_cast<unsigned short*>(to_lower), nz, nxy);
    return cudaGetLastError();
}

cudaError_t launch_halo_unpack_z(void* f, const void* from_lower, const void* from_upper, int nz, int64_t nxy,
                                 size_t elem, cudaStream_t st) {
    int64_t blocks = (nxy + 255) / 256;
    if (blocks > 148 * 4) blocks = 148 * 4;
    const dim3 grid((unsigned)blocks, 10);
    if (elem == 4)
        halo_unpack_kernel<float><<<grid, 256, 0, st>>>(static_cast<float*>(f), static_cast<const float*>(from_lower),
                                                        static_cast<const float*>(from_upper), nz, nxy);
    else
        halo_unpack_kernel<unsigned short><<<grid, 256, 0, st>>>(static_cast<unsigned short*>(f),
                                                                 static_cast<const unsigned short*>(from_lower),
                                                                 static_cast<const unsigned short*>(from_upper), nz,
                                                                 nxy);
    return cudaGetLastError();
}

// ---- moment storage ------------------------------------------------------------------------
// A pull from a ghost plane reads Q_k / 8 and J*_k,z of the ghost cell (the +z population from plane
// 0, the -z one from plane nz - 1), so the exchange carries those two of the four moment rows
// per field: slice 2 k + h holds row 4 k (h = 0, w_1 Q_k) or 4 k + 3 (h = 1, J*_k,z), 10 slices of
// nx ny values per direction.
__device__ __forceinline__ int mom_halo_row(int slice) { return 4 * (slice >> 1) + ((slice & 1) ? 3 : 0); }

__global__ void __launch_bounds__(256) halo_z_mom_kernel(float* __restrict__ lower, float* __restrict__ upper,
                                                         int nzl, int64_t nxy) {
    const int s = blockIdx.y % 10, row = mom_halo_row(s);
    const bool up = blockIdx.y < 10;  // lower top interior -> upper ghost plane 0
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nxy; c += (int64_t)gridDim.x * blockDim.x) {
        if (up) GRLB_ST(upper + mom_at(c) + row * kBrick, GRLB_LD(lower + mom_at((int64_t)(nzl - 2) * nxy + c) + row * kBrick));
        else GRLB_ST(lower + mom_at((int64_t)(nzl - 1) * nxy + c) + row * kBrick, GRLB_LD(upper + mom_at(nxy + c) + row * kBrick));
    }
}

__global__ void __launch_bounds__(256) halo_pack_mom_kernel(const float* __restrict__ f, float* __restrict__ to_upper,
                                                            float* __restrict__ to_lower, int nz, int64_t nxy) {
    const int s = blockIdx.y % 10, row = mom_halo_row(s);
    const bool up = blockIdx.y < 10;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nxy; c += (int64_t)gridDim.x * blockDim.x) {
        if (up) GRLB_ST(to_upper + s * nxy + c, GRLB_LD(f + mom_at((int64_t)(nz - 2) * nxy + c) + row * kBrick));
        else GRLB_ST(to_lower + s * nxy + c, GRLB_LD(f + mom_at(nxy + c) + row * kBrick));
    }
}

__global__ void __launch_bounds__(256) halo_unpack_mom_kernel(float* __restrict__ f, const float* __restrict__ from_lower,
                                                              const float* __restrict__ from_upper, int nz, int64_t nxy) {
    const int s = blockIdx.y % 10, row = mom_halo_row(s);
    const bool low = blockIdx.y < 10;  // from the lower neighbour into ghost plane 0
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nxy; c += (int64_t)gridDim.x * blockDim.x) {
        if (low) GRLB_ST(f + mom_at(c) + row * kBrick, GRLB_LD(from_lower + s * nxy + c));
        else GRLB_ST(f + mom_at((int64_t)(nz - 1) * nxy + c) + row * kBrick, GRLB_LD(from_upper + s * nxy + c));
    }
}

static dim3 halo_grid(int64_t nxy, int slices) {
    int64_t blocks = (nxy + 255) / 256;
    if (blocks > 148 * 4) blocks = 148 * 4;
    return dim3((unsigned)blocks, slices);
}

cudaError_t launch_halo_z_mom(void* lower, void* upper, int nzl, int64_t nxy, cudaStream_t st) {
    halo_z_mom_kernel<<<halo_grid(nxy, 20), 256, 0, st>>>(static_cast<float*>(lower), static_cast<float*>(upper), nzl,
                                                          nxy);
    return cudaGetLastError();
}

cudaError_t launch_halo_pack_z_mom(const void* f, void* to_upper, void* to_lower, int nz, int64_t nxy,
                                   cudaStream_t st) {
    halo_pack_mom_kernel<<<halo_grid(nxy, 20), 256, 0, st>>>(static_cast<const float*>(f), static_cast<float*>(to_upper),
                                                             static_cast<float*>(to_lower), nz, nxy);
    return cudaGetLastError();
}

cudaError_t launch_halo_unpack_z_mom(void* f, const void* from_lower, const void* from_upper, int nz, int64_t nxy,
                                     cudaStream_t st) {
    halo_unpack_mom_kernel<<<halo_grid(nxy, 20), 256, 0, st>>>(static_cast<float*>(f), static_cast<const float*>(from_lower),
                                                               static_cast<const float*>(from_upper), nz, nxy);
    return cudaGetLastError();
}

}  // namespace grlb
