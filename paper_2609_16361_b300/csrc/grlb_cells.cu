// grlb_cells.cu -- populations of listed cells (point probes of the state).
//
// The state of a domain is the set of post-collision populations f*_{k,i}(x) of every cell
// (what a pull sweep writes at x).  Where they sit depends on the streaming pattern:
//   two buffers:                   slot i of x in the current buffer;
//   one buffer, even steps done:   slot opp(i) of x (the AA-even write, and the initial state);
//   one buffer, odd steps done:    slot i of x + c_i (the AA-odd push), or, for the +x / -x
//                                  populations leaving an X_DIRICHLET_EQ tube, the outflow
//                                  record [side][k][y + ny z];
//   moments:                       rebuilt from the cell's own w_1 Q_k, J*_k (mom_at layout).
// One thread per (population row, listed cell): out[q n + j] = f_q(cells[j]) in FP64 lattice
// units, the stored deviation decoded and the reference equilibrium added back.
#include <cuda_runtime.h>

#include "grlb_device.cuh"
#include "grlb_kernels.h"

namespace grlb {

template <int S>
__global__ void __launch_bounds__(256) read_cells_kernel(const __grid_constant__ DomainDev D, const void* buf_v,
                                                         const int64_t* __restrict__ cells, int64_t n, int layout,
                                                         const __grid_constant__ CellDecode dec,
                                                         double* __restrict__ out) {
    using T = typename Store<S>::T;
    const T* buf = static_cast<const T*>(buf_v);
    const T* outflow = static_cast<const T*>(D.outflow);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < NP * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(t / n);
        const int64_t j = t - (int64_t)q * n;
        const int k = q / NQ, i = q - NQ * k;
        const int64_t c = GRLB_LD(cells + j);  // in [0, N): checked by the host
        const int64_t nx = D.nx, ny = D.ny, nz = D.nz;
        const int64_t x = c % nx, r = c / nx, y = r % ny, z = r / ny;
        const T* src;
        if (layout == 3) {  // moments: f*_q rebuilt from the cell's own Q_k, J*_k
            const T* m = buf + mom_at(c) + (int64_t)(4 * k) * kBrick;
            const float mq = Store<S>::ld(m);
            const float v = i == 0 ? 2.0f * mq  // mq = w_1 Q_k
                                   : fmaf(((i & 1) ? 0.5f : -0.5f), Store<S>::ld(m + (1 + ((i - 1) >> 1)) * kBrick), mq);
            GRLB_ST(out + t, fma((double)v, dec.dec[k], dec.shift[q]));
            continue;
        }
        if (layout == 0) {
            src = buf + brick_at(c) + (int64_t)q * kBrick;
        } else if (layout == 1) {
            const int o = i == 0 ? 0 : (i & 1 ? i + 1 : i - 1);  // opp(i)
            src = buf + brick_at(c) + (int64_t)(NQ * k + o) * kBrick;
        } else {
            int64_t xs = x, ys = y, zs = z;
            if (i == 1) xs = x + 1 == nx ? 0 : x + 1;
            if (i == 2) xs = x == 0 ? nx - 1 : x - 1;
            if (i == 3) ys = y + 1 == ny ? 0 : y + 1;
            if (i == 4) ys = y == 0 ? ny - 1 : y - 1;
            if (i == 5) zs = z + 1 == nz ? 0 : z + 1;
            if (i == 6) zs = z == 0 ? nz - 1 : z - 1;
            const int64_t yz = y + ny * z;
            if (D.bc == 1 && i == 1 && x == nx - 1) src = outflow + (5 + k) * ny * nz + yz;
            else if (D.bc == 1 && i == 2 && x == 0) src = outflow + k * ny * nz + yz;
            else src = buf + brick_at(xs + nx * (ys + ny * zs)) + (int64_t)q * kBrick;
        }
        const float v = Store<S>::ld(src);
        GRLB_ST(out + t, fma((double)v, dec.dec[k], dec.shift[q]));
    }
}

cudaError_t launch_read_cells(const DomainDev& D, int storage, const void* buf, const int64_t* cells, int64_t n,
                              int layout, const CellDecode& dec, double* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    int64_t blocks = (NP * n + threads - 1) / threads;
    if (blocks > 148 * 16) blocks = 148 * 16;
    if (storage == S_F32)
        read_cells_kernel<S_F32><<<(int)blocks, threads, 0, st>>>(D, buf, cells, n, layout, dec, out);
    else if (storage == S_F16)
        read_cells_kernel<S_F16><<<(int)blocks, threads, 0, st>>>(D, buf, cells, n, layout, dec, out);
    else
        read_cells_kernel<S_BF16><<<(int)blocks, threads, 0, st>>>(D, buf, cells, n, layout, dec, out);
    return cudaGetLastError();
}

}  // namespace grlb
