// grlb_kernels.cu -- sweep, initialisation, readback and diagnostic-reduction kernels.
//
// Layout in HBM (per domain, per buffer): 35 planes of N = nx*ny*nz elements, plane index
// q = 7k + i (field k, link i), x fastest inside a plane.  One CTA covers a tile of
// blockDim.x consecutive cells of blockDim.y rows at one z; consecutive lanes touch
// consecutive addresses of every plane, so each of the 35 loads and 35 stores of a warp is a
// fully used 128-byte line (FP32).  The +-y / +-z pulls read whole neighbouring rows; the +-x
// pulls are the same row shifted by one element, served from L1/L2 lines already fetched for
// the row (no extra DRAM traffic).
#include <cuda_runtime.h>

#include "grlb_device.cuh"
#include "grlb_kernels.h"

namespace grlb {

struct PullIdx {
    int32_t c, xm, xp, ym, yp, zm, zp;  // cell offsets of the 7 pull sources
    bool gl, gr;                        // +x / -x source is a Dirichlet ghost
};

__device__ __forceinline__ PullIdx pull_index(const DomainDev& D, int x, int y, int z) {
    PullIdx P;
    const int nx = D.nx, ny = D.ny, nz = D.nz;
    const int row = (y + ny * z) * nx;
    const int xm = (x == 0) ? nx - 1 : x - 1;
    const int xp = (x == nx - 1) ? 0 : x + 1;
    const int ym = (y == 0) ? ny - 1 : y - 1;
    const int yp = (y == ny - 1) ? 0 : y + 1;
    const int zm = (z == 0) ? nz - 1 : z - 1;
    const int zp = (z == nz - 1) ? 0 : z + 1;
    P.c = row + x;
    P.xm = row + xm;
    P.xp = row + xp;
    P.ym = (ym + ny * z) * nx + x;
    P.yp = (yp + ny * z) * nx + x;
    P.zm = (y + ny * zm) * nx + x;
    P.zp = (y + ny * zp) * nx + x;
    P.gl = (D.bc == 1) && (x == 0);
    P.gr = (D.bc == 1) && (x == nx - 1);
    return P;
}

template <int S>
__device__ __forceinline__ void load_cell(const DomainDev& D, const typename Store<S>::T* __restrict__ fin,
                                          const PullIdx& P, float (&d)[NF][NQ]) {
    using St = Store<S>;
    const int64_t pl = D.plane;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const typename St::T* b = fin + (int64_t)(7 * k) * pl;
        const float sc = D.dec[k];
        d[k][0] = St::ld(b + P.c) * sc;
        d[k][1] = P.gl ? D.ghostL[k] : St::ld(b + pl + P.xm) * sc;
        d[k][2] = P.gr ? D.ghostR[k] : St::ld(b + 2 * pl + P.xp) * sc;
        d[k][3] = St::ld(b + 3 * pl + P.ym) * sc;
        d[k][4] = St::ld(b + 4 * pl + P.yp) * sc;
        d[k][5] = St::ld(b + 5 * pl + P.zm) * sc;
        d[k][6] = St::ld(b + 6 * pl + P.zp) * sc;
    }
}

template <int S>
__device__ __forceinline__ void store_cell(const DomainDev& D, typename Store<S>::T* __restrict__ fout,
                                           int32_t c, const float (&o)[NF][NQ]) {
    using St = Store<S>;
    const int64_t pl = D.plane;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const float sc = D.enc[k];
#pragma unroll
        for (int i = 0; i < NQ; ++i) St::st(fout + (int64_t)(7 * k + i) * pl + c, o[k][i] * sc);
    }
}

// Block-level FP64 reduction of the per-cell diagnostics into one NDIAG record.
// Order is fixed by the block shape: FP32 butterfly inside each warp (<= 32 cells), FP64
// across warps in warp order.  rec: [dQ0..4, ke, eps_s, eps_d, rho_min, p_min, n_floor,
// n_nan, n_sensor].
__device__ __forceinline__ void block_reduce_diag(const CellDiag& cd, bool active,
                                                  double* __restrict__ out) {
    __shared__ double sh[32][NDIAG];
    float v[8];
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] = active ? cd.dQ[k] : 0.0f;
    v[5] = active ? cd.ke : 0.0f;
    v[6] = active ? cd.eps_s : 0.0f;
    v[7] = active ? cd.eps_d : 0.0f;
    float rmin = active ? cd.rho_raw : 3.0e38f;
    float pmin = active ? cd.p_raw : 3.0e38f;
    int cnt[3] = {active ? cd.floored : 0, active ? cd.nan : 0, active ? cd.sensor : 0};
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
        rmin = fminf(rmin, __shfl_xor_sync(0xffffffffu, rmin, off));
        pmin = fminf(pmin, __shfl_xor_sync(0xffffffffu, pmin, off));
#pragma unroll
        for (int k = 0; k < 3; ++k) cnt[k] += __shfl_xor_sync(0xffffffffu, cnt[k], off);
    }
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 8; ++k) sh[warp][k] = (double)v[k];
        sh[warp][8] = (double)rmin;
        sh[warp][9] = (double)pmin;
#pragma unroll
        for (int k = 0; k < 3; ++k) sh[warp][10 + k] = (double)cnt[k];
    }
    __syncthreads();
    if (tid < NDIAG) {
        double acc = sh[0][tid];
        for (int w = 1; w < nwarps; ++w) {
            const double x = sh[w][tid];
            acc = (tid == 8 || tid == 9) ? fmin(acc, x) : acc + x;
        }
        out[tid] = acc;
    }
}

// ---- single-domain sweep -----------------------------------------------------------------
template <int S, int COLL, bool DIAG>
__global__ void __launch_bounds__(128) sweep_kernel(const __grid_constant__ DomainDev D,
                                                    const void* __restrict__ fin_v,
                                                    void* __restrict__ fout_v,
                                                    double* __restrict__ partials) {
    using T = typename Store<S>::T;
    const T* __restrict__ fin = static_cast<const T*>(fin_v);
    T* __restrict__ fout = static_cast<T*>(fout_v);
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    const bool active = (x < D.nx) && (y < D.ny);
    CellDiag cd;
    if (active) {
        const PullIdx P = pull_index(D, x, y, z);
        float d[NF][NQ], o[NF][NQ];
        load_cell<S>(D, fin, P, d);
        collide<COLL, DIAG>(D, d, o, &cd);
        store_cell<S>(D, fout, P.c, o);
    }
    if (DIAG) {
        const int64_t blk = blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
        block_reduce_diag(cd, active, partials + blk * NDIAG);
    }
}

// ---- batched sweep over a tile table -----------------------------------------------------
// tiles[t] = (domain, x0, y0, z); the domain record supplies buffers, constants and its
// tile width tile_x (one-dimensional CTA: thread t -> (x0 + t % tile_x, y0 + t / tile_x)).
// `parity` flips every step so that each domain reads buf[cur ^ parity], writes the other.
template <int S, int COLL>
__global__ void __launch_bounds__(128) batch_sweep_kernel(const DomainDev* __restrict__ doms,
                                                          const int4* __restrict__ tiles,
                                                          int parity) {
    using T = typename Store<S>::T;
    __shared__ DomainDev sD;
    const int4 tl = tiles[blockIdx.x];
    {
        const int nwords = sizeof(DomainDev) / 4;
        const uint32_t* src = reinterpret_cast<const uint32_t*>(doms + tl.x);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&sD);
        for (int w = threadIdx.x; w < nwords; w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();
    const DomainDev& D = sD;
    const int x = tl.y + (int)threadIdx.x % D.tile_x;
    const int y = tl.z + (int)threadIdx.x / D.tile_x;
    const int z = tl.w;
    if (x >= D.nx || y >= D.ny) return;
    const int c = D.cur ^ parity;
    const T* __restrict__ fin = static_cast<const T*>(D.buf[c]);
    T* __restrict__ fout = static_cast<T*>(D.buf[c ^ 1]);
    const PullIdx P = pull_index(D, x, y, z);
    float d[NF][NQ], o[NF][NQ];
    load_cell<S>(D, fin, P, d);
    collide<COLL, false>(D, d, o, nullptr);
    store_cell<S>(D, fout, P.c, o);
}

// ---- diagnostics: fixed-order sum of the block partials ----------------------------------
// One CTA of 256 threads: thread t sums partials t, t+256, ... in order (FP64), then a fixed
// shared-memory tree.  Writes the NDIAG record to out.
__global__ void __launch_bounds__(256) diag_finalize_kernel(const double* __restrict__ partials,
                                                            int64_t nblocks, double* __restrict__ out) {
    __shared__ double sh[256];
    for (int f = 0; f < NDIAG; ++f) {
        const bool isMin = (f == 8 || f == 9);
        double acc = isMin ? 3.0e38 : 0.0;
        for (int64_t b = threadIdx.x; b < nblocks; b += 256) {
            const double x = partials[b * NDIAG + f];
            acc = isMin ? fmin(acc, x) : acc + x;
        }
        sh[threadIdx.x] = acc;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                const double a = sh[threadIdx.x], b2 = sh[threadIdx.x + s];
                sh[threadIdx.x] = isMin ? fmin(a, b2) : a + b2;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) out[f] = sh[0];
        __syncthreads();
    }
}

// ---- initialisation: primitive (physical, FP64) -> equilibrium deviations ----------------
// Populations f = w_i (Q + c_i . Phi^adv / cs^2) (zero non-equilibrium), stored as
// deviations from the reference equilibrium.  Lattice conversion with s = dt/dx.
template <int S>
__global__ void init_kernel(const DomainDev D, void* __restrict__ fout_v, const double* __restrict__ rho,
                            const double* __restrict__ u, const double* __restrict__ p, double s,
                            double gm1, double rho_ref, double p_ref) {
    using T = typename Store<S>::T;
    T* fout = static_cast<T*>(fout_v);
    const int64_t N = D.plane;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * blockDim.x) {
        const double r = rho[c];
        const double ux = u[c] * s, uy = u[N + c] * s, uz = u[2 * N + c] * s;
        const double pp = p[c] * s * s;
        const double uv[3] = {ux, uy, uz};
        const double m[3] = {r * ux, r * uy, r * uz};
        const double ke = 0.5 * (m[0] * ux + m[1] * uy + m[2] * uz);
        const double dE = (pp - p_ref) / gm1 + ke;
        const double dQ[5] = {r - rho_ref, m[0], m[1], m[2], dE};
        const double E = p_ref / gm1 + dE;
        double Pd[5][3];
        for (int a = 0; a < 3; ++a) {
            Pd[0][a] = m[a];
            for (int j = 0; j < 3; ++j) Pd[1 + j][a] = m[j] * uv[a] + (j == a ? pp - p_ref : 0.0);
            Pd[4][a] = (E + pp) * uv[a];
        }
        for (int k = 0; k < NF; ++k) {
            const double sc = (double)D.enc[k];
            const double q1 = 0.125 * dQ[k];
            const double v[NQ] = {0.25 * dQ[k], q1 + 0.5 * Pd[k][0], q1 - 0.5 * Pd[k][0],
                                  q1 + 0.5 * Pd[k][1], q1 - 0.5 * Pd[k][1],
                                  q1 + 0.5 * Pd[k][2], q1 - 0.5 * Pd[k][2]};
            for (int i = 0; i < NQ; ++i)
                Store<S>::st(fout + (int64_t)(7 * k + i) * N + c, (float)(v[i] * sc));
        }
    }
}

// ---- readback: conserved fields in physical units (FP64) ---------------------------------
template <int S>
__global__ void conserved_kernel(const DomainDev D, const void* __restrict__ fin_v,
                                 double* __restrict__ out, double s, double rho_ref, double E_ref) {
    using T = typename Store<S>::T;
    const T* fin = static_cast<const T*>(fin_v);
    const int64_t N = D.plane;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < NF; ++k) {
            double acc = 0.0;
            const double sc = (double)D.dec[k];
            for (int i = 0; i < NQ; ++i) acc += (double)Store<S>::ld(fin + (int64_t)(7 * k + i) * N + c) * sc;
            double q = acc;
            if (k == 0) q += rho_ref;
            if (k == 4) q += E_ref;
            if (k >= 1 && k <= 3) q /= s;
            if (k == 4) q /= s * s;
            out[(int64_t)k * N + c] = q;
        }
    }
}

// ---- host-side launchers ------------------------------------------------------------------
template <int S, int COLL>
static cudaError_t launch_sweep_t(const DomainDev& D, const void* fin, void* fout, bool diag,
                                  double* partials, dim3 grid, dim3 block, cudaStream_t st) {
    if (diag)
        sweep_kernel<S, COLL, true><<<grid, block, 0, st>>>(D, fin, fout, partials);
    else
        sweep_kernel<S, COLL, false><<<grid, block, 0, st>>>(D, fin, fout, partials);
    return cudaGetLastError();
}

cudaError_t launch_sweep(const DomainDev& D, int storage, int coll, const void* fin, void* fout,
                         bool diag, double* partials, dim3 grid, dim3 block, cudaStream_t st) {
#define GRLB_CASE(SS, CC) \
    if (storage == SS && coll == CC) return launch_sweep_t<SS, CC>(D, fin, fout, diag, partials, grid, block, st);
    GRLB_CASE(S_F32, C_RLB) GRLB_CASE(S_F32, C_BGK) GRLB_CASE(S_F16, C_RLB)
    GRLB_CASE(S_F16, C_BGK) GRLB_CASE(S_BF16, C_RLB) GRLB_CASE(S_BF16, C_BGK)
#undef GRLB_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_sweep(int storage, int coll, const DomainDev* doms, const int4* tiles,
                               int ntiles, int threads, int parity, cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
#define GRLB_CASE(SS, CC)                                                                  \
    if (storage == SS && coll == CC) {                                                     \
        batch_sweep_kernel<SS, CC><<<ntiles, threads, 0, st>>>(doms, tiles, parity);         \
        return cudaGetLastError();                                                         \
    }
    GRLB_CASE(S_F32, C_RLB) GRLB_CASE(S_F32, C_BGK) GRLB_CASE(S_F16, C_RLB)
    GRLB_CASE(S_F16, C_BGK) GRLB_CASE(S_BF16, C_RLB) GRLB_CASE(S_BF16, C_BGK)
#undef GRLB_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_diag_finalize(const double* partials, int64_t nblocks, double* out, cudaStream_t st) {
    diag_finalize_kernel<<<1, 256, 0, st>>>(partials, nblocks, out);
    return cudaGetLastError();
}

cudaError_t launch_init(const DomainDev& D, int storage, void* fout, const double* rho, const double* u,
                        const double* p, double s, double gm1, double rho_ref, double p_ref,
                        cudaStream_t st) {
    const int threads = 256;
    int64_t blocks = (D.plane + threads - 1) / threads;
    if (blocks > 148 * 32) blocks = 148 * 32;
    if (storage == S_F32) init_kernel<S_F32><<<(int)blocks, threads, 0, st>>>(D, fout, rho, u, p, s, gm1, rho_ref, p_ref);
    else if (storage == S_F16) init_kernel<S_F16><<<(int)blocks, threads, 0, st>>>(D, fout, rho, u, p, s, gm1, rho_ref, p_ref);
    else init_kernel<S_BF16><<<(int)blocks, threads, 0, st>>>(D, fout, rho, u, p, s, gm1, rho_ref, p_ref);
    return cudaGetLastError();
}

cudaError_t launch_conserved(const DomainDev& D, int storage, const void* fin, double* out, double s,
                             double rho_ref, double E_ref, cudaStream_t st) {
    const int threads = 256;
    int64_t blocks = (D.plane + threads - 1) / threads;
    if (blocks > 148 * 32) blocks = 148 * 32;
    if (storage == S_F32) conserved_kernel<S_F32><<<(int)blocks, threads, 0, st>>>(D, fin, out, s, rho_ref, E_ref);
    else if (storage == S_F16) conserved_kernel<S_F16><<<(int)blocks, threads, 0, st>>>(D, fin, out, s, rho_ref, E_ref);
    else conserved_kernel<S_BF16><<<(int)blocks, threads, 0, st>>>(D, fin, out, s, rho_ref, E_ref);
    return cudaGetLastError();
}

}  // namespace grlb
