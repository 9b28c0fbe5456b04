// grlb_kernels.cu -- sweep, initialisation, readback and diagnostic-reduction kernels.
//
// Compiled without multiply-add contraction (-fmad=false): each fused multiply-add is an
// explicit fmaf, so every kernel the collide is instantiated in rounds each operation the same
// way, whatever its launch bounds or register budget.
//
// Layout in HBM (per domain, per buffer): cell bricks (grlb_device.cuh) -- 128 consecutive
// cells in storage order (x fastest) keep their 35 population rows q = 7k + i (field k, link i)
// together, 128 elements each.  One CTA covers a tile of blockDim.x consecutive cells of
// blockDim.y rows at one z (or 128 consecutive cells); consecutive lanes touch consecutive
// elements of every population row, so each of the 35 loads and 35 stores of a warp is a fully
// used 128-byte line (FP32).  The +-y / +-z pulls read whole neighbouring rows; the +-x pulls
// are the same row shifted by one element, served from L1/L2 lines already fetched for the row
// (no extra DRAM traffic).  A thread forms one 64-bit address per pull source and reaches the
// five fields' populations of that source by constant offsets q * 128.
#include <cuda_runtime.h>

#include "grlb_device.cuh"
#include "grlb_kernels.h"

namespace grlb {

struct PullIdx {
    int32_t c, xm, xp, ym, yp, zm, zp;  // cell offsets of the 7 pull sources
    int32_t yz;                         // y + ny z (row index)
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
    P.yz = y + ny * z;
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

// ---- population access patterns ----------------------------------------------------------
// PULL: two buffers; read f_i(x - c_i) from the input, write f*_i(x) to the output (row i).
// AA (one buffer, in place, alternating):
//   AA_ODD : read f*_i(x - c_i) from slot opp(i) of the neighbour x - c_i, collide, write
//            f*_i(x) to slot i of the neighbour x + c_i (the streamed population arrives there);
//   AA_EVEN: read slot i of x itself, collide, write f*_i(x) to slot opp(i) of x.
// In an AA_ODD step the location a thread writes is one it read itself and no other thread
// touches it, so the in-place update has no races.  Ghost cells (X_DIRICHLET_EQ): an AA_ODD
// step reads the ghost value instead of the missing neighbour, drops the population that
// leaves the domain, and writes the ghost's incoming population into the boundary cell's own
// slot (nobody else reads it in that step) for the AA_EVEN step to find.
// MOM: two buffers of moments (mom_at layout, regularized collision): the pull rebuilds
// f*_i(x - c_i) from the source cell's w_1 Q_k and J*_k with the collide's own operations, so the
// sweep computes bit for bit what PULL computes on the populations those moments stand for,
// reading 20 values per cell (each used by up to 7 cells, the reuse caught by L1 / L2) and
// writing 20 instead of 35.
enum Pattern { PULL = 0, AA_ODD = 1, AA_EVEN = 2, MOM = 3 };

template <int S, int PAT>
__device__ __forceinline__ float ld_pop(const typename Store<S>::T* p) {
    if (PAT == PULL) return Store<S>::ld(p);  // read-only path: the input is not written
    return Store<S>::ld_plain(p);             // in place: plain (coherent) load
}

// Element offsets (cell bricks) of population row 0 of the cell and of its 6 pull sources.
struct PullAt {
    int64_t c, xm, xp, ym, yp, zm, zp;
};

__device__ __forceinline__ PullAt pull_at(const PullIdx& P) {
    PullAt A;
    A.c = brick_at_u32((uint32_t)P.c);
    A.xm = brick_at_u32((uint32_t)P.xm);
    A.xp = brick_at_u32((uint32_t)P.xp);
    A.ym = brick_at_u32((uint32_t)P.ym);
    A.yp = brick_at_u32((uint32_t)P.yp);
    A.zm = brick_at_u32((uint32_t)P.zm);
    A.zp = brick_at_u32((uint32_t)P.zp);
    return A;
}

// element offsets (moment storage) of the cell and its 6 pull sources
__device__ __forceinline__ PullAt pull_at_m(const PullIdx& P) {
    PullAt A;
    A.c = mom_at_u32((uint32_t)P.c);
    A.xm = mom_at_u32((uint32_t)P.xm);
    A.xp = mom_at_u32((uint32_t)P.xp);
    A.ym = mom_at_u32((uint32_t)P.ym);
    A.yp = mom_at_u32((uint32_t)P.yp);
    A.zm = mom_at_u32((uint32_t)P.zm);
    A.zp = mom_at_u32((uint32_t)P.zp);
    return A;
}

// Population i of the outgoing set of a field from its stored moments (w_1 Q, J): 2 w_1 Q = Q / 4
// at rest, fmaf(+-1/2, J_a, w_1 Q) along axis a -- the regularized collide's own operations
// (w_1 Q = Q / 8 is its q1, an exact scaling).
__device__ __forceinline__ float mom_pop(float s1, float j, float sign) { return fmaf(sign * 0.5f, j, s1); }

template <int S, int PAT>
__device__ __forceinline__ void load_cell(const DomainDev& D, const typename Store<S>::T* fin,
                                          const PullIdx& P, const PullAt& A, float (&d)[NF][NQ]) {
    using St = Store<S>;
    using T = typename St::T;
    if constexpr (PAT == MOM) {
        static_assert(S == S_F32, "moment storage is FP32");
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            const int q = 4 * k * kBrick;
            d[k][0] = 2.0f * St::ld(fin + A.c + q);
            d[k][1] = P.gl ? D.ghostL_st[k] : mom_pop(St::ld(fin + A.xm + q), St::ld(fin + A.xm + q + kBrick), 1.0f);
            d[k][2] = P.gr ? D.ghostR_st[k] : mom_pop(St::ld(fin + A.xp + q), St::ld(fin + A.xp + q + kBrick), -1.0f);
            d[k][3] = mom_pop(St::ld(fin + A.ym + q), St::ld(fin + A.ym + q + 2 * kBrick), 1.0f);
            d[k][4] = mom_pop(St::ld(fin + A.yp + q), St::ld(fin + A.yp + q + 2 * kBrick), -1.0f);
            d[k][5] = mom_pop(St::ld(fin + A.zm + q), St::ld(fin + A.zm + q + 3 * kBrick), 1.0f);
            d[k][6] = mom_pop(St::ld(fin + A.zp + q), St::ld(fin + A.zp + q + 3 * kBrick), -1.0f);
        }
    } else {
        const T* bc = fin + A.c;
        const T* bxm = fin + A.xm;
        const T* bxp = fin + A.xp;
        const T* bym = fin + A.ym;
        const T* byp = fin + A.yp;
        const T* bzm = fin + A.zm;
        const T* bzp = fin + A.zp;
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            const int q = 7 * k * kBrick;
            const float gl = D.ghostL_st[k], gr = D.ghostR_st[k];  // stored units
            if (PAT == AA_EVEN) {
#pragma unroll
                for (int i = 0; i < NQ; ++i) d[k][i] = ld_pop<S, PAT>(bc + q + i * kBrick);
            } else {
                // PULL reads row i of the neighbour; AA_ODD reads row opp(i) of it
                const int o1 = PAT == PULL ? 1 : 2, o2 = PAT == PULL ? 2 : 1;
                const int o3 = PAT == PULL ? 3 : 4, o4 = PAT == PULL ? 4 : 3;
                const int o5 = PAT == PULL ? 5 : 6, o6 = PAT == PULL ? 6 : 5;
                d[k][0] = ld_pop<S, PAT>(bc + q);
                d[k][1] = P.gl ? gl : ld_pop<S, PAT>(bxm + q + o1 * kBrick);
                d[k][2] = P.gr ? gr : ld_pop<S, PAT>(bxp + q + o2 * kBrick);
                d[k][3] = ld_pop<S, PAT>(bym + q + o3 * kBrick);
                d[k][4] = ld_pop<S, PAT>(byp + q + o4 * kBrick);
                d[k][5] = ld_pop<S, PAT>(bzm + q + o5 * kBrick);
                d[k][6] = ld_pop<S, PAT>(bzp + q + o6 * kBrick);
            }
        }
    }
}

template <int S, int PAT>
__device__ __forceinline__ void store_cell(const DomainDev& D, typename Store<S>::T* fout,
                                           const PullIdx& P, const PullAt& A, const float (&o)[NF][NQ]) {
    using St = Store<S>;
    using T = typename St::T;
    T* bc = fout + A.c;
    if constexpr (PAT == MOM) {  // o[k][0..3] = Q_k, J*_k
#pragma unroll
        for (int k = 0; k < NF; ++k)
#pragma unroll
            for (int m = 0; m < 4; ++m) St::st(bc + (4 * k + m) * kBrick, o[k][m]);
    } else {
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            const int q = 7 * k * kBrick;
            if (PAT == PULL) {
#pragma unroll
                for (int i = 0; i < NQ; ++i) St::st(bc + q + i * kBrick, o[k][i]);
            } else if (PAT == AA_EVEN) {
                St::st(bc + q, o[k][0]);
                St::st(bc + q + 2 * kBrick, o[k][1]);
                St::st(bc + q + 1 * kBrick, o[k][2]);
                St::st(bc + q + 4 * kBrick, o[k][3]);
                St::st(bc + q + 3 * kBrick, o[k][4]);
                St::st(bc + q + 6 * kBrick, o[k][5]);
                St::st(bc + q + 5 * kBrick, o[k][6]);
            } else {  // AA_ODD: push to the neighbour the population streams to
                St::st(bc + q, o[k][0]);
                const int64_t nyz = (int64_t)D.ny * D.nz;
                T* out = static_cast<T*>(D.outflow);
                if (P.gr) {
                    St::st(bc + q + 2 * kBrick, D.ghostR_st[k]);
                    St::st(out + (5 + k) * nyz + P.yz, o[k][1]);
                } else {
                    St::st(fout + A.xp + q + 1 * kBrick, o[k][1]);
                }
                if (P.gl) {
                    St::st(bc + q + 1 * kBrick, D.ghostL_st[k]);
                    St::st(out + k * nyz + P.yz, o[k][2]);
                } else {
                    St::st(fout + A.xm + q + 2 * kBrick, o[k][2]);
                }
                St::st(fout + A.yp + q + 3 * kBrick, o[k][3]);
                St::st(fout + A.ym + q + 4 * kBrick, o[k][4]);
                St::st(fout + A.zp + q + 5 * kBrick, o[k][5]);
                St::st(fout + A.zm + q + 6 * kBrick, o[k][6]);
            }
        }
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
        GRLB_ST(out + tid, acc);
    }
}

// (unused in the checked build, which issues no prefetch)
[[maybe_unused]] constexpr int kPrefetchPlanes = 2;           // L2 prefetch distance (planes)
[[maybe_unused]] constexpr int kPrefetchMaxPlane = 256 * 256;  // largest plane (cells) prefetched for

// ---- single-domain sweep -----------------------------------------------------------------
// One CTA per tile of blockDim.x x blockDim.y cells at one z.  The domain record is a kernel
// parameter, so its constants are read as constant-bank operands of the arithmetic (a record
// held in shared memory costs a load per use and ~15% of the sweep's time).
// LIN: cells are taken in storage order, thread t of CTA b updating cell 128 b + t, so no lane
// idles whatever nx is (x, y, z from one division each); otherwise a CTA is a tile of
// blockDim.x x blockDim.y cells of one z plane.
template <int S, int COLL, bool DIAG, bool SRC, int PAT, bool LIN>
__device__ __forceinline__ void sweep_body(const DomainDev& D, const void* fin_v, void* fout_v,
                                           double* __restrict__ partials) {
    using T = typename Store<S>::T;
    const T* fin = static_cast<const T*>(fin_v);
    T* fout = static_cast<T*>(fout_v);
    int x, y, z;
    bool active;
    if (LIN) {
        const int64_t t = (int64_t)blockIdx.x * 128 + threadIdx.x;
        active = t < D.plane;
        const uint32_t c = active ? (uint32_t)t : 0u;
        const uint32_t r = c / (uint32_t)D.nx;
        x = (int)(c - r * (uint32_t)D.nx);
        z = (int)(r / (uint32_t)D.ny);
        y = (int)(r - (uint32_t)z * (uint32_t)D.ny);
    } else {
        x = blockIdx.x * blockDim.x + threadIdx.x;
        y = blockIdx.y * blockDim.y + threadIdx.y;
        z = blockIdx.z;
        active = (x < D.nx) && (y < D.ny);
    }
    CellDiag cd;
#ifndef GRLB_CHECKED
    // 16-bit plain two-buffer sweeps of tiled domains whose rows are whole bricks: lane 0 of each
    // row of a tile that starts a brick prefetches that brick (35 rows, 8.75 KB) two planes
    // ahead into L2 with one bulk prefetch (the plane's CTAs run about a plane later).  256^3:
    // FP16 0.426 -> 0.417 ms, BF16 0.422 -> 0.406 ms.  Not for FP32, HBM-bound at the copy
    // bandwidth: 0.678 -> 0.803 ms with it; nor for the one-buffer patterns (1024^3 FP16: 29.0 ->
    // 33.3 ms); planes of up to 256^2 cells only, as for the moment sweep.
    if constexpr (S != S_F32 && !LIN && PAT == PULL && !DIAG) {
        if (threadIdx.x == 0 && (D.nx & (kBrick - 1)) == 0 && (x & (kBrick - 1)) == 0 && y < D.ny &&
            z + kPrefetchPlanes < D.nz && D.nx * D.ny <= kPrefetchMaxPlane) {
            const T* brick = fin + brick_at_u32((uint32_t)((y + D.ny * (z + kPrefetchPlanes)) * D.nx + x));
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(brick), "r"((int)(NP * kBrick * sizeof(T)))
                         : "memory");
        }
    }
#endif
    if (active) {
        const PullIdx P = pull_index(D, x, y, z);
        const PullAt A = PAT == MOM ? pull_at_m(P) : pull_at(P);
        float d[NF][NQ], o[NF][NQ];
        load_cell<S, PAT>(D, fin, P, A, d);
        collide<S, COLL, DIAG, PAT == MOM>(D, d, o, &cd);
        if (SRC) add_source<S>(D, P.c, o);
        store_cell<S, PAT>(D, fout, P, A, o);
    }
    if (DIAG) {
        const int64_t blk = blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
        block_reduce_diag(cd, active, partials + blk * NDIAG);
    }
}

template <int S, int COLL, bool DIAG, bool SRC, int PAT, bool LIN>
__global__ void __launch_bounds__(128) sweep_kernel(const __grid_constant__ DomainDev D,
                                                    const void* fin_v, void* fout_v,
                                                    double* __restrict__ partials) {
    sweep_body<S, COLL, DIAG, SRC, PAT, LIN>(D, fin_v, fout_v, partials);
}

// The gated FP32 collision keeps both updates live in a warp that straddles the gate (114
// registers, 4 CTAs per SM, with IEEE divisions in the collide); capped at 5 CTAs per SM it
// needs 96 registers, without spills since the collide divides approximately, and takes 0.670
// ms at 256^3 (0.701 with the IEEE divisions' 52 bytes of spills, 0.719 uncapped).  A separate
// kernel carries the cap, so the other instantiations keep their own register allocation.
template <bool DIAG, bool SRC, int PAT, bool LIN>
__global__ void __launch_bounds__(128, 5) sweep_kernel_gated_f32(const __grid_constant__ DomainDev D,
                                                                 const void* fin_v, void* fout_v,
                                                                 double* __restrict__ partials) {
    sweep_body<S_F32, C_GATED, DIAG, SRC, PAT, LIN>(D, fin_v, fout_v, partials);
}

// The plain moment-storage sweep waits mostly on its 65 loads per cell (L1 / L2 hits of the
// sources' moments).  With IEEE divisions in the collide it held 92 registers (5 CTAs per SM)
// and ran 1.7 % faster capped at 6 CTAs; with the approximate divisions it fits the 6-CTA cap
// (80 registers) without spills; 6 or 8 CTAs per SM ran alike (33.2 GLUP/s) before the column
// kernel's L2 prefetch, with it 6 CTAs 35.0 against 34.4 GLUP/s at 8 (64 registers).  The
// diagnostic variant (72 registers) keeps the plain bound.  The rounding of every operation
// is fixed by the source (no compiler contraction in this file), so the cap does not change
// results.
template <bool LIN>
__global__ void __launch_bounds__(128, 6) sweep_kernel_mom(const __grid_constant__ DomainDev D, const void* fin_v,
                                                           void* fout_v, double* __restrict__ partials) {
    sweep_body<S_F32, C_RLB, false, false, MOM, LIN>(D, fin_v, fout_v, partials);
}

// ---- moment sweep marching along z ---------------------------------------------------------
// As sweep_kernel_mom, but a thread updates the cells (x, y, z) of lz consecutive planes in
// turn: the -z / +z sources of plane z are the thread's own column, whose moments it touched in
// the two previous steps (L1 hits), and the tile's rows march through the planes together.
// 256^3: 0.501 ms with 4 planes per thread, 0.513 / 0.532 / 0.544 with 8 / 16 / 32, 0.519 with
// 1 (the loop costs 40 bytes of spills at the 6-CTA register cap); the one-cell kernel 0.511.
// L2 prefetch two planes ahead: when the domain's rows are whole bricks (nx a multiple of 128),
// lane 0 of each row of the CTAs whose tile starts a brick issues one bulk prefetch of that
// brick at plane z + 2 (its 20 moment rows, 10 KB; at the first plane also z + 1), so the
// rows a tile reaches next are on their way from DRAM while it collides.  256^3: 35.2 against
// 33.1 GLUP/s in the benchmark (0.461 against 0.493 ms per sweep, at a lower clock under the
// power cap); three planes ahead the same.  One instruction per row and plane: an earlier
// prefetch of one 128-byte line per lane cost 5 % more instructions and lost under the power cap,
// and one thread per band of rows prefetching the band's bricks (fewer warps take the branch)
// ran 34.8 against 35.8 GLUP/s.
// Only for planes of up to 256^2 cells: at 512^3 and 1024^3 the cap held a lower clock with it
// (1680 against 1845 MHz) and the sweep lost 3 % / 2.4 % (4.42 against 4.28 ms, 34.7 against
// 33.9 ms); at 128^3 it changes nothing.  Not in the checked build (a prefetch reads nothing the
// kernel uses).
// Staging the tile's planes in shared memory (cp.async, a ring of three planes, 96 KB per
// 256-thread CTA) ran 0.821 ms: two CTAs per SM leave too few warps for the collide.
// Carrying the column's z-window in registers (per field the arriving +z population and the
// cell's own w_1 Q, J*_z, so a plane reads 2 values per field along z instead of 5: 55 loads
// per cell instead of 65) spills 120 bytes at 6 CTAs per SM and ran 28.2 against 32.0 GLUP/s;
// at 5 CTAs (96 registers) 32.1, within run-to-run spread (both with IEEE divisions in the
// collide).  The loads are not the limit.
constexpr int kZChunk = 4;  // planes per thread

__global__ void __launch_bounds__(128, 6) sweep_kernel_mom_col(const __grid_constant__ DomainDev D, const void* fin_v,
                                                               void* fout_v, int lz) {
    const float* fin = static_cast<const float*>(fin_v);
    float* fout = static_cast<float*>(fout_v);
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= D.nx || y >= D.ny) return;
    const int zb = blockIdx.z * lz, ze = min(zb + lz, D.nz);
#ifndef GRLB_CHECKED
    // x is a multiple of kBrick and so is every row start: cell (x, y, zz) begins a brick, which
    // lies whole inside the buffer for zz < nz
    const bool pf = threadIdx.x == 0 && (D.nx & (kBrick - 1)) == 0 && (x & (kBrick - 1)) == 0 &&
                    D.nx * D.ny <= kPrefetchMaxPlane;
#endif
    for (int z = zb; z < ze; ++z) {
#ifndef GRLB_CHECKED
        if (pf) {
            for (int zz = z == zb ? z + 1 : z + kPrefetchPlanes; zz <= z + kPrefetchPlanes && zz < D.nz; ++zz) {
                const float* brick = fin + mom_at_u32((uint32_t)((y + D.ny * zz) * D.nx + x));
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(brick), "r"(NM * kBrick * 4) : "memory");
            }
        }
#endif
        const PullIdx P = pull_index(D, x, y, z);
        const PullAt A = pull_at_m(P);
        float d[NF][NQ], o[NF][NQ];
        load_cell<S_F32, MOM>(D, fin, P, A, d);
        collide<S_F32, C_RLB, false, true>(D, d, o, nullptr);
        store_cell<S_F32, MOM>(D, fout, P, A, o);
    }
}

// ---- batched sweep: persistent CTAs over a tile table ------------------------------------
// tiles[t] = (domain, x0, y0, z), or (domain, first cell, 0, 0) for a domain whose tile_x is 1
// (linear tiles: 128 consecutive cells in storage order, no idle lanes for any nx).
// A CTA of 128 threads takes tiles blockIdx.x, + gridDim.x,
// ... (grid-stride, so consecutive CTAs stream consecutive rows); the domain record (buffers,
// constants, tile width tile_x) is copied to shared memory whenever the domain changes;
// thread t handles cell (x0 + t % tile_x, y0 + t / tile_x, z).  Each domain reads
// buf[cur ^ parity] and writes the other buffer, so `parity` flips every step.  A domain's
// result does not depend on which other domains share the launch.
template <int S, int COLL>
__global__ void __launch_bounds__(128) batch_sweep_kernel(const DomainDev* __restrict__ doms,
                                                          const int4* __restrict__ tiles, int ntiles,
                                                          int parity) {
    using T = typename Store<S>::T;
    __shared__ DomainDev sD;
    int loaded = -1;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = GRLB_LD(tiles + t);
        if (tl.x != loaded) {  // uniform across the CTA
            __syncthreads();
            const int nwords = sizeof(DomainDev) / 4;
            const uint32_t* src = reinterpret_cast<const uint32_t*>(doms + tl.x);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&sD);
            for (int w = threadIdx.x; w < nwords; w += blockDim.x) dst[w] = GRLB_LD(src + w);
            __syncthreads();
            loaded = tl.x;
        }
        const DomainDev& D = sD;
        int x, y, z;
        bool active;
        if (D.tile_x == 1) {  // linear tile: 128 consecutive cells from cell tl.y
            const int64_t cidx = (int64_t)tl.y + threadIdx.x;
            active = cidx < D.plane;
            const uint32_t c = active ? (uint32_t)cidx : 0u;
            const uint32_t r = c / (uint32_t)D.nx;
            x = (int)(c - r * (uint32_t)D.nx);
            z = (int)(r / (uint32_t)D.ny);
            y = (int)(r - (uint32_t)z * (uint32_t)D.ny);
        } else {
            x = tl.y + (int)threadIdx.x % D.tile_x;
            y = tl.z + (int)threadIdx.x / D.tile_x;
            z = tl.w;
            active = x < D.nx && y < D.ny;
        }
        if (active) {
            const int c = D.cur ^ parity;
            const T* __restrict__ fin = static_cast<const T*>(D.buf[c]);
            T* __restrict__ fout = static_cast<T*>(D.buf[c ^ 1]);
            const PullIdx P = pull_index(D, x, y, z);
            const PullAt A = pull_at(P);
            float d[NF][NQ], o[NF][NQ];
            load_cell<S, PULL>(D, fin, P, A, d);
            collide<S, COLL, false>(D, d, o, nullptr);
            store_cell<S, PULL>(D, fout, P, A, o);
        }
    }
}

// ---- batched sweep with the domain records in constant memory -----------------------------
// The records of a batch's small domains sit in slots of a constant table, written before each
// batched step.  One CTA per tile, no tile table: CTA t of a launch finds its domain by a
// search over the launch's tile prefix sums (kernel parameters), so the domain index, the
// record's address and every constant read from it are the same for all threads of the CTA,
// and the constants are read through the constant cache as in the single-domain sweep instead
// of with a shared-memory load per use.
static_assert(kBatchSlots * sizeof(DomainDev) <= 60 * 1024, "constant record table exceeds its budget");
__constant__ DomainDev c_batch_doms[kBatchSlots];

template <int S, int COLL>
__global__ void __launch_bounds__(128) batch_sweep_const_kernel(const __grid_constant__ BatchLaunch L) {
    using T = typename Store<S>::T;
    const int t = blockIdx.x;
    int lo = 0, hi = L.nd - 1;  // domain of tile t: the last i with tile0[i] <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (L.tile0[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    const DomainDev& D = c_batch_doms[L.slot[lo]];
    const int lt = t - L.tile0[lo];
    int x, y, z;
    bool active;
    if (D.tile_x == 1) {  // linear tile: 128 consecutive cells in storage order
        const int64_t cidx = (int64_t)lt * 128 + threadIdx.x;
        active = cidx < D.plane;
        const uint32_t c = active ? (uint32_t)cidx : 0u;
        const uint32_t r = c / (uint32_t)D.nx;
        x = (int)(c - r * (uint32_t)D.nx);
        z = (int)(r / (uint32_t)D.ny);
        y = (int)(r - (uint32_t)z * (uint32_t)D.ny);
    } else {  // tile of tile_x cells x 128 / tile_x rows of one z plane, x fastest
        const int tx = D.tile_x, ty = 128 / tx;
        const int ntx = (D.nx + tx - 1) / tx, nty = (D.ny + ty - 1) / ty;
        const int r = lt / ntx;
        x = (lt - r * ntx) * tx + (int)threadIdx.x % tx;
        y = (r % nty) * ty + (int)threadIdx.x / tx;
        z = r / nty;
        active = x < D.nx && y < D.ny;
    }
    if (active) {
        const int c = D.cur ^ L.parity;
        const T* __restrict__ fin = static_cast<const T*>(D.buf[c]);
        T* __restrict__ fout = static_cast<T*>(D.buf[c ^ 1]);
        const PullIdx P = pull_index(D, x, y, z);
        const PullAt A = pull_at(P);
        float d[NF][NQ], o[NF][NQ];
        load_cell<S, PULL>(D, fin, P, A, d);
        collide<S, COLL, false>(D, d, o, nullptr);
        store_cell<S, PULL>(D, fout, P, A, o);
    }
}

template <int S, int COLL>
static cudaError_t launch_batch_const_t(const BatchLaunch& L, int ntiles, cudaStream_t st) {
    batch_sweep_const_kernel<S, COLL><<<ntiles, 128, 0, st>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_batch_sweep_const(int storage, int coll, const BatchLaunch& L, cudaStream_t st) {
    if (L.nd <= 0) return cudaSuccess;
    const int ntiles = L.tile0[L.nd];
#define GRLB_CASE(SS, CC) \
    if (storage == SS && coll == CC) return launch_batch_const_t<SS, CC>(L, ntiles, st);
    GRLB_CASE(S_F32, C_RLB) GRLB_CASE(S_F32, C_BGK) GRLB_CASE(S_F32, C_GATED)
    GRLB_CASE(S_F16, C_RLB) GRLB_CASE(S_F16, C_BGK) GRLB_CASE(S_F16, C_GATED)
    GRLB_CASE(S_BF16, C_RLB) GRLB_CASE(S_BF16, C_BGK) GRLB_CASE(S_BF16, C_GATED)
#undef GRLB_CASE
    return cudaErrorInvalidValue;
}

cudaError_t upload_batch_records(const DomainDev* recs, int first_slot, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (first_slot < 0 || first_slot + n > kBatchSlots) return cudaErrorInvalidValue;
    return cudaMemcpyToSymbolAsync(c_batch_doms, recs, (size_t)n * sizeof(DomainDev),
                                   (size_t)first_slot * sizeof(DomainDev), cudaMemcpyHostToDevice, st);
}

// ---- diagnostics: fixed-order sum of the block partials ----------------------------------
// Two deterministic stages.  Stage 1: CTA g sums the partial records [g*per, (g+1)*per) --
// thread t takes records g*per + t, + 256, ... in order (FP64), then a fixed shared-memory
// tree -- and writes one record.  Stage 2: one CTA sums the G stage-1 records the same way.
__device__ __forceinline__ void reduce_records(const double* __restrict__ rec, int64_t begin, int64_t end,
                                               double* __restrict__ out) {
    __shared__ double sh[NDIAG][256];
    double acc[NDIAG];
#pragma unroll
    for (int f = 0; f < NDIAG; ++f) acc[f] = (f == 8 || f == 9) ? 3.0e38 : 0.0;
    for (int64_t b = begin + threadIdx.x; b < end; b += 256) {
#pragma unroll
        for (int f = 0; f < NDIAG; ++f) {
            const double x = GRLB_LD(rec + (b * NDIAG + f));
            acc[f] = (f == 8 || f == 9) ? fmin(acc[f], x) : acc[f] + x;
        }
    }
#pragma unroll
    for (int f = 0; f < NDIAG; ++f) sh[f][threadIdx.x] = acc[f];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
#pragma unroll
            for (int f = 0; f < NDIAG; ++f) {
                const double a = sh[f][threadIdx.x], c = sh[f][threadIdx.x + s];
                sh[f][threadIdx.x] = (f == 8 || f == 9) ? fmin(a, c) : a + c;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < NDIAG) GRLB_ST(out + threadIdx.x, sh[threadIdx.x][0]);
}

__global__ void __launch_bounds__(256) diag_stage1_kernel(const double* __restrict__ partials, int64_t nblocks,
                                                          int64_t per, double* __restrict__ stage) {
    const int64_t begin = (int64_t)blockIdx.x * per;
    const int64_t end = begin + per < nblocks ? begin + per : nblocks;
    reduce_records(partials, begin, end, stage + (int64_t)blockIdx.x * NDIAG);
}

__global__ void __launch_bounds__(256) diag_stage2_kernel(const double* __restrict__ stage, int64_t g,
                                                          double* __restrict__ out) {
    reduce_records(stage, 0, g, out);
}

// ---- initialisation: primitive (physical, FP64) -> equilibrium deviations ----------------
// Populations f = w_i (Q + c_i . Phi^adv / cs^2) (zero non-equilibrium), stored as
// deviations from the reference equilibrium.  Lattice conversion with s = dt/dx.
template <int S>
__global__ void __launch_bounds__(256) init_kernel(const DomainDev D, void* __restrict__ fout_v,
                                                   const double* __restrict__ rho, const double* __restrict__ u,
                                                   const double* __restrict__ p, double s, double gm1,
                                                   double rho_ref, double p_ref, int swap) {
    using T = typename Store<S>::T;
    T* fout = static_cast<T*>(fout_v);
    const int64_t N = D.plane;
    const float g1 = (float)gm1;
    const float Hp_ref = (float)(p_ref / gm1 + p_ref);  // E_ref + p_ref
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * blockDim.x) {
        // the two differences against the reference state are taken in FP64, the rest in FP32
        const double r = GRLB_LD(rho + c);
        const float drho = (float)(r - rho_ref);
        const float dp = (float)(GRLB_LD(p + c) * s * s - p_ref);
        const float rf = (float)r;
        const float uv[3] = {(float)(GRLB_LD(u + c) * s), (float)(GRLB_LD(u + N + c) * s),
                             (float)(GRLB_LD(u + 2 * N + c) * s)};
        const float m[3] = {rf * uv[0], rf * uv[1], rf * uv[2]};
        const float ke = 0.5f * fmaf(m[0], uv[0], fmaf(m[1], uv[1], m[2] * uv[2]));
        const float dE = dp / g1 + ke;
        const float Hp = Hp_ref + dE + dp;  // E + p
        const float dQ[5] = {drho, m[0], m[1], m[2], dE};
        float Pd[5][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Pd[0][a] = m[a];
#pragma unroll
            for (int j = 0; j < 3; ++j) Pd[1 + j][a] = j == a ? fmaf(m[j], uv[a], dp) : m[j] * uv[a];
            Pd[4][a] = Hp * uv[a];
        }
        if (swap == 2) {  // moment storage (FP32): w_1 Q_k and the first moment Phi^adv_k
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                T* m = fout + mom_at(c) + 4 * k * kBrick;
                Store<S>::st(m, 0.125f * dQ[k]);
#pragma unroll
                for (int a = 0; a < 3; ++a) Store<S>::st(m + (1 + a) * kBrick, Pd[k][a]);
            }
            continue;
        }
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            const float sc = D.enc[k];
            const float q1 = 0.125f * dQ[k];
            const float v[NQ] = {0.25f * dQ[k], q1 + 0.5f * Pd[k][0], q1 - 0.5f * Pd[k][0],
                                 q1 + 0.5f * Pd[k][1], q1 - 0.5f * Pd[k][1],
                                 q1 + 0.5f * Pd[k][2], q1 - 0.5f * Pd[k][2]};
            // swap: the one-buffer (AA) layout keeps population i in slot opp(i) before an
            // odd step
#pragma unroll
            for (int i = 0; i < NQ; ++i) {
                const int slot = swap ? (i == 0 ? 0 : (i & 1 ? i + 1 : i - 1)) : i;
                Store<S>::st(fout + brick_at(c) + (7 * k + slot) * kBrick, v[i] * sc);
            }
        }
    }
}

// ---- readback: conserved fields in physical units (FP64) ---------------------------------
template <int S>
// gather = 1: one-buffer state after an odd step, where f*_i(x) sits in slot i of x + c_i
// (or in the outflow record when x + c_i is outside an X_DIRICHLET_EQ domain); gather = 2:
// moment storage, f*_i(x) rebuilt from the cell's own Q_k, J*_k.
__global__ void conserved_kernel(const DomainDev D, const void* __restrict__ fin_v,
                                 double* __restrict__ out, double s, double rho_ref, double E_ref, int gather) {
    using T = typename Store<S>::T;
    const T* fin = static_cast<const T*>(fin_v);
    const T* outflow = static_cast<const T*>(D.outflow);
    const int64_t N = D.plane;
    const int64_t nyz = (int64_t)D.ny * D.nz;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(c % D.nx), r = (int)(c / D.nx);
        const int y = r % D.ny, z = r / D.ny;
        const PullIdx P = pull_index(D, x, y, z);
        // where population i of this cell lives
        int32_t at[NQ] = {P.c, P.c, P.c, P.c, P.c, P.c, P.c};
        if (gather == 1) {
            at[1] = P.xp; at[2] = P.xm; at[3] = P.yp; at[4] = P.ym; at[5] = P.zp; at[6] = P.zm;
        }
        for (int k = 0; k < NF; ++k) {
            double acc = 0.0;
            const double sc = (double)D.dec[k];
            float mq = 0.0f, mj[3] = {0.0f, 0.0f, 0.0f};
            if (gather == 2) {  // moment storage: the cell's own outgoing set (mq = w_1 Q)
                const T* m = fin + mom_at(c) + 4 * k * kBrick;
                mq = Store<S>::ld(m);
#pragma unroll
                for (int a = 0; a < 3; ++a) mj[a] = Store<S>::ld(m + (1 + a) * kBrick);
            }
            for (int i = 0; i < NQ; ++i) {
                double v;
                if (gather == 2) v = (double)(i == 0 ? 2.0f * mq : mom_pop(mq, mj[(i - 1) >> 1], (i & 1) ? 1.0f : -1.0f));
                else if (gather && i == 1 && P.gr) v = (double)Store<S>::ld(outflow + (5 + k) * nyz + P.yz);
                else if (gather && i == 2 && P.gl) v = (double)Store<S>::ld(outflow + k * nyz + P.yz);
                else v = (double)Store<S>::ld(fin + brick_at(at[i]) + (7 * k + i) * kBrick);
                acc = fma(v, sc, acc);
            }
            double q = acc;
            if (k == 0) q += rho_ref;
            if (k == 4) q += E_ref;
            if (k >= 1 && k <= 3) q /= s;
            if (k == 4) q /= s * s;
            GRLB_ST(out + (int64_t)k * N + c, q);
        }
    }
}

// ---- host-side launchers ------------------------------------------------------------------
// grid.y == 0 is not a valid launch, so the linear mapping is signalled by block.y == 0
template <int S, int COLL, bool DIAG, bool SRC, int PAT, bool LIN>
static void launch_one(const DomainDev& D, const void* fin, void* fout, double* partials, dim3 grid,
                       dim3 block, cudaStream_t st) {
    if constexpr (PAT == MOM && !DIAG)
        sweep_kernel_mom<LIN><<<grid, block, 0, st>>>(D, fin, fout, partials);
    else if constexpr (S == S_F32 && COLL == C_GATED)
        sweep_kernel_gated_f32<DIAG, SRC, PAT, LIN><<<grid, block, 0, st>>>(D, fin, fout, partials);
    else
        sweep_kernel<S, COLL, DIAG, SRC, PAT, LIN><<<grid, block, 0, st>>>(D, fin, fout, partials);
}

template <int S, int COLL, int PAT, bool SRC>
static cudaError_t launch_sweep_p(const DomainDev& D, const void* fin, void* fout, bool diag,
                                  double* partials, dim3 grid, dim3 block, cudaStream_t st) {
    const bool lin = block.y == 0;
    if (lin) block = dim3(128, 1, 1);
    if (diag && lin) launch_one<S, COLL, true, SRC, PAT, true>(D, fin, fout, partials, grid, block, st);
    else if (diag) launch_one<S, COLL, true, SRC, PAT, false>(D, fin, fout, partials, grid, block, st);
    else if (lin) launch_one<S, COLL, false, SRC, PAT, true>(D, fin, fout, partials, grid, block, st);
    else launch_one<S, COLL, false, SRC, PAT, false>(D, fin, fout, partials, grid, block, st);
    return cudaGetLastError();
}

// column-marching moment sweep (plain sweeps of tiled domains): the grid's z extent split into
// chunks of kZChunk planes
// (The diagnostic sweep stays one cell per thread: 0.689 ms per 256^3 sweep, 1 in 50.)
static cudaError_t launch_sweep_mom_col(const DomainDev& D, const void* fin, void* fout, dim3 grid, dim3 block,
                                        cudaStream_t st) {
    const int lz = D.nz < kZChunk ? D.nz : kZChunk;
    grid.z = (unsigned)((D.nz + lz - 1) / lz);
    sweep_kernel_mom_col<<<grid, block, 0, st>>>(D, fin, fout, lz);
    return cudaGetLastError();
}

template <int S, int COLL>
static cudaError_t launch_sweep_t(const DomainDev& D, int pattern, const void* fin, void* fout, bool diag,
                                  double* partials, dim3 grid, dim3 block, cudaStream_t st) {
    if (pattern == MOM) {
        if constexpr (S == S_F32 && COLL == C_RLB) {
            if (!diag && block.y != 0) return launch_sweep_mom_col(D, fin, fout, grid, block, st);
            return launch_sweep_p<S, COLL, MOM, false>(D, fin, fout, diag, partials, grid, block, st);
        }
        return cudaErrorInvalidValue;
    }
    if (pattern == AA_ODD) return launch_sweep_p<S, COLL, AA_ODD, false>(D, fin, fout, diag, partials, grid, block, st);
    if (pattern == AA_EVEN) return launch_sweep_p<S, COLL, AA_EVEN, false>(D, fin, fout, diag, partials, grid, block, st);
    if (D.src != nullptr)  // sources: two-buffer sweeps only
        return launch_sweep_p<S, COLL, PULL, true>(D, fin, fout, diag, partials, grid, block, st);
    return launch_sweep_p<S, COLL, PULL, false>(D, fin, fout, diag, partials, grid, block, st);
}

cudaError_t launch_sweep(const DomainDev& D, int storage, int coll, int pattern, const void* fin, void* fout,
                         bool diag, double* partials, dim3 grid, dim3 block, cudaStream_t st) {
#define GRLB_CASE(SS, CC) \
    if (storage == SS && coll == CC)                                                               \
        return launch_sweep_t<SS, CC>(D, pattern, fin, fout, diag, partials, grid, block, st);
    GRLB_CASE(S_F32, C_RLB) GRLB_CASE(S_F32, C_BGK) GRLB_CASE(S_F32, C_GATED)
    GRLB_CASE(S_F16, C_RLB) GRLB_CASE(S_F16, C_BGK) GRLB_CASE(S_F16, C_GATED)
    GRLB_CASE(S_BF16, C_RLB) GRLB_CASE(S_BF16, C_BGK) GRLB_CASE(S_BF16, C_GATED)
#undef GRLB_CASE
    return cudaErrorInvalidValue;
}

// Persistent grid of the batched sweep: as many CTAs as can be resident at once on the current
// device (queried once per kernel instantiation and device ordinal), capped by the number of
// tiles.
template <typename K>
static int resident_ctas(K kernel) {
    constexpr int kMaxDev = 64;
    static int cached[kMaxDev] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    const bool slot = dev >= 0 && dev < kMaxDev;
    if (slot && cached[dev] > 0) return cached[dev];
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 128, 0);
    const int n = (sms > 0 ? sms : 148) * (per > 0 ? per : 4);
    if (slot) cached[dev] = n;
    return n;
}

template <int S, int COLL>
static cudaError_t launch_batch_t(const DomainDev* doms, const int4* tiles, int ntiles, int parity,
                                  cudaStream_t st) {
    auto k = batch_sweep_kernel<S, COLL>;
    int grid = resident_ctas(k);
    if (grid > ntiles) grid = ntiles;
    k<<<grid, 128, 0, st>>>(doms, tiles, ntiles, parity);
    return cudaGetLastError();
}

cudaError_t launch_batch_sweep(int storage, int coll, const DomainDev* doms, const int4* tiles, int ntiles,
                               int parity, cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
#define GRLB_CASE(SS, CC) \
    if (storage == SS && coll == CC) return launch_batch_t<SS, CC>(doms, tiles, ntiles, parity, st);
    GRLB_CASE(S_F32, C_RLB) GRLB_CASE(S_F32, C_BGK) GRLB_CASE(S_F32, C_GATED)
    GRLB_CASE(S_F16, C_RLB) GRLB_CASE(S_F16, C_BGK) GRLB_CASE(S_F16, C_GATED)
    GRLB_CASE(S_BF16, C_RLB) GRLB_CASE(S_BF16, C_BGK) GRLB_CASE(S_BF16, C_GATED)
#undef GRLB_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_diag_finalize(const double* partials, int64_t nblocks, double* out, cudaStream_t st) {
    // stage-1 records are written right after the nblocks partial records
    const int64_t g = nblocks < kDiagStageRecords ? nblocks : kDiagStageRecords;
    const int64_t per = (nblocks + g - 1) / g;
    double* stage = const_cast<double*>(partials) + nblocks * NDIAG;
    diag_stage1_kernel<<<(int)g, 256, 0, st>>>(partials, nblocks, per, stage);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_stage2_kernel<<<1, 256, 0, st>>>(stage, g, out);
    return cudaGetLastError();
}

cudaError_t launch_init(const DomainDev& D, int storage, void* fout, const double* rho, const double* u,
                        const double* p, double s, double gm1, double rho_ref, double p_ref, int swap,
                        cudaStream_t st) {
    const int threads = 256;
    int64_t blocks = (D.plane + threads - 1) / threads;
    if (blocks > 148 * 32) blocks = 148 * 32;
    if (storage == S_F32) init_kernel<S_F32><<<(int)blocks, threads, 0, st>>>(D, fout, rho, u, p, s, gm1, rho_ref, p_ref, swap);
    else if (storage == S_F16) init_kernel<S_F16><<<(int)blocks, threads, 0, st>>>(D, fout, rho, u, p, s, gm1, rho_ref, p_ref, swap);
    else init_kernel<S_BF16><<<(int)blocks, threads, 0, st>>>(D, fout, rho, u, p, s, gm1, rho_ref, p_ref, swap);
    return cudaGetLastError();
}

cudaError_t launch_conserved(const DomainDev& D, int storage, const void* fin, double* out, double s,
                             double rho_ref, double E_ref, int gather, cudaStream_t st) {
    const int threads = 256;
    int64_t blocks = (D.plane + threads - 1) / threads;
    if (blocks > 148 * 32) blocks = 148 * 32;
    if (storage == S_F32) conserved_kernel<S_F32><<<(int)blocks, threads, 0, st>>>(D, fin, out, s, rho_ref, E_ref, gather);
    else if (storage == S_F16) conserved_kernel<S_F16><<<(int)blocks, threads, 0, st>>>(D, fin, out, s, rho_ref, E_ref, gather);
    else conserved_kernel<S_BF16><<<(int)blocks, threads, 0, st>>>(D, fin, out, s, rho_ref, E_ref, gather);
    return cudaGetLastError();
}

// ---- finiteness scan: one read-only pass over a population buffer ------------------------
// Stored values are non-finite exactly when their exponent field is all ones (FP32 8 bits,
// FP16 5 bits, BF16 8 bits); a thread tests 16 bytes per load (4 FP32 or 8 16-bit values), a
// warp writes *flag = 1 once if any lane saw one.  The buffer holds whole cell bricks (35 x 128
// elements each), so its size is a multiple of 16 bytes.
__global__ void __launch_bounds__(256) check_finite_kernel(const uint4* __restrict__ buf, int64_t n16,
                                                           uint32_t mask_lo, uint32_t mask_hi,
                                                           int32_t* __restrict__ flag) {
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 v = GRLB_LDG(buf + i);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 4; ++j)
            bad = bad || ((w[j] & mask_lo) == mask_lo) || ((w[j] & mask_hi) == mask_hi);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) GRLB_ST(flag, 1);
}

cudaError_t launch_check_finite(const void* buf, int64_t bytes, int storage, int32_t* flag, cudaStream_t st) {
    // exponent masks of the value(s) in one 32-bit word: FP32 one value; 16-bit types two
    uint32_t lo = 0x7f800000u, hi = 0x7f800000u;
    if (storage == S_F16) { lo = 0x00007c00u; hi = 0x7c000000u; }
    if (storage == S_BF16) { lo = 0x00007f80u; hi = 0x7f800000u; }
    const int64_t n16 = bytes / 16;
    int64_t blocks = (n16 + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    if (blocks < 1) blocks = 1;
    check_finite_kernel<<<(int)blocks, 256, 0, st>>>(static_cast<const uint4*>(buf), n16, lo, hi, flag);
    return cudaGetLastError();
}

}  // namespace grlb
