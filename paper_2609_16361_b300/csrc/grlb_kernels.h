// grlb_kernels.h -- host-side launchers of the sweep kernels (internal to libgrlb).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "grlb_device.cuh"

namespace grlb {
// One sweep of one domain (record by value).  pattern: 0 two-buffer pull (fin -> fout),
// 1 / 2 odd / even step of the one-buffer AA pattern (fin == fout), 3 two-buffer pull of
// moments (FP32, regularized collision).  diag: one partial record
// per CTA in partials.
cudaError_t launch_sweep(const DomainDev& D, int storage, int coll, int pattern, const void* fin, void* fout,
                         bool diag, double* partials, dim3 grid, dim3 block, cudaStream_t st);
// One sweep of every tile in tiles[0, ntiles) (domain records in device memory): one launch
// of the persistent batched kernel.
cudaError_t launch_batch_sweep(int storage, int coll, const DomainDev* doms, const int4* tiles, int ntiles,
                               int parity, cudaStream_t st);
// Constant-table batched sweep: the records of up to kBatchSlots small domains live in a
// __constant__ table (slots written by upload_batch_records, stream-ordered); one launch covers
// the tiles of nd domains, domain i owning CTAs [tile0[i], tile0[i+1]) and its record in slot
// slot[i].  Tiles as in the tile-table sweep (tile_x cells x 128 / tile_x rows, or 128
// consecutive cells when tile_x == 1).
constexpr int kBatchSlots = 160;  // 160 x 336-byte records: 53.8 KB of the 64 KB constant bank
constexpr int kTableLanes = 8;    // at most this many streams for the one-launch-per-step schedule
struct BatchLaunch {
    int32_t nd;
    int32_t parity;
    int32_t slot[kBatchSlots];
    int32_t tile0[kBatchSlots + 1];
};
cudaError_t launch_batch_sweep_const(int storage, int coll, const BatchLaunch& L, cudaStream_t st);
cudaError_t upload_batch_records(const DomainDev* recs, int first_slot, int n, cudaStream_t st);
cudaError_t launch_diag_finalize(const double* partials, int64_t nblocks, double* out,
                                 cudaStream_t st);
// swap = 1 writes the one-buffer layout (population i in slot opp(i)).
cudaError_t launch_init(const DomainDev& D, int storage, void* fout, const double* rho,
                        const double* u, const double* p, double s, double gm1, double rho_ref,
                        double p_ref, int swap, cudaStream_t st);
// Chapman-Enskog initialisation (grlb_init_ce.cu): FP64 parameters in lattice units, ghost
// primitives (rho, ux, uy, uz, p) in physical units, nominal tau_k = 1 / omega_k.
struct CeInit {
    double s, gm1, mu, kap, inv_T_ref, T_S;
    double tau[5];
    double ghostL[5], ghostR[5];
    int sutherland, bc;
};
cudaError_t launch_init_ce(const DomainDev& D, int storage, void* fout, const double* rho, const double* u,
                           const double* p, double rho_ref, double p_ref, int swap, const CeInit& C,
                           cudaStream_t st);
// gather = 1 for a one-buffer (AA) state after an odd number of steps, 2 for moment storage.
cudaError_t launch_conserved(const DomainDev& D, int storage, const void* fin, double* out,
                             double s, double rho_ref, double E_ref, int gather, cudaStream_t st);

// ---- spectral post-processing (grlb_spectral.cu) ------------------------------------------
// Cubes (lgz > 0, n >= 16) or squares (lgz = 0, n >= 32) of extent n = 2^lg <= 1024.  grid1,
// grid3, grid5: the persistent grids of K1, K3, K5 (set by the launchers to the resident CTA
// count; the plan's values are upper bounds for sizing the partial-sum buffers); scale =
// 2^fx / N^2 for the fixed-point shell sums (set after K1).
struct SpectralPlan {
    int lg, lgx, lgy, lgz;
    int64_t N;
    int nbins;
    float scale;
    int grid1, grid3, grid5;
};
SpectralPlan spectral_plan(int lgx, int lgy, int lgz, int nbins, int sms);
// K1: populations -> x-transformed velocity planes U (3 N complex), mu (N), per-CTA sums of
// 1/2 |u|^2 (grid1 doubles).  gather as for launch_conserved.
cudaError_t launch_spectral_k1(const DomainDev& D, int storage, const void* fin, int gather, SpectralPlan& P,
                               const float2* tw, float2* U, float* mu, double* partials, cudaStream_t st);
// K2..K5: shell sums into bins (nbins, zeroed by the caller), per-CTA dissipation sums
// (2 grid5 doubles); U needs 4 N complex.
cudaError_t launch_spectral_k2_to_k5(SpectralPlan& P, const float2* tw, float2* U, const float* mu,
                                     unsigned long long* bins, double* partials, cudaStream_t st);
// z-slab ghost exchange (grlb_halo.cu): lower's top interior +z slices -> upper's ghost plane
// 0; upper's bottom interior -z slices -> lower's top ghost plane (nzl = lower's planes).
cudaError_t launch_halo_z(void* lower, void* upper, int nzl, int64_t nxy, size_t elem, cudaStream_t st);
// Cross-device form of the same exchange: pack the two outgoing slices of a slab (nz planes
// including its ghosts) into contiguous buffers of 5 nxy elements, unpack received ones into its
// ghost planes.
cudaError_t launch_halo_pack_z(const void* f, void* to_upper, void* to_lower, int nz, int64_t nxy, size_t elem,
                               cudaStream_t st);
cudaError_t launch_halo_unpack_z(void* f, const void* from_lower, const void* from_upper, int nz, int64_t nxy,
                                 size_t elem, cudaStream_t st);
// The same for moment storage: per direction 10 slices of nx ny FP32 values, slice 2 k + h = row
// 4 k (h = 0: Q_k / 8) or 4 k + 3 (h = 1: J*_k,z) of the moment bricks.
cudaError_t launch_halo_z_mom(void* lower, void* upper, int nzl, int64_t nxy, cudaStream_t st);
cudaError_t launch_halo_pack_z_mom(const void* f, void* to_upper, void* to_lower, int nz, int64_t nxy,
                                   cudaStream_t st);
cudaError_t launch_halo_unpack_z_mom(void* f, const void* from_lower, const void* from_upper, int nz, int64_t nxy,
                                     cudaStream_t st);
// Populations of listed cells (grlb_cells.cu): out[q n + j] = f_q(cells[j]) in FP64 lattice
// units, f = stored x dec[k] + shift[q].  layout 0: slot q of the cell (two buffers); 1: slot
// opp(i) of the cell (one buffer, even steps done); 2: slot q of the neighbour x + c_i or the
// outflow record (one buffer, odd steps done); 3: rebuilt from the cell's moments (moment
// storage).  cells[j] must lie in [0, N).
struct CellDecode {
    double dec[5];
    double shift[35];
};
cudaError_t launch_read_cells(const DomainDev& D, int storage, const void* buf, const int64_t* cells, int64_t n,
                              int layout, const CellDecode& dec, double* out, cudaStream_t st);
// Writes *flag = 1 (device-accessible) if any stored value of the buffer (bytes, a multiple of
// 16) is non-finite; never writes 0.
cudaError_t launch_check_finite(const void* buf, int64_t bytes, int storage, int32_t* flag, cudaStream_t st);
// FP32 FFMA issue-rate probe: ctas x 256 threads x iters x 128 FFMAs.
cudaError_t launch_ffma_probe(float* sink, int ctas, int iters, cudaStream_t st);
}  // namespace grlb
