// grlb_kernels.h -- host-side launchers of the sweep kernels (internal to libgrlb).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "grlb_device.cuh"

namespace grlb {
// One sweep of one domain (record by value).  pattern: 0 two-buffer pull (fin -> fout),
// 1 / 2 odd / even step of the one-buffer AA pattern (fin == fout).  diag: one partial record
// per CTA in partials.
cudaError_t launch_sweep(const DomainDev& D, int storage, int coll, int pattern, const void* fin, void* fout,
                         bool diag, double* partials, dim3 grid, dim3 block, cudaStream_t st);
// One sweep of every tile in tiles[0, ntiles) (domain records in device memory): one launch
// of the persistent batched kernel.
cudaError_t launch_batch_sweep(int storage, int coll, const DomainDev* doms, const int4* tiles, int ntiles,
                               int parity, cudaStream_t st);
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
// gather = 1 for a one-buffer (AA) state after an odd number of steps.
cudaError_t launch_conserved(const DomainDev& D, int storage, const void* fin, double* out,
                             double s, double rho_ref, double E_ref, int gather, cudaStream_t st);

// ---- spectral post-processing (grlb_spectral.cu) ------------------------------------------
// One batched FFT pass: lines of 2^log2n complex values `stride` apart; line l starts at
// (l & inner_mask) * inner_stride + (l >> lg_inner) * outer_stride (inner_mask = 2^lg_inner - 1);
// L = 2^lgL lines per CTA, L divides nlines.
struct FftAxis {
    int log2n, L, lgL, lg_inner;
    int64_t stride, inner_mask, inner_stride, outer_stride, nlines;
};
constexpr int kFftSmemBytes = 32768;
int fft_lines_per_cta(int log2n, int64_t nlines);
cudaError_t launch_fft_axis(float2* data, const float2* tw, const FftAxis& A, bool inverse, cudaStream_t st);
// Populations -> u (3 complex planes) and mu(T) (float plane), per-CTA sums of 1/2 |u|^2
// (lattice units).  gather as for launch_conserved.
cudaError_t launch_spectral_prep(const DomainDev& D, int storage, const void* fin, int gather, float2* U, float* mu,
                                 double* partials, int grid, cudaStream_t st);
// scale = 2^fx / N^2 (a power of two): shell sums in fixed point with 2^-fx resolution
cudaError_t launch_spectral_modes(float2* U, float2* TH, int lgx, int lgy, int lgz, int nbins, float scale,
                                  unsigned long long* bins, int grid, cudaStream_t st);
cudaError_t launch_spectral_eps(const float2* W, const float* mu, int64_t N, double* partials, int grid,
                                cudaStream_t st);
// FP32 FFMA issue-rate probe: ctas x 256 threads x iters x 128 FFMAs.
cudaError_t launch_ffma_probe(float* sink, int ctas, int iters, cudaStream_t st);
}  // namespace grlb
