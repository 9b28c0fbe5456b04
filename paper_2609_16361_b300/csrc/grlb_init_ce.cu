// grlb_init_ce.cu -- initialisation with the Chapman-Enskog non-equilibrium part.
//
// The equilibrium start f = f^eq(Q, Phi^adv) has no non-equilibrium first moment, so the first
// sweep reconstructs its gradients from the streaming shift alone; with omega near 2 the
// non-equilibrium part then relaxes by the factor (1 - omega) ~ -1 per step and alternates for
// thousands of steps between about zero and twice its value.  This kernel writes instead the
// state a Chapman-Enskog flow has after a collision (Sec. 2.3: the non-equilibrium first moment
// of field k carries its gradient).  Before a collision the streamed first moment is
// J_k = Phi^adv_k + Phi^diff_k - tau_k cs^2 grad Q_k; a regularized or BGK collision with the
// nominal tau_k = 1 / omega_k leaves Phi^adv_k + A_k with
//     A_k = Phi^diff_k - (tau_k - 1) cs^2 grad Q_k,
// so the stored populations are w_i (Q_k + c_i . (Phi^adv_k + A_k) / cs^2).  Gradients are
// central differences (phi(x + e_a) - phi(x - e_a)) / 2 in lattice units of Q_k, u and T, with
// periodic wrap or the Dirichlet ghost state beyond a tube's ends; Phi^diff is 0 (rho),
// -tau_visc (momentum) and -tau_visc u + q (energy) with tau_visc = mu (grad u + grad u^T -
// 2/3 div u I), q = -kappa grad T at the local temperature.  A_k is formed in FP32 from
// differences of the FP64 inputs (B300's FP64 units are a small fraction of its FP32 ones: the
// same arithmetic in FP64 took 11.2 ms at 256^3); the equilibrium part repeats the FP32
// deviation arithmetic of the plain initialisation, so a uniform field gives bitwise the plain
// initial state.
#include <cuda_runtime.h>

#include "grlb_device.cuh"
#include "grlb_kernels.h"

namespace grlb {

namespace {

struct Prim {  // physical units, as in the input fields
    double r, u[3], p;
};

__device__ __forceinline__ Prim prim(double r, double ux, double uy, double uz, double p) {
    Prim q;
    q.r = r;
    q.u[0] = ux;
    q.u[1] = uy;
    q.u[2] = uz;
    q.p = p;
    return q;
}

}  // namespace

template <int S>
__global__ void __launch_bounds__(256) init_ce_kernel(const DomainDev D, void* __restrict__ fout_v,
                                                      const double* __restrict__ rho, const double* __restrict__ u,
                                                      const double* __restrict__ p, double rho_ref, double p_ref,
                                                      int swap, const CeInit C) {
    using T = typename Store<S>::T;
    T* fout = static_cast<T*>(fout_v);
    const int64_t N = D.plane;
    const int nx = D.nx, ny = D.ny, nz = D.nz;
    const float g1 = (float)C.gm1;
    const float Hp_ref = (float)(p_ref / C.gm1 + p_ref);
    auto load = [&](int64_t i) {
        return prim(GRLB_LD(rho + i), GRLB_LD(u + i), GRLB_LD(u + N + i), GRLB_LD(u + 2 * N + i), GRLB_LD(p + i));
    };
    const float sl = (float)C.s, sl2 = (float)(C.s * C.s);  // lattice scaling of u and p
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx);
        const int64_t r = c / nx;
        const int y = (int)(r % ny), z = (int)(r / ny);
        // neighbours along +-x, +-y, +-z: [2a] = +e_a, [2a + 1] = -e_a
        Prim nb[6];
        if (C.bc == 1 && x == nx - 1)
            nb[0] = prim(C.ghostR[0], C.ghostR[1], C.ghostR[2], C.ghostR[3], C.ghostR[4]);
        else
            nb[0] = load(c - x + (x == nx - 1 ? 0 : x + 1));
        if (C.bc == 1 && x == 0)
            nb[1] = prim(C.ghostL[0], C.ghostL[1], C.ghostL[2], C.ghostL[3], C.ghostL[4]);
        else
            nb[1] = load(c - x + (x == 0 ? nx - 1 : x - 1));
        nb[2] = load(c + (int64_t)((y == ny - 1) ? -(ny - 1) : 1) * nx);
        nb[3] = load(c + (int64_t)((y == 0) ? (ny - 1) : -1) * nx);
        const int64_t pl = (int64_t)nx * ny;
        nb[4] = load(c + ((z == nz - 1) ? -(int64_t)(nz - 1) : 1) * pl);
        nb[5] = load(c + ((z == 0) ? (int64_t)(nz - 1) : -1) * pl);
        const int ext[3] = {nx, ny, nz};

        const Prim q0 = load(c);
        // Differences of neighbouring states without cancellation: the primitive differences
        // are taken in FP64 (the inputs' precision), everything else in FP32 through the
        // product rule on pairs, e.g. r+ u+ - r- u- = rb du + ub dr with the pair means rb, ub
        // (exact identities), so each gradient carries FP32 rounding of itself, not of the
        // states it is the difference of.  Lattice units: u s, p s^2.
        float gQ[5][3], gu[3][3], gT[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const Prim& P = nb[2 * a];
            const Prim& M = nb[2 * a + 1];
            const float h = ext[a] > 1 ? 0.5f : 0.0f;
            const float rP = (float)P.r, rM = (float)M.r;
            const float dr = (float)(P.r - M.r), dp = (float)(P.p - M.p) * sl2;
            const float rb = 0.5f * (rP + rM), pb = 0.5f * ((float)P.p + (float)M.p) * sl2;
            float du[3], ub[3], du2 = 0.0f, u2b = 0.0f;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float uP = (float)P.u[j] * sl, uM = (float)M.u[j] * sl;
                du[j] = (float)(P.u[j] - M.u[j]) * sl;
                ub[j] = 0.5f * (uP + uM);
                du2 = fmaf(2.0f * ub[j], du[j], du2);                         // d |u|^2
                u2b = fmaf(0.5f, fmaf(uP, uP, uM * uM), u2b);
            }
            gQ[0][a] = h * dr;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                gQ[1 + j][a] = h * fmaf(rb, du[j], ub[j] * dr);                // d (r u_j)
                gu[j][a] = h * du[j];
            }
            gQ[4][a] = h * fmaf(0.5f, fmaf(rb, du2, u2b * dr), dp / g1);      // d (p/(g-1) + r|u|^2/2)
            gT[a] = h * fmaf(rb, dp, -(pb * dr)) / (rP * rM);                 // d (p / r)
        }
        const float T0 = (float)q0.p * sl2 / (float)q0.r;
        float fac = 1.0f;
        if (C.sutherland) {
            const float t = T0 * (float)C.inv_T_ref, ts = (float)C.T_S;
            fac = (1.0f + ts) * t * sqrtf(t) / (t + ts);
        }
        const float mu = (float)C.mu * fac, kap = (float)C.kap * fac;
        const float th = gu[0][0] + gu[1][1] + gu[2][2];
        float tv[3][3];
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int a = 0; a < 3; ++a)
                tv[j][a] = mu * (gu[j][a] + gu[a][j] - (j == a ? (2.0f / 3.0f) * th : 0.0f));
        const float u0[3] = {(float)q0.u[0] * sl, (float)q0.u[1] * sl, (float)q0.u[2] * sl};
        float A[5][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float qa = -kap * gT[a];
            const float dE = qa - fmaf(tv[a][0], u0[0], fmaf(tv[a][1], u0[1], tv[a][2] * u0[2]));
            A[0][a] = -((float)C.tau[0] - 1.0f) * 0.25f * gQ[0][a];
#pragma unroll
            for (int j = 0; j < 3; ++j) A[1 + j][a] = fmaf(-((float)C.tau[1 + j] - 1.0f) * 0.25f, gQ[1 + j][a], -tv[j][a]);
            A[4][a] = fmaf(-((float)C.tau[4] - 1.0f) * 0.25f, gQ[4][a], dE);
        }

        // equilibrium part: the plain initialisation's deviation arithmetic
        const double rr = GRLB_LD(rho + c);
        const float drho = (float)(rr - rho_ref);
        const float dp = (float)(GRLB_LD(p + c) * C.s * C.s - p_ref);
        const float rf = (float)rr;
        const float uv[3] = {(float)(GRLB_LD(u + c) * C.s), (float)(GRLB_LD(u + N + c) * C.s),
                             (float)(GRLB_LD(u + 2 * N + c) * C.s)};
        const float m[3] = {rf * uv[0], rf * uv[1], rf * uv[2]};
        const float ke = 0.5f * fmaf(m[0], uv[0], fmaf(m[1], uv[1], m[2] * uv[2]));
        const float dEd = dp / g1 + ke;
        const float Hp = Hp_ref + dEd + dp;
        const float dQ[5] = {drho, m[0], m[1], m[2], dEd};
        float Pd[5][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Pd[0][a] = m[a];
#pragma unroll
            for (int j = 0; j < 3; ++j) Pd[1 + j][a] = j == a ? fmaf(m[j], uv[a], dp) : m[j] * uv[a];
            Pd[4][a] = Hp * uv[a];
        }
        if (swap == 2) {  // moment storage (FP32): w_1 Q_k and the first moment Phi^adv_k + A_k
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                T* m = fout + mom_at(c) + 4 * k * kBrick;
                Store<S>::st(m, 0.125f * dQ[k]);
#pragma unroll
                for (int a = 0; a < 3; ++a) Store<S>::st(m + (1 + a) * kBrick, Pd[k][a] + A[k][a]);
            }
            continue;
        }
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            const float sc = D.enc[k];
            const float q1 = 0.125f * dQ[k];
            const float P0 = Pd[k][0] + A[k][0], P1 = Pd[k][1] + A[k][1], P2 = Pd[k][2] + A[k][2];
            const float v[NQ] = {0.25f * dQ[k], q1 + 0.5f * P0, q1 - 0.5f * P0, q1 + 0.5f * P1,
                                 q1 - 0.5f * P1, q1 + 0.5f * P2, q1 - 0.5f * P2};
#pragma unroll
            for (int i = 0; i < NQ; ++i) {
                const int slot = swap ? (i == 0 ? 0 : (i & 1 ? i + 1 : i - 1)) : i;
                Store<S>::st(fout + brick_at(c) + (7 * k + slot) * kBrick, v[i] * sc);
            }
        }
    }
}

cudaError_t launch_init_ce(const DomainDev& D, int storage, void* fout, const double* rho, const double* u,
                           const double* p, double rho_ref, double p_ref, int swap, const CeInit& C,
                           cudaStream_t st) {
    const int threads = 256;
    int64_t blocks = (D.plane + threads - 1) / threads;
    if (blocks > 148 * 32) blocks = 148 * 32;
    if (storage == S_F32)
        init_ce_kernel<S_F32><<<(int)blocks, threads, 0, st>>>(D, fout, rho, u, p, rho_ref, p_ref, swap, C);
    else if (storage == S_F16)
        init_ce_kernel<S_F16><<<(int)blocks, threads, 0, st>>>(D, fout, rho, u, p, rho_ref, p_ref, swap, C);
    else
        init_ce_kernel<S_BF16><<<(int)blocks, threads, 0, st>>>(D, fout, rho, u, p, rho_ref, p_ref, swap, C);
    return cudaGetLastError();
}

}  // namespace grlb
