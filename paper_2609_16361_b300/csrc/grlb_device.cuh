// grlb_device.cuh -- device side of the fused stream-and-collide sweep (sm_103a).
//
// One thread updates one cell: pull the 35 populations f_{k,i}(x - c_i) (exact streaming,
// Sec. 2.2), run the in-collide update of Algorithm 1 in FP32 registers, write the 35
// post-collision populations at x into the other buffer.  Nothing but populations touches
// HBM: the reconstructed gradients, stress, heat flux and the sensor chi stay in registers
// (Sec. 2.5 "cell-local").
//
// Storage is the equilibrium shift of Sec. 2.2: the buffers hold d_{k,i} = f_{k,i} -
// w_i (Q_ref,k + c_i . J_ref,k / cs^2), the deviation from the equilibrium of a reference
// state at rest (Q_ref = (rho_ref, 0, 0, 0, p_ref/(gamma-1)), J_ref,m_j = p_ref e_j).  All
// moment arithmetic is done on deviations (dQ, dJ, dp) so the FP32 significand is spent on
// the fluctuation, not the mean.  FP16/BF16 storage multiplies the deviation by a per-field
// power of two before rounding (RN-even) and divides after loading.
//
// D3Q7 links i = 0, +x, -x, +y, -y, +z, -z; w0 = 1/4, w1..6 = 1/8; cs^2 = 1/4.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "grlb_check.cuh"

namespace grlb {

constexpr int NF = 5;
constexpr int NQ = 7;
constexpr int NP = NF * NQ;
constexpr int NDIAG = 13;  // per-block partial record of the diagnostic sweep
// Diagnostic scratch = nblocks partial records followed by up to kDiagStageRecords records of
// the first finalize stage.
constexpr int kDiagStageRecords = 256;

// Population layout in HBM: cell bricks.  Cells are grouped in storage order (x fastest) into
// bricks of kBrick consecutive cells; a brick holds its 35 population rows q = 7k + i one after
// the other, kBrick elements each, so population q of cell c is element
//     brick_at(c) + q * kBrick,   brick_at(c) = (c / kBrick) * 35 kBrick + c % kBrick.
// A warp of consecutive cells reads and writes whole contiguous row segments (as in 35 separate
// planes), while the 35 populations of one cell lie within 35 kBrick elements of one base
// address: a sweep forms 7 addresses per cell (its own and the 6 pull sources) and reaches
// the 35 populations by constant offsets, instead of forming 35 + 35 64-bit addresses.  A
// buffer holds ceil(N / kBrick) bricks; the cells past N in the last brick are never updated.
constexpr int kBrick = 128;
__host__ __device__ __forceinline__ int64_t brick_at(int64_t c) {  // c >= 0
    const uint64_t u = (uint64_t)c;
    return (int64_t)((u / kBrick) * (uint64_t)(NP * kBrick) + (u % kBrick));
}
__device__ __forceinline__ int64_t brick_at_u32(uint32_t c) {
    return (int64_t)(c >> 7) * (NP * kBrick) + (c & (kBrick - 1));
}
// elements of one population buffer for N cells
__host__ __device__ __forceinline__ int64_t brick_elems(int64_t N) {
    return (N + kBrick - 1) / kBrick * (int64_t)(NP * kBrick);
}
static_assert(kBrick == 128, "brick_at_u32 shifts by log2(kBrick)");
// Moment storage (regularized collision): the outgoing set of field k is w_i (Q_k + c_i . J*_k /
// cs^2), so a cell's state is the 4 numbers (Q_k, J*_k) per field: bricks of kBrick cells with
// NM = 20 rows r = 4 k + m (m = 0: w_1 Q_k = Q_k / 8, the share of Q_k each moving population
// carries, as a deviation; 1..3: J*_k,x..z), so value m of field k of cell c is element
// mom_at(c) + (4 k + m) kBrick.  Keeping Q_k / 8 spares the pull a multiplication per population.  A pull reads Q_k and one component of J*_k
// of each source: scalar loads of whole 128-byte row segments per warp, no unused components.
constexpr int NM = 4 * NF;
__host__ __device__ __forceinline__ int64_t mom_at(int64_t c) {
    const uint64_t u = (uint64_t)c;
    return (int64_t)((u / kBrick) * (uint64_t)(NM * kBrick) + (u % kBrick));
}
__device__ __forceinline__ int64_t mom_at_u32(uint32_t c) {
    return (int64_t)(c >> 7) * (NM * kBrick) + (c & (kBrick - 1));
}
__host__ __device__ __forceinline__ int64_t brick_elems_m(int64_t N) {  // floats of one buffer
    return (N + kBrick - 1) / kBrick * (int64_t)(NM * kBrick);
}

enum Storage { S_F32 = 0, S_F16 = 1, S_BF16 = 2 };
// C_GATED: BGK where the sensor is off (chi = 0), the regularized collision with omega_h where
// it fires (chi > 0).
enum Collision { C_BGK = 0, C_RLB = 1, C_GATED = 2 };

// Per-domain lattice-unit constants.  Plain old data: passed by value as a kernel
// parameter for single-domain launches, read from a device array by the batched sweep.
struct DomainDev {
    void* buf[2];          // population buffers A, B (cell bricks, brick_elems(N) elements each)
    int64_t plane;         // cells N = nx*ny*nz
    int32_t nx, ny, nz, bc;
    int32_t cur;           // index of the buffer holding the current state (batched sweep)
    int32_t tile_x;        // cells along x per CTA in the batched sweep (divides blockDim.x);
                           // 1: linear tiles of 128 consecutive cells
    float gm1;             // gamma - 1
    float mu_ref, kap_ref; // lattice-unit transport at T_ref
    float inv_T_ref, T_S;  // Sutherland law: mu = mu_ref (1+T_S) t^{3/2}/(t+T_S), t = T/T_ref
    int32_t sutherland;
    float omega[3];        // rho, momentum, energy (nominal 1/tau_LB)
    float omega_red[3];    // max(omega_k - omega_min, 0): chi-scaled reduction (Listing 2)
    float gain, J_min, rho_min, p_min;
    float rho_ref, p_ref, E_ref;
    float ghostL[5];       // deviation of f_{k,+x} in the x = -1 ghost (X_DIRICHLET_EQ)
    float ghostR[5];       // deviation of f_{k,-x} in the x = nx ghost
    float dec[5];          // per-field storage scale: value = stored * dec[k]
    float enc[5];          // stored = value * enc[k] (a power of two)
    float enc_q0[5], enc_q1[5], enc_j[5];  // w_0 enc[k], w_1 enc[k], enc[k] / 2: the scale
                                           // folded into the constants of the outgoing set
    float ghostL_st[5];    // ghostL[k] enc[k], ghostR[k] enc[k]: the ghost values in stored units,
    float ghostR_st[5];    // rounded to the storage type (as a one-buffer slot holds them)
    void* outflow;         // one-buffer X_DIRICHLET_EQ: populations leaving through x = -1 / nx in
                           // an odd step, [side][k][y + ny z] (side 0: -x at x = 0, 1: +x at nx-1)
    const float* src;      // optional source S_k (5 planes, physical rates), or null
    float src_scale[3];    // physical rate -> lattice units per step (rho, momentum, energy)
    int32_t pad1;
};

// ---- storage traits ----------------------------------------------------------------------
// `scaled`: the stored value is deviation x enc[k] (FP16 only; FP32 and BF16 store the
// deviation itself, so no scale multiplications are compiled in for them).
template <int S> struct Store;
template <> struct Store<S_F32> {
    static constexpr bool scaled = false;
    using T = float;
    // read-only path with a 256-byte L2 prefetch hint: consecutive warps of a row stream
    // consecutive lines of every plane (measured 0.4% faster than a plain read-only load)
    static __device__ __forceinline__ float ld(const float* p) {
        float v;
        asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(GRLB_CHK_SRC(p)));
        return v;
    }
    static __device__ __forceinline__ float ld_plain(const float* p) { return GRLB_LD(p); }
    // default write-back store (measured 0.8% faster than the evict-first .cs hint)
    static __device__ __forceinline__ void st(float* p, float v) { GRLB_ST(p, v); }
};
template <> struct Store<S_F16> {
    static constexpr bool scaled = true;
    using T = __half;
    static __device__ __forceinline__ float ld(const __half* p) { return __half2float(GRLB_LDG(p)); }
    static __device__ __forceinline__ float ld_plain(const __half* p) { return __half2float(GRLB_LD(p)); }
    static __device__ __forceinline__ void st(__half* p, float v) { GRLB_ST(p, __float2half_rn(v)); }
};
template <> struct Store<S_BF16> {
    static constexpr bool scaled = false;
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) {
        return __bfloat162float(GRLB_LDG(p));
    }
    static __device__ __forceinline__ float ld_plain(const __nv_bfloat16* p) { return __bfloat162float(GRLB_LD(p)); }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) {
        GRLB_ST(p, __float2bfloat16_rn(v));
    }
};

// Division in the collide: the approximate reciprocal-and-multiply (__fdividef, within 2 ulp
// for the divisors here: rho >= rho_min, t + T_S, 1 + beta >= 1 and 1 + 4 omega_E (g-1) kappa /
// rho >= 1, all far inside its range), for every storage.  Without the IEEE division's slow
// path the sweeps need 64 registers instead of 89: the 16-bit sweeps (limited by instruction
// issue and latency) run 8-10 % faster, the moment-storage sweep 4 % (33.2 against 31.8
// GLUP/s, and at a higher clock under the power cap); the FP32 population sweep, HBM-bound,
// 0.8 % slower (0.678 against 0.673 ms).  Moment and population storage share the one
// division, so they stay bit for bit the same.
template <int S>
__device__ __forceinline__ float coll_div(float a, float b) {
    return __fdividef(a, b);
}

// Per-cell diagnostic values (FP32, reduced later in FP64).
struct CellDiag {
    float dQ[5];           // deviations of the conserved moments from Q_ref
    float ke, eps_s, eps_d;
    float rho_raw, p_raw;  // unfloored
    int floored, nan, sensor;
};

// Source projection of Alg. 1 step 9: o_{k,i} += w_i S_k (lattice units, storage units).
template <int S>
__device__ __forceinline__ void add_source(const DomainDev& D, int32_t c, float (&o)[NF][NQ]) {
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const int r = (k == 0) ? 0 : (k == 4 ? 2 : 1);
        float sk = GRLB_LDG(D.src + (int64_t)k * D.plane + c) * D.src_scale[r];
        if (Store<S>::scaled) sk *= D.enc[k];
        o[k][0] = fmaf(0.25f, sk, o[k][0]);
#pragma unroll
        for (int i = 1; i < NQ; ++i) o[k][i] = fmaf(0.125f, sk, o[k][i]);
    }
}

// ---- Algorithm 1 on one cell --------------------------------------------------------------
// moments (Alg. 1): dQ_k = sum_i d_ki, dJ_k = sum_i d_ki c_i of the stored values of one field,
// in deviation units (the storage scale is applied to the 4 moments, not the 7 populations).
template <int S>
__device__ __forceinline__ void field_moments(const DomainDev& D, int k, float d0, float d1, float d2,
                                              float d3, float d4, float d5, float d6, float& dQ,
                                              float (&dJ)[3]) {
    dQ = ((d0 + d1) + (d2 + d3)) + ((d4 + d5) + d6);
    dJ[0] = d1 - d2;
    dJ[1] = d3 - d4;
    dJ[2] = d5 - d6;
    if (Store<S>::scaled) {
        dQ *= D.dec[k];
        dJ[0] *= D.dec[k];
        dJ[1] *= D.dec[k];
        dJ[2] *= D.dec[k];
    }
}

template <int S, int COLL, bool DIAG, bool MOM = false>
__device__ __forceinline__ void collide_moments(const DomainDev& D, const float (&dQ)[NF],
                                                const float (&dJ)[NF][3], const float (&d)[NF][NQ],
                                                float (&o)[NF][NQ], CellDiag* cd);

// In: d[k][i] = pulled stored values (deviations, x enc[k] when scaled).  Out: o[k][i] = the
// values to store (post-collision deviations in the same units).
// MOM: the outgoing set as moments, o[k][0] = w_1 Q_k = Q_k / 8, o[k][1..3] = J*_k (regularized
// collision only: its outgoing set is w_i (Q_k + c_i . J*_k / cs^2), population i being
// fmaf(+-1/2, J*_k,a, Q_k / 8) for the links along axis a and Q_k / 4 = 2 (Q_k / 8) at rest).
template <int S, int COLL, bool DIAG, bool MOM = false>
__device__ __forceinline__ void collide(const DomainDev& D, const float (&d)[NF][NQ],
                                        float (&o)[NF][NQ], CellDiag* cd) {
    float dQ[NF], dJ[NF][3];
#pragma unroll
    for (int k = 0; k < NF; ++k)
        field_moments<S>(D, k, d[k][0], d[k][1], d[k][2], d[k][3], d[k][4], d[k][5], d[k][6], dQ[k], dJ[k]);
    collide_moments<S, COLL, DIAG, MOM>(D, dQ, dJ, d, o, cd);
}

// Everything after the moments: primitives and floors, reconstruction, sensor, closures,
// equilibrium and collision.  The regularized collision needs only (dQ, dJ); BGK also reads d.
// Each multiply-add that is to be fused is written as fmaf and the files that instantiate the
// collide are compiled without contraction, so its rounding is the same in every kernel.
template <int S, int COLL, bool DIAG, bool MOM>
__device__ __forceinline__ void collide_moments(const DomainDev& D, const float (&dQ)[NF],
                                                const float (&dJ)[NF][3], const float (&d)[NF][NQ],
                                                float (&o)[NF][NQ], CellDiag* cd) {
    static_assert(!MOM || (COLL == C_RLB && S == S_F32), "moment storage: FP32, regularized collision");
    constexpr bool SC = Store<S>::scaled;
    const float gm1 = D.gm1;
    // primitives with positivity floors (Alg. 1); Q_k themselves stay unfloored
    const float rho_raw = D.rho_ref + dQ[0];
    const float rho = fmaxf(rho_raw, D.rho_min);
    const float irho = coll_div<S>(1.0f, rho);
    const float m0 = dQ[1], m1 = dQ[2], m2 = dQ[3];
    const float u0 = m0 * irho, u1 = m1 * irho, u2 = m2 * irho;
    const float uu = fmaf(u0, u0, fmaf(u1, u1, u2 * u2));
    const float ke = 0.5f * fmaf(m0, u0, fmaf(m1, u1, m2 * u2));
    // p - p_ref = (gamma-1)(dE - ke): the pressure fluctuation without cancellation
    float dp = gm1 * (dQ[4] - ke);
    const float p_raw = D.p_ref + dp;
    float p = p_raw;
    if (p_raw < D.p_min) { p = D.p_min; dp = D.p_min - D.p_ref; }
    const float T = p * irho;
    const float E = D.E_ref + dQ[4];
    // transport (Listing 1)
    float fac = 1.0f;
    if (D.sutherland) {
        const float t = T * D.inv_T_ref;
        fac = coll_div<S>((1.0f + D.T_S) * t * sqrtf(t), t + D.T_S);
    }
    const float mu = D.mu_ref * fac;
    const float kap = D.kap_ref * fac;

    // non-equilibrium first moments J - Phi^adv (Eq. gradrecon), in deviation form
    const float Hp = E + p;  // (E + p)
    float nA[NF][3];
    nA[0][0] = dJ[0][0] - m0;
    nA[0][1] = dJ[0][1] - m1;
    nA[0][2] = dJ[0][2] - m2;
    const float mm[3] = {m0, m1, m2};
    const float uv[3] = {u0, u1, u2};
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float v = fmaf(-mm[j], uv[c], dJ[1 + j][c]);
            nA[1 + j][c] = j == c ? v - dp : v;
        }
#pragma unroll
    for (int c = 0; c < 3; ++c) nA[4][c] = fmaf(-Hp, uv[c], dJ[4][c]);

    // direct reconstruction grad Q~ = -omega Pi / cs^2 (cs^-2 = 4)
    const float w4r = -4.0f * D.omega[0], w4m = -4.0f * D.omega[1], w4e = -4.0f * D.omega[2];
    float gr[3], G[3][3], ge[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        gr[c] = w4r * nA[0][c];  // mass row of M is zero: grad rho passes through
        ge[c] = w4e * nA[4][c];
    }
    // momentum block (Eq. cnsfM row 2, Sec. 2.4): (I + b S) grad m = g~_m + b S(u (x) grad rho)
    // with b = omega_m mu / (cs^2 rho); solved in closed form: the antisymmetric part and the
    // trace pass through, the symmetric-deviatoric part is divided by 1 + beta, beta = 2b.
    const float a_mu = mu * irho;
    const float b = 4.0f * D.omega[1] * a_mu;
    const float ugr = fmaf(u0, gr[0], fmaf(u1, gr[1], u2 * gr[2]));
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float sg = fmaf(uv[j], gr[c], uv[c] * gr[j]);
            if (j == c) sg = fmaf(-(2.0f / 3.0f), ugr, sg);
            G[j][c] = fmaf(b, sg, w4m * nA[1 + j][c]);
        }
    {
        const float trG3 = (G[0][0] + G[1][1] + G[2][2]) * (1.0f / 3.0f);
        const float kdamp = coll_div<S>(2.0f * b, fmaf(2.0f, b, 1.0f));  // beta / (1 + beta)
        float Dv[3][3];
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                Dv[j][c] = j == c ? fmaf(0.5f, G[j][c] + G[c][j], -trG3) : 0.5f * (G[j][c] + G[c][j]);
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int c = 0; c < 3; ++c) G[j][c] = fmaf(-kdamp, Dv[j][c], G[j][c]);  // G := grad m
    }
    // energy row (Eq. cnsfE): scalar division with the corrected upstream gradients
    const float kr = kap * irho;
    float gmTu[3], Su[3];
    {
        const float trm23 = (2.0f / 3.0f) * (G[0][0] + G[1][1] + G[2][2]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            gmTu[c] = fmaf(G[0][c], u0, fmaf(G[1][c], u1, G[2][c] * u2));  // ((grad m)^T u)_c
            // (S(grad m) u)_c = sum_j (G_cj + G_jc) u_j - 2/3 tr(G) u_c
            Su[c] = fmaf(-trm23, uv[c],
                         fmaf(G[c][0] + G[0][c], u0, fmaf(G[c][1] + G[1][c], u1, (G[c][2] + G[2][c]) * u2)));
        }
    }
    {
        const float cT = kr * fmaf(-0.5f * gm1, uu, T);
        const float w4 = 4.0f * D.omega[2];
        const float gkr = gm1 * kr;
        const float inv = coll_div<S>(1.0f, fmaf(w4, gkr, 1.0f));
        const float ugr3 = (1.0f / 3.0f) * ugr;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float MEr = fmaf(a_mu, fmaf(uu, gr[c], ugr3 * uv[c]), cT * gr[c]);
            const float MEm = fmaf(-a_mu, Su[c], gkr * gmTu[c]);
            ge[c] = fmaf(w4, MEr + MEm, ge[c]) * inv;
        }
    }
    // chain rule (Sec. 2.4): grad u and grad T
    float gu[3][3], gT[3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int c = 0; c < 3; ++c) gu[j][c] = fmaf(-uv[j], gr[c], G[j][c]) * irho;
    {
        const float cr = fmaf(0.5f * gm1, uu, -T) * irho;
        const float cg = gm1 * irho;
#pragma unroll
        for (int c = 0; c < 3; ++c) gT[c] = fmaf(cg, ge[c] - gmTu[c], cr * gr[c]);
    }
    const float theta = gu[0][0] + gu[1][1] + gu[2][2];
    // compression sensor (Listing 2): s = -div u / cs, cs = 1/2
    float chi = 0.0f;
    if (COLL == C_RLB || COLL == C_GATED) {
        const float s = -2.0f * theta;
        if (theta < 0.0f && s > D.J_min) chi = fminf(fmaxf(D.gain * s, 0.0f), 1.0f);
    }
    // Newtonian stress and Fourier flux (Eq. system), full flux in deviation form:
    // Phi_rho = m; Phi_m_j - p_ref e_j = m_j u + dp e_j - tau_j; Phi_E = (E+p) u - tau u + q
    const float t23 = (2.0f / 3.0f) * theta;
    float tau[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int c = 0; c < 3; ++c) tau[j][c] = mu * (gu[j][c] + gu[c][j] - (j == c ? t23 : 0.0f));
    float Pd[NF][3];  // Phi_k - J_ref,k
    float Fd[NF][3];  // Phi^diff_k
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Pd[0][c] = mm[c];
        Fd[0][c] = 0.0f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            Fd[1 + j][c] = -tau[j][c];
            Pd[1 + j][c] = j == c ? fmaf(mm[j], uv[c], dp) - tau[j][c] : fmaf(mm[j], uv[c], -tau[j][c]);
        }
        const float tu = fmaf(tau[c][0], u0, fmaf(tau[c][1], u1, tau[c][2] * u2));
        Fd[4][c] = fmaf(-kap, gT[c], -tu);
        Pd[4][c] = fmaf(Hp, uv[c], Fd[4][c]);
    }

    // C_GATED takes one of the two per cell (chi is uniform over the cell's five fields)
    const bool regularized = COLL == C_RLB || (COLL == C_GATED && chi > 0.0f);
    if (regularized) {
        // regularized collision with reduced rate (Sec. 2.5):
        // f* = f^eq + (1 - omega_h) r, r = first-moment part of f - f^eq, so the outgoing
        // set is w_i (Q + c_i . J* / cs^2) with J* = Phi + (1 - omega_h)(J - Phi).
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            const int r = (k == 0) ? 0 : (k == 4 ? 2 : 1);
            const float omh = fmaf(-chi, D.omega_red[r], D.omega[r]);
            const float onem = 1.0f - omh;
            // storage scale (a power of two) folded into w_i and 1/2: every product is exact,
            // so the stored values equal those of scaling the outgoing set afterwards
            const float cq0 = SC ? D.enc_q0[k] : 0.25f;
            const float cq1 = SC ? D.enc_q1[k] : 0.125f;
            const float cj = SC ? D.enc_j[k] : 0.5f;
            float js[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) js[c] = fmaf(onem, nA[k][c] - Fd[k][c], Pd[k][c]);
            if (MOM) {
                o[k][0] = dQ[k] * cq1;  // w_1 Q_k: the rest of the set is rebuilt from it
                o[k][1] = js[0];
                o[k][2] = js[1];
                o[k][3] = js[2];
                continue;
            }
            const float q1 = dQ[k] * cq1;
            o[k][0] = dQ[k] * cq0;
            o[k][1] = fmaf(cj, js[0], q1);
            o[k][2] = fmaf(-cj, js[0], q1);
            o[k][3] = fmaf(cj, js[1], q1);
            o[k][4] = fmaf(-cj, js[1], q1);
            o[k][5] = fmaf(cj, js[2], q1);
            o[k][6] = fmaf(-cj, js[2], q1);
        }
    } else {
        // BGK (Sec. 2.2): f* = f + omega (f^eq - f)
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            const int r = (k == 0) ? 0 : (k == 4 ? 2 : 1);
            const float om = D.omega[r];
            const float sc = SC ? D.enc[k] : 1.0f;
            const float q1 = 0.125f * dQ[k] * sc;
            const float px = 0.5f * Pd[k][0] * sc, py = 0.5f * Pd[k][1] * sc, pz = 0.5f * Pd[k][2] * sc;
            float fe[NQ];
            fe[0] = 0.25f * dQ[k] * sc;
            fe[1] = q1 + px;
            fe[2] = q1 - px;
            fe[3] = q1 + py;
            fe[4] = q1 - py;
            fe[5] = q1 + pz;
            fe[6] = q1 - pz;
#pragma unroll
            for (int i = 0; i < NQ; ++i) o[k][i] = fmaf(om, fe[i] - d[k][i], d[k][i]);
        }
    }

    if (DIAG) {
#pragma unroll
        for (int k = 0; k < NF; ++k) cd->dQ[k] = dQ[k];
        cd->ke = ke;
        const float wx = gu[2][1] - gu[1][2], wy = gu[0][2] - gu[2][0], wz = gu[1][0] - gu[0][1];
        cd->eps_s = mu * fmaf(wx, wx, fmaf(wy, wy, wz * wz));
        cd->eps_d = (4.0f / 3.0f) * mu * theta * theta;
        cd->rho_raw = rho_raw;
        cd->p_raw = p_raw;
        cd->floored = (rho_raw < D.rho_min) || (p_raw < D.p_min);
        bool fin = true;
#pragma unroll
        for (int k = 0; k < NF; ++k) fin = fin && isfinite(dQ[k]);
        cd->nan = !fin;
        cd->sensor = chi > 0.0f;
    }
}

}  // namespace grlb
