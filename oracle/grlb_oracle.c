/*
 * grlb_oracle.c -- plain FP64 CPU oracle of the five-field gradient-reconstruction
 * lattice Boltzmann scheme for the compressible Navier-Stokes-Fourier equations
 * (arxiv 2609.16361).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference that the
 * CUDA sweep is checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it; the product path never does.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Everything here runs in lattice units (dx = dt = 1) on FP64 populations that are NOT
 * shifted by any reference state.  Layout: f[(k*7 + i)*N + x + nx*(y + ny*z)], field k in
 * (rho, m_x, m_y, m_z, E), link i in (0, +x, -x, +y, -y, +z, -z).
 *
 * Per-cell update = Algorithm 1 of the paper, in its order:
 *   moments (Alg. 1 first step), floors (second step), non-equilibrium first moment
 *   Pi^(1) (Eq. gradrecon), direct reconstruction grad Q~ = -Pi^(1)/(cs^2 tau_LB),
 *   reconstruction operator R = (I - cs^-2 diag(omega) M)^-1 (Eq. feedback) applied by
 *   building the 15x15 Jacobian M of Eq. cnsfM literally and solving the linear system with
 *   Gaussian elimination (the definition of R, not the closed-form block solve),
 *   chain rule to grad u, grad T (Sec. 2.4), compression sensor chi (Sec. 2.5 /
 *   Listing 2), Newtonian stress and Fourier flux (Eq. system), linear equilibrium with the
 *   full flux in its first moment (Sec. 2.2), regularized collision with reduced rate
 *   (Sec. 2.5), BGK (Sec. 2.2), or the sensor-gated pair of the two (BGK where chi = 0, the
 *   regularized collision where chi > 0: the reading of Sec. 2.2 in which the compression
 *   sensor activates the regularized operator in place of BGK), exact streaming (pull form).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *  - D3Q7 weights for cs^2 = 1/4: w0 = 1/4, w1..6 = 1/8 (unique isotropic choice).
 *  - Q_k in the equilibrium is the unfloored zeroth moment (floors touch primitives only).
 *  - the nominal omega_k (never omega_h) enters Eq. gradrecon and R.
 *  - omega_h = omega - chi * max(omega - omega_min, 0): the sensor never raises the rate.
 *  - X_DIRICHLET_EQ: ghost cells at x = -1 and x = nx hold the equilibrium (zero
 *    non-equilibrium) populations of fixed left / right primitive states; y, z periodic.
 *
 * Pins (tests): exact conservation on periodic domains, invariance of a uniform
 * equilibrium, exact algebraic recovery of grad Q from a first moment built from the
 * physical stress and heat-flux definitions, the exact Sod Riemann solution, the Becker
 * viscous-shock closed form, low-Mach viscous decay of a Taylor-Green vortex.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NF 5
#define NQ 7
#define NP (NF * NQ)
#define NG 15

/* D3Q7 links: 0, +x, -x, +y, -y, +z, -z (Sec. 2.2). */
static const int CI[NQ][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0},
                              {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
static const double WI[NQ] = {0.25, 0.125, 0.125, 0.125, 0.125, 0.125, 0.125};
static const double CS2 = 0.25;

/* Lattice-unit parameters.  Mirrors what a case prescribes, already converted. */
typedef struct {
    int nx, ny, nz;
    int bc;          /* 0 periodic, 1 x-Dirichlet equilibrium ghosts */
    int collision;   /* 0 BGK, 1 regularized + compression sensor, 2 sensor-gated:
                        BGK where chi = 0, regularized with omega_h where chi > 0 */
    int sutherland;  /* 0 constant mu */
    double gamma;
    double mu_ref, kappa_ref, T_ref, T_S;
    double omega[NF];
    double omega_min, gain, J_min;
    double rho_min, p_min;
    double left[5], right[5]; /* primitive (rho, ux, uy, uz, p) of the ghost states */
} orc_params;

/* Per-cell byproducts, for diagnostics and unit tests. */
typedef struct {
    double Q[NF];        /* unfloored conserved moments */
    double rho, u[3], p, T, mu, kappa;
    double gradQ[NG];    /* reconstructed conserved gradients, (rho | m_x m_y m_z | E) x (d/dx..) */
    double gradu[9];     /* (grad u)_{jc} = d u_j / d x_c, row-major */
    double gradT[3];
    double chi;
    int floored;         /* 1 if rho or p hit its floor */
} orc_cell_info;

/* ---- transport coefficients (Listing 1) ----------------------------------------------- */
static void transport(const orc_params* P, double T, double* mu, double* kappa) {
    if (P->sutherland) {
        double t = T / P->T_ref;
        double f = (1.0 + P->T_S) * pow(t, 1.5) / (t + P->T_S);
        *mu = P->mu_ref * f;
        *kappa = P->kappa_ref * f; /* kappa scaled by mu_T / mu */
    } else {
        *mu = P->mu_ref;
        *kappa = P->kappa_ref;
    }
}

/* ---- advective flux Phi^adv(Q) = Phi|_{grad Q = 0} (Eq. system, Eq. gradrecon) -------- */
static void advective_flux(const double Q[NF], double rho, const double u[3], double p,
                           double Phi[NF][3]) {
    for (int c = 0; c < 3; ++c) {
        Phi[0][c] = Q[1 + c];
        for (int j = 0; j < 3; ++j) Phi[1 + j][c] = Q[1 + j] * u[c] + (j == c ? p : 0.0);
        Phi[4][c] = (Q[4] + p) * u[c];
    }
    (void)rho;
}

/* ---- diffusive-flux Jacobian M (Eq. cnsfM) ---------------------------------------------
 * Unknown vector g (15): g[0..2] = d rho/dx_c, g[3 + 3j + c] = d m_j / dx_c, g[12 + c] = d E/dx_c.
 * Row r indexes Phi^diff the same way (field-major, direction-minor).                     */
static int gi_rho(int c) { return c; }
static int gi_m(int j, int c) { return 3 + 3 * j + c; }
static int gi_E(int c) { return 12 + c; }

static void build_M(double rho, const double u[3], double T, double mu, double kappa,
                    double gamma, double M[NG][NG]) {
    memset(M, 0, sizeof(double) * NG * NG);
    const double a = mu / rho, kr = kappa / rho;
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    /* mass row: zero */
    /* momentum row m_j, direction c */
    for (int j = 0; j < 3; ++j)
        for (int c = 0; c < 3; ++c) {
            const int r = gi_m(j, c);
            /* (mu/rho) S(u (x) grad rho): S(X)_{jc} = X_jc + X_cj - 2/3 delta_jc tr X, X = u_j d_c rho */
            for (int d = 0; d < 3; ++d) {
                double s = (c == d ? u[j] : 0.0) + (j == d ? u[c] : 0.0) -
                           (j == c ? (2.0 / 3.0) * u[d] : 0.0);
                M[r][gi_rho(d)] += a * s;
            }
            /* -(mu/rho) S(grad m) */
            for (int l = 0; l < 3; ++l)
                for (int d = 0; d < 3; ++d) {
                    double s = (j == l && c == d ? 1.0 : 0.0) + (c == l && j == d ? 1.0 : 0.0) -
                               (j == c && l == d ? 2.0 / 3.0 : 0.0);
                    M[r][gi_m(l, d)] += -a * s;
                }
        }
    /* energy row, direction c */
    for (int c = 0; c < 3; ++c) {
        const int r = gi_E(c);
        for (int d = 0; d < 3; ++d) {
            double s = a * ((c == d ? uu : 0.0) + u[c] * u[d] / 3.0) +
                       kr * (T - 0.5 * (gamma - 1.0) * uu) * (c == d ? 1.0 : 0.0);
            M[r][gi_rho(d)] += s;
        }
        /* -(mu/rho) (S grad m) u + ((gamma-1) kappa/rho) (grad m)^T u */
        for (int l = 0; l < 3; ++l)
            for (int d = 0; d < 3; ++d) {
                /* (S(G) u)_c = sum_j S_cj u_j; dS_cj/dG_ld = d_cl d_jd + d_jl d_cd - 2/3 d_cj d_ld */
                double su = (c == l ? u[d] : 0.0) + (c == d ? u[l] : 0.0) -
                            (l == d ? (2.0 / 3.0) * u[c] : 0.0);
                double gtu = (c == d ? u[l] : 0.0); /* ((grad m)^T u)_c = sum_j d_c m_j u_j */
                M[r][gi_m(l, d)] += -a * su + (gamma - 1.0) * kr * gtu;
            }
        M[r][gi_E(c)] += -(gamma - 1.0) * kr;
    }
}

/* Gaussian elimination with partial pivoting, A x = b in place (b <- x). */
static int solve_dense(int n, double A[NG][NG], double b[NG]) {
    for (int col = 0; col < n; ++col) {
        int piv = col;
        double best = fabs(A[col][col]);
        for (int r = col + 1; r < n; ++r)
            if (fabs(A[r][col]) > best) { best = fabs(A[r][col]); piv = r; }
        if (!(best > 0.0)) return -1;
        if (piv != col) {
            for (int c = 0; c < n; ++c) { double t = A[col][c]; A[col][c] = A[piv][c]; A[piv][c] = t; }
            double t = b[col]; b[col] = b[piv]; b[piv] = t;
        }
        for (int r = col + 1; r < n; ++r) {
            double f = A[r][col] / A[col][col];
            if (f == 0.0) continue;
            for (int c = col; c < n; ++c) A[r][c] -= f * A[col][c];
            b[r] -= f * b[col];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int c = r + 1; c < n; ++c) s -= A[r][c] * b[c];
        b[r] = s / A[r][r];
    }
    return 0;
}

/* Linear equilibrium of one field: f^eq_i = w_i (Q + c_i . Phi / cs^2) (Sec. 2.2). */
static void equilibrium(double Q, const double Phi[3], double feq[NQ]) {
    for (int i = 0; i < NQ; ++i) {
        double cphi = CI[i][0] * Phi[0] + CI[i][1] * Phi[1] + CI[i][2] * Phi[2];
        feq[i] = WI[i] * (Q + cphi / CS2);
    }
}

/* Zero-non-equilibrium populations of a primitive state (rho, ux, uy, uz, p). */
void orc_equilibrium_state(const orc_params* P, const double prim[5], double f[NP]) {
    double rho = prim[0], u[3] = {prim[1], prim[2], prim[3]}, p = prim[4];
    double Q[NF];
    Q[0] = rho;
    for (int j = 0; j < 3; ++j) Q[1 + j] = rho * u[j];
    Q[4] = p / (P->gamma - 1.0) + 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double Phi[NF][3];
    advective_flux(Q, rho, u, p, Phi);
    for (int k = 0; k < NF; ++k) equilibrium(Q[k], Phi[k], f + k * NQ);
}

/* One cell of Algorithm 1: post-streaming populations fhat -> post-collision fstar. */
int orc_cell(const orc_params* P, const double fhat[NP], double fstar[NP], orc_cell_info* info) {
    const double g = P->gamma;
    /* Alg. 1, moments */
    double Q[NF], J[NF][3];
    for (int k = 0; k < NF; ++k) {
        double q = 0.0, j0 = 0.0, j1 = 0.0, j2 = 0.0;
        for (int i = 0; i < NQ; ++i) {
            double f = fhat[k * NQ + i];
            q += f;
            j0 += f * CI[i][0];
            j1 += f * CI[i][1];
            j2 += f * CI[i][2];
        }
        Q[k] = q;
        J[k][0] = j0; J[k][1] = j1; J[k][2] = j2;
    }
    /* Alg. 1, primitives with positivity floor */
    int floored = 0;
    double rho = Q[0];
    if (rho < P->rho_min) { rho = P->rho_min; floored = 1; }
    double u[3] = {Q[1] / rho, Q[2] / rho, Q[3] / rho};
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double p = (g - 1.0) * (Q[4] - 0.5 * rho * uu);
    if (p < P->p_min) { p = P->p_min; floored = 1; }
    double T = p / rho;
    double mu, kappa;
    transport(P, T, &mu, &kappa);

    /* Alg. 1, non-equilibrium first moment and direct reconstruction (Eq. gradrecon) */
    double Phiadv[NF][3];
    advective_flux(Q, rho, u, p, Phiadv);
    double gt[NG];
    for (int c = 0; c < 3; ++c) {
        gt[gi_rho(c)] = -P->omega[0] * (J[0][c] - Phiadv[0][c]) / CS2;
        for (int j = 0; j < 3; ++j)
            gt[gi_m(j, c)] = -P->omega[1 + j] * (J[1 + j][c] - Phiadv[1 + j][c]) / CS2;
        gt[gi_E(c)] = -P->omega[4] * (J[4][c] - Phiadv[4][c]) / CS2;
    }
    /* Eq. feedback: (I - cs^-2 diag(omega) M) grad Q = grad Q~ */
    double M[NG][NG], A[NG][NG];
    build_M(rho, u, T, mu, kappa, g, M);
    for (int r = 0; r < NG; ++r) {
        double om = (r < 3) ? P->omega[0] : (r < 12 ? P->omega[1 + (r - 3) / 3] : P->omega[4]);
        for (int c = 0; c < NG; ++c) A[r][c] = (r == c ? 1.0 : 0.0) - om / CS2 * M[r][c];
    }
    double gq[NG];
    memcpy(gq, gt, sizeof gq);
    if (solve_dense(NG, A, gq) != 0) return -1;

    /* chain rule: grad u = (grad m - u (x) grad rho)/rho (Sec. 2.4) */
    double gu[9];
    for (int j = 0; j < 3; ++j)
        for (int c = 0; c < 3; ++c) gu[3 * j + c] = (gq[gi_m(j, c)] - u[j] * gq[gi_rho(c)]) / rho;
    /* grad T = (gamma-1)/rho (grad E - sum_j u_j grad m_j) + (1/rho)((gamma-1)/2 |u|^2 - T) grad rho */
    double gT[3];
    for (int c = 0; c < 3; ++c) {
        double s = gq[gi_E(c)];
        for (int j = 0; j < 3; ++j) s -= u[j] * gq[gi_m(j, c)];
        gT[c] = (g - 1.0) / rho * s + (0.5 * (g - 1.0) * uu - T) / rho * gq[gi_rho(c)];
    }

    /* Alg. 1, compression sensor (Listing 2); cs = 1/2 in lattice units */
    double div = gu[0] + gu[4] + gu[8];
    double chi = 0.0;
    if (P->collision == 1 || P->collision == 2) {
        double s = -div / sqrt(CS2);
        if (div < 0.0 && s > P->J_min) {
            chi = P->gain * s;
            if (chi > 1.0) chi = 1.0;
            if (chi < 0.0) chi = 0.0;
        }
    }

    /* Alg. 1, Newtonian stress and Fourier flux (Eq. system) */
    double tau[3][3], q[3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            tau[a][b] = mu * (gu[3 * a + b] + gu[3 * b + a] - (a == b ? (2.0 / 3.0) * div : 0.0));
    for (int c = 0; c < 3; ++c) q[c] = -kappa * gT[c];

    /* full flux: Phi_rho = m; Phi_m_j = m_j u + p e_j - tau_j; Phi_E = (E+p)u - tau u + q */
    double Phi[NF][3];
    for (int c = 0; c < 3; ++c) {
        Phi[0][c] = Phiadv[0][c];
        for (int j = 0; j < 3; ++j) Phi[1 + j][c] = Phiadv[1 + j][c] - tau[j][c];
        double tu = tau[c][0] * u[0] + tau[c][1] * u[1] + tau[c][2] * u[2];
        Phi[4][c] = Phiadv[4][c] - tu + q[c];
    }

    /* Alg. 1, equilibrium and collision */
    for (int k = 0; k < NF; ++k) {
        double feq[NQ];
        equilibrium(Q[k], Phi[k], feq);
        const int regularized = P->collision == 1 || (P->collision == 2 && chi > 0.0);
        if (regularized) {
            /* regularized: keep only the first-moment part r of f - f^eq (Sec. 2.5) */
            double om = P->omega[k];
            double red = om - P->omega_min;
            if (red < 0.0) red = 0.0;
            double omh = om - chi * red;
            double d[3];
            for (int c = 0; c < 3; ++c) {
                double s = 0.0;
                for (int i = 0; i < NQ; ++i) s += (fhat[k * NQ + i] - feq[i]) * CI[i][c];
                d[c] = s;
            }
            for (int i = 0; i < NQ; ++i) {
                double r = WI[i] * (CI[i][0] * d[0] + CI[i][1] * d[1] + CI[i][2] * d[2]) / CS2;
                fstar[k * NQ + i] = feq[i] + (1.0 - omh) * r;
            }
        } else {
            double om = P->omega[k];
            for (int i = 0; i < NQ; ++i) {
                double f = fhat[k * NQ + i];
                fstar[k * NQ + i] = f - om * (f - feq[i]);
            }
        }
    }

    if (info) {
        for (int k = 0; k < NF; ++k) info->Q[k] = Q[k];
        info->rho = rho;
        for (int j = 0; j < 3; ++j) info->u[j] = u[j];
        info->p = p; info->T = T; info->mu = mu; info->kappa = kappa;
        memcpy(info->gradQ, gq, sizeof gq);
        memcpy(info->gradu, gu, sizeof gu);
        memcpy(info->gradT, gT, sizeof gT);
        info->chi = chi;
        info->floored = floored;
    }
    return 0;
}

/* Reconstruction alone, for unit tests: given fhat return grad Q, grad u, grad T, chi ... */
int orc_cell_info_only(const orc_params* P, const double fhat[NP], orc_cell_info* info) {
    double fstar[NP];
    return orc_cell(P, fhat, fstar, info);
}

size_t orc_cell_info_size(void) { return sizeof(orc_cell_info); }

/* ---- streaming + collision over the whole domain ---------------------------------------
 * fin holds post-collision populations at time n; fout receives those at time n+1.
 * Pull form of the exact streaming f(x + c_i, n+1) = f*(x, n).
 * cell_out (nullable): per-cell info records (N entries) of the pre-collision state n+1.   */
/* src (nullable): per-cell source S_k in lattice units per step, layout src[k*N + idx]; its
 * projection w_i S_k is added to the post-collision populations (Alg. 1 step 9). */
int orc_step_src(const orc_params* P, const double* fin, double* fout, orc_cell_info* cell_out,
                 const double* src);
int orc_step(const orc_params* P, const double* fin, double* fout, orc_cell_info* cell_out) {
    return orc_step_src(P, fin, fout, cell_out, NULL);
}

int orc_step_src(const orc_params* P, const double* fin, double* fout, orc_cell_info* cell_out,
                 const double* src) {
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    const long N = (long)nx * ny * nz;
    double gl[NP], gr[NP];
    orc_equilibrium_state(P, P->left, gl);
    orc_equilibrium_state(P, P->right, gr);
    int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
    for (int z = 0; z < nz; ++z) {
        double fhat[NP], fstar[NP];
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long idx = x + (long)nx * (y + (long)ny * z);
                for (int k = 0; k < NF; ++k)
                    for (int i = 0; i < NQ; ++i) {
                        int xs = x - CI[i][0], ys = y - CI[i][1], zs = z - CI[i][2];
                        ys = (ys + ny) % ny;
                        zs = (zs + nz) % nz;
                        double v;
                        if (P->bc == 1 && xs < 0) {
                            v = gl[k * NQ + i];
                        } else if (P->bc == 1 && xs >= nx) {
                            v = gr[k * NQ + i];
                        } else {
                            xs = (xs + nx) % nx;
                            v = fin[(long)(k * NQ + i) * N + xs + (long)nx * (ys + (long)ny * zs)];
                        }
                        fhat[k * NQ + i] = v;
                    }
                orc_cell_info* inf = cell_out ? &cell_out[idx] : NULL;
                if (orc_cell(P, fhat, fstar, inf) != 0) err |= 1;
                if (src)
                    for (int k = 0; k < NF; ++k)
                        for (int i = 0; i < NQ; ++i) fstar[k * NQ + i] += WI[i] * src[(long)k * N + idx];
                for (int q = 0; q < NP; ++q) fout[(long)q * N + idx] = fstar[q];
            }
    }
    return err ? -1 : 0;
}

/* Initial populations: equilibrium of the given primitive fields (zero non-equilibrium). */
void orc_init_equilibrium(const orc_params* P, const double* rho, const double* ux,
                          const double* uy, const double* uz, const double* p, double* f) {
    const long N = (long)P->nx * P->ny * P->nz;
#pragma omp parallel for schedule(static)
    for (long idx = 0; idx < N; ++idx) {
        double prim[5] = {rho[idx], ux[idx], uy[idx], uz[idx], p[idx]};
        double fe[NP];
        orc_equilibrium_state(P, prim, fe);
        for (int q = 0; q < NP; ++q) f[(long)q * N + idx] = fe[q];
    }
}

/* Conserved moments Q_k = sum_i f_{k,i} (unchanged by collision, so read locally). */
void orc_moments(const orc_params* P, const double* f, double* Q) {
    const long N = (long)P->nx * P->ny * P->nz;
#pragma omp parallel for schedule(static)
    for (long idx = 0; idx < N; ++idx)
        for (int k = 0; k < NF; ++k) {
            double s = 0.0;
            for (int i = 0; i < NQ; ++i) s += f[(long)(k * NQ + i) * N + idx];
            Q[(long)k * N + idx] = s;
        }
}

#ifdef _OPENMP
#include <omp.h>
#endif
/* Threads the OpenMP loops use (1 without OpenMP). */
int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
