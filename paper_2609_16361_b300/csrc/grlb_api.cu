// grlb_api.cu -- the C ABI of include/grlb.h: parameter validation and lattice conversion,
// device memory ownership, launch configuration, readback, checkpoints and batching.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "grlb.h"
#include "grlb_kernels.h"

using grlb::DomainDev;
using grlb::NDIAG;

namespace {

thread_local std::string g_err;

grlb_status fail(grlb_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

grlb_status cuda_fail(cudaError_t e, const char* what) {
    return fail(GRLB_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define GRLB_CU(call)                                      \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

size_t elem_bytes(int storage) { return storage == GRLB_STORE_F32 ? 4 : 2; }
// one population buffer: N cells in cell bricks (whole bricks of 35 x 128 elements)
size_t pop_bytes(size_t N, int storage) { return (size_t)grlb::brick_elems((int64_t)N) * elem_bytes(storage); }
// streaming = 1: one population buffer (AA pattern); 2: two buffers of moments (FP32, regularized
// collision: 20 values per cell instead of 35)
bool one_buffer(const grlb_params& p) { return p.streaming == 1; }
bool moment_storage(const grlb_params& p) { return p.streaming == 2; }
// one state buffer of N cells
size_t state_bytes(size_t N, const grlb_params& p) {
    if (moment_storage(p)) return (size_t)grlb::brick_elems_m((int64_t)N) * sizeof(float);
    return pop_bytes(N, p.storage);
}

// One-buffer Dirichlet domains keep the populations that leave through the ends in an odd step.
size_t outflow_bytes(const grlb_params& p) {
    return (one_buffer(p) && p.bc == GRLB_BC_X_DIRICHLET_EQ) ? 10 * (size_t)p.ny * p.nz * elem_bytes(p.storage) : 0;
}

// Power-of-two storage scale for the 16-bit modes: deviations of field k are divided by a
// reference magnitude M_k (rho_ref, rho_ref c_ref, E_ref) and multiplied by 2^8 so that
// typical fluctuations sit well inside the FP16 normal range.  FP32 and BF16 use 1.
float storage_scale(int storage, double Mk) {
    if (storage != GRLB_STORE_F16) return 1.0f;
    const int e = (int)std::lround(std::log2(Mk));
    return std::ldexp(1.0f, 8 - e);
}

// A value in stored units as the storage type holds it (round to nearest even for FP16 / BF16):
// the Dirichlet ghost populations are kept so, because the one-buffer pattern writes them to a
// slot of the boundary cell and reads them back, and the two-buffer sweep must pull the same
// number.
float as_stored(int storage, float v) {
    if (storage == GRLB_STORE_F16) return __half2float(__float2half_rn(v));
    if (storage == GRLB_STORE_BF16) return __bfloat162float(__float2bfloat16_rn(v));
    return v;
}

// Device memory of domains and batches comes from the device's stream-ordered pool
// (cudaMallocAsync / cudaFreeAsync): freeing does not synchronise the device, so a serving loop
// can release a finished request while the others keep running.  The pool keeps released
// memory for reuse (this process only).
void retain_pool() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    done[dev] = true;
}

}  // namespace

struct grlb_domain {
    grlb_params P;
    DomainDev D;
    cudaStream_t stream = nullptr;
    int device = 0;
    double s = 1.0, gm1 = 0.4, rho_ref = 1.0, p_ref = 1.0, E_ref = 1.0;
    double* partials = nullptr;
    int64_t nblocks = 0;
    double* diag_dev = nullptr;
    int64_t steps = 0;
    int64_t diag_step = -1;
    dim3 grid, block;
    size_t bytes = 0;
    // pipelined initialisation (grlb_stage_primitive / grlb_init_from_stage)
    double* stage[2] = {nullptr, nullptr};   // allocated when filled, released when consumed
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t staged[2] = {nullptr, nullptr};
    int stage_head = 0, stage_count = 0;
    int ce_init = 0;  // grlb_set_init_mode
    // grlb_step replays kStepGraphSweeps plain sweeps from a CUDA graph on small domains; the
    // graph starts from buffer graph_cur at step parity graph_parity
    cudaGraphExec_t step_graph = nullptr;
    int graph_cur = 0, graph_parity = 0;
};

extern "C" {

const char* grlb_last_error(void) { return g_err.c_str(); }
const char* grlb_version(void) { return "grlb 0.1 (sm_103a)"; }

static grlb_status validate(const grlb_params* p) {
    if (!p) return fail(GRLB_EINVAL, "params is NULL");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail(GRLB_EINVAL, "nx, ny, nz must be >= 1");
    const long double N = (long double)p->nx * p->ny * p->nz;
    if (N >= 2147483647.0L) return fail(GRLB_EINVAL, "nx*ny*nz must be < 2^31");
    if (p->nz > 65535) return fail(GRLB_EINVAL, "nz must be <= 65535");
    if (p->bc != GRLB_BC_PERIODIC && p->bc != GRLB_BC_X_DIRICHLET_EQ) return fail(GRLB_EINVAL, "bad bc");
    if (p->collision != GRLB_COLL_BGK && p->collision != GRLB_COLL_RLB_SENSOR &&
        p->collision != GRLB_COLL_RLB_GATED)
        return fail(GRLB_EINVAL, "bad collision");
    if (p->storage < GRLB_STORE_F32 || p->storage > GRLB_STORE_BF16) return fail(GRLB_EINVAL, "bad storage");
    if (p->streaming < 0 || p->streaming > 2) return fail(GRLB_EINVAL, "streaming must be 0, 1 or 2");
    if (p->streaming == 2 && (p->storage != GRLB_STORE_F32 || p->collision != GRLB_COLL_RLB_SENSOR))
        return fail(GRLB_EINVAL, "moment storage (streaming = 2) needs FP32 storage and the regularized collision");
    if (!(p->dx > 0) || !(p->dt > 0)) return fail(GRLB_EINVAL, "dx, dt must be > 0");
    if (!(p->gamma > 1)) return fail(GRLB_EINVAL, "gamma must be > 1");
    if (!(p->mu_ref >= 0) || !(p->prandtl > 0) || !(p->T_ref > 0) || !(p->T_S >= 0))
        return fail(GRLB_EINVAL, "bad transport parameters");
    const double om[3] = {p->omega_rho, p->omega_mom, p->omega_E};
    for (double w : om)
        if (!(w > 0 && w <= 2)) return fail(GRLB_EINVAL, "omega must be in (0, 2]");
    if (!(p->ref_rho > 0) || !(p->ref_p > 0)) return fail(GRLB_EINVAL, "reference state must be positive");
    if (!(p->rho_min > 0) || !(p->p_min > 0)) return fail(GRLB_EINVAL, "floors must be > 0");
    if (p->bc == GRLB_BC_X_DIRICHLET_EQ)
        for (int s = 0; s < 2; ++s) {
            const double* g = s ? p->right_prim : p->left_prim;
            if (!(g[0] > 0) || !(g[4] > 0)) return fail(GRLB_EINVAL, "ghost states must have rho, p > 0");
        }
    return GRLB_OK;
}

// Deviation of the +x (sign=+1) or -x (sign=-1) equilibrium population of field k of a
// primitive state (lattice units) from the reference equilibrium.
static void ghost_dev(const grlb_domain* d, const double prim[5], int sign, float out[5]) {
    const double s = d->s, g1 = d->gm1;
    const double r = prim[0], u[3] = {prim[1] * s, prim[2] * s, prim[3] * s}, p = prim[4] * s * s;
    const double m[3] = {r * u[0], r * u[1], r * u[2]};
    const double ke = 0.5 * (m[0] * u[0] + m[1] * u[1] + m[2] * u[2]);
    const double dQ[5] = {r - d->rho_ref, m[0], m[1], m[2], (p - d->p_ref) / g1 + ke};
    const double E = d->E_ref + dQ[4];
    double Px[5];  // x component of Phi^adv - J_ref
    Px[0] = m[0];
    Px[1] = m[0] * u[0] + (p - d->p_ref);
    Px[2] = m[1] * u[0];
    Px[3] = m[2] * u[0];
    Px[4] = (E + p) * u[0];
    for (int k = 0; k < 5; ++k) out[k] = (float)(0.125 * dQ[k] + sign * 0.5 * Px[k]);
}

static void fill_domain_dev(grlb_domain* d) {
    const grlb_params& p = d->P;
    DomainDev& D = d->D;
    const double s = p.dt / p.dx;
    d->s = s;
    d->gm1 = p.gamma - 1.0;
    d->rho_ref = p.ref_rho;
    d->p_ref = p.ref_p * s * s;
    d->E_ref = d->p_ref / d->gm1;
    D.plane = (int64_t)p.nx * p.ny * p.nz;
    D.nx = p.nx;
    D.ny = p.ny;
    D.nz = p.nz;
    D.bc = p.bc;
    D.cur = 0;
    D.tile_x = 128;
    D.gm1 = (float)d->gm1;
    const double mu_L = p.mu_ref * p.dt / (p.dx * p.dx);
    const double cp = p.gamma / (p.gamma - 1.0);
    D.mu_ref = (float)mu_L;
    D.kap_ref = (float)(mu_L * cp / p.prandtl);
    D.inv_T_ref = (float)(1.0 / (p.T_ref * s * s));
    D.T_S = (float)p.T_S;
    D.sutherland = p.sutherland ? 1 : 0;
    const double om[3] = {p.omega_rho, p.omega_mom, p.omega_E};
    for (int r = 0; r < 3; ++r) {
        D.omega[r] = (float)om[r];
        D.omega_red[r] = (float)std::max(om[r] - p.omega_min, 0.0);
    }
    D.gain = (float)p.sensor_gain;
    D.J_min = (float)p.J_min;
    D.rho_min = (float)p.rho_min;
    D.p_min = (float)(p.p_min * s * s);
    D.rho_ref = (float)d->rho_ref;
    D.p_ref = (float)d->p_ref;
    D.E_ref = (float)d->E_ref;
    if (p.bc == GRLB_BC_X_DIRICHLET_EQ) {
        ghost_dev(d, p.left_prim, +1, D.ghostL);
        ghost_dev(d, p.right_prim, -1, D.ghostR);
    } else {
        for (int k = 0; k < 5; ++k) D.ghostL[k] = D.ghostR[k] = 0.0f;
    }
    const double c_ref = std::sqrt(p.gamma * d->p_ref / d->rho_ref);
    const double M[5] = {d->rho_ref, d->rho_ref * c_ref, d->rho_ref * c_ref, d->rho_ref * c_ref, d->E_ref};
    for (int k = 0; k < 5; ++k) {
        D.enc[k] = storage_scale(p.storage, M[k]);
        D.dec[k] = 1.0f / D.enc[k];
        D.enc_q0[k] = 0.25f * D.enc[k];
        D.enc_q1[k] = 0.125f * D.enc[k];
        D.enc_j[k] = 0.5f * D.enc[k];
        D.ghostL_st[k] = as_stored(p.storage, D.ghostL[k] * D.enc[k]);
        D.ghostR_st[k] = as_stored(p.storage, D.ghostR[k] * D.enc[k]);
    }
    D.src = nullptr;
    D.outflow = nullptr;
    D.src_scale[0] = (float)p.dt;
    D.src_scale[1] = (float)(p.dt * s);
    D.src_scale[2] = (float)(p.dt * s * s);
    D.pad1 = 0;
}

// CTA of 128 threads = bx cells along x times by rows.  bx in {128, 64, 32} is the width that
// pads the row least (idle lanes cost throughput: nx = 130 on 128-wide tiles leaves half the
// lanes of every row idle), the wider one on ties -- the narrower one for moment storage, whose
// sweep reads every cell's moments from up to 7 threads: with 4 rows per CTA the +-y sources
// are mostly L1 hits (256^3: 0.518 ms on 32 x 4 tiles, 0.522 on 64 x 2, 0.532 on 128 x 1).
static void choose_launch(grlb_domain* d) {
    const int nx = d->P.nx;
    const bool narrow = moment_storage(d->P);
    int bx = 128;
    long best = -1;
    for (int w = 128; w >= 32; w /= 2) {
        const long padded = (long)((nx + w - 1) / w) * w;
        if (best < 0 || padded < best || (narrow && padded == best)) {
            best = padded;
            bx = w;
        }
    }
    int by = 128 / bx;
    while (by > 1 && by / 2 >= d->P.ny) by /= 2;
    const double padded = (double)((nx + bx - 1) / bx * bx) * ((d->P.ny + by - 1) / by * by);
    if (padded > 1.05 * (double)nx * d->P.ny) {
        // rows do not fill whole tiles: take cells in storage order instead (block.y == 0
        // tells the launcher), one 128-cell CTA after another
        const int64_t N = (int64_t)nx * d->P.ny * d->P.nz;
        d->block = dim3(128, 0, 1);
        d->grid = dim3((unsigned)((N + 127) / 128), 1, 1);
    } else {
        d->block = dim3(bx, by, 1);
        d->grid = dim3((d->P.nx + bx - 1) / bx, (d->P.ny + by - 1) / by, d->P.nz);
    }
    d->nblocks = (int64_t)d->grid.x * d->grid.y * d->grid.z;
}

size_t grlb_bytes_for(const grlb_params* p) {
    if (validate(p) != GRLB_OK) return 0;
    grlb_domain tmp;
    tmp.P = *p;
    choose_launch(&tmp);
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    const size_t nbuf = one_buffer(*p) ? 1 : 2;
    return nbuf * state_bytes(N, *p) + (size_t)(tmp.nblocks + grlb::kDiagStageRecords) * NDIAG * 8 +
           NDIAG * 8 + outflow_bytes(*p);
}

grlb_status grlb_create(const grlb_params* p, void* stream, grlb_domain** out) {
    if (!out) return fail(GRLB_EINVAL, "out is NULL");
    *out = nullptr;
    grlb_status st = validate(p);
    if (st != GRLB_OK) return st;
    grlb_domain* d = new (std::nothrow) grlb_domain();
    if (!d) return fail(GRLB_ENOMEM, "host allocation failed");
    d->P = *p;
    d->stream = static_cast<cudaStream_t>(stream);
    cudaGetDevice(&d->device);
    fill_domain_dev(d);
    choose_launch(d);
    const size_t N = (size_t)d->D.plane;
    const size_t pb = state_bytes(N, *p);
    retain_pool();
    cudaStream_t s = d->stream;
    cudaError_t e = cudaSuccess;
    d->D.buf[0] = d->D.buf[1] = nullptr;
    e = grlb::dev_alloc(&d->D.buf[0], pb, s);
    if (e == cudaSuccess) {
        if (one_buffer(*p)) d->D.buf[1] = d->D.buf[0];  // one buffer, updated in place
        else e = grlb::dev_alloc(&d->D.buf[1], pb, s);
    }
    // the last brick's cells past N are never written by a kernel: zero them once so that
    // checkpoints of equal states are equal bytes
    const size_t tail = (moment_storage(*p) ? grlb::NM : grlb::NP) * grlb::kBrick * elem_bytes(p->storage);
    for (int b = 0; b < (one_buffer(*p) ? 1 : 2) && e == cudaSuccess; ++b)
        e = cudaMemsetAsync(static_cast<char*>(d->D.buf[b]) + pb - tail, 0, tail, s);
    if (e == cudaSuccess && one_buffer(*p) && p->bc == GRLB_BC_X_DIRICHLET_EQ)
        e = grlb::dev_alloc(&d->D.outflow, outflow_bytes(*p), s);
    if (e == cudaSuccess)
        e = grlb::dev_alloc(&d->partials, (size_t)(d->nblocks + grlb::kDiagStageRecords) * NDIAG * sizeof(double), s);
    if (e == cudaSuccess) e = grlb::dev_alloc(&d->diag_dev, NDIAG * sizeof(double), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        grlb_destroy(d);
        return fail(e == cudaErrorMemoryAllocation ? GRLB_ENOMEM : GRLB_ECUDA,
                    std::string("grlb_create: ") + cudaGetErrorString(e));
    }
    d->bytes = (one_buffer(*p) ? 1 : 2) * pb + (size_t)(d->nblocks + grlb::kDiagStageRecords) * NDIAG * 8 +
               NDIAG * 8 + outflow_bytes(*p);
    *out = d;
    return GRLB_OK;
}

// Releases in the order of the domain's stream (no device synchronisation).
void grlb_destroy(grlb_domain* d) {
    if (!d) return;
    cudaStream_t s = d->stream;
    if (d->D.src) grlb::chk_release(d->D.src, s);  // the caller's source field, lent since it was set
    grlb::dev_free(d->D.buf[0], s);
    if (d->D.buf[1] != d->D.buf[0]) grlb::dev_free(d->D.buf[1], s);
    grlb::dev_free(d->D.outflow, s);
    grlb::dev_free(d->partials, s);
    grlb::dev_free(d->diag_dev, s);
    for (int i = 0; i < 2; ++i) {
        if (d->stage[i]) grlb::dev_free(d->stage[i], d->copy_stream);  // staged, never consumed
        if (d->staged[i]) cudaEventDestroy(d->staged[i]);
    }
    if (d->copy_stream) cudaStreamDestroy(d->copy_stream);
    if (d->step_graph) cudaGraphExecDestroy(d->step_graph);
    cudaGetLastError();
    delete d;
}

grlb_status grlb_set_stream(grlb_domain* d, void* stream) {
    if (!d) return fail(GRLB_EINVAL, "domain is NULL");
    d->stream = static_cast<cudaStream_t>(stream);
    return GRLB_OK;
}

size_t grlb_device_bytes(const grlb_domain* d) { return d ? d->bytes : 0; }
int64_t grlb_steps_done(const grlb_domain* d) { return d ? d->steps : -1; }


// The initialisation kernel the domain's init mode asks for (equilibrium or Chapman-Enskog).
static cudaError_t launch_domain_init(grlb_domain* d, const double* rho, const double* u, const double* p) {
    if (!d->ce_init)
        return grlb::launch_init(d->D, d->P.storage, d->D.buf[0], rho, u, p, d->s, d->gm1, d->rho_ref, d->p_ref,
                                 d->P.streaming, d->stream);
    const grlb_params& P = d->P;
    grlb::CeInit C;
    C.s = d->s;
    C.gm1 = d->gm1;
    C.mu = P.mu_ref * P.dt / (P.dx * P.dx);
    C.kap = C.mu * (P.gamma / (P.gamma - 1.0)) / P.prandtl;
    C.inv_T_ref = 1.0 / (P.T_ref * d->s * d->s);
    C.T_S = P.T_S;
    const double om[5] = {P.omega_rho, P.omega_mom, P.omega_mom, P.omega_mom, P.omega_E};
    for (int k = 0; k < 5; ++k) {
        C.tau[k] = 1.0 / om[k];
        C.ghostL[k] = P.left_prim[k];
        C.ghostR[k] = P.right_prim[k];
    }
    C.sutherland = P.sutherland;
    C.bc = P.bc;
    return grlb::launch_init_ce(d->D, P.storage, d->D.buf[0], rho, u, p, d->rho_ref, d->p_ref, P.streaming, C,
                                d->stream);
}

grlb_status grlb_init_primitive(grlb_domain* d, const double* rho, const double* u, const double* p) {
    if (!d || !rho || !u || !p) return fail(GRLB_EINVAL, "grlb_init_primitive: NULL argument");
    const size_t N = (size_t)d->D.plane;
    double* stage = nullptr;
    GRLB_CU(grlb::dev_alloc(&stage, 5 * N * sizeof(double), d->stream));
    cudaError_t e = cudaMemcpyAsync(stage, rho, N * sizeof(double), cudaMemcpyHostToDevice, d->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(stage + N, u, 3 * N * sizeof(double), cudaMemcpyHostToDevice, d->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(stage + 4 * N, p, N * sizeof(double), cudaMemcpyHostToDevice, d->stream);
    if (e == cudaSuccess) {
        d->D.cur = 0;
        e = launch_domain_init(d, stage, stage + N, stage + 4 * N);
    }
    cudaError_t e2 = grlb::dev_free(stage, d->stream);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if (e != cudaSuccess) return cuda_fail(e, "grlb_init_primitive");
    d->steps = 0;
    d->diag_step = -1;
    return GRLB_OK;
}

grlb_status grlb_init_primitive_device(grlb_domain* d, const double* rho, const double* u, const double* p) {
    if (!d || !rho || !u || !p) return fail(GRLB_EINVAL, "grlb_init_primitive_device: NULL argument");
    d->D.cur = 0;
    const size_t N = (size_t)d->D.plane;
    cudaError_t e;
    {
        grlb::Lent lr(rho, N * sizeof(double), d->stream), lu(u, 3 * N * sizeof(double), d->stream),
            lp(p, N * sizeof(double), d->stream);
        e = launch_domain_init(d, rho, u, p);
    }
    if (e != cudaSuccess) return cuda_fail(e, "grlb_init_primitive_device");
    d->steps = 0;
    d->diag_step = -1;
    return GRLB_OK;
}

// Two buffers: read buf[cur], write the other.  One buffer (AA): the state after an even
// number of steps sits in swapped slots, so step n+1 is an odd-type step when n is even.
grlb_status grlb_stage_primitive(grlb_domain* d, const double* rho, const double* u, const double* p) {
    if (!d || !rho || !u || !p) return fail(GRLB_EINVAL, "grlb_stage_primitive: NULL argument");
    if (d->stage_count == 2) return fail(GRLB_ESTATE, "both staging slots hold unconsumed states");
    const size_t N = (size_t)d->D.plane;
    if (!d->copy_stream) {  // the copy stream and its two events exist together or not at all
        cudaEvent_t ev[2] = {nullptr, nullptr};
        cudaStream_t cs = nullptr;
        cudaError_t e = cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (cudaEvent_t x : ev)
                if (x) cudaEventDestroy(x);
            return cuda_fail(e, "grlb_stage_primitive (copy stream)");
        }
        d->staged[0] = ev[0];
        d->staged[1] = ev[1];
        d->copy_stream = cs;
    }
    retain_pool();
    const int slot = d->stage_head;
    GRLB_CU(grlb::dev_alloc(&d->stage[slot], 5 * N * sizeof(double), d->copy_stream));
    double* st = d->stage[slot];
    cudaError_t e = cudaMemcpyAsync(st, rho, N * sizeof(double), cudaMemcpyHostToDevice, d->copy_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(st + N, u, 3 * N * sizeof(double), cudaMemcpyHostToDevice, d->copy_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(st + 4 * N, p, N * sizeof(double), cudaMemcpyHostToDevice, d->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(d->staged[slot], d->copy_stream);
    if (e != cudaSuccess) {  // the slot stays empty; its buffer goes back to the pool
        grlb::dev_free(st, d->copy_stream);
        d->stage[slot] = nullptr;
        return cuda_fail(e, "grlb_stage_primitive");
    }
    d->stage_head ^= 1;
    d->stage_count += 1;
    return GRLB_OK;
}

grlb_status grlb_init_from_stage(grlb_domain* d) {
    if (!d) return fail(GRLB_EINVAL, "domain is NULL");
    if (d->stage_count == 0) return fail(GRLB_ESTATE, "no staged state to initialise from");
    const int slot = (d->stage_head + 2 - d->stage_count) & 1;  // oldest filled slot
    const size_t N = (size_t)d->D.plane;
    GRLB_CU(cudaStreamWaitEvent(d->stream, d->staged[slot], 0));
    d->D.cur = 0;
    const double* st = d->stage[slot];
    GRLB_CU(launch_domain_init(d, st, st + N, st + 4 * N));
    GRLB_CU(grlb::dev_free(d->stage[slot], d->stream));  // released once the init has read it
    d->stage[slot] = nullptr;
    d->stage_count -= 1;
    d->steps = 0;
    d->diag_step = -1;
    return GRLB_OK;
}

static grlb_status sweep_once(grlb_domain* d, bool diag) {
    const int c = d->D.cur;
    cudaError_t e;
    if (one_buffer(d->P)) {
        const int pattern = (d->steps % 2 == 0) ? 1 : 2;
        e = grlb::launch_sweep(d->D, d->P.storage, d->P.collision, pattern, d->D.buf[0], d->D.buf[0], diag,
                               d->partials, d->grid, d->block, d->stream);
    } else {  // pull from one buffer into the other: populations (pattern 0) or moments (3)
        e = grlb::launch_sweep(d->D, d->P.storage, d->P.collision, moment_storage(d->P) ? 3 : 0, d->D.buf[c],
                               d->D.buf[c ^ 1], diag, d->partials, d->grid, d->block, d->stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "sweep launch");
    if (!one_buffer(d->P)) d->D.cur = c ^ 1;
    d->steps += 1;
    return GRLB_OK;
}

grlb_status grlb_set_source_device(grlb_domain* d, const float* S) {
    if (!d) return fail(GRLB_EINVAL, "domain is NULL");
    if (S && d->P.streaming) return fail(GRLB_EINVAL, "a source needs two-buffer streaming (streaming = 0)");
    if (d->D.src) GRLB_CU(grlb::chk_release(d->D.src, d->stream));
    if (S) GRLB_CU(grlb::chk_register(S, 5 * (size_t)d->D.plane * sizeof(float), d->stream));
    d->D.src = S;
    if (d->step_graph) {  // the captured sweeps carry the old source pointer
        cudaGraphExecDestroy(d->step_graph);
        d->step_graph = nullptr;
    }
    return GRLB_OK;
}

// A small domain's sweep is shorter than a kernel launch (a 400-cell tube: ~4 us per sweep,
// all of it launch latency), so grlb_step replays its sweeps from a CUDA graph of
// kStepGraphSweeps launches.  The count is even, so a replay returns to the buffer (and step
// parity) it started from; the graph is captured once, on the domain's stream, and used
// whenever the domain is at that buffer and parity.  Not used on the legacy default stream,
// while the caller is capturing the stream, for domains above kStepGraphMaxCells cells (there
// the launch latency is negligible), or for fewer than 2 kStepGraphSweeps steps.
constexpr int kStepGraphSweeps = 8;
constexpr int64_t kStepGraphMaxCells = (int64_t)1 << 22;

static grlb_status capture_step_graph(grlb_domain* d) {
    const int cur = d->D.cur;
    const int64_t steps = d->steps;
    cudaGraph_t g = nullptr;
    GRLB_CU(cudaStreamBeginCapture(d->stream, cudaStreamCaptureModeThreadLocal));
    grlb_status st = GRLB_OK;
    for (int n = 0; n < kStepGraphSweeps && st == GRLB_OK; ++n) st = sweep_once(d, false);
    cudaError_t e = cudaStreamEndCapture(d->stream, &g);
    d->D.cur = cur;  // nothing ran yet: the captured sweeps run at each replay
    d->steps = steps;
    if (st != GRLB_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture (step graph)");
    e = cudaGraphInstantiate(&d->step_graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        d->step_graph = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate (step graph)");
    }
    d->graph_cur = cur;
    d->graph_parity = (int)(steps & 1);
    return GRLB_OK;
}

// The captured sweeps read buf[graph_cur] first; a one-buffer domain's sweeps also depend on
// the step parity (the AA pattern alternates), a two-buffer domain's do not.
static bool at_graph_start(const grlb_domain* d) {
    if (one_buffer(d->P)) return (int)(d->steps & 1) == d->graph_parity;
    return d->D.cur == d->graph_cur;
}

static grlb_status step_domain(grlb_domain* d, int nsteps);

grlb_status grlb_step(grlb_domain* d, int nsteps) {
    if (!d) return fail(GRLB_EINVAL, "domain is NULL");
    if (nsteps < 0) return fail(GRLB_EINVAL, "nsteps must be >= 0");
    return step_domain(d, nsteps);
}

// nsteps sweeps on d->stream: graph replays where they apply, plain sweeps otherwise.
static grlb_status step_domain(grlb_domain* d, int nsteps) {
    int n = 0;
    if (d->stream && nsteps >= 2 * kStepGraphSweeps && d->D.plane <= kStepGraphMaxCells) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(d->stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
            if (!d->step_graph) {
                grlb_status st = capture_step_graph(d);
                if (st != GRLB_OK) return st;
            }
            // one plain sweep aligns the buffer (two buffers) or the step parity (one buffer,
            // whose access pattern alternates) with the graph's start
            if (!at_graph_start(d)) {
                grlb_status st = sweep_once(d, false);
                if (st != GRLB_OK) return st;
                ++n;
            }
            if (at_graph_start(d)) {
                for (; n + kStepGraphSweeps <= nsteps; n += kStepGraphSweeps) {
                    GRLB_CU(cudaGraphLaunch(d->step_graph, d->stream));
                    d->steps += kStepGraphSweeps;
                }
            }
        }
    }
    for (; n < nsteps; ++n) {
        grlb_status st = sweep_once(d, false);
        if (st != GRLB_OK) return st;
    }
    return GRLB_OK;
}

grlb_status grlb_step_diag(grlb_domain* d) {
    if (!d) return fail(GRLB_EINVAL, "domain is NULL");
    grlb_status st = sweep_once(d, true);
    if (st != GRLB_OK) return st;
    GRLB_CU(grlb::launch_diag_finalize(d->partials, d->nblocks, d->diag_dev, d->stream));
    d->diag_step = d->steps;
    return GRLB_OK;
}

grlb_status grlb_diag_read(grlb_domain* d, grlb_diag* out) {
    if (!d || !out) return fail(GRLB_EINVAL, "grlb_diag_read: NULL argument");
    if (d->diag_step < 0) return fail(GRLB_ESTATE, "no diagnostic sweep since init");
    double h[NDIAG];
    GRLB_CU(cudaMemcpyAsync(h, d->diag_dev, NDIAG * sizeof(double), cudaMemcpyDeviceToHost, d->stream));
    GRLB_CU(cudaStreamSynchronize(d->stream));
    const double N = (double)d->D.plane;
    const double Qref[5] = {d->rho_ref, 0.0, 0.0, 0.0, d->E_ref};
    for (int k = 0; k < 5; ++k) out->totals[k] = N * Qref[k] + h[k];
    out->ke = h[5];
    out->eps_s = h[6];
    out->eps_d = h[7];
    out->rho_min = h[8];
    out->p_min = h[9];
    out->n_floor = (int64_t)h[10];
    out->n_nan = (int64_t)h[11];
    out->n_sensor = (int64_t)h[12];
    out->step = d->diag_step;
    out->s = d->s;
    out->ncells = d->D.plane;
    if (out->n_nan > 0)
        return fail(GRLB_ENUMERIC, "grlb_diag_read: " + std::to_string(out->n_nan) +
                                       " cells with a non-finite conserved moment at step " +
                                       std::to_string(out->step));
    return GRLB_OK;
}

grlb_status grlb_check_finite(grlb_domain* d, int32_t* flag) {
    if (!d || !flag) return fail(GRLB_EINVAL, "grlb_check_finite: NULL argument");
    const size_t bytes = state_bytes((size_t)d->D.plane, d->P);
    grlb::Lent lf(flag, sizeof(int32_t), d->stream);
    GRLB_CU(grlb::launch_check_finite(d->D.buf[d->D.cur], (int64_t)bytes, d->P.storage, flag, d->stream));
    return GRLB_OK;
}

grlb_status grlb_read_conserved(grlb_domain* d, double* out) {
    if (!d || !out) return fail(GRLB_EINVAL, "grlb_read_conserved: NULL argument");
    const size_t N = (size_t)d->D.plane;
    double* stage = nullptr;
    GRLB_CU(grlb::dev_alloc(&stage, 5 * N * sizeof(double), d->stream));
    const int gather = moment_storage(d->P) ? 2 : (one_buffer(d->P) && (d->steps & 1)) ? 1 : 0;
    cudaError_t e = grlb::launch_conserved(d->D, d->P.storage, d->D.buf[d->D.cur], stage, d->s, d->rho_ref,
                                           d->E_ref, gather, d->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, stage, 5 * N * sizeof(double), cudaMemcpyDeviceToHost, d->stream);
    cudaError_t e2 = grlb::dev_free(stage, d->stream);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if (e != cudaSuccess) return cuda_fail(e, "grlb_read_conserved");
    return GRLB_OK;
}

grlb_status grlb_read_cells(grlb_domain* d, const int64_t* cells, int64_t n, double* f_out) {
    if (!d) return fail(GRLB_EINVAL, "domain is NULL");
    if (n < 0) return fail(GRLB_EINVAL, "grlb_read_cells: n must be >= 0");
    if (n == 0) return GRLB_OK;
    if (!cells || !f_out) return fail(GRLB_EINVAL, "grlb_read_cells: NULL argument");
    const int64_t N = d->D.plane;
    for (int64_t j = 0; j < n; ++j)
        if (cells[j] < 0 || cells[j] >= N)
            return fail(GRLB_EINVAL, "grlb_read_cells: cell " + std::to_string(cells[j]) + " (entry " +
                                         std::to_string(j) + ") outside [0, " + std::to_string(N) + ")");
    // decoding: f = stored x dec[k] + w_i (Q_ref,k + c_i . J_ref,k / cs^2), J_ref,m_j = p_ref e_j
    grlb::CellDecode dec;
    const double Qref[5] = {d->rho_ref, 0.0, 0.0, 0.0, d->E_ref};
    const int cx[7] = {0, 1, -1, 0, 0, 0, 0}, cy[7] = {0, 0, 0, 1, -1, 0, 0}, cz[7] = {0, 0, 0, 0, 0, 1, -1};
    for (int k = 0; k < 5; ++k) {
        dec.dec[k] = (double)d->D.dec[k];
        for (int i = 0; i < 7; ++i) {
            const double w = i == 0 ? 0.25 : 0.125;
            const int c = k == 1 ? cx[i] : k == 2 ? cy[i] : k == 3 ? cz[i] : 0;
            dec.shift[7 * k + i] = w * (Qref[k] + 4.0 * c * d->p_ref);
        }
    }
    const int layout = moment_storage(d->P) ? 3 : !one_buffer(d->P) ? 0 : (d->steps & 1) ? 2 : 1;
    cudaStream_t s = d->stream;
    char* stage = nullptr;
    const size_t cb = (size_t)n * sizeof(int64_t), ob = (size_t)n * grlb::NP * sizeof(double);
    GRLB_CU(grlb::dev_alloc(&stage, cb + ob, s));
    int64_t* dcells = reinterpret_cast<int64_t*>(stage);
    double* dout = reinterpret_cast<double*>(stage + cb);
    cudaError_t e = cudaMemcpyAsync(dcells, cells, cb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = grlb::launch_read_cells(d->D, d->P.storage, d->D.buf[d->D.cur], dcells, n, layout, dec, dout, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f_out, dout, ob, cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = grlb::dev_free(stage, s);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "grlb_read_cells");
    return GRLB_OK;
}

grlb_status grlb_read_primitive(grlb_domain* d, double* rho, double* u, double* p, double* T) {
    if (!d) return fail(GRLB_EINVAL, "domain is NULL");
    const size_t N = (size_t)d->D.plane;
    std::vector<double> Q;
    try {
        Q.resize(5 * N);
    } catch (...) {
        return fail(GRLB_ENOMEM, "host allocation failed");
    }
    grlb_status st = grlb_read_conserved(d, Q.data());
    if (st != GRLB_OK) return st;
    const double g1 = d->gm1;
    for (size_t c = 0; c < N; ++c) {
        const double r = Q[c];
        const double ux = Q[N + c] / r, uy = Q[2 * N + c] / r, uz = Q[3 * N + c] / r;
        const double pp = g1 * (Q[4 * N + c] - 0.5 * r * (ux * ux + uy * uy + uz * uz));
        if (rho) rho[c] = r;
        if (u) { u[c] = ux; u[N + c] = uy; u[2 * N + c] = uz; }
        if (p) p[c] = pp;
        if (T) T[c] = pp / r;
    }
    return GRLB_OK;
}

namespace {
struct SaveHeader {
    uint64_t magic;
    int64_t steps;
    int64_t N;
    int32_t storage, layout;  // layout: grlb_params.streaming of the saving domain
};
const uint64_t kMagic = 0x3242524c47ULL;  // "GLRB2": cell-brick population layout
}  // namespace

grlb_status grlb_save(grlb_domain* d, void* buf, size_t* bytes) {
    if (!d || !bytes) return fail(GRLB_EINVAL, "grlb_save: NULL argument");
    const size_t pop = state_bytes((size_t)d->D.plane, d->P);
    const size_t ob = outflow_bytes(d->P);
    const size_t need = sizeof(SaveHeader) + pop + ob;
    if (!buf) {
        *bytes = need;
        return GRLB_OK;
    }
    if (*bytes < need) return fail(GRLB_EINVAL, "grlb_save: buffer too small");
    SaveHeader h{kMagic, d->steps, d->D.plane, d->P.storage, d->P.streaming};
    std::memcpy(buf, &h, sizeof h);
    GRLB_CU(cudaMemcpyAsync(static_cast<char*>(buf) + sizeof h, d->D.buf[d->D.cur], pop, cudaMemcpyDeviceToHost,
                            d->stream));
    if (ob)
        GRLB_CU(cudaMemcpyAsync(static_cast<char*>(buf) + sizeof h + pop, d->D.outflow, ob, cudaMemcpyDeviceToHost,
                                d->stream));
    GRLB_CU(cudaStreamSynchronize(d->stream));
    *bytes = need;
    return GRLB_OK;
}

grlb_status grlb_load(grlb_domain* d, const void* buf, size_t bytes) {
    if (!d || !buf) return fail(GRLB_EINVAL, "grlb_load: NULL argument");
    const size_t pop = state_bytes((size_t)d->D.plane, d->P);
    const size_t ob = outflow_bytes(d->P);
    if (bytes < sizeof(SaveHeader) + pop + ob) return fail(GRLB_EINVAL, "grlb_load: buffer too small");
    SaveHeader h;
    std::memcpy(&h, buf, sizeof h);
    if (h.magic != kMagic || h.N != d->D.plane || h.storage != d->P.storage || h.layout != d->P.streaming)
        return fail(GRLB_EINVAL, "grlb_load: checkpoint does not match this domain (cells, storage or layout)");
    d->D.cur = 0;
    GRLB_CU(cudaMemcpyAsync(d->D.buf[0], static_cast<const char*>(buf) + sizeof h, pop, cudaMemcpyHostToDevice,
                            d->stream));
    if (ob)
        GRLB_CU(cudaMemcpyAsync(d->D.outflow, static_cast<const char*>(buf) + sizeof h + pop, ob,
                                cudaMemcpyHostToDevice, d->stream));
    GRLB_CU(cudaStreamSynchronize(d->stream));
    d->steps = h.steps;
    d->diag_step = -1;
    if (d->step_graph) {  // captured at another buffer / parity: re-captured at the loaded state
        cudaGraphExecDestroy(d->step_graph);
        d->step_graph = nullptr;
    }
    return GRLB_OK;
}

}  // extern "C"

// =========================================================================================
// Batching: one launch per step over the concatenated tile table of all active domains.
// =========================================================================================
struct grlb_batch {
    std::vector<grlb_domain*> doms;
    std::vector<int> active;
    std::vector<int> tile_x;  // per-domain override (0 = rule from cfg.block_x)
    std::vector<int> solo;    // 1: large domain, advanced by the single-domain sweep
    grlb_batch_config cfg{};
    cudaStream_t stream = nullptr;
    DomainDev* d_doms = nullptr;
    std::vector<DomainDev> h_doms;  // records copied before each step (pageable: staged by the copy)
    // tiles grouped by (storage, collision): group g = 3 storage + collision occupies
    // [off[g], off[g+1])
    int4* d_tiles = nullptr;
    int ntiles = 0;
    int group_off[10] = {0};
    cudaGraphExec_t graph = nullptr;
    bool dirty = true;
    // constant-table path: the small domains' records in slots [slot0, slot0 + nsmall) of the
    // constant table (small_idx[i]: domain i's offset in that range, -1 for large domains), one
    // launch per group; slot0 < 0 when no slots were free (then the tile-table path above runs)
    int slot0 = -1, nsmall = 0;
    std::vector<int> small_idx;
    std::vector<DomainDev> h_recs;
    std::vector<grlb::BatchLaunch> launch;  // [lane * kGroups + group]
    // the small domains split into nlanes groups of about equal tile counts (up to
    // kTableLanes when there are enough tiles), each stepped on its own stream (lane 0:
    // `stream`, lane l > 0: lane_stream[l - 1], forked from and joined back into `stream`) with
    // its own graph: the domains are independent, so one lane's launches fill the others' wave
    // ramp and tail
    int nlanes = 1;
    cudaGraphExec_t lane_graph[grlb::kTableLanes] = {};
    cudaStream_t lane_stream[grlb::kTableLanes - 1] = {};
    cudaEvent_t lane_done[grlb::kTableLanes - 1] = {};
    cudaEvent_t lane_fork = nullptr;
    std::vector<std::shared_ptr<void>> slot_waits;  // release events of the slots' last holders
    // large domains step on streams of their own, forked from and joined back into `stream`,
    // so that their launches overlap one another's tails and the table launches
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> aux_done;
    cudaEvent_t fork = nullptr;
};

namespace {
constexpr int kGroups = 9;  // 3 storage types x 3 collisions
constexpr size_t kSoloLanes = 32;  // side streams of the single-domain path of a batch
int group_of(const grlb_params& p) { return p.storage * 3 + p.collision; }

// Tile width of domain i: the override, else block_x if the config fixes it, else the width
// in {128, 64, 32} that pads its rows least, or 1 (linear tiles) when rows do not fill tiles.
int tile_width(const grlb_batch* b, size_t i) {
    if (b->tile_x[i] > 0) return b->tile_x[i];
    const grlb_domain* d = b->doms[i];
    const int nx = d->P.nx, ny = d->P.ny;
    if (b->cfg.block_x > 0) {
        int tx = b->cfg.block_x;
        while (tx > 32 && tx / 2 >= nx) tx /= 2;
        return tx;
    }
    int tx = 128;
    long best = -1;
    for (int w = 128; w >= 32; w /= 2) {
        const long padded = (long)((nx + w - 1) / w) * w;
        if (best < 0 || padded < best) {
            best = padded;
            tx = w;
        }
    }
    const int ty = 128 / tx;
    const double padded = (double)((nx + tx - 1) / tx * tx) * ((ny + ty - 1) / ty * ty);
    return padded > 1.05 * (double)nx * ny ? 1 : tx;
}

// Slots of the constant record table (grlb_kernels.cu), shared by every batch of the process.
// A batch takes a contiguous range at creation and gives it back when destroyed; the event
// recorded then on its stream stays with the slots, and the next batch that takes them makes
// its stream wait for it before writing its own records, so no record is overwritten while a
// kernel of the previous holder may still read it.
struct EventRef {
    cudaEvent_t ev = nullptr;
    ~EventRef() {
        if (ev) cudaEventDestroy(ev);
    }
};
std::mutex g_slot_mu;
bool g_slot_used[grlb::kBatchSlots] = {};
// never destroyed: the events must not be released after the CUDA runtime has shut down
std::shared_ptr<void>* const g_slot_release = new std::shared_ptr<void>[grlb::kBatchSlots];

int take_slots(int n, std::vector<std::shared_ptr<void>>* waits) {
    if (n <= 0) return -1;
    std::lock_guard<std::mutex> lk(g_slot_mu);
    for (int s0 = 0; s0 + n <= grlb::kBatchSlots; ++s0) {
        int k = 0;
        while (k < n && !g_slot_used[s0 + k]) ++k;
        if (k < n) {
            s0 += k;
            continue;
        }
        for (int j = s0; j < s0 + n; ++j) {
            g_slot_used[j] = true;
            if (g_slot_release[j]) {
                bool dup = false;
                for (auto& w : *waits) dup = dup || w == g_slot_release[j];
                if (!dup) waits->push_back(g_slot_release[j]);
                g_slot_release[j].reset();
            }
        }
        return s0;
    }
    return -1;
}

void give_slots(int s0, int n, cudaStream_t st) {
    if (s0 < 0) return;
    auto ref = std::make_shared<EventRef>();
    if (cudaEventCreateWithFlags(&ref->ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ref->ev, st) != cudaSuccess) {
        cudaGetLastError();  // no event: wait for the device before the slots are reused
        cudaDeviceSynchronize();
        ref.reset();
    }
    std::lock_guard<std::mutex> lk(g_slot_mu);
    for (int j = s0; j < s0 + n; ++j) {
        g_slot_used[j] = false;
        g_slot_release[j] = ref;
    }
}

// Number of CTAs (tiles) of small domain i.
int64_t tiles_of(const grlb_batch* b, size_t i) {
    const grlb_domain* d = b->doms[i];
    const int tx = tile_width(b, i);
    if (tx == 1) return (d->D.plane + 127) / 128;
    const int ty = 128 / tx;
    return (int64_t)((d->P.nx + tx - 1) / tx) * ((d->P.ny + ty - 1) / ty) * d->P.nz;
}

void drop_lane_graphs(grlb_batch* b) {
    for (cudaGraphExec_t& g : b->lane_graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

// One lane per kLaneTiles tiles of the small domains (four waves of one CTA per SM each), at
// most max_lanes (config; 0 = kDefaultLanes) and at most one per domain.  Measured on the
// 48-tube class (0.79 / 0.85 / 0.83 / 0.79 of the copy bandwidth with 1 / 2 / 4 / 8 lanes): two
// lanes fill each other's ramp and tail, more split the steps into launches too short to
// reach full bandwidth themselves.
constexpr int64_t kLaneTiles = 4 * 148;
constexpr int kDefaultLanes = 2;

grlb_status rebuild_launches(grlb_batch* b) {
    std::vector<size_t> small;
    std::vector<int64_t> tiles(b->doms.size(), 0);
    int64_t total = 0;
    for (size_t i = 0; i < b->doms.size(); ++i) {
        if (!b->active[i] || b->solo[i]) continue;
        small.push_back(i);
        tiles[i] = tiles_of(b, i);
        total += tiles[i];
    }
    const int max_lanes = b->cfg.max_lanes > 0 ? std::min(b->cfg.max_lanes, grlb::kTableLanes) : kDefaultLanes;
    b->nlanes = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)max_lanes, (int64_t)small.size(),
                                                               total / kLaneTiles}));
    // lane of each domain: largest first into the lane with the fewest tiles
    std::vector<int> lane_of(b->doms.size(), 0);
    if (b->nlanes > 1) {
        std::vector<size_t> order = small;
        std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t c) { return tiles[a] > tiles[c]; });
        std::vector<int64_t> load(b->nlanes, 0);
        for (size_t i : order) {
            const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            lane_of[i] = l;
            load[l] += tiles[i];
        }
    }
    b->launch.assign(grlb::kTableLanes * kGroups, grlb::BatchLaunch{});
    for (grlb::BatchLaunch& L : b->launch) L.nd = 0;
    for (size_t i : small) {
        grlb::BatchLaunch& L = b->launch[lane_of[i] * kGroups + group_of(b->doms[i]->P)];
        const int64_t first = L.nd == 0 ? 0 : L.tile0[L.nd];
        const int64_t end = first + tiles[i];
        if (end > 2147483647LL) return fail(GRLB_EINVAL, "batch: more than 2^31 tiles in one launch");
        L.slot[L.nd] = b->slot0 + b->small_idx[i];
        L.tile0[L.nd] = (int32_t)first;
        L.tile0[L.nd + 1] = (int32_t)end;
        L.nd += 1;
    }
    b->ntiles = (int)std::min<int64_t>(total, 2147483647LL);
    drop_lane_graphs(b);
    b->dirty = false;
    return GRLB_OK;
}

grlb_status rebuild_tiles(grlb_batch* b) {
    if (b->slot0 >= 0) return rebuild_launches(b);
    std::vector<int4> groups[kGroups];
    for (size_t i = 0; i < b->doms.size(); ++i) {
        if (!b->active[i] || b->solo[i]) continue;
        const grlb_domain* d = b->doms[i];
        const int tx = tile_width(b, i);
        std::vector<int4>& g = groups[group_of(d->P)];
        if (tx == 1) {
            for (int64_t c = 0; c < d->D.plane; c += 128) g.push_back(make_int4((int)i, (int)c, 0, 0));
            continue;
        }
        const int ty = 128 / tx;
        for (int z = 0; z < d->P.nz; ++z)
            for (int y = 0; y < d->P.ny; y += ty)
                for (int x = 0; x < d->P.nx; x += tx) g.push_back(make_int4((int)i, x, y, z));
    }
    std::vector<int4> all;
    for (int g = 0; g < kGroups; ++g) {
        b->group_off[g] = (int)all.size();
        all.insert(all.end(), groups[g].begin(), groups[g].end());
    }
    b->group_off[kGroups] = (int)all.size();
    grlb::dev_free(b->d_tiles, b->stream);
    b->d_tiles = nullptr;
    b->ntiles = (int)all.size();
    if (b->ntiles > 0) {
        GRLB_CU(grlb::dev_alloc(&b->d_tiles, all.size() * sizeof(int4), b->stream));
        GRLB_CU(cudaMemcpyAsync(b->d_tiles, all.data(), all.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                b->stream));
    }
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->dirty = false;
    return GRLB_OK;
}

cudaError_t order_after_domains(grlb_batch* b) {
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    for (size_t i = 0; e == cudaSuccess && i < b->doms.size(); ++i) {
        if (b->doms[i]->stream == b->stream) continue;
        e = cudaEventRecord(ev, b->doms[i]->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, ev, 0);
    }
    if (ev) cudaEventDestroy(ev);
    return e;
}

cudaError_t enqueue_batch_step(grlb_batch* b, int parity, int lane = 0, cudaStream_t st = nullptr) {
    if (b->slot0 >= 0) {
        for (int g = 0; g < kGroups; ++g) {
            grlb::BatchLaunch& L = b->launch[lane * kGroups + g];
            if (L.nd == 0) continue;
            L.parity = parity;
            cudaError_t e = grlb::launch_batch_sweep_const(g / 3, g % 3, L, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    for (int g = 0; g < kGroups; ++g) {
        const int n = b->group_off[g + 1] - b->group_off[g];
        if (n == 0) continue;
        cudaError_t e = grlb::launch_batch_sweep(g / 3, g % 3, b->d_doms, b->d_tiles + b->group_off[g], n, parity,
                                                 st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
}  // namespace

extern "C" {

grlb_status grlb_batch_create(grlb_domain* const* domains, int n, const grlb_batch_config* cfg, grlb_batch** out) {
    if (!out || !domains || n <= 0) return fail(GRLB_EINVAL, "grlb_batch_create: bad arguments");
    *out = nullptr;
    grlb_batch* b = new (std::nothrow) grlb_batch();
    if (!b) return fail(GRLB_ENOMEM, "host allocation failed");
    if (cfg) b->cfg = *cfg;
    const int bx = b->cfg.block_x;
    if (bx != 0 && bx != 32 && bx != 64 && bx != 128) {
        delete b;
        return fail(GRLB_EINVAL, "block_x must be 32, 64 or 128");
    }
    if (b->cfg.max_lanes < 0 || b->cfg.max_lanes > grlb::kTableLanes) {
        delete b;
        return fail(GRLB_EINVAL, "max_lanes must be in [0, 8]");
    }
    const int sched = b->cfg.schedule;
    if (sched != GRLB_SCHED_CONCURRENT && sched != GRLB_SCHED_TABLE_CONST && sched != GRLB_SCHED_TABLE) {
        delete b;
        return fail(GRLB_EINVAL, "schedule must be GRLB_SCHED_CONCURRENT, _TABLE_CONST or _TABLE");
    }
    for (int i = 0; i < n; ++i) {
        if (!domains[i]) {
            delete b;
            return fail(GRLB_EINVAL, "NULL domain in batch");
        }
        const int64_t thr = b->cfg.solo_min_cells == 0 ? 262144 : b->cfg.solo_min_cells;
        // moment-storage domains always run their own sweep (the table kernels pull populations)
        const int solo = sched == GRLB_SCHED_CONCURRENT || moment_storage(domains[i]->P) ||
                                 (thr > 0 && domains[i]->D.plane >= thr)
                             ? 1
                             : 0;
        // the batched kernel runs two-buffer domains without a source; a domain advanced on its
        // own (solo) may use one-buffer streaming or moment storage
        if (domains[i]->D.src || (domains[i]->P.streaming && !solo)) {
            delete b;
            return fail(GRLB_EINVAL, "batched domains need two-buffer streaming (unless at least solo_min_cells "
                                     "cells) and no source term");
        }
        b->doms.push_back(domains[i]);
        b->active.push_back(1);
        b->tile_x.push_back(0);
        b->solo.push_back(solo);
    }
    b->stream = domains[0]->stream;
    retain_pool();
    b->small_idx.assign(n, -1);
    for (int i = 0; i < n; ++i)
        if (!b->solo[i]) b->small_idx[i] = b->nsmall++;
    if (sched == GRLB_SCHED_TABLE_CONST) b->slot0 = take_slots(b->nsmall, &b->slot_waits);
    b->h_recs.resize(b->nsmall);
    b->h_doms.resize(n);
    cudaError_t e = cudaSuccess;
    if (b->slot0 < 0) e = grlb::dev_alloc(&b->d_doms, n * sizeof(DomainDev), b->stream);
    // the batch stream must not run ahead of work already queued on the domains' streams
    if (e == cudaSuccess) e = order_after_domains(b);
    if (e != cudaSuccess) {
        grlb_batch_destroy(b);
        return cuda_fail(e, "grlb_batch_create");
    }
    grlb_status st = rebuild_tiles(b);
    if (st != GRLB_OK) {
        grlb_batch_destroy(b);
        return st;
    }
    *out = b;
    return GRLB_OK;
}

// Releases in the order of the batch stream; each domain's stream is made to wait for the
// batch's queued work, so a later grlb_destroy of a domain cannot overtake it.
void grlb_batch_destroy(grlb_batch* b) {
    if (!b) return;
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(ev, b->stream);
        for (grlb_domain* d : b->doms)
            if (d->stream != b->stream) cudaStreamWaitEvent(d->stream, ev, 0);
        cudaEventDestroy(ev);
    }
    if (b->graph) cudaGraphExecDestroy(b->graph);
    grlb::dev_free(b->d_doms, b->stream);
    grlb::dev_free(b->d_tiles, b->stream);
    // slots taken but never written (no step ran): their previous holders' release events have
    // not been waited for yet, so this batch's release must follow them too
    for (const auto& w : b->slot_waits) {
        const EventRef* r = static_cast<const EventRef*>(w.get());
        if (r && r->ev) cudaStreamWaitEvent(b->stream, r->ev, 0);
    }
    give_slots(b->slot0, b->nsmall, b->stream);
    drop_lane_graphs(b);
    for (int l = 0; l < grlb::kTableLanes - 1; ++l) {  // pending work completes first
        if (b->lane_stream[l]) cudaStreamDestroy(b->lane_stream[l]);
        if (b->lane_done[l]) cudaEventDestroy(b->lane_done[l]);
    }
    if (b->lane_fork) cudaEventDestroy(b->lane_fork);
    // pending work on the side streams completes before their resources are released
    for (cudaStream_t s : b->aux) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->aux_done) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    cudaGetLastError();
    delete b;
}

grlb_status grlb_batch_set_stream(grlb_batch* b, void* stream) {
    if (!b) return fail(GRLB_EINVAL, "batch is NULL");
    cudaEvent_t ev = nullptr;
    GRLB_CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaEventRecord(ev, b->stream);  // the batch's own allocations and copies come first
    b->stream = static_cast<cudaStream_t>(stream);
    cudaStreamWaitEvent(b->stream, ev, 0);
    cudaEventDestroy(ev);
    GRLB_CU(order_after_domains(b));
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    drop_lane_graphs(b);  // lane 0's graph was captured on the old stream
    return GRLB_OK;
}

grlb_status grlb_batch_set_active(grlb_batch* b, const int* active) {
    if (!b) return fail(GRLB_EINVAL, "batch is NULL");
    for (size_t i = 0; i < b->doms.size(); ++i) b->active[i] = active ? (active[i] != 0) : 1;
    return rebuild_tiles(b);
}

grlb_status grlb_batch_set_tile_x(grlb_batch* b, const int* tile_x) {
    if (!b) return fail(GRLB_EINVAL, "batch is NULL");
    for (size_t i = 0; i < b->doms.size(); ++i) {
        const int t = tile_x ? tile_x[i] : 0;
        if (t != 0 && t != 1 && t != 32 && t != 64 && t != 128)
            return fail(GRLB_EINVAL, "tile_x must be 0, 1, 32, 64 or 128");
    }
    for (size_t i = 0; i < b->doms.size(); ++i) b->tile_x[i] = tile_x ? tile_x[i] : 0;
    return rebuild_tiles(b);
}

static grlb_status batch_table_steps(grlb_batch* b, int nsteps);

grlb_status grlb_batch_step(grlb_batch* b, int nsteps) {
    if (!b) return fail(GRLB_EINVAL, "batch is NULL");
    if (nsteps < 0) return fail(GRLB_EINVAL, "nsteps must be >= 0");
    if (nsteps == 0) return GRLB_OK;
    // domains advanced by the single-domain sweep (every domain under GRLB_SCHED_CONCURRENT, the
    // large ones otherwise): grlb_step's stepping (graph replays where they apply), bitwise its
    // result, on up to kSoloLanes side streams forked from the batch stream -- the largest
    // domains first, dealt round-robin, so that the lanes carry similar work and their kernels
    // run concurrently, filling one another's waves
    std::vector<size_t> solo;
    for (size_t i = 0; i < b->doms.size(); ++i)
        if (b->active[i] && b->solo[i]) solo.push_back(i);
    std::stable_sort(solo.begin(), solo.end(),
                     [&](size_t a, size_t c) { return b->doms[a]->D.plane > b->doms[c]->D.plane; });
    const int nlanes = (int)std::min<size_t>(solo.size(), kSoloLanes);
    if (nlanes > 0) {
        if (!b->fork) GRLB_CU(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
        while ((int)b->aux.size() < nlanes) {  // aux[k] and aux_done[k] are created in pairs
            cudaStream_t s;
            cudaEvent_t ev;
            GRLB_CU(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
            const cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e != cudaSuccess) {
                cudaStreamDestroy(s);
                return cuda_fail(e, "cudaEventCreateWithFlags (batch aux stream)");
            }
            b->aux.push_back(s);
            b->aux_done.push_back(ev);
        }
        GRLB_CU(cudaEventRecord(b->fork, b->stream));
        for (int k = 0; k < nlanes; ++k) GRLB_CU(cudaStreamWaitEvent(b->aux[k], b->fork, 0));
        for (size_t j = 0; j < solo.size(); ++j) {
            grlb_domain* d = b->doms[solo[j]];
            cudaStream_t keep = d->stream;
            d->stream = b->aux[j % nlanes];
            const grlb_status st = step_domain(d, nsteps);
            d->stream = keep;
            if (st != GRLB_OK) return st;
        }
        for (int k = 0; k < nlanes; ++k) GRLB_CU(cudaEventRecord(b->aux_done[k], b->aux[k]));
    }
    grlb_status tst = GRLB_OK;
    if (b->ntiles > 0) tst = batch_table_steps(b, nsteps);
    for (int k = 0; k < nlanes; ++k) GRLB_CU(cudaStreamWaitEvent(b->stream, b->aux_done[k], 0));
    return tst;
}

// The small domains' part of grlb_batch_step: nsteps launches of the batched sweep over the
// tile table (pairs of steps replayed from a CUDA graph).
static grlb_status batch_table_steps(grlb_batch* b, int nsteps) {
    if (b->slot0 >= 0) {
        for (const auto& w : b->slot_waits) {  // the slots' previous holder is done with them
            const EventRef* r = static_cast<const EventRef*>(w.get());
            if (r && r->ev) GRLB_CU(cudaStreamWaitEvent(b->stream, r->ev, 0));
        }
        b->slot_waits.clear();
        for (size_t i = 0; i < b->doms.size(); ++i) {
            if (b->small_idx[i] < 0) continue;
            DomainDev& r = b->h_recs[b->small_idx[i]];
            r = b->doms[i]->D;
            r.tile_x = tile_width(b, i);
        }
        // from pageable memory: the host copy is staged before the call returns
        GRLB_CU(grlb::upload_batch_records(b->h_recs.data(), b->slot0, b->nsmall, b->stream));
    } else {
        for (size_t i = 0; i < b->doms.size(); ++i) {
            b->h_doms[i] = b->doms[i]->D;
            b->h_doms[i].tile_x = tile_width(b, i);
        }
        // from pageable memory: the host copy is staged before the call returns, no stream wait
        GRLB_CU(cudaMemcpyAsync(b->d_doms, b->h_doms.data(), b->doms.size() * sizeof(DomainDev),
                                cudaMemcpyHostToDevice, b->stream));
    }
    const int nl = b->slot0 >= 0 ? b->nlanes : 1;
    if (nl > 1) {
        if (!b->lane_fork) GRLB_CU(cudaEventCreateWithFlags(&b->lane_fork, cudaEventDisableTiming));
        for (int l = 0; l + 1 < nl; ++l) {
            if (b->lane_stream[l]) continue;  // a lane stream and its event exist together or not at all
            cudaStream_t ls = nullptr;
            cudaEvent_t ev = nullptr;
            cudaError_t e = cudaStreamCreateWithFlags(&ls, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e != cudaSuccess) {
                if (ls) cudaStreamDestroy(ls);
                return cuda_fail(e, "batch lane stream");
            }
            b->lane_stream[l] = ls;
            b->lane_done[l] = ev;
        }
        GRLB_CU(cudaEventRecord(b->lane_fork, b->stream));  // after the record upload
        for (int l = 0; l + 1 < nl; ++l) GRLB_CU(cudaStreamWaitEvent(b->lane_stream[l], b->lane_fork, 0));
    }
    for (int lane = 0; lane < nl; ++lane) {
        cudaStream_t st = lane == 0 ? b->stream : b->lane_stream[lane - 1];
        cudaGraphExec_t& G = b->slot0 >= 0 ? b->lane_graph[lane] : b->graph;
        int done = 0;
        if (b->cfg.use_graph && st != nullptr && nsteps >= 2) {
            if (!G) {
                cudaGraph_t g;
                GRLB_CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                cudaError_t e = enqueue_batch_step(b, 0, lane, st);
                if (e == cudaSuccess) e = enqueue_batch_step(b, 1, lane, st);
                cudaError_t e2 = cudaStreamEndCapture(st, &g);
                if (e != cudaSuccess) return cuda_fail(e, "batch graph capture");
                if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
                e = cudaGraphInstantiate(&G, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) {
                    G = nullptr;
                    return cuda_fail(e, "cudaGraphInstantiate");
                }
            }
            for (; done + 2 <= nsteps; done += 2) GRLB_CU(cudaGraphLaunch(G, st));
        }
        for (; done < nsteps; ++done) GRLB_CU(enqueue_batch_step(b, done & 1, lane, st));
    }
    for (int l = 0; l + 1 < nl; ++l) {
        GRLB_CU(cudaEventRecord(b->lane_done[l], b->lane_stream[l]));
        GRLB_CU(cudaStreamWaitEvent(b->stream, b->lane_done[l], 0));
    }
    for (size_t i = 0; i < b->doms.size(); ++i) {
        if (!b->active[i] || b->solo[i]) continue;
        grlb_domain* d = b->doms[i];
        d->D.cur ^= (nsteps & 1);
        d->steps += nsteps;
    }
    return GRLB_OK;
}

}  // extern "C"

// =========================================================================================
// Diagnostic sweep for callers that cannot allocate device memory: the block partials live
// in a file-scope static device array instead of scratch from cudaMalloc.
// =========================================================================================
namespace {
// Block partials followed by the records of the first finalize stage.
static __device__ __align__(256) double
    g_noalloc_partials[((size_t)GRLB_NOALLOC_MAX_BLOCKS + grlb::kDiagStageRecords) * NDIAG];

// Device address of g_noalloc_partials on the current device (host code cannot use the symbol
// itself as a device pointer).  Looked up on every call: the lookup allocates nothing, and an
// address kept from an earlier call would be stale after a device reset, which unloads the
// library's device code (the next lookup loads it again).
grlb_status noalloc_scratch(double** out) {
    double* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_partials);
    if (e != cudaSuccess || !ptr) return cuda_fail(e, "cudaGetSymbolAddress(static diagnostic scratch)");
    *out = ptr;
    return GRLB_OK;
}
}  // namespace

extern "C" grlb_status grlb_step_diag_noalloc(const grlb_params* p, const void* f_in, void* f_out,
                                              double* diag_out, void* stream) {
    grlb_status st = validate(p);
    if (st != GRLB_OK) return st;
    if (!f_in || !f_out || !diag_out) return fail(GRLB_EINVAL, "grlb_step_diag_noalloc: NULL pointer");
    if (f_in == f_out) return fail(GRLB_EINVAL, "grlb_step_diag_noalloc: f_in and f_out must differ");
    if (p->streaming) return fail(GRLB_EINVAL, "grlb_step_diag_noalloc: two-buffer streaming only");
    grlb_domain tmp;  // host-side description only; owns no memory
    tmp.P = *p;
    fill_domain_dev(&tmp);
    choose_launch(&tmp);
    tmp.D.buf[0] = tmp.D.buf[1] = nullptr;
    if (tmp.nblocks > GRLB_NOALLOC_MAX_BLOCKS)
        return fail(GRLB_EINVAL, "grlb_step_diag_noalloc: domain needs " + std::to_string(tmp.nblocks) +
                                     " CTAs, more than the static scratch holds (" +
                                     std::to_string(GRLB_NOALLOC_MAX_BLOCKS) + ")");
    double* scratch = nullptr;
    st = noalloc_scratch(&scratch);
    if (st != GRLB_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t pb = pop_bytes((size_t)tmp.D.plane, p->storage);
    grlb::Lent li(f_in, pb, s), lo(f_out, pb, s), ld(diag_out, NDIAG * sizeof(double), s),
        lsc(scratch, sizeof(g_noalloc_partials), s);
    GRLB_CU(grlb::launch_sweep(tmp.D, p->storage, p->collision, 0, f_in, f_out, true, scratch, tmp.grid, tmp.block,
                               s));
    GRLB_CU(grlb::launch_diag_finalize(scratch, tmp.nblocks, diag_out, s));
    return GRLB_OK;
}

// ---- spectral post-processing -------------------------------------------------------------
namespace {

int ilog2_exact(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return (1 << l) == n ? l : -1;
}

// Extent n shared by every axis longer than 1, and how many such axes; 0 if they differ.
int spectral_extent(const grlb_params& p, int* dims) {
    int n = 0;
    *dims = 0;
    for (int e : {p.nx, p.ny, p.nz}) {
        if (e <= 1) continue;
        if (n && e != n) return 0;
        n = e;
        ++*dims;
    }
    return n;
}

int64_t shell_of_host(int64_t M) {
    int64_t b = (int64_t)std::floor(std::sqrt((double)M) + 0.5);
    while (b * b + b < M) ++b;
    while (b > 0 && b * b - b + 1 > M) --b;
    return b;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" int32_t grlb_spectrum_shells(const grlb_params* p) {
    if (!p) return -1;
    int dims = 0;
    const int n = spectral_extent(*p, &dims);
    if (dims == 0) return 1;
    if (n == 0) return -1;
    const int64_t h = n / 2;
    return (int32_t)(shell_of_host(dims * h * h) + 1);
}

extern "C" grlb_status grlb_spectral_diag(grlb_domain* d, int32_t nbins, double* spectrum, double* sums) {
    if (!d || !sums || nbins < 0 || (nbins > 0 && !spectrum))
        return fail(GRLB_EINVAL, "grlb_spectral_diag: NULL or negative argument");
    const grlb_params& P = d->P;
    if (P.bc != GRLB_BC_PERIODIC) return fail(GRLB_EINVAL, "grlb_spectral_diag: periodic domains only");
    const int n = P.nx;
    const int lg = n > 1 ? ilog2_exact(n) : -1;
    if (P.ny != n || (P.nz != 1 && P.nz != n) || lg < (P.nz > 1 ? 4 : 5) || lg > 10)
        return fail(GRLB_EINVAL, "grlb_spectral_diag: needs an n^3 cube (n in [16, 1024]) or an n x n x 1 square "
                                 "(n in [32, 1024]), n a power of two");
    const int shells = grlb_spectrum_shells(&P);
    const int nb = std::min<int>(nbins, shells);
    const int64_t N = d->D.plane;
    cudaStream_t st = d->stream;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grlb::SpectralPlan plan = grlb::spectral_plan(lg, lg, P.nz > 1 ? lg : 0, nb, sms);
    const int np = std::max(plan.grid1, 2 * plan.grid5);

    // scratch: 4 complex planes, mu plane, twiddles, per-CTA partials, shell bins
    const size_t oU = 0, oMu = align256(oU + 4 * (size_t)N * sizeof(float2));
    const size_t oTw = align256(oMu + (size_t)N * sizeof(float));
    const size_t oPart = align256(oTw + (size_t)n * sizeof(float2));
    const size_t oBins = align256(oPart + (size_t)np * sizeof(double));
    const size_t bytes = align256(oBins + (size_t)std::max(nb, 1) * sizeof(unsigned long long));
    char* base = nullptr;
    GRLB_CU(cudaMallocAsync(reinterpret_cast<void**>(&base), bytes, st));
    float2* U = reinterpret_cast<float2*>(base + oU);
    float* mu = reinterpret_cast<float*>(base + oMu);
    float2* tw = reinterpret_cast<float2*>(base + oTw);
    double* part = reinterpret_cast<double*>(base + oPart);
    unsigned long long* bins = reinterpret_cast<unsigned long long*>(base + oBins);
    // the checked build registers each part of the scratch on its own, without the padding
    const void* parts[5] = {U, mu, tw, part, bins};
    const size_t part_bytes[5] = {4 * (size_t)N * sizeof(float2), (size_t)N * sizeof(float),
                                  (size_t)n * sizeof(float2), (size_t)np * sizeof(double),
                                  (size_t)std::max(nb, 1) * sizeof(unsigned long long)};
    for (int i = 0; i < 5; ++i) grlb::chk_register(parts[i], part_bytes[i], st);
    auto release_scratch = [&]() {
        for (int i = 0; i < 5; ++i) grlb::chk_release(parts[i], st);
        return cudaFreeAsync(base, st);
    };

    std::vector<float2> htw(n);
    for (int j = 0; j < n; ++j) {
        const double a = -2.0 * M_PI * (double)j / (double)n;
        htw[j] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    std::vector<double> hpart(np);
    std::vector<unsigned long long> hbins(std::max(nb, 1));
    const int gather = moment_storage(P) ? 2 : (one_buffer(P) && (d->steps & 1)) ? 1 : 0;
    double ke_sum = 0.0;
    cudaError_t e = cudaMemcpyAsync(tw, htw.data(), htw.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bins, 0, std::max(nb, 1) * sizeof(unsigned long long), st);
    if (e == cudaSuccess)
        e = grlb::launch_spectral_k1(d->D, P.storage, d->D.buf[d->D.cur], gather, plan, tw, U, mu, part, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hpart.data(), part, plan.grid1 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
        for (int i = 0; i < plan.grid1; ++i) ke_sum += hpart[i];
        // fixed point for the shell sums: total 1/2|u^|^2/N^2 = ke_sum / N stays below 2^60
        int ex = 0;
        const double mean = ke_sum / (double)N;
        if (mean > 0) std::frexp(mean, &ex);
        // 2^fx / N^2 must stay a normal FP32 number: fx within [-126 + lg N^2, 127 + lg N^2]
        const int lgN2 = 2 * (plan.lgx + plan.lgy + plan.lgz);
        const int fx = std::max(-126 + lgN2, std::min(127 + lgN2, 60 - ex));
        const double fx_scale = std::ldexp(1.0, fx);
        plan.scale = std::ldexp(1.0f, fx - lgN2);
        e = grlb::launch_spectral_k2_to_k5(plan, tw, U, mu, bins, part, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hpart.data(), part, 2 * plan.grid5 * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && nb > 0)
            e = cudaMemcpyAsync(hbins.data(), bins, nb * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
        cudaError_t e2 = release_scratch();
        if (e == cudaSuccess) e = e2;
        base = nullptr;
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) {
            double es = 0.0, ed = 0.0;
            for (int i = 0; i < plan.grid5; ++i) {
                es += hpart[2 * i];
                ed += hpart[2 * i + 1];
            }
            const double inv_N2 = 1.0 / ((double)N * (double)N);
            sums[0] = es * inv_N2;
            sums[1] = ed * inv_N2;
            sums[2] = ke_sum;
            for (int b = 0; b < nbins; ++b) spectrum[b] = b < nb ? (double)hbins[b] / fx_scale : 0.0;
        }
    }
    if (base) release_scratch();
    if (e != cudaSuccess) return cuda_fail(e, "grlb_spectral_diag");
    return GRLB_OK;
}

extern "C" grlb_status grlb_halo_exchange_z(grlb_domain* lower, grlb_domain* upper) {
    if (!lower || !upper) return fail(GRLB_EINVAL, "grlb_halo_exchange_z: NULL domain");
    const grlb_params& a = lower->P;
    const grlb_params& b = upper->P;
    if (a.nx != b.nx || a.ny != b.ny || a.storage != b.storage)
        return fail(GRLB_EINVAL, "grlb_halo_exchange_z: slabs differ in nx, ny or storage");
    if (one_buffer(a) || a.streaming != b.streaming)
        return fail(GRLB_EINVAL, "grlb_halo_exchange_z: two-buffer slabs of one kind (populations or moments)");
    if (a.bc != GRLB_BC_PERIODIC || b.bc != GRLB_BC_PERIODIC)
        return fail(GRLB_EINVAL, "grlb_halo_exchange_z: slabs are periodic domains");
    if (a.nz < 3 || b.nz < 3) return fail(GRLB_EINVAL, "grlb_halo_exchange_z: a slab needs nz >= 3 (2 ghost planes)");
    if (lower->stream != upper->stream)
        return fail(GRLB_EINVAL, "grlb_halo_exchange_z: slabs must share one stream");
    if (moment_storage(a))
        GRLB_CU(grlb::launch_halo_z_mom(lower->D.buf[lower->D.cur], upper->D.buf[upper->D.cur], a.nz,
                                        (int64_t)a.nx * a.ny, lower->stream));
    else
        GRLB_CU(grlb::launch_halo_z(lower->D.buf[lower->D.cur], upper->D.buf[upper->D.cur], a.nz,
                                    (int64_t)a.nx * a.ny, elem_bytes(a.storage), lower->stream));
    return GRLB_OK;
}

// values per cell of one exchanged slab face: the population along z of each field, or Q_k / 8 and
// J*_k,z of each field (moment storage)
static int halo_slices(const grlb_params& p) { return moment_storage(p) ? 10 : 5; }

static grlb_status check_slab(const grlb_domain* d, const char* who) {
    const grlb_params& a = d->P;
    if (one_buffer(a)) return fail(GRLB_EINVAL, std::string(who) + ": two-buffer streaming only");
    if (a.bc != GRLB_BC_PERIODIC) return fail(GRLB_EINVAL, std::string(who) + ": slabs are periodic domains");
    if (a.nz < 3) return fail(GRLB_EINVAL, std::string(who) + ": a slab needs nz >= 3 (2 ghost planes)");
    return GRLB_OK;
}

extern "C" grlb_status grlb_halo_pack_z(grlb_domain* d, void* to_upper, void* to_lower) {
    if (!d || !to_upper || !to_lower) return fail(GRLB_EINVAL, "grlb_halo_pack_z: NULL argument");
    grlb_status st = check_slab(d, "grlb_halo_pack_z");
    if (st != GRLB_OK) return st;
    const grlb_params& a = d->P;
    const size_t slice = halo_slices(a) * (size_t)a.nx * a.ny * elem_bytes(a.storage);
    grlb::Lent lu(to_upper, slice, d->stream), ll(to_lower, slice, d->stream);
    if (moment_storage(a))
        GRLB_CU(grlb::launch_halo_pack_z_mom(d->D.buf[d->D.cur], to_upper, to_lower, a.nz, (int64_t)a.nx * a.ny,
                                             d->stream));
    else
        GRLB_CU(grlb::launch_halo_pack_z(d->D.buf[d->D.cur], to_upper, to_lower, a.nz, (int64_t)a.nx * a.ny,
                                         elem_bytes(a.storage), d->stream));
    return GRLB_OK;
}

extern "C" grlb_status grlb_halo_unpack_z(grlb_domain* d, const void* from_lower, const void* from_upper) {
    if (!d || !from_lower || !from_upper) return fail(GRLB_EINVAL, "grlb_halo_unpack_z: NULL argument");
    grlb_status st = check_slab(d, "grlb_halo_unpack_z");
    if (st != GRLB_OK) return st;
    const grlb_params& a = d->P;
    const size_t slice = halo_slices(a) * (size_t)a.nx * a.ny * elem_bytes(a.storage);
    grlb::Lent ll(from_lower, slice, d->stream), lu(from_upper, slice, d->stream);
    if (moment_storage(a))
        GRLB_CU(grlb::launch_halo_unpack_z_mom(d->D.buf[d->D.cur], from_lower, from_upper, a.nz,
                                               (int64_t)a.nx * a.ny, d->stream));
    else
        GRLB_CU(grlb::launch_halo_unpack_z(d->D.buf[d->D.cur], from_lower, from_upper, a.nz, (int64_t)a.nx * a.ny,
                                           elem_bytes(a.storage), d->stream));
    return GRLB_OK;
}

extern "C" grlb_status grlb_set_init_mode(grlb_domain* d, int32_t ce_init) {
    if (!d) return fail(GRLB_EINVAL, "domain is NULL");
    if (ce_init != 0 && ce_init != 1) return fail(GRLB_EINVAL, "grlb_set_init_mode: ce_init must be 0 or 1");
    d->ce_init = ce_init;
    return GRLB_OK;
}

extern "C" grlb_status grlb_ffma_probe(int32_t ctas, int32_t iters, float* sink, void* stream,
                                       double* warp_instructions) {
    if (ctas < 1 || iters < 1 || !sink || !warp_instructions)
        return fail(GRLB_EINVAL, "grlb_ffma_probe: ctas and iters must be >= 1, pointers non-NULL");
    grlb::Lent ls(sink, (size_t)ctas * 256 * sizeof(float), static_cast<cudaStream_t>(stream));
    GRLB_CU(grlb::launch_ffma_probe(sink, ctas, iters, static_cast<cudaStream_t>(stream)));
    *warp_instructions = (double)ctas * 8.0 * (double)iters * 128.0;
    return GRLB_OK;
}

// ---- bounds-checked build ---------------------------------------------------------------------
extern "C" int32_t grlb_checked_build(void) { return grlb::kChecked ? 1 : 0; }

extern "C" grlb_status grlb_check_read(grlb_check_counts* out, int32_t reset) {
    if (!out) return fail(GRLB_EINVAL, "grlb_check_read: out is NULL");
#ifdef GRLB_CHECKED
    grlb::ChkCounts c{};
    GRLB_CU(grlb::chk_read(&c, reset != 0));
    out->violations = (int64_t)c.violations;
    out->first_addr = c.first;
    out->live_regions = c.live;
    out->unmatched = (int64_t)c.unmatched;
    out->overflow = (int64_t)c.overflow;
    return GRLB_OK;
#else
    (void)reset;
    return fail(GRLB_ESTATE, "grlb_check_read: not a bounds-checked build (GRLB_CHECKED)");
#endif
}

extern "C" grlb_status grlb_check_probe(const void* base, uint64_t bytes, int64_t offset, uint64_t access_bytes,
                                        void* stream) {
#ifdef GRLB_CHECKED
    if (bytes == 0 || access_bytes == 0 || access_bytes > 0xffffffffull)
        return fail(GRLB_EINVAL, "grlb_check_probe: bytes and access_bytes must be positive (access < 4 GB)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const char* at = static_cast<const char*>(base) + offset;
    GRLB_CU(grlb::chk_register(base, bytes, s));
    GRLB_CU(grlb::chk_probe(at, access_bytes, s));
    GRLB_CU(grlb::chk_release(base, s));
    return GRLB_OK;
#else
    (void)base; (void)bytes; (void)offset; (void)access_bytes; (void)stream;
    return fail(GRLB_ESTATE, "grlb_check_probe: not a bounds-checked build (GRLB_CHECKED)");
#endif
}

// ---- device memory cached by the pool ---------------------------------------------------------
extern "C" grlb_status grlb_trim_pool(void) {
    int dev = 0;
    GRLB_CU(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    GRLB_CU(cudaDeviceGetDefaultMemPool(&pool, dev));
    GRLB_CU(cudaDeviceSynchronize());  // releases still in flight on any stream complete first
    GRLB_CU(cudaMemPoolTrimTo(pool, 0));
    return GRLB_OK;
}
