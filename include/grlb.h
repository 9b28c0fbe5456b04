/*
 * grlb.h -- C ABI of the B300 (sm_103a) gradient-reconstruction lattice Boltzmann sweep for
 * the compressible Navier-Stokes-Fourier equations (arxiv 2609.16361).
 *
 * One domain = five conserved-field D3Q7 lattices (rho, m_x, m_y, m_z, E), 35 populations per
 * cell (Sec. 2.2), advanced by the fused stream-and-collide sweep of Algorithm 1.
 *
 * Conventions shared by every entry point:
 *  - Ownership: the library allocates and owns all device memory of a domain or batch; the
 *    caller owns every host array it passes and keeps it alive for the duration of the call.
 *  - Fields on the host are FP64, physical units, structure of arrays, x fastest:
 *    a[x + nx*(y + ny*z)], N = nx*ny*nz entries per field plane.
 *  - Streams: work is enqueued on the stream given at creation (a cudaStream_t passed as
 *    void*, e.g. a torch stream handle; NULL = legacy default stream).  grlb_step,
 *    grlb_step_diag and grlb_batch_step only enqueue.  Calls that return host data
 *    (grlb_read_*, grlb_diag_read, grlb_save) synchronize that stream first.
 *  - Errors: every call returns a grlb_status; on failure grlb_last_error() returns a
 *    thread-local message.  No call aborts the process.  A numeric blow-up is reported by
 *    the diagnostics (n_nan, n_floor; grlb_diag_read then returns GRLB_ENUMERIC) or by
 *    grlb_check_finite, not by the plain sweep.
 *  - Lattice units: dx = dt = 1 inside the kernels.  With s = dt/dx: rho unchanged,
 *    u_L = s u, (p, E, T)_L = s^2 (p, E, T), (mu, kappa)_L = (mu, kappa) dt/dx^2.
 */
#ifndef GRLB_H
#define GRLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GRLB_OK = 0,
    GRLB_EINVAL = -1,   /* bad argument (null pointer, size, enum, parameter range)      */
    GRLB_ENOMEM = -2,   /* device or host allocation failed                              */
    GRLB_ECUDA = -3,    /* a CUDA runtime call failed; message carries cudaGetErrorString */
    GRLB_ENUMERIC = -4, /* non-finite state: grlb_diag_read returns it (after filling its
                           output) when the diagnostic sweep counted n_nan > 0 cells      */
    GRLB_ETIMEOUT = -5, /* reserved: no kernel of the library waits on another           */
    GRLB_ESTATE = -6    /* call not valid in the object's current state                  */
} grlb_status;

typedef enum { GRLB_BC_PERIODIC = 0, GRLB_BC_X_DIRICHLET_EQ = 1 } grlb_bc;
/* Collision operators.  BGK: f* = f + omega_k (f^eq - f) (Sec. 2.2).  RLB_SENSOR: the
 * regularized collision of Sec. 2.5 / Algorithm 1 in every cell: f* = f^eq + (1 - omega_h) r,
 * r the first-moment part of f - f^eq, omega_h = omega_k - chi max(omega_k - omega_min, 0).
 * RLB_GATED: the reading of Sec. 2.2 in which the compression sensor activates the regularized
 * collision in place of BGK: the RLB_SENSOR update where chi > 0, BGK at the nominal omega_k
 * where chi = 0 (the sensor, reconstruction and flux are those of RLB_SENSOR). */
typedef enum { GRLB_COLL_BGK = 0, GRLB_COLL_RLB_SENSOR = 1, GRLB_COLL_RLB_GATED = 2 } grlb_collision;
typedef enum { GRLB_STORE_F32 = 0, GRLB_STORE_F16 = 1, GRLB_STORE_BF16 = 2 } grlb_storage;

/* Physical description of one domain (Sec. 2.1 system, Listing 1 closures, Listing 2
 * sensor, Tab. run_params numerical parameters). */
typedef struct {
    int32_t nx, ny, nz;         /* cells; N = nx*ny*nz must be < 2^31                       */
    int32_t bc;                 /* grlb_bc.  X_DIRICHLET_EQ: ghost cells at x=-1 and x=nx
                                   hold the equilibrium of left_prim / right_prim; y, z
                                   periodic.  PERIODIC: every axis periodic.                 */
    int32_t collision;          /* grlb_collision (Sec. 2.2 BGK, Sec. 2.5 regularized, or
                                   the sensor-gated pair of the two)                        */
    int32_t storage;            /* grlb_storage: population storage type; arithmetic is FP32
                                   in every mode (FP64 for the diagnostic sums), and with FP16 /
                                   BF16 storage the collision's four divisions are the
                                   approximate reciprocal-and-multiply (within 2 ulp)         */
    double dx, dt;              /* physical cell size and time step (> 0)                  */
    double gamma;               /* ratio of specific heats (> 1)                            */
    double mu_ref;              /* dynamic viscosity at T_ref (>= 0)                        */
    double prandtl;             /* kappa = mu c_p / Pr, c_p = gamma/(gamma-1)  (> 0)        */
    double T_ref;               /* Sutherland reference temperature (T = p/rho, > 0)        */
    int32_t sutherland;         /* 1: mu(T) by the Sutherland law of Listing 1; 0: constant */
    int32_t streaming;          /* 0: two population buffers (pull); 1: one buffer updated in
                                   place by the AA pattern (half the memory, same traffic, the
                                   same collisions: results agree with 0 to FP32 rounding);
                                   2: two buffers of moments -- the regularized collision's
                                   outgoing set of field k is w_i (Q_k + c_i . J*_k / cs^2),
                                   so the state is kept as (Q_k, J*_k), 20 values per cell
                                   instead of 35, and the pull rebuilds each population with
                                   the collide's own FP32 operations: results bitwise those of
                                   0 (FP32 storage and GRLB_COLL_RLB_SENSOR only; 160 instead
                                   of 280 bytes per cell update); sources need 0, batches 0
                                   for domains they run in the batched kernel (below
                                   solo_min_cells; moment domains always run their own sweep)
                                   */
    double T_S;                 /* Sutherland constant relative to T_ref (0.4042)           */
    double omega_rho, omega_mom, omega_E; /* per-field relaxation 1/tau_LB, in (0, 2]       */
    double omega_min;           /* sensor floor rate (Listing 2)                            */
    double sensor_gain;         /* g (Listing 2)                                            */
    double J_min;               /* compression dead band (Listing 2)                        */
    double rho_min, p_min;      /* positivity floors, physical units (Alg. 1)               */
    double ref_rho, ref_p;      /* reference state at rest of the equilibrium shift (Sec. 2.2) */
    double left_prim[5];        /* (rho, ux, uy, uz, p) of the x = -1 ghost                 */
    double right_prim[5];       /* (rho, ux, uy, uz, p) of the x = nx ghost                 */
} grlb_params;

/* Diagnostics of the state a diagnostic sweep lands on (lattice units, FP64 sums). */
typedef struct {
    double totals[5];   /* sum over cells of Q_k (rho, m_x, m_y, m_z, E), lattice units      */
    double ke;          /* sum of 1/2 |m|^2 / rho                                            */
    double eps_s;       /* sum of mu |curl u|^2 (solenoidal dissipation, Sec. 3.4)          */
    double eps_d;       /* sum of (4/3) mu (div u)^2 (dilatational dissipation, Sec. 3.4)   */
    double rho_min;     /* minimum unfloored density                                        */
    double p_min;       /* minimum unfloored pressure, lattice units                        */
    int64_t n_floor;    /* cells where rho or p hit its floor                               */
    int64_t n_nan;      /* cells with a non-finite conserved moment                         */
    int64_t n_sensor;   /* cells with chi > 0                                                */
    int64_t step;       /* time step the values refer to                                     */
    double s;           /* dt/dx of the domain, for conversion to physical units            */
    int64_t ncells;
} grlb_diag;

typedef struct grlb_domain grlb_domain;
typedef struct grlb_batch grlb_batch;

/* Last error message of the calling thread ("" if none). Never NULL. */
const char* grlb_last_error(void);
/* Library version string. */
const char* grlb_version(void);

/* Create a domain: validates p, allocates two population buffers (storage type per
 * p->storage, in the cell-brick layout below) and the diagnostic scratch on the current CUDA
 * device.  stream is a
 * cudaStream_t (may be NULL).  On success *out owns the memory; free with grlb_destroy. */
grlb_status grlb_create(const grlb_params* p, void* stream, grlb_domain** out);
void grlb_destroy(grlb_domain* d);
grlb_status grlb_set_stream(grlb_domain* d, void* stream);
/* Device bytes the domain holds (populations + scratch). */
size_t grlb_device_bytes(const grlb_domain* d);
/* Device bytes grlb_create would allocate for these parameters (0 if invalid). */
size_t grlb_bytes_for(const grlb_params* p);

/* Initialise from primitive fields (host FP64, physical units, x fastest): rho[N],
 * u[3*N] (three planes ux, uy, uz), p[N].  Populations are set to the linear equilibrium of
 * each cell with the advective flux (zero non-equilibrium), Sec. 2.2.  Resets the step
 * counter.  Blocks until the host arrays have been copied. */
grlb_status grlb_init_primitive(grlb_domain* d, const double* rho, const double* u,
                                const double* p);

/* Same as grlb_init_primitive with the fields already resident on the domain's device (FP64,
 * physical units, same layout, device pointers).  Only enqueues on the domain's stream; the
 * caller keeps the arrays alive until the stream has passed this point. */
grlb_status grlb_init_primitive_device(grlb_domain* d, const double* rho, const double* u,
                                       const double* p);

/* Source term of the conservation laws (d_t Q + div Phi = S, Sec. 2.1), projected onto the
 * lattice weights after the collision (Algorithm 1, last step: + w_i S_k) in every following
 * sweep of this domain.  S is a device pointer to 5 planes of N FP32 values (rho, m_x, m_y,
 * m_z, E rates per unit physical time, x fastest), or NULL to remove it.  The library keeps
 * the pointer, does not own the memory, and reads it when each sweep runs: the caller may
 * rewrite it between sweeps in stream order (e.g. S at the mid-point time of the next step).
 * Domains with a source cannot join a batch. */
grlb_status grlb_set_source_device(grlb_domain* d, const float* S);

/* Pipelined initialisation, for loops that upload the next initial state while the current
 * one is being advanced.  grlb_stage_primitive enqueues the copy of host fields (the layout of
 * grlb_init_primitive; page-locked host memory for the copy to overlap) into one of two device
 * staging slots on a copy stream of the domain and returns at once; it fails with GRLB_ESTATE
 * when both slots hold states not yet consumed.  grlb_init_from_stage enqueues on the domain's
 * stream the initialisation from the oldest staged slot, ordered after its copy (GRLB_ESTATE if
 * nothing is staged), and resets the step counter.  The host arrays must stay unchanged until
 * that initialisation has run.  The slots (2 x 5 N doubles) are allocated on the first call and
 * freed with the domain. */
grlb_status grlb_stage_primitive(grlb_domain* d, const double* rho, const double* u,
                                 const double* p);
grlb_status grlb_init_from_stage(grlb_domain* d);

/* Enqueue nsteps >= 0 plain sweeps (Algorithm 1 on every cell + exact streaming).  A domain of
 * at most 4,194,304 cells on a stream other than the legacy default stream, asked for at least
 * 16 sweeps while its stream is not being captured, replays them from a CUDA graph of 8 sweeps
 * (captured on the first such call, re-captured after grlb_set_source_device; at most one
 * plain sweep first to match the graph's buffer and step parity, plain sweeps for the
 * remainder): the same kernels in the same order, so the state is bitwise that of one launch
 * per sweep.  Otherwise every sweep is one launch. */
grlb_status grlb_step(grlb_domain* d, int nsteps);

/* Enqueue one diagnostic sweep: the same update as grlb_step(d, 1), which also reduces
 * the grlb_diag quantities of the state it lands on into a device-side record, with
 * FP64 block partials summed in a fixed order (bitwise deterministic). */
grlb_status grlb_step_diag(grlb_domain* d);
/* Synchronize and copy the record of the last diagnostic sweep to *out.  Returns GRLB_ENUMERIC
 * (with *out filled in) when that sweep found cells with a non-finite conserved moment
 * (out->n_nan > 0): the state has blown up and further steps keep it non-finite; GRLB_ESTATE
 * if no diagnostic sweep ran since the last initialisation. */
grlb_status grlb_diag_read(grlb_domain* d, grlb_diag* out);

/* Failure check without a diagnostic sweep: enqueue on the domain's stream one read-only pass
 * over the stored populations of the current state (140 bytes per cell in FP32, 70 in FP16 /
 * BF16; about half a sweep's traffic) that sets *flag = 1 if any stored value is non-finite
 * (NaN or infinite).  It never writes 0: the caller clears the flag before the check.  flag must
 * be device-accessible: device memory, or page-locked host memory (with unified addressing its
 * host pointer is valid on the device), e.g. one slot per domain that a serving loop reads
 * once the stream has passed the check.  A state the diagnostics would report with
 * n_nan > 0 always sets the flag (a non-finite moment needs a non-finite population).
 * Errors: GRLB_EINVAL for NULL arguments; GRLB_ECUDA on launch failure. */
grlb_status grlb_check_finite(grlb_domain* d, int32_t* flag);

/* Conserved fields in physical units: out[5*N] = planes rho, m_x, m_y, m_z, E. */
grlb_status grlb_read_conserved(grlb_domain* d, double* out);
/* Primitive fields in physical units (no floors): rho[N], u[3*N], p[N], T[N]; any pointer
 * may be NULL to skip that field. */
grlb_status grlb_read_primitive(grlb_domain* d, double* rho, double* u, double* p, double* T);
/* Point probes: the 35 populations of listed cells without reading the whole state.  The state
 * of a domain is the post-collision population set f*_{k,i}(x) of its cells (Alg. 1 step 9
 * before streaming: what a two-buffer sweep writes at x), whatever the streaming pattern
 * (grlb_params.streaming) keeps where.
 *  cells  host array of n cell indices x + nx (y + ny z), each in [0, N); n >= 0 (0: no-op).
 *  f_out  host array of 35 n doubles, row-major by population: f_out[q n + j] = f*_q of
 *         cells[j], q = 7 k + i (field k = rho, m_x, m_y, m_z, E; link i = 0, +x, -x, +y, -y,
 *         +z, -z), in lattice units with the reference equilibrium added back, so that
 *         sum_i f_out[(7 k + i) n + j] is conserved field k of the cell in lattice units
 *         (rho; m s; E s^2 with s = dt/dx).
 * Synchronises the domain's stream.  Errors: GRLB_EINVAL for a NULL argument, n < 0 or a cell
 * outside [0, N) (checked before anything is enqueued); GRLB_ENOMEM / GRLB_ECUDA from the
 * staging allocation or the copies. */
grlb_status grlb_read_cells(grlb_domain* d, const int64_t* cells, int64_t n, double* f_out);

/* Raw checkpoint: stored populations + step counter.  grlb_save with buf == NULL sets
 * *bytes to the size needed; otherwise *bytes must be at least that size.  grlb_load
 * requires a buffer written by grlb_save of a domain with the same cells, storage and
 * streaming (the header's last 32-bit field records grlb_params.streaming).  Moment storage
 * (streaming 2) saves its moment buffer: bricks of 128 cells, each holding 20 rows 4 k + m
 * (m = 0: Q_k / 8, the share w_1 Q_k of each moving population; 1..3: J*_k,x..z; deviations
 * from the reference state), 128 FP32 values each.
 * Otherwise the format is a 32-byte header, then the population buffer as the library keeps it in device
 * memory -- the cell-brick layout: cells in storage order (x fastest) are grouped into
 * ceil(N / 128) bricks of 128 cells; a brick holds its 35 population rows q = 7k + i (field k
 * = rho, m_x, m_y, m_z, E; link i = 0, +x, -x, +y, -y, +z, -z) one after the other, 128
 * elements each, so population q of cell c is element (c / 128) 4480 + 128 q + c % 128 (the
 * cells past N in the last brick hold zeros).  Elements are the storage type's deviations
 * from the reference equilibrium (FP16: times a per-field power of two), followed, for a
 * one-buffer X_DIRICHLET_EQ domain, by its outflow record. */
grlb_status grlb_save(grlb_domain* d, void* buf, size_t* bytes);
grlb_status grlb_load(grlb_domain* d, const void* buf, size_t bytes);
int64_t grlb_steps_done(const grlb_domain* d);

/* ---- batching: many domains advanced by one call ------------------------------------------
 * A batch references existing domains (it does not own them; destroy the batch first) and
 * advances every active one by nsteps per grlb_batch_step, on the stream of domains[0] (or the
 * one set with grlb_batch_set_stream).  All domains must live on the same device.  A domain's
 * result never depends on the other domains of the batch.  Three schedules:
 *  GRLB_SCHED_CONCURRENT (default): every domain is advanced by the single-domain sweep that
 *    grlb_step runs (its record a kernel parameter, so its constants are constant-bank operands;
 *    domains of at most 4,194,304 cells replay their sweeps from their own CUDA graph), and the
 *    domains are dealt, largest first, over up to 32 side streams forked from and joined back
 *    into the batch stream, so that the kernels of different domains run concurrently and fill
 *    one another's waves.  Results are bitwise those of grlb_step.  Domains may use one-buffer
 *    streaming or moment storage.
 *  GRLB_SCHED_TABLE_CONST: the small domains (below solo_min_cells) advance together in one
 *    launch per step and (storage, collision) group of the batched sweep, one 128-thread CTA per
 *    tile, their records in a constant table of 160 slots shared by the process (a batch that
 *    finds too few free slots runs as GRLB_SCHED_TABLE); with enough tiles they are split into
 *    groups of about equal tile counts on up to max_lanes streams.  Large domains as under GRLB_SCHED_CONCURRENT.
 *  GRLB_SCHED_TABLE: as GRLB_SCHED_TABLE_CONST with the records in device memory, staged in
 *    shared memory by a persistent kernel walking a tile table.
 * Under the two table schedules a CTA covers tile_x cells along x times 128/tile_x rows, a
 * small domain's result matches grlb_step within FP32 rounding (16-bit storage: up to a few
 * stored values one 16-bit rounding apart; the two kernels read the constants from different
 * memory spaces) and small domains need two-buffer streaming.  No schedule takes a domain with a
 * source term. */
typedef enum { GRLB_SCHED_CONCURRENT = 0, GRLB_SCHED_TABLE_CONST = 1, GRLB_SCHED_TABLE = 2 } grlb_schedule;
typedef struct {
    int32_t block_x;        /* table schedules: default tile width 32, 64 or 128 (0 = 128,
                               narrowed for domains with fewer cells along x)                */
    int32_t solo_min_cells; /* table schedules: 0 = 262144 (64^3); < 0: every domain goes
                               through the table                                            */
    int32_t use_graph;      /* table schedules: 1 = replay the table launches of two steps
                               from a CUDA graph                                            */
    int32_t schedule;       /* grlb_schedule                                                */
    int32_t max_lanes;      /* GRLB_SCHED_TABLE_CONST: at most this many streams (1..8; 0 = 2)
                               over which the small domains are split, one per 592 tiles    */
} grlb_batch_config;

grlb_status grlb_batch_create(grlb_domain* const* domains, int n, const grlb_batch_config* cfg,
                              grlb_batch** out);
void grlb_batch_destroy(grlb_batch* b);
grlb_status grlb_batch_set_stream(grlb_batch* b, void* stream);
/* Mark which domains advance (active[i] != 0); rebuilds the tile table.  active == NULL
 * activates all. */
grlb_status grlb_batch_set_active(grlb_batch* b, const int* active);
/* Per-domain tile shape of the table schedules, e.g. from an autotuner: 32, 64 or 128 cells
 * along x of a 128-thread CTA (times 4, 2, 1 rows); 1 = linear tiles of 128 consecutive cells in
 * storage order; 0 = the default (block_x if the config sets it, else the least-padding width,
 * or linear tiles when rows do not fill whole tiles).  tile_x == NULL resets all to 0.  Rebuilds
 * the tile table.  Results do not depend on the tile shape; GRLB_SCHED_CONCURRENT ignores it. */
grlb_status grlb_batch_set_tile_x(grlb_batch* b, const int* tile_x);
/* Enqueue nsteps sweeps of every active domain by the batch's schedule (above). */
grlb_status grlb_batch_step(grlb_batch* b, int nsteps);

/* ---- diagnostic sweep without device allocation ---------------------------------------
 * The paper has no counterpart to this entry point.  It exists for callers that cannot call
 * cudaMalloc: an application whose memory manager reserved the device memory up front (a
 * further cudaMalloc would fail or fragment its pool), or a time-critical loop that cannot
 * afford the implicit device synchronisation cudaMalloc and cudaFree may cause.  It performs exactly
 * what grlb_step_diag does for one sweep, on population buffers the caller owns, and keeps
 * its block partials in a fixed array of device memory that the library declares statically
 * ((GRLB_NOALLOC_MAX_BLOCKS + 256) x GRLB_NDIAG doubles, 6.8 MB, held by every device that
 * loads the library until the process exits).  It never calls cudaMalloc, cudaFree or any other
 * allocating routine.
 *
 *  p        domain description (as for grlb_create); validated on the host.
 *  f_in     device pointer, current populations: 4480 ceil(N / 128) elements of the storage
 *           type in the cell-brick layout and equilibrium-shift format of the library's own
 *           buffers (the bytes grlb_save writes after its 32-byte header).
 *  f_out    device pointer, same size, receives the populations one step later; must not
 *           overlap f_in.
 *  diag_out device pointer to GRLB_NDIAG doubles: sums over cells of (Q_k - Q_ref,k) for
 *           k = rho, m_x, m_y, m_z, E, then ke, eps_s, eps_d, rho_min, p_min, n_floor,
 *           n_nan, n_sensor (the grlb_diag fields; totals[k] = N Q_ref,k + diag_out[k] with
 *           Q_ref = (ref_rho, 0, 0, 0, ref_p s^2/(gamma-1))).
 *  stream   cudaStream_t (may be NULL); the call only enqueues work on it.
 * Limits and behaviour: the launch may use at most GRLB_NOALLOC_MAX_BLOCKS CTAs of 128 cells
 * (8,388,608 cells, e.g. 128^3 or 256 x 256 x 128); larger domains return GRLB_EINVAL.  Each
 * call looks up the device address of the static array on the current device (a lookup that
 * allocates nothing); the first call on a device, and the first after a device reset, may load
 * the library's device code for it, so make that call before any stream capture begins.  Every
 * call on a device shares the
 * one array, which keeps the previous call's contents (each call overwrites every entry it
 * reads, so nothing needs clearing); calls whose sweeps overlap on the GPU race on it, so
 * serialise them (one stream, or events). */
#define GRLB_NDIAG 13
#define GRLB_NOALLOC_MAX_BLOCKS 65536
grlb_status grlb_step_diag_noalloc(const grlb_params* p, const void* f_in, void* f_out,
                                   double* diag_out, void* stream);


/* ---- initialisation mode ------------------------------------------------------------------
 * ce_init = 0 (default): grlb_init_primitive, grlb_init_primitive_device and
 * grlb_init_from_stage write the equilibrium f^eq(Q, Phi^adv) (no non-equilibrium part).
 * ce_init = 1: they write the Chapman-Enskog state of the fields instead (Sec. 2.3: the
 * non-equilibrium first moment of field k carries its gradient), the state a smooth flow has
 * after a collision: w_i (Q_k + c_i . (Phi^adv_k + A_k) / cs^2) with
 *   A_k = Phi^diff_k - (tau_k - 1) cs^2 grad Q_k,   tau_k = 1 / omega_k (nominal rates),
 * Phi^diff = (0, -tau_visc, -tau_visc u + q) from tau_visc = mu (grad u + grad u^T -
 * 2/3 div u I) and q = -kappa grad T at the local temperature, and gradients by central
 * differences (phi(x + e_a) - phi(x - e_a)) / 2 in lattice units of Q, u and T (periodic
 * wrap, or the ghost state beyond the ends of an X_DIRICHLET_EQ tube; zero along an axis of
 * extent 1).  With omega near 2 the equilibrium start leaves a non-equilibrium part that
 * changes sign every step for thousands of steps, and the cell-local diagnostics alternate
 * with it; the Chapman-Enskog start does not.  The conserved fields are the same in both modes.
 * The mode stays with the domain until changed.  Errors: GRLB_EINVAL for a NULL domain or a
 * value other than 0 / 1. */
grlb_status grlb_set_init_mode(grlb_domain* d, int32_t ce_init);

/* ---- z-slab decomposition (one periodic domain split along z) -----------------------------
 * The scheme's streaming moves one population per field across a z-face per step, so a domain
 * splits into z-slabs that exchange two planes of 5 populations per step (the decomposition a
 * multi-device run uses, here with both slabs on one device).  A slab of nz_s interior planes
 * is an ordinary periodic domain of nz_s + 2 planes (ghost plane 0 below, nz_s + 1 above),
 * initialised with the fields of the whole domain's planes z0 - 1 .. z0 + nz_s (periodic
 * wrap).  Before every step call grlb_halo_exchange_z for every adjacent pair (lower, upper),
 * including (last, first) of a periodic ring: it copies, for the five fields, the +z population
 * of lower's top interior plane into upper's ghost plane 0 and the -z population of upper's
 * bottom interior plane into lower's top ghost plane -- the only ghost values an interior cell
 * pulls.  The interior cells then evolve bitwise as in the undivided domain (same kernel, same
 * inputs); ghost-plane cells carry no meaning and enter the slab's own diagnostics, so interior
 * totals are taken from the readback.  Enqueued on the slabs' common stream.
 * Moment storage (streaming 2) exchanges Q_k / 8 and J*_k,z of the same planes (what a pull from a
 * ghost plane reads of it); both slabs must keep the same kind of state.
 * Errors: GRLB_EINVAL for NULL domains, slabs that differ in nx, ny, storage or streaming,
 * one-buffer streaming, non-periodic slabs, nz < 3, or different streams; GRLB_ECUDA on launch
 * failure. */
grlb_status grlb_halo_exchange_z(grlb_domain* lower, grlb_domain* upper);

/* The same exchange between slabs on different devices (one slab per rank of a multi-device
 * run): before every step each slab packs its two outgoing slices, the ranks swap them (e.g.
 * NCCL send / receive of device buffers, on the domain's stream order), and each slab unpacks
 * what it received.  Slices hold 5 x nx x ny stored values of the storage type (raw equilibrium-
 * shift deviations, FP16 scaled), field-major (rho, m_x, m_y, m_z, E), x fastest within a field.
 *  grlb_halo_pack_z:   to_upper <- the +z populations of the top interior plane (z = nz - 2),
 *                      to_lower <- the -z populations of the bottom interior plane (z = 1).
 *  grlb_halo_unpack_z: ghost plane z = 0 (+z populations) <- from_lower (the lower neighbour's
 *                      to_upper), ghost plane z = nz - 1 (-z populations) <- from_upper.
 * All buffers are device memory of the domain's device, 5 nx ny elements each, owned by the
 * caller; both calls only enqueue on the domain's stream.  Moment storage (streaming 2): a pull
 * from a ghost plane reads Q_k / 8 and J*_k,z of the ghost cell, so the slices hold those: 10 nx ny
 * FP32 values per buffer, slice 2 k + h = Q_k / 8 (h = 0) or J*_k,z (h = 1) of field k;
 * grlb_halo_exchange_z copies the same rows (both slabs must store moments).  A slab that is its own neighbour (one
 * rank, periodic) unpacks its own packed slices: the slab then evolves as the periodic domain.
 * Errors: GRLB_EINVAL for NULL arguments, one-buffer streaming, a non-periodic domain or
 * nz < 3; GRLB_ECUDA on launch failure. */
grlb_status grlb_halo_pack_z(grlb_domain* d, void* to_upper, void* to_lower);
grlb_status grlb_halo_unpack_z(grlb_domain* d, const void* from_lower, const void* from_upper);

/* ---- spectral post-processing (Sec. 3.4) ------------------------------------------------
 * The paper evaluates the Taylor-Green dissipation spectrally and shows the shell-averaged
 * velocity spectrum.  grlb_spectral_diag computes both from the domain's current state (the
 * state grlb_read_conserved returns), in lattice units, on the device with the library's own
 * FFT kernels (FP32 complex, radix 2), and returns FP64 results:
 *   u = m / rho_f with rho_f = max(rho, rho_min); p = max((gamma-1)(E - |m|^2/(2 rho_f)), p_min);
 *   T = p / rho_f; mu(T) the closure of the collision (constant or Sutherland);
 *   u^(m) = sum_x u(x) exp(-2 pi i m.x / n), integer wavevector m, m_a in [-n/2, n/2);
 *   spectrum[b] = sum over m with b - 1/2 <= |m| < b + 1/2 of 1/2 |u^(m)|^2 / N^2, so that
 *                 sum_b spectrum[b] = (1/N) sum_x 1/2 |u|^2 (Parseval);
 *   derivatives d/dx_a <-> i k_a, k_a = 2 pi m_a / n (zero for the Nyquist index m_a = -n/2);
 *   sums[0] = eps_s = sum_x mu |curl u|^2, sums[1] = eps_d = sum_x 4/3 mu (div u)^2 (the units
 *   of grlb_diag's cell-local eps_s / eps_d), sums[2] = sum_x 1/2 |u|^2.
 *  d         domain: periodic, an n^3 cube (n in [16, 1024]) or an n x n x 1 square (n in
 *            [32, 1024]), n a power of two.
 *  nbins     entries of spectrum to fill; shells beyond grlb_spectrum_shells(p) - 1 read 0,
 *            shells at or beyond nbins are left out of spectrum (not of sums).
 *  spectrum  host array of nbins doubles (may be NULL when nbins == 0).
 *  sums      host array of 3 doubles.
 * Five kernels (cubes; three for squares) move 372 bytes per cell (FP32 populations).  Scratch:
 * 36 bytes per cell plus small tables, taken from the stream-ordered pool on the domain's
 * stream and returned before the call ends.  The call synchronises the domain's stream
 * (twice).  Shell sums are accumulated in 64-bit fixed point (resolution 2^-60 of the total),
 * so the result does not depend on the order of the additions and is reproducible run to run.
 * Errors: GRLB_EINVAL for NULL pointers, negative nbins, a non-periodic domain or unsupported
 * extents; GRLB_ENOMEM / GRLB_ECUDA from the allocation or a launch. */
int32_t grlb_spectrum_shells(const grlb_params* p);  /* shells of the domain's spectrum, -1 if unsupported */
grlb_status grlb_spectral_diag(grlb_domain* d, int32_t nbins, double* spectrum, double* sums);

/* ---- FP32 issue-rate probe ----------------------------------------------------------------
 * Measurement helper with no counterpart in the paper: the 16-bit storage sweeps are bound by
 * instruction issue, and this probe measures that ceiling.  Enqueues one launch of ctas CTAs of
 * 256 threads; every thread runs iters x 128 FP32 fused multiply-adds in 8 independent chains.
 * *warp_instructions receives the launch's FFMA warp-instruction count (ctas x 8 x iters x 128);
 * that count divided by the launch's duration (events on `stream`) is the FFMA issue rate, and
 * 64 times it the FP32 FLOP rate.  sink: device array of ctas x 256 floats (in practice never
 * written: a thread stores to its own element only if its chain sum is exactly 0).
 * Errors: GRLB_EINVAL for ctas or iters < 1 or NULL pointers; GRLB_ECUDA on launch failure. */
grlb_status grlb_ffma_probe(int32_t ctas, int32_t iters, float* sink, void* stream, double* warp_instructions);

/* ---- cached device memory ----------------------------------------------------------------
 * Domains and batches take device memory from the device's stream-ordered pool, which keeps what
 * they release for reuse by this process (no device synchronisation on release).  grlb_trim_pool
 * synchronises the current device and returns the pool's unused memory to the system, e.g.
 * before creating a domain larger than any released before, or to leave the memory to another
 * process.  Errors: GRLB_ECUDA. */
grlb_status grlb_trim_pool(void);

/* ---- bounds-checked build ------------------------------------------------------------------
 * A debugging aid with no counterpart in the paper, standing in for a memory checker.
 * libgrlb_checked.so is this library compiled with GRLB_CHECKED.  In it every load and store of
 * every kernel first tests its byte range against a device-side registry of live regions: each
 * device allocation the library makes (live from its allocation to its release, in the order of
 * the allocating / releasing stream), the caller's device buffers lent to one call (the init,
 * halo, finiteness, allocation-free and probe calls: live while that call's kernels run) and a
 * source field set with grlb_set_source_device (live until replaced, cleared or the domain is
 * destroyed).  An access outside every live region is counted and not made (a load reads zero,
 * a store goes to a sink).  The test is a call per access, which can change which multiplies and
 * adds the compiler fuses, so results agree with the plain library's to rounding.  It costs a
 * scan of the registry per access: use small domains.
 *  grlb_checked_build  1 in the checked build, 0 in the plain one.
 *  grlb_check_read     synchronises the device and fills *out (violations: accesses outside
 *                      every live region; first_addr: the address of the first one, 0 if none;
 *                      live_regions: regions registered and not yet released -- 0 once every
 *                      domain, batch and staged buffer is gone; unmatched: releases of a region
 *                      that was not live; overflow: registrations that found the registry
 *                      (4096 regions) full).  reset != 0 zeroes every count but live_regions.
 *  grlb_check_probe    makes [base, base + bytes) live on `stream`, tests the range
 *                      [base + offset, base + offset + access_bytes) as a kernel access would
 *                      (counting a violation when it is outside every live region), then
 *                      releases the region.  Nothing at either address is read or written:
 *                      base may be any value.  For testing the checker itself.
 * In the plain build grlb_check_read and grlb_check_probe return GRLB_ESTATE. */
typedef struct {
    int64_t violations;
    uint64_t first_addr;
    int64_t live_regions;
    int64_t unmatched;
    int64_t overflow;
} grlb_check_counts;
int32_t grlb_checked_build(void);
grlb_status grlb_check_read(grlb_check_counts* out, int32_t reset);
grlb_status grlb_check_probe(const void* base, uint64_t bytes, int64_t offset, uint64_t access_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GRLB_H */
