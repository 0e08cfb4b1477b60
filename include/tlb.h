/*
 * tlb.h -- C ABI of the GB300 (sm_103a) ternary free-energy lattice Boltzmann
 * library: one fused time step of the model of Bala, Pepona, Karlin,
 * Kusumaatmaja & Semprebon, "Wetting boundaries for a ternary high density
 * ratio lattice Boltzmann method" (arXiv:1904.06881), Sec. II-IV.
 *
 * Every entry point returns an int: TLB_OK (0) or a negative TLB_E_* code;
 * tlb_strerror() names it and tlb_last_error_message() gives the detail of
 * the last failure on the calling thread.  Pointers marked (host) are read or
 * written synchronously and not retained; pointers marked (device) must be
 * device memory of the context's GPU.  Contexts and servers are owned by the
 * library and freed only by tlb_destroy / tlb_server_destroy.  A context may
 * be used from one host thread at a time.
 *
 * Layout: a lattice has N = nx*ny*nz nodes, node n = x + nx*(y + ny*z),
 * x fastest; every axis is periodic and walls come from the solid mask.
 * Vector fields are component-major (u[a*N + n]).  D2Q9 lattices have nz = 1.
 * Phases: C1 gas; C2 liquid with phi = +chi; C3 liquid with phi = -chi
 * (Sec. II.A, Eqs. definitionC1-C3).
 */
#ifndef TLB_H
#define TLB_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---- */
#define TLB_OK              0
#define TLB_E_INVAL        -1   /* bad argument, size or parameter */
#define TLB_E_NOMEM        -2   /* device or host allocation failed */
#define TLB_E_CUDA         -3   /* a CUDA runtime call failed */
#define TLB_E_UNSUPPORTED  -4   /* valid request this library does not implement */
#define TLB_E_UNCALIBRATED -5   /* force wetting: angles != 90 deg, no kappa^w and no matching calibration */
#define TLB_E_DIVERGED     -6   /* a non-positive density or population was met */
#define TLB_E_TIMEOUT      -7   /* a bounded device wait gave up */
#define TLB_E_BUSY         -8   /* no capacity (server queue or memory budget) */
#define TLB_E_NOTFOUND     -9   /* unknown ticket */
#define TLB_E_BOUNDS      -10   /* bounds-checked builds (-DTLB_BOUNDS_CHECK) only: a kernel computed a
                                   node index outside its array; the access was skipped */

enum { TLB_D2Q9 = 0, TLB_D3Q27 = 1 };
enum { TLB_WET_FORCE = 0, TLB_WET_GEOM_EXTRAP = 1, TLB_WET_GEOM_INTERP = 2 };

/* Full parameter set.  tlb_params_default() fills Table 1 set 1 (lambda =
 * 0.6, 1, 1; kappa = 0.01, 1, 1), chi = 5, the printed Carnahan-Starling
 * constants a = 0.037, b = 0.2, R = 1 (Sec. II.A), tau = 1 for f and g
 * (beta = 0.5, nu = 1/6; Sec. II.C), Gamma = 1 and coexistence densities at
 * T = 0.8 T_c.  All values are FP64 on the host. */
typedef struct {
    int    lattice;              /* TLB_D2Q9 or TLB_D3Q27 */
    int    nx, ny, nz;
    double lambda[3], kappa[3];  /* Eqs. BulkEnergy, InterfEnergy */
    double chi;
    double a, b, R;              /* EOS constants before rescaling (Eq. PsiEOS) */
    double rho_l, rho_g;         /* coexistence densities to reach, rho_l > rho_g > 0 */
    double beta;                 /* ELBM beta; nu = (1/beta - 1)/6 */
    double tau_g;                /* LBGK relaxation time of g (Eq. CahnHilliardLBM) */
    double Gamma;                /* mobility constant of g^eq */
    int    wetting;              /* TLB_WET_* (Sec. IV.A-B) */
    double theta_deg[3];         /* theta_21, theta_31, theta_23 (Sec. IV.A convention) */
    double kw_rho, kw_phi;       /* force-method strengths (Eq. forceBC) */
    int    g_fp16;               /* 1: reduced-precision g storage: the rest population g_0 in
                                    FP32, the moving populations in FP16 scaled by 16 */
    int    eos;                  /* TLB_EOS_*: the equation of state behind Psi_eos (Sec. II.A names
                                    Carnahan-Starling, used throughout the paper, van der Waals and
                                    Peng-Robinson as EOS the model hosts); default Carnahan-Starling */
    double omega;                /* Peng-Robinson acentric factor (default 0.344) */
    double nu[3];                /* kinematic viscosity of C1 (gas), C2, C3; all 0 (default): one
                                    beta for the whole fluid, as in the paper.  Otherwise the local
                                    beta = 1/(6 nu + 1) with nu the concentration-weighted mean of
                                    the three (concentrations clipped to [0, 1]); an extension, the
                                    paper has one viscosity (Sec. II.C) */
} tlb_params;
enum { TLB_EOS_CS = 0, TLB_EOS_VDW = 1, TLB_EOS_PR = 2 };

/* Constants derived at creation (host FP64). */
typedef struct {
    double T, a, b, R;           /* temperature; a, b after rescaling */
    double rho_l, rho_g;         /* coexistence densities actually used */
    double C, Psi0;              /* constants of Eq. PsiEOS */
    double Tc;                   /* critical temperature of the EOS */
    double kappa_rr, kappa_pp, kappa_rp;   /* gradient coefficients (Sec. II.B) */
    double aA;                   /* attraction constant in use: a (CS, vdW) or a A(T) (PR) */
} tlb_derived;

typedef struct tlb_ctx tlb_ctx;

const char *tlb_strerror(int code);
const char *tlb_last_error_message(void);
/* Library version and the compute capability the kernels were built for. */
int tlb_version(int *major, int *minor, int *sm);

/* Device allocator used for every later allocation (NULL restores
 * cudaMalloc/cudaFree).  alloc(bytes, user) returns device memory or NULL;
 * free_(ptr, user) releases it. */
int tlb_set_allocator(void *(*alloc)(size_t bytes, void *user), void (*free_)(void *ptr, void *user),
                      void *user);

int tlb_params_default(tlb_params *p);

/* Create a lattice (Sec. II).  densities = {rho_liquid, rho_gas} (both
 * liquids share rho_l, Sec. II.A); kappas = {kappa1, kappa2, kappa3} with
 * lambdas of Table 1 set 1; viscosities = kinematic viscosity of the three
 * phases, which must be equal (one beta, Sec. II.C) else TLB_E_UNSUPPORTED;
 * angles_deg = {theta_21, theta_31, theta_23}.  The density ratio fixes the
 * temperature of the Carnahan-Starling EOS; a and b are scaled so that the
 * coexistence densities are the ones given.  Force wetting takes its
 * strengths from a registered calibration table (tlb_set_force_calibration)
 * when an angle differs from 90 deg; without a matching table, or outside
 * its range, the call returns TLB_E_UNCALIBRATED. */
int tlb_create(int lattice, int nx, int ny, int nz, const double densities[2], const double kappas[3],
               const double viscosities[3], int wetting, const double angles_deg[3], tlb_ctx **out);
int tlb_create_ex(const tlb_params *p, tlb_ctx **out);
/* Host only (no device call): the constants a context created from p would
 * use -- temperature from the density ratio, a and b after rescaling,
 * coexistence densities, C and Psi0 of Psi_eos (Sec. II.A), T_c, gradient
 * coefficients (Sec. II.B).  TLB_E_INVAL for invalid parameters or no
 * coexistence. */
int tlb_derive(const tlb_params *p, tlb_derived *out);

/* Force-wetting calibration.  Eq. forceBC (Sec. IV) sets the wall's wetting
 * through strengths kappa^w, not angles; the paper maps one to the other by
 * measurement.  This registers such a measurement: n pairs (kappa_w[i],
 * theta_deg[i]) of a liquid drop on a wall (kappa_phi^w = 0), kappa_w
 * increasing and theta decreasing, for the lattice and thermodynamic
 * parameter set of *p (lattice, lambda, kappa, chi, a, b, R, rho_l, rho_g;
 * the other fields are ignored).  tlb_create / tlb_create_ex / tlb_submit with
 * TLB_WET_FORCE, kw_rho = kw_phi = 0 and theta_21 or theta_31 != 90 deg then
 * set s2 = kappa(theta_21), s3 = kappa(theta_31) by linear interpolation and
 * kw_rho = (s2 + s3)/2, kw_phi = (s2 - s3)/2 (theta_23 is not an input of this
 * scheme).  Explicit kw_rho / kw_phi always take precedence.  Tables are
 * process-wide; registering the same lattice and parameter set again
 * replaces its table.  Host data, copied.  TLB_E_INVAL for fewer than two
 * points, non-finite or non-monotone data.  The Python binding registers the
 * tables shipped in paper_1904_06881_gb300/force_wetting_calibration.json. */
int tlb_set_force_calibration(const tlb_params *p, const double *kappa_w, const double *theta_deg, int n);
void tlb_destroy(tlb_ctx *ctx);
int tlb_get_params(const tlb_ctx *ctx, tlb_params *out);
int tlb_get_derived(const tlb_ctx *ctx, tlb_derived *out);

/* Work stream of the context (cudaStream_t); NULL is the legacy default
 * stream.  tlb_step and the *_device calls are asynchronous on it. */
int tlb_set_stream(tlb_ctx *ctx, void *cuda_stream);

/* Solid mask (host, N bytes, 1 = solid).  Resets the ghost-node list and the
 * wall flags used by the wall rules of Sec. IV. */
int tlb_set_solid(tlb_ctx *ctx, const uint8_t *mask);

/* Initial fields (host FP64): rho, phi (N each), u = fluid velocity (D*N) or
 * NULL for rest.  f = f^eq(rho, u - F/(2 rho)) and g = g^eq(phi, u, mu_phi)
 * with F and mu_phi of the initial fields (Sec. II.C). Synchronous. */
int tlb_init_fields(tlb_ctx *ctx, const double *rho, const double *phi, const double *u);
/* Same with device FP32 inputs; asynchronous on the context stream. */
int tlb_init_fields_device(tlb_ctx *ctx, const float *rho, const float *phi, const float *u);

/* Advance nsteps time steps (Eqs. ELBMequation, CahnHilliardLBM with the
 * wall rules and wetting scheme of Sec. IV).  Asynchronous; returns the
 * sticky error status seen by the last synchronising call. */
int tlb_step(tlb_ctx *ctx, int nsteps);
/* One phase of a time step, for per-kernel timing: phase 0 computes the
 * moments rho, phi (D3Q27; empty for D2Q9, whose step kernel sums the moments
 * of its tile and halo itself); phase 1 is empty (kept for callers that issue
 * 0, 1, 2); phase 2 runs the fused kernel -- ghost layer, stencils, force,
 * collision, streaming -- and completes the step.  Issuing 0, 1, 2 (or 0, 2)
 * in order is exactly one tlb_step.  A step is one launch (D2Q9) or two
 * (D3Q27).  Asynchronous. */
int tlb_step_phase(tlb_ctx *ctx, int phase);
/* Wait for the context stream and report what the kernels flagged since the
 * last check: TLB_E_TIMEOUT if a tile's tensor copies of its populations
 * (D3Q27) did not complete within the kernel's one-second bound (the tile
 * was skipped), else TLB_E_DIVERGED for a non-positive density or
 * population; bounds-checked builds also report TLB_E_BOUNDS.  The error
 * sticks to the context. */
int tlb_sync(tlb_ctx *ctx);

/* Fields of the current state (host FP64; any pointer may be NULL): rho,
 * phi (N), bare velocity u = sum f c / rho (D*N), concentrations C (3*N,
 * Eqs. definitionC1-C3).  Solid nodes read 0.  Synchronous. */
int tlb_get_fields(tlb_ctx *ctx, double *rho, double *phi, double *u, double *C);
/* Device FP32 outputs (rho, phi: N; u: D*N; any may be NULL); asynchronous. */
int tlb_get_fields_device(tlb_ctx *ctx, float *rho, float *phi, float *u);

/* FP64 sums over fluid nodes: out = {sum rho, sum phi, sum C1, sum C2,
 * sum C3, 0.5 sum rho |u|^2}.  Synchronous. */
int tlb_diagnostics(tlb_ctx *ctx, double out[6]);

/* Auxiliary fields recomputed from the current state, as FP64 on the host:
 * which = 0 p0, 1 mu_rho, 2 mu_phi, 3..5 F (total force incl. wetting force),
 * 6..11 P_xx,P_yy,P_zz,P_xy,P_xz,P_yz, 12 rho incl. ghost layer, 13 phi incl.
 * ghost layer.  Solid nodes read 0 for which < 12. */
int tlb_get_aux(tlb_ctx *ctx, int which, double *out);

/* Pre-collision populations (host FP64, Q*N each, f[i*N + n]); the lattice
 * direction order is that of tlb_lattice_directions.  Synchronous. */
int tlb_get_populations(tlb_ctx *ctx, double *f, double *g);
int tlb_set_populations(tlb_ctx *ctx, const double *f, const double *g);
/* Lattice directions: c (Q*3 ints) and weights w (Q doubles); returns Q. */
int tlb_lattice_directions(int lattice, int *c, double *w);

/* Checkpoint: the populations and step counter in an opaque host buffer. */
size_t tlb_snapshot_bytes(const tlb_ctx *ctx);
int tlb_snapshot(tlb_ctx *ctx, void *host, size_t bytes);
int tlb_restore(tlb_ctx *ctx, const void *host, size_t bytes);
long long tlb_steps_done(const tlb_ctx *ctx);
/* Device bytes held by the context. */
size_t tlb_device_bytes(const tlb_ctx *ctx);
/* Kernel launches issued by the context since creation. */
long long tlb_launch_count(const tlb_ctx *ctx);

/* ---- allocation-free stepping (no counterpart in the paper) ----
 * For callers that must not allocate device memory while they run: code that
 * owns a fixed device-memory budget carved up in advance, hosts whose
 * allocator is a framework pool that raw cudaMalloc would bypass, and loops
 * that cannot afford the device-wide synchronisation cudaMalloc/cudaFree may
 * imply.  tlb_step_noalloc advances caller-owned populations by nsteps with
 * the kernels of tlb_step (the same populations, bit for bit) and allocates
 * nothing: its scratch (moments, tile table, node flags, error word, the two
 * batch entries) is one static device array of TLB_NOALLOC_MAX_NODES * 25 +
 * 1280 bytes (26.2 MB) that every GPU loading this library holds until exit.
 *   p          lattice, sizes and physics; at most TLB_NOALLOC_MAX_NODES
 *              (1048576) nodes, else TLB_E_INVAL; g_fp16 must be 0.  Force
 *              wetting given by angles takes its strengths from the
 *              registered calibration tables, as tlb_create_ex does
 *              (TLB_E_UNCALIBRATED without a matching table).
 *   mask       host, N bytes (1 = solid) or NULL for no walls.
 *   f, f_tmp   device, Q*N floats each: f holds the pre-collision populations
 *              minus the lattice weights (the layout tlb_get_populations
 *              describes, minus w_i, as float); f_tmp is work space.
 *   g, g_tmp   device, Q*N floats each, same roles for the order parameter.
 *   On return the advanced populations are in f and g (asynchronously, on
 *   cuda_stream; NULL = legacy default stream).
 * The first call on a device looks up the scratch array's device address
 * (once per device, with that device current).  All calls share the one
 * array and it keeps the last call's contents.  Every call resets the error
 * word and rewrites the batch entries (they hold f, g and their work
 * buffers).  The node flags and the tile table are built on the host and
 * uploaded when the lattice, the sizes, the mask's contents or the
 * stream differ from the previous call's on this device; otherwise the copy
 * in the array is used again (one N-byte comparison instead of the host pass
 * over the mask and its upload).  Calls that overlap on the GPU --
 * concurrent streams or host threads on one device -- race and must be
 * serialised by the caller.  Divergence is not reported by this call; use a
 * context (tlb_sync) to get it. */
#define TLB_NOALLOC_MAX_NODES (1 << 20)
int tlb_step_noalloc(const tlb_params *p, const uint8_t *mask, float *f, float *f_tmp, void *g, void *g_tmp,
                     int nsteps, void *cuda_stream);

/* ---- batched lattices: many contexts advanced by one launch per phase ---- */
/* Advance every context in ctxs[0..n) by nsteps, with one launch per kernel
 * phase covering all lattices (a tile -> lattice table).  All contexts must
 * share the lattice type and the stream of ctxs[0]. */
int tlb_step_batch(tlb_ctx *const *ctxs, int n, int nsteps);

/* ---- resident batches: a table built once, graph replays, tuned launches ----
 * Many independent lattices (one lattice type and g storage) advanced
 * together by one launch per kernel phase over a tile -> lattice table, the
 * same kernels as tlb_step (a lattice gives bit-identical results alone and
 * in a batch).  The table lives on the device for the batch's lifetime, so
 * tlb_batch_step allocates nothing and does not synchronise the host; steps
 * are replayed from CUDA graphs of graph_depth steps (captured on first use
 * for each buffer parity).  The contexts must outlive the batch; stepping a
 * context on its own between batch steps is allowed (the batch notices and
 * rewrites its table). */
typedef struct tlb_batch tlb_batch;
enum { TLB_ORDER_LATTICE = 0,        /* tiles of lattice 0, then lattice 1, ... */
       TLB_ORDER_INTERLEAVED = 1,    /* tile j of every lattice in turn */
       TLB_ORDER_LARGEST_FIRST = 2   /* lattice-major, largest lattices first */ };
typedef struct {
    int variant;        /* D2Q9 register budget: 0 = 3 CTAs/SM, 1 = 4 CTAs/SM,
                           -1 = chosen by launch size; D3Q27: ignored */
    int tile_order;     /* TLB_ORDER_*: order of the tile table (CTA dispatch order) */
    int graph_depth;    /* steps per CUDA-graph replay: 0 (direct launches) or even */
    double us_per_step; /* set by tlb_batch_tune: measured time of one step */
} tlb_batch_config;
/* Build the batch over ctxs[0..n), which must share one stream (TLB_E_INVAL
 * otherwise); the batch's work is issued on it.  cfg NULL =
 * variant -1, lattice order, graph depth 8.  The table upload is ordered on
 * the stream (no host synchronisation).  TLB_E_INVAL for mixed lattice types
 * or g storage, or a repeated context. */
int tlb_batch_create(tlb_ctx *const *ctxs, int n, const tlb_batch_config *cfg, tlb_batch **out);
/* Advance every lattice by nsteps, asynchronously on the batch's stream. */
int tlb_batch_step(tlb_batch *b, int nsteps);
/* Autotuner: times every candidate configuration (register budget, tile
 * order, graph depth 2/8/32) on this batch's own lattices -- graph replays
 * of launches that recompute the current step, so the lattices' state is
 * unchanged -- and keeps the fastest; `reps` scales the timed replays.
 * Synchronous.  The chosen configuration is written to *chosen (may be NULL). */
int tlb_batch_tune(tlb_batch *b, int reps, tlb_batch_config *chosen);
int tlb_batch_get_config(const tlb_batch *b, tlb_batch_config *out);
/* Waits for the batch's stream, then frees its tables and graphs (not the contexts). */
void tlb_batch_destroy(tlb_batch *b);

/* ---- request server (continuous batching) ---- */
typedef struct tlb_server tlb_server;
typedef struct {
    tlb_params params;           /* lattice, sizes and physics */
    const uint8_t *mask;         /* host, N bytes (may be NULL: no walls) */
    const double *rho, *phi;     /* host initial fields, N each */
    int nsteps;                  /* steps to run */
} tlb_request;
typedef struct {
    int state;                   /* TLB_REQ_* */
    int status;                  /* TLB_OK or the error that failed it */
    double submit_s, start_s, done_s;   /* host wall-clock seconds */
    double mass[6];              /* tlb_diagnostics at completion */
} tlb_result;
enum { TLB_REQ_QUEUED = 0, TLB_REQ_RUNNING = 1, TLB_REQ_DONE = 2, TLB_REQ_FAILED = 3 };

/* Server with a device-memory budget for resident lattices and a cap on
 * lattices advanced together; steps_per_round steps run between admissions.
 * cuda_stream NULL: the server steps each group of lattices (lattice type x
 * g storage) on a stream of its own, so that the groups' rounds overlap on the
 * GPU; otherwise every group uses cuda_stream.  Each pump issues one round of
 * the active lattices through resident batches (one per group, rebuilt when
 * its members change) and admits queued requests while that round runs on
 * the GPU (their initial fields go through another stream); requests
 * admitted in a round join the next one. */
int tlb_server_create(size_t hbm_budget_bytes, int max_active, int steps_per_round, void *cuda_stream,
                      tlb_server **out);
/* Copy a request in; returns a ticket.  TLB_E_INVAL if the request can never
 * fit the budget. */
int tlb_submit(tlb_server *s, const tlb_request *req, uint64_t *ticket);
/* Advance the server by one round (admit, step all active lattices together,
 * retire finished ones).  Returns the number of active lattices or < 0. */
int tlb_server_pump(tlb_server *s);
/* State of a ticket; when DONE, rho/phi (host, N each, may be NULL) receive
 * the final fields and the ticket is released. */
int tlb_poll(tlb_server *s, uint64_t ticket, tlb_result *res, double *rho, double *phi);
int tlb_server_stats(tlb_server *s, int *queued, int *active, size_t *bytes_in_use);
/* Admission order (no paper counterpart).  TLB_SCHED_FIFO (the default):
 * arrival order, the head of the queue waits until its memory is free and
 * nothing overtakes it.  TLB_SCHED_SHORTEST: the queued request with the least
 * work (nodes x steps) among those whose memory fits is admitted first (ties
 * in arrival order); with max_wait_s > 0, requests queued longer than that
 * come first, in arrival order, and are not overtaken.  Takes effect at the
 * next pump.  TLB_E_INVAL for an unknown policy or max_wait_s < 0. */
enum { TLB_SCHED_FIFO = 0, TLB_SCHED_SHORTEST = 1 };
int tlb_server_set_policy(tlb_server *s, int policy, double max_wait_s);
void tlb_server_destroy(tlb_server *s);

#ifdef __cplusplus
}
#endif
#endif
