/*
 * lb.h - C ABI of the GB300 free-energy lattice Boltzmann library (liblb.so).
 *
 * The library advances the free-energy lattice Boltzmann scheme of Pooley &
 * Furtado ("Eliminating spurious velocities in the free energy lattice
 * Boltzmann method") for a van der Waals liquid-gas system on the D2Q9 and
 * D3Q19 lattices:
 *   - van der Waals bulk pressure p0 (Eq. 2) and lambda = nu (1 - 3 c_s^2) (Eq. 36);
 *   - isotropic gradient / Laplacian stencils (Eq. 32 in 2D, Eq. 29 with the
 *     coefficients of Eq. 31 in 3D);
 *   - the tuned equilibrium distribution (Eqs. 5, 6 with the weights of
 *     Sec. VIII / Eq. 31) - "equilibrium scheme";
 *   - the momentum-conserving forcing variant (Sec. VI, Eqs. 27, 28), whose
 *     update reads density two sites away - "forcing scheme";
 *   - BGK collision and streaming (Eq. 4).
 * Lattice units: dx = dt = c = 1.  Every domain is periodic in all directions.
 *
 * Conventions shared by every call
 *   - Host arrays are owned by the caller and only read/written during the
 *     call.  Fields are float64, structure of arrays, site index
 *     x + nx*(y + ny*z), x fastest.  Vector fields are stored component by
 *     component (all x components, then all y, then all z).
 *   - Population arrays exchanged with the host are float64 with layout
 *     [i][z][y][x], i the velocity index in the paper's order (Sec. II for
 *     D2Q9, Sec. VII for D3Q19).  They hold f_i(r, t), the distribution after
 *     streaming (the left-hand side of Eq. 4).
 *   - Device memory belongs to the context and is released by lb_destroy.
 *   - Every call returns an lb_status and never throws.  On error the
 *     thread-local message of lb_last_error() says why.  A device error seen
 *     by a context (a CUDA failure or a non-finite density) is sticky: every
 *     later call on that context returns it until lb_destroy.
 *   - Work is queued on the context's CUDA stream; calls that return host
 *     data synchronise that stream.
 */
#ifndef LB_H
#define LB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_ctx lb_ctx;

typedef enum {
    LB_OK = 0,
    LB_EINVAL = 1,     /* invalid argument or parameter set */
    LB_ENOMEM = 2,     /* device or host allocation failed */
    LB_ECUDA = 3,      /* a CUDA runtime call failed */
    LB_EUNSTABLE = 4,  /* a density became non-finite or non-positive */
    LB_ETIMEOUT = 5,   /* a bounded device wait expired */
    LB_ESTATE = 6      /* call made in the wrong order (e.g. step before init) */
} lb_status;

typedef enum { LB_D2Q9 = 0, LB_D3Q19 = 1 } lb_lattice;

/* LB_SCHEME_EQUILIBRIUM: M_ab = kappa d_a rho d_b rho terms inside f^eq (Eq. 5).
 * LB_SCHEME_FORCING: M_ab terms moved into the body force g (Sec. VI). */
typedef enum { LB_SCHEME_EQUILIBRIUM = 0, LB_SCHEME_FORCING = 1 } lb_scheme;

/* Storage of the populations in HBM.  Arithmetic is float64 for LB_F64 and
 * float32 otherwise.  LB_F16DEV / LB_BF16DEV keep f_0 in float32 and store
 * f_i - w_i p0(rho_ref) (i >= 1) in fp16 / bf16: w_i p0(rho_ref) is the rest
 * equilibrium of Eq. 5 at u = 0 and zero gradients, the same in bulk liquid
 * and gas at coexistence. */
typedef enum { LB_F64 = 0, LB_F32 = 1, LB_F16DEV = 2, LB_BF16DEV = 3 } lb_storage;

typedef struct {
    int lattice;          /* lb_lattice */
    int nx, ny, nz;       /* sites per direction, >= 1; nz must be 1 for D2Q9 */
    double a, b, T;       /* van der Waals p0 = rho T/(1 - b rho) - a rho^2 (Eq. 2); 0 < T < 8a/27b */
    double kappa;         /* gradient coefficient of Eq. 1, > 0 */
    double tau;           /* BGK relaxation time of Eq. 4, > 1/2 */
    int scheme;           /* lb_scheme */
    int storage;          /* lb_storage */
    double rho_ref;       /* reference density of the deviation storage; 0 => liquid coexistence density */
} lb_params;

typedef struct {
    double mass;          /* sum_r rho (float64, fixed summation order) */
    double momentum[3];   /* sum_r rho u (Eq. 3); unused components are 0 */
    double max_u;         /* max_r |u|, u the lattice velocity of Eq. 3 */
    double max_v;         /* max_r |v|, v = u + g/(2 rho) (Eq. 40); = max_u for the equilibrium scheme */
    double min_rho, max_rho;
    long long step;       /* time steps taken since the last init (or the step of an imported state) */
    int status;           /* lb_status of the context */
    double dP;            /* p0(rho at the inside probe) - p0(rho at the outside probe): the pressure
                             jump across the interface of Sec. IV (Eq. 2); probes: lb_set_probes */
    double max_du;        /* max_r |u(r) - u_prev(r)|, u_prev the u of the previous lb_stats_get on this
                             context: the steady-state test of Sec. IV runs; -1 on the first call after an
                             init, a population or state import */
    long long du_steps;   /* steps between this call and that previous call (0 when max_du = -1) */
} lb_stats;

/* Library version string (static storage). */
const char* lb_version(void);

/* Thread-local message describing the last error on this thread ("" if none). */
const char* lb_last_error(void);

/* Maxwell coexistence densities of the van der Waals fluid (Eq. 2, Sec. II):
 * rho_l > rho_g with equal p0 and equal chemical potential
 * mu0 = T ln(rho/(1 - b rho)) + T b rho/(1 - b rho) - 2 a rho.
 * float64 Newton iteration on the host.  LB_EINVAL unless a, b > 0 and
 * 0 < T < 8a/(27b) and both outputs are non-NULL. */
lb_status lb_coexistence(double a, double b, double T, double* rho_l, double* rho_g);

/* Create a context: validates *p, solves the coexistence densities and
 * allocates the two population buffers on the current CUDA device.
 * cuda_stream is a cudaStream_t (NULL = the legacy default stream); it must
 * outlive the context.  *out receives the context, or NULL on error.
 * LB_EINVAL also for more than 2^31 - 1 sites (the kernels index sites with
 * 32-bit integers). */
lb_status lb_create(const lb_params* p, void* cuda_stream, lb_ctx** out);

/* Bytes of the two population buffers a context with parameters *p holds
 * (host only; LB_EINVAL for invalid parameters or a NULL bytes). */
lb_status lb_population_bytes(const lb_params* p, size_t* bytes);

/* lb_create with the two population buffers in caller-owned device memory
 * (for instance a framework's allocator): `populations` must be a device
 * pointer on the current device, 256-byte aligned, with at least
 * lb_population_bytes(p) bytes; it is used as is (no copy), must outlive the
 * context and is not freed by lb_destroy.  Both are checked on the host
 * before any device work (LB_EINVAL).  Everything else as lb_create. */
lb_status lb_create_with_buffers(const lb_params* p, void* cuda_stream, void* populations, size_t bytes,
                                 lb_ctx** out);

/* Release every device allocation of the context (not a buffer given to
 * lb_create_with_buffers).  NULL-safe. */
lb_status lb_destroy(lb_ctx* ctx);

/* Coexistence densities the context uses (liquid, gas). */
lb_status lb_get_coexistence(const lb_ctx* ctx, double* rho_l, double* rho_g);

/* Initialise drops (synthetic workload of Sec. IV): density
 *   rho0 = rho_g + (rho_l - rho_g) * max_k 1/2 (1 + tanh((R_k - d_k)/width)),
 * d_k the periodic minimum-image distance of integer site coordinates from
 * centre k; then f = f^eq(rho0, u = 0) of the context's scheme (Eqs. 5, 6),
 * gradients taken with the stencils.  centres: ndrops*dim doubles (x, y[, z]);
 * radii: ndrops doubles > 0.  ndrops = 0 gives uniform gas.  Resets the step
 * counter.  The first initialisation allocates one float64 per site (the
 * density); lb_fields / lb_stats_get and velocity uploads later allocate the
 * other float64 field arrays (13 doubles per site in all, kept until
 * lb_destroy). */
lb_status lb_init_drops(lb_ctx* ctx, int ndrops, const double* centres, const double* radii,
                        double width);

/* Initialise from a host density field rho (N doubles) and velocity u
 * (dim*N doubles, NULL => 0): f = f^eq(rho, u) of the context's scheme. */
lb_status lb_init_fields(lb_ctx* ctx, const double* rho, const double* u);

/* Load / read the populations f_i(r, t) (Q*N float64, layout [i][z][y][x]).
 * Loading converts to the context's storage (rounding for reduced storage)
 * and resets the step counter. */
lb_status lb_set_populations(lb_ctx* ctx, const double* f);
lb_status lb_get_populations(lb_ctx* ctx, double* f);

/* Read the populations of a box of the periodic lattice: sites (x0 + x, y0 + y, z0 + z)
 * wrapped into the lattice, 0 <= x < bx, 0 <= y < by, 0 <= z < bz, decoded to float64
 * into f (caller-owned host array of Q*bx*by*bz doubles, layout [i][z][y][x] of the
 * box).  For lattices too large to read whole.  Origins in [0, n) and sizes in [1, n]
 * per axis (n the lattice size; D2Q9: z0 = 0, bz = 1), at most 2^LB_BOX_MAX_LOG2_SITES
 * sites; otherwise LB_EINVAL.  Allocates and frees a device staging buffer of the
 * box's size and synchronises the context's stream. */
#define LB_BOX_MAX_LOG2_SITES 24
lb_status lb_get_populations_box(lb_ctx* ctx, int x0, int y0, int z0, int bx, int by, int bz, double* f);

/* Advance nsteps >= 0 time steps of Eq. 4: one fused kernel per step
 * (moments, stencils, equilibrium, force, BGK, streaming).  Asynchronous on
 * the context's stream; a non-finite density raises the context's status,
 * reported by the next synchronising call.  With nsteps > 64 the steps run
 * as replays of a CUDA graph of 64 kernel launches (captured once per
 * starting buffer on a private stream of the context, after one ordinary
 * launch) plus ordinary launches for the rest; the results are identical. */
lb_status lb_step(lb_ctx* ctx, int nsteps);

/* Wait for queued work; returns the context's status. */
lb_status lb_synchronize(lb_ctx* ctx);

/* Host copies of rho (N), u (dim*N) and v = u + g/(2 rho) (dim*N; Eq. 40,
 * = u for the equilibrium scheme).  Any output may be NULL.  Synchronises. */
lb_status lb_fields(lb_ctx* ctx, double* rho, double* u, double* v);

/* float64 reductions of the current state (see lb_stats).  Synchronises.
 * Keeps a float64 copy of u (dim * N doubles, allocated by the first call)
 * as the reference of the next call's max_du. */
lb_status lb_stats_get(lb_ctx* ctx, lb_stats* out);

/* Probe sites of lb_stats.dP: inside[3], outside[3] = (x, y, z), each in
 * [0, n) per axis (z = 0 for D2Q9); LB_EINVAL otherwise.  lb_create sets
 * inside = (nx/2, ny/2, nz/2), outside = (0, 0, 0) (a centred drop);
 * lb_init_drops sets inside = the site nearest to the first drop centre and
 * outside = the site farthest (periodic minimum image) from every centre,
 * searched on a grid of step ceil(n/64) per axis. */
lb_status lb_set_probes(lb_ctx* ctx, const int* inside, const int* outside);
lb_status lb_get_probes(const lb_ctx* ctx, int* inside, int* outside);

/* ---- Checkpoint / restart (no counterpart in the paper) ---------------------
 *
 * lb_get_state exports the raw stored state: a fixed header (magic "LBGBSTA1",
 * version 1, lattice, nx, ny, nz, scheme, storage, population layout, the step
 * counter, the parameter hash of lb_params_hash and the payload size) followed
 * by the bytes of the current population buffer exactly as stored (float64 /
 * float32 / fp16 or bf16 deviations, in the context's layout).  buf = NULL:
 * *bytes receives the size needed; otherwise *bytes is the capacity of the
 * caller-owned host buffer buf (LB_EINVAL if smaller) and receives the size
 * written.  Synchronises.  LB_ESTATE before the first init.
 * lb_set_state imports such a buffer into a context created with the same
 * lb_params (LB_EINVAL if the header, the parameter hash or the size differ),
 * sets the step counter from it and clears the context's device status; the
 * next steps continue the exported run bit for bit (N + N steps with an
 * export and import in between equal 2N steps).  Synchronises. */
lb_status lb_get_state(lb_ctx* ctx, void* buf, size_t* bytes);
lb_status lb_set_state(lb_ctx* ctx, const void* buf, size_t bytes);

/* ---- Index checks (no counterpart in the paper) ---------------------------
 *
 * A library built with -DLB_DEBUG_BOUNDS (paper_0710_5470_gb300.build,
 * debug=True: _build_debug/liblb_debug.so) tests the site index of every
 * global population access of the fused step kernels against the lattice
 * before making it; an out-of-range access is skipped and the first one is
 * recorded (no trap).  lb_debug_bounds returns whether this library has the
 * checks (*checked = 1) and the first recorded violation since the last call
 * (*violation: 0 if none, else bit 63 set, the kind of access in bits 48..55 -
 * 1/2/3 pair-kernel load/store/shared write, 4/5 D3Q19 tile load/store, 6/7
 * D2Q9 load/store - and the site index in bits 0..47), then clears it.
 * Synchronises the device.  Either pointer may be NULL. */
lb_status lb_debug_bounds(int* checked, unsigned long long* violation);

/* 64-bit FNV-1a hash of the parameters that define a run (lattice, sizes,
 * scheme, storage, a, b, T, kappa, tau, rho_ref); host only.  LB_EINVAL for
 * an invalid parameter set (the checks of lb_create). */
lb_status lb_params_hash(const lb_params* p, unsigned long long* hash);

/* Free parameters of the D2Q9 model (Sec. III, Eq. 16): the diagonal weights w^p_{5-8} (pressure),
 * w^t_{5-8} (interface term) and w^xx_{5-8} (M term) of the equilibrium, and the diagonal
 * coefficients B of the gradient stencil (Eq. 10), D of the Laplacian (Eq. 11) and F of the force
 * stencil (Eq. 28).  The other weights follow from the constraints after Eqs. 14-15 and from
 * 2A + 4B = 1, C + 2D = 1, 2E + 4F = 1.  The optimum of Sec. III is 1/12, 1/12, -1/24, 1/12, 1/6,
 * 1/12 (what the fused kernels hard-wire); other values give the scans of Fig. 2 and the prior-art
 * choices of Sec. III. */
typedef struct {
    double wp58, wt58, wxx58, B, D, F;
} lb_free_params;

/* Run a D2Q9 float64 context with these free parameters: later lb_init_drops / lb_init_fields,
 * lb_step and the v of lb_fields / lb_stats_get use them, through plain float64 kernels (three
 * launches per step; for parameter studies, not for throughput).  NULL returns the context to
 * the fused kernels.  LB_EINVAL for another lattice or storage or a non-finite value; the first
 * call allocates 6 float64 per site of work arrays. */
lb_status lb_set_free_params(lb_ctx* ctx, const lb_free_params* params);

/* Number of sites N and populations Q of the context. */
lb_status lb_shape(const lb_ctx* ctx, long long* n_sites, int* q);

/* Device pointer of the current population buffer and its byte size, for
 * callers that stage inputs in device memory themselves.  Layout: population
 * 0 as one array of pitch = N rounded up to a multiple of 128 elements, then
 * populations 1..Q-1, each one array of pitch elements; except for D3Q19
 * contexts with fp16 / bf16 deviation storage and nx a multiple of 32 (both
 * schemes), whose populations 1..18 are interleaved in blocks of 32 sites (the 18
 * rows of 32 values of a block contiguous, 1152 bytes; site q in block q/32). */
lb_status lb_device_state(lb_ctx* ctx, void** dptr, size_t* bytes);

/* Launch form of the context's fused step kernel (Eq. 4 per site, one launch
 * per time step): a short description written into name (at most cap bytes,
 * NUL-terminated; name may be NULL), the CTA's column tile (tile_x x tile_y
 * sites), threads per CTA, dynamic shared memory per CTA, and the number of
 * CTAs per launch.  Any output pointer may be NULL. */
lb_status lb_kernel_info(const lb_ctx* ctx, char* name, size_t cap, int* tile_x, int* tile_y, int* threads,
                         size_t* smem, int* ctas);

/* ------------------------------------------------------------------------
 * Batched sweeps of independent D2Q9 drop runs (parameter sweeps of the
 * Sec. IV test problem).  Every instance has its own lattice size, T, kappa
 * and tau and one centred drop; all share a, b, the scheme and the storage.
 * One kernel launch advances every active instance by one time step (work
 * items = (instance, tile)); lb_batch_run_to_steady replays a CUDA graph of
 * `every` steps plus a float64 convergence check and retires instances whose
 * max_r |u(t) - u(t - every)| < tol (u of Eq. 3).  Tile shapes (32x8, 32x16,
 * 64x8) are chosen by lb_batch_autotune, which times each on the live state
 * and restores it.
 */
typedef struct lb_batch lb_batch;
typedef struct {
    int nx, ny;            /* lattice of the instance, >= 1 */
    double T, kappa, tau;  /* van der Waals temperature, gradient coefficient, relaxation time */
    double radius;         /* radius of its centred drop (lb_batch_init_drops); <= 0: no drop */
} lb_instance;

/* n in 1..4096 instances, each with at most 2^20 tiles of 32 x 8 sites (LB_EINVAL otherwise);
 * cuda_stream NULL => the batch creates its own stream. */
lb_status lb_batch_create(int scheme, int storage, double a, double b, int n, const lb_instance* inst,
                          void* cuda_stream, lb_batch** out);
lb_status lb_batch_destroy(lb_batch* batch);   /* NULL-safe */
/* f = f^eq of a tanh drop (same profile as lb_init_drops) in every instance; resets the run state. */
lb_status lb_batch_init_drops(lb_batch* batch, double width);
/* f = f^eq(rho, u) for instance k from host fields (u may be NULL). */
lb_status lb_batch_init_fields(lb_batch* batch, int k, const double* rho, const double* u);
/* Advance every active instance nsteps time steps. */
lb_status lb_batch_step(lb_batch* batch, int nsteps);
/* Time each tile variant for `steps` steps on a copy of the state and keep the fastest. */
lb_status lb_batch_autotune(lb_batch* batch, int steps, int* tile_x, int* tile_y);
/* Run until every instance is retired or max_steps: steps_out[k] = steps at retirement (-1: not
 * converged), status_out[k] = LB_OK (converged), LB_ETIMEOUT (not converged within max_steps) or
 * LB_EUNSTABLE (non-finite density).  every must be even; no instance retires before min_steps. */
lb_status lb_batch_run_to_steady(lb_batch* batch, double tol, int every, long long min_steps, long long max_steps,
                                 long long* steps_out, int* status_out, long long* total_steps);
/* Steady-state test against a reference, for storage whose rounding keeps max|u(t) - u(t - every)|
 * above any useful tol: instance k with umax_ref > 0 is converged once, for `hold` consecutive checks,
 * max|u| is within band * umax_ref of umax_ref and, if rho_max_ref > 0, the largest and smallest
 * densities are within tol_rho of rho_max_ref and rho_min_ref (bulk liquid and gas; these do not
 * change when rounding noise translates the drop, which the periodic lattice allows).  umax_ref = 0
 * restores the max|du| < tol test for k.  The paper defines no steady-state test (Sec. IV runs to a
 * fixed time); the reference is typically the float64 steady state, so runs in other storage formats
 * stop at equal accuracy.  LB_EINVAL for k out of range, umax_ref < 0 or a non-finite value.  Applies
 * to later lb_batch_run_to_steady calls. */
lb_status lb_batch_set_reference(lb_batch* batch, int k, double umax_ref, double rho_max_ref, double rho_min_ref);
/* Parameters of the reference test (defaults band 0.05, tol_rho 1e-3, hold 10); LB_EINVAL for a
 * negative band or tol_rho or hold < 1. */
lb_status lb_batch_set_band(lb_batch* batch, double band, double tol_rho, int hold);
/* Self-contained steady-state test for instances without a reference (the
 * paper defines no test; Sec. IV runs to a fixed time): an instance is steady
 * once, for `hold` consecutive checks, its max|u| changed by at most
 * rtol_u * max|u| and its max rho and min rho by at most tol_rho since the
 * previous check.  It needs no steady values known in advance, and its
 * thresholds can sit above the rounding floor of reduced storage, whose
 * max|u(t) - u(t - every)| never falls below ~1e-8.  rtol_u = 0 switches it off
 * (the max|u(t) - u(t - every)| < tol test of lb_batch_run_to_steady).  Resets
 * every instance's count of consecutive checks.  LB_EINVAL for negative or
 * non-finite thresholds or hold < 1. */
lb_status lb_batch_set_self_test(lb_batch* batch, double rtol_u, double tol_rho, int hold);
/* max|u(t) - u(t - every)|, max|u|, max rho and min rho of each instance at its last check (0 before
 * the first check; frozen at retirement).  Any output may be NULL.  Synchronises. */
lb_status lb_batch_last_check(lb_batch* batch, double* du, double* umax, double* rho_max, double* rho_min);
/* Host copies of rho (N) and u (2N) of instance k, and of its populations (9N, layout as lb_get_populations). */
lb_status lb_batch_fields(lb_batch* batch, int k, double* rho, double* u);
lb_status lb_batch_populations(lb_batch* batch, int k, double* f);
lb_status lb_batch_info(const lb_batch* batch, int* tile_x, int* tile_y, long long* sites, long long* steps);

/* ------------------------------------------------------------------------
 * Learned warm start (a build addition; the paper has no learned component).
 * A 4-layer fully convolutional network (periodic 3x3 convolutions, 5 -> 32
 * -> 32 -> 32 -> 3 channels, tanh between layers, fp16 weights with float32
 * accumulation) maps the planes (tanh-start density, T, kappa, tau, 10/R) of
 * a D2Q9 drop to its steady (density correction, 1000 u_x, 1000 u_y), so a
 * run can start from lb_init_fields(predicted rho, u) instead of the tanh
 * profile.  Training (forward, backward, MSE, Adam) runs in the library's
 * kernels.  Image arrays are float32, layout [sample][channel][y][x].
 * Parameters are packed as W_1 (32x5x3x3), b_1, W_2, b_2, W_3, b_3, W_4 (3x32x3x3), b_4.
 */
#define LB_WS_IN 5
#define LB_WS_HIDDEN 32
#define LB_WS_OUT 3
typedef struct lb_ws lb_ws;
lb_status lb_ws_create(int seed, void* cuda_stream, lb_ws** out);
lb_status lb_ws_destroy(lb_ws* ws);   /* NULL-safe */
lb_status lb_ws_num_params(const lb_ws* ws, long long* n);
lb_status lb_ws_set_params(lb_ws* ws, const float* params, size_t count);   /* resets the Adam state */
lb_status lb_ws_get_params(lb_ws* ws, float* params, size_t count);
/* y (n x 3 x H x W) = network(x (n x 5 x H x W)).  At most 65535 samples per call (and per
 * training minibatch); more is LB_EINVAL. */
lb_status lb_ws_forward(lb_ws* ws, const float* x, int n, int H, int W, float* y);
/* Prediction for one drop (x: 5 x H x W) averaged over the symmetries of the periodic lattice
 * that fix the domain centre (reflections about W/2 and H/2, and the transpose when H == W), with
 * the velocity channels transformed as a vector: the result has the symmetry of the input. */
lb_status lb_ws_predict_sym(lb_ws* ws, const float* x, int H, int W, float* y);
/* Mean squared error of network(x) against t and its parameter gradients (packed; may be NULL). */
lb_status lb_ws_loss_grad(lb_ws* ws, const float* x, const float* t, int n, int H, int W, double* loss,
                          float* grads);
/* Adam (beta 0.9, 0.999) on minibatches of `batch` samples, reshuffled every epoch;
 * loss_history[e] = mean minibatch loss of epoch e (may be NULL). */
lb_status lb_ws_train(lb_ws* ws, const float* x, const float* t, int n, int H, int W, int epochs, int batch,
                      float lr, int seed, double* loss_history);
/* Input planes of one drop, and the decoding of a prediction into rho (N) and u (2N); decoding
 * keeps the mass of the tanh start (the mass residual of the predicted density correction is
 * removed with weight 1 - 4c^2, c the normalised tanh density, i.e. inside the interface). */
lb_status lb_ws_features(int nx, int ny, const double* rho_tanh, double rho_l, double rho_g, double T, double kappa,
                         double tau, double R, float* x);
lb_status lb_ws_decode(int nx, int ny, const double* rho_tanh, double rho_l, double rho_g, const float* y,
                       double* rho, double* u);

/* 3D variant for D3Q19 drops: the same network with periodic 3x3x3 convolutions (5 -> 32 -> 32 ->
 * 32 -> 4 channels); outputs (density correction, 1000 u_x, 1000 u_y, 1000 u_z).  Volumes are
 * float32 [sample][channel][z][y][x]; W_l packed as [C_out][C_in][3][3][3].  The input features are
 * those of lb_ws_features, which works site by site (call it with ny * nz as ny).  Same call
 * conventions and errors as the 2D functions (with samples x depth at most 65535 per call and per
 * minibatch); lb_ws3_predict_sym averages over the eight axis
 * reflections that fix the centre of the box (velocity components change sign accordingly). */
#define LB_WS3_OUT 4
typedef struct lb_ws3 lb_ws3;
lb_status lb_ws3_create(int seed, void* cuda_stream, lb_ws3** out);
lb_status lb_ws3_destroy(lb_ws3* ws);   /* NULL-safe */
lb_status lb_ws3_num_params(const lb_ws3* ws, long long* n);
lb_status lb_ws3_set_params(lb_ws3* ws, const float* params, size_t count);
lb_status lb_ws3_get_params(lb_ws3* ws, float* params, size_t count);
lb_status lb_ws3_forward(lb_ws3* ws, const float* x, int n, int D, int H, int W, float* y);
lb_status lb_ws3_loss_grad(lb_ws3* ws, const float* x, const float* t, int n, int D, int H, int W, double* loss,
                           float* grads);
lb_status lb_ws3_train(lb_ws3* ws, const float* x, const float* t, int n, int D, int H, int W, int epochs, int batch,
                       float lr, int seed, double* loss_history);
lb_status lb_ws3_predict_sym(lb_ws3* ws, const float* x, int D, int H, int W, float* y);
/* rho = rho_tanh + (rho_l - rho_g) * (y_0 minus its mass residual spread over the interface);
 * u (3N, SoA) = 1e-3 y_{1..3}. */
lb_status lb_ws3_decode(int nx, int ny, int nz, const double* rho_tanh, double rho_l, double rho_g, const float* y,
                        double* rho, double* u);

/* ------------------------------------------------------------------------
 * Allocation-free reductions.  The paper has no counterpart: this is a
 * library service for callers that cannot allocate device memory when they
 * need the numbers, e.g. an application whose allocator has already reserved
 * the device memory it may use, or a stepping loop that must not pay for
 * cudaMalloc/cudaFree (which can synchronise the device) or risk running out
 * of memory mid-run.
 *
 * lb_field_stats_noalloc computes the same float64 reductions as
 * lb_stats_get, but from caller-provided device fields, writing 8 doubles to
 * the caller's device buffer out: {mass, momentum x, y, z, max|u|, max|v|,
 * min rho, max rho} (momentum components beyond dim are 0).
 *   rho: n doubles; u, v: dim*n doubles (component-major, as lb_fields);
 *   all device pointers owned by the caller; dim in 1..3;
 *   1 <= n <= LB_NOALLOC_MAX_SITES, larger n returns LB_EINVAL;
 *   asynchronous on cuda_stream (a cudaStream_t, NULL = legacy stream).
 * It calls no cudaMalloc/cudaFree and no allocating routine: its per-block
 * partial sums live in a file-scope device array of LB_NOALLOC_MAX_BLOCKS*8
 * doubles (256 KiB), present on every GPU that loads the library until the
 * process exits.  The first call on a device looks up that array's address
 * (cudaGetSymbolAddress) with the device current; make that first call before
 * any stream capture.  All calls share the array; each call rewrites the
 * partials it reads, but calls whose kernels overlap on the GPU (other
 * streams, other host threads) race on it.
 */
#define LB_NOALLOC_MAX_BLOCKS 4096
#define LB_NOALLOC_SITES_PER_BLOCK 4096
#define LB_NOALLOC_MAX_SITES ((long long)LB_NOALLOC_MAX_BLOCKS * LB_NOALLOC_SITES_PER_BLOCK)
lb_status lb_field_stats_noalloc(const double* rho, const double* u, const double* v, int dim, long long n,
                                 double* out, void* cuda_stream);

/* ---- D3Q19 work list (host-only inspection helper; no counterpart in the paper) ----
 *
 * lb_work_list returns the CTA work list that lb_create builds for the D3Q19
 * step (a lattice split into column tiles of tile_x x tile_y sites and z chunks):
 * 4 ints (x0, y0, z0, z1) per CTA, in launch order, for a GPU with `sms` SMs and
 * `ctas_per_sm` resident CTAs of the step kernel per SM (2 for the 32-bit kernels
 * on a GB300, tiles 32 x 8; float64: tiles 32 x 4).  *count receives the number
 * of CTAs; if out is not NULL, the first min(count, capacity) entries are written
 * to it (caller-owned, 4 * capacity ints).  Runs on the host only (no CUDA call).
 * Non-positive sizes, more than 2^31 - 1 sites or a NULL count return LB_EINVAL. */
lb_status lb_work_list(int sms, int ctas_per_sm, int nx, int ny, int nz, int tile_x, int tile_y, int* out,
                       int capacity, int* count);

/* ---- FMA rate (measurement helper; no counterpart in the paper) --------------
 *
 * lb_fma_peak measures the fused multiply-add rate of the current GPU, the
 * denominator of the ALU roofline of the step kernels (the float64 step is
 * bound by the FP64 units rather than by HBM).  precision: 0 = float64,
 * 1 = float32.  It launches 4 CTAs of 256 threads per SM; every thread runs 8
 * independent chains of iters FMAs each.  The launch is timed with CUDA
 * events on the legacy default stream and the call returns after it, with
 * the rate in TFLOP/s (2 flops per FMA) in *tflops.  A warm-up launch of at
 * most 64 iterations precedes it.  It allocates and frees one element of
 * device memory.  iters outside [1, 2^24], another precision or a NULL tflops
 * return LB_EINVAL; a CUDA failure returns LB_ECUDA.  Pick iters so that the
 * launch runs for milliseconds (float64 ~4000, float32 ~2e5 on a GB300). */
lb_status lb_fma_peak(int precision, int iters, double* tflops);

/* ---- Binary fluid (D2Q9, D3Q19) -------------------------------------------
 *
 * The paper states (Sec. I) that its analysis applies equally to other
 * multiphase systems solved by the free-energy method, binary fluids among
 * them, and prints no equations for them.  This context runs the reading
 * that carries the liquid-gas construction over to a symmetric binary fluid
 * with an order parameter phi (the conserved concentration difference):
 *   free energy   psi = rho/3 ln rho + A/2 phi^2 + B/4 phi^4 + kappa/2 |grad phi|^2
 *                 (A < 0 < B: bulk phases phi = +-sqrt(-A/B));
 *   mu            = A phi + B phi^3 - kappa lap(phi);
 *   p0            = rho/3 + A/2 phi^2 + 3B/4 phi^4;
 *   f^eq          Eqs. 5, 6 with this p0, w^t kappa phi lap(phi) and
 *                 w^ab kappa d_a phi d_b phi (optimum weights of Sec. VIII),
 *                 lambda = 0 (c_s^2 = dp0/drho = 1/3);
 *   g^eq          sum g = phi, sum g e = phi u, sum g e_a e_b = Gamma mu d_ab
 *                 + phi u_a u_b, from the same weights (w^p for the mu term);
 *   relaxation    f with tau (BGK, Eq. 4), g with tau_phi (mobility
 *                 Gamma (tau_phi - 1/2)), both pushed to r + e_i;
 *   forcing       (LB_SCHEME_FORCING, Sec. VI) the M terms leave f^eq and act
 *                 as the body force of Eq. 28 with M_ab = kappa d_a phi d_b phi,
 *                 F_i of Eq. 27, and g^eq takes the fluid velocity
 *                 v = u + g/(2 rho) of Eq. 40 in place of u.
 * Stencils: the gradient and Laplacian of phi by Eqs. 10 and 11 at the
 * optimum (B = 1/12, D = 1/6), the force stencil with F = 1/12; in 3D
 * Eq. 29 with A = 1/6, B = 1/12, C = 1/3, D = 1/6 and the weights of Eq. 31.
 * Storage: LB_F64 (float64 arithmetic), LB_F32 (float32 arithmetic), or for
 * D2Q9 with an even nx LB_F16DEV (float32 arithmetic; f_0 and g_0 stored in
 * float32, f_i - w_i p_ref and g_i (i >= 1) in fp16, p_ref = p0 of a bulk
 * phase at rho = 1: 1/3 + A^2 / (4 B) for A < 0 < B, else 1/3).
 * Populations exchanged with the host: float64 [i][z][y][x] for f and for g,
 * i in the paper's order (Sec. II, Sec. VII), after streaming.  Conventions otherwise as
 * above (caller-owned host arrays, status codes, sticky device errors). */
typedef struct lb_binary lb_binary;

typedef struct {
    int lattice;          /* lb_lattice: LB_D2Q9 or LB_D3Q19 (Sec. VII weights, reading R7 for forcing) */
    int nx, ny, nz;       /* sites per direction, >= 1 (periodic); nz = 1 for D2Q9 */
    double A, B;          /* free-energy coefficients: A < 0 < B */
    double kappa;         /* gradient coefficient, >= 0 */
    double Gamma;         /* mobility coefficient of g^eq, > 0 */
    double tau;           /* relaxation time of f, > 1/2 */
    double tau_phi;       /* relaxation time of g, > 1/2 */
    int scheme;           /* lb_scheme */
    int storage;          /* LB_F64, LB_F32, or LB_F16DEV (D2Q9, even nx) */
} lb_binary_params;

typedef struct {
    double mass;          /* sum rho */
    double phi_total;     /* sum phi */
    double momentum[3];   /* sum rho u (the z component 0 for D2Q9) */
    double max_u;         /* max |u| (Eq. 3) */
    double max_v;         /* max |v| (Eq. 40 in the forcing scheme; = max_u otherwise) */
    double min_phi, max_phi;
    long long step;       /* steps taken since the last initialisation */
    int status;           /* 0, or LB_EUNSTABLE once a density became non-finite or non-positive */
} lb_binary_stats;

/* Creates a context: validates the parameters (LB_EINVAL), allocates two
 * population sets (f and g, double-buffered) on the device and returns it in
 * *out.  stream: the cudaStream_t to queue work on (NULL = the legacy default
 * stream); graphs of 64 steps are captured on a private stream and launched
 * on it. */
lb_status lb_binary_create(const lb_binary_params* p, void* stream, lb_binary** out);
lb_status lb_binary_destroy(lb_binary* ctx);
/* f = f^eq, g = g^eq of host fields rho [N], phi [N] and u [D][N] (NULL: u = 0),
 * stencils of phi taken on the device (the oracle's initial state); resets the
 * step counter.  rho must be positive and finite (LB_EINVAL otherwise). */
lb_status lb_binary_init_fields(lb_binary* ctx, const double* rho, const double* phi, const double* u);
/* Replaces / reads the populations: host f [Q][N] and g [Q][N], float64 (rounded
 * to float32 for LB_F32 storage).  set resets the step counter. */
lb_status lb_binary_set_populations(lb_binary* ctx, const double* f, const double* g);
lb_status lb_binary_get_populations(lb_binary* ctx, double* f, double* g);
/* nsteps steps (D2Q9: one fused kernel launch each; D3Q19: a phi pass and the
 * fused step; CUDA-graph replay on long runs). */
lb_status lb_binary_step(lb_binary* ctx, int nsteps);
lb_status lb_binary_synchronize(lb_binary* ctx);
/* Host float64 fields of the current state; any pointer may be NULL.
 * rho [N], phi [N], u [D][N] (Eq. 3), v [D][N] (Eq. 40; = u in the equilibrium
 * scheme), mu [N]. */
lb_status lb_binary_fields(lb_binary* ctx, double* rho, double* phi, double* u, double* v, double* mu);
/* Totals and extremes of the current state: the float64 fields of
 * lb_binary_fields (computed on the device), summed in site order on the host;
 * allocates (2 + 2 D) N doubles of host memory per call.  Returns
 * LB_EUNSTABLE (with out filled) once a density became non-finite. */
lb_status lb_binary_stats_get(lb_binary* ctx, lb_binary_stats* out);

#ifdef __cplusplus
}
#endif

#endif /* LB_H */
