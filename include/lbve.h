/*
 * lbve.h -- C ABI of the GB300 (sm_103a) hybrid lattice-Boltzmann library for the integral nonlinear
 * Maxwell fluid of Papenkort & Voigtmann, "Lattice Boltzmann simulations of a viscoelastic
 * shear-thinning fluid" (arXiv:1504.06123).
 *
 * Every function is extern "C", takes plain pointers and sizes, returns an int status (LBVE_OK = 0 or
 * a negative LBVE_E* code) and never lets a C++ exception cross it.  Device work is enqueued on the
 * CUDA stream passed as `void* stream` (NULL = the legacy default stream); calls that return data
 * to host memory synchronise that stream first.  A handle is not thread-safe: use one handle per host
 * thread.
 *
 * Conventions (all arrays):
 *   - lattice units dt = dx = 1;
 *   - node index n = x + nx*(y + ny*z), x fastest; x is periodic; walls (half-way bounce-back) at
 *     y = -1/2 and ny-1/2, and, for a D3Q19 duct, at z = -1/2 and nz-1/2;
 *   - kappa[a][b] = d v_a / d x_b (kappa = (grad v)^T, Sec. I), d*d components, row-major;
 *   - sigma (symmetric) components: 2D xx, yy, xy; 3D xx, yy, zz, xy, xz, yz.
 */
#ifndef LBVE_H
#define LBVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------------- */
#define LBVE_OK           0
#define LBVE_EINVAL      -1  /* an argument is out of range; nothing was changed */
#define LBVE_ENOMEM      -2  /* device memory could not be allocated */
#define LBVE_ECUDA       -3  /* a CUDA call or kernel launch failed (see lbve_last_cuda_error) */
#define LBVE_ENONFINITE  -4  /* a NaN or Inf appeared in the state */
#define LBVE_ESTATE      -6  /* the call does not fit the handle's state */
#define LBVE_ENOSUPPORT  -7  /* a valid combination this library does not implement */
#define LBVE_ETOOBIG     -8  /* request larger than the fixed device buffer of lbve_fields_host_fixed */

/* ---- enumerations ---------------------------------------------------------------------------- */
#define LBVE_D2Q9   9    /* planar channel, Sec. III velocity set */
#define LBVE_D3Q19 19    /* square duct: the three-dimensional form of the Sec. III scheme */

#define LBVE_F32 0       /* populations / history stored in float */
#define LBVE_F64 1       /* populations / history stored in double */
#define LBVE_BF16 2      /* reserved: plain bfloat16 history is not built (its 2^-9 rounding, identical at
                            every point of a steady flow, cannot meet 1e-3); use LBVE_S16 */
#define LBVE_S16 3       /* precision variant of the history: 16-bit block-scaled storage (d*d int16
                            mantissas + one shared power-of-two exponent per vector) of kappa and of
                            Q = E(t_b, t') in a per-node FP32 frame R = E(t, t_b) re-based every 32
                            steps; FP32 arithmetic */

#define LBVE_FORM_P 0     /* history form P: every point keeps X = E(t,t') - 1, advanced in place every step by
                             the left factor exp(kappa(t-1)) of Eq. (eeval), and its kappa (16-bit storage:
                             the frame form described at LBVE_S16) */
#define LBVE_FORM_F 1     /* history form F, the paper's factor storage (Sec. III): every point keeps, written
                             once, its factor deviation F - 1 -- exp(kappa(t')) - 1, or for a merged point the
                             product of the two merged factors, newer on the left -- and its rate of strain
                             kappa + kappa^T (averaged on merge); every step re-forms E(t,t') as the ordered
                             product of the factors from the newest point on (Eq. eeval).  Storage LBVE_F32,
                             LBVE_F64 or LBVE_S16 (16-bit block-scaled F - 1 and rate of strain, FP32
                             arithmetic); the sweep only reads the history.  Not with LBVE_MODEL_WM, nor for
                             differentiation (LBVE_ENOSUPPORT) */

#define LBVE_TRACE_FULL 0 /* Eq. (bodyforce) with the density source d_t(delta rho) as written */
#define LBVE_TRACE_NONE 1 /* both d_t(delta rho) terms dropped, rho = sum n (channel simplification) */

#define LBVE_MODEL_NLM  0 /* integral nonlinear Maxwell model: Eq. (gitt) with the modulus of Eq. (nlmax) */
#define LBVE_MODEL_INLM 1 /* instantaneous nlM, Eq. (inlM) of Sec. IV read as a stress / strain-rate law at
                             time t: sigma_struc(t) = G_inf sum_{n>=1} tau_M^n d^(n)[kappa(t)],
                             tau_M = (1/tau + gammadot(t)/gamma_c)^-1.  No history is kept (hist_C, hist_B
                             are checked but unused).  The series is summed until two consecutive terms
                             are below 1e-18 of the sum; where that takes more than 1000 terms or the
                             terms overflow (no steady state, e.g. strong extension) sigma_struc is NaN
                             and lbve_fields reports LBVE_ENONFINITE */
#define LBVE_MODEL_WM   2 /* White-Metzner form named in Sec. II: the second exponential of Eq. (nlmax)
                             takes the strain accumulated between t' and t, sum_{s=t'}^{t-1} gammadot(s),
                             in place of (t - t') gammadot(t').  History storage LBVE_F32 or LBVE_F64 */

#define LBVE_X_PERIODIC 0 /* x (the flow axis) plainly periodic; the flow is driven by the body force g */
#define LBVE_X_PRESSURE 1 /* pressure-step boundary along x (Sec. III: the generalised periodic boundary that
                             fixes a constant pressure step between inlet and outlet of the periodic lattice).
                             Populations crossing the seam stream from ghost images of the opposite boundary
                             node: its post-collision non-equilibrium part on an equilibrium at the ghost
                             density and the node's velocity.  The ghosts sit on the linear profile of a
                             pressure drop dp per period (nx spacings) around rho0:
                             rho_in/out = rho0 +- (dp / c_s^2) (nx + 1) / (2 nx).  Equivalent, in the
                             incompressible limit, to g = dp / (rho0 nx); it also fixes the mean density */

#define LBVE_FIELD_RHO   1u  /* [N]        hydrodynamic density of Eq. (hydrofields) */
#define LBVE_FIELD_U     2u  /* [d][N]     velocity u = (sum c n + f/2)/rho */
#define LBVE_FIELD_SIGMA 4u  /* [nsig][N]  sigma_struc of Eq. (gitt) */
#define LBVE_FIELD_KAPPA 8u  /* [d*d][N]   velocity gradient of the last step */
#define LBVE_FIELD_N1   16u  /* [N]        first normal-stress difference sigma_xx - sigma_yy */

/* ---- channel description (problem statement of Sec. III/IV) ----------------------------------- */
typedef struct {
    int32_t lattice;          /* LBVE_D2Q9 (nz must be 1) or LBVE_D3Q19 */
    int32_t nx, ny, nz;       /* fluid nodes; ny >= 2 (walled); a duct needs nz >= 2 */
    int32_t wall_z;           /* D3Q19: 1 = walls in z as well (square duct), 0 = z periodic */
    double  tau_lb;           /* BGK relaxation time (> 1/2); eta_N = rho0 c_s^2 (tau_lb - 1/2) */
    double  rho0;             /* reference density (populations are stored as n_i - w_i rho0) */
    double  G_inf;            /* plateau modulus G_inf of Eq. (nlmax) (>= 0) */
    double  tau;              /* structural relaxation time tau of Eq. (nlmax), in steps (> 0) */
    double  gamma_c;          /* strain scale gamma_c of Eq. (nlmax) (> 0; +INFINITY = UCM limit) */
    double  g[3];             /* body force per unit mass; force density f = rho0 g (Sec. IV driving) */
    int32_t hist_C;           /* points per history block C (Sec. III; the paper uses 128), >= 4 */
    int32_t hist_B;           /* number of blocks B, 1..16; B*C points span about C (2^B - 1) steps */
    int32_t hist_storage;     /* LBVE_F32 | LBVE_F64 | LBVE_S16: storage and arithmetic of the history */
    int32_t pop_precision;    /* LBVE_F32 | LBVE_F64: storage and collision arithmetic of the populations
                                 (independent of hist_storage; node fields are always double) */
    int32_t trace_coupling;   /* LBVE_TRACE_FULL | LBVE_TRACE_NONE */
    int32_t model;            /* LBVE_MODEL_NLM (0) | LBVE_MODEL_INLM | LBVE_MODEL_WM; the same for every
                                 channel of a batch.  LBVE_MODEL_WM with LBVE_S16, and differentiation
                                 (lbve_create_tangent / lbve_create_adjoint) of any model but
                                 LBVE_MODEL_NLM, return LBVE_ENOSUPPORT */
    int32_t x_boundary;       /* LBVE_X_PERIODIC (0) | LBVE_X_PRESSURE; per channel */
    double  dp;               /* LBVE_X_PRESSURE: pressure drop per period along x (lattice units, finite);
                                 ignored for LBVE_X_PERIODIC.  Differentiation of a channel with
                                 LBVE_X_PRESSURE returns LBVE_ENOSUPPORT */
    int32_t hist_form;        /* LBVE_FORM_P (0) | LBVE_FORM_F: how the history stores its points (Sec. III);
                                 the same for every channel of a batch */
} lbve_channel_desc;

typedef struct lbve lbve_t;   /* opaque; owns every device buffer of one channel or of a batch */

/*
 * Create a channel on the current CUDA device: fluid at rest, n_i = w_i rho_init(n) (rho0 where
 * rho_init is NULL; otherwise a host array of N doubles, copied), every history point at rest
 * (E = 1, kappa = 0).  The history grid of Sec. III starts full, so the first steps already run the
 * block merges.  Device memory: 2 Q N populations, (d^2 + d^2) (B C + ... ) N history words and a few
 * fields; sizes in lbve_memory_bytes.  *out is NULL on failure.
 * Errors: EINVAL (bad sizes or parameters, including a shear-wave speed sqrt(G_inf/rho0) > 0.5 that
 * the explicit stress coupling cannot carry), ENOMEM, ECUDA, ENOSUPPORT.
 */
int lbve_create(const lbve_channel_desc* desc, const double* rho_init, lbve_t** out);

/*
 * Create a batch of n_channels independent channels (for instance the paper's channels of different
 * width, Sec. IV) advanced together by every lbve_step: one set of launches for all channels.  Each
 * channel has its own sizes, G_inf, tau, gamma_c, g, tau_lb and trace coupling; the lattice, the history
 * grid (hist_C, hist_B), the precisions and rho0 must be the same for all.  Channels are stored one
 * after the other (node order x fastest within each); lbve_channel_nodes gives a channel's range in
 * the node arrays of lbve_fields.  rho_init: NULL or the initial densities of all nodes in that order.
 * Errors as lbve_create; EINVAL also when the shared settings differ or n_channels is outside 1..65536.
 */
int lbve_create_batch(const lbve_channel_desc* descs, int32_t n_channels, const double* rho_init, lbve_t** out);

/*
 * Device-memory provider of a handle (the ownership rule of the boundary: the handle owns its device state,
 * taken from the caller's allocator -- for instance PyTorch's caching allocator -- or from cudaMalloc; the
 * paper has no counterpart).  alloc returns device memory of at least `bytes` on the current device,
 * aligned to 256 bytes, or NULL; free returns it.  `stream` is the stream the memory is first used on (the
 * legacy default stream, NULL, for the handle's own buffers, which the handle frees only after a device
 * synchronisation); ctx is passed through.  Both are called from the host thread that calls the library.
 */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void (*free)(void* ptr, void* stream, void* ctx);
    void* ctx;
} lbve_allocator;

/*
 * lbve_create_batch (n_channels = 1: lbve_create) with every device buffer of the handle and of its later
 * calls (probe buffers, field staging, checkpoints) taken from `allocator` (NULL, or alloc == NULL: cudaMalloc).
 * ENOMEM when the allocator returns NULL or memory not aligned to 256 bytes; whatever was allocated is freed
 * again through the allocator, and *out is NULL.  EINVAL when alloc is set and free is not.
 */
int lbve_create_ex(const lbve_channel_desc* descs, int32_t n_channels, const double* rho_init,
                   const lbve_allocator* allocator, lbve_t** out);

/* First node and node count of a channel (0 for a handle made by lbve_create). */
int lbve_channel_nodes(const lbve_t* h, int32_t channel, int64_t* offset, int64_t* count);

/* Free every device buffer of the handle (synchronises the device).  NULL is ignored. */
void lbve_destroy(lbve_t* h);

/*
 * Replace the body force of one channel (channel = -1: all) -- startup / cessation, Sec. IV.  Stream
 * ordered: steps enqueued earlier on `stream` still use the old value, later steps the new one.
 */
int lbve_set_force(lbve_t* h, int32_t channel, const double g[3], void* stream);

/*
 * Replace the pressure drop per period dp of the pressure-step boundary (LBVE_X_PRESSURE) of one channel
 * (-1: all) -- startup / cessation with the pressure drive of Sec. III-IV.  Ordered like lbve_set_force.
 * ESTATE when a selected channel was created with LBVE_X_PERIODIC; EINVAL for a non-finite dp.
 */
int lbve_set_pressure_step(lbve_t* h, int32_t channel, double dp, void* stream);

/* Replace G_inf, tau, gamma_c of Eq. (nlmax) for one channel (-1: all); ordered like lbve_set_force. */
int lbve_set_params(lbve_t* h, int32_t channel, double G_inf, double tau, double gamma_c, void* stream);

/*
 * Advance n_steps >= 0 full hybrid steps (Sec. III): moments -> kappa by finite differences -> stress
 * history (advance E, insert/merge per the quasi-logarithmic grid, -d_t'B, modulus of Eq. (nlmax),
 * trapezoidal sum of Eq. (gitt)) -> trace split, density source, BGK collision with the forcing of
 * Eq. (bodyforce) -> streaming with bounce-back.  Asynchronous on `stream`.  Runs of 16 steps are
 * replayed from a CUDA graph captured on first use (unless lbve_profile is on).
 */
int lbve_step(lbve_t* h, int64_t n_steps, void* stream);

/* Number of completed steps (host-side counter; no synchronisation). */
int lbve_get_time(const lbve_t* h, int64_t* t);

/*
 * Write the fields selected by field_mask (LBVE_FIELD_*) of the last completed step as doubles into
 * dst, one block per field in increasing bit order, each block component-major ([comp][N]).
 * dst_is_device = 1: dst is device memory (stream-ordered, asynchronous); 0: host memory (the call
 * synchronises `stream`).  The caller owns dst; its size must be lbve_fields_count(h, mask) doubles.
 * Returns ENONFINITE (after copying) when a copied value is NaN or Inf and dst is host memory (a
 * device-side flag set by the copy kernel).
 */
int lbve_fields(lbve_t* h, uint32_t field_mask, double* dst, int32_t dst_is_device, void* stream);

/*
 * lbve_fields for one channel of a batch and in a chosen precision: the fields selected by field_mask of the
 * nodes of `channel` (-1: all nodes, as lbve_fields), one block per field in increasing bit order, each block
 * component-major ([comp][nodes of the channel], node order of lbve_channel_nodes), written as dst_dtype values
 * (LBVE_F64: double; LBVE_F32: float, each value rounded once from the double field).  dst holds
 * (components of the selected fields) x (nodes of the channel) values; device or host memory as in
 * lbve_fields, with the same synchronisation and the same ENONFINITE report for host destinations.
 * Errors: EINVAL (channel outside -1 .. n_channels-1, another dst_dtype, bad mask), ENOSUPPORT for tangent
 * handles (lbve_tangent_fields).
 */
int lbve_fields_ex(lbve_t* h, int32_t channel, uint32_t field_mask, void* dst, int32_t dst_is_device,
                   int32_t dst_dtype, void* stream);

/* Number of doubles lbve_fields writes for field_mask. */
int lbve_fields_count(const lbve_t* h, uint32_t field_mask, size_t* count);

/*
 * Probe time series (Sec. IV: the transients of Figs. Qall, QT and figtau are the velocity, shear stress
 * and normal-stress difference at one wall distance y/H of each channel, recorded through startup and
 * cessation).  Set n_probes node indices (host array `nodes`, the node numbering of lbve_fields; for a
 * batch the batch-wide index, channel offset from lbve_channel_nodes plus the in-channel index); from
 * then on every step whose completed-step count t (lbve_get_time after the step) is a multiple of
 * `every` appends one record, written on the device by a small kernel launched after each step (and
 * captured in the step graphs), so recording needs no host round trip.  A record is
 *   [t, then for each probe: rho, u[d], sigma[nsig]]      (1 + n_probes (1 + d + nsig) doubles),
 * the same values lbve_fields returns at step t.  The handle owns a device buffer of `capacity` records;
 * records past it are counted but not stored.  Setting probes clears earlier records; n_probes = 0
 * removes the recorder.  Synchronises the device (the step graphs are re-captured).
 * Errors: EINVAL (a node index outside 0..N-1, n_probes < 0 or > 65536, every < 1, capacity < 1 when
 * n_probes > 0), ENOMEM, ENOSUPPORT for tangent and adjoint handles.
 */
int lbve_set_probes(lbve_t* h, int32_t n_probes, const int64_t* nodes, int32_t every, int64_t capacity);

/*
 * Copy the stored probe records to host memory `dst_host` (room for `capacity` records of the layout
 * above, caller-owned).  *n_stored = records copied (at most capacity), *n_total = records taken since
 * lbve_set_probes (n_total > n_stored means the buffer overflowed).  Synchronises `stream`.
 * Errors: EINVAL (no recorder set), ECUDA.
 */
int lbve_probe_read(lbve_t* h, double* dst_host, int64_t* n_stored, int64_t* n_total, void* stream);

/*
 * Test hook for the stress history alone (steps of Sec. III on a prescribed gradient): advance every
 * node's history by one step with kappa(t) taken from kappa_dev (device, [d*d][N] doubles) instead of
 * the finite differences of the flow, and write sigma_struc(t) to sigma_dev (device, [nsig][N]
 * doubles).  Uses and advances the same history and step counter as lbve_step.  Asynchronous.
 */
int lbve_history_apply(lbve_t* h, const double* kappa_dev, double* sigma_dev, void* stream);

/*
 * Mass bookkeeping of the density source (Sec. III): *sum_n = total of all populations, *sum_drho =
 * total of delta rho(t-1) = -tr sigma(t-1)/(d c_s^2).  With LBVE_TRACE_FULL their difference is
 * conserved by the scheme.  Synchronises `stream`.
 */
int lbve_mass(lbve_t* h, double* sum_n, double* sum_drho, void* stream);

/*
 * The retained history points after step t >= 0 for blocks of C points and B blocks (identical at
 * every node): their creation times t' newest first and trapezoidal weights.  tp_out and w_out must
 * hold B*C entries; *n_out receives the count.  Pure host function (no device, no handle).
 */
int lbve_schedule(int32_t C, int32_t B, int64_t t, int64_t* tp_out, double* w_out, int32_t* n_out);

/*
 * Differentiation: a channel whose every state value also carries its derivatives with respect to the
 * four model parameters theta = (G_inf, tau, gamma_c, g_x) -- the tangent-linear model of the same
 * hybrid step (Sec. III), in double precision, one channel.  lbve_step, lbve_fields, lbve_set_force,
 * lbve_set_params and lbve_destroy work on it as on any handle (derivatives are taken at the current
 * parameter values; a later parameter change does not reset the accumulated derivatives).
 * lbve_tangent_fields writes d(field)/d(theta_k) for k = 0..3 to host memory: four consecutive blocks,
 * each in the layout of lbve_fields (lbve_fields_count(h, mask) doubles per block).  Synchronises.
 * ESTATE when h is not a tangent handle.
 */
int lbve_create_tangent(const lbve_channel_desc* desc, const double* rho_init, lbve_t** out);
int lbve_tangent_fields(lbve_t* h, uint32_t field_mask, double* dst_host, void* stream);

/*
 * Checkpoint / resume of the whole state of a handle: populations, history (and the frame of the 16-bit
 * form), node fields, step counter and per-channel parameters.  lbve_checkpoint_size gives the bytes of
 * the image; save writes it to dst (device memory if dst_is_device, else host memory), restore reads it
 * back into a handle created with the same descriptions.  Both synchronise `stream`.  Restore returns
 * EINVAL when the image does not match the handle.
 */
int lbve_checkpoint_size(lbve_t* h, size_t* bytes);
int lbve_checkpoint_save(lbve_t* h, void* dst, int32_t dst_is_device, void* stream);
int lbve_checkpoint_restore(lbve_t* h, const void* src, int32_t src_is_device, void* stream);

/*
 * Reverse mode (adjoint).  lbve_create_adjoint makes a channel (form P history; pop_precision and
 * hist_storage LBVE_F64 or LBVE_F32, ENOSUPPORT otherwise) that records a state image every checkpoint_every
 * steps while it is stepped from t = 0.  The replayed states are kept in the channel's own storage; the
 * adjoint itself, and dL/dtheta, are computed in FP64 (with FP32 storage the gradient is that of the FP32
 * trajectory).  lbve_backward then returns grad_out = dL/d(G_inf, tau, gamma_c, g_x) for a loss L
 * of the fields of the last completed step, given dL_du ([d][N], host) and dL_dsigma ([nsig][N], host):
 * it replays every segment from its image, keeps the per-step states of that segment, and runs the
 * adjoint of the hybrid step (collision and streaming, history commit and sweep, finite differences,
 * moments) backwards through it.  The handle's state is the same before and after the call; stepping
 * further and calling again is allowed.  ESTATE before the first step.  Synchronises `stream`.
 */
int lbve_create_adjoint(const lbve_channel_desc* desc, const double* rho_init, int32_t checkpoint_every,
                        lbve_t** out);
int lbve_backward(lbve_t* h, const double* dL_du, const double* dL_dsigma, double grad_out[4], void* stream);

/* Device bytes held by the handle (populations, history, fields). */
int lbve_memory_bytes(const lbve_t* h, size_t* bytes);

/*
 * Launch shape of the history sweep chosen at create by the autotuner: the number of slot chunks each
 * node's points are split into (tasks = node tiles x chunks), the number of persistent CTAs, and the task
 * mode (*cta_tasks = 0: a task is one warp's; 1: a task is one CTA's, its warps splitting the chunk;
 * 2, 16-bit form F only: balanced ranges -- every warp of the resident grid takes an equal run of the
 * tile-major sequence of (node tile, point), a tile being cut into at most *slot_chunks pieces).
 * The tuner times candidate shapes once per process for each (device, lattice, history storage and model,
 * history grid, padded node count); later handles of the same kind take the shape found then.
 * The shape fixes the order in which the trapezoidal sum of Eq. (gitt) is added up: results are bitwise
 * reproducible for a given shape, and differ in the last bits between shapes.
 */
int lbve_sweep_config(const lbve_t* h, int32_t* slot_chunks, int32_t* ctas, int32_t* cta_tasks);

/*
 * Replace the autotuned launch shape (for bitwise-reproducible runs across handles, whose autotuner may
 * choose differently): slot_chunks in 1 .. max(1, B*C/8), cta_tasks 0, 1 (only with an FP32 or FP64
 * history) or 2 (only with the 16-bit form F; slot_chunks is then set from the grid, and EINVAL if that
 * exceeds B*C/8).  Synchronises the device; the step graphs are re-captured.  EINVAL outside those ranges,
 * ENOSUPPORT for a handle without a history sweep (instantaneous model, tangent and adjoint handles).
 */
int lbve_set_sweep_config(lbve_t* h, int32_t slot_chunks, int32_t cta_tasks);

/*
 * Kernel timing for benchmarks: with enable = 1, every later lbve_step records a CUDA event pair on
 * its stream around each of its launches (moments, history, collide-stream).  lbve_profile_read waits
 * for the last event, returns the summed device milliseconds and launch counts per kernel in that
 * order (ms_out[3], launches_out[3]) and clears the record.  enable = 0 stops recording.
 */
int lbve_profile(lbve_t* h, int32_t enable);
int lbve_profile_read(lbve_t* h, double ms_out[3], int64_t launches_out[3]);

/*
 * lbve_fields with a host destination, for callers that must not allocate device memory once their set-up
 * is done.  (The paper has no counterpart: this is a library service.)  lbve_fields stages a host copy in
 * a device buffer that it allocates on first use and keeps; some callers cannot allow that allocation:
 * an application that has handed the whole GPU to a memory pool of its own, a service that runs with a
 * fixed device-memory budget, or a time-stepping loop in which an allocation (and the device-wide
 * synchronisation it implies) is not acceptable.  This variant allocates nothing: it stages through one
 * fixed device array of LBVE_FIXED_STAGING_DOUBLES doubles (16 MiB) that every GPU which loads the library
 * holds until the process exits.
 *
 * Same fields, layout and synchronisation as lbve_fields with dst_is_device = 0: dst is host memory of
 * lbve_fields_count(h, mask) doubles, owned by the caller; `stream` is synchronised before return.
 * Returns LBVE_ETOOBIG (nothing copied) when that count exceeds LBVE_FIXED_STAGING_DOUBLES, ENONFINITE
 * (after copying) when a copied value is NaN or Inf, EINVAL for bad arguments.
 * The first call on a device looks up the array's device address (once per device, on the current
 * device; again only if the device's CUDA context has been destroyed and re-made since, e.g. by
 * cudaDeviceReset); make that first call before any stream capture.  All calls on a device share the one array,
 * so calls that overlap on the GPU (other streams, other host threads) race with each other: serialise
 * them.  The non-finite flag kept in the array is cleared at the start of every call.
 */
#define LBVE_FIXED_STAGING_DOUBLES (1u << 21)
int lbve_fields_host_fixed(lbve_t* h, uint32_t field_mask, double* dst_host, void* stream);

/* Static description of a status code. */
const char* lbve_strerror(int status);

/* Text of the last CUDA error seen by this library in the calling thread ("" if none). */
const char* lbve_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBVE_H */
