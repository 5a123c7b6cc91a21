/*
 * kt.h -- C ABI of the GB300 (sm_103a) per-cell stiff thermochemistry integrator.
 *
 * The operation (Wang 2025, "The Kratos Framework ...", Sec. 2.2-2.3): every cell
 * carries species densities n^s (and, when the network has the energy equation, its
 * temperature T) and is advanced independently over a time dt by an implicit
 * ("semi-implicit", Sec. 2.2) solver with adaptive sub-steps.  Each Newton
 * iteration evaluates the modified-Arrhenius rates (Sec. 2.2.1), assembles the dense
 * species-and-temperature Jacobian (Eq. method-jacobian), LU-factorises the iteration
 * matrix with Crout's scaled row pivoting (Algorithm lu-decomp) and solves it.  The
 * result is post-processed (Sec. 2.2.3): negative densities are clipped and the
 * element totals of the initial state restored; failed cells are retried with a
 * smaller first step and reverted to their input if they fail again.
 *
 * Conventions
 *   - Every function returns 0 (KT_OK) or a negative KT_E* code; the message of the
 *     last failure on the calling thread is kt_last_error().
 *   - Cell arrays are structure-of-arrays: y[s * ncells + c] for species s of cell c,
 *     T[c], rho[c], all float64; status / counters are int32.
 *   - Device pointers must stay valid until the work on `stream` has reached them;
 *     streams are borrowed (a cudaStream_t cast to void*, NULL = legacy default).
 *   - Calls that take a stream are asynchronous unless stated otherwise.
 *   - Per-cell numerical failures are not call errors: they are reported in status[].
 */
#ifndef KT_H
#define KT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define KT_API __attribute__((visibility("default")))
#else
#define KT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define KT_OK 0
#define KT_EINVAL (-1)    /* bad argument */
#define KT_ENOMEM (-2)    /* host or device allocation failed */
#define KT_ECUDA (-3)     /* a CUDA runtime call failed */
#define KT_EPARSE (-4)    /* network file unreadable or malformed */
#define KT_ENETWORK (-5)  /* a reaction does not conserve every element */
#define KT_ETIMEOUT (-6)  /* a bounded device wait (TMA barrier) gave up */
#define KT_EUNSUPPORTED (-7) /* network size beyond what the kernels are built for */

/* per-cell status */
#define KT_STATUS_OK 0
#define KT_STATUS_RETRIED 1      /* first attempt failed, the retry succeeded */
#define KT_STATUS_REVERTED 2     /* both attempts failed: state reverted to the input */
#define KT_STATUS_NONFINITE 3    /* NaN / Inf in the input: cell left untouched */

/* forms of the iteration */
#define KT_FORM_FP64 0     /* full Newton, FP64 Jacobian and LU (the plain form) */
#define KT_FORM_FP32LU 1   /* simplified Newton: FP32 Jacobian + LU, FP64 residual/update */

/* Newton starting iterate */
#define KT_GUESS_PREV 0    /* the state at the start of the step (plain predictor) */
#define KT_GUESS_MLP 1     /* learned initial guess (needs kt_mlp_load) */
#define KT_GUESS_FULLSTEP 2 /* second half step starts from the full step's result
                               (same end time; differs by the local error only) */

/* one-step scheme of the sub-steps (the paper names a semi-implicit solver with
 * adaptive sub-steps, Sec. 2.2, without fixing it) */
#define KT_SCHEME_BE 0      /* backward Euler; error by step doubling (one step h vs two
                               of h/2, the two-half-step result kept); first order */
#define KT_SCHEME_TRBDF2 1  /* TR-BDF2 (Bank et al. 1985): a trapezoidal stage to
                               t + gamma h and a BDF2 stage to t + h, gamma = 2 - sqrt(2),
                               both solving y = r + d h f(y), d = gamma/2, with one
                               iteration matrix I - d h J per step; error estimated from
                               f at the three points, 2 C h (f_n/gamma - f_g/(gamma(1-gamma))
                               + f_{n+1}/(1-gamma)), C = (-3 gamma^2 + 4 gamma - 2)/(12(2-gamma));
                               h_new = h min(facmax, max(0.2, 0.9 err^(-1/3))); second
                               order.  The second stage starts from the first stage's
                               result whatever `guess` says; KT_GUESS_MLP is refused. */

/* storage of the FP32-LU lane-per-cell kernels under TR-BDF2 (kt_options.lane_variant) */
#define KT_LANE_AUTO 0      /* KT_LANE_LEAN where it applies */
#define KT_LANE_JCACHE 1    /* the FP32 Jacobian is kept beside the iteration matrix (a
                               rejected attempt re-uses it) and a failed FP32 solve is
                               redone in FP64 Newton from its start before h halves;
                               52 KB of shared memory per warp for 11 unknowns */
#define KT_LANE_LEAN 2      /* the iteration matrix I - d h J is assembled directly in
                               FP32 (no Jacobian copy), the step's start state and rate
                               stay in registers, and a failed FP32 solve halves h (no
                               FP64 rescue); 27 KB per warp for 11 unknowns, so twice as
                               many warps share an SM */

typedef struct kt_network kt_network;
typedef struct kt_state kt_state;
typedef struct kt_mlp kt_mlp;

/* Integration options.  Fill with kt_options_default() and override fields.
 * Sub-step control: one backward-Euler step of h and two of h/2 per attempt; the
 * weighted RMS of their difference with weights atol_i + rtol*max(|y_i|,|y2_i|)
 * must be <= 1; the next h is h*min(facmax, max(0.2, 0.9/sqrt(err))).  Newton on
 * each step stops when every |delta_i| <= newton_atol_frac*atol_i + newton_rtol*|y_i|
 * (temperature: newton_rtol*|T|) and fails after max_newton iterations (h halves).
 * The FP32-LU form also stops one iteration earlier when the contraction rate theta
 * of its simplified Newton iteration (< 1/2) predicts that the error left,
 * theta/(1-theta)*|delta_i|, is within newton_rtol*|y_i| for every component. */
typedef struct {
    double rtol;             /* relative error weight                          (1e-6) */
    double atol;             /* absolute error weight of every species         (1e-10) */
    double h_init;           /* first trial sub-step [s]                       (1e-6) */
    double h_min;            /* a sub-step below this fails the attempt [s]    (1e-30) */
    double newton_rtol;      /* Newton relative tolerance                      (1e-12) */
    double newton_atol_frac; /* Newton absolute tolerance as a fraction of atol (1e-2) */
    double facmax;           /* largest step growth per accepted step           (4) */
    double retry_h_factor;   /* retry's first step = h_init * retry_h_factor   (1e-3) */
    double retry_facmax;     /* retry's facmax                                  (2) */
    int max_substeps;        /* attempts (accepted + rejected) per integration (100000) */
    int max_newton;          /* Newton iterations per factorisation            (8) */
    int form;                /* KT_FORM_*                                       (FP64) */
    int guess;               /* KT_GUESS_*                                      (PREV) */
    int persistent;          /* 1: persistent kernel pulling cells from a device
                                work queue; 0: one cell per lane, one pass     (0) */
    int retry;               /* 1: retry failed cells once                      (1) */
    int atol_mode;           /* 0: atol absolute; 1: atol times the cell's
                                initial total of element 0                     (0) */
    int block_warps;         /* warps per block, 0 = automatic                   (0) */
    int blocks_per_sm;       /* persistent grid = blocks_per_sm x SMs, 0 = automatic (0) */
    int use_graph;           /* 1: kt_integrate replays a captured CUDA graph    (0) */
    int cells_per_warp;      /* 32: one cell per lane (networks with <= 16 unknowns);
                                1: one cell per warp (<= 96 unknowns); 0: automatic (0) */
    int schedule;            /* kt_integrate on a state with persistent = 1: 1 hands
                                out the cells with the most Newton iterations in the
                                previous call first (the state's n_newton counters;
                                zero after kt_state_create), 0 in index order.  The
                                order changes no result, only the load balance (0) */
    int scheme;              /* KT_SCHEME_*: the one-step scheme of each sub-step      (BE) */
    int lane_variant;        /* KT_LANE_*: storage of the FP32-LU lane-per-cell kernels
                                with TR-BDF2 (3 or 11 unknowns); ignored elsewhere (AUTO) */
    int reserved[2];
} kt_options;

/* Defaults listed above. */
KT_API int kt_options_default(kt_options *opts);

/* Load a reaction network from the plain-text format written by the package's
 * input generators ("kratos_network 1" header, species with molar mass, heat of
 * formation, heat capacity and element counts, reactions with up to three reactants
 * and products and modified-Arrhenius A, b, theta: k = A (T/t_ref)^b exp(-theta/T),
 * Sec. 2.2.1).  Optional sections before "end":
 *   cv_poly t_mid, then "cvp s a0..a4 b0..b4" per species: heat capacities
 *     cv_s(T) = sum_k a_k T^k below t_mid, sum_k b_k T^k above [J/(mol K)] (Sec. 4.2,
 *     NASA-style fits); C_V(T) = sum_s n0_s cv_s(T) with the cell's input composition;
 *   photo m, then "ph r sigma_r" m times: one-reactant photo-reactions (see
 *     kt_integrate_rad);
 *   rate_table nT T0 T1 nR rho0 rho1 m, then "tab r" and nR x nT values of ln k m times:
 *     tabulated rates (Sec. 2.2.1 item 3) on log-spaced nodes; each cell takes ln k
 *     linear in ln rho at its density (pre-processing, Sec. 2.2.2), then ln k linear in
 *     ln T between nodes (dk/dT from that slope), constant beyond the grid.
 * Every reaction must conserve every element (Eq. method-const-elem), else
 * KT_ENETWORK.  The caller owns *out and frees it with kt_network_free. */
KT_API int kt_network_load(const char *path, kt_network **out);

/* Sizes of a loaded network.  Any output pointer may be NULL. */
KT_API int kt_network_info(const kt_network *net, int *n_species, int *n_elements,
                    int *n_reactions, int *has_temperature);

KT_API void kt_network_free(kt_network *net);

/* Device state for ncells cells on the current CUDA device: what the thermochemistry
 * step keeps per cell (Sec. 2.2, Eq. method-ode-thermochem: the species number
 * densities, the temperature, the density), y [n_species][ncells], T, rho, plus the
 * status, the counters and the scratch of the integrate call.  The library owns every
 * buffer; free with kt_state_free.  ncells may be 0. */
KT_API int kt_state_create(const kt_network *net, int64_t ncells, kt_state **out);

/* Copy cell data into the state (host or device source, SoA float64): the cells'
 * state before the step, which the step pre-processes (Sec. 2.2.2).  rho may be
 * NULL (then 1).  Asynchronous on stream; host sources must stay valid until the
 * copy has run (pinned memory makes the copy truly asynchronous). */
KT_API int kt_state_upload(kt_state *st, const double *y, const double *T, const double *rho,
                    int src_is_device, void *cuda_stream);

/* Set the per-cell cost estimate that the longest-first queue order (opts->schedule)
 * reads: cost [ncells] int32 (host or device), e.g. the Newton counts of the previous
 * step of an operator-split simulation, or any estimate the caller has.  It is copied
 * into the state's n_newton counters, which every kt_integrate overwrites with the
 * counts it measured.  The order changes no result, only the load balance (a
 * scheduling aid of this library; the paper has no counterpart).  Asynchronous on
 * stream, same source rules as kt_state_upload. */
KT_API int kt_state_set_cost(kt_state *st, const int32_t *cost, int src_is_device, void *cuda_stream);

/* Advance every cell of the state by dt in place (asynchronous on stream): one
 * thermochemistry step of Sec. 2.2 per cell, i.e. pre-processing (Sec. 2.2.2), implicit
 * sub-steps with the rates and Jacobian of Sec. 2.2.1 factorised by Algorithm
 * lu-decomp, post-processing and failure handling (Sec. 2.2.3).  With
 * opts->use_graph the call (scratch reset + kernel) is captured once into a CUDA graph
 * on a private stream and replayed on `stream` while dt and *opts are unchanged. */
KT_API int kt_integrate(kt_state *st, double dt, const kt_options *opts, void *cuda_stream);

/* Copy results out (host or device destination): the cells' state after the step and
 * their status (Sec. 2.2.3: OK, retried, reverted, non-finite input), accepted
 * sub-steps and Newton iterations.  Any output pointer may be NULL.
 * With a host destination the call synchronises the stream and also reports a device
 * error recorded by the integrate kernels (KT_ETIMEOUT). */
KT_API int kt_state_download(const kt_state *st, double *y, double *T, int32_t *status,
                      int32_t *n_substeps, int32_t *n_newton, int dst_is_device,
                      void *cuda_stream);

/* Synchronise the stream and report a device error recorded by the kernels. */
KT_API int kt_state_check(const kt_state *st, void *cuda_stream);

KT_API void kt_state_free(kt_state *st);

/* Bytes of device scratch one kt_integrate_ptrs call needs (queue counter and error
 * word); the caller passes a zero-or-not buffer of at least this size, 16-B aligned. */
KT_API size_t kt_scratch_bytes(void);

/* Same operation on caller-owned DEVICE buffers (e.g. torch tensors):
 * y_in [n_species][ncells], T_in [ncells], rho [ncells] (may be NULL); outputs may
 * alias the inputs (in-place integration); status/n_substeps/n_newton may be NULL.
 * scratch: device buffer of kt_scratch_bytes() bytes, reused by the call (its
 * content on entry does not matter).  Calls sharing a scratch buffer must be ordered
 * on one stream. */
KT_API int kt_integrate_ptrs(const kt_network *net, int64_t ncells, const double *y_in,
                      const double *T_in, const double *rho, double dt,
                      const kt_options *opts, double *y_out, double *T_out,
                      int32_t *status, int32_t *n_substeps, int32_t *n_newton,
                      void *scratch, void *cuda_stream);

/* Launch-configuration search (warps per block, persistent queue or one pass; the
 * kernel family is base->cells_per_warp, or by size when 0: one cell per lane up to
 * 16 unknowns, else one per warp) on a caller-supplied sample of cells in device
 * buffers: each candidate integrates the sample once untimed and once timed with
 * CUDA events on stream; *best receives base with the fastest configuration and
 * *best_seconds its time.  Same buffer rules as kt_integrate_ptrs; synchronises. */
KT_API int kt_autotune(const kt_network *net, int64_t ncells, const double *y_in,
                       const double *T_in, double dt, const kt_options *base,
                       double *y_out, double *T_out, void *scratch, void *cuda_stream,
                       kt_options *best, double *best_seconds);

/* kt_integrate_ptrs for networks with photo-reactions (Sec. 2.2.1 item 2, Eq.
 * photo-reaction-single): per cell the photo flux factor flux[c] = L dl / dV
 * [photons cm^-2 s^-1 per unit cross-section] and the path length path[c] = dl [cm]
 * (device float64 [ncells]; either may be NULL: flux 1, path 0).  A photo-reaction of
 * reactant i with cross-section sigma_r runs at k = flux sigma_r (1 - e^-tau)/tau,
 * tau = path sum_s n_s sigma_s over every absorbing species (the optically thin limit
 * flux sigma_r when path = 0), with the exact Jacobian of tau's dependence on every
 * absorber.  rho (may be NULL: 1) also selects the cell's slice of the network's rate
 * tables.  Same buffer rules as kt_integrate_ptrs.  Networks with tabulated or photo
 * rates run in the warp-per-cell kernels (cells_per_warp 0 or 1). */
KT_API int kt_integrate_rad(const kt_network *net, int64_t ncells, const double *y_in,
                            const double *T_in, const double *rho, const double *flux,
                            const double *path, double dt, const kt_options *opts, double *y_out,
                            double *T_out, int32_t *status, int32_t *n_substeps, int32_t *n_newton,
                            void *scratch, void *cuda_stream);

/* kt_integrate_ptrs with a per-cell time step: dt_cells [ncells] (device, float64,
 * each > 0; a cell whose dt is not a positive finite number gets status
 * KT_STATUS_NONFINITE and is left untouched). */
KT_API int kt_integrate_dt(const kt_network *net, int64_t ncells, const double *y_in,
                           const double *T_in, const double *rho, const double *dt_cells,
                           const kt_options *opts, double *y_out, double *T_out,
                           int32_t *status, int32_t *n_substeps, int32_t *n_newton,
                           void *scratch, void *cuda_stream);

/* kt_integrate_ptrs for callers that must not allocate device memory (a host
 * framework that owns every allocation, a step running inside a fixed memory pool or a
 * real-time budget).  The paper has no counterpart; it is an interface of this library.
 * The call allocates nothing: the work-queue counter, the device error word and the
 * network tables live in one static device array of 64 KiB per device, held by every
 * device that loads the library until the process exits.  Networks whose tables need
 * more (256 bytes of counters plus the tables) are rejected with KT_EINVAL and a
 * message.  The first call on a device looks up the array's device address (make that
 * first call before any stream capture).  Every call shares the array and resets the
 * counter and refreshes the tables itself; calls that overlap on the GPU (two streams,
 * two host threads) race on it and must be ordered by the caller.  Same arguments and
 * buffer rules as kt_integrate_ptrs except the scratch, which is internal; the
 * learned guess is not available here (KT_EUNSUPPORTED).  Each call copies the network
 * tables from host memory into the array on cuda_stream.  status is required (NULL is
 * KT_EINVAL): it is the call's only report of a device-side failure, since the device
 * error word sits in the internal array; cells the kernels did not reach because of a
 * device error keep status -1. */
KT_API int kt_integrate_noalloc(const kt_network *net, int64_t ncells, const double *y_in,
                                const double *T_in, const double *rho, double dt,
                                const kt_options *opts, double *y_out, double *T_out,
                                int32_t *status, int32_t *n_substeps, int32_t *n_newton,
                                void *cuda_stream);

/* Read and clear the device error word of a scratch buffer (synchronises stream). */
KT_API int kt_scratch_check(void *scratch, void *cuda_stream);

/* ---------------------------------------------------------------- learned guess
 * A small MLP predicts the Newton starting iterate of each sub-step (the paper's
 * closing section points at DeepODE-style learned solvers; there is no further
 * specification).  Architecture: n_in (<= 16) -> 128 -> 128 -> 128 -> n_out (<= 16),
 * SiLU, BF16 weights, FP32 accumulation (mma.sync tensor-core kernels).
 * For a network with ns species and N unknowns the guess uses n_in = ns + 3 features
 * (log max(y_s,1e-30), log T, log rho, log h), normalised as (x - mu_in)/sd_in, and
 * n_out = N outputs: the normalised change of log y (and log T) over the step,
 * un-normalised as mu_out + sd_out * out.  If Newton does not converge from the guess
 * the step is retried from the plain predictor, so the answer is the solver's.
 * Master parameters (float32, kt_mlp_sizes() of them) in this order:
 * W1 [128][16], W2 [128][128], W3 [128][128], W4 [16][128], b1 [128], b2 [128],
 * b3 [128], b4 [16]; row n of W_l holds the weights of output n (z = h W^T + b);
 * entries beyond n_in / n_out are zero and stay zero. */
KT_API int kt_mlp_sizes(int *n_master_params, int *packed_bytes);

/* New MLP on the current device with PyTorch-style uniform initialisation from seed. */
KT_API int kt_mlp_create(int n_in, int n_out, unsigned long long seed, kt_mlp **out);
KT_API void kt_mlp_free(kt_mlp *mlp);

/* Feature / output normalisation (host arrays of n_in and n_out floats; sd > 0). */
KT_API int kt_mlp_set_norm(kt_mlp *mlp, const float *mu_in, const float *sd_in,
                           const float *mu_out, const float *sd_out);

/* One Adam step (lr; betas 0.9, 0.999; eps 1e-8) on the MSE loss
 * 1/(2B) sum (out - target)^2 of a batch: X [B][16] and targets [B][16] are
 * normalised float32 device arrays (padding columns ignored).  *loss (host, may be
 * NULL; non-NULL synchronises) receives the loss before the update. */
KT_API int kt_mlp_train_step(kt_mlp *mlp, const float *X, const float *targets, int B,
                             float lr, double *loss, void *cuda_stream);

/* Gradients of that loss (host float array in the master order) without updating;
 * synchronises. */
KT_API int kt_mlp_gradients(kt_mlp *mlp, const float *X, const float *targets, int B,
                            float *grads, double *loss, void *cuda_stream);

/* Batch inference: X [n][16] -> out [n][16] (normalised), device arrays, asynchronous. */
KT_API int kt_mlp_forward(const kt_mlp *mlp, const float *X, float *out, int64_t n,
                          void *cuda_stream);

/* Copy the float32 master parameters out / in (host arrays; set re-packs BF16). */
KT_API int kt_mlp_get_params(const kt_mlp *mlp, float *master);
KT_API int kt_mlp_set_params(kt_mlp *mlp, const float *master);

/* Flat binary file: "KTMLP2", n_in, n_out, hidden, layers, seed, step, dtype tag,
 * normalisation, float32 masters. */
KT_API int kt_mlp_save(const kt_mlp *mlp, const char *path);
KT_API int kt_mlp_load_file(const char *path, kt_mlp **out);

/* Load a saved MLP into a state (owned by the state) for opts.guess = KT_GUESS_MLP. */
KT_API int kt_mlp_load(kt_state *st, const char *weights_path);

/* Use mlp (not owned; must outlive the calls) for kt_integrate_ptrs / kt_integrate_dt
 * with opts.guess = KT_GUESS_MLP on this network; NULL detaches. */
KT_API int kt_network_attach_mlp(kt_network *net, const kt_mlp *mlp);

/* Diagnostics: out[i] = exp(x[i]) for device arrays, which = 0 CUDA's exp, 1 the
 * library's table-driven exponential (valid for -708 <= x <= 709). */
KT_API int kt_debug_exp(const double *x, double *out, int64_t n, int which, void *cuda_stream);

/* Stoichiometry-compatible species advection, one directional sweep (Sec. 2.1.3,
 * Eqs. method-flux-sp, method-plm-general, method-sto-plm-proj, method-sto-plm-recon):
 * on nlines periodic lines of L >= 3 uniform cells of width dx, x^s = n^s / rho is
 * reconstructed piecewise-linearly with the modified van Leer limiter (slope
 * sgn(a) min(2|a||b|/(|a|+|b|), |b|) from the forward and backward differences a, b;
 * zero at extrema), the corrections are projected onto the null space of the network's
 * element matrix (project = 1; the element abundances of every interface state then
 * equal the cell's), the upwind state by the sign of the mass flux gives the species
 * fluxes F^s = x^s F^rho, and
 *   n_out = alpha n_base + (1 - alpha) (n_in - dtdx (F_{j+1/2} - F_{j-1/2}))
 * (n_base may be NULL: n_out = the plain update).  Device float64 arrays: n_in, n_base,
 * n_out [n_species][nlines][L]; rho, mass_flux [nlines][L], mass_flux[j] at the interface
 * j-1/2.  n_out must not alias n_in.  scratch: device buffer of kt_advect_scratch_bytes(),
 * 16-B aligned, reused by the call (calls sharing it must be ordered on one stream).
 * nlines <= 65535.  Asynchronous on stream. */
KT_API int kt_advect_sweep(const kt_network *net, int64_t nlines, int64_t L, const double *n_in,
                           const double *rho, const double *mass_flux, double dx, double dtdx,
                           double alpha, const double *n_base, double *n_out, int project,
                           void *scratch, void *cuda_stream);

/* Bytes of device scratch one kt_advect_sweep call needs. */
KT_API size_t kt_advect_scratch_bytes(void);

/* Ray tracing on a Cartesian mesh with Beer-Lambert deposition (Sec. 3, Eqs. cart-dl,
 * method-rad-equiv-flux, method-rt-abs).  The box [0, nx hx] x [0, ny hy] x [0, nz hz]
 * holds nx*ny*nz cells; kappa [nbins][nx][ny][nz] is each cell's inverse absorption
 * length per energy bin.  Ray q starts at origins[3q..3q+2] with unit direction
 * dirs[3q..3q+2] and photon counts n0[q*nbins + b]; in every cell it crosses, over the
 * length dl between its entry and exit (the nearest axis plane of Eq. cart-dl), it adds
 * N dl/(dV dt) (1 - e^-tau)/tau to feff and N (1 - e^-tau) to absorbed (tau = kappa dl,
 * both [nbins][nx][ny][nz], accumulated: the caller zeroes them) and leaves with
 * N e^-tau; escaped [nrays][nbins] (may be NULL) receives what leaves the box.  Rays
 * starting outside the box deposit nothing.  Accumulation uses FP64 atomics, so sums
 * over rays crossing one cell are order-dependent at rounding level.  nbins <= 8.
 * Device float64 arrays; asynchronous on stream. */
KT_API int kt_raytrace(int nx, int ny, int nz, double hx, double hy, double hz, int nbins,
                       const double *kappa, int64_t nrays, const double *origins, const double *dirs,
                       const double *n0, double dt, double *feff, double *absorbed, double *escaped,
                       void *cuda_stream);

/* Rays of an isotropic point source (Eq. method-rt-ph-num): nrays directions on a
 * Fibonacci lattice (z_k = 1 - (2k+1)/nrays, azimuth k pi (3 - sqrt 5)), each of solid
 * angle 4 pi / nrays, carrying lum[b] dt / nrays photons per bin.  src (3) and lum
 * (nbins <= 8) are host arrays; origins, dirs [nrays][3] and n0 [nrays][nbins] are
 * device outputs.  Asynchronous on stream. */
KT_API int kt_rays_point_source(const double *src, const double *lum, int nbins, double dt,
                                int64_t nrays, double *origins, double *dirs, double *n0,
                                void *cuda_stream);

/* Diagnostics: peak probe of the FP64 (fp32 = 0) or FP32 (fp32 = 1) pipe, the
 * denominator of the library's roofline figures.  Launches `blocks` blocks (0: 8 per
 * SM) of 256 threads, each thread running 8 independent fused multiply-add chains for
 * `iters` rounds; *flops (host, may be NULL) receives the flops launched
 * (2 x 8 x iters x threads).  The caller times the launch on `stream` with events.
 * sink: device buffer of at least 8 bytes, written only to keep the loop alive. */
KT_API int kt_fma_peak(int fp32, int64_t iters, int blocks, double *sink, void *cuda_stream,
                       double *flops);

/* Thread-local message of the last failed call ("" if none). */
KT_API const char *kt_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* KT_H */
