/*
 * lbhpde.h -- C ABI of a GB300 (sm_103a) lattice Boltzmann solver for
 *
 *     phi_t + sum_{k=1..m} alpha_k d_x^k Pi_k(phi) = 0,     1 <= m <= 6,
 *
 * the general LBGK model of B. Shi, N. He, Z. Guo, "Lattice Boltzmann Model for
 * High-Order Nonlinear Partial Differential Equations", arXiv:0907.1720
 * (Eq. (NPDE), Sec. II A).
 *
 * Conventions for every function below:
 *   - Return value: an LBHPDE_* status code (0 = success).  No function aborts or
 *     prints; lbhpde_strerror() turns a code into text.
 *   - Host pointers are owned by the caller and are only read or written during
 *     the call (inputs are copied).  Device memory that a handle needs is
 *     allocated by the library through the allocator given at creation (or
 *     cudaMalloc when none is given) and released by the matching destroy call.
 *   - Distribution arrays live in HBM as structure-of-arrays rows of length ld
 *     (ld >= N, a multiple of 32 elements): row 0 holds phi, rows 1..b-1 hold
 *     the post-collision populations f*_j, j = 1..b-1, of the velocities
 *     e = {1,-1,2,-2[,3,-3]} (Sec. III A/B).  The rest population is implied by
 *     sum_j f*_j = phi, which collision preserves (first relation of Eq. (moments)).
 *   - Work is enqueued on the handle's CUDA stream; calls that return data to the
 *     host synchronise that stream.  A handle may be used by one host thread at
 *     a time; the server (lbhpde_server_*) is internally synchronised.
 *   - Grids are periodic (LBHPDE_PERIODIC) or bounded (LBHPDE_NEE): nodes
 *     x_0..x_{N-1} with prescribed phi at the max|e| outer nodes of each end,
 *     applied by the non-equilibrium extrapolation that Sec. IV uses for its
 *     test problems (see LBHPDE_NEE).
 */
#ifndef LBHPDE_H
#define LBHPDE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define LBHPDE_OK 0
#define LBHPDE_ERR_ARG 1          /* invalid argument (sizes, orders, lattice, pointers) */
#define LBHPDE_ERR_TAU_SINGULAR 2 /* tau_k = 0 for a needed k: beta_k or A_k0 undefined  */
#define LBHPDE_ERR_OOM 3          /* device allocation failed / over the memory budget   */
#define LBHPDE_ERR_DIVERGED 4     /* a non-finite phi was found                          */
#define LBHPDE_PENDING 5          /* request accepted but not finished (lbhpde_poll)     */
#define LBHPDE_ERR_TIMEOUT 6      /* a bounded wait ran out                              */
#define LBHPDE_ERR_CUDA 7         /* a CUDA runtime call failed                          */
#define LBHPDE_ERR_NOT_FOUND 8    /* unknown request id                                  */
#define LBHPDE_ERR_UNSUPPORTED 9  /* valid request this build does not handle            */

/* -------------------------------------------------------------- enumerations */
#define LBHPDE_FP64 0      /* populations and arithmetic in IEEE double                   */
#define LBHPDE_FP32_DEV 1  /* float populations stored as deviations from the rest         */
                           /* equilibrium (phi kept apart), float arithmetic               */
#define LBHPDE_PERIODIC 0
/* Bounded grid with the non-equilibrium extrapolation boundary of Sec. IV (after Guo et al.;
 * the paper gives no formula).  After each collide+stream step the W = max|e| outer nodes at
 * each end (nodes 0..W-1 and N-W..N-1) are rebuilt as
 *     f_j(x_b) = f^eq_j(phi_b) + [f_j(x_f) - f^eq_j(phi(x_f))],
 * phi_b the prescribed value and x_f = W - 1 + depth (left), N - W - depth (right).  The plain
 * code LBHPDE_NEE means depth 2, which reproduces the paper's printed errors for its D1Q5 and
 * c = 10 D1Q7 examples; LBHPDE_NEE_DEPTH(d) chooses another depth (d >= 1; d = 1 is the
 * nearest node whose populations all come from inside the grid).  Needs N >= 2 (W + depth).
 * Bounded instances are stepped with lbhpde_step_nee / lbhpde_batch_step_nee, which take the
 * boundary values of every step. */
#define LBHPDE_NEE 1
#define LBHPDE_NEE_DEPTH(d) (LBHPDE_NEE | ((d) << 8))

/* Flag or-ed into `scheme`: leave the A_40, A_50, A_60 corrections of Eqs. (Pi4)-(Pi6) out of
 * the auxiliary moments.  The paper derives them for exact recovery, but its printed errors
 * for the Kuramoto-Sivashinsky examples (Tables I and II) are those of a model without A_40.
 * The model is then flagged inexact wherever a correction would be present. */
#define LBHPDE_NO_AUX_CORRECTION 0x100

#define LBHPDE_PI_ZERO 0   /* Pi_k = 0                         */
#define LBHPDE_PI_PHI 1    /* Pi_k = phi                       */
#define LBHPDE_PI_POWER 2  /* Pi_k = phi^power, 1 <= power <= 7 */
#define LBHPDE_PI_POLY 3   /* Pi_k = sum_p coef[p] phi^p        */
#define LBHPDE_PI_POLY_NU 4 /* Pi_k = sum_p coef[p] phi^p + sum_{p>=1} coef_nu[p] phi^(p + nu), nu > 0 real:
                              * the u^n u_x terms of class (1), Sec. III C, with a real n */
#define LBHPDE_PI_NCOEF 8
#define LBHPDE_MAX_DEG 31  /* highest degree of f^eq_j(phi) the kernels accept */
#define LBHPDE_NU_TERMS 64 /* capacity of the generalised f^eq tables: (A + 1)(Dg + 1) <= 64 */

#define LBHPDE_KERNEL_AUTO 0    /* the on-chip kernel (ONCHIP)                                 */
#define LBHPDE_KERNEL_STREAM 1  /* one fused collide+stream launch per step through HBM        */
#define LBHPDE_KERNEL_ONCHIP 2  /* instances that fit one CTA stay resident in registers for   */
                                /* all steps; longer ones advance in temporally blocked        */
                                /* windows (HALO)                                              */
#define LBHPDE_KERNEL_HALO 3    /* every instance in temporally blocked windows: a CTA loads a */
                                /* window plus a halo from HBM, advances it several steps in   */
                                /* registers and writes back the exact middle                  */

/* One flux function Pi_k of Eq. (NPDE): the paper requires "known differential
 * functions of phi"; this library takes polynomials in phi (every worked class of
 * Sec. III C is of that form), optionally with terms phi^(p + nu) of one real exponent
 * nu > 0 (class (1) with a real n: Pi_1 = a u^2/2 + b u^(n+1)/(n+1), nu = n).  All Pi_k of
 * kind LBHPDE_PI_POLY_NU of one equation must share nu.  The phi^(p + nu) terms are taken
 * as zero where phi <= 0 (the paper's class has u > 0; this is the continuous extension). */
typedef struct {
    int kind;                        /* LBHPDE_PI_*                                      */
    int power;                       /* for LBHPDE_PI_POWER                              */
    double coef[LBHPDE_PI_NCOEF];    /* for LBHPDE_PI_POLY(_NU): coef[p] phi^p           */
    double nu;                       /* for LBHPDE_PI_POLY_NU: the real exponent, > 0    */
    double coef_nu[LBHPDE_PI_NCOEF]; /* for LBHPDE_PI_POLY_NU: coef_nu[p] phi^(p + nu);  */
                                     /* coef_nu[0] must be 0                             */
} lbhpde_pi;

/* The model the library derives from an equation (Secs. II and III): step a0 of the
 * hot path.  P_j(phi) = sum_p coef[j][p] phi^p equals omega * f^eq_j(phi) with
 * omega = 1/tau; feq[j][p] are the unscaled coefficients of f^eq_j.  Row j follows
 * the velocity order e = {0,1,-1,2,-2,3,-3}. */
typedef struct {
    int b;                 /* lattice velocities: 5 (D1Q5) or 7 (D1Q7)                    */
    int m;                 /* order of the equation                                        */
    int scheme;            /* 1 = all b moments, 2 = highest moment set to zero (Sec. IV) */
    int D;                 /* degree of the f^eq_j polynomials                             */
    int inexact;           /* 1 if a precondition of exact recovery fails (Remarks 2, 4, 5)*/
    double c;              /* lattice speed dx/dt                                          */
    double omega;          /* 1/tau                                                         */
    double tk[7];          /* tau_k, k = 2..6, Eq. (taus)                                   */
    double beta[7];        /* beta_k, k = 2..6: alpha_k = dt^{k-1} tau_k beta_k             */
    double A[3];           /* A_40, A_50, A_60, Eqs. (Pi4)-(Pi6)                            */
    double feq[7][LBHPDE_MAX_DEG + 1];
    double coef[7][LBHPDE_MAX_DEG + 1];
    /* The same in generalised form, for every model:
     *   f^eq_j(phi) = sum_{a=0}^{A} (phi^nu)^a sum_{i=0}^{Dg} gfeq[j][a (Dg + 1) + i] phi^i,
     * A = nu_rows - 1, Dg = nu_deg; gcoef = omega gfeq.  Without real exponents nu = 0,
     * nu_rows = 1, nu_deg = D and the rows equal feq and coef; with them, D = (A + 1)(Dg + 1) - 1
     * (the flattened row length minus one) and feq, coef are zero. */
    double nu;
    int nu_rows, nu_deg;
    double gfeq[7][LBHPDE_NU_TERMS];
    double gcoef[7][LBHPDE_NU_TERMS];
} lbhpde_model_info;

/* Optional device allocator (e.g. a framework's caching allocator).  alloc returns a
 * device pointer with at least 256-byte alignment or NULL; release frees it. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*release)(void *ptr, size_t bytes, void *stream, void *user);
    void *user;
} lbhpde_allocator;

/* ------------------------------------------------------------------ step a0 */

/* Build the model of Secs. II-III on the host (no GPU is touched):
 * tau_k (Eq. (taus)), beta_k (Eqs. (NPDE3)-(NPDE6)), A_40/A_50/A_60 (Eqs. (Pi4)-(Pi6)),
 * the auxiliary moments Pi_k0 = int_0^phi [...] dphi (Sec. II C-F, integration constant
 * zero), the scaled moments Pibar_k = (Pi_k0 + beta_k Pi_k)/c^k (Sec. III A/B) and
 * f^eq = M^-1 Pibar (Eqs. (EDF5), (EDF7)), folded into polynomial coefficients.
 *   m          order, 1..6; m <= b-1
 *   alpha      [m], alpha[k-1] = alpha_k; alpha[0] scales Pi_1 (the paper fixes alpha_1 = 1)
 *   pi         [m], Pi_1..Pi_m
 *   dx, dt     lattice spacing and time step (> 0, finite); c = dx/dt
 *   tau        dimensionless relaxation time (> 0)
 *   lattice    0 = auto (5 for m <= 4, else 7), 5 or 7
 *   scheme     1 or 2 (scheme 2 needs m < b-1), optionally | LBHPDE_NO_AUX_CORRECTION
 * Errors: LBHPDE_ERR_ARG, LBHPDE_ERR_TAU_SINGULAR (tau_k = 0 where beta_k or A_k0 needs it). */
int lbhpde_model(int m, const double *alpha, const lbhpde_pi *pi, double dx, double dt, double tau,
                 int lattice, int scheme, lbhpde_model_info *out);

/* --------------------------------------------------------- single instance */

typedef struct lbhpde_ctx *lbhpde_t;

/* Create one instance of N nodes: periodic (N >= 2 * max|e_j|, i.e. 4 on D1Q5 and 6 on D1Q7)
 * or bounded (boundary = LBHPDE_NEE or LBHPDE_NEE_DEPTH(d); N >= 2 (max|e_j| + depth)).
 * precision is LBHPDE_FP64 or LBHPDE_FP32_DEV.  Other boundary codes: LBHPDE_ERR_UNSUPPORTED.
 * cuda_stream is a cudaStream_t (NULL = the legacy default stream); alloc may be NULL.
 * The state is undefined until lbhpde_set_phi. */
int lbhpde_create(lbhpde_t *out, int m, const double *alpha, const lbhpde_pi *pi, long N, double dx,
                  double dt, double tau, int lattice, int scheme, int precision, int boundary,
                  void *cuda_stream, const lbhpde_allocator *alloc);

/* Step a1: f_j(x, 0) = f^eq_j(phi0(x)) (the paper sets initial conditions from the
 * analytic solution, Sec. IV; equilibrium initial populations are this library's reading).
 * phi0 is [N] doubles in host memory (phi0_on_device = 0) or device memory (= 1). */
int lbhpde_set_phi(lbhpde_t h, const double *phi0, int phi0_on_device);

/* Steps a2-a6, nsteps times: stream (pull form), phi = sum_j f_j, f^eq_j(phi), BGK relaxation
 * f*_j = f_j - (f_j - f^eq_j)/tau (Eq. (LBE)).  Asynchronous on the handle's stream.
 * LBHPDE_ERR_ARG on a bounded instance (it needs boundary values: lbhpde_step_nee). */
int lbhpde_step(lbhpde_t h, long nsteps);

/* nsteps steps of a bounded instance (LBHPDE_NEE): each step as lbhpde_step, then the outer
 * nodes are rebuilt from the prescribed values.  phib: [nsteps][2W] doubles, W = max|e_j|;
 * row n holds phi_b at time (steps taken + n + 1) dt at nodes 0..W-1 followed by nodes
 * N-W..N-1.  phib is host memory (phib_on_device = 0: copied before the call returns, unless it
 * is page-locked, in which case it must stay unchanged until the stream reaches the step) or
 * device memory (= 1: read by the kernels, so it must stay valid until they have run).  On a
 * periodic instance phib is ignored (may be NULL). */
int lbhpde_step_nee(lbhpde_t h, long nsteps, const double *phib, int phib_on_device);

/* Step a7: copy phi (t = steps taken * dt) into phi_out ([N] doubles, host or device).
 * Synchronises the stream (host output: the copy; device output: the 4-byte non-finite flag the
 * copy kernel raises).  Returns LBHPDE_ERR_DIVERGED (after copying) if phi has a non-finite
 * value. */
int lbhpde_read_phi(lbhpde_t h, double *phi_out, int out_on_device);

/* Diagnostics of step a7, reduced on the GPU in double precision. */
typedef struct {
    double sum_phi;     /* sum_x phi: invariant on periodic grids                        */
    double max_abs_phi;
    long nonfinite;     /* nodes whose phi is NaN or Inf                                  */
    double err_E;       /* sum|phi - phi*| / sum|phi*| (Sec. IV), when phi* is given     */
    double err_L2;      /* ||phi - phi*||_2 / ||phi*||_2, when phi* is given             */
    long steps;         /* time steps taken since lbhpde_set_phi                         */
} lbhpde_diag;

/* phistar: [N] doubles in device memory, or NULL.  Synchronises the stream. */
int lbhpde_diagnostics(lbhpde_t h, const double *phistar_device, lbhpde_diag *out);

/* Kernels the handle has launched since it was made (instrumentation; no counterpart in the
 * paper), into *count: every step, initialisation, readout and diagnostics kernel (a replay of
 * a captured graph counts each kernel in it).  Host only; LBHPDE_ERR_ARG for a NULL argument. */
int lbhpde_kernel_launches(lbhpde_t h, long long *count);

/* Which kernel lbhpde_step uses (LBHPDE_KERNEL_*).  For the on-chip kernels: the nodes each
 * thread holds (FP32: 2, 4 or 8 on D1Q5, 4 or 8 on D1Q7; FP64: 2 or 4 on D1Q5, 4 on D1Q7; 16 on
 * FP32 D1Q5 polynomial models selects the 16-node resident kernel, which holds instances of up
 * to 8192 nodes and is the automatic choice there, longer ones taking windows of the default
 * size) and the steps per launch (resident instances: launch chunk; windows: steps per window, which
 * sets the halo to steps * max|e| nodes); 0 = automatic.  Returns LBHPDE_ERR_UNSUPPORTED for a
 * combination the library was not built with, leaving the previous choice in place. */
int lbhpde_set_kernel(lbhpde_t h, int kernel, int nodes_per_thread, int steps_per_launch);

/* Autotuner of the on-chip kernel (tile width and time-block depth; the paper has no
 * counterpart).  Times the compiled (nodes per thread, steps per window)
 * candidates for one precision, lattice (5 or 7) and f^eq degree on a synthetic periodic grid
 * of 2^22 (FP32) or 2^21 (FP64) nodes in temporally blocked windows, and keeps the fastest in a
 * process-wide table.  Batches and handles created afterwards use the tuned pair wherever
 * lbhpde_set_kernel did not fix one.  Outputs (each may be NULL): the chosen pair and its
 * measured node-updates per second.  Allocates and frees about 235 MB of device memory on the
 * current device and synchronises. */
int lbhpde_autotune(int precision, int lattice, int degree, int *nodes_per_thread, int *steps_per_launch,
                    double *node_updates_per_s);

/* Records a tuned (nodes per thread, steps per window) pair for one precision, lattice and f^eq
 * degree without timing anything (no counterpart in the paper), as lbhpde_autotune would have
 * left it: e.g. a pair found in an earlier process, or a fixed choice for a profiling run.
 * Host only (no device work).
 * LBHPDE_ERR_ARG for an invalid precision, lattice or degree, or steps_per_launch < 1;
 * LBHPDE_ERR_UNSUPPORTED for nodes per thread the library was not built with, or a window
 * whose halo (2 * steps * max|e|) leaves fewer than half of its nodes valid. */
int lbhpde_set_tuning(int precision, int lattice, int degree, int nodes_per_thread, int steps_per_launch);

int lbhpde_get_model(lbhpde_t h, lbhpde_model_info *out);
int lbhpde_destroy(lbhpde_t h);
const char *lbhpde_strerror(int code);

/* ------------------------------------------------------------------ batches */

/* One member of a batch (the same arguments as lbhpde_create). */
typedef struct {
    int m;
    double alpha[6];
    lbhpde_pi pi[6];
    long N;
    double dx, dt, tau;
    int lattice, scheme;
    int boundary;          /* LBHPDE_PERIODIC (0), LBHPDE_NEE or LBHPDE_NEE_DEPTH(d) */
} lbhpde_instance;

typedef struct lbhpde_batch_s *lbhpde_batch_t;

/* Many independent instances of one precision, stepped together: the on-chip kernel packs
 * whole periodic instances onto CTAs (one launch advances all of them) and keeps each bounded
 * instance of up to 2048 nodes resident in one CTA; longer instances use the streaming kernel.
 * Members may mix lattices, orders, sizes and boundaries. */
int lbhpde_batch_create(lbhpde_batch_t *out, int count, const lbhpde_instance *members, int precision,
                        void *cuda_stream, const lbhpde_allocator *alloc);
/* phi0: the members' initial profiles concatenated ([sum N] doubles, host or device). */
int lbhpde_batch_set_phi(lbhpde_batch_t b, const double *phi0, int phi0_on_device);
/* LBHPDE_ERR_ARG if the batch has a bounded member (use lbhpde_batch_step_nee). */
int lbhpde_batch_step(lbhpde_batch_t b, long nsteps);
/* As lbhpde_step_nee for every member: the boundary values of member i are the [nsteps][2W_i]
 * doubles at phib + i * member_stride.  member_stride = 0 lets all bounded members share one
 * array (they must then have the same W); otherwise member_stride >= nsteps * 2W_i for every
 * bounded member.  Periodic members ignore phib. */
int lbhpde_batch_step_nee(lbhpde_batch_t b, long nsteps, const double *phib, long member_stride,
                          int phib_on_device);
/* phi_out: [sum N] doubles, host or device.  LBHPDE_ERR_DIVERGED if any phi is non-finite. */
int lbhpde_batch_read_phi(lbhpde_batch_t b, double *phi_out, int out_on_device);
/* out: [count] records.  phistar: [sum N] doubles in device memory, or NULL. */
int lbhpde_batch_diagnostics(lbhpde_batch_t b, const double *phistar_device, lbhpde_diag *out);
/* As lbhpde_kernel_launches, for a batch. */
int lbhpde_batch_kernel_launches(lbhpde_batch_t b, long long *count);
int lbhpde_batch_set_kernel(lbhpde_batch_t b, int kernel, int nodes_per_thread, int steps_per_launch);
/* Total node count (sum N) and device bytes held. */
int lbhpde_batch_size(lbhpde_batch_t b, long *total_nodes, size_t *device_bytes);
int lbhpde_batch_destroy(lbhpde_batch_t b);

/* ------------------------------------------------------------ checkpoint / resume */

/* The paper has no checkpoint; these keep a long solve restartable.  A checkpoint holds the
 * batch's full state (every member's phi and stored populations, in the batch's precision, as
 * on the device), the steps taken, and a fingerprint of the layout (member count, sizes,
 * lattices, depths, precision).  Loading it into a batch created with the same members
 * continues bit for bit as the saved batch would have; the members' models are the loading
 * batch's own.  Both calls copy through host memory and synchronise the batch's stream.
 *   bytes: the size of buf; checkpoint_size gives the size needed.
 * Errors: LBHPDE_ERR_ARG for a NULL argument, a buffer that is too small, saving a batch whose
 * phi was never set, or loading a checkpoint of another layout or precision (nothing changes). */
int lbhpde_batch_checkpoint_size(lbhpde_batch_t b, size_t *bytes);
int lbhpde_batch_save(lbhpde_batch_t b, void *buf, size_t bytes);
int lbhpde_batch_load(lbhpde_batch_t b, const void *buf, size_t bytes);
/* The same for a single instance. */
int lbhpde_checkpoint_size(lbhpde_t h, size_t *bytes);
int lbhpde_save(lbhpde_t h, void *buf, size_t bytes);
int lbhpde_load(lbhpde_t h, const void *buf, size_t bytes);

/* ------------------------------------------------------------------ serving */

/* A request server: continuous batching of independent solves on one GPU (the paper has no
 * serving layer).  Requests are admitted as device memory and slots
 * free up, keep their distributions resident in the server's device arena, and advance
 * together in step blocks on the on-chip kernel; a request that arrives while others run is
 * admitted at the next block boundary.  Each request's arithmetic is that of a single-instance
 * solve with the same kernel, so its result does not depend on what else is in the mix.
 * The server owns one scheduler thread and one CUDA stream; all entry points are thread-safe. */
typedef struct lbhpde_server_s *lbhpde_server_t;

typedef struct {
    int m;
    double alpha[6];
    lbhpde_pi pi[6];
    long N;
    double dx, dt, tau;
    int lattice, scheme;
    long nsteps;           /* time steps to take (>= 0)                                  */
    const double *phi0;    /* [N] host doubles, copied by lbhpde_submit                   */
} lbhpde_request;

typedef struct {
    int status;            /* LBHPDE_PENDING, LBHPDE_OK, LBHPDE_ERR_DIVERGED, LBHPDE_ERR_CUDA */
    long steps_done;
    double submit_s;       /* host clock, seconds since the server started                */
    double admit_s;        /* -1 while queued                                             */
    double finish_s;       /* -1 while pending; latency = finish_s - submit_s             */
    double sum_phi;        /* sum of the final phi (FP64)                                  */
    long nonfinite;        /* nodes whose final phi is not finite                          */
} lbhpde_result;

typedef struct {
    long queued, in_flight, completed;
    double node_updates;   /* completed requests' N * nsteps                               */
    size_t bytes_in_use, bytes_total;
    long launches;
    int error;             /* sticky status of the scheduler (LBHPDE_OK unless a CUDA call failed) */
    double gpu_busy_s;     /* summed GPU time of the step blocks, from their uploads to their last
                            * launch (CUDA events): busy / wall time is the device's share of work */
    /* host time of the scheduler thread by phase (seconds, summed over step blocks): admission,
     * set-up of admitted requests (uploads, initialisation), planning (packing and table
     * uploads), issuing the launches, waiting for the block, retiring finished requests */
    double host_admit_s, host_setup_s, host_plan_s, host_launch_s, host_wait_s, host_retire_s;
} lbhpde_server_info;

/* device_bytes (>= 1 MiB) is the state arena, allocated at creation; each request holds
 * 2 * b * ceil32(N) elements of the chosen precision while admitted.  max_active (1..65536)
 * bounds the admitted requests; steps_per_block (0 = 256) is the admission granularity. */
int lbhpde_server_create(lbhpde_server_t *out, int precision, size_t device_bytes, int max_active,
                         int steps_per_block, int device);
/* Step a0 runs here on the caller's thread.  Any model lbhpde_model accepts, real exponents
 * included (served by the on-chip kernels' real-exponent variant).  Errors: LBHPDE_ERR_ARG
 * (invalid request), LBHPDE_ERR_OOM (larger than the whole arena), LBHPDE_ERR_CUDA (the server
 * has failed). */
int lbhpde_submit(lbhpde_server_t s, const lbhpde_request *req, uint64_t *id);
/* As lbhpde_submit for a bounded request (the non-equilibrium extrapolation boundary of Sec. IV,
 * as for lbhpde_create).  boundary: LBHPDE_NEE or LBHPDE_NEE_DEPTH(d), N >= 2 (W + depth).
 * phib: [nsteps][2W] host doubles, W = max|e_j|, row n holding phi_b at time (n + 1) dt at nodes
 * 0..W-1 followed by nodes N-W..N-1 (the layout of lbhpde_step_nee); copied by the call (may
 * be NULL when nsteps = 0).  The request stays resident in one CTA of the bounded kernel, whose
 * arithmetic is that of lbhpde_step_nee on a single instance with LBHPDE_KERNEL_ONCHIP at 4 nodes
 * a thread, so its result is the same alone and in the mix.
 * Errors: LBHPDE_ERR_ARG (boundary LBHPDE_PERIODIC or malformed, N too small, phib NULL with
 * nsteps > 0); LBHPDE_ERR_UNSUPPORTED for real-exponent models and for grids the bounded kernel
 * does not hold (N > 2048, or no placement of both ends' extrapolation nodes in one warp). */
int lbhpde_submit_nee(lbhpde_server_t s, const lbhpde_request *req, int boundary, const double *phib,
                      uint64_t *id);
/* Non-blocking.  LBHPDE_PENDING while the request is queued or running (info is filled);
 * otherwise its final status, phi copied to phi_out ([N] host doubles, may be NULL), and the
 * request released (a later poll returns LBHPDE_ERR_NOT_FOUND). */
int lbhpde_poll(lbhpde_server_t s, uint64_t id, double *phi_out, lbhpde_result *info);
/* As lbhpde_poll, waiting at most timeout_s seconds; LBHPDE_ERR_TIMEOUT when it runs out. */
int lbhpde_wait(lbhpde_server_t s, uint64_t id, double timeout_s, double *phi_out, lbhpde_result *info);
int lbhpde_server_stats(lbhpde_server_t s, lbhpde_server_info *out);
/* Stops the scheduler after its current step block and frees everything; requests not yet
 * polled are dropped. */
int lbhpde_server_destroy(lbhpde_server_t s);

/* ------------------------------------------------- diagnostics, no allocation */

/* Largest N lbhpde_phi_diagnostics_noalloc accepts (2^24 nodes). */
#define LBHPDE_NOALLOC_MAX_NODES 16777216L

/* The diagnostics reduction of lbhpde_diagnostics for a phi array the caller owns, in a form
 * that allocates no memory at all.  The paper has no counterpart: this entry point exists for
 * callers that cannot let a library call cudaMalloc -- applications that reserve all device
 * memory up front for their own pool, or latency-critical loops where the implicit
 * device-wide synchronisation of cudaMalloc/cudaFree is not acceptable.
 *   phi_device      [N] doubles in device memory (e.g. from lbhpde_read_phi with out_on_device)
 *   N               1 .. LBHPDE_NOALLOC_MAX_NODES; larger N returns LBHPDE_ERR_ARG
 *   phistar_device  [N] doubles in device memory, or NULL (then err_E = err_L2 = 0)
 *   out             host record; steps is set to 0
 *   cuda_stream     stream for the two kernels and the copy of the result (NULL = legacy)
 * The per-block partial sums live in a file-scope device array of about 1 MiB that every GPU
 * loading the library keeps until the process exits.  The first call on a device (with that
 * device current) looks up the array's device address and keeps it for the life of the
 * process; make that first call before any stream capture, and make no call on a device after
 * cudaDeviceReset() on it in the same process (the kept address belonged to the context the
 * reset destroyed).  Every call writes each record it reads, so nothing is carried over between
 * calls, but all calls share the one array: calls that overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.  The call synchronises
 * cuda_stream.  Returns LBHPDE_ERR_DIVERGED (after filling out) if phi has a non-finite
 * value, LBHPDE_ERR_CUDA if a CUDA call fails.  Calls no cudaMalloc, cudaFree or allocating
 * library routine. */
int lbhpde_phi_diagnostics_noalloc(const double *phi_device, long N, const double *phistar_device,
                                   lbhpde_diag *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* LBHPDE_H */
