/*
 * fdwave.h - C ABI of the GB300 shaped-stencil acoustic wave library
 * (libfdwave.so, built for sm_103a).
 *
 * The library advances the constant-density acoustic wave equation with a
 * damping (sponge) term,
 *     u_tt + eta(x) u_t - c(x)^2 Lap u = f(x, t)            (paper Eq. wave_eq
 *                                                             and Section 3.1)
 * with the centred second-order leapfrog in time (Eq. time_derivative1) and a
 * symmetric shaped Laplacian stencil of radius M in space
 * (Eq. spacexz_derivative2_sym; shapes of Section 4.1; weight schemes of
 * Sections 3.3-3.4), on a regular grid of spacing h and time step tau.
 *
 * Discrete step on the padded grid (field zero outside it):
 *   u^{n+1} = [2 u^n - (1 - g) u^{n-1} + k * sum_o a_o u^n(x + o) + a_src^n] / (1 + g)
 * with k = (c tau / h)^2 per node, g = eta tau / 2, a_o the orbit weights
 * (the Laplacian is h^-2 sum_o a_o u(x+o)), a_src^n = tau^2 s(t^n) / h^dim at
 * a source node.  Traces: trace[n][r] = u^{n+1} at receiver r.
 *
 * Conventions for every call:
 *   - Layout: 2D arrays are [z][x], 3D arrays are [z][y][x], x contiguous,
 *     row-major, FP32 unless stated.  "Physical" arrays have the problem's
 *     n[] nodes per axis; "padded" arrays have n[] + 2 nb nodes per axis.
 *   - Indices of sources/receivers are linear row-major indices into the
 *     physical grid, int64, HOST memory.
 *   - Pointers suffixed _d are device pointers (cudaMalloc'd or torch
 *     tensors); the caller owns all memory.  The library never allocates
 *     device memory except where a call says so: scratch comes from a
 *     caller-provided workspace of the size the *_workspace_size call gives,
 *     256-byte aligned.
 *   - All device work is enqueued on the caller's stream (a cudaStream_t,
 *     NULL for the legacy default stream) and is asynchronous; host-side
 *     argument errors are reported synchronously.
 *   - Errors: every call returns an fd_status; nothing is thrown across the
 *     ABI.  fd_last_error() gives a thread-local message for the last failing
 *     call of the calling thread.  Conditions detected on the device (time-out
 *     of a bounded wait, a velocity above vmax, a wavefield that grew beyond
 *     1e30 or became non-finite, checked every 32 steps and at the last step)
 *     are recorded in a status word in the workspace and returned by
 *     fd_status_read().
 */
#ifndef FDWAVE_H
#define FDWAVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FD_OK = 0,
    FD_ERR_ARG = -1,          /* invalid argument (message in fd_last_error) */
    FD_ERR_CUDA = -2,         /* a CUDA runtime/driver call failed */
    FD_ERR_UNSTABLE = -3,     /* dt above the von Neumann limit, or vmax exceeded */
    FD_ERR_SINGULAR = -4,     /* weight system singular / not solvable */
    FD_ERR_TIMEOUT = -5,      /* a bounded device wait expired (kernel returned early) */
    FD_ERR_NOMEM = -6,        /* workspace too small or host allocation failed */
    FD_ERR_UNSUPPORTED = -7   /* combination not implemented */
} fd_status;

/* Stencil shapes of Section 4.1 (3D: union of the 2D shape in the three
 * coordinate planes). */
typedef enum {
    FD_CROSS = 0,             /* axes only, 4M+1 points (2D) */
    FD_CROSS_RHOMBUS = 1,     /* axes to M plus {|p|+|q| <= N} */
    FD_RHOMBUS = 2,           /* {|p|+|q| <= M} */
    FD_CROSS_SQUARE = 3,      /* axes to M plus {min(|p|,|q|) <= N, max <= M} */
    FD_SQUARE = 4             /* {max(|p|,|q|) <= M} */
} fd_shape;

/* Weight schemes of Sections 3.3 (spatial) and 3.4 (dispersion-based). */
typedef enum {
    FD_SPATTE = 0,            /* Taylor, Eq. taylor_system (off-axis weights 0) */
    FD_SPECTE_THETA = 1,      /* polar Taylor at angle theta, Eqs. taylor_system_r*_spec */
    FD_SPECLS = 2,            /* least squares of the spatial symbol, Section 3.3.3 */
    FD_DISPTE = 3,            /* time-space Taylor, Eqs. taylor_system_r*_disp */
    FD_DISPTE_THETA = 4,      /* polar variant at angle theta, Eqs. *_disp_theta */
    FD_DISPLS = 5             /* least squares of the dispersion relation, Section 3.4.3 */
} fd_scheme;

/* Basis of the least-squares schemes: the one the paper adopts (Taylor basis
 * for SpecLS, Eq. taylor_laplacian_spec_disp_linsys; cosine basis for DispLS,
 * Eq. displs_cont_linsys), or either basis explicitly. */
typedef enum { FD_LS_PAPER = 0, FD_LS_TAYLOR = 1, FD_LS_COSINE = 2 } fd_ls_basis;

typedef struct {
    int32_t dim;              /* 2 or 3 */
    int32_t shape;            /* fd_shape */
    int32_t M;                /* radius, 1 <= M <= 16 */
    int32_t N;                /* inner size of CROSS_RHOMBUS (1..M) / CROSS_SQUARE (0..M) */
    int32_t scheme;           /* fd_scheme */
    int32_t ls_basis;         /* fd_ls_basis (LS schemes only) */
    double courant;           /* C = c_max tau / h for the Disp* schemes (Eq. courant) */
    double theta;             /* wave-number angle of the *_THETA schemes (2D only) */
    double band;              /* LS band: beta = k h in [0, band]; <= 0 selects pi/2 */
} fd_stencil_desc;

/* Maximum number of orbits any supported stencil has. */
#define FD_MAX_ORBITS 160

/*
 * fd_weights - stencil weights, one per symmetry orbit (HOST, FP64, pure).
 * Orbits are keyed by sorted absolute offsets (p >= q >= s >= 0; s = 0 in
 * 2D); orbit 0 is the centre.  mult[i] is the orbit's number of offsets.
 *   desc      stencil description
 *   cap       capacity of the output arrays (>= number of orbits)
 *   n_orbits  out: number of orbits written
 *   orbits    out: [cap][3] (p, q, s)
 *   mult      out: [cap]
 *   w         out: [cap] weights a (the Laplacian is h^-2 sum a u)
 * Errors: FD_ERR_ARG (bad desc or cap), FD_ERR_SINGULAR, FD_ERR_UNSUPPORTED
 * (theta schemes in 3D).
 */
int fd_weights(const fd_stencil_desc *desc, int cap, int *n_orbits,
               int32_t *orbits, int32_t *mult, double *w);

/*
 * fd_cfl_limit - von Neumann stability limit of the leapfrog with this
 * stencil, from the symbol S(k) = sum_o a_o cos(k.o) of Eq. full_disp.  The
 * amplification equation lambda^2 - (2 + C^2 S(k)) lambda + 1 = 0 has both
 * roots on the unit circle iff -4 <= C^2 S(k) <= 0 for every k, so:
 *   - C_max = 2 / sqrt(max_k -S(k)); a run is stable when c_max tau / h <= C_max;
 *   - a stencil whose symbol is positive somewhere (above 1e-9 max(-S), far
 *     beyond the round-off of S(0) = 0) is unstable at every time step and
 *     gets FD_ERR_UNSTABLE (fd_last_error names the wave number).
 * HOST, FP64.  Errors: as fd_weights, and FD_ERR_UNSTABLE.
 */
int fd_cfl_limit(const fd_stencil_desc *desc, double *courant_max);

/*
 * fd_weights_conditioning - how well the system fd_weights solves determines
 * the weights (Section 4.2 names the ill-posed shapes; the LS schemes are
 * solved as minimum-norm least squares):
 *   cond        out: sigma_max / sigma_min of the system's matrix (HUGE_VAL when
 *               a singular value is zero).  LS schemes: the quadrature-weighted
 *               design matrix of Sections 3.3.3 / 3.4.3 (one column per
 *               non-centre orbit); DispTE / theta schemes: the moment or polar
 *               system; SpatTE: the Taylor system of the axis orbits
 *   rank        out: LS: singular values above 1e-10 sigma_max (those the
 *               solution keeps); other schemes: the number of independent
 *               equations
 *   n_unknowns  out: number of unknowns (columns)
 * A rank below n_unknowns means the minimum-norm choice, not the equations,
 * fixes part of the weights.  HOST, FP64.  Errors: as fd_weights.
 */
int fd_weights_conditioning(const fd_stencil_desc *desc, double *cond, int *rank,
                            int *n_unknowns);

/*
 * fd_ricker - Ricker wavelet s(t^n), t^n = n dt, n = 0..nt-1, with peak
 * frequency f0 and delay 1/f0 (the source named in Section 3.1):
 * s(t) = (1 - 2 pi^2 f0^2 (t - 1/f0)^2) exp(-pi^2 f0^2 (t - 1/f0)^2).
 * out: HOST float[nt].  Errors: FD_ERR_ARG.
 */
int fd_ricker(double f0, double dt, int nt, float *out);

/* Problem on the physical grid; the sponge of nb nodes is added per side. */
typedef struct {
    int32_t dim;              /* 2 or 3 */
    int32_t nb;               /* sponge width in nodes (>= 0) */
    int64_t n[3];             /* physical nodes (nz, ny, nx); ny = 1 in 2D */
    int32_t nt;               /* number of time steps */
    int32_t reserved;
    double h;                 /* grid spacing (m) */
    double dt;                /* time step tau (s) */
    double vmax;              /* largest velocity of any model used (m/s) */
    double damp_R;            /* sponge reflection target R (<= 0 selects 1e-3):
                                 eta(d) = eta_max (d/nb)^2 summed over axes,
                                 eta_max = 3 vmax ln(1/R) / (2 nb h) */
} fd_problem;

typedef struct fd_plan fd_plan;

/* Model parameterisation of the model_d arrays. */
typedef enum { FD_MODEL_VELOCITY = 0, FD_MODEL_SLOWNESS2 = 1 } fd_model_kind;

/*
 * fd_plan_create - validate a problem and stencil, solve the weights (host
 * FP64, rounded to FP32 for the kernels), check vmax dt / h <= C_max of
 * fd_cfl_limit (FD_ERR_UNSTABLE otherwise, and for a stencil that no time
 * step makes stable) and choose the kernel variant.  The plan owns
 * only host memory.  Errors: FD_ERR_ARG, FD_ERR_UNSTABLE, FD_ERR_SINGULAR,
 * FD_ERR_UNSUPPORTED, FD_ERR_NOMEM.
 */
int fd_plan_create(const fd_problem *prob, const fd_stencil_desc *stencil, fd_plan **out);
void fd_plan_destroy(fd_plan *plan);

typedef struct {
    int64_t padded[3];        /* padded nodes per axis (nz, ny, nx) */
    int64_t pitch;            /* row pitch (floats) of the internal field buffers */
    int32_t n_orbits;         /* orbits of the stencil (after zero-weight reduction) */
    int32_t kernel;           /* kernel variant id chosen by the plan */
    double courant_max;       /* fd_cfl_limit of the stencil */
    int32_t tile[3];          /* tile (x, y/z, z-chunk) of the chosen variant */
    int32_t effective_shape;  /* shape after dropping all-zero off-axis orbits */
} fd_plan_info;
int fd_plan_get_info(const fd_plan *plan, fd_plan_info *info);

/*
 * fd_plan_autotune - pick the plan's kernel variant by measurement: each
 * candidate tile shape (rows per thread in 2D; y tile and z-chunk length in
 * 3D) is timed per step on this plan's problem on `model_d` with no sources
 * or receivers (best of three 64-step runs minus best of three 16-step runs,
 * over 48, as captured graphs); a candidate must be 2 % faster than the best
 * before it to replace it; the choice is kept in the plan and in a
 * per-process cache
 * keyed by device name, dimension, shape, M, N and padded size (appended to
 * the file named by the environment variable FDWAVE_TUNE_CACHE, and read
 * from it, when that is set).  Synchronises `stream`.  Results of the plan's
 * calls do not depend on the variant.  ws_d: >= fd_forward_workspace_size(plan,
 * 0, 0) + 1 KiB.  Errors: FD_ERR_ARG, FD_ERR_NOMEM, FD_ERR_CUDA.
 */
int fd_plan_autotune(fd_plan *plan, int model_kind, const float *model_d, void *ws_d,
                     size_t ws_bytes, void *stream);

/*
 * fd_plan_variants / fd_plan_set_variant - the kernel variants built for the
 * plan's stencil, and choosing one by hand instead of the default or
 * fd_plan_autotune (the paper has no counterpart: these are schedules of the
 * same arithmetic, and results do not depend on the variant).
 *   2D: rows per thread R (1, 2 or 4) of the 64 x 16R tile.
 *   3D: rows TY (8 or 16) of the 64 x TY column a CTA marches in z.
 * fd_plan_variants writes up to cap entries and sets n to the number built
 * (0 for the generic 2D kernel).  fd_plan_set_variant takes one of them and
 * a z-chunk in planes per CTA (3D; 0 lets the cost model choose).
 * Errors: FD_ERR_ARG, FD_ERR_UNSUPPORTED (variant not built).
 */
int fd_plan_variants(const fd_plan *plan, int cap, int *n, int *variants);
int fd_plan_set_variant(fd_plan *plan, int variant, int z_chunk);

/*
 * fd_forward_workspace_size - bytes of device workspace fd_forward needs for
 * nsrc sources and nrec receivers (three padded field buffers, tile-bucketed
 * source/receiver tables, the status word).  The tables are sized for the
 * plan's largest tile count, so the size does not depend on the kernel
 * variant fd_plan_autotune chooses.
 */
int fd_forward_workspace_size(const fd_plan *plan, int nsrc, int nrec, size_t *bytes);

/*
 * fd_forward - run the plan's nt steps from u^0 = u^{-1} = 0 (or a given
 * state), injecting sources and recording traces (Section 3.1, Data objects of
 * Section 5.2).
 *   model_kind  fd_model_kind of model_d
 *   model_d     physical [nz][ny][nx] velocity (m/s) or slowness squared m = 1/v^2
 *   nsrc, src_idx    sources: HOST int64 physical linear indices
 *   wavelet_d   [nt][nsrc] source time functions s(t^n) (e.g. fd_ricker)
 *   nrec, rec_idx    receivers: HOST int64 physical linear indices
 *   traces_d    out [nt][nrec]: u^{n+1} at the receivers (may be NULL if nrec = 0)
 *   state_in_d  NULL for zero initial state, else padded [2][..] = (u^0, u^{-1})
 *   state_out_d NULL, or out padded [2][..] = (u^{nt}, u^{nt-1})
 *   ws_d, ws_bytes   workspace (>= fd_forward_workspace_size)
 *   stream      cudaStream_t
 * The model's maximum must not exceed the plan's vmax; a larger value is
 * recorded in the status word (FD_ERR_UNSTABLE from fd_status_read).
 */
int fd_forward(fd_plan *plan, int model_kind, const float *model_d,
               int nsrc, const int64_t *src_idx, const float *wavelet_d,
               int nrec, const int64_t *rec_idx, float *traces_d,
               const float *state_in_d, float *state_out_d,
               void *ws_d, size_t ws_bytes, void *stream);

/*
 * fd_status_read - synchronise `stream` and return the device status word of
 * the last call that used workspace ws_d, then clear it:
 *   FD_ERR_TIMEOUT   a bounded device wait gave up (the kernel returned early;
 *                    the results of that call are not valid);
 *   FD_ERR_UNSTABLE  the model exceeded the plan's vmax, or the wavefield grew
 *                    without bound (|u| > 1e30 or non-finite at a checked step:
 *                    every 32nd step and the last; the gradient checks its
 *                    forward and adjoint sweeps);
 *   FD_OK            none of these.
 * This is how the von Neumann analysis of Eq. full_disp is enforced at run
 * time for models and states the plan's checks did not see.
 */
int fd_status_read(const fd_plan *plan, void *ws_d, void *stream);

/*
 * fd_gradient_workspace_size / fd_adjoint_gradient - gradient of a misfit
 * J(traces) with respect to m = 1/v^2 on the physical grid by the exact
 * discrete adjoint of the step above (the paper names FWI as the target use,
 * Section 1 and 7; the adjoint is derived from the discrete step).
 *   resid_d     [nt][nrec] dJ/dtrace (for J = 1/2 ||d - d_obs||^2: d - d_obs)
 *   ckpt_every  k >= 1: the forward sweep stores (u^n, u^{n-1}) every k steps;
 *               the backward sweep recomputes each segment of k steps and runs
 *               the adjoint steps over it.  k >= nt keeps the D field of every
 *               step (nt fields, e.g. 124 GB for 296^3 x 1200 steps): the
 *               forward sweep stores D itself, with no checkpoint and no
 *               recompute.  The gradient is bitwise the same for every k.
 *   grad_d      out physical [nz][ny][nx] dJ/dm (overwritten)
 *   traces_d    optional out [nt][nrec] traces of the forward sweep (NULL: none)
 *   wavelet_grad_d  optional out [nt][nsrc] dJ/ds(t^n) for each source, the
 *               adjoint of the source-injection map (NULL: none)
 * Other arguments as fd_forward.  Workspace: three field buffers, (2 nt/k)
 * checkpoint fields, k segment fields and the gradient accumulator.
 */
int fd_gradient_workspace_size(const fd_plan *plan, int nsrc, int nrec, int ckpt_every,
                               size_t *bytes);
int fd_adjoint_gradient(fd_plan *plan, int model_kind, const float *model_d,
                        int nsrc, const int64_t *src_idx, const float *wavelet_d,
                        int nrec, const int64_t *rec_idx, const float *resid_d,
                        int ckpt_every, float *grad_d, float *traces_d,
                        float *wavelet_grad_d, void *ws_d, size_t ws_bytes, void *stream);

/*
 * fd_gradient_forward / fd_gradient_adjoint - fd_adjoint_gradient with
 * ckpt_every = nt split in two calls, for callers that need the traces before
 * they can form the residual (a misfit J(d, d_obs), an autograd backward).  No
 * counterpart in the paper (whose FWI outlook implies the same gradient).
 * fd_gradient_forward runs the forward sweep, writes the traces (traces_d
 * optional) and keeps the D field of every step in ws_d;
 * fd_gradient_adjoint then runs the adjoint sweep from them for a residual and
 * writes dJ/dm (and dJ/ds if wavelet_grad_d is not NULL).  The forward sweep
 * is not repeated, so a misfit gradient costs one forward and one adjoint
 * sweep.  Both calls take the same plan, sources, receivers and workspace,
 * sized by fd_gradient_workspace_size with ckpt_every = nt; nothing may write
 * ws_d in between, and fd_gradient_adjoint may be called several times (other
 * residuals) after one fd_gradient_forward.  The gradient and traces are
 * bitwise those of fd_adjoint_gradient.  A plan keeps up to 64 stored
 * forwards (workspace and a hash of the source and receiver indices), so the
 * forwards of several shots may precede their adjoints.  Errors: as
 * fd_adjoint_gradient, and FD_ERR_ARG from fd_gradient_adjoint when no stored
 * forward of the plan has this workspace and these sources and receivers:
 * none was made, another call on the plan
 * (fd_forward, fd_adjoint_gradient) has since written the workspace, or the
 * kernel variant changed (fd_plan_set_variant, fd_plan_autotune).
 */
int fd_gradient_forward(fd_plan *plan, int model_kind, const float *model_d,
                        int nsrc, const int64_t *src_idx, const float *wavelet_d,
                        int nrec, const int64_t *rec_idx, float *traces_d,
                        void *ws_d, size_t ws_bytes, void *stream);
int fd_gradient_adjoint(fd_plan *plan, int nsrc, const int64_t *src_idx,
                        int nrec, const int64_t *rec_idx, const float *resid_d,
                        float *grad_d, float *wavelet_grad_d,
                        void *ws_d, size_t ws_bytes, void *stream);

/*
 * Batched shots (no counterpart in the paper, whose experiments run one
 * source at a time): independent forward problems, possibly on grids of
 * different size, with the same stencil, dt and nt, advanced together.  For
 * 2D cross stencils with M = 2, 4, 8 each time step is one launch of
 * persistent CTAs over a table of every shot's tiles; other
 * batches launch each shot's step kernel in turn.  The whole time loop is
 * captured once into a CUDA graph and replayed on repeat calls.  Fields of
 * every shot must fit the workspace at once.  With the environment variable
 * FDWAVE_BATCH_2STEP=1, Cross(2) and Cross(4) batches advance two time steps
 * per pass instead (temporal blocking; two more fields per shot in the
 * workspace, same results bit for bit).  With FDWAVE_BATCH_PERSISTENT=1, a
 * single-launch batch runs all nt steps in one cooperative launch, with a
 * bounded grid barrier between steps (same results bit for bit).
 * fd_forward_batched: traces only (no final states).  Errors: FD_ERR_ARG
 * (shots that differ in dim, stencil, dt or nt), FD_ERR_NOMEM, FD_ERR_CUDA.
 */
typedef struct {
    const fd_plan *plan;      /* plan of this shot's grid (shared stencil/dt/nt) */
    int32_t model_kind;
    int32_t nsrc;
    int32_t nrec;
    int32_t reserved;
    const float *model_d;
    const int64_t *src_idx;   /* HOST */
    const float *wavelet_d;   /* [nt][nsrc] */
    const int64_t *rec_idx;   /* HOST */
    float *traces_d;          /* [nt][nrec] */
} fd_shot;

int fd_forward_batched_workspace_size(int nshots, const fd_shot *shots, size_t *bytes);
int fd_forward_batched(int nshots, const fd_shot *shots, void *ws_d, size_t ws_bytes,
                       void *stream);

/*
 * Tile shape of single-launch batches: the batched tile kernel has 64 x 16R
 * tiles with R rows per thread (R = 2 by default, or 4).
 * fd_forward_batched_autotune times each R on this batch (best of three
 * 64-step runs minus best of three 16-step runs, launched step by step,
 * copies of the plans) and keeps the fastest (a candidate must win by 2 %)
 * for batches of the same stencil, shot count and total padded size on this
 * device, for the rest of the process; fd_forward_batched_set_variant sets R
 * by hand.  The batched gradient uses the same choice.  Results do not depend
 * on R.  The workspace sizes above cover every R.  Synchronises `stream`.
 * Errors: FD_ERR_ARG, FD_ERR_NOMEM, FD_ERR_CUDA, FD_ERR_UNSUPPORTED (R not
 * built for the stencil).
 */
int fd_forward_batched_autotune(int nshots, const fd_shot *shots, void *ws_d, size_t ws_bytes,
                                void *stream);
int fd_forward_batched_set_variant(int nshots, const fd_shot *shots, int rows);

/*
 * Batched gradients (the paper has no counterpart; its FWI outlook sums the
 * gradients of many shots): the checkpointed adjoint gradient of
 * fd_adjoint_gradient for several shots in one call, each shot with its own
 * plan (grids may differ; stencil, dt and nt are shared), model, sources,
 * receivers, residuals and gradient output.  For 2D cross stencils with
 * M = 2, 4 or 8 every time step of each sweep is one launch of persistent
 * CTAs over the tiles of every shot; other batches run the shots one after
 * another.  Each shot's gradient (and traces) are bit for bit those of
 * fd_adjoint_gradient with the same ckpt_every (and so with any ckpt_every;
 * ckpt_every >= nt keeps every D and recomputes nothing).  Workspace: every shot's
 * gradient workspace plus the batch's tables.  Device status: the first
 * shot's status word (fd_status_read with the first plan and ws_d).
 * Errors: FD_ERR_ARG (shots that differ in dim, stencil, dt or nt, missing
 * outputs), FD_ERR_NOMEM, FD_ERR_CUDA.
 */
typedef struct {
    const fd_plan *plan;      /* plan of this shot's grid (shared stencil/dt/nt) */
    int32_t model_kind;
    int32_t nsrc;
    int32_t nrec;
    int32_t reserved;
    const float *model_d;
    const int64_t *src_idx;   /* HOST */
    const float *wavelet_d;   /* [nt][nsrc] */
    const int64_t *rec_idx;   /* HOST */
    const float *resid_d;     /* [nt][nrec] dJ/dtrace */
    float *grad_d;            /* out: physical dJ/dm of this shot */
    float *traces_d;          /* optional out [nt][nrec] of the forward sweep (NULL: none) */
} fd_grad_shot;

int fd_adjoint_gradient_batched_workspace_size(int nshots, const fd_grad_shot *shots,
                                               int ckpt_every, size_t *bytes);
int fd_adjoint_gradient_batched(int nshots, const fd_grad_shot *shots, int ckpt_every,
                                void *ws_d, size_t ws_bytes, void *stream);

/*
 * fd_forward_noalloc - fd_forward for callers that cannot allocate device
 * memory (an allocator that owns all device memory, a real-time loop where an
 * allocation would stall, a plugin host that hands out none).  The paper has
 * no counterpart; this is a deployment convenience.
 * Arguments are those of fd_forward without the workspace: the scratch comes
 * from a static device array of 32 MiB compiled into the library, which every
 * GPU that loads the library holds until the process exits.  The call makes
 * no cudaMalloc or cudaFree call, and no allocation through any library; its
 * time steps are launched one by one on `stream` (no CUDA graph is captured
 * or instantiated, no stream is created and the device is not synchronised).
 *   - Problems whose forward workspace (fd_forward_workspace_size) exceeds
 *     32 MiB are rejected with FD_ERR_NOMEM before any device work.
 *   - The first call on a device resolves the array's address on that device
 *     (cudaGetSymbolAddress, with that device current); make that first call
 *     before any stream capture.
 *   - All calls share the array, which keeps the last call's contents.  Each
 *     call clears what must start at zero, but calls that overlap on the GPU
 *     (other streams, other host threads, other plans) race on it: serialise
 *     them.
 *   - Host-side errors are returned; conditions detected on the device go to
 *     a status word in the array, read by fd_status_read_noalloc.
 */
int fd_forward_noalloc(fd_plan *plan, int model_kind, const float *model_d,
                       int nsrc, const int64_t *src_idx, const float *wavelet_d,
                       int nrec, const int64_t *rec_idx, float *traces_d,
                       const float *state_in_d, float *state_out_d, void *stream);

/*
 * fd_status_read_noalloc - fd_status_read for fd_forward_noalloc: synchronise
 * `stream`, return the device status word of the last fd_forward_noalloc call
 * on the current device (FD_OK, FD_ERR_TIMEOUT, FD_ERR_UNSTABLE) and clear it.
 * The paper has no counterpart.  Errors: FD_ERR_ARG, FD_ERR_CUDA.
 */
int fd_status_read_noalloc(const fd_plan *plan, void *stream);

/*
 * Evaluation metrics (Section 2.4 and Appendix A), computed on the GPU in
 * FP64 from FP32 data.  All pointers are DEVICE pointers the caller owns;
 * the calls are asynchronous on `stream` and allocate nothing.
 *
 * fd_error_norms - classical error norms of a numerical data object against a
 * reference (Eqs. snapnorm1, snapnorm2, snapnormmax): out_d[3] = (scale1 *
 * sum |num - ref|, scale2 * sqrt(sum (num - ref)^2), max |num - ref|) over n
 * values.  A 2D snapshot takes scale1 = 1/h^2, scale2 = 1/h; traces and
 * receiver gathers take the paper's analogous factors with tau for h.
 * Errors: FD_ERR_ARG, FD_ERR_CUDA.
 */
int fd_error_norms(const float *num_d, const float *ref_d, int64_t n, double scale1,
                   double scale2, double *out_d, void *stream);

/*
 * fd_dft_gamma - DFT dispersion metric of Appendix A for nrec traces of nt
 * samples, numerical against reference, both [nt][nrec] like the traces of
 * fd_forward:
 *   spec_num_d, spec_ref_d  out [nrec][nfreq] complex (re, im) DFT
 *                 coefficients A_k, k < nfreq (Eq. dft); 16-byte aligned
 *   gamma_d       out [nrec][nfreq] gamma_k (Eq. gammadft), or NULL: phase
 *                 difference num - ref brought into [-pi, pi] by one 2 pi
 *                 shift (Eq. phasesdifdftajusted), over pi, times |A_k^num|
 *                 over the trace's largest |A_k^num|; 0 for a zero trace
 *   norm_d        out [nrec] sqrt(mean_k gamma_k^2) (Eq. norm2gammastdft,
 *                 averaged over the nfreq frequencies computed)
 *   agg_d         out [2] (average, maximum) of norm_d over the receivers
 *                 (Eqs. norm2gammarecdftavg, norm2gammarecdftmax), or NULL
 * 1 <= nfreq <= nt (nt/2 + 1 covers the frequencies of a real trace).
 * Errors: FD_ERR_ARG, FD_ERR_CUDA.
 */
int fd_dft_gamma(const float *num_d, const float *ref_d, int nt, int nrec, int nfreq,
                 double *spec_num_d, double *spec_ref_d, float *gamma_d, double *norm_d,
                 double *agg_d, void *stream);

/*
 * fd_cwt_gamma - wavelet (CWT) dispersion metric of Appendix A for nrec traces
 * of nt samples, numerical against reference, both [nt][nrec].  The printed
 * transform (Eqs. cwt1, cwt) is read as the DFT-based Morlet transform of
 * Torrence and Compo that the appendix follows, one inverse DFT:
 *   S_{n,k} = (1/nt) sum_{k'=1}^{nt/2} A_k' Psi(s_k omega_k') exp(+2 pi i k' n / nt)
 * with A the DFT of Eq. dft, omega_k' = 2 pi k' / (nt tau) (Eq. omegak; the
 * Heaviside factor drops k' = 0 and k' > nt/2), Psi(s omega) = (2 pi s / tau)^(1/2)
 * pi^(-1/4) exp(-(s omega - omega0)^2 / 2) (Eqs. cwt2, cwt3), and scale k >= 1
 * the one whose Fourier period is DFT line k's: s_k omega_k = (omega0 +
 * sqrt(2 + omega0^2)) / 2.  Scale 0 has no finite scale: S_{n,0} = 0.  tau
 * cancels and is not an argument.
 *   omega0        Morlet centre frequency (> 0; 6 is the usual choice)
 *   spec_num_d, spec_ref_d  out [nrec][nt/2 + 1] complex DFT lines (re, im)
 *   cwt_num_d, cwt_ref_d    out [nrec][nscale][nt] complex S_{n,k} (re, im)
 *   gamma_d       out [nrec][nscale][nt] gamma_{n,k} (Eq. gammacwt), or NULL:
 *                 wrapped phase difference num - ref (Eqs. phasesdifcwt,
 *                 phasesdifcwtajusted) over pi, times |S^num_{n,k}| over amax
 *   amax_d        out [nrec] largest |S^num_{n,k}| of each trace (Eq.
 *                 amplmaxcwt); gamma is 0 where it is 0
 *   norm_d        out [nrec] sqrt(mean over n and k of gamma^2) (Eq.
 *                 norm2gammastcwt)
 *   agg_d         out [2] (average, maximum) of norm_d (Eqs.
 *                 norm2gammareccwtavg, norm2gammareccwtmax), or NULL
 * 1 <= nscale <= nt, 1 <= nrec <= 65535, nt <= 29054 (one trace's DFT lines
 * are staged in shared memory).  Cost: nrec nscale nt (nt/2) complex
 * multiply-adds per trace set, in FP64.  All buffers are DEVICE pointers,
 * 16-byte aligned where complex.
 * Errors: FD_ERR_ARG, FD_ERR_CUDA.
 */
int fd_cwt_gamma(const float *num_d, const float *ref_d, int nt, int nrec, int nscale,
                 double omega0, double *spec_num_d, double *spec_ref_d, double *cwt_num_d,
                 double *cwt_ref_d, float *gamma_d, double *amax_d, double *norm_d,
                 double *agg_d, void *stream);

/* Thread-local message of the last failing call ("" if none). */
const char *fd_last_error(void);

/* Library version string. */
const char *fd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FDWAVE_H */
