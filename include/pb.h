/*
 * pb.h -- C ABI of libpb: GB300-native (sm_103a) Jacobi-preconditioned CG for
 * the linear finite-difference Poisson-Boltzmann equation of Qi,
 * Botello-Smith & Luo, "Acceleration of Linear Finite-Difference
 * Poisson-Boltzmann Methods on GPUs" (arXiv:1704.02745).
 *
 * Problem (Sec. 2.1, Eq. 2-4).  On a uniform nx*ny*nz grid of spacing h the
 * library solves the h^2-scaled seven-point discretisation of Eq. (3),
 *
 *   sum over the six edges e of c:  eps_e (phi_c - phi_nb)
 *       + kbar^2 h^2 lambda_c phi_c  =  4 pi q_c / h,
 *
 * i.e. A phi = b of Eq. (4), where eps_e is the dielectric on the edge between
 * two nodes (eps_i(i,j,k) of Eq. 3 sits between (i,j,k) and (i+1,j,k)),
 * lambda is the ion-exclusion mask of Eq. (1)-(2), kbar^2 = eps_out kappa^2
 * collects the coefficients of the linearised Boltzmann term, and q_c is the
 * charge of the cube centred on node c.  Units: lengths in Angstrom, charges
 * in e, phi in e/Angstrom, energies in kcal/mol.
 *
 * Conventions shared by every entry point:
 *  - Node arrays are dense, x fastest: index i + nx*(j + ny*k).
 *  - Every call returns a pb_status.  Nothing calls exit/abort or traps on the
 *    device; pb_last_error() returns a message for the calling thread.
 *  - Host inputs are copied before the call returns.  Device pointers passed
 *    in are borrowed (the caller keeps ownership).  Grids and servers are
 *    owned by the library and freed by pb_free_grid / pb_server_destroy.
 *  - All device work is issued on the context's stream; calls that return
 *    results to the host synchronise that stream.
 */
#ifndef PB_H
#define PB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int pb_status;
enum {
    PB_OK = 0,
    PB_ERR_ARG = 1,           /* bad argument: empty grid, h <= 0, eps <= 0, an atom whose
                                 trilinear cell leaves the grid, unknown enum value */
    PB_ERR_OOM = 2,           /* a device allocation failed */
    PB_ERR_CUDA = 3,          /* a CUDA runtime call failed (message in pb_last_error) */
    PB_ERR_NOT_CONVERGED = 5, /* iteration cap reached before the tolerance */
    PB_ERR_BREAKDOWN = 6,     /* p.Ap <= 0 or a non-finite CG scalar */
    PB_ERR_TIMEOUT = 7,       /* pb_batch_poll: result not ready within the timeout; a solve:
                                 a bounded device wait (a TMA tile load, ~50 ms of clock) gave
                                 up, so the solve could not finish */
    PB_ERR_BUSY = 8,          /* pb_batch_submit: over the memory budget and queue full */
    PB_ERR_NOT_FOUND = 9,     /* unknown ticket */
    PB_ERR_CANCELLED = 10     /* pb_batch_poll: the request was cancelled (pb_batch_cancel) */
};

/* Storage of the dielectric coefficients used by the FP32 operator. */
enum {
    PB_COEF_PACKED = 0, /* one byte per node: six edge flags (eps_in / eps_out) + lambda */
    PB_COEF_F32 = 1,    /* explicit eps_x, eps_y, eps_z and diagonal arrays, FP32 */
    PB_COEF_BF16 = 2,   /* explicit eps arrays in BF16 (exact for eps 1 and 80);
                           the diagonal is rebuilt in FP32 from eps and lambda */
    PB_COEF_F64 = 3     /* explicit arrays in FP64 (used by the FP64 operator) */
};

typedef enum { PB_F64 = 0, PB_F32 = 1 } pb_dtype;

/* Arithmetic of a solve. */
enum {
    PB_PREC_F64 = 0,        /* the paper's PCG (Sec. 2.2) in FP64 throughout */
    PB_PREC_F32 = 1,        /* PCG in FP32 (the paper's precision, Sec. 2.7), result
                               accumulated into FP64 */
    PB_PREC_F32_REFINE = 2  /* FP32 inner PCG, FP64 outer iterative refinement: true
                               residual b - A x, accumulation x += d (not in the paper) */
};

/* NONE: plain CG; JACOBI: M = diag A (Sec. 2.4); GMG: a geometric-multigrid
 * V-cycle (Sec. 2 lists GMG; Sec. 4 names multigrid as the next step): coarse
 * levels rediscretised at 2h with series-combined edges, trilinear transfer,
 * two damped-Jacobi sweeps before and after, the outer CG in FP64 (its
 * scalars on the device, iterations launched as CUDA graphs of three) and the
 * V-cycle in FP32 whatever opts->precision says; free-space boundary only,
 * not served by pb_server. */
enum { PB_PRECOND_NONE = 0, PB_PRECOND_JACOBI = 1, PB_PRECOND_GMG = 2 };

/* Grid and physical parameters (Sec. 2.7: h = 0.5 A, eps 1 / 80, phi0 = 0). */
typedef struct {
    int nx, ny, nz;           /* nodes per axis, each >= 1 */
    double h;                 /* spacing, A, > 0 */
    double origin[3];         /* position of node (0,0,0), A */
    double eps_in, eps_out;   /* solute / solvent dielectric, > 0 */
    double ionic_strength;    /* mol/L of 1:1 salt, >= 0 */
    double temperature;       /* K, > 0 */
    int kappa_mask;           /* 1: lambda = 0 at nodes strictly inside an atom; 0: lambda = 1 */
    int coef;                 /* PB_COEF_*: storage of the FP32 operator's coefficients */
    int dh_precision;         /* pb_dtype of the Debye-Hueckel boundary sum */
    int periodic;             /* 1: every axis periodic with period n*h (the periodic boundary
                                 of Fig. 2): node i's neighbours are i-1, i+1 modulo n, an edge
                                 or node is inside an atom if some periodic image is, charges
                                 spread modulo n, no boundary sum.  Needs n >= 3 per axis and
                                 ionic_strength > 0 (without salt, or with every node inside
                                 an atom under kappa_mask, A is singular) */
    int eps_model;            /* PB_EPS_*: the boundary dielectric (Sec. 2.7) */
} pb_grid_desc;

/* Boundary dielectric.  MIDPOINT: an edge takes eps_in when its midpoint is
 * strictly inside an atom sphere, else eps_out (the packed one-byte map).
 * HARMONIC: the weighted harmonic average Sec. 2.7 uses, 1 / (w/eps_in +
 * (1-w)/eps_out) with w the fraction of the edge strictly inside the union of
 * the spheres; needs explicit coefficients (coef F32, BF16 or F64: the FP32
 * inner solve keeps FP32 or BF16 copies, the FP64 residual and FP64 solves
 * the FP64 edges) and the free-space boundary; not served by pb_server. */
enum { PB_EPS_MIDPOINT = 0, PB_EPS_HARMONIC = 1 };

typedef struct {
    int precond;      /* PB_PRECOND_* (Sec. 2.4: Jacobi, M = diag A; or multigrid) */
    int precision;    /* PB_PREC_* */
    double rel_tol;   /* stop when ||r|| / ||b|| < rel_tol (Sec. 2.2 stopping rule) */
    int max_iter;     /* cap on CG iterations summed over all inner solves */
    double inner_tol; /* PB_PREC_F32_REFINE: inner solve to ||r_in|| / ||r_outer|| < inner_tol */
    int max_outer;    /* PB_PREC_F32_REFINE: cap on inner solves */
    int warm_start;   /* 1: phi holds phi0 on entry; 0: phi0 = 0 */
    int poll_every;   /* CG iterations per device-graph launch between host checks (0: auto) */
    int profile;      /* 1: launch kernels one by one with CUDA events around each and report
                         their device time in pb_solve_info (slower; for measurement only) */
} pb_solve_opts;

typedef struct {
    int status;          /* pb_status of the solve */
    int iterations;      /* CG iterations (alpha updates), summed over inner solves */
    int outer_steps;     /* inner solves run (1 for PB_PREC_F64 / PB_PREC_F32) */
    double relres;       /* recursive residual of the last inner solve, relative to its rhs */
    double relres_true;  /* ||b - A phi|| / ||b|| evaluated in FP64 at exit */
    /* profile = 1 only: summed device time (ms) and count of the launches of
     * the stencil pass doing CG work, of the update pass doing CG work, and of
     * the residual pass doing the FP64 residual (refinement) work */
    double ms_stencil, ms_update, ms_resid;
    int n_stencil, n_update, n_resid;
} pb_solve_info;

typedef struct pb_ctx pb_ctx;
typedef struct pb_grid pb_grid;
typedef struct pb_server pb_server;

/* Message of the last failed call on this thread ("" if none). */
const char *pb_last_error(void);

/* Context on CUDA device `device`, issuing work on `cuda_stream` (a
 * cudaStream_t, borrowed).  NULL: the context creates and owns a
 * non-blocking stream (the legacy default stream cannot hold device graphs). */
pb_status pb_create(pb_ctx **out, int device, void *cuda_stream);
pb_status pb_destroy(pb_ctx *ctx);

/* Running totals of a context since pb_create: CUDA kernels the library has
 * launched on the device (kernels inside device graphs counted one by one),
 * and bytes it copied host->device and device->host.  Any pointer may be NULL. */
pb_status pb_ctx_stats(pb_ctx *ctx, uint64_t *kernel_launches, uint64_t *h2d_bytes,
                       uint64_t *d2h_bytes);

/* Measured arithmetic rates of ctx's device (the paper has no counterpart: its
 * solver ran in FP32 on a GPU of its day).  A pure FMA loop -- eight
 * independent chains per thread, one store per thread, a full wave of CTAs --
 * timed with CUDA events, best of three launches after one untimed; FMAs per
 * second in FP64 and FP32.  It is the roofline of the kernels whose FP64
 * arithmetic sets their time (the FP64 true residual of the refinement, plain
 * FP64 solves).  Allocates and frees a small device buffer; synchronises the
 * context's stream.  Errors: PB_ERR_ARG (NULL), PB_ERR_OOM, PB_ERR_CUDA. */
typedef struct {
    double fp64_fma_per_s, fp32_fma_per_s;
    int sms;                 /* streaming multiprocessors of the device */
    double sm_max_mhz;       /* the device's maximum SM clock */
} pb_alu_rates;
pb_status pb_measure_alu(pb_ctx *ctx, pb_alu_rates *out);

/* Grid setup on the device (Eq. 3 coefficients; Sec. 2.7 conditions):
 *  - eps on every edge: eps_in when the edge midpoint lies strictly inside an
 *    atom sphere (|m - x_a|^2 < r_a^2), else eps_out;
 *  - lambda = 0 at nodes strictly inside an atom (kappa_mask), else 1;
 *  - grid charges by trilinear spreading, b = 4 pi q_node / h;
 *  - Debye-Hueckel Dirichlet values on the ghost faces,
 *    phi_g = sum_a q_a exp(-kappa r) / (eps_out r), folded into b.
 * xyz (n_atoms x 3), q and radius are HOST arrays, copied.  n_atoms may be 0.
 * On success *out owns all device arrays of the grid.  PB_ERR_ARG if an
 * atom's trilinear cell leaves the grid. */
pb_status pb_setup_grid(pb_ctx *ctx, const pb_grid_desc *desc, int n_atoms, const double *xyz,
                        const double *q, const double *radius, pb_grid **out);
pb_status pb_free_grid(pb_grid *grid);

/* Redo the setup of an existing grid for new atoms (a new snapshot of the same
 * molecule on the same grid): same steps as pb_setup_grid, no allocation
 * unless n_atoms exceeds every earlier call's.  Host arrays, copied.  The
 * grid's solve workspace is kept, so the next pb_pcg_solve may warm-start. */
pb_status pb_grid_update_atoms(pb_grid *grid, int n_atoms, const double *xyz, const double *q,
                               const double *radius);

/* Au = A u (Eq. 3-4, h^2-scaled; ghost values excluded: they live in b).
 * u and Au are DEVICE arrays of nx*ny*nz elements of `dtype`, borrowed.
 * PB_F64 uses the exact FP64 coefficients; PB_F32 uses the grid's FP32
 * coefficient storage (desc.coef). */
pb_status pb_apply_operator(pb_grid *grid, const void *u, void *Au, int dtype);

/* Solve A phi = b (Sec. 2.2 preconditioned CG with the Jacobi preconditioner
 * of Sec. 2.4, or plain CG).  phi is a DEVICE array of nx*ny*nz doubles,
 * borrowed: phi0 on entry if opts->warm_start, the solution on return.
 * Returns the solve's status (also in info->status). */
pb_status pb_pcg_solve(pb_grid *grid, const pb_solve_opts *opts, double *phi,
                       pb_solve_info *info);

/* Autotuner of a grid's stencil tile plan (the paper has no counterpart: its
 * SpMV is a library call).  Times the stencil pass of each candidate plan --
 * the fewest x tiles or one more, three tile heights, two z chunkings, and
 * the analytic default -- on this grid with the kernels of `precision`
 * (PB_PREC_*), keeps the fastest, and reports it in *info (may be NULL).
 * The grid's later solves use that plan; their results do not depend on it
 * beyond the order of the partial sums.  The grid's internal work vectors
 * are scratch to the timing runs; its setup and the caller's arrays are
 * untouched.  Errors: PB_ERR_ARG (NULL grid, bad precision), PB_ERR_OOM,
 * PB_ERR_CUDA. */
typedef struct {
    int W, H, tz, n_tiles;      /* the plan kept: tile width, height, z planes, tiles */
    int candidates;             /* plans timed */
    double us_default, us_best; /* stencil pass (microseconds): default plan, plan kept */
} pb_tune_info;
pb_status pb_grid_autotune(pb_grid *grid, int precision, pb_tune_info *info);

/* Electrostatic energy 1/2 * 332.0637 * sum_nodes q_node phi_node (kcal/mol)
 * of a DEVICE potential phi (nx*ny*nz doubles, borrowed); the energies that
 * Sec. 3.1 compares.  Evaluated in FP64 as sum_atoms q_a * (trilinear
 * interpolation of phi at x_a), the adjoint of the charge spreading. */
pb_status pb_energy(pb_grid *grid, const double *phi, double *energy_kcal);

/* Electrostatic solvation energy, the quantity Sec. 3.1 (Figs. 1-2) compares:
 * dG = E_solv - E_ref (kcal/mol), where E_solv is the energy of the solved
 * system `desc` and E_ref that of the reference system with eps_out replaced
 * by eps_in (the solute's own dielectric everywhere) and no salt, on the same
 * grid and atoms.  Runs setup, solve (opts) and energy for the solvated
 * system, then for the reference system cold-started; one grid is held at a
 * time.  phi: DEVICE array of nx*ny*nz doubles, borrowed: phi0 of the
 * solvated solve if opts->warm_start, its solution on return.  Returns the
 * first non-OK solve status (the results are still filled in).  A periodic
 * desc is PB_ERR_ARG: its reference system (no salt) has a singular A. */
typedef struct {
    double dG, e_solv, e_ref;   /* kcal/mol */
    pb_solve_info solv, ref;    /* the two solves */
} pb_solvation;
pb_status pb_solvation_energy(pb_ctx *ctx, const pb_grid_desc *desc, int n_atoms,
                              const double *xyz, const double *q, const double *radius,
                              const pb_solve_opts *opts, double *phi, pb_solvation *out);

/* Export a setup array to HOST memory for inspection (dense layouts):
 *   PB_EXPORT_EPS_X  double (nz, ny, nx+1): edge between x-nodes i-1 and i at [.., i]
 *   PB_EXPORT_EPS_Y  double (nz, ny+1, nx)
 *   PB_EXPORT_EPS_Z  double (nz+1, ny, nx)
 *   PB_EXPORT_LAMBDA uint8  (nz, ny, nx)
 *   PB_EXPORT_B      double (nz, ny, nx)
 *   PB_EXPORT_GHOST  double, faces x-, x+ (nz, ny), y-, y+ (nz, nx), z-, z+ (ny, nx)
 * `bytes` must equal the array's size. */
enum { PB_EXPORT_EPS_X = 0, PB_EXPORT_EPS_Y = 1, PB_EXPORT_EPS_Z = 2, PB_EXPORT_LAMBDA = 3,
       PB_EXPORT_B = 4, PB_EXPORT_GHOST = 5 };
pb_status pb_grid_export(pb_grid *grid, int what, void *host_dst, size_t bytes);

/* Device bytes a grid of these dimensions holds after setup and a solve of
 * `precision` (the admission model of the server). */
size_t pb_grid_bytes(const pb_grid_desc *desc, int precision);

/* Energy of a potential with no device allocation.  The paper has no
 * counterpart: this is for callers that cannot allocate device memory -- for
 * example an MD engine whose memory manager owns all device memory, or a
 * time-critical loop in which cudaMalloc / cudaFree (which synchronise the
 * device) are not allowed.  It computes what pb_energy computes,
 * 1/2 * 332.0637 * sum_atoms q_a * (trilinear interpolation of phi at x_a),
 * from the caller's arrays only:
 *   xyzq    DEVICE array, n_atoms x 4 doubles (x, y, z, charge), 32-byte aligned
 *   nx, ny, nz, h, origin[3] (HOST)  the grid of phi (as pb_grid_desc)
 *   phi     DEVICE array of nx*ny*nz doubles, x fastest
 *   energy  DEVICE pointer to one double that receives the result
 *   cuda_stream  stream to run on (NULL: the legacy default stream)
 * Work is queued on the stream; the call does not wait for it.  The
 * reduction's partial sums use a fixed array inside the library's device
 * memory (room for n_atoms <= 1,048,576; larger returns PB_ERR_ARG).  The
 * first call on a device looks up that array's device address (make it
 * before any stream capture); every later call on that device reuses it.
 * That cached address assumes one CUDA context per device for the life of
 * the process (the runtime's primary context): after cudaDeviceReset, or if
 * the caller switches the device to another context, the cached address is
 * stale and must not be used -- such callers should not use this entry
 * point.  All calls share the array, so calls that overlap on the GPU race. */
pb_status pb_energy_noalloc(int n_atoms, const double *xyzq, int nx, int ny, int nz, double h,
                            const double *origin, const double *phi, double *energy,
                            void *cuda_stream);

/* ------------------------------------------------------------------------ */
/* Continuous-batching server.  The paper's motivation is PB on thousands to
 * millions of MD snapshots (Sec. 1); the server solves many snapshots at once:
 * requests are admitted as device memory allows, grids stay resident per
 * trajectory (a snapshot warm-starts from the trajectory's latest solution;
 * snapshots of one trajectory may solve at the same time on separate grids),
 * and all active grids advance together through the same persistent phase
 * kernels, each under its own convergence mask.  A result
 * does not depend on which other requests share the device (each grid's
 * reductions are summed in its own fixed order). */

typedef struct {
    int64_t trajectory_id;   /* snapshots of one trajectory share a resident grid; -1: none */
    pb_grid_desc desc;       /* grid of this snapshot (a trajectory keeps one desc) */
    int n_atoms;
    const double *xyz, *q, *radius; /* HOST arrays, copied by pb_batch_submit */
    double *phi_out;         /* optional HOST buffer of nx*ny*nz doubles that receives phi;
                                borrowed until pb_batch_poll returns the result.  Page-
                                locked memory (pb_pinned_alloc, cudaHostAlloc) takes the
                                device's copy directly, beside the next solves; pageable
                                memory is filled from a pinned staging copy by the
                                server's worker thread */
} pb_request;

/* Page-locked host memory for phi_out buffers (cudaHostAlloc; the paper has
 * no counterpart).  pb_pinned_alloc: *out = bytes of page-locked memory,
 * PB_ERR_OOM if none is left.  pb_pinned_free: releases a pointer that
 * pb_pinned_alloc returned (NULL: no-op). */
pb_status pb_pinned_alloc(size_t bytes, void **out);
pb_status pb_pinned_free(void *p);

typedef struct {
    int status;              /* pb_status of the request */
    double energy;           /* kcal/mol, as pb_energy */
    pb_solve_info info;
    double seconds;          /* submit -> result ready (host clock) */
    int warm_started;        /* 1 if the solve started from the trajectory's last solution */
} pb_result;

/* Server on ctx's device with a device-memory budget (bytes; grids are
 * admitted while the sum of pb_grid_bytes stays within it) and the solve
 * options applied to every request (precision, preconditioner, tolerances;
 * warm_start = 1: later snapshots of a trajectory start from its last
 * solution).  NULL opts: FP32 + FP64 refinement, Jacobi, rel_tol 1e-6.  The
 * server runs a worker thread; pb_server_destroy stops it and frees all.
 * Failures reach the requests they concern, and the server goes on serving:
 * a grid the device has no memory for (after idle grids are released and the
 * allocation retried once) fails its request with PB_ERR_OOM; a timed-out
 * device wait in a batch fails every solve then on the device with
 * PB_ERR_TIMEOUT (their grids are released). */
pb_status pb_server_create(pb_ctx *ctx, size_t hbm_budget_bytes, const pb_solve_opts *opts,
                           pb_server **out);
pb_status pb_server_destroy(pb_server *server);
/* Queue a request (inputs copied).  PB_ERR_BUSY when the queue is full;
 * PB_ERR_ARG for a bad request (checked on the host before queueing). */
pb_status pb_batch_submit(pb_server *server, const pb_request *req, uint64_t *ticket);
/* Wait up to timeout_ms (0: do not wait; < 0: wait until ready) for a
 * ticket.  PB_OK when the result is handed out (the ticket is then spent);
 * the request's own outcome is result->status (PB_OK, or e.g. PB_ERR_ARG,
 * PB_ERR_OOM, PB_ERR_TIMEOUT for a timed-out device wait, PB_ERR_CANCELLED).
 * PB_ERR_TIMEOUT if not ready within timeout_ms (the ticket stays valid);
 * PB_ERR_NOT_FOUND for an unknown or already returned ticket.  Never blocks
 * forever when timeout_ms >= 0. */
pb_status pb_batch_poll(pb_server *server, uint64_t ticket, int timeout_ms, pb_result *result);
/* Cancel a request (the paper has no counterpart).  A request still queued
 * leaves the queue; one on the device is stopped at the worker's next round
 * (between graph launches), and its grid stays resident for the trajectory's
 * next snapshot (which then starts cold).  *cancelled (may be NULL) = 1: the
 * request's pb_batch_poll returns PB_ERR_CANCELLED, with no energy and phi_out
 * unwritten; 0: its result was complete already and stands.  PB_ERR_NOT_FOUND
 * for an unknown or already returned ticket.  Never blocks on the device. */
pb_status pb_batch_cancel(pb_server *server, uint64_t ticket, int *cancelled);
/* Counters: requests queued, active on the device, grids resident, bytes
 * resident, solves completed.  Any pointer may be NULL. */
pb_status pb_server_stats(pb_server *server, int *queued, int *active, int *resident,
                          size_t *bytes_resident, uint64_t *completed);

/* Tile plan of a server's batch (the paper has no counterpart: its SpMV was a
 * library call).  Every grid of the batch is cut into W x H column tiles --
 * the fewest tiles of width <= 64 across x, then height_pct percent of the
 * tallest height a tile of that width allows (W*H <= 1024) -- and the columns
 * into z chunks of at least min_planes planes (as many chunks as fill the
 * device's resident stencil CTAs, no more).  occupancy: resident CTAs per SM
 * of the stencil pass, 3 (the batch build) or 2 (the build whose shared
 * memory admits two).  Results do not depend on the plan beyond the order of
 * the partial sums of each reduction.  Default: {32, 100, 3}. */
typedef struct {
    int min_planes;   /* >= 1 */
    int height_pct;   /* 1 .. 100 */
    int occupancy;    /* 2 or 3 */
} pb_batch_plan;
/* Use `plan` for the batch from the worker's next round on (every resident
 * grid is re-planned between graph launches; solves in flight continue).
 * PB_ERR_ARG for an out-of-range field. */
pb_status pb_server_set_plan(pb_server *server, const pb_batch_plan *plan);

/* Autotuner of the batch's tile plan, on the live batch.  At the worker's
 * next round with solves on the device, every candidate plan -- min_planes
 * 16, 32, 64, 128 or whole grids; height_pct 100 or 67; occupancy 3 or 2 --
 * is applied to all active grids in turn and the stencil and update passes
 * of two CG ticks are timed with CUDA events (the solves advance meanwhile);
 * the four fastest by HBM bytes per second are timed again, and the fastest
 * plan is kept for the batch and for grids admitted later.  Waits up to
 * timeout_ms (< 0: without limit) for the tuning to finish; PB_ERR_TIMEOUT if
 * it has not (it still runs once a batch is active).  *out (may be NULL):
 * the plan kept, and bytes per second of the default and of the kept plan. */
typedef struct {
    pb_batch_plan plan;                /* the plan kept */
    int candidates;                    /* plans timed */
    double gbs_default, gbs_best;      /* stencil + update passes: algorithmic GB/s */
} pb_server_tune_info;
pb_status pb_server_autotune(pb_server *server, int timeout_ms, pb_server_tune_info *out);

/* Kernel measurement of a running server.  Between begin and end the worker
 * launches each phase kernel on its own between CUDA events (slower, for
 * measurement) and sums, per kind of launch, the device time and the
 * algorithmic HBM bytes of the grids active in it.  Per grid node, FP32 inner
 * solves with one-byte coefficients: 21 B for a CG stencil pass (read z,
 * p_old, the x increment d and the code byte; write p and d -- a server's
 * stencil pass stores no Ap), 13 B for an update pass (read p, z and the code
 * byte; write z -- Ap is formed again from p), 37 B for an FP64 residual pass
 * (read x, d, p, the code byte and b; write x and the new z).  FP64 solves:
 * 41 B and 25 B for the two CG passes.  Launches with no grid in the phase
 * they serve are not counted. */
typedef struct {
    double ms_stencil, bytes_stencil;  /* CG stencil-pass launches */
    double ms_update, bytes_update;    /* update-pass launches */
    int launches_stencil, launches_update;
    double ms_resid, bytes_resid;      /* residual-pass launches */
    int launches_resid;
    /* the algorithmic bytes of the first 64 stencil-pass and update-pass
     * launches between begin and end, in launch order, counting launches
     * with no grid in their phase too (0 bytes), so that a counter capture
     * of those same launches can be divided by the grid nodes they covered */
    double first_bytes_stencil[64], first_bytes_update[64];
    int first_stencil, first_update;   /* entries filled (at most 64) */
} pb_kernel_profile;
pb_status pb_server_profile_begin(pb_server *server);
pb_status pb_server_profile_end(pb_server *server, pb_kernel_profile *out);

/* Admission decision of the server, exposed for testing.  Requests are
 * considered in queue order.  A request whose trajectory has an idle
 * resident grid of the same dims reuses it (the most recently used one);
 * any other request needs req_bytes[i] new bytes (a trajectory whose grids
 * are all busy gets one more grid), for which idle grids of the same
 * trajectory with other dims, then idle grids least recently used first, are
 * evicted.  The first request that does not fit stops admission of requests
 * that need new memory (no overtaking).  Outputs: admit[i] = index of the
 * reused slot, -1 for a new slot, -2 not admitted; evict[j] = 1 for slots to
 * evict.  Returns the number admitted. */
typedef struct {
    int64_t trajectory_id;
    int nx, ny, nz;
    size_t bytes;
    int busy;                /* 1 while a request of this grid is on the device */
    uint64_t last_used;      /* larger = more recent */
} pb_slot_state;
int pb_plan_admission(size_t budget, const pb_slot_state *slots, int n_slots,
                      const int64_t *req_traj, const int *req_dims /* 3 per request */,
                      const size_t *req_bytes, int n_reqs, int *admit, int *evict);

#ifdef __cplusplus
}
#endif
#endif /* PB_H */
