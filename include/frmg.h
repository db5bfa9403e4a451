/*
 * frmg.h -- C ABI of the GB300 (sm_103a) FAS multigrid solver for the
 * Hu-Sawicki f(R) scalaron equation (n = 1), after Li, Zhao, Teyssier &
 * Koyama, "ECOSMOG" (arXiv:1110.1379).
 *
 * Equation (Sec. IV, Eq. discrete_fR, multiplied by c~^2 as in Sec. V.B.1,
 * Eq. bc_modified_fR_op), written in u = ln(f_R / fbar_R(a)):
 *
 *   L_i(u) = (alpha/2) sum_{6 faces j} (e^{u_i} + e^{u_j}) (u_j - u_i)
 *            + beta (e^{-u_i/2} - 1) - gamma (rho_i - 1)            = 0
 *
 *   alpha = c~^2 |fbar~_R(a)| / h^2,  beta = Om a^4 (a^-3 + 4 OL/Om),
 *   gamma = Om a,  c~ = c/(B H0),  OL = 1 - Om,
 *   |fbar~_R(a)| = a^2 xi / (3 (a^-3 + 4 OL/Om))^2  (Sec. VI.A.1),
 *   xi = |f_R0| (3 (1 + 4 OL/Om))^2.
 *
 * h is the cell size in code units (box side 1): h = 1/dims[0] on the domain
 * grid, halved per refinement level.  The solution returned in u is
 * u = ln(f_R/fbar_R); f_R = fbar_R(a) e^u with fbar_R(a) = -|fbar~_R(a)|/a^2.
 *
 * Conventions for every entry point:
 *  - Grids are [n2][n1][n0] with x (dims[0]) fastest; dims must be even and >= 2.
 *  - Pointers may be CUDA device memory or host memory.  Host arrays are
 *    staged through library-owned device buffers (copies in both directions
 *    are part of the call).  The caller keeps ownership of every array.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call
 *    that takes a context is synchronous on return: results and stats are
 *    valid when it returns (fr_residual_norm_noalloc, which takes none, is
 *    asynchronous on its stream).
 *  - Return values are fr_status codes.  On FR_ENOCONV / FR_EDIVERGED the last
 *    iterate is still written to u.  fr_status_string() names a code;
 *    fr_last_error() returns a message for the last failing call on the
 *    calling thread.
 *  - A context is not thread-safe: use one context per host thread.
 */
#ifndef FRMG_H
#define FRMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct frmg_ctx frmg_ctx;

typedef enum {
    FR_OK = 0,
    FR_EINVAL = 1,     /* invalid argument (dims, a, |f_R0|, density, patch nesting) */
    FR_ENOMEM = 2,     /* device or pinned host allocation failed */
    FR_ECUDA = 3,      /* a CUDA call failed */
    FR_ENOCONV = 4,    /* max_vcycles reached before tol */
    FR_EDIVERGED = 5,  /* NaN/Inf or a residual growing for several cycles */
    FR_ETIMEOUT = 6    /* reserved for a bounded device-side wait that ran out; no
                          kernel of this library waits on another, so no entry
                          point returns it */
} fr_status;

typedef enum {
    FR_FP64 = 0,  /* every step in FP64 (the plain method) */
    FR_MIXED = 1  /* FP32 smoothing and coarse levels inside an FP64 defect /
                     update / convergence loop (iterative refinement) */
} fr_precision;

typedef struct {
    double tol;             /* rms of L(u) on the finest grid; 1e-8 */
    int max_vcycles;        /* cap on V-cycles (FP64) or on inner V-cycles (mixed); 100 */
    int pre, post;          /* NGS sweeps before / after the coarse correction; 2, 2 */
    fr_precision prec;      /* FR_FP64 */
    double newton_step_cap; /* |du| per Newton-Gauss-Seidel update; 1.0 */
    int inner_cycles;       /* mixed: FP32 V-cycles per FP64 defect after the first; 2 */
    int max_outer;          /* mixed: cap on FP64 defect evaluations; 40 */
    int allow_negative_density; /* 0: reject rho < 0 (the paper's sine test needs 1) */
    int use_graph;          /* capture repeated V-cycles in CUDA graphs; 1 */
    int temporal_depth;     /* FP32 sweeps per pass of the tiled smoother: 1 or 2;
                               0 = library default */
    int tiling;             /* FP32 shared-memory kernels: 0 = where the grids fill the
                               GPU, 1 = wherever possible (grids >= 16 a side), -1 = never */
    int defect_precision;   /* mixed: arithmetic of the fine-grid defect, the update of u
                               and the convergence test: 0 = double-float (pairs of FP32
                               values, ~48-bit significands, on the FP32 pipes),
                               1 = native FP64 */
    double tau_alpha;       /* > 0: also stop once rms(L(u)) <= tau_alpha * rms(tau), tau the
                               truncation-error estimate L^H(R u) - R L^h(u) of Sec. V.B.2
                               on the first coarser grid (the paper asks tau_alpha <= 1/3);
                               0 = off (default) */
    double relax;           /* relaxation factor w of every Newton-Gauss-Seidel update,
                               u += w * du (the Newton-GS step of Sec. V.B.2 is w = 1, the default);
                               0 < w < 2.
                               Over-relaxing the red-black sweeps (w ~ 1.1-1.25) can lower
                               the V-cycle's convergence factor; the solution is the
                               same, only the path to it changes.  On strongly nonlinear
                               fields it can also slow convergence down (fr_autotune tries
                               it per field).  FR_EINVAL outside (0, 2). */
    int fmg;                /* mixed solves of one field from u = 0: 1 = full-multigrid start
                               (the density term averaged to every level, the coarsest level
                               solved, then at each finer level the interpolated coarser
                               solution and one V-cycle from there; the last one, on the
                               finest grid, counts as the first V-cycle); 0 = start the
                               V-cycles from u = 0 (default).  Ignored otherwise. */
    int initial_guess;      /* fr_solve, fr_solve_batch, fr_solve_levels (domain grid):
                               1 = u holds the initial guess (default); 0 = start from
                               u = 0: the contents of u are not read (a host u is not
                               copied to the device), u is output only. */
    int smooth_tile;        /* mixed: kernel and tile of the one-sweep FP32 smoothers on
                               tiled levels: 8 or 16 = register-column kernels (each
                               thread keeps its x-pairs' last four planes in registers),
                               the plain (full-variable) form on 64 x 8 or 64 x 16
                               tiles and the correction form on 64 x 8 tiles; -1 =
                               shared-memory plane-ring kernels on 64 x 16 tiles;
                               0 = library default.  Every choice performs the same
                               sweeps (identical results); only the speed differs. */
} fr_opts;

#define FR_HIST 64
typedef struct {
    int vcycles;      /* V-cycles on the finest grid (all precisions) */
    int outer;        /* mixed: FP64-accurate defect evaluations; FP64: 0 */
    double res0_rms;  /* rms of L(u0) */
    double res_rms;   /* rms of L(u) on return (FP64-accurate evaluation) */
    double res_max;   /* max |L(u)| on return */
    double seconds;   /* wall time of the call */
    int nhist;        /* entries in hist (at most FR_HIST) */
    double hist[FR_HIST]; /* residual rms per V-cycle: FP64 mode, after each cycle;
                             mixed, the fine residual after pre-smoothing of each
                             FP32 cycle, and the FP64-accurate defect (negated)
                             at each outer step */
    double tau_rms;   /* rms of the truncation-error estimate (tau_alpha > 0: of the
                         last evaluation; FP64: after the last V-cycle; mixed: after
                         the FP32 full-variable phase), NaN when not evaluated */
    int host_copies;  /* fr_solve with a host u: copies of the result to the host.  A
                         mixed solve with a page-locked u starts one when an outer step
                         predicts convergence, overlapping the last defect check; a
                         later update makes it stale and the result is copied again
                         (2 or more).  0 for a device u. */
} fr_stats;

/* Refinement patch (Sec. V.A.1, V.B.1, VI.B): a box of fine cells at twice the
 * resolution of its parent, with Dirichlet boundary values interpolated from
 * the parent solution.  The footprint plus one parent cell on every side must
 * lie inside a patch parent; a domain-grid parent wraps periodically. */
typedef struct {
    int parent;          /* -1: the domain grid; else index of an earlier patch */
    int origin[3];       /* lower corner in parent cells (x, y, z) */
    int n[3];            /* fine cells (x, y, z); even, >= 4 */
    const double *density; /* rho~ on the patch cells, [n2][n1][n0] */
    double *u;           /* out: patch solution, [n2][n1][n0] */
} fr_patch;

void fr_opts_default(fr_opts *opts);
const char *fr_status_string(int status);
const char *fr_last_error(void);

/* Library-owned context: device, workspace, streams, captured graphs.
 * The environment variable FRMG_WORKSPACE_LIMIT (bytes), read when the
 * context is created, caps the device workspace the context holds (in use and
 * cached); a call that would need more fails with FR_ENOMEM, as it does when
 * cudaMalloc fails. */
int fr_ctx_create(frmg_ctx **out, int device);
void fr_ctx_destroy(frmg_ctx *ctx);

/* Derived constants {alpha(h = 1/n0), beta, gamma, c~, |fbar~_R(a)|, ubar} for
 * one grid; out has 6 doubles (host). */
int fr_constants(double box_mpc_h, int n0, double a, double omega_m, double fr0_abs,
                 double *out6);

/*
 * Solve one periodic domain grid: FAS V-cycles of red-black Newton-Gauss-Seidel
 * (Sec. V.B) from the initial guess in u_inout until rms(L(u)) <= tol.
 * density: rho~ (mean ~1, Sec. III.A), [n2][n1][n0] FP64.
 * u_inout: in the initial guess, out the solution, FP64.
 * opts NULL = defaults (tol from the argument overrides opts->tol);
 * stats may be NULL.
 * Errors: FR_EINVAL for odd/small dims, a <= 0, |f_R0| <= 0, Om outside
 * (0,1), box <= 0, NaN density or (unless allowed) negative density.
 */
int fr_solve(frmg_ctx *ctx, const double *density, const int dims[3], double box_mpc_h,
             double a, double omega_m, double fr0_abs, double tol, double *u_inout,
             const fr_opts *opts, fr_stats *stats, void *stream);

/*
 * Domain grid plus nested refinement patches, solved one way coarse to fine
 * (Sec. V.A.1: boundary values come from the parent solution; Sec. VI.B).
 * Patches must be ordered so that every parent precedes its children.  For
 * each patch: the initial u and the ghost values are the trilinear (27/9/3/1)
 * interpolation of the parent's solution, u_b = (ghost + first interior)/2 is
 * fixed, and the patch is solved with FAS V-cycles to tol_patch.
 * per_grid (optional, 1 + npatch entries): stats of the domain then each patch.
 */
int fr_solve_levels(frmg_ctx *ctx, const double *density, const int dims[3], double box_mpc_h,
                    double a, double omega_m, double fr0_abs, double tol, double tol_patch,
                    double *u_inout, fr_patch *patches, int npatch, const fr_opts *opts,
                    fr_stats *per_grid, void *stream);

/*
 * Many independent periodic fields solved together: every kernel launch of a
 * V-cycle level covers all fields still iterating (a field drops out once its
 * rms(L(u)) <= tol).  Arrays of nfields entries; density[i] and u_inout[i]
 * must all be device pointers or all host pointers.  omega_m and tol are
 * shared.  stats (optional) has nfields entries.
 */
int fr_solve_batch(frmg_ctx *ctx, int nfields, const double *const *density,
                   const int (*dims)[3], const double *box_mpc_h, const double *a,
                   const double *fr0_abs, double omega_m, double tol, double *const *u_inout,
                   const fr_opts *opts, fr_stats *stats, void *stream);

/*
 * Cloud-in-cell density assignment (Sec. VI.C): np particles at pos[np][3]
 * (x, y, z in box units, [0, 1)), each of mass n0 n1 n2 / np, spread over the 8
 * nearest cell centres with weights prod_d (1 - |x_d - x_c,d| / h_d), periodic.
 * density_out: [n2][n1][n0] FP64, overwritten; its mean is 1 (Sec. VI.C).
 */
int fr_cic_assign(frmg_ctx *ctx, const double *pos, long long np, const int dims[3],
                  double *density_out, void *stream);

/* ---- Single-step entry points (one level, FP64, the same kernels as the
 *      solver uses); parity checks call these step by step.  Arrays follow
 *      the conventions above (caller-owned, device or host, [n2][n1][n0]);
 *      bad dims, sizes or model parameters give FR_EINVAL, checked before
 *      anything is written. ---- */

/* nsweeps red-black Newton-Gauss-Seidel sweeps (Sec. V.B.1: u <- u - (L - f) /
 * (dL/du), the step clamped to |du| <= step_cap; red = (i+j+k) even first) on
 * L(u) = f (f NULL = 0), u updated in place; cell size h; ub NULL = periodic,
 * else the six packed boundary faces of a patch (Eq. u_i-1jk with mask ratio
 * -1; faces -x,+x,-y,+y,-z,+z; the face normal to axis a indexed by the other
 * axes p < q as c[q]*n[p] + c[p]). */
int fr_smooth(frmg_ctx *ctx, double *u, const double *density, const double *f,
              const int dims[3], double h, double box_mpc_h, double a, double omega_m,
              double fr0_abs, const double *ub, int nsweeps, double step_cap, void *stream);

/* FP32 smoothing as the mixed path runs it, on one level: nsweeps red-black
 * sweeps of A(u) = f (f NULL = 0, no density term) in FP32.  bg NULL: u is the
 * unknown.  bg non-NULL: u is a correction delta on the FP32 background bg and
 * the equation is A(bg + delta) - A(bg) = f.  tiled != 0 selects the
 * shared-memory temporally blocked kernel (grids of at least 16 cells a side),
 * 8 or 16 the register-column kernel (plain form on 64 x 8 or 64 x 16 tiles,
 * correction form on 64 x 8 tiles), 0 the one-colour-per-launch kernel; all
 * give the same sweeps. */
int fr_smooth_f32(frmg_ctx *ctx, float *u, const float *bg, const float *f, const int dims[3],
                  double h, double box_mpc_h, double a, double omega_m, double fr0_abs,
                  const float *ub, int nsweeps, double step_cap, int tiled, void *stream);

/* d = L(u) - f on one level (Sec. IV Eq. discrete_fR, with patch faces
 * Eq. bc_modified_fR_op; arguments as fr_smooth); d: dims cells, overwritten. */
int fr_residual(frmg_ctx *ctx, const double *u, const double *density, const double *f,
                const int dims[3], double h, double box_mpc_h, double a, double omega_m,
                double fr0_abs, const double *ub, double *d, void *stream);

/* d = L(u) - f (f = 0) evaluated as the mixed-precision loop evaluates its
 * fine-grid defect: in double-float arithmetic (FP32 pairs, ~48-bit
 * significands) from u split into a double-float pair; arguments as
 * fr_residual.  Lets callers compare it with an FP64 evaluation. */
int fr_residual_df(frmg_ctx *ctx, const double *u, const double *density, const int dims[3],
                   double h, double box_mpc_h, double a, double omega_m, double fr0_abs,
                   const double *ub, double *d, void *stream);

/* Restriction of Sec. V.B.2 (read as the average of the 8 children of each
 * coarse cell): coarse [n2/2][n1/2][n0/2] from fine [n2][n1][n0], overwritten;
 * every fine dim even and >= 2. */
int fr_restrict(frmg_ctx *ctx, const double *fine, const int dims_fine[3], double *coarse,
                void *stream);

/* u_fine += P(uH - uR), trilinear 27/9/3/1 over 64 (Sec. V.A.3, V.B.3);
 * uH and uR have dims_fine / 2; periodic wrap, or with dirichlet != 0 coarse
 * neighbours outside the grid contribute 0 (no renormalisation). */
int fr_prolong_correct(frmg_ctx *ctx, double *u_fine, const int dims_fine[3], const double *uH,
                       const double *uR, int dirichlet, void *stream);

/* Patch boundary set-up (Sec. V.A.1, V.B.1: ghost values from the parent):
 * a patch of n[3] fine cells (refinement factor 2) whose lower corner is
 * parent cell origin[3] (x, y, z).  u_init (n cells) and every ghost value are
 * the trilinear 27/9/3/1 interpolation of uparent (dims_parent); ub (packed
 * faces as fr_smooth) receives u_b = (ghost + first interior) / 2.  periodic
 * != 0 wraps the parent; otherwise a stencil leaving it gives FR_EINVAL
 * (found while interpolating: device outputs may then hold partial values,
 * host outputs are left unchanged). */
int fr_patch_bc(frmg_ctx *ctx, const double *uparent, const int dims_parent[3], int periodic,
                const int origin[3], const int n[3], double *u_init, double *ub, void *stream);

/* Run exactly ncycles FAS V-cycles of Sec. V.B.2 (no convergence test) on one
 * periodic grid in the precision of opts, u_inout updated in place;
 * stats->res_rms is the FP64 residual afterwards. */
int fr_vcycles(frmg_ctx *ctx, const double *density, const int dims[3], double box_mpc_h,
               double a, double omega_m, double fr0_abs, double *u_inout, int ncycles,
               const fr_opts *opts, fr_stats *stats, void *stream);

/*
 * Residual norm of one grid without allocating anything (no cudaMalloc,
 * cudaFree or allocating library call), for callers that cannot allocate
 * device memory at that point: code whose device memory is owned by another
 * allocator (a caching pool that leaves nothing for cudaMalloc, or that must
 * account for every allocation), and loops that cannot afford the device
 * synchronisation an allocation or a free may bring.  The paper has no
 * counterpart; this is a service entry point of the library.
 * out2 (device) receives {rms of L(u) over the cells, max |L(u)|}; u, density,
 * ub (optional patch faces, as fr_smooth) and out2 must be device memory of
 * the current device (or managed memory): the kernels run on the current
 * device, and a pointer to another GPU's memory is refused with FR_EINVAL.
 * No context is needed.  Grids are limited to 33,554,432 cells (FR_EINVAL
 * beyond, with a message in fr_last_error()).  The call is asynchronous on
 * `stream`: out2 is valid once the stream reaches it.
 * Scratch: a fixed 16 KB array of this library's module on each GPU that
 * loads the library, held until the process exits and shared by every call on
 * that GPU; each call overwrites all of it before reading it, but calls that
 * overlap on the GPU (different streams, no ordering) race on it.  The first
 * call on each device looks up the array's device address (with that device
 * current) and keeps it.  The kept address belongs to the device's primary
 * context: after cudaDeviceReset (or anything else that destroys that
 * context) the module is loaded again, possibly at another address, and the
 * kept one is stale, so do not call this entry point on that device again in
 * the same process.
 */
int fr_residual_norm_noalloc(const double *u, const double *density, const int dims[3],
                             double h, double box_mpc_h, double a, double omega_m,
                             double fr0_abs, const double *ub, double *out2, void *stream);

/*
 * Autotuner: solves the given problem from u = 0 (into library scratch; the
 * caller's arrays are only read) with every combination of the V-cycle shape
 * (pre, post) in {(1,1), (2,1), (1,2), (2,2), (3,3)} and the relaxation factor
 * relax in {1, 1.15, 1.25} at one sweep per tiled pass, then, one at a time on
 * top of the fastest setting so far, two sweeps per pass (temporal_depth 2),
 * the full-multigrid start (fmg 1) and tiling 1, then the smoother's kernel
 * and tile shape (smooth_tile 16, 8 and -1), on top of *base (NULL =
 * defaults), twice each, and writes the fastest setting that reaches tol to
 * *best (and its time in seconds to *best_seconds, if not NULL; best->smooth_tile
 * names the chosen tile, never 0).  Device or host density pointer.
 * FR_ENOCONV if no candidate converged.
 */
int fr_autotune(frmg_ctx *ctx, const double *density, const int dims[3], double box_mpc_h,
                double a, double omega_m, double fr0_abs, double tol, const fr_opts *base,
                fr_opts *best, double *best_seconds, void *stream);

/*
 * Autotuner of a batch (the arguments of fr_solve_batch): solves the batch
 * from u = 0 (into library scratch; the caller's arrays are only read) with
 * every combination of the V-cycle shape (pre, post) in {(1,1), (2,1), (1,2),
 * (2,2), (3,3)}, the relaxation factor in {1, 1.15, 1.25} and tiling in
 * {0, 1} at one sweep per tiled pass, then the smoother's kernel and tile
 * (smooth_tile 16, 8, -1) on the fastest, on top of *base (NULL = defaults),
 * twice each, and writes the fastest setting that reaches tol for every field
 * to *best (its time in seconds to *best_seconds if not NULL).  Device or host
 * densities.  FR_ENOCONV if no candidate converged.
 */
int fr_autotune_batch(frmg_ctx *ctx, int nfields, const double *const *density,
                      const int (*dims)[3], const double *box_mpc_h, const double *a,
                      const double *fr0_abs, double omega_m, double tol, const fr_opts *base,
                      fr_opts *best, double *best_seconds, void *stream);

/*
 * Triangle-shaped-cloud density assignment (Sec. VI.C, the code's default
 * scheme): arguments and result as fr_cic_assign; each particle spreads over
 * the 27 nearest cell centres with weights prod_d W(x_d), W = 3/4 - d^2 for the
 * nearest centre (d = offset in cells, |d| <= 1/2) and (1/2 -+ d)^2 / 2 for its
 * two neighbours; periodic.  FR_EINVAL if a position is outside [0, 1).
 */
int fr_tsc_assign(frmg_ctx *ctx, const double *pos, long long np, const int dims[3],
                  double *density_out, void *stream);

#define FR_SCHEME_CIC 0
#define FR_SCHEME_TSC 1
/*
 * Force interpolation (Sec. VI.C): force_out[np][3] = -grad Phi at the
 * particles pos[np][3] (box units, [0, 1)), the gradient by central
 * differences on the periodic grid of phi ([n2][n1][n0], box units: h_d = 1/n_d)
 * and interpolated with the weights of `scheme` (FR_SCHEME_CIC or
 * FR_SCHEME_TSC: use the scheme of the density assignment, which conserves
 * momentum).  Host or device pointers; dims >= 3; synchronous on return.
 * FR_EINVAL for positions outside [0, 1) (their forces are set to 0).
 */
int fr_particle_forces(frmg_ctx *ctx, const double *phi, const int dims[3], const double *pos,
                       long long np, int scheme, double *force_out, void *stream);

/*
 * Modified Poisson equation for the potential Phi (Sec. III.B; Eq. discrete_poisson):
 *   (1/h^2) [sum of the six neighbours - 6 phi_i] = s_i,
 *   s_i = 2 gamma (rho_i - 1) - (beta/2) (e^{-u_i/2} - 1),
 * the paper's right-hand side for n = 1 written in u = ln(f_R / fbar_R), the
 * variable of fr_solve (gamma = Omega_m a, beta = Omega_m a^4 (a^-3 + 4 OL/Om),
 * as fr_constants returns them).  density, u: [n2][n1][n0] FP64 (u is normally
 * fr_solve's solution on the same grid); phi_inout: initial guess in, solution
 * out.  Host or device pointers (host arrays are staged).
 * phib == NULL: periodic grid.  The equation has a solution only for a source
 * of zero mean, so the source's mean is removed (returned in *src_mean when
 * not NULL) and phi is returned with zero mean.
 * phib != NULL: refinement patch with the packed boundary values phi_b of its
 * six faces (layout as fr_smooth's ub); a neighbour outside the patch is the
 * ghost 2 phi_b - phi_i (Eq. phi_b with mask ratio -1, Eq. bc_modified_poisson);
 * h = the patch's cell size in code units (h <= 0: 1 / dims[0]).
 * Multigrid in the correction scheme (Sec. V.A.2, Eq. bc_modified_poisson_coarse;
 * trilinear prolongation of Sec. V.A.3): FP32 V-cycles (opts->pre / opts->post
 * red-black Gauss-Seidel sweeps, over-relaxed by opts->relax) on the
 * correction equation inside a defect
 * correction whose defect and update are evaluated in double-float (~48-bit)
 * arithmetic.  Stops when the rms of L(phi) - s is <= tol (FR_OK); FR_ENOCONV
 * after opts->max_outer outer steps or opts->max_vcycles V-cycles (phi holds
 * the last iterate).  stats (optional): vcycles, outer, res0_rms, res_rms,
 * res_max, seconds, hist.  Synchronous on return.
 */
int fr_poisson_solve(frmg_ctx *ctx, const double *density, const double *u, const int dims[3],
                     double box_mpc_h, double a, double omega_m, double fr0_abs,
                     const double *phib, double h, double tol, double *phi_inout,
                     const fr_opts *opts, fr_stats *stats, double *src_mean, void *stream);

/* The source s of fr_poisson_solve (before any mean removal), FP64 out
 * (host or device), evaluated in double-float arithmetic. */
int fr_poisson_source(frmg_ctx *ctx, const double *density, const double *u, const int dims[3],
                      double box_mpc_h, double a, double omega_m, double fr0_abs,
                      double *s_out, void *stream);

/*
 * General mask scheme (Sec. V; Eqs. u_i-1jk, bc_modified_fR_op and
 * bc_modified_fR_dop of Sec. V.B.1; the masked multigrid of Sec. V.B.2,
 * V.A.2 and V.A.3): FAS solve of the f(R) equation on a refinement region of
 * any shape.  The region is a box of dims = (n0, n1, n2) cells of size h (code
 * units, box side 1) with a mask value per cell in [-1, 1]: cells with
 * mask > 0 are active and relaxed, the others are ghosts whose values stay
 * fixed; every cell of the box's outer layer must be a ghost (FR_EINVAL
 * otherwise).  density: rho~ on every cell; mask: [n2][n1][n0]; u_inout: in,
 * the initial values of the active cells and the ghost values (interpolated
 * from the parent level in an AMR code), out, the solution on the active
 * cells (ghost values unchanged).  Host or device pointers.
 * Across a face from an active cell i to a ghost g the ghost enters as
 * u_g = u_b - r u_b + r u_i with r = m_g / m_i and b_g = exp(u_g); u_b is
 * fixed from the initial values, u_b = (m_i u_g - m_g u_i) / (m_i - m_g).
 * Coarser levels: masks, densities and initial values restricted as the mean
 * of the 8 children, active where the coarse mask is > 0; R d^h sums the
 * active children only; the correction reaches active fine cells only and a
 * masked coarse cell contributes nothing to it.  Levels halve while the sizes
 * stay even and >= 4, the coarser level's outer layer stays masked and it
 * keeps an active cell.  The paper's masks are +1 (active) and -1 on the
 * finest level; a small positive mask puts the boundary close to the cell
 * centre and makes |r| large (the ghost then amplifies changes of u_i by |r|).
 * V(pre,post) red-black Newton-Gauss-Seidel (opts->pre, post,
 * newton_step_cap, relax), until the rms of L(u) over the active cells is
 * <= tol (FR_OK) or opts->max_vcycles V-cycles (FR_ENOCONV).
 * opts->prec = FR_FP64: every step in FP64.  FR_MIXED: the same V-cycles in
 * FP32 first (mask, density and ghost boundary values read from the FP64
 * copies), until their residual stalls (ratio >= 0.75 per cycle), grows past
 * three times its best, or falls to 1e-6 of its start or to tol (a
 * non-finite FP32 residual discards this phase); then outer steps: the FP64
 * residual d, opts->inner_cycles FP32 V-cycles of the correction form
 * L(g + v) - L(g) = -d (g the FP64 iterate rounded to FP32), u += v; a step
 * that does not halve the FP64 residual hands over to FP64 V-cycles.  The
 * convergence test is always the FP64 residual.
 * stats: vcycles (both phases), res0_rms, res_rms, res_max, seconds, hist (the
 * rms after each V-cycle; mixed: the FP32 phase's values, then the FP64
 * residual (negated) after each outer step and FP64 V-cycle), outer (mixed:
 * FP64 residual evaluations after the FP32 phase).
 * Synchronous on return.
 */
int fr_solve_masked(frmg_ctx *ctx, const double *density, const double *mask, const int dims[3],
                    double h, double box_mpc_h, double a, double omega_m, double fr0_abs,
                    double tol, double *u_inout, const fr_opts *opts, fr_stats *stats,
                    void *stream);

/*
 * Symmetron field equation (a second scalar-field model on the same FAS
 * machinery; the paper's Sec. I and VII name the symmetron of Hinterbichler &
 * Khoury 2010 among the models its solver carries over to).  In
 * chi = phi / phi_0 (phi_0 the vacuum value), with the vacuum range lambda0
 * (Mpc/h) and the expansion factor a_ssb at which the mean matter density
 * falls to the symmetry-breaking density, the quasi-static comoving equation
 *   laplacian chi = (a^2 / (2 lambda0^2)) [ ((a_ssb / a)^3 rho - 1) chi + chi^3 ]
 * is discretised with the 7-point Laplacian (Sec. IV) on a periodic grid of
 * cells of box / dims[0] Mpc/h and solved as
 *   L_i = A sum_{6 faces} (chi_j - chi_i) - [ (s rho_i - 1) chi_i + chi_i^3 ] = 0,
 *   A = 2 lambda0^2 / (a^2 (box / dims[0])^2),  s = (a_ssb / a)^3,
 * by FAS V-cycles of red-black Newton-Gauss-Seidel (Sec. V.B.2: 8-child
 * average restriction, trilinear prolongation, A / 4 per coarser level) until
 * rms(L) <= tol.  The field is symmetric under chi -> -chi; the solution
 * sought is the positive branch, reached from a positive initial guess.
 * density: rho (mean 1, finite and >= 0), [n2][n1][n0]; chi_inout: initial
 * guess in (opts->initial_guess = 0: start from the homogeneous positive
 * solution sqrt(1 - s), or 1 before symmetry breaking), solution out.  Host
 * or device pointers.  opts: pre, post, newton_step_cap, relax, max_vcycles,
 * max_outer, initial_guess, tiling (FR_MIXED: the FP32 sweeps of a level run
 * as one register-column kernel per sweep on 64 x 8 tiles where the level
 * fills the GPU with tiles (0), wherever it is at least 16 cells a side (1),
 * or never (-1: one launch per colour)), prec: FR_FP64 = every step in FP64; FR_MIXED =
 * the residual, the update of chi and the convergence test in double-float
 * (chi and rho as pairs of FP32 values, ~48-bit significands, on the FP32
 * pipes) around FP32 FAS V-cycles of
 * the correction equation L(g + delta) - L(g) = -L(chi), g = fp32(chi), run
 * until their fine residual is predicted below max(0.1 tol, 1e-6 rms L(chi))
 * (at most max_vcycles per outer step).  stats: vcycles, outer, res0_rms,
 * res_rms, res_max, seconds, hist.  FR_EINVAL for bad arguments or density,
 * FR_ENOCONV if tol is not reached (chi holds the last iterate),
 * FR_EDIVERGED for a non-finite or growing residual.  Synchronous on return.
 */
int fr_symmetron_solve(frmg_ctx *ctx, const double *density, const int dims[3],
                       double box_mpc_h, double a, double a_ssb, double lambda0, double tol,
                       double *chi_inout, const fr_opts *opts, fr_stats *stats, void *stream);

/* Number of kernel launches this context issued since it was created. */
long long fr_launch_count(const frmg_ctx *ctx);

/* Per-kernel timing: when enabled, every launch is bracketed by CUDA events
 * recorded on its own stream and the elapsed times are accumulated per kernel
 * family.  fr_profile(ctx, 1) enables and clears, fr_profile(ctx, 0) disables
 * and clears.  fr_profile_entry reads entry idx (FR_EINVAL past the end):
 * name (NUL-terminated, truncated to namelen), launch count, total ms. */
int fr_profile(frmg_ctx *ctx, int enable);
int fr_profile_entry(frmg_ctx *ctx, int idx, char *name, int namelen, long long *count,
                     double *total_ms);

#ifdef __cplusplus
}
#endif

#endif /* FRMG_H */
