/*
 * mg.h -- C ABI of the GB300 geometric-multigrid Poisson solver.
 *
 * The library solves the discrete Poisson equation of self-gravity
 *     (sum of the six face neighbours - 6 phi_ijk) / h^2 = 4 pi G rho_ijk
 * (Tomida & Stone 2023, Sec. 2.1, Eqs. poisson and discretized2) on a uniform
 * Cartesian grid of nx*ny*nz cells with spacing h, by full multigrid
 * (Algorithm 2) followed by V(M,N) cycles (Algorithm 1) with a red-black SOR
 * smoother (Sec. 2.3.2, Eqs. rbsor1-rbsor2), volume-average restriction and
 * trilinear prolongation (Sec. 2.3.1), until the volume-weighted RMS defect
 * (Sec. 2.3.7, Eq. threshold) divided by the RMS of the source falls below
 * a tolerance.
 *
 * Conventions shared by every entry point:
 *  - Arrays are contiguous, z-major: element (i, j, k) of an nx*ny*nz field
 *    is at index (k*ny + j)*nx + i (x fastest).  Cell (i, j, k) has its centre
 *    at ((i + 1/2 - nx/2) h, (j + 1/2 - ny/2) h, (k + 1/2 - nz/2) h): the
 *    domain is centred on the origin.
 *  - Pointers whose name ends in _dev are device pointers on the current CUDA
 *    device; other pointers are host pointers.  The caller owns every array
 *    it passes; the library never frees or keeps them past the call.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Device work
 *    is issued on that stream in order; entry points that return values to
 *    host memory synchronise that stream before returning.
 *  - Every entry point returns an mg_status and never aborts the process.
 *    mg_status_str() names a status; mg_last_error() gives the message of the
 *    last failure of a context (or of the process, for NULL).
 *  - Red cells are those with (i + j + k) even (0-based); red is updated first
 *    (Sec. 2.2, Eqs. rbgs1-rbgs2).
 */
#ifndef MG_GB300_H
#define MG_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MG_OK = 0,
  MG_ERR_ARG = 1,           /* invalid argument (sizes, kinds, null pointers)     */
  MG_ERR_OOM = 2,           /* device or host allocation failed / over budget     */
  MG_ERR_CUDA = 3,          /* a CUDA call failed; see mg_last_error()            */
  MG_ERR_NOT_CONVERGED = 4, /* tolerance not met within max_cycles or it stalled  */
  MG_ERR_DIVERGED = 5,      /* NaN/Inf, or the defect grew tenfold                */
  MG_ERR_TIMEOUT = 6,       /* a bounded device wait ran out                      */
  MG_ERR_BUSY = 7           /* the resource is in use (server full)               */
} mg_status;

/* Boundary kinds (Sec. 2.3.6).  Periodic and zero-gradient ghosts copy cell
 * centres; fixed and open ghosts are 2 b - (adjacent active cell), so that the
 * value on the domain surface equals b (a constant for FIXED, the multipole
 * potential of App. A for OPEN).  Coarse correction levels use the
 * homogeneous counterpart (periodic, zero fixed, zero gradient).  MIXED is a
 * rule per face, made by mg_create_faces only. */
typedef enum {
  MG_BC_PERIODIC = 0,
  MG_BC_FIXED = 1,
  MG_BC_ZEROGRAD = 2,
  MG_BC_OPEN = 3,
  MG_BC_MIXED = 4
} mg_bc;

/* Arithmetic of a solve.  FP64: every step in double.  MIXED: an FP64
 * defect-correction loop (outer residual, correction update, source,
 * multipole moments and boundary values in double) around FP32 multigrid
 * solves of the correction equation. */
typedef enum { MG_FP64 = 0, MG_MIXED = 1 } mg_precision;

typedef struct {
  int prec;           /* mg_precision; default MG_FP64                             */
  int mode_fmg;       /* 1: FMG start (Algorithm 2); 0: MGI, phi_dev holds the      */
                      /*    initial guess (Sec. 2.3.7).  Default 1                  */
  int pre, post;      /* V(M,N) smoothing steps, each in {0,1,2}; default 1, 1      */
  double omega;       /* SOR over-relaxation (Sec. 2.3.2); default 1.15             */
  int max_cycles;     /* V-cycles (FP64) or outer iterations (MIXED); default 50    */
  double fixed_value; /* b for MG_BC_FIXED; default 0                               */
  int lmax;           /* multipole order for MG_BC_OPEN, 0..4 (App. A); default 4   */
  int use_com;        /* 1: expansion about the centre of mass (default); 0: origin */
  double origin[3];   /* expansion origin when use_com = 0                          */
  double stall_ratio; /* stop when d_n > stall_ratio * d_{n-1} twice; default 0.9   */
  int inner_fmg;      /* MIXED: start each inner FP32 solve with FMG (default 0:    */
                      /*    V-cycles from a zero correction)                         */
  int inner_cycles;   /* MIXED: FP32 V-cycles per outer iteration after the start;  */
                      /*    default 3                                               */
  int outer_fixed;    /* MIXED: 1 (default): from the second outer iteration on,    */
                      /*    phi and h^2 f are held as 64-bit integers scaled by 2^S  */
                      /*    and the outer residual is exact integer arithmetic,     */
                      /*    rounded once to FP32; 0: FP64 residual and update        */
  int fas;            /* FP64: 1 runs the full approximation scheme (Algorithm 3,   */
                      /*    Sec. 2.3.5) in place of the correction scheme in every  */
                      /*    V-cycle and in FMG; 0 (default) the correction scheme   */
  int coarse_literal; /* 1: the coarse correction levels of a zero-gradient grid   */
                      /*    take zero fixed values (Sec. 2.3.6 read word for word)  */
                      /*    instead of the homogeneous zero-gradient rule; other    */
                      /*    rules are unaffected.  Converges, but slowly (about     */
                      /*    0.9 per V-cycle on 16^3-32^3 grids against 0.15), so    */
                      /*    give stall_ratio >= 1 and room in max_cycles.  Not in    */
                      /*    mg_batch_create.  Default 0                              */
  int leg_pairs;      /* MIXED: the up leg of each inner V-cycle on the finest     */
                      /*    level and the down leg of the next (Algorithm 1, steps   */
                      /*    5-7 then 1-3) as one fused pass, two SMOOTH steps per    */
                      /*    pass over HBM, or as two passes; same bits either way.   */
                      /*    0 (default): two passes, unless mg_ctx_autotune timed    */
                      /*    the fused pass faster; 1: always fused; 2: never         */
  int batch_small;    /* serving loop only: 1 serves requests of at most 64^3 cells  */
                      /*    with a periodic, fixed or zero-gradient rule by batched  */
                      /*    hierarchies (continuous batching into one persistent     */
                      /*    launch, see mg_server_create); 0 (default): one solve    */
                      /*    per request                                              */
  int tensor_copies;  /* MIXED, periodic levels at least 64 cells wide: the fused  */
                      /*    legs' planes of u and f brought into shared memory by    */
                      /*    tensor copies (cp.async.bulk.tensor, one thread per CTA) */
                      /*    instead of per-thread asynchronous copies (down leg:     */
                      /*    rows in 32s, 64 x 32 tiles; up leg: 64 x 16 tiles); same */
                      /*    bits either way.  0 (default): per-thread copies, unless */
                      /*    mg_ctx_autotune timed the tensor copies faster for that  */
                      /*    leg and level; 1: always (where they apply); 2: never    */
  int first_cycles;   /* MIXED: V-cycles (counting the FMG start when inner_fmg = 1) */
                      /*    of the first outer iteration's inner solve, 1..65; 0    */
                      /*    (default): 1 + inner_cycles like the others.  The first  */
                      /*    inner solve corrects the whole source: its residual      */
                      /*    levels off where FP32 rounding of the correction sets    */
                      /*    the floor, and cycles past that point change little     */
  int reserved[1];    /* must be zero                                               */
} mg_opts;

typedef struct mg_ctx mg_ctx;

/* Fill *opts with the defaults listed above. */
void mg_opts_init(mg_opts *opts);

/* Create a solver for an nx*ny*nz grid of spacing dx with boundary kind bc
 * (periodic, fixed, zero gradient or open).  Each dimension must be a power
 * of two >= 2 with nx a longest side.  Levels are halved until the shortest
 * side has one cell (Sec. 3.2.1): for a cube the coarsest level is one cell,
 * solved exactly; for a box it has several, smoothed by N_0,max Gauss-Seidel
 * sweeps (Sec. 2.3.2).  The level hierarchy and all scratch are allocated on
 * the current device here.  opts may be NULL for defaults; it is copied.  On
 * success *ctx owns the device memory until mg_destroy.  Errors: MG_ERR_ARG
 * (sizes, kinds, options), MG_ERR_OOM, MG_ERR_CUDA. */
mg_status mg_create(int nx, int ny, int nz, double dx, mg_bc bc, const mg_opts *opts,
                    mg_ctx **ctx);

/* Create a solver whose six faces have rules of their own (Sec. 2.3.6 lets
 * the rules differ between boundaries).  face_bc[q], face_value[q] for the
 * faces q = 0..5 = x-, x+, y-, y+, z-, z+ (host arrays of 6):
 *   MG_BC_PERIODIC   both faces of that axis must be periodic;
 *   MG_BC_FIXED      phi on the face is face_value[q];
 *   MG_BC_ZEROGRAD   zero normal gradient.
 * face_value may be NULL for all zeros; it is read on fixed faces only.  Any
 * fixed face sets the zero point of phi; without one the means of f and phi
 * are removed, as for periodic grids.  Coarse correction levels use each
 * face's homogeneous rule (opts->coarse_literal: zero fixed on zero-gradient
 * faces too).  Six equal rules (and, if fixed, equal values) give the
 * context mg_create gives for that rule; otherwise the context's rule is
 * MG_BC_MIXED.  Its levels run with the face rules in their ghost synthesis
 * (the fused FP32 legs, the single-CTA coarse levels and MG_MIXED's exact
 * fixed-point outer step for any combination of periodic axes).  Other
 * arguments and errors as mg_create. */
mg_status mg_create_faces(int nx, int ny, int nz, double dx, const mg_bc *face_bc,
                          const double *face_value, const mg_opts *opts, mg_ctx **ctx);

/* mg_solve, then the gravitational acceleration at cell centres (Sec. 3.2.3):
 * per axis the average of the two face accelerations -(phi_{i+1} - phi_i)/h
 * and -(phi_i - phi_{i-1})/h, neighbours outside the grid from the boundary
 * rule.  g_dev (caller-owned, FP64, 3*nx*ny*nz) receives g_x, g_y, g_z one
 * after the other, each (nz, ny, nx).  In the fixed-point mixed solve the
 * acceleration is formed from the exact integer potential in the same pass
 * that writes phi.  Other arguments, results and errors as mg_solve. */
mg_status mg_solve_gravity(mg_ctx *ctx, const double *rho_dev, double four_pi_G, double tol,
                           double *phi_dev, double *g_dev, double *hist, int hist_cap,
                           int *n_hist, void *stream);

/* Device bytes mg_create would allocate for this grid and these options
 * (the level hierarchy and scratch, as requested from cudaMalloc; the
 * allocator's rounding is not included).  Allocates nothing.  Errors:
 * MG_ERR_ARG as mg_create. */
mg_status mg_required_bytes(int nx, int ny, int nz, mg_bc bc, const mg_opts *opts,
                            size_t *bytes);

/* Solve for phi given rho: f = four_pi_G * rho; for periodic and
 * zero-gradient grids the mean of f is removed and the returned phi has zero
 * mean (Sec. 2.3.6); for open grids phi -> 0 at infinity.  rho_dev and
 * phi_dev are FP64 nx*ny*nz device arrays; phi_dev is the initial guess in
 * MGI mode and is overwritten with the result.  Iteration stops when
 * ||d||/||f|| < tol (RMS norms over the finest level, Eq. threshold); tol = 0
 * iterates until the reduction stalls (Sec. 2.3.7).
 * hist (host, capacity hist_cap >= 1) receives ||d||/||f|| after the FMG
 * sweep (FP64) or after the first outer iteration (MIXED), then after each
 * further V-cycle / outer iteration; *n_hist is the count written.
 * Returns MG_OK, MG_ERR_NOT_CONVERGED (phi still holds the last iterate),
 * MG_ERR_DIVERGED, MG_ERR_ARG, MG_ERR_CUDA.  Synchronises `stream`. */
mg_status mg_solve(mg_ctx *ctx, const double *rho_dev, double four_pi_G, double tol,
                   double *phi_dev, double *hist, int hist_cap, int *n_hist, void *stream);

/* Same as mg_solve with rho and phi in HOST memory (phi read as the initial
 * guess in MGI mode): the transfers and the solve all run on `stream` inside
 * the call, and phi holds the result when it returns.  Page-locked buffers
 * (cudaHostAlloc / cudaHostRegister, mapped for this device) are read and
 * written in place by the solve's first pass over rho and its last pass over
 * phi; other host memory goes through copies into device buffers the context
 * keeps.  Same bits either way. */
mg_status mg_solve_host(mg_ctx *ctx, const double *rho, double four_pi_G, double tol,
                        double *phi, double *hist, int hist_cap, int *n_hist, void *stream);

/* Release the context and its device memory.  NULL is accepted. */
mg_status mg_destroy(mg_ctx *ctx);

/* Bytes of device memory the context holds. */
size_t mg_ctx_device_bytes(const mg_ctx *ctx);

/* Number of kernel launches issued by the last mg_solve / mg_solve_host of
 * this context. */
long long mg_ctx_last_launches(const mg_ctx *ctx);

/* Kernel classes for per-kernel timing of finest-level launches. */
typedef enum {
  MG_K_SOR = 0,             /* one colour of the smoother                         */
  MG_K_DEFECT_RESTRICT = 1, /* fused defect + restriction                         */
  MG_K_PROLONG = 2,         /* trilinear prolongation + correction                */
  MG_K_FMG_PROLONG = 3,     /* FMG prolongation I'                                */
  MG_K_DEFECT_NORM = 4,     /* FP64 defect norm of the stopping test              */
  MG_K_OUTER_RESIDUAL = 5,  /* MIXED: FP64 residual -> FP32                       */
  MG_K_CORRECT = 6,         /* MIXED: FP64 correction update                      */
  MG_K_SOURCE = 7,          /* f = 4 pi G rho and its sums                         */
  MG_K_FUSED_DOWN = 8,      /* FP32 fused SMOOTH + defect + restriction           */
  MG_K_FUSED_UP = 9,        /* FP32 fused prolongation + correction + SMOOTH      */
  MG_K_GRAVITY = 10,        /* acceleration g = -grad phi (mg_solve_gravity)       */
  MG_K_FUSED_DOWN0 = 11,    /* MG_K_FUSED_DOWN from a zero start (reads f only)   */
  MG_K_FUSED_UPDOWN = 12,   /* FP32 up leg of one V-cycle and down leg of the     */
                            /* next in one pass (two SMOOTH steps)                */
  MG_K_COUNT = 13
} mg_kernel;

/* Enable (on = 1) or disable per-kernel timing: every finest-level launch of
 * a later solve is bracketed by CUDA events on the solve's stream and its
 * duration added to its class.  Enabling resets the totals. */
mg_status mg_ctx_set_timing(mg_ctx *ctx, int on);

/* Total milliseconds and launch count of kernel class k since timing was
 * enabled. */
mg_status mg_ctx_kernel_time(const mg_ctx *ctx, int k, double *total_ms, long long *launches);

const char *mg_status_str(mg_status s);
const char *mg_last_error(const mg_ctx *ctx);

/* ------------------------------------------------------------------------
 * Single-step operators on one level, for testing each kernel on its own.
 * u_dev, f_dev, d_dev are nx*ny*nz device arrays of the precision `prec`
 * (MG_FP64: double, MG_MIXED: float).  bc and bc_value as above; for
 * MG_BC_OPEN, faces_dev holds the boundary value at every face point of the
 * level: faces 0..5 (x-lo, x-hi, y-lo, y-hi, z-lo, z-hi) in turn, face 0/1
 * indexed [k][j] with k, j in 0..nz+1, 0..ny+1 (index 0 and n+1 are the
 * extended points used by edge and corner ghosts), faces 2/3 [k][i], faces
 * 4/5 [j][i]; it is always FP64.  Edge and corner ghosts apply the face rule
 * along x, then y, then z.  Each returns after the work is queued on stream.
 * ---------------------------------------------------------------------- */

/* `steps` SMOOTH applications (Eqs. rbsor1-rbsor2): colours 0 = red then
 * black per step, 1 = red half-sweep only, 2 = black half-sweep only. */
mg_status mg_op_smooth(int prec, int nx, int ny, int nz, double h, mg_bc bc, double bc_value,
                       const double *faces_dev, double omega, int steps, int colours,
                       void *u_dev, const void *f_dev, void *stream);

/* d = f - L_h u (Eq. defect). */
mg_status mg_op_defect(int prec, int nx, int ny, int nz, double h, mg_bc bc, double bc_value,
                       const double *faces_dev, const void *u_dev, const void *f_dev,
                       void *d_dev, void *stream);

/* The exact conversions of the fixed-point outer loop (binary64 / binary32 to
 * and from 64-bit integers, round to nearest with ties to even, computed in
 * integer arithmetic), applied elementwise to n device values: kind 0 double
 * -> int64, 1 int64 -> double, 2 double -> float, 3 float -> int64, 4 int64
 * -> float.  in_dev and out_dev hold n elements of the kind's input and output
 * types and must not overlap.  Results are the correctly rounded values (the
 * IEEE 754 conversion); out-of-range inputs saturate.  Errors: MG_ERR_ARG for
 * a bad kind, n < 0 or a null pointer with n > 0. */
mg_status mg_op_convert(int kind, long long n, const void *in_dev, void *out_dev, void *stream);

/* Acceleration g = [g_x | g_y | g_z] (3 N doubles) of an FP64 potential at
 * cell centres (Sec. 3.2.3), as in mg_solve_gravity. */
mg_status mg_op_gravity(int nx, int ny, int nz, double h, mg_bc bc, double bc_value,
                        const double *faces_dev, const double *phi_dev, double *g_dev,
                        void *stream);

/* Fused defect + restriction: fc = I_l^{l-1}(f - L_h u) on the
 * (nx/2)*(ny/2)*(nz/2) coarse grid (Algorithm 1, steps 2-3). */
mg_status mg_op_defect_restrict(int prec, int nx, int ny, int nz, double h, mg_bc bc,
                                double bc_value, const double *faces_dev, const void *u_dev,
                                const void *f_dev, void *fc_dev, void *stream);

/* uc = I_l^{l-1} uf: mean of each 2x2x2 block (Eq. restriction); nx, ny, nz
 * are the fine sizes. */
mg_status mg_op_restrict(int prec, int nx, int ny, int nz, const void *uf_dev, void *uc_dev,
                         void *stream);

/* Prolongation of the coarse (nx/2)*(ny/2)*(nz/2) array uc to the fine grid,
 * with coarse ghosts from (bc, bc_value, coarse faces_dev):
 * high_order = 0: trilinear (Eq. trilinear); 1: FMG operator I' (weights
 * 5/32, 30/32, -3/32).  add = 1: uf += I uc (correction); 0: uf = I uc. */
mg_status mg_op_prolong(int prec, int nx, int ny, int nz, mg_bc bc, double bc_value,
                        const double *coarse_faces_dev, int high_order, int add,
                        const void *uc_dev, void *uf_dev, void *stream);

/* COARSEST (Sec. 2.3.2) on a 1x1x1 level from a zero guess: the 1-cell
 * equation solved exactly with its ghosts; 0 for periodic / zero gradient. */
mg_status mg_op_coarsest(int prec, double h, mg_bc bc, double bc_value, const double *faces_dev,
                         const void *f_dev, void *u_dev, void *stream);

/* Fused FP32 legs of a V-cycle (Algorithm 1) on one level with a homogeneous
 * rule (bc = MG_BC_PERIODIC, MG_BC_FIXED meaning zero fixed, or
 * MG_BC_ZEROGRAD).  u_in and u_out are distinct float arrays.
 * down: u_out = SMOOTH(u_in, or 0 if zero_guess), then fc = I_l^{l-1}(f - L u_out)
 *       on the (nx/2)*(ny/2)*(nz/2) grid (steps 1-3).
 * up:   u_out = SMOOTH(u_in + I_{l-1}^l ec), ec on the coarse grid (steps 5-7).
 * Levels the fused kernels do not cover (narrower than 32 cells) run the
 * per-step kernels instead, with the same result. */
mg_status mg_op_vcycle_down(int nx, int ny, int nz, double h, mg_bc bc, double omega,
                            int zero_guess, const float *u_in_dev, float *u_out_dev,
                            const float *f_dev, float *fc_dev, void *stream);
mg_status mg_op_vcycle_up(int nx, int ny, int nz, double h, mg_bc bc, double omega,
                          const float *u_in_dev, float *u_out_dev, const float *f_dev,
                          const float *ec_dev, void *stream);

/* The fused FP32 kernels of the two legs above, called directly (no
 * fallback to the per-step kernels), with a rule per face and an explicit
 * launch shape, so that every compiled variant can be checked on its own.
 * leg 0: down (steps 1-3 of Algorithm 1: u_out = SMOOTH(u_in, or 0 when
 * zero_guess), fc = restriction of f - L u_out); leg 1: up (steps 5-7:
 * u_out = SMOOTH(u_in + trilinear(ec))); leg 2: the up leg of one V-cycle and
 * the down leg of the next in one pass (steps 5-7, then 1-3 of the next cycle:
 * u_out = SMOOTH(SMOOTH(u_in + trilinear(ec))), fc = restriction of
 * f - L u_out; tx 0 or 64, nx a multiple of 64, nz >= 16); leg 3: leg 0 with
 * the planes of u_in and f brought into shared memory by tensor copies
 * (cp.async.bulk.tensor) on the tiles whose window does not wrap (all faces
 * periodic, tx 0 or 64, ty 0 or 32, nx a multiple of 64, ny of 32; same bits
 * as leg 0); leg 4: leg 1 with the planes of u_in and f brought in the same
 * way (tx 0 or 64, ty 0 or 16, nx a multiple of 64; same bits as leg 1).  A
 * leg-3 or leg-4 kernel that waits too long for a copy sets a process-wide
 * flag; the next such call that finds it set clears it and returns
 * MG_ERR_TIMEOUT.  face_bc[6] (host) gives each face's
 * homogeneous rule (x-, x+, y-, y+, z-, z+): MG_BC_PERIODIC on both faces of an
 * axis, MG_BC_FIXED (value 0) or MG_BC_ZEROGRAD.  tx (0, 32 or 64 cells), ty
 * (0, 16 or 32 rows) and cz (0 or a multiple of 4 planes; of 8 for leg 2)
 * choose the CTA tile
 * and z-chunk; 0 takes the built-in choice.  Arrays as in mg_op_vcycle_down
 * and mg_op_vcycle_up.  Errors: MG_ERR_ARG for bad arguments and for grids or
 * shapes the fused kernels do not take (sides below 32, nx not a multiple of
 * the tile width, ny of the tile height, nz of 8). */
mg_status mg_op_fused_leg(int leg, int nx, int ny, int nz, double h, const int *face_bc,
                          double omega, int zero_guess, int tx, int ty, int cz,
                          const float *u_in_dev, float *u_out_dev, const float *f_dev,
                          const float *ec_dev, float *fc_dev, void *stream);

/* The fixed-point outer step of MG_MIXED (not in the paper: the exact form
 * of the FP64 defect correction, with phi and h^2 f held as 64-bit integers
 * P and F scaled by 2^S):
 *   P' = P + round(e * c)   (e * c the FP32 product rounded to the nearest
 *                            integer, ties to even; phi_in_dev NULL: P = 0;
 *                            e_dev must not be NULL)
 *   R  = F - (sum of the six neighbours of P' - 6 P')   exactly (Eq. defect)
 *   r32 = fl32(R) * factor.
 * phi_out_dev receives P', r32_dev the residual.  face_bc[6] as in
 * mg_op_fused_leg; a fixed face's neighbour is B - P' with B = round(2 b 2^S),
 * b from faces_dev (the faces layout above, FP64; NULL: b = 0); two_pow_S =
 * 2^S.  cz: planes per CTA (0 built-in, else >= 4).  int64 arrays
 * nx*ny*nz; nx a multiple of 32 and ny of 16.  Synchronises `stream`.
 * Errors: MG_ERR_ARG, MG_ERR_CUDA. */
mg_status mg_op_fx_step(int nx, int ny, int nz, const int *face_bc, const double *faces_dev,
                        double two_pow_S, int cz, const long long *phi_in_dev, const float *e_dev,
                        float c, const long long *F_dev, long long *phi_out_dev, float factor,
                        float *r32_dev, void *stream);

/* Multipole moments of rho_dev (FP64, nx*ny*nz, spacing h) for App. A:
 * Q_host receives (lmax+1)^2 moments ordered l*l + (m + l) (25 slots are
 * written, zero above lmax); origin_host is the expansion origin on input
 * (use_com = 0) or receives the centre of mass (use_com = 1; kept as given
 * when the total mass is 0).  Synchronises `stream`. */
mg_status mg_op_multipole_moments(int nx, int ny, int nz, double h, const double *rho_dev,
                                  int lmax, int use_com, double *origin_host, double *Q_host,
                                  void *stream);

/* Multipole boundary potential -G sum Q_lm sqrt(4 pi/(2l+1)) Y_lm / r^(l+1)
 * (App. A) at every face point of an nx*ny*nz level of spacing h, in the
 * faces layout described above.  Q_host and origin_host as returned by
 * mg_op_multipole_moments. */
mg_status mg_op_open_faces(int nx, int ny, int nz, double h, const double *Q_host, int lmax,
                           double G, const double *origin_host, double *faces_dev, void *stream);

/* Same result as mg_op_multipole_moments, for callers that cannot allocate
 * device memory -- for instance a host application whose device memory is
 * all reserved by its own pool allocator and that forbids allocations by
 * plugins, or code that must not meet an out-of-memory failure or the
 * allocator's latency mid-step.  The paper has no counterpart: this entry
 * point exists only for such callers.
 * It allocates nothing (no cudaMalloc, cudaFree or other allocating call):
 * its scratch is one fixed device array of 8192 * 35 + 32 doubles (2.24 MiB)
 * that every device which loads the library holds until the process exits.
 * Limit: ny * nz <= 262144 rows (32 rows per partial block, 8192 blocks);
 * larger grids are rejected with MG_ERR_ARG and a message on stderr (use
 * mg_op_multipole_moments for them).  The first call on a device looks up the
 * array's device address with cudaGetSymbolAddress and loads the polynomial
 * tables into constant memory, with that device current; make that first call
 * before any stream capture.  Every call uses the same array, which keeps the
 * last call's contents: calls whose work overlaps on the GPU (on different
 * streams, or from several host threads) race and must be serialised by the
 * caller.  Synchronises `stream`. */
mg_status mg_op_multipole_moments_noalloc(int nx, int ny, int nz, double h, const double *rho_dev,
                                          int lmax, int use_com, double *origin_host,
                                          double *Q_host, void *stream);

/* ------------------------------------------------------------------------
 * Batched solve: many independent grids in one persistent launch.
 * ---------------------------------------------------------------------- */
typedef struct mg_batch mg_batch;

/* Create a batch of n grids: grid g has dims[3g..3g+2] cells (cubic, a power
 * of two from 2 to 1024), spacing dx[g], rule bcs[g] (periodic, fixed or zero
 * gradient; fixed_values[g] is b for a fixed rule, NULL means 0).  Every grid
 * is solved by the mixed-precision method (a defect-correction loop whose
 * source, norms and residual are FP64-accurate -- the residual exact in 64-bit
 * fixed point, as in mg_solve -- around FP32 V(1,1) cycles): opts->prec must
 * be MG_MIXED, pre = post = 1, mode_fmg = 1 (phi starts at 0), inner_fmg = 0;
 * max_cycles (outer iterations, <= 64) and inner_cycles (V-cycles per outer
 * iteration after the one from a zero correction, 0..16; first_cycles, 0..17,
 * for the first outer iteration) are shared.  All
 * level storage is allocated here.  Errors: MG_ERR_ARG, MG_ERR_OOM. */
mg_status mg_batch_create(int n, const int *dims, const double *dx, const mg_bc *bcs,
                          const double *fixed_values, const mg_opts *opts, mg_batch **batch);

/* Solve every grid: rho_dev[g], phi_dev[g] are the FP64 device arrays of grid
 * g, four_pi_G[g] and tol[g] its constants (host arrays of n).  rho_dev[g] =
 * NULL leaves slot g out of this solve (phi_dev[g] is not touched, status[g]
 * = MG_OK, n_hist[g] = 0); at least one grid must be given.  A grid's result
 * does not depend on the other slots.  One persistent
 * cooperative kernel runs every phase of every grid; the first call captures
 * the upload of the per-grid arguments, the kernel and the download of the
 * results as a CUDA graph (so make it outside any capture of your own) and
 * later calls replay it; each grid stops by the
 * rule of mg_solve (Sec. 2.3.7).  hist (host, n * hist_cap, may be NULL)
 * receives each grid's ||d||/||f|| after every outer iteration, n_hist[g] the
 * count, status[g] its result.  Returns MG_OK when every grid converged, else
 * the first failing grid's status, MG_ERR_TIMEOUT if a grid-wide barrier wait
 * ran out (about 2 s), MG_ERR_CUDA.  Synchronises `stream`. */
mg_status mg_batch_solve(mg_batch *batch, const double *const *rho_dev, const double *four_pi_G,
                         const double *tol, double *const *phi_dev, double *hist, int hist_cap,
                         int *n_hist, mg_status *status, void *stream);

mg_status mg_batch_destroy(mg_batch *batch);

/* Total cells of the finest levels of the batch. */
long long mg_batch_cells(const mg_batch *batch);

/* 1 when the solve runs as a captured CUDA graph (captured on the first
 * mg_batch_solve and replayed after), 0 when it is launched directly. */
int mg_batch_graph(const mg_batch *batch);

/* Device time of the last mg_batch_solve by phase kind, in milliseconds
 * (from the GPU's global timer at each grid-wide barrier): ms_by_type[k] for
 * k < n_types in the order source, mean, first residual, norms of the
 * source and first residual, fused down leg, bottom levels, fused up leg, max |e|,
 * fixed-point scale, conversion to fixed point, outer step (correction and
 * residual), stopping rule, phi sum, phi mean, phi conversion and mean
 * removal.
 * Synchronises the device.  Errors: MG_ERR_ARG, MG_ERR_CUDA. */
mg_status mg_batch_phase_ms(mg_batch *batch, double *ms_by_type, int n_types);

/* CTAs of the persistent launch: 0 (default) as many as fit on the device at
 * once, else at most that many (fewer CTAs leave SMs to other streams' work,
 * for a batch of small grids).  Takes effect at the next mg_batch_solve,
 * which captures its CUDA graph again.  Errors: MG_ERR_ARG (blocks < 0). */
mg_status mg_batch_set_blocks(mg_batch *batch, int blocks);

/* Limit of one wait at the persistent kernel's grid-wide barriers, in GPU
 * clock cycles (default 4e9, about 2 s at 2 GHz); a wait that runs out makes
 * every block return and mg_batch_solve report MG_ERR_TIMEOUT, leaving the
 * batch usable.  Takes effect at the next mg_batch_solve, which captures its
 * CUDA graph again.  Errors: MG_ERR_ARG (cycles < 0). */
mg_status mg_batch_set_barrier_limit(mg_batch *batch, long long cycles);

const char *mg_batch_last_error(const mg_batch *batch);

/* Number of doubles in a faces array of an nx*ny*nz level. */
size_t mg_faces_count(int nx, int ny, int nz);

/* Autotune the launch shapes of this context's hot kernels on `stream`: for
 * every level the fused FP32 legs run on (tiles of 32 or 64 cells by 16 or 32
 * rows, 8..64 z-planes per CTA) and for the fixed-point outer step (4..64
 * planes),
 * each candidate is timed with CUDA events on the context's own buffers and
 * the fastest kept.  Choices are shared by every context of the same shape
 * in the process (so they give identical bits) and, when the environment
 * variable MG_TUNE_CACHE names a file, read from and appended to it.  Results
 * do not depend on the shapes except for the rounding order of the residual
 * norm.  Overwrites the context's scratch only; synchronises `stream`.
 * Errors: MG_ERR_ARG, MG_ERR_CUDA. */
mg_status mg_ctx_autotune(mg_ctx *ctx, void *stream);

/* The shape (tile width tx, height ty, planes cz) chosen for a kernel class on
 * a level (MG_K_FUSED_DOWN, MG_K_FUSED_DOWN0, MG_K_FUSED_UP, MG_K_FUSED_UPDOWN,
 * MG_K_SOR for extra fused smoothing steps, MG_K_OUTER_RESIDUAL for the
 * fixed-point step on the finest level); 0 means the built-in choice.  Where a
 * leg takes its planes by tensor copies (mg_ctx_tensor_copies) the shape is
 * that variant's (64 x 32 down, 64 x 16 up). */
mg_status mg_ctx_tile_config(const mg_ctx *ctx, int level, int kernel, int *tx, int *ty,
                             int *cz);

/* Whether the fused legs of a level of the mixed path bring their planes into
 * shared memory by tensor copies: the down leg (Algorithm 1, steps 1-3 in one
 * pass) from a nonzero start (*down) and from zero (*down0), and the up leg
 * (steps 5-7, *up): 1 or 0, as fixed by opts.tensor_copies and
 * mg_ctx_autotune.  Errors: MG_ERR_ARG (null pointer, level outside
 * 0..L-1). */
mg_status mg_ctx_tensor_copies(const mg_ctx *ctx, int level, int *down, int *down0, int *up);

/* ---------------------------------------------------------------------------
 * Serving loop.  Requests (solves of any supported size and boundary rule)
 * are submitted one at a time and return a ticket at once.  `slots` worker
 * threads, each with its own CUDA stream, take queued requests in arrival
 * order as soon as a slot is free and the request's level hierarchy is
 * resident and idle or fits in the HBM budget (idle hierarchies of other
 * sizes are evicted least recently used first); a later request may pass a
 * waiting one up to 64 times, then the waiting one holds the next free slot.
 * Hierarchies stay resident between requests of the same key (cells, dx,
 * rule, fixed value, lmax).  Requests on different slots run concurrently on
 * the device; each result equals the result of the same request alone.
 * With opts->batch_small = 1, requests of at most 64^3 cells with a periodic,
 * fixed or zero-gradient rule (when the options allow mg_batch_create's solve)
 * are served by batched hierarchies of up to 16 grids of one shape and rule (as
 * many as the budget holds): the slot that takes one also takes the queued
 * requests of that shape and rule and solves them in one persistent launch
 * (mg_batch_solve), whatever their tolerances; a grid's result there does not
 * depend on the others.  The server is internally synchronised: any thread
 * may submit, poll and wait.
 * --------------------------------------------------------------------------- */
typedef struct mg_server mg_server;

typedef struct {
  int nx, ny, nz;        /* cubic power of two >= 2 */
  double dx;             /* cell width */
  mg_bc bc;
  double fixed_value;    /* boundary value b of MG_BC_FIXED */
  int lmax;              /* multipole order 0..4 of MG_BC_OPEN */
  const double *rho;     /* FP64 array, nx*ny*nz, caller-owned: device memory, or */
                         /* host memory (then phi is host memory too)            */
  double four_pi_G;
  double tol;            /* ||d||/||f|| target of this request */
  double *phi;           /* FP64 array written with the result, in the same memory as rho */
  int per_face;          /* 1: a rule per face (Sec. 2.3.6) from the two arrays below,  */
                         /*    as in mg_create_faces (bc and fixed_value are ignored);  */
                         /*    0 (zero-initialised requests): the one rule bc           */
  mg_bc face_bc[6];      /* x-, x+, y-, y+, z-, z+: periodic (in pairs), fixed or zero  */
                         /*    gradient                                                  */
  double face_value[6];  /* b on each fixed face                                         */
} mg_request;

typedef struct {
  int done;              /* 0 while queued or running */
  mg_status status;      /* the solve's status (as mg_solve) once done */
  int n_hist;            /* entries written to hist */
  int reserved;
  double queue_ms;       /* submission -> a slot took it */
  double solve_ms;       /* slot took it -> result in phi (stream synchronised) */
  double total_ms;       /* submission -> result: the request's latency */
  double h2d_ms;         /* host arrays on a single hierarchy: device time of the  */
  double d2h_ms;         /* copies of rho in and phi out (0 otherwise)              */
} mg_result;

typedef struct {
  long long submitted, completed, rejected, evictions, created, cells_completed;
  long long batched;     /* requests solved in one batched launch with others */
  size_t budget_bytes, resident_bytes, peak_bytes; /* hierarchy bytes as mg_required_bytes */
  int queued, running, slots, resident;
} mg_server_stats;

/* Start a server on the current device: hbm_budget_bytes bounds the bytes of
 * all resident hierarchies together (mg_required_bytes of each); slots
 * (1..64) worker threads; at most max_queue (>= 1) requests wait at a time.
 * opts (NULL: defaults) apply to every request except lmax and fixed_value,
 * which come with each request.  Errors: MG_ERR_ARG. */
mg_status mg_server_create(size_t hbm_budget_bytes, int slots, int max_queue,
                           const mg_opts *opts, mg_server **server);

/* Queue one request; *ticket names it.  rho and phi must stay valid and phi
 * untouched by the caller until the request is done.  With host arrays the
 * slot copies rho in and phi out on its own stream by the copy engines (the
 * other slots keep computing meanwhile; page-locked buffers move fastest) and
 * the request's hierarchy holds device copies of both (counted in the
 * budget).  Errors: MG_ERR_ARG (invalid request, or rho and phi in different
 * memories), MG_ERR_OOM (its hierarchy alone exceeds the budget),
 * MG_ERR_BUSY (the queue is full; nothing was queued). */
mg_status mg_server_submit(mg_server *server, const mg_request *request, long long *ticket);

/* State of a ticket without waiting.  Once it reports done = 1 the ticket
 * is retired: a later poll or wait of it returns MG_ERR_ARG.  hist (host,
 * hist_cap entries, may be NULL) receives the residual history as
 * mg_solve's. */
mg_status mg_server_poll(mg_server *server, long long ticket, mg_result *result, double *hist,
                         int hist_cap);

/* Wait up to timeout_s seconds for a ticket; retires it when done.  Returns
 * MG_ERR_TIMEOUT (ticket kept, result->done = 0) when time ran out.  Several
 * threads may wait on one ticket (and others poll it) at once: every thread
 * already waiting when the request finishes receives its result, even if a
 * poll retired the ticket meanwhile; calls made after the retirement return
 * MG_ERR_ARG. */
mg_status mg_server_wait(mg_server *server, long long ticket, double timeout_s,
                         mg_result *result, double *hist, int hist_cap);

mg_status mg_server_get_stats(mg_server *server, mg_server_stats *stats);

/* Finish every queued and running request, free all hierarchies, stop the
 * workers. */
mg_status mg_server_destroy(mg_server *server);

const char *mg_server_last_error(const mg_server *server);

#ifdef __cplusplus
}
#endif

#endif /* MG_GB300_H */
