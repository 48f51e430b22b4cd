/*
 * lbm13.h -- C ABI of the GB300 (sm_103a) D2Q13 energy-conserving multiple-
 * relaxation-time lattice Boltzmann time step of Lallemand & Dubois,
 * "Comparison of Simulations of Convective Flows" (Commun. Comput. Phys. 2015).
 *
 * One time step (lbm13_step) streams the 13 populations -- the D2Q9 set plus
 * the four distance-2 links of Sec. 2, Eq. (d2q13-vitesses) -- applies the wall
 * rules of Sec. 7, Eq. (d2q13-cl-abb) at the domain edges, and relaxes the nine
 * non-conserved moments of the orthogonal basis of Sec. 2, Eq.
 * (d2q13-polynomes) toward the equilibria of Eq. (d2q13-moments-equil), with
 * the forcing of Sec. 5 / Sec. 8.  All of it runs in one fused CUDA kernel per
 * step; the read-outs (lbm13_moments, lbm13_residual) are CUDA kernels too.
 *
 * Conventions shared by every entry point
 *  - Every call returns an lbm13_status (int); no C++ exception crosses the
 *    ABI.  On failure lbm13_last_error(h) holds a message.
 *  - Lattice arrays are row-major [ny][nx] (x fastest), in double precision.
 *    Population arrays are [13][ny][nx], population j in the paper's order:
 *    (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1) (2,0) (0,2)
 *    (-2,0) (0,-2).  Moment planes are in the order rho, E, eps, varpi, jx,
 *    jy, qx, qy, rx, ry, XX, XY, XXe.
 *  - Host pointers are owned by the caller and only read or written during
 *    the call (those calls synchronise the lattice's stream).  Device
 *    pointers (the *_device calls) are owned by the caller and used in stream
 *    order on the lattice's stream; the call returns before the work ends.
 *  - The library owns the lattice's device buffers and obtains them from the
 *    caller's allocator (or cudaMalloc when none is given).  Calls on one
 *    handle are stream-ordered and not thread-safe.
 *  - Units are lattice units: spacing 1, time step 1.
 */
#ifndef LBM13_H
#define LBM13_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM13_OK = 0,
    LBM13_EINVAL = 1,    /* bad argument: sizes, rates outside (0,2), unpaired periodic sides, NULL */
    LBM13_ENOMEM = 2,    /* the allocator returned NULL */
    LBM13_EUNSTABLE = 3, /* derived relaxation time sigma_q <= 0 (Eq. d2q13-sigma-qx) */
    LBM13_EDIVERGED = 4, /* a non-finite population was found by lbm13_residual */
    LBM13_ETIMEOUT = 5,  /* a bounded device-side wait ran out */
    LBM13_ECUDA = 6      /* a CUDA runtime call failed; see lbm13_last_error */
} lbm13_status;

typedef enum {
    LBM13_FP64 = 0,          /* populations stored and computed in double */
    LBM13_FP32_DEVIATION = 1 /* stored as f_j - w_j in float, computed in float;
                                read-outs and reductions in double */
} lbm13_precision;

/* Free parameters of Sec. 2 (the list after Eq. (d2q13-sigma-qx)).  The rest
 * follows from them: h1, k1, h2 (Eq. d2q13-diffusion), sigma_q, c_erho, c2
 * (Eq. d2q13-sigma-qx), s = 1/(sigma + 1/2) (Eq. d2q13-henon), and the shear
 * rate from the viscosity, sigma_XX = 104 nu / (13 c1 + 95 + 2 E0).  Rates of
 * the y components equal those of the x components (s_qy = s_qx, s_ry = s_rx,
 * s_XY = s_XX). */
typedef struct {
    double E0;        /* reference energy moment at rho = 1 */
    double c1;        /* q equilibrium constant */
    double k2;        /* r equilibrium E coefficient */
    double c_epsE;    /* eps equilibrium E coefficient */
    double c_vpi_rho; /* varpi equilibrium rho coefficient */
    double c_vpi_E;   /* varpi equilibrium E coefficient */
    double Pr;        /* Prandtl number: viscosity / decay rate of the entropy mode */
    double nu;        /* kinematic (shear) viscosity */
    double s_eps, s_vpi, s_r, s_XXe; /* free relaxation rates, each in (0, 2) */
} lbm13_params;

typedef enum {
    LBM13_PERIODIC = 0,   /* opposite sides must both be periodic */
    LBM13_WALL_BB = 1,    /* adiabatic no-slip wall: every crossing link bounces back (Sec. 9) */
    LBM13_WALL_MIXED = 2, /* velocity + temperature wall: links normal to the wall use
                             anti-bounce-back, diagonal links bounce-back (Sec. 7) */
    LBM13_HALO = 3        /* south or north only: the lattice is one y-slab of a larger one, and
                             its two rows next to this side are halo rows holding the
                             neighbouring slab's rows (the paper's own lattice has no such
                             side: its stencil, Sec. 2, reaches two rows, hence two halo
                             rows).  The step never writes halo rows and pulls from them
                             like any row; lbm13_halo_unpack fills them after each step. */
} lbm13_wall_kind;

/* A wall lies half a link outside the first/last node.  u_t is its velocity
 * along the wall (+x for south/north walls, +y for west/east walls); T is its
 * temperature (used by LBM13_WALL_MIXED only).  The wall density is the
 * linear extrapolation 1.5 rho(first node) - 0.5 rho(second node).  Where two
 * walls meet (the paper gives no corner rule), the diagonal that leaves a
 * corner node across both bounces back with the moving-wall correction of
 * each wall, at that wall's own state; a closed box then keeps its mass
 * whatever its walls' speeds (with bounce-back walls, its energy too). */
typedef struct {
    int kind;   /* lbm13_wall_kind */
    double u_t;
    double T;
} lbm13_wall;

/* Wall density of the velocity+temperature walls.  Sec. 7 takes it from an
 * extrapolation of the fluid's values without giving the rule; EXTRAPOLATE
 * uses 1.5 rho(first node) - 0.5 rho(second node).  Those walls are not mass-tight
 * (mass drifts slowly through them, ~1e-8 per step per node in a cavity), so
 * ZERO_FLUX offers the density that makes the wall's net normal mass flux
 * zero, estimated from the outgoing populations; the total mass is then
 * conserved to round-off and steady states are reached. */
#define LBM13_WALL_DENSITY_EXTRAPOLATE 0
#define LBM13_WALL_DENSITY_ZERO_FLUX 1

/* Sides, body force and energy source.  The force per node is
 * F = (rho - rho_ref) (gx, gy): rho_ref = 0 gives the body force rho g of the
 * Poiseuille test (Sec. 8), rho_ref = 1 the buoyancy force proportional to
 * rho - rho_0 of Sec. 5.  `heat` is the uniform volumetric energy source of
 * the adiabatic-wall test (Sec. 9): every node gains `heat` of internal-energy
 * density p = (E + 28 rho)/26 - |j|^2/(2 rho) per step (E* += 26 heat), with
 * the equilibria taken half-way (at E + 13 heat) and T read half-way,
 * (p* - heat/2)/rho.  Zero for no source; must be finite. */
typedef struct {
    lbm13_wall west, east, south, north;
    double gx, gy;
    double rho_ref;
    int wall_density;  /* LBM13_WALL_DENSITY_EXTRAPOLATE or LBM13_WALL_DENSITY_ZERO_FLUX */
    double heat;       /* energy source per node and step, in units of p */
} lbm13_boundary;

/* Device-memory provider.  alloc returns a device pointer of at least `bytes`
 * bytes, aligned to 256 bytes, or NULL; free releases it.  They are called from
 * lbm13_create (two population buffers), lbm13_residual (first call: the
 * reduction buffers), lbm13_set_state and lbm13_moments (a staging buffer,
 * released before they return) and lbm13_destroy. */
typedef struct {
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, void *ctx);
    void *ctx;
} lbm13_allocator;

typedef struct lbm13_lattice *lbm13_t;

/* Number of doubles written by lbm13_derive. */
#define LBM13_DERIVED_COUNT 48

/* Moment / field selection bits for lbm13_moments. Bits 0..12 select the 13
 * moments of the stored post-collision state (order above); the others select
 * derived fields. */
#define LBM13_MOMENT(k) (1u << (k))
#define LBM13_FIELD_UX (1u << 13)   /* (j_x - F_x/2) / rho */
#define LBM13_FIELD_UY (1u << 14)   /* (j_y - F_y/2) / rho */
#define LBM13_FIELD_T (1u << 15)    /* p / rho, p = (E + 28 rho)/26 - |j|^2/(2 rho) */
#define LBM13_FIELD_P (1u << 16)    /* p */
#define LBM13_FIELD_E_SEC7 (1u << 17) /* E - (13/2)(ux^2 + uy^2), the read-out printed in Sec. 7 */
#define LBM13_ALL_MOMENTS 0x1FFFu

/* Layout of the 16 doubles written by lbm13_residual. */
enum {
    LBM13_R_RESIDUAL = 0, /* max(r_u, r_T): r_u = ||u^n - u^{n-K}||_2 / (K max(||u^n - mean u^n||_2, 1e-6 sqrt(N)))
                             with the velocity u = (ux, uy) as one vector field over N nodes, K steps since
                             the previous call; r_T the same for T */
    LBM13_R_UX = 1,       /* the ux part of r_u: ||ux^n - ux^{n-K}||_2 / (K max(||u^n - mean u^n||_2, 1e-6 sqrt(N))) */
    LBM13_R_UY = 2,       /* the uy part of r_u */
    LBM13_R_T = 3,        /* r_T */
    LBM13_R_MASS = 4,     /* sum rho over the lattice */
    LBM13_R_JX = 5,       /* sum j_x (stored post-collision moments) */
    LBM13_R_JY = 6,       /* sum j_y */
    LBM13_R_ENERGY = 7,   /* sum E */
    LBM13_R_NUSSELT = 8,  /* (1/(ny kappa dT)) sum [ux (T - Tm) - kappa D_x T], kappa = nu/Pr,
                             dT = T_west - T_east; 0 unless both are LBM13_WALL_MIXED with dT != 0 */
    LBM13_R_ASYM_U = 9,   /* max |u(i,j) + u(nx-1-i, ny-1-j)| (Sec. 10, Fig. 14) */
    LBM13_R_ASYM_T = 10,  /* max |(T - Tm)(i,j) + (T - Tm)(mirror)| */
    LBM13_R_UMAX = 11,    /* max |u| */
    LBM13_R_NONFINITE = 12, /* number of non-finite stored populations */
    LBM13_R_K = 13,       /* steps since the previous lbm13_residual (0 on the first call) */
    LBM13_R_STEP = 14,    /* time step counter */
    LBM13_R_TMEAN = 15    /* mean T */
};

/* Library version string (static storage). */
const char *lbm13_version(void);

/* Message for a status code (static storage). */
const char *lbm13_status_string(int status);

/* Host-only: derived constants of Sec. 2 for a parameter set, no GPU needed.
 * out[LBM13_DERIVED_COUNT] receives: 0 A = 13c1+95+2E0, 1 B = 114404+51051c1-11492c_epsE+7854E0,
 * 2 h1, 3 k1, 4 h2, 5 c2, 6 c_erho, 7 sigma_XX, 8 sigma_q, 9..21 the 13 rates s_k
 * (0 for rho, E, jx, jy), 22..34 the rest populations w_j = f_eq(rho=1, E=E0, j=0),
 * 35 T0 = (E0 + 28)/26, 36 adiabatic sound speed squared A/52, 37 kappa = nu/Pr.
 * Returns LBM13_EINVAL for a NULL argument or a rate outside (0, 2) and
 * LBM13_EUNSTABLE when sigma_q <= 0 (out is filled in both cases). */
int lbm13_derive(const lbm13_params *params, double *out);

/* Host-only: linear stability of the time step about the uniform state
 * rho = 1, u = (ux, uy), T = T0 (no force), the procedure of the end of Sec. 2:
 * *growth = max |z| - 1 over the eigenvalues z of the linearised step for the
 * n x n wave vectors k = (-pi + 2 pi a/(n-1), -pi + 2 pi b/(n-1)) (k = 0 for
 * n = 1).  The step is linearly stable when *growth <= ~1e-12 (round-off).
 * n in 1..129.  LBM13_EINVAL for NULL, n out of range or an eigenvalue
 * iteration that does not converge; lbm13_derive's status when it rejects the
 * parameter set. */
int lbm13_linear_growth(const lbm13_params *params, double ux, double uy, int n, double *growth);

/* The scan of lbm13_linear_growth for `count` cases at once on the current
 * device (the dispersion-root procedure of the end of Sec. 2, run for many
 * candidate parameter sets and flows): case c is parameter set params[c]
 * about u = (ux[c], uy[c]) on the n x n k-grid; growth[c] = max |z| - 1.  The
 * collision Jacobians are assembled on the host; one GPU thread per (case, k)
 * reduces the 13 x 13 amplification matrix to Hessenberg form and runs the
 * shifted QR iteration (the same code as the host scan).  Host arrays of
 * `count` entries, owned by the caller; `stream` is a cudaStream_t (NULL =
 * legacy default) that the call synchronises; its scratch comes from the
 * stream-ordered allocator and is released before it returns.  LBM13_EINVAL
 * for NULL, count < 1, n outside 1..129, a rejected parameter set or an
 * eigenvalue iteration that does not converge; LBM13_ECUDA on a CUDA error. */
int lbm13_linear_growth_batch(const lbm13_params *params, const double *ux, const double *uy, int count, int n,
                              double *growth, void *stream);

/* Create an nx x ny lattice (nx, ny >= 2; >= 4 along an axis that has walls,
 * plus 2 rows per halo side; nx <= 2^20, ny <= 32768, nx * ny < 2^31) on the
 * current CUDA device.  `alloc` may be NULL (cudaMalloc),
 * `stream` is a cudaStream_t (NULL = legacy default stream).  The state starts
 * at rest: rho = 1, u = 0, T = T0.  On success *out is a new handle.
 * LBM13_EUNSTABLE when sigma_q <= 0 or when the linearised step amplifies a
 * Fourier mode (lbm13_linear_growth on a 9 x 9 k-grid above 1e-9) at rest or,
 * where a wall moves, in a uniform flow at the largest wall speed along x and
 * along y. */
int lbm13_create(int nx, int ny, const lbm13_params *params, const lbm13_boundary *boundary,
                 int precision, const lbm13_allocator *alloc, void *stream, lbm13_t *out);

/* Release the device buffers (through the allocator) and the handle.  NULL is a no-op. */
void lbm13_destroy(lbm13_t h);

/* Last error message of this handle (static storage per handle). */
const char *lbm13_last_error(lbm13_t h);

/* Debug builds (compiled with LBM13_DEBUG): *count = the number of population
 * loads and stores of the step kernels on this lattice so far that fell
 * outside it (plane >= 13, row >= ny or column >= nx); each was counted and
 * redirected to the buffer's first element instead of being performed.
 * Release builds return LBM13_EINVAL with *count = 0 (nothing is checked). */
int lbm13_debug_violations(lbm13_t h, unsigned long long *count);

/* Change the stream the following calls are ordered on. */
int lbm13_set_stream(lbm13_t h, void *stream);

/* Lattice geometry: out[0] nx, out[1] ny, out[2] pitch (elements per row of a
 * population plane), out[3] precision, out[4] bytes per stored population,
 * out[5] device bytes held, out[6] time step counter, out[7] grid size of the
 * persistent multi-step launch (0 until one was considered, or if impossible). */
int lbm13_info(lbm13_t h, int64_t out[8]);

/* How lbm13_step runs n >= 2 steps: per-step launches (replayed from CUDA
 * graphs in runs of 32), or a persistent launch that advances the lattice by
 * up to 1024 steps in one cooperative launch whose co-resident blocks separate
 * the phases of each step by grid barriers (results are bit-identical).
 * AUTO (default) and OFF: per-step launches (on GB300 they are faster at every
 * size measured, 64^2 to 512^2); ON: persistent whenever a cooperative launch
 * is possible.  Every barrier wait is bounded (1 s); a timeout leaves the
 * state incomplete and is reported as LBM13_ETIMEOUT by the next synchronising
 * call (lbm13_synchronize, lbm13_residual, lbm13_moments, lbm13_project,
 * lbm13_get_raw_state, lbm13_save).  LBM13_EINVAL for another mode. */
#define LBM13_PERSISTENT_AUTO 0
#define LBM13_PERSISTENT_OFF 1
#define LBM13_PERSISTENT_ON 2
int lbm13_set_persistent(lbm13_t h, int mode);

/* Paired steps (FP32-deviation lattices periodic in x and y): lbm13_step
 * advances such a lattice two time steps per launch when it steps n >= 2 (an
 * odd n ends with one single step).  A paired launch reads the current buffer
 * once and writes the state two steps later to the other buffer: persistent
 * blocks take 28 x 28 tiles in turn, each stepping the tile and the two nodes
 * around it in shared memory, then the tile, while the next tile's input
 * arrives by tensor copy (the intermediate state never reaches HBM; DRAM
 * traffic 52 bytes per update instead of 104, with 15% more collisions).
 * Results are bit-identical to single steps.  AUTO (default): lattices of
 * 2^20 nodes or more (smaller ones step faster singly); ON: every such
 * lattice; OFF: one launch per step.  Every tensor copy's wait is bounded
 * (1 s); a timeout is reported as LBM13_ETIMEOUT like a persistent launch's.
 * Walled, slab (halo) and FP64 lattices, and persistent mode, step singly.
 * LBM13_EINVAL for another mode. */
#define LBM13_PAIR_AUTO 0
#define LBM13_PAIR_OFF 1
#define LBM13_PAIR_ON 2
int lbm13_set_pair_steps(lbm13_t h, int mode);

/* Kernel launches lbm13_step(h, n) makes with the lattice's current modes
 * (n per-step launches, n / 2 rounded up paired ones, or one per 1024 steps
 * of a persistent launch). */
int lbm13_step_launches(lbm13_t h, int64_t n, int64_t *launches);

/* Self-check of the paired steps' bounded wait: one paired launch from the
 * current state with its wait limited to timeout_s (1e-3 .. 2 s) and, when
 * withhold != 0, no tensor copy issued, so that every staged tile's wait runs
 * out, reports and leaves without writing.  *timed_out = 1 when the error
 * word was set (it is cleared again); the state and the step counter stay
 * as they were.  LBM13_EINVAL for a lattice that does not take paired steps. */
int lbm13_pair_check(lbm13_t h, double timeout_s, int withhold, int *timed_out);

/* Self-check of the grid barrier's bounded wait on the current device: a
 * cooperative launch of `blocks` blocks runs 4 barriers that wait for
 * blocks + extra_blocks arrivals.  With extra_blocks = 0 every barrier
 * completes (*timed_out = 0); with extra_blocks > 0 no barrier can, every wait
 * runs out after timeout_s and *timed_out = 1, and the context stays usable.
 * blocks in 1..1024 (and co-resident), extra_blocks in 0..1024, timeout_s in
 * [1e-3, 2]; LBM13_EINVAL outside, LBM13_ECUDA on a CUDA error. */
int lbm13_barrier_check(int blocks, int extra_blocks, double timeout_s, int *timed_out);

/* Set the state to the equilibrium of the given fields (host arrays [ny][nx];
 * any NULL field takes its rest value: rho 1, u 0, T T0):
 * f*_j = f_eq,j(rho, j = rho u, E = rho (26 T - 28) + 13 rho |u|^2).
 * Resets the step counter and the residual snapshot.  Returns when the state
 * is set (synchronises).  A lattice of 2^22 nodes or more is uploaded in eight
 * row bands on a second stream of the library's, each band's copies
 * overlapping the set-up of the band before (host arrays in page-locked
 * memory let the copies run asynchronously); the result is the same. */
int lbm13_set_state(lbm13_t h, const double *rho, const double *ux, const double *uy, const double *T);

/* As lbm13_set_state, with device arrays (no NULLs), stream-ordered. */
int lbm13_set_state_device(lbm13_t h, const double *rho, const double *ux, const double *uy, const double *T);

/* Checkpoint: write / read the stored post-collision populations, host
 * [13][ny][nx] doubles (in FP32-deviation mode converted from / to float
 * deviations).  set_raw resets the residual snapshot and sets the step
 * counter to `step`; get_raw returns the counter in *step when step != NULL. */
int lbm13_set_raw_state(lbm13_t h, const double *f, int64_t step);
int lbm13_get_raw_state(lbm13_t h, double *f, int64_t *step);

/* Bit-exact checkpoint of the stored state (in the storage precision, as
 * stored), for resuming a run.  lbm13_checkpoint_bytes gives the size of the
 * image: a 64-byte header (magic "LBM13CK1", nx, ny, precision, pitch, step
 * counter as int64) followed by the 13 population planes.  lbm13_save writes
 * the image into a host buffer of at least that size; lbm13_restore reads one
 * back into a lattice of the same nx, ny and precision (EINVAL otherwise) and
 * resets the residual snapshot.  Both synchronise. */
int lbm13_checkpoint_bytes(lbm13_t h, size_t *bytes);
int lbm13_save(lbm13_t h, void *host, size_t bytes);
int lbm13_restore(lbm13_t h, const void *host, size_t bytes);

/* Advance n >= 0 time steps: one fused stream + wall + collide kernel each,
 * launched on the lattice's stream (asynchronous); a large FP32 lattice
 * periodic in x and y takes two steps per launch (lbm13_set_pair_steps), a
 * lattice in persistent mode many (lbm13_set_persistent).  Runs of 32 steps
 * are replayed from CUDA graphs. */
int lbm13_step(lbm13_t h, int64_t n);

/* Selected moments/fields of the stored state (mask bits above), planes of
 * [ny][nx] doubles in increasing bit order, into a host buffer of
 * popcount(mask) * nx * ny doubles (synchronises).  A lattice of 2^22 nodes
 * or more is read out in eight row bands, each band's download (on a second
 * stream) overlapping the computation of the next. */
int lbm13_moments(lbm13_t h, double *out, unsigned mask);

/* As lbm13_moments into a device buffer (stream-ordered, asynchronous). */
int lbm13_moments_device(lbm13_t h, double *out, unsigned mask);

/* FP64 reductions of the stored state into out[16] (host; layout above;
 * synchronises).  Stores (ux, uy, T) as the snapshot for the next call.
 * Returns LBM13_EDIVERGED (after filling out) when a population is not finite.
 * The first call allocates the snapshot and reduction buffers. */
int lbm13_residual(lbm13_t h, double *out);

/* Fourier aggregates of Sec. 6, Eq. (d2q13-mesure) (V~_y = sum v_y cos kx,
 * rho~ and E~ at 2k), generalised: for the wave vector
 * k = 2 pi (kx / nx, ky / ny) (integers, any sign; reduced modulo nx, ny) and
 * its double 2k,
 *   out[LBM13_PROJ(f, h, c)] = sum over all nx*ny nodes of F_f trig_c((h+1) k . (x, y)),
 * h = 0 for k, 1 for 2k; c = 0 cos, 1 sin; (x, y) node indices.  The fields
 * F_f are deviations from the rest state: rho - 1, ux, uy, T - T0, E - E0,
 * p - T0, with u, T, p read as by lbm13_moments (half-way through the force
 * and the source); for a non-zero wave vector this equals the projection of
 * the field itself.  Sums run in FP64 in a fixed order (deterministic).
 * out: host, LBM13_PROJ_COUNT doubles.  Synchronises the lattice's stream.
 * LBM13_EINVAL for NULL; LBM13_ENOMEM if the small partial-sum buffer cannot
 * be allocated (allocated on the first call, kept until lbm13_destroy). */
enum { LBM13_P_RHO = 0, LBM13_P_UX = 1, LBM13_P_UY = 2, LBM13_P_T = 3, LBM13_P_E = 4, LBM13_P_P = 5 };
#define LBM13_PROJ_COUNT 24
#define LBM13_PROJ(f, h, c) (4 * (f) + 2 * (h) + (c))
int lbm13_project(lbm13_t h, int kx, int ky, double *out);

/* Time step counter. */
int64_t lbm13_time(lbm13_t h);

/* Wait for the lattice's stream. */
int lbm13_synchronize(lbm13_t h);

/* ---------------------------------------------------------------- plans
 * A plan steps many lattices together: one batched launch per time step
 * covers every tile of every lattice (uneven sizes, each with its own
 * parameters, walls and force), and runs of 32 steps are replayed as CUDA
 * graphs.  The per-node arithmetic is that of lbm13_step, so a lattice gives
 * bit-identical results alone or in a plan.  Each lattice's step counter and
 * buffers advance as with lbm13_step; the lattices must not be destroyed while
 * a plan holds them, and their own streams are not used by the plan. */
typedef struct lbm13_plan *lbm13_plan_t;

/* Plan over `count` distinct lattices of one precision and device.  The plan's
 * device table and work list come from `alloc` (NULL: cudaMalloc); `stream`
 * orders the plan's launches.  Default tile: 32 x 8 nodes, 8 CTAs per SM,
 * lattice-by-lattice order. */
int lbm13_plan_create(const lbm13_t *lattices, int count, const lbm13_allocator *alloc, void *stream,
                      lbm13_plan_t *out);
void lbm13_plan_destroy(lbm13_plan_t p);
const char *lbm13_plan_last_error(lbm13_plan_t p);

/* Advance every lattice of the plan by n >= 0 steps (asynchronous). */
int lbm13_plan_step(lbm13_plan_t p, int64_t n);

/* Per-lattice admission and retirement (the paper has no counterpart: they
 * serve a request loop that steps many solves together).  lbm13_plan_add
 * appends lattice h (same precision and device as the plan, not already in
 * it): the plan's stream first waits (event, no host synchronisation) for the
 * work already issued on h's own stream -- its creation and initial state --
 * then h's entry and tensor maps are written into a free slot of the plan's
 * device table by stream-ordered copies (the table doubles its capacity when
 * full, re-writing every entry once) and the work list is rebuilt.
 * lbm13_plan_remove takes h out (the last lattice moves into its slot, so the
 * order of the others in lbm13_plan_residual changes the same way) and makes
 * h's own stream wait for the plan's launches issued so far; h keeps its state
 * and step counter and may be stepped alone, added again or destroyed once its
 * stream has reached that point.  A plan keeps at least one lattice.  Neither
 * call synchronises the host with the device; the configuration (tile shape,
 * order) is kept, and captured step graphs are rebuilt on the next step.
 * LBM13_EINVAL for NULL, a mismatched or duplicate lattice (add), a lattice not
 * in the plan or the last one (remove). */
int lbm13_plan_add(lbm13_plan_t p, lbm13_t h);
int lbm13_plan_remove(lbm13_plan_t p, lbm13_t h);

/* Autotuner: times every candidate (rows per thread R and warps per block BY
 * of the tile, row groups per tile 1, 4 or 16, persistent CTAs per SM or one
 * CTA per tile, and the order of the tiles: by lattice, round robin, largest
 * first: 180 candidates; FP32 plans also the ring-staged strips of 64 and 32
 * columns with 4, 8, 16 or 32 groups in the three orders: 24 more) over steps_per_candidate real
 * steps each (+1 warm-up), then keeps the fastest.  The steps taken count as
 * simulation steps.  *best_ms_per_step (may be NULL) gets the best time. */
int lbm13_plan_tune(lbm13_plan_t p, int steps_per_candidate, double *best_ms_per_step);

/* Choose a configuration: (R, BY) in {(1,4), (2,4), (4,4), (2,2), (1,8)},
 * ctas_per_sm 0 (one CTA per tile) .. 64, order 0 by lattice, 1 round robin,
 * 2 largest first, groups 1 .. 64 row groups of BY * R rows per tile (a tile
 * is 32 columns x groups * BY * R rows).  LBM13_EINVAL outside these.  In an
 * FP32 plan, (4,4) with one CTA per tile stages each tile's populations
 * through shared memory by tensor copies (TMA), 8 rows at a time; and
 * (R, BY) = (0, 8) or (0, 4) (FP32 only; ctas_per_sm ignored) selects the
 * ring-staged strips: one CTA of BY warps per strip of 8 BY columns x groups
 * 4-row groups, whose input rows stream through a four-slot shared-memory ring
 * by tensor copies while the lattice's collision coefficients stay in
 * registers; the strips step the nodes two or more links from every edge, and
 * each lattice's edge nodes are further CTAs of the same launch (one node per
 * thread, global loads). */
int lbm13_plan_set_config(lbm13_plan_t p, int R, int BY, int ctas_per_sm, int order, int groups);

/* Self-check of the staged tiles' bounded wait (FP32 plan set to R = 4,
 * BY = 4, one CTA per tile, or to the ring-staged strips R = 0, BY = 8 or 4; else
 * LBM13_EINVAL): one staged launch with every
 * wait limited to timeout_s (1e-3 .. 2 s) and, when withhold != 0, no tensor
 * copy issued, so that every wait runs out and each block reports and leaves
 * without writing (the ring's edge-node CTAs, which do not wait, write nothing
 * in such a launch either).  *timed_out = 1 when the error word was set (it is cleared
 * again).  The plan does not advance: the lattices keep their states. */
int lbm13_plan_tma_check(lbm13_plan_t p, double timeout_s, int withhold, int *timed_out);

/* out: R, BY, ctas_per_sm, order, tiles, grid, total nodes, candidates tried
 * by the last tune, groups. */
int lbm13_plan_config(lbm13_plan_t p, int64_t out[9]);

/* FP64 reductions of every lattice of the plan, host out[count * 16] in the
 * layout of lbm13_residual (lattice i at out + 16 i), with a single
 * synchronisation of the plan's stream.  Each lattice's residual snapshot
 * advances as with lbm13_residual (a lattice's first call allocates its
 * reduction buffers through its own allocator).  Returns LBM13_EDIVERGED,
 * after filling out, when a lattice holds non-finite populations, and
 * LBM13_ETIMEOUT when a staged tile's tensor copy did not complete within
 * 1 s since the last call (its tile was left unstepped). */
int lbm13_plan_residual(lbm13_plan_t p, double *out);

/* y-slab halo exchange (the paper has no counterpart: it runs one lattice on
 * one GPU; this splits a lattice into y-slabs, one per device or one per
 * stream, that exchange two rows per side after every step).  A slab is a
 * lattice whose south and/or north side is LBM13_HALO; with nx columns and
 * ny rows (halo rows included) it must keep at least four rows that are not
 * halo rows.  A packed halo is [2 rows][4 populations][nx] in the lattice's
 * storage type (double, or float deviations f_j - w_j), *bytes of
 * lbm13_halo_bytes.
 *
 * lbm13_halo_pack(h, side, out): the two rows next to the halo rows of
 * `side` (rows 2, 3 for LBM13_HALO_SOUTH; ny-4, ny-3 for LBM13_HALO_NORTH) of
 * the stored state, populations that move across that side (v_y < 0:
 * 4, 7, 8, 12 at south; v_y > 0: 2, 5, 6, 10 at north), into the caller's
 * DEVICE buffer `out`, in stream order on h's stream.
 * lbm13_halo_unpack(h, side, in): writes a packed halo of the neighbouring
 * slab into h's halo rows of `side` (rows 0, 1 at south, ny-2, ny-1 at
 * north: the populations that move into h across that side), in stream order.
 * The lower slab's north pack is the upper slab's south unpack and vice versa;
 * the caller orders the streams of the two slabs (and moves the buffer between
 * devices where they differ).  LBM13_EINVAL for NULL, a side that is not
 * LBM13_HALO on h, or a lattice with fewer than four non-halo rows. */
#define LBM13_HALO_SOUTH 2
#define LBM13_HALO_NORTH 3
int lbm13_halo_bytes(lbm13_t h, size_t *bytes);
int lbm13_halo_pack(lbm13_t h, int side, void *out);
int lbm13_halo_unpack(lbm13_t h, int side, const void *in);

/* Measured FP64 instruction rate of the current device, the denominator of
 * the FP64 time step's roofline (that step is bound by its FP64 pipe, not by
 * HBM).  The paper has no counterpart.  Every SM runs 8 blocks of 256 threads,
 * each thread 8 independent FMA chains of `iters` FMAs (iters in 1..2^24),
 * timed with CUDA events after a warm-up launch on a stream of its own:
 * *fma_per_s = FMAs retired per second, *seconds (may be NULL) the timed
 * launch's duration.  LBM13_EINVAL for NULL fma_per_s or iters out of range,
 * LBM13_ECUDA if a CUDA call fails. */
int lbm13_fp64_fma_rate(int iters, double *fma_per_s, double *seconds);

/* Largest lattice (nx * ny) that lbm13_totals_noalloc accepts. */
#define LBM13_NOALLOC_MAX_NODES 67108864

/* Conserved totals of the stored state without allocating anything.
 * The paper has no counterpart; this is a service for callers that cannot
 * allocate device memory at the moment they need the totals: a serving loop
 * that has handed every byte of its HBM budget to lattices through another
 * allocator (one more buffer would break the budget or fail), a latency-bound
 * loop that cannot afford the device-wide synchronisation cudaMalloc and
 * cudaFree may impose, and code running inside an allocator callback, which
 * must not re-enter that allocator.  lbm13_residual allocates its reduction
 * buffers on its first call; this call never calls cudaMalloc, cudaFree or
 * any allocating routine.
 *
 * out is a caller-owned DEVICE buffer of 8 doubles, written in stream order on
 * the lattice's stream (the call returns before the work ends): 0 sum rho,
 * 1 sum j_x, 2 sum j_y, 3 sum E (stored post-collision moments, as
 * LBM13_R_MASS..LBM13_R_ENERGY of lbm13_residual), 4 number of non-finite
 * populations, 5 max |u|, 6 mean T, 7 nx * ny.  The call reads the population
 * buffer that holds the lattice's state when the call is made.
 *
 * Scratch: a file-scope device array of 256 KiB (4096 x 8 doubles) that every
 * GPU loading the library holds until the process exits; lattices of up to
 * LBM13_NOALLOC_MAX_NODES nodes fit (larger ones return LBM13_EINVAL).  The
 * first call on a device (and the first after that device's context was
 * replaced, e.g. by cudaDeviceReset) looks up that array's device address with
 * the device current; make that first call before any stream capture.  Every
 * call reuses the same array and each call's blocks overwrite their rows before
 * they are read, so nothing needs clearing; calls whose work overlaps on the
 * GPU (other streams, other lattices) race on it.  Returns LBM13_EINVAL for a
 * NULL argument or an oversized lattice, LBM13_ECUDA if the lattice's device
 * cannot be made current or one of the call's own launches fails. */
int lbm13_totals_noalloc(lbm13_t h, double *out);

#ifdef __cplusplus
}
#endif

#endif /* LBM13_H */
