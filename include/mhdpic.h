/*
 * mhdpic.h - C ABI of the GB300 (sm_103a) cosmic-ray particle update of the
 * MHD-PIC method (Bai, Caprioli, Sironi & Spitkovsky, arXiv:1412.1087).
 *
 * One particle step, as the paper defines it:
 *   - the cell-centred electric field E = E0 - F_CR/n_g with E0 = -v_g x B
 *     (Section 2.1, eq:emf0, eq:lorentz2, eq:emfcr2; used by the particles as
 *     stated in Section 2.2);
 *   - drift half a step, TSC interpolation of E and B (Section 3), removal of
 *     the E component along B, relativistic Boris kick-rotate-kick with an
 *     artificial light speed C, drift half a step (Appendix A.2);
 *   - TSC deposit of -m dv and -m dE_k at the half-step position (the
 *     corrector of Appendix A.3) and of the charge and current densities
 *     n_CR, J_CR at the new position (Appendix A.1, eq:nJCR);
 *   - applying the corrector deposit to the gas momentum and energy
 *     (Section 2.1: Newton's third law and eq:eng; Appendix A.3).
 * Units are the paper's code units: the factor c is absorbed into E and J.
 *
 * All calls are asynchronous on the stream given at init unless stated; none
 * aborts.  Every call returns MHDPIC_OK (0) or a negative MHDPIC_E* code;
 * mhdpic_strerror() gives a message and mhdpic_last_error() the detail of the
 * last failure on the calling thread.
 *
 * Ownership: the caller owns every particle and gas buffer (plain pointers,
 * device memory unless options.memory is MHDPIC_MEM_HOST, where all of them
 * are host memory, or MHDPIC_MEM_HOST_GAS, where the gas buffers are).  The
 * library owns only its scratch (sort keys, permutation, a second particle
 * set, staged fields, fixed-point deposit grids, work list, status word),
 * allocated by mhdpic_init and freed by mhdpic_destroy.  The particle state
 * alternates between the caller's buffers and the second set (see
 * mhdpic_sort); mhdpic_sync_particles brings it back into the caller's.
 * Buffers must stay valid and unmoved between init and destroy.
 *
 * Layouts (np = total particles of all boxes, nc = total cells of all boxes):
 *   particles, box-major: box b owns particles [box_start[b], box_start[b+1]);
 *   MIXED:  pos[np]          mhdpic_pos, 16 bytes: the linear cell of the
 *                            particle inside its box, c = (k*ny + j)*nx + i,
 *                            and its offset in [0,1) inside the cell along
 *                            each dimension (off[2] = 0 in 2-D);
 *           vel[np]          mhdpic_vel, 16 bytes: the four-velocity
 *                            v = gamma*u (eq:4vel) as a two-word number, an
 *                            FP32 leading word per component plus a packed
 *                            residual (below);
 *   FP64:   x[ndim*np]       double, absolute position, plane-major;
 *           p64[3*np]        double, four-velocity;
 *   gas (cells box-major, box b's cells start at the sum of earlier boxes'
 *   cell counts, c as above inside a box):
 *           rho[nc], mom[3*nc] (momentum density rho*v_g, plane-major),
 *           egas[nc] (total energy density), B[3*nc] (cell-centred field).
 */
#ifndef MHDPIC_H
#define MHDPIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define MHDPIC_OK 0
#define MHDPIC_E_ARG (-1)      /* invalid argument (message in mhdpic_last_error) */
#define MHDPIC_E_CUDA (-2)     /* a CUDA runtime call failed */
#define MHDPIC_E_NOMEM (-3)    /* device allocation failed */
#define MHDPIC_E_STATUS (-4)   /* a device status flag is set (mhdpic_get_status) */
#define MHDPIC_E_CAPACITY (-5) /* a size limit of the library was exceeded */
#define MHDPIC_E_STATE (-6)    /* call made in the wrong state (e.g. destroyed ctx) */

/* ---- enumerations ---- */
#define MHDPIC_BC_PERIODIC 0
#define MHDPIC_BC_REFLECT 1 /* conducting wall: specular particle reflection, mirror-folded stencil */
/* conducting wall at the lower face, open (inflow) upper face, as the paper's
 * shock box along x (Section 5): a particle that reaches the open face is held
 * just inside it for its gather and corrector deposit, then leaves the box;
 * stencil cells beyond the open face take the last cell's fields and deposits.
 * Only for single-box contexts.  A particle that left is marked (MIXED:
 * cell = -1; FP64: x[0] = NaN; four-velocity 0) and dropped to the end of the
 * particle arrays by the next mhdpic_sort; mhdpic_live_particles counts the
 * rest, and the free slots at the end take injected particles. */
#define MHDPIC_BC_WALL_OPEN 2
#define MHDPIC_SHAPE_TSC 2  /* triangular-shaped cloud (quadratic spline), Section 3 */
#define MHDPIC_PREC_FP64 0  /* all particle arithmetic in double */
#define MHDPIC_PREC_MIXED 1 /* int32 cell + f32 offsets, f32 push, two-word four-velocity, int64 fixed-point deposits */
#define MHDPIC_MEM_DEVICE 0 /* caller buffers are device pointers */
#define MHDPIC_MEM_HOST 1   /* caller buffers are (pinned) host pointers; each call copies */
#define MHDPIC_MEM_HOST_GAS 2 /* particle buffers on the device, gas buffers (pinned) host pointers:
                               * the particles stay resident and each call copies only the gas
                               * arrays it reads or writes (a host MHD solver coupled to the push);
                               * the gas upload of a feedback that directly follows a push runs on
                               * a second stream of the library's beside that push, still after
                               * the call is made and after the work queued before the push */

#define MHDPIC_SPEC_ENERGY 0     /* spectrum of E_k = v^2/(gamma+1) per unit mass (eq:parEk) */
#define MHDPIC_SPEC_MOMENTUM 1   /* spectrum of |v| = p/m (four-velocity magnitude) */
#define MHDPIC_SPEC_MAX_BINS 2048

/* ---- device status flags (sticky until mhdpic_clear_status) ---- */
#define MHDPIC_ST_FAST_MOVER 1u /* a particle moved more than 2 cells in one half step (App. A.4) */
#define MHDPIC_ST_NONFINITE 2u  /* a non-finite position or four-velocity was produced */
#define MHDPIC_ST_OVERFLOW 4u   /* a fixed-point deposit exceeded its headroom */
#define MHDPIC_ST_SORT_CAP 8u   /* a cell held more particles than the sort's segment limit */
#define MHDPIC_ST_CELL_RANGE 16u/* a particle's cell index was outside its box */
#define MHDPIC_ST_INJECT_CAP 32u/* mhdpic_inject ran out of free particle slots */
#define MHDPIC_ST_BARRIER 64u   /* a grid-wide barrier of the one-launch step waited beyond its limit:
                                 * that step's results are not valid */
#define MHDPIC_ST_COPY_TIMEOUT 128u /* a tensor copy of a push's field tile did not complete within its
                                     * limit: that push's results are not valid */

typedef struct mhdpic_ctx mhdpic_ctx;

/* Grid of one box.  2-D boxes have ndim = 2, n[2] = 1; dx[2] is then the cell
 * depth that enters the cell volume dV = dx[0]*dx[1]*dx[2]. */
typedef struct {
    int32_t ndim;  /* 2 or 3 */
    int32_t n[3];  /* cells per dimension */
    double dx[3];  /* cell widths (> 0) */
    double x0[3];  /* lower corner of the box */
    int32_t bc[3]; /* MHDPIC_BC_PERIODIC, MHDPIC_BC_REFLECT or MHDPIC_BC_WALL_OPEN, per dimension */
} mhdpic_grid;

/* Physical parameters of one box (Sections 2.2, App. A.1). */
typedef struct {
    double qm_cr;  /* (q/mc) of the CR species */
    double qm_gas; /* (q/mc)_g of the gas ions: n_g = qm_gas * rho (eq:ng) */
    double C;      /* artificial speed of light (Section 2.2) */
    double m_cr;   /* particle "mass" m_CR (App. A.1) */
    int32_t hall;  /* 1: E = E0 - F_CR/n_g (eq:emfcr2); 0: E = E0 */
    int32_t shape; /* MHDPIC_SHAPE_TSC (the only shape the paper uses) */
} mhdpic_params;

/* Library options, shared by all boxes of a context. */
typedef struct {
    int32_t precision; /* MHDPIC_PREC_MIXED or MHDPIC_PREC_FP64 */
    int32_t memory;    /* MHDPIC_MEM_DEVICE, MHDPIC_MEM_HOST or MHDPIC_MEM_HOST_GAS */
    int32_t brick[3];  /* cells per sort brick and per push tile (0: 4x4x4 in 3-D, 8x8 in 2-D) */
    int32_t reserved[8];
} mhdpic_options;

/* Mixed-precision particle position: 16 bytes, one 128-bit load or store. */
typedef struct {
    int32_t cell;  /* linear cell inside the box; -1 marks a free slot or a particle that left */
    float off[3];  /* offset in [0,1) inside the cell per dimension (unused entries 0) */
} mhdpic_pos;

/*
 * Mixed-precision four-velocity: 16 bytes, one 128-bit load or store.  The
 * value of component d is the exact sum
 *     v[d] + r_d * 2^(e_d - 33),
 * with e_d the binary exponent of v[d] (|v[d]| in [2^e_d, 2^(e_d+1)), taken
 * as -90 when |v[d]| < 2^-90, zero included) and r_d the signed 10-bit field
 * of lo in bits 10d .. 10d+9 (|r_d| <= 511): 34 significant bits, about
 * 2^-35 of |v[d]| per rounding.  The push adds each step's change dv, the
 * very value it deposits as the corrector (App. A.3), to this two-word
 * number, so what the particle stores changes by what the gas is given up to
 * that last rounding (an FP32 word alone would round every step at 2^-25 and
 * drift measurably over 1000 steps).  The leading words alone are the FP32
 * four-velocity the push computes with; lo = 0 is a plain FP32 value.
 */
typedef struct {
    float v[3];
    uint32_t lo;
} mhdpic_vel;

/* Caller-owned particle buffers (see the layout above). */
typedef struct {
    int64_t np;               /* total particles (may be 0) */
    const int64_t *box_start; /* HOST array [nbox+1], box_start[0] = 0, box_start[nbox] = np */
    mhdpic_pos *pos;          /* MIXED, 16-byte aligned */
    mhdpic_vel *vel;          /* MIXED, 16-byte aligned */
    double *x;                /* FP64 */
    double *p64;              /* FP64 */
} mhdpic_particles;

/* Caller-owned gas buffers (see the layout above). rho and B are read only. */
typedef struct {
    double *rho;
    double *mom;
    double *egas;
    double *B;
} mhdpic_gas;

/*
 * mhdpic_init - validate a batch of nbox independent boxes, allocate scratch,
 * choose the fixed-point scales, sort the particles (as mhdpic_sort), deposit
 * their charge and current (as mhdpic_deposit) and stage the fields.
 *   ctx     out: new context (NULL on failure)
 *   grids, params: host arrays [nbox]
 *   stream: cudaStream_t (NULL = legacy default stream) used by every call
 * Positions must lie inside their box; the caller's particle buffers are
 * sorted in place.  Synchronises the stream once (it reads per-cell counts
 * back).
 */
int mhdpic_init(mhdpic_ctx **ctx, int32_t nbox, const mhdpic_grid *grids,
                const mhdpic_params *params, const mhdpic_options *options,
                const mhdpic_particles *particles, const mhdpic_gas *gas, void *stream);

/*
 * mhdpic_sort - stable counting sort of each box's particles by cell key: the
 * brick number (bricks of options.brick cells, numbered x fastest) times the
 * brick volume plus the cell's x-fastest number inside its brick.  The paper
 * has no sort (cell ordering is this library's layout).  The push work list is
 * rebuilt at once; the particle arrays are permuted by the next
 * mhdpic_interp_push, which reads its particles through the permutation and
 * writes them, sorted and advanced, into the library's second particle set
 * (no separate pass over the particles).  Until mhdpic_sync_particles the
 * caller's device buffers may therefore hold an earlier state; in
 * MHDPIC_MEM_HOST mode the host buffers are sorted on return.
 *   perm_out   device int64[np] or NULL: perm_out[r] = index, in the order
 *              the caller last saw, of the particle now at rank r (global
 *              indices); asking for it applies any earlier pending sort
 *   counts_out device int32[nkeys] or NULL: particles per key, keys of box b
 *              after those of earlier boxes (nkeys from mhdpic_num_keys)
 */
int mhdpic_sort(mhdpic_ctx *ctx, int64_t *perm_out, int32_t *counts_out);

/*
 * mhdpic_interp_push - nsub particle sub-steps of length dt with the staged
 * fields held fixed (App. A.2; sub-cycling as in App. A.4).  Each sub-step
 * drifts, interpolates E and B by TSC at x^(n+1/2), removes E along B, applies
 * the relativistic Boris kick-rotate-kick and drifts again; it adds
 * (-m dv, -m dE_k) at x^(n+1/2) to the corrector accumulators (App. A.3).  The
 * last sub-step also deposits n_CR and J_CR at the new positions (eq:nJCR),
 * which the next field staging uses.  dt must be > 0, nsub >= 1.
 * Conservation: with MHDPIC_PREC_FP64 the corrector deposit is the change the
 * particle stores, so gas + CR momentum and energy pass through
 * mhdpic_apply_feedback to roundoff.  With MHDPIC_PREC_MIXED dv is formed
 * without cancellation from the two kicks and the rotation (accurate to
 * about 1e-7 of dv itself), deposited, and added to the particle's two-word
 * four-velocity (mhdpic_vel), which holds it to about 2^-35 of |v|: the
 * stored change is the deposited one to that rounding, and dE_k is the
 * change of the two half kicks (the rotation keeps |v|).
 */
int mhdpic_interp_push(mhdpic_ctx *ctx, double dt, int32_t nsub);

/*
 * mhdpic_set_subcycle_sort - with every > 0, mhdpic_interp_push re-sorts the
 * particles after every `every` sub-steps of one call (not after the last),
 * so that long sub-cycles keep their particles near their cells' tiles.  The
 * results do not depend on it, bit for bit (the fixed-point sums depend
 * neither on the order of the particles nor on how they fall into work
 * items); only the particle order and the speed do.  0 (the default) never sorts
 * inside a call.  Returns MHDPIC_E_ARG for every < 0.
 */
int mhdpic_set_subcycle_sort(mhdpic_ctx *ctx, int32_t every);

/*
 * mhdpic_set_sort_lookahead - from the next sort on (mhdpic_sort, the sorts of
 * mhdpic_run and of sub-cycles), key each particle by the cell it reaches
 * after moving for time t at its current velocity, instead of its current
 * cell: with t = dt/2 the cell of the half-step position where the next push
 * gathers E, B and deposits the corrector (App. A.2-A.3), so that the push
 * finds its particles in the cells it works on.  The sorts of mhdpic_run,
 * made every k steps, look k t ahead (with t = dt/2 the mean half-step
 * position of the k pushes of the cycle); mhdpic_sort looks t ahead.  Per dimension the cell moves
 * by -1, 0 or +1 (a half step moves a particle well under one cell): +1 when
 * v_d > 0 and (a_d v_d)^2 >= ((1 - o_d)(1 - o_d)) g2, -1 when v_d < 0 and
 * (a_d v_d)^2 > (o_d o_d) g2, with g2 = 1 + v^2 w (gamma^2), v^2 =
 * (vx vx + vy vy) + vz vz, a_d = t/dx_d rounded from double to float and
 * w = 1/(C C) in FP32, o_d the offset in the cell (FP64 precision:
 * (x_d - x0_d)/dx_d minus its cell, as float) and v the FP32 four-velocity
 * (the FP64 one rounded to float), every operation a correctly rounded FP32
 * one in this order (the faces of o_d + a_d v_d/gamma tested on squares: no
 * square root, no division); the cell wraps on periodic faces and is clamped
 * into the box otherwise.  The call is ordered on the context's stream.  Only
 * the order of the particles and the speed depend on t: the deposits, the gas
 * and the particle states are the same bit for bit.
 * 0 (the default) sorts by the current cell.  The paper has no sort.
 * Errors: MHDPIC_E_STATE, MHDPIC_E_ARG for a non-finite t.
 */
int mhdpic_set_sort_lookahead(mhdpic_ctx *ctx, double t);

/*
 * mhdpic_sync_particles - make the caller's particle buffers hold the current
 * particle state: apply a pending sort and copy the library's second set back
 * if it is the current one.  Call it before reading or writing the caller's
 * particle buffers in MHDPIC_MEM_DEVICE / MHDPIC_MEM_HOST_GAS mode; the
 * caller's buffers then stay current until the next mhdpic_sort (a no-op in
 * MHDPIC_MEM_HOST mode, where the host buffers are current once the stream
 * has finished each call: synchronise it before reading them).
 * Asynchronous; ordered on the context's stream.
 */
int mhdpic_sync_particles(mhdpic_ctx *ctx);

/*
 * mhdpic_spectrum - particle spectrum of every box (the diagnostics of
 * Section 4.3: the energy spectrum f(E) of eq:dpdE, its momentum form, and
 * the E_max of eq:emax).  The binned quantity q of a particle is
 * E_k = v^2/(gamma+1) with gamma = sqrt(C^2 + v^2)/C (kind
 * MHDPIC_SPEC_ENERGY) or |v| (MHDPIC_SPEC_MOMENTUM), v the four-velocity and
 * v^2 = (vx^2 + vy^2) + vz^2, all in IEEE double arithmetic in this order.
 *   kind        MHDPIC_SPEC_ENERGY or MHDPIC_SPEC_MOMENTUM
 *   nbins       1 .. MHDPIC_SPEC_MAX_BINS
 *   edges       host double[nbins + 1], finite and strictly ascending; a
 *               particle counts in bin b when edges[b] <= q < edges[b+1]
 *               (outside [edges[0], edges[nbins]) it is not counted)
 *   region      host double[6] {lo_x, hi_x, lo_y, hi_y, lo_z, hi_z} or NULL:
 *               only particles with lo_d <= x_d < hi_d for every d < ndim
 *               count (x_d = x0_d + (i_d + offset_d) dx_d in double in mixed
 *               precision); NULL counts the whole box
 *   n_moment    the integer n of eq:emax, 0 .. 64
 *   counts_out  host int64[nbox * nbins], box-major
 *   sums_out    host double[2 * nbox] or NULL: per box, the sums of
 *               q^(n+1) and q^n over the counted particles (E_max of eq:emax
 *               is their ratio for the energy kind)
 * Reads the current particle state (a pending sort does not change the
 * counts).  Synchronises the stream.
 */
int mhdpic_spectrum(mhdpic_ctx *ctx, int32_t kind, int32_t nbins, const double *edges, const double *region,
                    int32_t n_moment, int64_t *counts_out, double *sums_out);

/*
 * mhdpic_lambda_map - the CR-Hall parameter Lambda = R (u_CR - v_g)/v_A of
 * eq:lambda per cell, with R = n_CR/(n_g + n_CR) (eq:defR), n_g = (q/mc)_g rho
 * (eq:ng), u_CR = J_CR/n_CR, v_g = (rho v)/rho and v_A = |B|/sqrt(rho),
 * evaluated as (J_CR - n_CR v_g) / ((n_g + n_CR) v_A) from the latest charge
 * and current deposit and the gas state; 0 where |B| = 0.
 *   out  device double[3 * nc], plane-major (component d at out[d*nc + c])
 * In host-memory modes the gas is read from the caller's host buffers.
 */
int mhdpic_lambda_map(mhdpic_ctx *ctx, double *out);

/*
 * mhdpic_deposit - TSC deposit of n_CR = (q/mc) m_CR W/dV and
 * J_CR = (q/mc) m_CR u W/dV (App. A.1, eq:nJCR) at the current positions,
 * replacing the current moments, then restage the fields from the gas and
 * these moments.  The corrector accumulators are left untouched.  Mixed
 * precision deposits through the push's shared tile over the work list of a
 * sort of the current particles: a pending sort is used, else the call sorts
 * (the next push applies it; the caller's order is unchanged until then);
 * each particle adds the same fixed-point integers as the push that put it
 * where it is, so right after a push the moments come out bit for bit the
 * same.  FP64 deposits straight into the global accumulators.
 */
int mhdpic_deposit(mhdpic_ctx *ctx);

/*
 * mhdpic_apply_feedback - add the accumulated corrector deposit to the gas:
 * rho*v += dM/dV, egas += dE/dV (Section 2.1, App. A.3), zero the
 * accumulators, and restage E, B for the next push from the updated gas and
 * the latest moments (eq:emf0, eq:lorentz2, eq:emfcr2).
 *   totals_out HOST double[8*nbox] or NULL.  When given, the call also forms
 *   per box the FP64 totals {P_gas x,y,z, E_gas, P_CR x,y,z, E_CR} with
 *   P_gas = sum rho*v dV, E_gas = sum egas dV, P_CR = sum m v,
 *   E_CR = sum m E_k (eq:parEk) in a fixed-order reduction, and synchronises
 *   the stream to return them.
 */
int mhdpic_apply_feedback(mhdpic_ctx *ctx, double *totals_out);

/*
 * mhdpic_live_particles - number of particles that have not left the box
 * through an open face (MHDPIC_BC_WALL_OPEN), counted over the current state.
 *   live_out  host int64
 * Synchronises the stream.
 */
int mhdpic_live_particles(mhdpic_ctx *ctx, int64_t *live_out);

/*
 * mhdpic_inject - shock front tracking and CR injection (Section 5), for a
 * single box with MHDPIC_BC_WALL_OPEN along x (the wall at x0, the inflow
 * face at the far end).
 *   front: the transverse average of v_x = (rho v_x)/rho per x cell, smoothed
 *   with a Gaussian of standard deviation 4 cells (truncated at 3 standard
 *   deviations and at the box ends, renormalised); v_up, rho_up are the
 *   smoothed values of the last (inflow) cell; x_s is where, coming from
 *   upstream, |v_x| first falls to 0.6 |v_up| (linear interpolation between
 *   cell centres); the tail x_t is the centre of the first cell at or below
 *   the front cell whose smoothed pressure P = (gamma-1)(egas - rho v^2/2 -
 *   B^2/2) reaches 2/3 of P1 = r/(r-1) rho_up v_up^2 (eq:rh,
 *   r = (gamma+1)/(gamma-1)), x0 if none.
 *   injection: the gas mass swept in this step, rho_up (|v_up| + max(V, 0))
 *   dt A (A the box cross-section, V the front speed since the previous call,
 *   0 on the first), times eta, becomes CR particles of mass m_CR; the
 *   fraction of a particle left over is carried to the next call.  Particle
 *   k sits at x = x_s, uniform across the box, with an isotropic direction
 *   and kinetic energy per unit mass energy_factor * v_up^2/2 in the frame of
 *   the front (the paper: 10 E_sh), boosted by V along x.  Random numbers:
 *   Philox4x32-10, counter (k, call number, 0, 0), key = seed.
 *   compensation: the gas gives the injected mass, momentum (m_CR sum v) and
 *   energy (m_CR sum E_k) evenly from the cells with centres in [x_t, x_s)
 *   (the front's cell column when there are none), so gas + CR momentum and
 *   energy are unchanged.
 * The new particles take the free slots past the live particles of the last
 * sort (which puts particles that left the box, and caller slots marked free
 * with cell -1 / x NaN, after all others; particles that left since are
 * collected by the next sort); when they run out the count is cut and
 * MHDPIC_ST_INJECT_CAP is raised.  The call sorts after injecting (the next
 * push applies the sort); the charge/current deposit is not redone
 * (mhdpic_deposit does), and the next push (or mhdpic_run) first stages the
 * fields of the compensated gas.  Without a front nothing is injected.
 *   dt, eta, energy_factor, gamma_gas  as above (dt > 0, eta >= 0)
 *   seed       key of the random numbers
 *   front_out  host double[2] {x_s (NaN without a front), x_t} or NULL
 *   ninj_out   host int64, particles injected, or NULL
 * Synchronises the stream.  Errors: MHDPIC_E_ARG for a context that is not a
 * single box with MHDPIC_BC_WALL_OPEN along x, or bad arguments.
 */
int mhdpic_inject(mhdpic_ctx *ctx, double dt, double eta, double energy_factor, double gamma_gas, uint64_t seed,
                  double *front_out, int64_t *ninj_out);

/*
 * mhdpic_set_injection_times - early-particle removal (Section 5: the CRs
 * injected before the Bell instability has grown cross the upstream
 * unscattered, so every particle with injection time t_i < t_early is
 * removed at t = 2 t_i).  Turns on a per-particle injection time and a
 * clock, or resets them.
 *   t_inj    host double[np], t_i of each slot in the order of the caller's
 *            particle arrays as they stand after this call (the call brings
 *            them up to date, like mhdpic_sync_particles), or NULL for +inf
 *            (never removed); free slots' values are not used
 *   t_now    the current time (finite)
 *   t_early  the threshold (not NaN; -inf removes nothing)
 * From then on each push sub-step advances the clock by its dt first; a live
 * particle with t_i < t_early and clock >= 2 t_i is removed at the end of
 * that push, the same way as a particle that leaves through an open face
 * (its corrector deposit of the step stands, no charge/current deposit, cell
 * -1 / x NaN and velocity 0, collected by the next sort).  mhdpic_inject sets
 * t_i of each new particle to the clock.  The injection times follow every
 * sort.  A graph captured by mhdpic_run before the call is discarded.
 * Synchronises the stream.  Errors: MHDPIC_E_ARG for a non-finite t_now or a
 * NaN t_early; MHDPIC_E_NOMEM.
 */
int mhdpic_set_injection_times(mhdpic_ctx *ctx, const double *t_inj, double t_now, double t_early);

/*
 * mhdpic_get_injection_times - read back the injection times and the clock.
 *   t_inj  host double[np] (order of the caller's arrays after the call, which
 *          brings them up to date), or NULL
 *   t_now  host double, the clock, or NULL
 * Synchronises the stream.  Errors: MHDPIC_E_STATE when
 * mhdpic_set_injection_times was never called.
 */
int mhdpic_get_injection_times(mhdpic_ctx *ctx, double *t_inj, double *t_now);

/* ---- gas models of the coupled step ---- */
#define MHDPIC_GAS_SOURCES 0   /* the gas changes by the CR sources alone; B is held */
#define MHDPIC_GAS_LINEAR_X 1  /* plus plane-parallel linear MHD along x (below) */

/*
 * mhdpic_gas_predict - predictor of the coupled MHD-PIC step (App. A.3,
 * eq:scheme, first line): the half-step gas state
 *   g^(n+1/2) = g^n + G(f^n, g^n) dt/2
 * into library scratch (the caller's gas is not changed), and the cell fields
 * of g^(n+1/2) staged for the next mhdpic_interp_push.  The CR part of G comes
 * from the latest charge and current deposit (n, J at x^n): momentum
 * -F_CR = -(1-R)(n E0 + J x B) (eq:gasmotion, eq:lorentz2) and energy
 * -(1-R) J.E0 (eq:engeq), with R = n/(n_g + n) when the box has the CR-Hall
 * term and R = 0 otherwise; the staged field is E0 = -v_g x B, minus F_CR/n_g
 * with the CR-Hall term (eq:emfcr2), from the half state and the same n, J.
 *   dt     the step (> 0); the push and mhdpic_gas_correct take the same dt
 *   model  MHDPIC_GAS_SOURCES: no other gas evolution;
 *          MHDPIC_GAS_LINEAR_X: rho and B_x taken as uniform and v_x = 0 to
 *          first order, the transverse momentum and field follow the 1-D
 *          linear MHD equations d(rho v_y,z)/dt = B_x dB_y,z/dx,
 *          dB_y,z/dt = B_x dv_y,z/dx plus the curl of the CR-Hall field
 *          (dB_y/dt -= d(F_z/n_g)/dx, dB_z/dt += d(F_y/n_g)/dx), with centred
 *          differences; every box must be periodic along x.  The gas energy
 *          takes only the CR sources in both models.
 * The first call allocates the half-state scratch (8 doubles per cell) with
 * cudaMalloc.  Errors: MHDPIC_E_ARG for dt <= 0, an unknown model or a box
 * that is not periodic along x under MHDPIC_GAS_LINEAR_X.
 */
int mhdpic_gas_predict(mhdpic_ctx *ctx, double dt, int32_t model);

/*
 * mhdpic_gas_correct - corrector of the coupled step (App. A.3, eq:scheme,
 * third line): the caller's gas advances to
 *   g^(n+1) = g^n + G((f^n + f^(n+1))/2, g^(n+1/2)) dt,
 * where the CR part is the corrector deposit accumulated by the pushes since
 * the predictor (rho v += dM/dV, egas += dE/dV, App. A.3) and the gas part is
 * the model's, evaluated at the half state of mhdpic_gas_predict; with the
 * CR-Hall term the induction takes the curl of -F_CR/n_g with
 * F_CR = -dM/(dV dt), the force the deposit implies.  rho is unchanged; mom,
 * egas and B are written (back to the caller's host buffers in host-memory
 * modes).  The accumulators are zeroed.  The staged fields are then stale:
 * mhdpic_gas_predict stages the next step's half-step fields, and a push or
 * mhdpic_run called first stages the fields of the corrected gas itself (as
 * mhdpic_apply_feedback would, without a corrector to apply).
 *   dt, model  as given to mhdpic_gas_predict
 *   totals_out HOST double[8*nbox] or NULL, as for mhdpic_apply_feedback
 * Errors: MHDPIC_E_STATE when no predictor ran since the last corrector,
 * MHDPIC_E_ARG when dt or model differ from the predictor's.
 */
int mhdpic_gas_correct(mhdpic_ctx *ctx, double dt, int32_t model, double *totals_out);

/*
 * mhdpic_run - nsteps full steps, each mhdpic_interp_push(dt, 1) followed by
 * mhdpic_apply_feedback(NULL), with mhdpic_sort after every sort_every-th
 * step (counted across calls).  sort_every = 0 lets the library choose the
 * cadence: the first call runs one warm-up step, then times whole cycles of
 * 1, 2, 3 and 4 steps (at least four steps per candidate, 19 steps in all
 * while nsteps lasts) on real steps that count toward nsteps, and keeps the
 * fastest (mhdpic_sort_cadence).
 * Whole cycles are captured once into a CUDA graph and replayed (re-captured
 * when dt or the cadence changes); with the legacy default stream or host
 * buffers the steps run eagerly.  Each step without a sort is one kernel
 * launch where mhdpic_set_step_fusion allows it; with a sort every step and
 * device buffers or the gas in host memory, the feedback runs on a second
 * stream beside the sort.
 * Asynchronous except while tuning.
 */
int mhdpic_run(mhdpic_ctx *ctx, double dt, int32_t nsteps, int32_t sort_every);

/*
 * mhdpic_set_step_fusion - with enable != 0 (the default) each step of
 * mhdpic_run is one kernel launch where it can be: the corrector scales, the
 * push with both deposits, and the feedback with the field staging for the
 * next step run in one persistent cooperative kernel, its phases separated by
 * grid-wide barriers (the paper's particle step of App. A.2-A.3 followed by
 * the corrector's feedback, eq:scheme); a step with a sort adds the sort's
 * launches.  At a sort cadence of 1 with device buffers or the gas in host
 * memory (either precision) it instead puts each step's feedback and field
 * staging (and the gas copies of MHDPIC_MEM_HOST_GAS) on a second stream
 * beside the sort that follows the push, the two joined before the next
 * step; with enable == 0 they run in turn on the context's stream.  The
 * one-launch step applies to mixed precision with device buffers and no open
 * face or injection times (mhdpic_step_fusion tells whether it does); the
 * results are the same bit for bit as those of mhdpic_interp_push(dt, 1)
 * followed by mhdpic_apply_feedback(NULL).  Each barrier waits at most one
 * second by default; a wait that runs out raises MHDPIC_ST_BARRIER (the step's
 * results are then not valid) instead of hanging.  A captured cycle is
 * discarded.  The paper has no counterpart.  Errors: MHDPIC_E_STATE.
 */
int mhdpic_set_step_fusion(mhdpic_ctx *ctx, int32_t enable);

/* 1 when mhdpic_run's steps of this context are one-launch steps, 0 when not,
 * -1 for an invalid context. */
int32_t mhdpic_step_fusion(const mhdpic_ctx *ctx);

/*
 * mhdpic_set_field_tma - with enable != 0 (the default where possible) a push
 * stages each work item's field tile, the cell-centred E and B of the tile's
 * cells (Section 3: the TSC gather reads them), with two tensor copies
 * (cp.async.bulk.tensor) of the padded staged-field planes, one per plane,
 * completed on a shared-memory barrier; otherwise its threads copy the tile.
 * Mixed precision only, and only where the brick's x extent is even (the copy
 * alignment rule); mhdpic_field_tma tells whether the copies are used.  The
 * results are the same bit for bit.  A copy that does not complete within one
 * second raises MHDPIC_ST_COPY_TIMEOUT and ends that push.  A captured cycle
 * is discarded.  The paper has no counterpart.  Errors: MHDPIC_E_STATE.
 */
int mhdpic_set_field_tma(mhdpic_ctx *ctx, int32_t enable);

/* 1 when pushes of this context stage their field tiles by tensor copies, 0
 * when their threads do, -1 for an invalid context. */
int32_t mhdpic_field_tma(const mhdpic_ctx *ctx);

/*
 * mhdpic_debug_set_barrier_limit - testing interface: the wait limit of the
 * one-launch step's grid barriers, in nanoseconds (<= 0 restores the default
 * of one second).  A short limit makes the barrier give up with
 * MHDPIC_ST_BARRIER where blocks arrive at different times (no kernel is made
 * to stall; mhdpic_clear_status resets the barrier).  A captured cycle is
 * discarded.  The paper has no counterpart.  Errors: MHDPIC_E_STATE.
 */
int mhdpic_debug_set_barrier_limit(mhdpic_ctx *ctx, int64_t ns);

/*
 * mhdpic_debug_set_copy_limit - testing interface: the wait limit, in
 * nanoseconds, for the tensor copies of the push's field tiles and of the
 * sort's key pass to land in shared memory (<= 0 restores the default of one
 * second).  A block whose wait runs out raises MHDPIC_ST_COPY_TIMEOUT, waits
 * (up to one second) for its copies still in flight and ends; the results of
 * that launch are then not valid, and mhdpic_clear_status resets the flag.
 * With a 1 ns limit the waits that find a copy still in flight give up (no
 * copy is held back).  A captured cycle is discarded.  The paper has no
 * counterpart.  Errors: MHDPIC_E_STATE.
 */
int mhdpic_debug_set_copy_limit(mhdpic_ctx *ctx, int64_t ns);

/* Sort cadence chosen by mhdpic_run's tuner (0 before tuning, -1: bad ctx). */
int32_t mhdpic_sort_cadence(const mhdpic_ctx *ctx);

/*
 * mhdpic_get_deposits - convert fixed-point accumulators to double.
 *   which 0: corrector (dMx, dMy, dMz, dE) as accumulated since the last
 *            apply (momentum and energy, not densities; the sign is the gas's)
 *   which 1: current moments (n, Jx, Jy, Jz) as densities
 *   out   device double[4*nc], plane-major.
 */
int mhdpic_get_deposits(mhdpic_ctx *ctx, int32_t which, double *out);

/*
 * mhdpic_get_velocities - the current four-velocities as double, out device
 * double[3*np] plane-major (component d of particle i at out[d*np + i]), in
 * the order of the caller's particle arrays after the call (which brings them
 * up to date, as mhdpic_sync_particles).  MIXED: the exact value of each
 * two-word mhdpic_vel component; FP64: a copy of p64.
 */
int mhdpic_get_velocities(mhdpic_ctx *ctx, double *out);

/* Staged cell-centred fields as double: out device double[6*nc] = Ex,Ey,Ez,Bx,By,Bz. */
int mhdpic_get_fields(mhdpic_ctx *ctx, double *out);

/* Number of sort keys of all boxes (length of counts_out). */
int64_t mhdpic_num_keys(const mhdpic_ctx *ctx);

/* Device status flags (MHDPIC_ST_*), OR-ed over all calls since the last
 * clear.  Synchronises the stream. */
int mhdpic_get_status(mhdpic_ctx *ctx, uint32_t *flags);
int mhdpic_clear_status(mhdpic_ctx *ctx);

/*
 * mhdpic_debug_fail_launch - host-side fault injection for testing the
 * library's error paths (no GPU fault is made): the n-th kernel-launch check
 * of this context from now on reports MHDPIC_E_CUDA as though that launch had
 * failed, and the call making it returns the error; n = 0 disarms.  The
 * launch itself is issued, so after an eager call fails this way the
 * context's state is unspecified; a failure inside the graph capture of
 * mhdpic_run leaves the context as it was before the capture (nothing
 * captured runs).  The paper has no counterpart: it is a testing interface of
 * this library.  Errors: MHDPIC_E_STATE, MHDPIC_E_ARG for n < 0.
 */
int mhdpic_debug_fail_launch(mhdpic_ctx *ctx, int64_t n);

/* Count of this library's kernel launches since init (for benchmarks). */
int64_t mhdpic_launch_count(const mhdpic_ctx *ctx);

/* Free the context and its scratch (synchronises the stream). NULL is a no-op. */
int mhdpic_destroy(mhdpic_ctx *ctx);

/*
 * mhdpic_deposit_moments_noalloc - the charge and current deposit of
 * mhdpic_deposit (n_CR and J_CR of one box at the given positions, as
 * densities) for callers that cannot allocate device memory once running:
 * codes that reserve a fixed device-memory budget at start-up, time-step loops
 * that must stay allocation-free, or call sites where the implicit device
 * synchronisation of cudaMalloc/cudaFree is not acceptable.  It needs no
 * context and calls no cudaMalloc, cudaFree or allocating library routine.
 * The paper has no counterpart: it is an interface of this library.
 *   grid, params: one box (host structs; any boundary, particles that left
 *   through an open face, cell -1 / x NaN, deposit nothing); precision:
 *   MHDPIC_PREC_MIXED (pos, vel) or MHDPIC_PREC_FP64 (x, p64), device
 *   arrays laid out as in mhdpic_init; out: device double[4*ncell] = n, Jx,
 *   Jy, Jz, plane-major; stream: cudaStream_t.
 * Its int64 fixed-point accumulators, per-cell counts and scales are one
 * file-scope device array of about 9 MiB (for MHDPIC_NOALLOC_MAX_CELLS cells)
 * that every GPU loading the library holds until the process exits; grids with
 * more than MHDPIC_NOALLOC_MAX_CELLS cells (or a side longer than that) are
 * rejected with MHDPIC_E_CAPACITY.  Each call made while the stream is not
 * capturing looks up the array's device address on the current device
 * (cudaGetSymbolAddress; a device reset reloads the module, so the address is
 * never kept across one); a call made during a stream capture reuses the
 * address of the last call on that device, so make the first call on a device
 * before any stream capture (MHDPIC_E_STATE otherwise).  Every call clears and
 * then reuses the same array, which keeps the last call's sums: calls that
 * overlap on the GPU (other streams, or a second caller) race and corrupt each
 * other, so serialise them.  The fixed-point scales are sized on the device
 * from the densest cell of the call's particles.
 * Errors: MHDPIC_E_ARG, MHDPIC_E_CAPACITY, MHDPIC_E_STATE, MHDPIC_E_CUDA
 * (message in mhdpic_last_error()).
 */
#define MHDPIC_NOALLOC_MAX_CELLS 262144
int mhdpic_deposit_moments_noalloc(const mhdpic_grid *grid, const mhdpic_params *params, int32_t precision,
                                   int64_t np, const mhdpic_pos *pos, const mhdpic_vel *vel,
                                   const double *x, const double *p64, double *out, void *stream);

/* Static message for a return code, and the detailed message of the last
 * failure on this thread. */
const char *mhdpic_strerror(int code);
const char *mhdpic_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MHDPIC_H */
