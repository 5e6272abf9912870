// Internal declarations of the sm_103a MHD-PIC particle library.
//
// The device-side box table, the work items of the push, fixed-point helpers
// and the host-side launchers that the C-ABI layer (mhdpic_api.cu) calls.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mhdpic.h"

namespace mhdpic {

// ---------------------------------------------------------------------------
// channel numbering of the fixed-point deposit grids
// ---------------------------------------------------------------------------
// corrector (momentum and energy given to the gas, App. A.3): 0..3
// moments (charge and current densities, eq:nJCR):          4..7
enum { CH_MX = 0, CH_MY, CH_MZ, CH_E, CH_N, CH_JX, CH_JY, CH_JZ, NCH };

// Push tile: a brick of cells plus a halo of HALO cells on every side.  A
// particle whose 3^D stencil lies inside the tile deposits into shared memory;
// any other particle takes the global-memory path, so the halo only decides
// speed, never correctness.
constexpr int HALO = 2;
// Ghost cells around each box in the staged mixed-precision fields: as many as
// the tile's halo, so that every tile is one block of the padded array.
constexpr int FGHOST = HALO;
constexpr int PUSH_THREADS = 256;
constexpr int ITEM_MAX_PARTICLES = 4096;

// Fast unsigned division by a runtime constant (Granlund-Montgomery
// round-up method): q = umulhi(n, mul) >> shift for n < 2^31.
struct FastDiv {
    uint32_t d, mul, shift;
};

inline FastDiv make_fastdiv(uint32_t d)
{
    FastDiv f;
    f.d = d;
    uint32_t l = 0;
    while ((1ull << l) < d)
        ++l;
    // mul = ceil(2^(32+l) / d) - 2^32 fits in 32 bits for d >= 1
    uint64_t m = ((1ull << (32 + l)) + d - 1) / d;
    f.mul = (uint32_t)(m - (1ull << 32));
    f.shift = l;
    if (d == 1) {
        f.mul = 0;
        f.shift = 0;
    }
    return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv &f)
{
    uint32_t t = __umulhi(n, f.mul);
    return (t + n) >> f.shift;   // exact for n < 2^31 (31-bit numerators)
}

// One box as the kernels see it.
struct BoxDev {
    int32_t n[3];
    int32_t bc[3];
    int32_t hall;
    int32_t ndim;
    double dx[3], inv_dx[3], x0[3];
    double dV, inv_dV;
    double qm_cr, qm_gas, C, m_cr;
    int64_t cell0;   // first global cell of the box
    int64_t ncell;
    int64_t part0, part1;
    int64_t key0;    // first sort key of the box
    int64_t nkeys;
    int32_t nb[3];   // bricks per dimension
    int32_t pn[3];   // staged-field (mixed) array per box: the brick grid nb*brick + 2 FGHOST per dimension
                     // (x rounded up to even; 1 for z in 2-D), so that every push tile lies inside it
    int64_t fcell0;  // first cell of the box in the padded staged-field planes
    int32_t nbricks;
    int64_t brick0;  // first global brick number
    FastDiv div_nx, div_nxy;
    double scale[NCH];     // fixed-point scale (a power of two) per channel
    double inv_scale[NCH];
    double qmax[NCH];      // particle quantity above which the overflow flag is raised
    double qbound[NCH];    // particle quantity bound the scale was sized for
    int32_t escale[NCH];   // scale = 2^escale
};

// Per-box maxima tracked on the device; they size the corrector scales.
// Non-negative floats are stored as their bit patterns so that an unsigned
// atomicMax orders them correctly.
struct BoxStats {
    uint32_t vmax;        // max |v| of the particles (four-velocity)
    uint32_t emax;        // max |E| of the cell fields staged since the last scale choice
    uint32_t bmax;        // max |B| of the cell fields staged since the last scale choice
    int32_t maxcount;     // max particles per cell at the last sort
    int32_t corr_dirty;   // corrector accumulators hold data: scales locked
    uint32_t emax_used;   // the field maxima the last scale choice used (the
    uint32_t bmax_used;   // fields still staged when nothing was staged since)
    int32_t pad;
};

// A work item: the sorted positions p0, p0 + step, ... below p1, all in one
// brick.  A brick of at most ITEM_MAX_PARTICLES is one item of step 1; when
// it is a whole 64-cell brick, [p0, pm) and [pm, p1) are its two 32-cell
// halves (one lane per cell), otherwise pm = -1.  A crowded brick becomes m
// interleaved items per half (per brick without halves), item t taking the
// positions t, t + m, ... of that part (step m, pm = -1), so that every item
// spans all the part's cells, as the lanes need.
struct WorkItem {
    int32_t box;
    int32_t brick;   // brick number inside the box
    int64_t p0, pm, p1;
    int32_t step;
    int32_t count;   // positions in the item: ceil((p1 - p0) / step) <= ITEM_MAX_PARTICLES
};

// Everything a kernel needs, passed by value.
struct Ctx {
    int32_t nbox, ndim, prec;
    int32_t brick[3];
    int32_t brick_sh[3];   // log2 of brick[d] when it is a power of two, else -1
    int32_t tile[3];       // brick + 2*HALO
    int32_t tile_vol;      // cells of the tile
    int32_t ts[3];         // tile strides in slots (x, y, z); padded to spread banks
    int32_t tile_slots;    // slots of the tile (>= tile_vol)
    int32_t fts[3];        // field tile strides (x 1, y ts[1], z dense): the layout a tensor copy writes
    int32_t ftile_slots;   // slots of the field tile
    int32_t tma;           // 1: field tiles staged by tensor copies (tmaps), 0: by the threads
    int32_t halves;        // 1: default 64-cell bricks split into 32-cell halves
    double sort_ahead;     // sort key: the cell after moving for this time at the current velocity
    const float4 *sort_k;  // per box {t/dx, t/dy, t/dz, 1/C^2} in FP32 for that key
    int64_t copy_limit_ns; // wait limit for a tensor copy to land (then MHDPIC_ST_COPY_TIMEOUT)
    int64_t np, nc, nkeys, nbricks_total;
    const BoxDev *boxes;   // device
    const int64_t *box_part_start; // device [nbox+1]
    const int64_t *box_cell_start; // device [nbox+1]
    // current particle set, device: the caller's buffers (or their mirrors in
    // host-memory mode) or the library's second set.  Mixed precision keeps
    // two 16-byte records per particle: pos = {cell, off[3]} (as int4, the
    // offsets' bits in y, z, w) and vel = {v[3], packed residual} (float4)
    int4 *pos;
    float4 *vel;
    double *x;
    double *p64;
    // what a push reads: the current set itself (perm_src null), or right
    // after a sort the previous set through the permutation, sorted position
    // j taking particle perm_src[j]; the push then writes the current set
    const int32_t *perm_src;
    const int4 *src_pos;
    const float4 *src_vel;
    const double *src_x;
    const double *src_p64;
    double *rho, *mom, *egas, *B;
    // scratch
    unsigned long long *corr;     // [4][nc]
    unsigned long long *momdep[2];// [4][nc] each
    float4 *fa;                   // mixed: padded planes of the staged fields, {Ex, Ey, Ez, Bx}
    float2 *fb;                   //        and {By, Bz}, per box pn[0] x pn[1] x pn[2] cells from fcell0
    const unsigned char *tmaps;   // mixed with tma: per box two 128-byte tensor maps (planes fa, fb)
    double *f64;                  // [nc][6]
    uint32_t *status;
    const int32_t *key_off;       // sort offsets: particles of key k are [key_off[k], key_off[k+1])
    BoxDev *boxes_rw;             // same table, writable by the scale kernel
    BoxStats *stats;              // [nbox]
    // early-particle removal (null when not tracked): the injection time t_i
    // of every slot of the set the kernel writes, and the clock
    // {t, t_early}; a push removes a particle with t_i < t_early at the end
    // of the step that reaches t >= 2 t_i
    double *tinj;
    const double *clock;
};

// ---------------------------------------------------------------------------
// launchers (each returns the number of kernel launches it made, or -1 on a
// launch error; the caller checks cudaGetLastError)
// ---------------------------------------------------------------------------
struct SortScratch {
    int32_t *count;     // [nkeys + 1]
    int32_t *offset;    // [nkeys + 1]
    int32_t *pkey;      // [np]
    int32_t *pslot;     // [np]
    int32_t *perm;      // [np]
    int32_t *scan_tmp;  // block sums
    int32_t *big_list;  // segments longer than a warp can sort
    int32_t *big_count; // [1]
    void *tmp;          // particle staging, np * (largest particle record)
    int32_t *brick_items;  // [nbricks + 1] items per brick
    int32_t *item_off;     // [nbricks + 1] exclusive scan of brick_items
    int64_t *brick_start;  // device [nbox + 1] first global brick of each box
    WorkItem *items;
    int32_t *nitems;       // [1]
    int32_t *max_count;    // [1]
};

// One set of particle arrays (the precision's arrays; the others null).
struct PSet {
    int4 *pos;
    float4 *vel;
    double *x;
    double *p64;
    double *tinj;   // injection times, when tracked
};

int launch_sort(const Ctx &c, const SortScratch &s, int64_t *perm_out, int32_t *counts_out,
                cudaStream_t st);
// dst[j] = src[perm[j]] for every particle plane (and the injection times
// when both sets track them)
int launch_gather(const Ctx &c, const int32_t *perm, const PSet &src, const PSet &dst, cudaStream_t st);
// dst[j] = src[perm[j]] for one plane of np doubles
int launch_gather_f64(int64_t np, const int32_t *perm, const double *src, double *dst, cudaStream_t st);
// clock[0] += dt (the time a push reaches, before the push reads it)
int launch_clock_advance(double *clock, double dt, cudaStream_t st);
int launch_max_count(const Ctx &c, const SortScratch &s, cudaStream_t st);
// after a push that applied a sort: slots past the live particles marked free
int launch_mark_free(const Ctx &c, const SortScratch &s, cudaStream_t st);
// number of particles that have not left the box (into out, device)
int launch_count_live(const Ctx &c, unsigned long long *out, cudaStream_t st);
int launch_vmax(const Ctx &c, cudaStream_t st);
int launch_prep(const Ctx &c, int cur, int apply, cudaStream_t st);
int launch_moments(const Ctx &c, int cur, cudaStream_t st);
int launch_push_mixed(const Ctx &c, const SortScratch &s, int32_t *work_ctr, int cur_out, int full,
                      double dt, int grid_blocks, cudaStream_t st);
int launch_push_f64(const Ctx &c, const SortScratch &s, int32_t *work_ctr, int cur_out, int full,
                    double dt, int grid_blocks, cudaStream_t st);
// mixed precision: charge/current deposit at the stored positions through the
// push's tile, over the work list of the last sort (particles read through
// c.perm_src when set); momdep[cur] must be zero
int launch_deposit_mixed(const Ctx &c, const SortScratch &s, int32_t *work_ctr, int cur, int grid_blocks,
                         cudaStream_t st);
int launch_scales(const Ctx &c, double dt, cudaStream_t st);
// The grid-wide barrier of the fused step kernel (zeroed at init and by
// mhdpic_clear_status).
struct GridBarrier {
    unsigned int count;
    unsigned int gen;
};
// One whole mixed-precision step in one cooperative launch: scales, push
// (moments into momdep[cur ^ 1]), feedback and staging from them; -1 when
// the launch is refused
int launch_step_mixed(const Ctx &c, const SortScratch &s, int32_t *work_ctr, int cur, double dt, int grid_blocks,
                      GridBarrier *bar, long long limit_ns, cudaStream_t st);
int step_blocks_per_sm_mixed(const Ctx &c);
// chunked reductions: a box takes ceil((particles + cells) / per_chunk)
// slices, at least one and at most nchunks
int launch_totals(const Ctx &c, double *partials, int nchunks, int64_t per_chunk, double *out, cudaStream_t st);
int launch_fixed_to_double(const Ctx &c, const unsigned long long *src, int ch0, double *out,
                           cudaStream_t st);
int launch_fields_to_double(const Ctx &c, double *out, cudaStream_t st);
// the current four-velocities as double, plane-major [3][np]
int launch_velocities_to_double(const Ctx &c, double *out, cudaStream_t st);

// Spectrum request (mhdpic_spectrum); edges is a device copy [nbins + 1].
struct SpecArgs {
    int32_t kind, nbins, n_moment, has_region;
    double region[6];
    const double *edges;
};
int launch_spectrum(const Ctx &c, const SpecArgs &a, int nchunks, int64_t per_chunk, unsigned long long *counts,
                    double *partials, double *sums, cudaStream_t st);
int launch_lambda(const Ctx &c, int cur, double *out, cudaStream_t st);
// coupled step (App. A.3): gas half state into half[8][nc] plus field
// staging; gas full step from the half state and the corrector deposit
// shock front and CR injection (single box, open x face): the device state
// (inject_state_bytes, initialised from init_inject_state's host image), the
// scratch (inject_scratch_doubles(nx) doubles), the host view of the outputs
size_t inject_state_bytes();
void init_inject_state(void *st_host);
size_t inject_scratch_doubles(int64_t nx);
void inject_outputs(const void *st_host, double front[2], int64_t *n, int *capped);
int launch_inject(const Ctx &c, const SortScratch &s, void *state, double *scratch, int64_t nx, double dt,
                  double eta, double energy_factor, double gamma_gas, uint64_t seed, uint32_t call, int use_perm,
                  cudaStream_t st);
int launch_gas_predict(const Ctx &c, int cur, double dt, int model, double *half, cudaStream_t st);
int launch_gas_correct(const Ctx &c, double dt, int model, const double *half, cudaStream_t st);

// sets the message mhdpic_last_error() returns on this thread
void set_last_error(const char *msg);

// occupancy helpers
int push_blocks_per_sm_mixed(const Ctx &c);
int push_blocks_per_sm_f64(const Ctx &c);
size_t push_smem_bytes_mixed(const Ctx &c);
size_t push_smem_bytes_f64(const Ctx &c);
// the largest exponent of a fixed-point scale (kept inside float range)
constexpr int SCALE_EXP_MAX = 120;

}  // namespace mhdpic
