// Mixed-precision particle step: int32 cell + f32 offset positions, f32
// Boris push, fixed-point deposits (App. A.1-A.3 of arXiv:1412.1087).
//
// A persistent CTA of 8 warps takes brick items from an atomic counter.  Per
// item it stages the brick's E, B plus a halo of HALO cells in shared memory,
// accumulates both deposits in a shared fixed-point tile, and adds the tile to
// the int64 global accumulators at the end.
//
//  * Lanes and cells: a 64-cell brick is two 32-cell halves; warps 0-3 work
//    on one half and warps 4-7 on the other, and lane l takes the l-th 1/32 of
//    its half's (cell-sorted) particles, so the 32 lanes of an instruction sit
//    in about 32 different cells.  The tile strides are padded (3-D: y 12,
//    z 112 slots; 2-D: y 24) so that 32 cells of a half fall on 32 different
//    banks for the 32-bit deposit atomics and on distinct bank groups for the
//    128-bit and 64-bit field loads.  (Giving each lane exactly one cell's
//    particles removes more conflicts but idles a quarter of the lanes, since
//    cell counts vary; the even split measured 11% faster.)
//  * Fixed point in the tile: each contribution x = a w (in tile units, the
//    product exact inside the FMA) is the integer round(x) split into
//    hi = round(x / 2^KLO) and lo = round(x - hi 2^KLO), two FFMAs and one
//    FADD in all: t = fma(a, w, M_H) holds hi in its bit pattern (M_H =
//    1.5*2^(23+KLO) fixes the exponent), and fma(a, w, (M_H + M) - t) with
//    M = 1.5*2^23 holds lo (the addend is exact and the residual is rounded
//    once).  The planes add the two bit patterns as they are, each carrying
//    a constant offset (the bit pattern of M_H, of M); every deposit also
//    counts itself once at its stencil corner, and the flush removes the
//    offsets of the contributions a slot received (mod 2^32) before it
//    rebuilds hi 2^KLO + lo in int64 and shifts it to the global scale.  The
//    tile scale is sized for the largest item (ITEM_MAX_PARTICLES), so
//    neither plane can overflow and every item of a box rounds a
//    contribution alike.  The charge density (all contributions positive, no
//    cancellation) uses the hi plane alone, as round(x) from one FFMA
//    against M.
//  * A particle whose stencil leaves the tile adds the very integers the tile
//    would have held, shifted, straight to the int64 global accumulators, so
//    the sums are exact, independent of the order of the additions and of how
//    the particles fall into items (sort cadence included).  A particle whose
//    quantities exceed the bound the scales were sized for deposits at the
//    global scale instead (a choice that depends on the particle alone).
//  * Particles are two 16-byte records (pos = {cell, offsets}, vel = the
//    two-word four-velocity), one 128-bit load or store each, read through
//    the sort's permutation by the push that applies it.  The stored
//    four-velocity takes exactly the deposited dv (two-word sum), so the
//    exchange with the gas conserves momentum to 2^-35 of |v| per step.
//  * 2-D: each thread copies its next two particles' records into a
//    three-stage shared-memory ring with 16-byte cp.async while it pushes
//    the current one.
#include "async_copy.cuh"
#include "cells_common.cuh"
#include "push_common.cuh"

namespace mhdpic {

namespace {

constexpr float MAGIC = 12582912.0f;  // 1.5 * 2^23: x + MAGIC has unit spacing for |x| < 2^22
constexpr int MAGIC_BITS = 0x4B400000;
constexpr int KLO = 19;               // bits of the low word of a split contribution
constexpr float MAGIC_HI = 6597069766656.0f;  // 1.5 * 2^(23+KLO)
constexpr int MAGIC_HI_BITS = 0x54C00000;     // bit pattern of MAGIC_HI
constexpr float MAGIC_HI_LO = 6597082349568.0f;  // MAGIC_HI + MAGIC, exact (bits 2^42 .. 2^22)
// A slot of the deposit tile is TILE_WORDS consecutive int words: the hi
// words of the 8 channels (0..7), their lo words (8..15; the density has
// none, and its place holds the moments deposit's contribution count) and
// the corrector deposit's count (16).  An odd number of words keeps slots
// that differ mod 32 on different banks, and every word of a slot is a
// constant offset from the slot's address.
constexpr int TILE_WORDS = 2 * NCH + 1;
constexpr int W_LO = NCH;               // lo word of channel ch: W_LO + ch
constexpr int W_CNT_M = NCH + CH_N;     // contributions of the moments deposit, by stencil corner
constexpr int W_CNT_C = 2 * NCH;        // the same for the corrector deposit

struct MixedConst {
    float hdx[3];    // dt / (2 dx)
    float invC2;     // 1 / C^2
    float hh;        // (q/mc) dt / 2
    float m;
    float qn;        // (q/mc) m / dV
    float st[NCH];   // tile scale
    float gs[NCH];   // global scale
    float qb[NCH];   // per-particle bound of the tile path
    int ksh[NCH];    // flush shift: global = tile * 2^ksh
};

// TSC weights of one particle, passed by value to the global-memory path.
struct Wts {
    float x[3], y[3], z[3];
};

__device__ __forceinline__ void item_const(const BoxDev &b, float dt, int64_t cnt, int D, MixedConst &k)
{
#pragma unroll
    for (int d = 0; d < 3; ++d)
        k.hdx[d] = 0.5f * dt * (float)b.inv_dx[d];
    float C = (float)b.C;
    k.invC2 = 1.f / (C * C);
    k.hh = 0.5f * (float)b.qm_cr * dt;
    k.m = (float)b.m_cr;
    k.qn = (float)(b.qm_cr * b.m_cr * b.inv_dV);
    const float wmax = D == 3 ? 0.421875f : 0.5625f;   // largest TSC weight of one cell
    // sized for the largest item, so that every item of a box has the same
    // tile scale and a contribution rounds the same whichever item holds it
    (void)cnt;
    const float fc = (float)ITEM_MAX_PARTICLES + 1.f;
    // split channels: |hi| sums <= cnt (X/2^KLO + 1) < 2^31 and |lo| sums <= cnt 2^(KLO-1) < 2^31;
    // the hi word also needs |x| < 2^(22+KLO) for the rounding FFMA
    const float cap_split = fminf(1099511627776.f /* 2^40 */, 524288.f * (2147483648.f / fc - 1.f));
    // single-word channel: |x| < 2^21 and sums <= cnt x < 2^31
    const float cap_single = fminf(2097152.f, 2147483648.f / fc);
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
        float Q = fmaxf((float)b.qbound[ch], 1e-30f);
        int eg = b.escale[ch];
        int et = ilogbf((ch == CH_N ? cap_single : cap_split) / (Q * wmax));   // 2^et Q wmax <= cap
        et = max(et, -SCALE_EXP_MAX);
        if (et > eg)
            et = eg;
        k.ksh[ch] = eg - et;
        k.st[ch] = ldexpf(1.f, et);
        k.gs[ch] = ldexpf(1.f, eg);
        k.qb[ch] = Q;
    }
}

template <int D>
__device__ __forceinline__ void gather_tile(const Ctx &c, int base, const Wts &w, const float4 *__restrict__ sFa,
                                            const float2 *__restrict__ sFb, float E[3], float Bf[3])
{
    E[0] = E[1] = E[2] = Bf[0] = Bf[1] = Bf[2] = 0.f;
    const int SY = c.fts[1], SZ = c.fts[2];   // the field tile's strides
    // the z layers are kept rolled in 3-D: a third of the code, fewer
    // instruction-cache misses (measured 2% faster); 2-D has one layer
#pragma unroll 1
    for (int cz = 0; cz < (D == 3 ? 3 : 1); ++cz)
#pragma unroll
        for (int cy = 0; cy < 3; ++cy) {
            float wyz = D == 3 ? w.y[cy] * w.z[cz] : w.y[cy];
#pragma unroll
            for (int cx = 0; cx < 3; ++cx) {
                float ww = w.x[cx] * wyz;
                int s = base + cx + SY * cy + SZ * cz;
                float4 a = sFa[s];
                float2 bb = sFb[s];
                E[0] = fmaf(ww, a.x, E[0]);
                E[1] = fmaf(ww, a.y, E[1]);
                E[2] = fmaf(ww, a.z, E[2]);
                Bf[0] = fmaf(ww, a.w, Bf[0]);
                Bf[1] = fmaf(ww, bb.x, Bf[1]);
                Bf[2] = fmaf(ww, bb.y, Bf[2]);
            }
        }
}

// An opaque register copy: the value is materialised here, once, and every
// later use reads these bits.  The deposit's inputs (TSC weights, scaled
// quantities) go through it, so that the inlined tile path and the global
// path cannot each recompute them with a different contraction of the same
// expression: the integers a particle deposits must not depend on the path.
__device__ __forceinline__ float pinned(float x)
{
    asm volatile("" : "+f"(x));
    return x;
}

__device__ __forceinline__ void pin_weights(Wts &w)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        w.x[a] = pinned(w.x[a]);
        w.y[a] = pinned(w.y[a]);
        w.z[a] = pinned(w.z[a]);
    }
}

struct F6 {
    float e[3], b[3];
};

template <int D>
__device__ __noinline__ F6 gather_global(const Ctx &c, const BoxDev &b, int ci0, int ci1, int ci2, Wts w)
{
    F6 r;
    r.e[0] = r.e[1] = r.e[2] = r.b[0] = r.b[1] = r.b[2] = 0.f;
    // the stencil's cells, ghosts included, are inside the padded planes
    for (int cz = 0; cz < (D == 3 ? 3 : 1); ++cz)
        for (int cy = 0; cy < 3; ++cy) {
            float wyz = D == 3 ? w.y[cy] * w.z[cz] : w.y[cy];
            for (int cx = 0; cx < 3; ++cx) {
                float ww = w.x[cx] * wyz;
                const int64_t f = fidx(b, ci0 + cx - 1, ci1 + cy - 1, D == 3 ? ci2 + cz - 1 : 0);
                const float4 f1 = __ldg(c.fa + f);
                const float2 f2 = __ldg(c.fb + f);
                r.e[0] = fmaf(ww, f1.x, r.e[0]);
                r.e[1] = fmaf(ww, f1.y, r.e[1]);
                r.e[2] = fmaf(ww, f1.z, r.e[2]);
                r.b[0] = fmaf(ww, f1.w, r.b[0]);
                r.b[1] = fmaf(ww, f2.x, r.b[1]);
                r.b[2] = fmaf(ww, f2.y, r.b[2]);
            }
        }
    return r;
}

// round(a * wx) as the words hi + MAGIC_HI_BITS and lo + MAGIC_BITS, with
// hi = round(a wx / 2^KLO) and lo = round(a wx - hi 2^KLO), |lo| <= 2^(KLO-1):
// the one place the tile path and the global path compute them
__device__ __forceinline__ void split_words(float a, float wx, int &hb, int &lb)
{
    const float t = fmaf(a, wx, MAGIC_HI);
    hb = __float_as_int(t);
    lb = __float_as_int(fmaf(a, wx, MAGIC_HI_LO - t));
}

// round(a * wx) as one word, plus MAGIC_BITS (|a wx| < 2^22)
__device__ __forceinline__ int single_word(float a, float wx)
{
    return __float_as_int(fmaf(a, wx, MAGIC));
}

// both words of a split contribution added to a tile slot as they are
__device__ __forceinline__ void add_split(int *hi, int *lo, float a, float wx)
{
    int hb, lb;
    split_words(a, wx, hb, lb);
    atomicAdd(hi, hb);
    atomicAdd(lo, lb);
}

// Contributions tile cell (tx, ty, tz) received from one deposit: the counts
// (word W_CNT_C or W_CNT_M) of the stencil corners at most 2 cells below it.
__device__ __forceinline__ uint32_t slot_count(const Ctx &c, const int *sD, int word, int tx, int ty, int tz, int D)
{
    const int *cnt = sD + word;
    uint32_t k = 0u;
    for (int dz = 0; dz < (D == 3 ? 3 : 1); ++dz) {
        if (tz - dz < 0)
            break;
        for (int dy = 0; dy < 3; ++dy) {
            if (ty - dy < 0)
                break;
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                if (tx - dx < 0)
                    break;
                k += (uint32_t)cnt[((tx - dx) + c.ts[1] * (ty - dy) + c.ts[2] * (tz - dz)) * TILE_WORDS];
            }
        }
    }
    return k;
}

// channel ch of tile slot s rebuilt as the sum of its rounded contributions
__device__ __forceinline__ long long slot_value(const int *sD, int s, int ch, uint32_t kc, uint32_t km)
{
    const int *w = sD + s * TILE_WORDS;
    const uint32_t k = ch < CH_N ? kc : km;
    const int hi = (int)((uint32_t)w[ch] - k * (uint32_t)(ch == CH_N ? MAGIC_BITS : MAGIC_HI_BITS));
    if (ch == CH_N)
        return hi;
    const int lo = (int)((uint32_t)w[W_LO + ch] - k * (uint32_t)MAGIC_BITS);
    return (long long)hi * (1ll << KLO) + lo;
}

// Four channels into the tile; q carries the tile scale.  Every channel is
// split into hi and lo words except the charge density, whose contributions
// are all positive and never cancel.  The words carry their offsets; the
// deposit counts itself at its stencil corner (base) for the flush.
template <int D>
__device__ __forceinline__ void deposit_tile(const Ctx &c, int base, const Wts &w, const float q[4], int ch0,
                                             int *__restrict__ sD)
{
    const int SY = c.ts[1], SZ = c.ts[2];
    const bool first_single = ch0 == CH_N;
#pragma unroll 1
    for (int cz = 0; cz < (D == 3 ? 3 : 1); ++cz)
#pragma unroll
        for (int cy = 0; cy < 3; ++cy) {
            float wyz = D == 3 ? w.y[cy] * w.z[cz] : w.y[cy];
            float a0 = q[0] * wyz, a1 = q[1] * wyz, a2 = q[2] * wyz, a3 = q[3] * wyz;
#pragma unroll
            for (int cx = 0; cx < 3; ++cx) {
                int *__restrict__ t = sD + (base + cx + SY * cy + SZ * cz) * TILE_WORDS + ch0;
                if (first_single)
                    atomicAdd(t, single_word(a0, w.x[cx]));
                else
                    add_split(t, t + W_LO, a0, w.x[cx]);
                add_split(t + 1, t + 1 + W_LO, a1, w.x[cx]);
                add_split(t + 2, t + 2 + W_LO, a2, w.x[cx]);
                add_split(t + 3, t + 3 + W_LO, a3, w.x[cx]);
            }
        }
    atomicAdd(sD + base * TILE_WORDS + (first_single ? W_CNT_M : W_CNT_C), 1);
}

// Four channels into the int64 global accumulators as exactly the integers
// the tile path would add (q carries the tile scale; each word is shifted to
// the global scale as the flush shifts the tile): used where the stencil
// leaves the tile, so that the sums do not depend on the tile a particle sits
// in.
template <int D>
__device__ __noinline__ void deposit_global_split(const Ctx &c, const BoxDev &b, int ci0, int ci1, int ci2, Wts w,
                                                  float q0, float q1, float q2, float q3, int ch0, int k0, int k1,
                                                  int k2, int k3, unsigned long long *__restrict__ g0)
{
    const int64_t nc = c.nc;
    const int ci[3] = {ci0, ci1, ci2};
    const float q[4] = {q0, q1, q2, q3};
    const int ksh[4] = {k0, k1, k2, k3};
    int gx[3], gy[3], gz[3];
    stencil_coords<D>(b, ci, gx, gy, gz);
    for (int cz = 0; cz < (D == 3 ? 3 : 1); ++cz)
        for (int cy = 0; cy < 3; ++cy) {
            float wyz = D == 3 ? w.y[cy] * w.z[cz] : w.y[cy];
            for (int cx = 0; cx < 3; ++cx) {
                int64_t g = b.cell0 + ((int64_t)gz[cz] * b.n[1] + gy[cy]) * b.n[0] + gx[cx];
                for (int k = 0; k < 4; ++k) {
                    const float a = q[k] * wyz;
                    long long v;
                    if (ch0 + k == CH_N) {
                        v = single_word(a, w.x[cx]) - MAGIC_BITS;
                    } else {
                        int hb, lb;
                        split_words(a, w.x[cx], hb, lb);
                        v = (long long)(hb - MAGIC_HI_BITS) * (1ll << KLO) + (lb - MAGIC_BITS);
                    }
                    if (v)
                        red_add(g0 + k * nc + g, (long long)((unsigned long long)v << ksh[k]));
                }
            }
        }
}

// Four channels straight into the int64 global accumulators; q carries the
// global scale.  Used for particles above the bound the tile scale was sized
// for (the choice depends only on the particle).
template <int D>
__device__ __noinline__ void deposit_global(const Ctx &c, const BoxDev &b, int ci0, int ci1, int ci2, Wts w,
                                            float q0, float q1, float q2, float q3,
                                            unsigned long long *__restrict__ g0)
{
    const int64_t nc = c.nc;
    const int ci[3] = {ci0, ci1, ci2};
    int gx[3], gy[3], gz[3];
    stencil_coords<D>(b, ci, gx, gy, gz);
    for (int cz = 0; cz < (D == 3 ? 3 : 1); ++cz)
        for (int cy = 0; cy < 3; ++cy) {
            float wyz = D == 3 ? w.y[cy] * w.z[cz] : w.y[cy];
            for (int cx = 0; cx < 3; ++cx) {
                float ww = w.x[cx] * wyz;
                int64_t g = b.cell0 + ((int64_t)gz[cz] * b.n[1] + gy[cy]) * b.n[0] + gx[cx];
                red_add(g0 + g, __float2ll_rn(q0 * ww));
                red_add(g0 + nc + g, __float2ll_rn(q1 * ww));
                red_add(g0 + 2 * nc + g, __float2ll_rn(q2 * ww));
                red_add(g0 + 3 * nc + g, __float2ll_rn(q3 * ww));
            }
        }
}

__device__ __forceinline__ bool within(const float q[4], const float *qb, int ch0)
{
    return fabsf(q[0]) <= qb[ch0] && fabsf(q[1]) <= qb[ch0 + 1] && fabsf(q[2]) <= qb[ch0 + 2] &&
           fabsf(q[3]) <= qb[ch0 + 3];
}

// Particle records staged per thread: pos and vel, 16 bytes each.
constexpr int RING_RECS = 2;
constexpr int RING_STAGES = 3;
// Per dimension: 2-D pushes are short, so the kernel hides the particle
// loads behind a three-stage shared-memory ring (two particles ahead) and
// runs 3 CTAs per SM (80 registers, no
// spills in the loop; 4 CTAs at 64 registers spilled and measured slower with
// a sort every step) with the item constants in shared memory; 3-D pushes
// keep everything in registers at 2 CTAs per SM (the ring measured no faster
// there and takes shared memory from L1).
template <int D>
constexpr bool STAGED = D == 2;
template <int D>
constexpr int MIN_BLOCKS = D == 3 ? 2 : 3;
template <int D>
constexpr bool CONST_IN_SMEM = D == 2;

__device__ __forceinline__ void cp_async16(int4 *dst, const void *src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_prev()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(RING_STAGES - 1) : "memory");
}

// Start the copy of source particle i's two records into one stage of this
// thread's ring (records PUSH_THREADS int4 apart).
__device__ __forceinline__ void stage_particle(const Ctx &c, int64_t i, int4 *dst)
{
    cp_async16(dst, c.src_pos + i);
    cp_async16(dst + PUSH_THREADS, c.src_vel + i);
}

struct PIn {
    int32_t cell;
    float o[3], v[3];
    uint32_t res;   // packed residuals of the two-word four-velocity
};

__device__ __forceinline__ PIn unpack(const int4 a, const float4 b)
{
    PIn r;
    r.cell = a.x;
    r.o[0] = __int_as_float(a.y);
    r.o[1] = __int_as_float(a.z);
    r.o[2] = __int_as_float(a.w);
    r.v[0] = b.x;
    r.v[1] = b.y;
    r.v[2] = b.z;
    r.res = __float_as_uint(b.w);
    return r;
}

__device__ __forceinline__ PIn load_staged(const int4 *in)
{
    const int4 a = in[0], bi = in[PUSH_THREADS];
    return unpack(a, make_float4(__int_as_float(bi.x), __int_as_float(bi.y), __int_as_float(bi.z),
                                 __int_as_float(bi.w)));
}

__device__ __forceinline__ PIn load_global(const Ctx &c, int64_t i)
{
    return unpack(__ldg(c.src_pos + i), __ldg(c.src_vel + i));
}

__device__ __forceinline__ void store_particle(const Ctx &c, int64_t j, int32_t cell, const float o[3],
                                               const float v[3], uint32_t res)
{
    c.pos[j] = make_int4(cell, __float_as_int(o[0]), __float_as_int(o[1]), __float_as_int(o[2]));
    c.vel[j] = make_float4(v[0], v[1], v[2], __uint_as_float(res));
}

// The push's dynamic shared memory: the deposit tile (`slots` slots of
// TILE_WORDS int words), the field tile (a float4 and a float2 plane of `fslots`, each on a
// 128-byte boundary for the tensor copies), then the particle ring (2-D).
struct PushLayout {
    size_t fa, fb, ring;
};

__host__ __device__ constexpr size_t align128(size_t x) { return (x + 127) / 128 * 128; }

__host__ __device__ inline PushLayout push_layout(int slots, int fslots)
{
    PushLayout l{};
    l.fa = align128(sizeof(int) * TILE_WORDS * (size_t)slots);
    l.fb = align128(l.fa + sizeof(float4) * (size_t)fslots);
    l.ring = align128(l.fb + sizeof(float2) * (size_t)fslots);
    return l;
}

__device__ __forceinline__ void store_dead(const Ctx &c, int64_t j)
{
    c.pos[j] = make_int4(DEAD_CELL, 0, 0, 0);
    c.vel[j] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Charge and current density deposit of one particle (eq:nJCR) at cell ci,
// offsets o, four-velocity v with ig = 1/gamma from rsqrtf(fmaf(vsq3(v),
// invC2, 1)): n = qn W, J = qn (v/gamma) W.  The push calls it at x^(n+1) and
// the standalone deposit at the stored positions, so the two give the same
// integers for the same particle state.
template <int D>
__device__ __forceinline__ void deposit_moments_one(const Ctx &c, const BoxDev &b, const ItemGeom &gm,
                                                    const MixedConst &k, const int ci[3], const float o[3],
                                                    const float v[3], float ig, int *sD, unsigned long long *mout)
{
    Wts w2;
    w2.z[0] = 0.f;
    w2.z[1] = 1.f;
    w2.z[2] = 0.f;
    int rel2[3] = {0, 0, 0};
    bool in2 = tile_rel(c, b, gm, 0, ci[0], rel2[0]);
    in2 &= tile_rel(c, b, gm, 1, ci[1], rel2[1]);
    tsc_from_offset<float>(o[0], w2.x);
    tsc_from_offset<float>(o[1], w2.y);
    if (D == 3) {
        in2 &= tile_rel(c, b, gm, 2, ci[2], rel2[2]);
        tsc_from_offset<float>(o[2], w2.z);
    }
    pin_weights(w2);
    const float qj = k.qn * ig;
    const float qm[4] = {pinned(k.qn), pinned(qj * v[0]), pinned(qj * v[1]), pinned(qj * v[2])};
    if (within(qm, k.qb, CH_N)) {
        const float qs[4] = {pinned(qm[0] * k.st[4]), pinned(qm[1] * k.st[5]), pinned(qm[2] * k.st[6]),
                             pinned(qm[3] * k.st[7])};
        if (in2) {
            const int base2 = (rel2[0] - 1) + c.ts[1] * (rel2[1] - 1) + (D == 3 ? c.ts[2] * (rel2[2] - 1) : 0);
            deposit_tile<D>(c, base2, w2, qs, CH_N, sD);
        } else {
            deposit_global_split<D>(c, b, ci[0], ci[1], ci[2], w2, qs[0], qs[1], qs[2], qs[3], CH_N, k.ksh[4],
                                    k.ksh[5], k.ksh[6], k.ksh[7], mout);
        }
    } else {
        deposit_global<D>(c, b, ci[0], ci[1], ci[2], w2, qm[0] * k.gs[4], qm[1] * k.gs[5], qm[2] * k.gs[6],
                          qm[3] * k.gs[7], mout);
    }
}

template <int D, bool FULL>
__device__ __forceinline__ float push_one(const Ctx &c, const BoxDev &b, const ItemGeom &gm, const MixedConst &k,
                                          int64_t j, const PIn &pin, const float4 *sFa, const float2 *sFb,
                                          int *sD, unsigned long long *mout)
{
    if (pin.cell == DEAD_CELL) {   // left the box earlier (kept until the next sort)
        store_dead(c, j);
        return 0.f;
    }
    int ci[3];
    decode_cell(b, pin.cell, ci);
    float o[3] = {pin.o[0], pin.o[1], pin.o[2]}, v[3] = {pin.v[0], pin.v[1], pin.v[2]};

    // drift to x^(n+1/2) with u = v / gamma (a particle at an open face is
    // held just inside it, deposits its corrector and then leaves)
    const float sn = fmaf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2], k.invC2, 1.f);   // gamma^2
    const float ign = rsqrtf(sn);
    bool leaving = false;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        o[d] = fmaf(k.hdx[d] * ign, v[d], o[d]);
        leaving |= renorm_mixed(b, d, ci[d], o[d], v[d], c.status);
    }

    Wts w;
    w.z[0] = 0.f;
    w.z[1] = 1.f;
    w.z[2] = 0.f;
    int rel[3] = {0, 0, 0};
    bool in_tile = tile_rel(c, b, gm, 0, ci[0], rel[0]);
    in_tile &= tile_rel(c, b, gm, 1, ci[1], rel[1]);
    tsc_from_offset<float>(o[0], w.x);
    tsc_from_offset<float>(o[1], w.y);
    if (D == 3) {
        in_tile &= tile_rel(c, b, gm, 2, ci[2], rel[2]);
        tsc_from_offset<float>(o[2], w.z);
    }
    pin_weights(w);
    const int base = (rel[0] - 1) + c.ts[1] * (rel[1] - 1) + (D == 3 ? c.ts[2] * (rel[2] - 1) : 0);
    const int fbase = (rel[0] - 1) + c.fts[1] * (rel[1] - 1) + (D == 3 ? c.fts[2] * (rel[2] - 1) : 0);

    float E[3], Bf[3];
    if (in_tile) {
        gather_tile<D>(c, fbase, w, sFa, sFb, E, Bf);
    } else {
        F6 f = gather_global<D>(c, b, ci[0], ci[1], ci[2], w);
        E[0] = f.e[0];
        E[1] = f.e[1];
        E[2] = f.e[2];
        Bf[0] = f.b[0];
        Bf[1] = f.b[1];
        Bf[2] = f.b[2];
    }

    // remove the component of E along B
    float B2 = Bf[0] * Bf[0] + Bf[1] * Bf[1] + Bf[2] * Bf[2];
    if (B2 > 0.f) {
        float eb = (E[0] * Bf[0] + E[1] * Bf[1] + E[2] * Bf[2]) / B2;
        E[0] = fmaf(-eb, Bf[0], E[0]);
        E[1] = fmaf(-eb, Bf[1], E[1]);
        E[2] = fmaf(-eb, Bf[2], E[2]);
    }

    // Boris: v0 = v + (h/2)E; b = (h/2)B/gamma(v0); v1 = v0 + 2(v0 + v0 x b) x b/(1+b^2)
    const float e0 = k.hh * E[0], e1 = k.hh * E[1], e2 = k.hh * E[2];
    const float v00 = v[0] + e0, v01 = v[1] + e1, v02 = v[2] + e2;
    const float s1 = fmaf(v00 * v00 + v01 * v01 + v02 * v02, k.invC2, 1.f);
    const float ig1 = rsqrtf(s1);
    const float hb = k.hh * ig1;
    const float b0 = hb * Bf[0], b1 = hb * Bf[1], b2 = hb * Bf[2];
    const float t0 = v00 + (v01 * b2 - v02 * b1), t1 = v01 + (v02 * b0 - v00 * b2),
                t2 = v02 + (v00 * b1 - v01 * b0);
    // the divisions below have denominators of 1 or more: the fast division
    // (2 ulp) in place of the IEEE sequence
    const float s2 = __fdividef(2.f, 1.f + b0 * b0 + b1 * b1 + b2 * b2);
    const float r0 = s2 * (t1 * b2 - t2 * b1), r1 = s2 * (t2 * b0 - t0 * b2), r2 = s2 * (t0 * b1 - t1 * b0);
    const float v10 = v00 + r0, v11 = v01 + r1, v12 = v02 + r2;
    const float vk[3] = {v10 + e0, v11 + e1, v12 + e2};   // after the second kick, FP32

    // dv = h E + rot without cancellation; the rotation keeps |v|, so dE_k is
    // the change of the two half kicks, E_k(a) - E_k(b) = (a-b).(a+b)/(ga+gb)
    const float s2k = fmaf(vsq3(vk), k.invC2, 1.f);
    const float ig2k = rsqrtf(s2k);
    const float gn = sn * ign, g1 = s1 * ig1, g2 = s2k * ig2k;   // gamma = gamma^2 / gamma
    const float dEk = __fdividef(e0 * (vk[0] + v10) + e1 * (vk[1] + v11) + e2 * (vk[2] + v12), g2 + g1) +
                      __fdividef(e0 * (v00 + v[0]) + e1 * (v01 + v[1]) + e2 * (v02 + v[2]), g1 + gn);
    const float dv[3] = {pinned(2.f * e0 + r0), pinned(2.f * e1 + r1), pinned(2.f * e2 + r2)};
    {
        const float qc[4] = {pinned(-k.m * dv[0]), pinned(-k.m * dv[1]), pinned(-k.m * dv[2]), pinned(-k.m * dEk)};
        if (within(qc, k.qb, CH_MX)) {
            const float qs[4] = {pinned(qc[0] * k.st[0]), pinned(qc[1] * k.st[1]), pinned(qc[2] * k.st[2]),
                                 pinned(qc[3] * k.st[3])};
            if (in_tile)
                deposit_tile<D>(c, base, w, qs, CH_MX, sD);
            else
                deposit_global_split<D>(c, b, ci[0], ci[1], ci[2], w, qs[0], qs[1], qs[2], qs[3], CH_MX, k.ksh[0],
                                        k.ksh[1], k.ksh[2], k.ksh[3], c.corr);
        } else {
            deposit_global<D>(c, b, ci[0], ci[1], ci[2], w, qc[0] * k.gs[0], qc[1] * k.gs[1], qc[2] * k.gs[2],
                              qc[3] * k.gs[3], c.corr);
        }
    }

    // the stored four-velocity takes exactly the deposited dv (two-word sum,
    // rounded once at 2^-35 of |v|): what the gas is given is what the
    // particle loses
    float vn[3] = {v[0], v[1], v[2]};   // the leading words (mirrored by a reflection at the half step)
    int rq[3] = {res_field(pin.res, 0), res_field(pin.res, 1), res_field(pin.res, 2)};
#pragma unroll
    for (int d = 0; d < D; ++d)
        if (v[d] != pin.v[d])
            rq[d] = -rq[d];
#pragma unroll
    for (int d = 0; d < 3; ++d)
        two_word_add(vn[d], rq[d], dv[d]);
    const float ig2 = rsqrtf(fmaf(vsq3(vn), k.invC2, 1.f));

    // drift to x^(n+1); a reflection mirrors both words of the component
#pragma unroll
    for (int d = 0; d < D; ++d) {
        o[d] = fmaf(k.hdx[d] * ig2, vn[d], o[d]);
        const float before = vn[d];
        leaving |= renorm_mixed(b, d, ci[d], o[d], vn[d], c.status);
        if (vn[d] != before)
            rq[d] = -rq[d];
    }
    leaving |= removed_early(c, j);
    if (leaving) {   // removed: no moments deposit; the next sort drops it
        store_dead(c, j);
        return 0.f;
    }

    if (FULL)
        deposit_moments_one<D>(c, b, gm, k, ci, o, vn, ig2, sD, mout);

    if (!isfinite(vn[0] + vn[1] + vn[2]))
        set_status(c.status, MHDPIC_ST_NONFINITE);
    store_particle(c, j, (int32_t)(((int64_t)ci[2] * b.n[1] + ci[1]) * b.n[0] + ci[0]), o, vn, res_pack(rq));
    return vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2];
}

// ---------------------------------------------------------------------------
// Tensor copies of the field tile (TMA): one cp.async.bulk.tensor per plane
// per work item, completed on a shared-memory mbarrier.  Each wait has a time
// limit; a copy that does not complete raises MHDPIC_ST_COPY_TIMEOUT.
// ---------------------------------------------------------------------------

// The copies read a box of the padded planes starting at the tile's first
// cell; the innermost coordinate counts floats (4 per cell in plane fa, 2 in
// fb), so it is a multiple of 16 bytes when the tile starts on an even cell.
template <int D>
__device__ __forceinline__ void tma_tile(void *dst, const unsigned char *tmap, int x, int y, int z, uint64_t *bar)
{
    if (D == 3)
        asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                     " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
                     "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
                     : "memory");
    else
        asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                     " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
                     "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
                     : "memory");
}

// The push over the work items of the last sort, taken from an atomic
// counter by the calling kernel's persistent blocks (smem: the dynamic shared
// memory, push_smem_bytes_mixed bytes).
template <int D, bool FULL>
__device__ __forceinline__ void push_items(const Ctx &c, const WorkItem *__restrict__ items, const int nit,
                                           int32_t *__restrict__ work_ctr, int cur_out, float dt,
                                           unsigned char *smem)
{
    const int S = c.tile_slots;
    const PushLayout lay = push_layout(S, c.ftile_slots);
    int *sD = reinterpret_cast<int *>(smem);
    float4 *sFa = reinterpret_cast<float4 *>(smem + lay.fa);
    float2 *sFb = reinterpret_cast<float2 *>(smem + lay.fb);
    int4 *ring = reinterpret_cast<int4 *>(smem + lay.ring) + threadIdx.x;
    constexpr int RS = RING_RECS * PUSH_THREADS;   // int4 per ring stage
    __shared__ __align__(8) uint64_t s_bar;   // completion of the field tile's tensor copies
    unsigned phase = 0;
    const unsigned copy_bytes = (unsigned)((sizeof(float4) + sizeof(float2)) * (size_t)c.ftile_slots);
    if (c.tma) {
        if (threadIdx.x == 0)
            mbar_init(&s_bar);
        __syncthreads();
    }
    __shared__ int s_item;
    __shared__ MixedConst s_k;
    unsigned long long *mout = c.momdep[cur_out];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int NW = PUSH_THREADS / 32;

    for (;;) {
        if (threadIdx.x == 0)
            s_item = atomicAdd(work_ctr, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= nit)
            break;
        const WorkItem it = items[item];
        const BoxDev &b = c.boxes[it.box];
        const ItemGeom gm = item_geom(c, b, it.brick, D);

        // stage the fields: the tile is one block of the padded planes
        // (ghosts included), copied by the tensor engine or by the threads
        if (c.tma) {
            if (threadIdx.x == 0) {
                // the previous item's reads of the tile ended at the barrier before
                fence_proxy_async();
                mbar_expect_tx(&s_bar, copy_bytes);
                const unsigned char *tm = c.tmaps + (size_t)it.box * 256;
                const int x0 = gm.org[0] + FGHOST, y0 = gm.org[1] + FGHOST, z0 = gm.org[2] + FGHOST;
                tma_tile<D>(sFa, tm, 4 * x0, y0, z0, &s_bar);
                tma_tile<D>(sFb, tm + 128, 2 * x0, y0, z0, &s_bar);
            }
        } else {
            for (int t = threadIdx.x; t < c.tile_vol; t += PUSH_THREADS) {
                const int tx = t % c.tile[0], r = t / c.tile[0];
                const int ty = r % c.tile[1], tz = r / c.tile[1];
                // the tile lies inside the padded planes (they cover the brick grid plus the halo)
                const int64_t f = fidx(b, gm.org[0] + tx, gm.org[1] + ty, gm.org[2] + tz);
                const int sl = tx + c.fts[1] * ty + c.fts[2] * tz;
                sFa[sl] = __ldg(c.fa + f);
                sFb[sl] = __ldg(c.fb + f);
            }
        }
        // clear the deposit tile and its counts
        for (int s = threadIdx.x; s < TILE_WORDS * S; s += PUSH_THREADS)
            sD[s] = 0;
        if (threadIdx.x == 0)
            item_const(b, dt, it.p1 - it.p0, D, s_k);
        __syncthreads();
        if (c.tma) {
            const bool ok = mbar_wait(&s_bar, phase, c.copy_limit_ns);
            if (__syncthreads_or(!ok)) {   // give up the launch, after the copies in flight have had their time
                if (threadIdx.x == 0)
                    set_status(c.status, MHDPIC_ST_COPY_TIMEOUT);
                mbar_wait(&s_bar, phase, COPY_LIMIT_NS);
                return;
            }
            phase ^= 1u;
        }
        // the item constants stay in shared memory where registers are short
        MixedConst kreg;
        if (!CONST_IN_SMEM<D>)
            kreg = s_k;
        const MixedConst &k = CONST_IN_SMEM<D> ? s_k : kreg;

        float vm2 = 0.f;
        {
            const LaneRange lr = lane_range(it, wid, NW);
            const int64_t base = lr.base, cnt = lr.cnt, lane0 = lane * lr.q, rb = lr.first, re = lr.q,
                          rs = lr.stride;
            const int32_t step = lr.step;
            // source particle of sorted position base + (lane0 + r) step; when the
            // push applies a sort the permutation entry is loaded one
            // iteration early.  (One code path for both cases, so that the
            // arithmetic is the same instruction for instruction.)
            const bool gather = c.perm_src != nullptr;
            auto valid = [&](int64_t r) { return r < re && lane0 + r < cnt; };
            auto src_of = [&](int64_t r) -> int64_t {
                const int64_t j = base + (int32_t)(lane0 + r) * step;
                return gather ? (int64_t)__ldg(c.perm_src + j) : j;
            };
            if (STAGED<D>) {
                // the next RING_STAGES - 1 particles' words are copied into
                // shared memory while the current one is pushed
                constexpr int NS = RING_STAGES;
#pragma unroll
                for (int s0 = 0; s0 < NS - 1; ++s0) {
                    if (valid(rb + s0 * rs))
                        stage_particle(c, src_of(rb + s0 * rs), ring + s0 * RS);
                    cp_async_commit();
                }
                int64_t sn = valid(rb + (NS - 1) * rs) ? src_of(rb + (NS - 1) * rs) : 0;
                int st = 0;
                for (int64_t r = rb; r < re; r += rs) {
                    const int stn = st == 0 ? NS - 1 : st - 1;
                    if (valid(r + (NS - 1) * rs))
                        stage_particle(c, sn, ring + stn * RS);
                    if (valid(r + NS * rs))
                        sn = src_of(r + NS * rs);
                    cp_async_commit();
                    cp_async_wait_prev();
                    if (lane0 + r < cnt)
                        vm2 = fmaxf(vm2, push_one<D, FULL>(c, b, gm, k, base + (int32_t)(lane0 + r) * step, load_staged(ring + st * RS),
                                                           sFa, sFb, sD, mout));
                    st = st + 1 == NS ? 0 : st + 1;
                }
            } else {
                int64_t sn = valid(rb) ? src_of(rb) : 0;
                for (int64_t r = rb; r < re; r += rs)
                    if (lane0 + r < cnt) {
                        const int64_t src = sn;
                        if (valid(r + rs))
                            sn = src_of(r + rs);
                        vm2 = fmaxf(vm2, push_one<D, FULL>(c, b, gm, k, base + (int32_t)(lane0 + r) * step, load_global(c, src), sFa,
                                                           sFb, sD, mout));
                    }
            }
        }
        unsigned vb = __reduce_max_sync(0xffffffffu, __float_as_uint(sqrtf(vm2)));
        if (lane == 0 && vb)
            atomicMax(&c.stats[it.box].vmax, vb);
        __syncthreads();

        // remove the offsets, rebuild hi 2^KLO + lo and shift the tile into
        // the global accumulators
        for (int t = threadIdx.x; t < c.tile_vol; t += PUSH_THREADS) {
            int tx = t % c.tile[0], r = t / c.tile[0];
            int ty = r % c.tile[1], tz = r / c.tile[1];
            int64_t g = tile_global(c, b, gm, tx, ty, tz, D);
            int s = tile_slot(c, tx, ty, tz);
            const uint32_t kc = slot_count(c, sD, W_CNT_C, tx, ty, tz, D);
            const uint32_t km = FULL ? slot_count(c, sD, W_CNT_M, tx, ty, tz, D) : 0u;
#pragma unroll
            for (int ch = 0; ch < NCH; ++ch) {
                if (!FULL && ch >= CH_N)
                    break;
                const long long v = slot_value(sD, s, ch, kc, km);
                if (v) {
                    unsigned long long *dst = ch < CH_N ? c.corr + ch * c.nc + g : mout + (ch - CH_N) * c.nc + g;
                    atomicAdd(dst, (unsigned long long)v << k.ksh[ch]);
                }
            }
        }
        __syncthreads();
    }
}

template <int D, bool FULL>
__global__ void __launch_bounds__(PUSH_THREADS, MIN_BLOCKS<D>) k_push_mixed(Ctx c, const WorkItem *__restrict__ items,
                                                                 const int32_t *__restrict__ nitems,
                                                                 int32_t *__restrict__ work_ctr, int cur_out,
                                                                 float dt)
{
    extern __shared__ __align__(128) unsigned char smem[];
    push_items<D, FULL>(c, items, *nitems, work_ctr, cur_out, dt, smem);
}

// ---------------------------------------------------------------------------
// The whole step in one launch (mhdpic_run's steps): the corrector scales of
// every box, the push with both deposits, then the feedback to the gas and
// the field staging for the next step (what mhdpic_interp_push(dt, 1) and
// mhdpic_apply_feedback launch as three kernels), separated by grid-wide
// barriers.  The blocks are co-resident (cooperative launch); a barrier that
// waits longer than its limit raises MHDPIC_ST_BARRIER and the kernel returns
// (the step's results are then not valid), so it never hangs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long global_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Sense-counting grid barrier: the last block to arrive resets the count and
// advances the generation the others wait on.  The fences make every block's
// writes before the barrier visible to every block after it.
__device__ __forceinline__ bool grid_sync(GridBarrier *bar, unsigned nblocks, long long limit_ns, uint32_t *status)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned *gen = &bar->gen;
        const unsigned g0 = *gen;   // read before arriving
        __threadfence();
        if (atomicAdd(&bar->count, 1u) == nblocks - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const long long t0 = global_ns();
            while (*gen == g0) {
                if (global_ns() - t0 > limit_ns) {
                    set_status(status, MHDPIC_ST_BARRIER);
                    ok = 0;
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <int D>
__global__ void __launch_bounds__(PUSH_THREADS, MIN_BLOCKS<D>) k_step_mixed(Ctx c, const WorkItem *__restrict__ items,
                                                                 const int32_t *__restrict__ nitems,
                                                                 int32_t *__restrict__ work_ctr, int cur, float dtf,
                                                                 double dt, GridBarrier *bar, long long limit_ns)
{
    extern __shared__ __align__(128) unsigned char smem[];
    if (blockIdx.x == 0) {   // the corrector scales, and the push's work counter
        for (int bx = threadIdx.x; bx < c.nbox; bx += blockDim.x)
            scales_box(c, bx, dt);
        if (threadIdx.x == 0)
            *work_ctr = 0;
    }
    if (!grid_sync(bar, gridDim.x, limit_ns, c.status))
        return;
    push_items<D, true>(c, items, *nitems, work_ctr, cur ^ 1, dtf, smem);
    if (!grid_sync(bar, gridDim.x, limit_ns, c.status))
        return;
    prep_cells<MHDPIC_PREC_MIXED>(c, cur ^ 1, 1);
}

// Standalone charge/current deposit (eq:nJCR) at the particles' positions,
// through the same shared fixed-point tile as the push: persistent CTAs over
// the brick items of the last sort, particles read through the pending
// permutation when there is one (nothing is written back), each deposited by
// deposit_moments_one, so a particle contributes the same integers as in
// the push that put it there.  Moments go to momdep[cur], which the caller
// has zeroed.
template <int D>
__global__ void __launch_bounds__(PUSH_THREADS) k_deposit_mixed(Ctx c, const WorkItem *__restrict__ items,
                                                               const int32_t *__restrict__ nitems,
                                                               int32_t *__restrict__ work_ctr, int cur)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int S = c.tile_slots;
    int *sD = reinterpret_cast<int *>(smem);
    __shared__ int s_item;
    __shared__ MixedConst s_k;
    unsigned long long *mout = c.momdep[cur];
    const int nit = *nitems;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int NW = PUSH_THREADS / 32;
    const bool gather = c.perm_src != nullptr;

    for (;;) {
        if (threadIdx.x == 0)
            s_item = atomicAdd(work_ctr, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= nit)
            break;
        const WorkItem it = items[item];
        const BoxDev &b = c.boxes[it.box];
        const ItemGeom gm = item_geom(c, b, it.brick, D);
        for (int s = threadIdx.x; s < TILE_WORDS * S; s += PUSH_THREADS)
            sD[s] = 0;
        if (threadIdx.x == 0)
            item_const(b, 0.f, it.p1 - it.p0, D, s_k);
        __syncthreads();
        const MixedConst &k = s_k;
        {
            const LaneRange lr = lane_range(it, wid, NW);
            const int64_t lane0 = lane * lr.q;
            for (int64_t r = lr.first; r < lr.q; r += lr.stride) {
                if (lane0 + r >= lr.cnt)
                    continue;
                const int64_t j = lr.base + (int32_t)(lane0 + r) * lr.step;
                const int64_t src = gather ? (int64_t)__ldg(c.perm_src + j) : j;
                const PIn pin = load_global(c, src);
                if (pin.cell == DEAD_CELL)
                    continue;
                int ci[3];
                decode_cell(b, pin.cell, ci);
                const float ig = rsqrtf(fmaf(vsq3(pin.v), k.invC2, 1.f));
                deposit_moments_one<D>(c, b, gm, k, ci, pin.o, pin.v, ig, sD, mout);
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < c.tile_vol; t += PUSH_THREADS) {
            int tx = t % c.tile[0], r = t / c.tile[0];
            int ty = r % c.tile[1], tz = r / c.tile[1];
            int64_t g = tile_global(c, b, gm, tx, ty, tz, D);
            int s = tile_slot(c, tx, ty, tz);
            const uint32_t km = slot_count(c, sD, W_CNT_M, tx, ty, tz, D);
#pragma unroll
            for (int ch = CH_N; ch < NCH; ++ch) {
                const long long v = slot_value(sD, s, ch, 0u, km);
                if (v)
                    atomicAdd(mout + (ch - CH_N) * c.nc + g, (unsigned long long)v << k.ksh[ch]);
            }
        }
        __syncthreads();
    }
}

constexpr int PUSH_SMEM_LIMIT = 200 * 1024;

template <int D, bool FULL>
int occupancy_mixed(size_t bytes)
{
    cudaFuncSetAttribute(k_push_mixed<D, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, PUSH_SMEM_LIMIT);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push_mixed<D, FULL>, PUSH_THREADS, bytes);
    return nb;
}

template <int D>
int occupancy_all(size_t bytes)
{
    occupancy_mixed<D, false>(bytes);
    return occupancy_mixed<D, true>(bytes);
}

template <int D>
void launch_d(const Ctx &c, const SortScratch &s, int32_t *work_ctr, int cur_out, int full, float dt, int grid,
              size_t bytes, cudaStream_t st)
{
    if (full)
        k_push_mixed<D, true><<<grid, PUSH_THREADS, bytes, st>>>(c, s.items, s.nitems, work_ctr, cur_out, dt);
    else
        k_push_mixed<D, false><<<grid, PUSH_THREADS, bytes, st>>>(c, s.items, s.nitems, work_ctr, cur_out, dt);
}

}  // namespace

size_t push_smem_bytes_mixed(const Ctx &c)
{
    const bool staged = c.ndim == 3 ? STAGED<3> : STAGED<2>;
    const size_t ring = staged ? sizeof(int4) * RING_STAGES * (size_t)RING_RECS * PUSH_THREADS : 0;
    return push_layout(c.tile_slots, c.ftile_slots).ring + ring;
}

int push_blocks_per_sm_mixed(const Ctx &c)
{
    const size_t bytes = push_smem_bytes_mixed(c);
    const int nb = c.ndim == 3 ? occupancy_all<3>(bytes) : occupancy_all<2>(bytes);
    return nb < 1 ? 1 : nb;
}

int launch_deposit_mixed(const Ctx &c, const SortScratch &s, int32_t *work_ctr, int cur, int grid_blocks,
                         cudaStream_t st)
{
    const size_t bytes = sizeof(int) * TILE_WORDS * (size_t)c.tile_slots;
    cudaMemsetAsync(work_ctr, 0, sizeof(int32_t), st);
    if (c.ndim == 3) {
        cudaFuncSetAttribute(k_deposit_mixed<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, PUSH_SMEM_LIMIT);
        k_deposit_mixed<3><<<grid_blocks, PUSH_THREADS, bytes, st>>>(c, s.items, s.nitems, work_ctr, cur);
    } else {
        cudaFuncSetAttribute(k_deposit_mixed<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, PUSH_SMEM_LIMIT);
        k_deposit_mixed<2><<<grid_blocks, PUSH_THREADS, bytes, st>>>(c, s.items, s.nitems, work_ctr, cur);
    }
    return 1;
}

int step_blocks_per_sm_mixed(const Ctx &c)
{
    const size_t bytes = push_smem_bytes_mixed(c);
    int nb = 0;
    if (c.ndim == 3) {
        cudaFuncSetAttribute(k_step_mixed<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, PUSH_SMEM_LIMIT);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_mixed<3>, PUSH_THREADS, bytes);
    } else {
        cudaFuncSetAttribute(k_step_mixed<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, PUSH_SMEM_LIMIT);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_mixed<2>, PUSH_THREADS, bytes);
    }
    return nb;
}

int launch_step_mixed(const Ctx &c, const SortScratch &s, int32_t *work_ctr, int cur, double dt, int grid_blocks,
                      GridBarrier *bar, long long limit_ns, cudaStream_t st)
{
    const size_t bytes = push_smem_bytes_mixed(c);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid_blocks);
    cfg.blockDim = dim3(PUSH_THREADS);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const float dtf = (float)dt;
    cudaError_t e;
    if (c.ndim == 3)
        e = cudaLaunchKernelEx(&cfg, k_step_mixed<3>, c, (const WorkItem *)s.items, (const int32_t *)s.nitems,
                               work_ctr, cur, dtf, dt, bar, limit_ns);
    else
        e = cudaLaunchKernelEx(&cfg, k_step_mixed<2>, c, (const WorkItem *)s.items, (const int32_t *)s.nitems,
                               work_ctr, cur, dtf, dt, bar, limit_ns);
    return e == cudaSuccess ? 1 : -1;
}

int launch_push_mixed(const Ctx &c, const SortScratch &s, int32_t *work_ctr, int cur_out, int full, double dt,
                      int grid_blocks, cudaStream_t st)
{
    const size_t bytes = push_smem_bytes_mixed(c);
    cudaMemsetAsync(work_ctr, 0, sizeof(int32_t), st);
    if (c.ndim == 3)
        launch_d<3>(c, s, work_ctr, cur_out, full, (float)dt, grid_blocks, bytes, st);
    else
        launch_d<2>(c, s, work_ctr, cur_out, full, (float)dt, grid_blocks, bytes, st);
    return 1;
}

}  // namespace mhdpic
