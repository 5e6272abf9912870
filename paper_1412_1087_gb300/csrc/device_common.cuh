// Device helpers shared by the library's kernels.
#pragma once

#include "mhdpic_internal.cuh"

namespace mhdpic {

// Value of a fixed-point accumulator word (two's complement) at 1/inv_scale.
__device__ __forceinline__ double from_fixed(unsigned long long v, double inv_scale)
{
    return (double)(long long)v * inv_scale;
}

// Box that owns global index i, given CSR starts [nbox+1] (empty boxes skipped).
__device__ __forceinline__ int find_box(const int64_t *__restrict__ starts, int nbox, int64_t i)
{
    int lo = 0, hi = nbox - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(starts + mid) <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Slices of a box in the chunked reductions (totals, spectrum): one per
// per_chunk particles and cells, at least one, at most nchunks, so that
// boxes of very different sizes keep the blocks evenly loaded.
__device__ __forceinline__ int box_chunks(const BoxDev &b, int64_t per_chunk, int nchunks)
{
    const int64_t work = (b.part1 - b.part0) + b.ncell;
    const int64_t k = (work + per_chunk - 1) / per_chunk;
    return (int)(k < 1 ? 1 : (k > nchunks ? nchunks : k));
}

// Map an unwrapped cell coordinate g along dimension d onto the box: periodic
// wrap, or mirror fold at a reflecting wall (cell -1-k mirrors cell k); beyond
// an open face the cells take the last cell's values (and deposits).
__device__ __forceinline__ int map_coord(int g, int n, int bc)
{
    if (bc == MHDPIC_BC_PERIODIC) {
        if (g >= 0 && g < n)
            return g;
        int r = g % n;
        return r < 0 ? r + n : r;
    }
    if (bc == MHDPIC_BC_WALL_OPEN) {
        if (g < 0)
            g = -1 - g;
        return g >= n ? n - 1 : g;
    }
    for (int it = 0; it < 64; ++it) {
        if (g < 0)
            g = -1 - g;
        else if (g >= n)
            g = 2 * n - 1 - g;
        else
            return g;
    }
    return 0;
}

// A particle that left the box through an open face: cell -1 in mixed
// precision, a NaN first coordinate in FP64 (its four-velocity is 0).
constexpr int32_t DEAD_CELL = -1;

template <int PREC>
__device__ __forceinline__ bool particle_dead(const Ctx &c, int64_t i)
{
    return PREC == MHDPIC_PREC_MIXED ? c.pos[i].x == DEAD_CELL : isnan(c.x[i]);
}

// ---------------------------------------------------------------------------
// Two-word four-velocity of the mixed-precision particle record (mhdpic_vel):
// component d is v[d] + r_d 2^(e_d - 33), e_d the binary exponent of v[d]
// (at least RES_EMIN) and r_d the signed 10-bit field d of the residual word.
// ---------------------------------------------------------------------------
constexpr int RES_EMIN = -90;
constexpr int RES_SHIFT = 33;   // 23 mantissa bits + 10 residual bits
constexpr int RES_QMAX = 511;

__device__ __forceinline__ int res_exp(float h)
{
    const int e = ((__float_as_int(h) >> 23) & 0xff) - 127;   // 0 and subnormals give -127
    return e < RES_EMIN ? RES_EMIN : e;
}

// 2^(e - 33) and 2^(33 - e) for e in [RES_EMIN, 127]: both normal floats
__device__ __forceinline__ float res_quantum(int e) { return __int_as_float((e - RES_SHIFT + 127) << 23); }
__device__ __forceinline__ float res_inv_quantum(int e) { return __int_as_float((RES_SHIFT - e + 127) << 23); }

__device__ __forceinline__ int res_field(uint32_t w, int d)
{
    return (int)(w << (22 - 10 * d)) >> 22;
}

// Error-free sum a + b = s + t (Knuth's TwoSum), in explicitly rounded
// operations so that no contraction changes it.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &t)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi, r) += d: the exact sum hi + r q + d is rounded once, to the nearest
// number the record can hold (34 significant bits).  TwoSum gives the
// leading word and the exact remainder; the remainder is quantised to the
// new word's residual grid.
__device__ __forceinline__ void two_word_add(float &hi, int &r, float d)
{
    const float rv = __fmul_rn((float)r, res_quantum(res_exp(hi)));   // exact
    float s, t;
    two_sum(hi, d, s, t);
    const float rem = __fadd_rn(t, rv);
    float h2, rem2;
    two_sum(s, rem, h2, rem2);
    const int e2 = res_exp(h2);
    const float q = rintf(__fmul_rn(rem2, res_inv_quantum(e2)));
    const int qi = q > (float)RES_QMAX ? RES_QMAX : (q < -(float)RES_QMAX ? -RES_QMAX : (int)q);
    hi = h2;
    r = isfinite(h2) ? qi : 0;
}

__device__ __forceinline__ uint32_t res_pack(const int r[3])
{
    return ((uint32_t)r[0] & 0x3ffu) | (((uint32_t)r[1] & 0x3ffu) << 10) | (((uint32_t)r[2] & 0x3ffu) << 20);
}

// Exact double value of component d of a record.
__device__ __forceinline__ double vel_f64(const float4 &w, int d)
{
    const float h = d == 0 ? w.x : (d == 1 ? w.y : w.z);
    const int r = res_field(__float_as_uint(w.w), d);
    return (double)h + (double)r * (double)res_quantum(res_exp(h));
}

__device__ __forceinline__ void set_status(uint32_t *status, uint32_t flag)
{
    atomicOr(status, flag);
}

// Signed 64-bit fixed-point value added to an unsigned accumulator: two's
// complement addition is the same operation, so the grid sum is exact and
// independent of the order of the additions.
__device__ __forceinline__ void red_add(unsigned long long *addr, long long v)
{
    atomicAdd(addr, (unsigned long long)v);
}

__device__ __forceinline__ long long to_fixed(float v)
{
    return __float2ll_rn(v);
}

__device__ __forceinline__ long long to_fixed(double v)
{
    return __double2ll_rn(v);
}

// TSC (quadratic spline) weights from the offset o in [0,1) inside the cell:
// with delta = o - 1/2 the weights of cells i-1, i, i+1 are
// (1/2)(1/2 - delta)^2 = (1/2)(1-o)^2, 3/4 - delta^2, (1/2)(1/2 + delta)^2 = (1/2)o^2.
// The centre weight is one explicit fused multiply-add, so every kernel that
// forms these weights gets the same bits.
template <typename R>
__device__ __forceinline__ void tsc_from_offset(R o, R w[3])
{
    R a = R(1) - o;
    R dl = o - R(0.5);
    w[0] = R(0.5) * a * a;
    w[1] = fma(-dl, dl, R(0.75));
    w[2] = R(0.5) * o * o;
}

// |v|^2 in one fixed order of explicit operations (the same bits wherever
// it is evaluated).
__device__ __forceinline__ float vsq3(const float v[3])
{
    return fmaf(v[2], v[2], fmaf(v[1], v[1], __fmul_rn(v[0], v[0])));
}

// Index in the padded staged-field planes of box coordinates (gx, gy, gz),
// each in [-FGHOST, n + FGHOST) (z 0 in 2-D).
__device__ __forceinline__ int64_t fidx(const BoxDev &b, int gx, int gy, int gz)
{
    const int gzz = b.ndim == 3 ? gz + FGHOST : 0;
    return b.fcell0 + ((int64_t)gzz * b.pn[1] + (gy + FGHOST)) * b.pn[0] + (gx + FGHOST);
}

// Store the staged mixed-precision fields of box-local cell (x, y, z) at its
// own position and at every ghost that copies it: along each dimension the
// padded positions u in [-FGHOST, 0) and [n, pn - FGHOST) (up to the brick
// grid's end plus the halo, so that every push tile is inside the planes)
// whose stencil cell mapping (map_coord: periodic image, mirror image at a
// reflecting wall, the last cell beyond an open face) is the cell itself.
__device__ __forceinline__ bool ghost_of(int u, int x, int n, int bc)
{
    return (u < 0 || u >= n) && map_coord(u, n, bc) == x;
}

// Candidate k of one dimension: the cell itself (k = 0), the lower ghosts
// -1 .. -FGHOST, then the upper ghosts n .. hi - 1; count 1 + FGHOST + hi - n.
__device__ __forceinline__ int ghost_candidate(int k, int x, int n)
{
    return k == 0 ? x : (k <= FGHOST ? -k : n + (k - 1 - FGHOST));
}

__device__ __forceinline__ void store_fields_mixed(float4 *fa, float2 *fb, const BoxDev &b, int x, int y, int z,
                                                   float4 a, float2 bb)
{
    const int kx = 1 + FGHOST + (b.pn[0] - FGHOST - b.n[0]);
    const int ky = 1 + FGHOST + (b.pn[1] - FGHOST - b.n[1]);
    const int kz = b.ndim == 3 ? 1 + FGHOST + (b.pn[2] - FGHOST - b.n[2]) : 1;
    for (int iz = 0; iz < kz; ++iz) {
        const int uz = b.ndim == 3 ? ghost_candidate(iz, z, b.n[2]) : 0;
        if (iz > 0 && !ghost_of(uz, z, b.n[2], b.bc[2]))
            continue;
        for (int iy = 0; iy < ky; ++iy) {
            const int uy = ghost_candidate(iy, y, b.n[1]);
            if (iy > 0 && !ghost_of(uy, y, b.n[1], b.bc[1]))
                continue;
            for (int ix = 0; ix < kx; ++ix) {
                const int ux = ghost_candidate(ix, x, b.n[0]);
                if (ix > 0 && !ghost_of(ux, x, b.n[0], b.bc[0]))
                    continue;
                const int64_t f = fidx(b, ux, uy, uz);
                fa[f] = a;
                fb[f] = bb;
            }
        }
    }
}

// Box-local linear cell -> integer coordinates.
__device__ __forceinline__ void decode_cell(const BoxDev &b, int32_t c, int ci[3])
{
    uint32_t uc = (uint32_t)c;
    uint32_t k = fdiv(uc, b.div_nxy);
    uint32_t r = uc - k * (uint32_t)b.div_nxy.d;
    uint32_t j = fdiv(r, b.div_nx);
    ci[0] = (int)(r - j * (uint32_t)b.div_nx.d);
    ci[1] = (int)j;
    ci[2] = (int)k;
}

}  // namespace mhdpic
