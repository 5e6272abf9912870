// Fused particle step: drift, TSC gather, E-parallel cleaning, relativistic
// Boris kick-rotate-kick, drift, corrector deposit at x^(n+1/2) and moments
// deposit at x^(n+1) (App. A.1-A.3 of arXiv:1412.1087).
//
// Work decomposition: the particles are cell-sorted by brick, and the work
// list cuts every brick's particle range into items of at most
// ITEM_MAX_PARTICLES.  A persistent CTA takes items from an atomic counter.
// For each item it stages the brick's fields plus a halo of HALO cells in
// shared memory, accumulates both deposits in a shared int64 fixed-point tile
// of the same shape, and adds the tile to the global accumulators at the end.
// A particle whose stencil leaves the tile (it drifted away from its brick
// since the last sort) reads fields and deposits through global memory, so the
// result does not depend on the sort cadence.  All deposits are integer adds,
// so the sums are exact and independent of the order of the additions.
//
// Lane mapping: lane l of every warp owns the l-th 1/32 of the item's
// particles and the warps interleave inside it, so at any instruction the 32
// lanes of a warp work on particles about (item size / 32) apart, i.e. in
// different cells, which keeps same-address shared atomics rare.
#include "device_common.cuh"

namespace mhdpic {

namespace {

struct ItemGeom {
    int org[3];    // unwrapped box coordinates of tile cell (0,0,0)
    int ctr[3];    // brick centre, for periodic unwrapping of particle cells
    int half[3];   // brick[d] / 2
};

__device__ __forceinline__ ItemGeom item_geom(const Ctx &c, const BoxDev &b, int brick, int D)
{
    ItemGeom g;
    int bi = brick % b.nb[0];
    int r = brick / b.nb[0];
    int bj = r % b.nb[1];
    int bk = r / b.nb[1];
    int bc3[3] = {bi, bj, bk};
    for (int d = 0; d < 3; ++d) {
        if (d < D) {
            g.org[d] = bc3[d] * c.brick[d] - HALO;
            g.half[d] = c.brick[d] / 2;
            g.ctr[d] = bc3[d] * c.brick[d] + g.half[d];
        } else {
            g.org[d] = 0;
            g.half[d] = 0;
            g.ctr[d] = 0;
        }
    }
    return g;
}

// Tile coordinate of a particle's cell along d (periodic unwrapping toward the
// brick centre).  Returns true when the whole 3-point stencil is in the tile.
__device__ __forceinline__ bool tile_rel(const Ctx &c, const BoxDev &b, const ItemGeom &g, int d,
                                         int ci, int &rel)
{
    int dd = ci - g.ctr[d];
    if (b.bc[d] == MHDPIC_BC_PERIODIC) {
        int n = b.n[d];
        if (dd > n / 2)
            dd -= n;
        else if (dd < -(n / 2))
            dd += n;
    }
    rel = dd + g.half[d] + HALO;
    return rel >= 1 && rel <= c.tile[d] - 2;
}

// ---------------------------------------------------------------------------
// mixed precision: int32 cell + f32 offset positions, f32 push
// ---------------------------------------------------------------------------

struct MixedConst {
    float hdx[3];    // dt / (2 dx)
    float invC2;     // 1 / C^2
    float hh;        // (q/mc) dt / 2
    float m;
    float qn;        // (q/mc) m / dV
    float scale[NCH];
    float vlim[NCH]; // particle quantity limits (overflow guard), pre-scaled
};

// Move the offset back into [0,1), carrying whole cells; apply the particle
// boundary (periodic wrap or specular reflection, which flips v[d]).
__device__ __forceinline__ void renorm_mixed(const BoxDev &b, int d, int &ci, float &o, float &vd,
                                             uint32_t *status)
{
    float f = floorf(o);
    if (f != 0.f) {
        int k = (int)f;
        if (k > 2 || k < -2)
            set_status(status, MHDPIC_ST_FAST_MOVER);
        ci += k;
        o -= f;
    }
    if (o >= 1.f) {   // o was a tiny negative number that rounded up
        o -= 1.f;
        ci += 1;
    }
    int n = b.n[d];
    if (ci >= 0 && ci < n)
        return;
    if (b.bc[d] == MHDPIC_BC_PERIODIC) {
        ci = map_coord(ci, n, MHDPIC_BC_PERIODIC);
        return;
    }
    // reflecting wall: position s = ci + o mirrors to -s or 2n - s
    if (ci < 0) {
        ci = -1 - ci;
        o = 1.f - o;
        if (o >= 1.f) {
            o = 0.f;
            ci += 1;
        }
    } else {
        ci = 2 * n - 1 - ci;
        o = 1.f - o;
        if (o >= 1.f) {
            if (ci + 1 >= n)
                o = 0x1.fffffep-1f;   // exactly on the wall: just inside it
            else {
                o = 0.f;
                ci += 1;
            }
        }
    }
    vd = -vd;
    if (ci < 0 || ci >= n) {   // moved by more than the box: clamp and flag
        set_status(status, MHDPIC_ST_FAST_MOVER);
        ci = ci < 0 ? 0 : n - 1;
    }
}

template <int D>
__device__ __forceinline__ void gather_mixed(const Ctx &c, const BoxDev &b, bool in_tile, const int rel[3],
                                             const int ci[3], const float wx[3], const float wy[3],
                                             const float wz[3], const float4 *__restrict__ sF,
                                             float E[3], float Bf[3])
{
    E[0] = E[1] = E[2] = Bf[0] = Bf[1] = Bf[2] = 0.f;
    const int TX = c.tile[0], TY = c.tile[1];
    if (in_tile) {
        int base = (rel[0] - 1) + TX * ((rel[1] - 1) + TY * (D == 3 ? rel[2] - 1 : 0));
#pragma unroll
        for (int cz = 0; cz < (D == 3 ? 3 : 1); ++cz)
#pragma unroll
            for (int cy = 0; cy < 3; ++cy) {
                float wyz = wy[cy] * (D == 3 ? wz[cz] : 1.f);
#pragma unroll
                for (int cx = 0; cx < 3; ++cx) {
                    float w = wx[cx] * wyz;
                    int idx = base + cx + TX * (cy + TY * cz);
                    float4 f1 = sF[2 * idx], f2 = sF[2 * idx + 1];
                    E[0] = fmaf(w, f1.x, E[0]);
                    E[1] = fmaf(w, f1.y, E[1]);
                    E[2] = fmaf(w, f1.z, E[2]);
                    Bf[0] = fmaf(w, f1.w, Bf[0]);
                    Bf[1] = fmaf(w, f2.x, Bf[1]);
                    Bf[2] = fmaf(w, f2.y, Bf[2]);
                }
            }
    } else {
        const float4 *__restrict__ gF = reinterpret_cast<const float4 *>(c.f32);
        int gx[3], gy[3], gz[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gx[a] = map_coord(ci[0] + a - 1, b.n[0], b.bc[0]);
            gy[a] = map_coord(ci[1] + a - 1, b.n[1], b.bc[1]);
            if (D == 3)
                gz[a] = map_coord(ci[2] + a - 1, b.n[2], b.bc[2]);
        }
        for (int cz = 0; cz < (D == 3 ? 3 : 1); ++cz)
            for (int cy = 0; cy < 3; ++cy) {
                float wyz = wy[cy] * (D == 3 ? wz[cz] : 1.f);
                for (int cx = 0; cx < 3; ++cx) {
                    float w = wx[cx] * wyz;
                    int64_t g = b.cell0 + ((int64_t)gz[cz] * b.n[1] + gy[cy]) * b.n[0] + gx[cx];
                    float4 f1 = __ldg(gF + 2 * g), f2 = __ldg(gF + 2 * g + 1);
                    E[0] = fmaf(w, f1.x, E[0]);
                    E[1] = fmaf(w, f1.y, E[1]);
                    E[2] = fmaf(w, f1.z, E[2]);
                    Bf[0] = fmaf(w, f1.w, Bf[0]);
                    Bf[1] = fmaf(w, f2.x, Bf[1]);
                    Bf[2] = fmaf(w, f2.y, Bf[2]);
                }
            }
    }
}

// Deposit 4 pre-scaled quantities q (channels ch0..ch0+3) with TSC weights.
template <int D, typename R>
__device__ __forceinline__ void deposit4(const Ctx &c, const BoxDev &b, bool in_tile, const int rel[3],
                                         const int ci[3], const R wx[3], const R wy[3], const R wz[3],
                                         const R q[4], int ch0, unsigned long long *__restrict__ sD,
                                         unsigned long long *__restrict__ g0,
                                         unsigned long long *__restrict__ g1,
                                         unsigned long long *__restrict__ g2,
                                         unsigned long long *__restrict__ g3)
{
    const int TX = c.tile[0], TY = c.tile[1], T = c.tile_vol;
    if (in_tile) {
        int base = (rel[0] - 1) + TX * ((rel[1] - 1) + TY * (D == 3 ? rel[2] - 1 : 0));
        unsigned long long *s0 = sD + (ch0 + 0) * T, *s1 = sD + (ch0 + 1) * T,
                           *s2 = sD + (ch0 + 2) * T, *s3 = sD + (ch0 + 3) * T;
#pragma unroll
        for (int cz = 0; cz < (D == 3 ? 3 : 1); ++cz)
#pragma unroll
            for (int cy = 0; cy < 3; ++cy) {
                R wyz = wy[cy] * (D == 3 ? wz[cz] : R(1));
#pragma unroll
                for (int cx = 0; cx < 3; ++cx) {
                    R w = wx[cx] * wyz;
                    int idx = base + cx + TX * (cy + TY * cz);
                    red_add(s0 + idx, to_fixed(q[0] * w));
                    red_add(s1 + idx, to_fixed(q[1] * w));
                    red_add(s2 + idx, to_fixed(q[2] * w));
                    red_add(s3 + idx, to_fixed(q[3] * w));
                }
            }
    } else {
        int gx[3], gy[3], gz[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gx[a] = map_coord(ci[0] + a - 1, b.n[0], b.bc[0]);
            gy[a] = map_coord(ci[1] + a - 1, b.n[1], b.bc[1]);
            if (D == 3)
                gz[a] = map_coord(ci[2] + a - 1, b.n[2], b.bc[2]);
        }
        for (int cz = 0; cz < (D == 3 ? 3 : 1); ++cz)
            for (int cy = 0; cy < 3; ++cy) {
                R wyz = wy[cy] * (D == 3 ? wz[cz] : R(1));
                for (int cx = 0; cx < 3; ++cx) {
                    R w = wx[cx] * wyz;
                    int64_t g = b.cell0 + ((int64_t)gz[cz] * b.n[1] + gy[cy]) * b.n[0] + gx[cx];
                    red_add(g0 + g, to_fixed(q[0] * w));
                    red_add(g1 + g, to_fixed(q[1] * w));
                    red_add(g2 + g, to_fixed(q[2] * w));
                    red_add(g3 + g, to_fixed(q[3] * w));
                }
            }
    }
}

template <int D, bool FULL>
__device__ __forceinline__ float push_one_mixed(const Ctx &c, const BoxDev &b, const ItemGeom &gm,
                                               const MixedConst &k, int64_t j, const float4 *sF,
                                               unsigned long long *sD, unsigned long long *mout)
{
    const int64_t np = c.np, nc = c.nc;
    int ci[3];
    decode_cell(b, c.cell[j], ci);
    float o[3] = {0.f, 0.f, 0.f}, v[3];
#pragma unroll
    for (int d = 0; d < D; ++d)
        o[d] = c.off[d * np + j];
#pragma unroll
    for (int d = 0; d < 3; ++d)
        v[d] = c.p[d * np + j];

    // drift to x^(n+1/2) with u = v / gamma
    const float ign = rsqrtf(fmaf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2], k.invC2, 1.f));
#pragma unroll
    for (int d = 0; d < D; ++d) {
        o[d] = fmaf(k.hdx[d] * ign, v[d], o[d]);
        renorm_mixed(b, d, ci[d], o[d], v[d], c.status);
    }

    // TSC weights and tile position at x^(n+1/2)
    float w[3][3] = {{0.f, 1.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 1.f, 0.f}};
    int rel[3] = {0, 0, 0};
    bool in_tile = true;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        tsc_from_offset<float>(o[d], w[d]);
        in_tile &= tile_rel(c, b, gm, d, ci[d], rel[d]);
    }

    float E[3], Bf[3];
    gather_mixed<D>(c, b, in_tile, rel, ci, w[0], w[1], w[2], sF, E, Bf);

    // remove the component of E along B
    float B2 = Bf[0] * Bf[0] + Bf[1] * Bf[1] + Bf[2] * Bf[2];
    if (B2 > 0.f) {
        float eb = (E[0] * Bf[0] + E[1] * Bf[1] + E[2] * Bf[2]) / B2;
        E[0] = fmaf(-eb, Bf[0], E[0]);
        E[1] = fmaf(-eb, Bf[1], E[1]);
        E[2] = fmaf(-eb, Bf[2], E[2]);
    }

    // Boris: v0 = v + (h/2)E; b = (h/2)B/gamma(v0); v1 = v0 + 2(v0 + v0 x b) x b/(1+b^2)
    float e[3] = {k.hh * E[0], k.hh * E[1], k.hh * E[2]};
    float v0[3] = {v[0] + e[0], v[1] + e[1], v[2] + e[2]};
    const float ig1 = rsqrtf(fmaf(v0[0] * v0[0] + v0[1] * v0[1] + v0[2] * v0[2], k.invC2, 1.f));
    float bb[3] = {k.hh * ig1 * Bf[0], k.hh * ig1 * Bf[1], k.hh * ig1 * Bf[2]};
    float t[3] = {v0[0] + (v0[1] * bb[2] - v0[2] * bb[1]), v0[1] + (v0[2] * bb[0] - v0[0] * bb[2]),
                  v0[2] + (v0[0] * bb[1] - v0[1] * bb[0])};
    float s2 = 2.f / (1.f + bb[0] * bb[0] + bb[1] * bb[1] + bb[2] * bb[2]);
    float rot[3] = {s2 * (t[1] * bb[2] - t[2] * bb[1]), s2 * (t[2] * bb[0] - t[0] * bb[2]),
                    s2 * (t[0] * bb[1] - t[1] * bb[0])};
    float v1[3] = {v0[0] + rot[0], v0[1] + rot[1], v0[2] + rot[2]};
    float vn[3] = {v1[0] + e[0], v1[1] + e[1], v1[2] + e[2]};

    // dv = v^(n+1) - v^(n) = h E + rot without cancellation; the rotation keeps
    // |v| so dE_k comes from the two half kicks only:
    // E_k(a) - E_k(b) = (a - b).(a + b)/(gamma_a + gamma_b)
    const float ig2 = rsqrtf(fmaf(vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2], k.invC2, 1.f));
    const float gn = 1.f / ign, g1 = 1.f / ig1, g2 = 1.f / ig2;
    float dEk = (e[0] * (vn[0] + v1[0]) + e[1] * (vn[1] + v1[1]) + e[2] * (vn[2] + v1[2])) / (g2 + g1) +
                (e[0] * (v0[0] + v[0]) + e[1] * (v0[1] + v[1]) + e[2] * (v0[2] + v[2])) / (g1 + gn);
    float qc[4] = {-k.m * (2.f * e[0] + rot[0]) * k.scale[CH_MX], -k.m * (2.f * e[1] + rot[1]) * k.scale[CH_MY],
                   -k.m * (2.f * e[2] + rot[2]) * k.scale[CH_MZ], -k.m * dEk * k.scale[CH_E]};
    if (fabsf(qc[0]) > k.vlim[CH_MX] || fabsf(qc[1]) > k.vlim[CH_MY] || fabsf(qc[2]) > k.vlim[CH_MZ] ||
        fabsf(qc[3]) > k.vlim[CH_E])
        set_status(c.status, MHDPIC_ST_OVERFLOW);
    deposit4<D, float>(c, b, in_tile, rel, ci, w[0], w[1], w[2], qc, CH_MX, sD, c.corr,
                       c.corr + nc, c.corr + 2 * nc, c.corr + 3 * nc);

    // drift to x^(n+1)
#pragma unroll
    for (int d = 0; d < D; ++d) {
        o[d] = fmaf(k.hdx[d] * ig2, vn[d], o[d]);
        renorm_mixed(b, d, ci[d], o[d], vn[d], c.status);
    }

    if (FULL) {
        float w2[3][3] = {{0.f, 1.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 1.f, 0.f}};
        int rel2[3] = {0, 0, 0};
        bool in2 = true;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            tsc_from_offset<float>(o[d], w2[d]);
            in2 &= tile_rel(c, b, gm, d, ci[d], rel2[d]);
        }
        float qm[4] = {k.qn * k.scale[CH_N], k.qn * ig2 * vn[0] * k.scale[CH_JX],
                       k.qn * ig2 * vn[1] * k.scale[CH_JY], k.qn * ig2 * vn[2] * k.scale[CH_JZ]};
        deposit4<D, float>(c, b, in2, rel2, ci, w2[0], w2[1], w2[2], qm, CH_N, sD, mout, mout + nc,
                           mout + 2 * nc, mout + 3 * nc);
    }

    if (!isfinite(vn[0] + vn[1] + vn[2]))
        set_status(c.status, MHDPIC_ST_NONFINITE);
    c.cell[j] = (int32_t)(((int64_t)ci[2] * b.n[1] + ci[1]) * b.n[0] + ci[0]);
#pragma unroll
    for (int d = 0; d < D; ++d)
        c.off[d * np + j] = o[d];
#pragma unroll
    for (int d = 0; d < 3; ++d)
        c.p[d * np + j] = vn[d];
    return vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2];
}

// ---------------------------------------------------------------------------
// FP64: absolute positions, the oracle's arithmetic order
// ---------------------------------------------------------------------------

struct F64Const {
    double dt, h, C, m, qn;
    double scale[NCH];
    double vlim[NCH];
};

__device__ __forceinline__ void boundary_f64(const BoxDev &b, int d, double &x, double &vd)
{
    double lo = b.x0[d];
    double L = b.n[d] * b.dx[d];
    double hi = lo + L;
    if (b.bc[d] == MHDPIC_BC_PERIODIC) {
        double r = x - lo;
        if (r < 0.0 || r >= L)
            r -= L * floor(r / L);
        if (r >= L)
            r -= L;
        x = lo + r;
    } else {
        if (x < lo) {
            x = 2.0 * lo - x;
            vd = -vd;
        } else if (x >= hi) {
            x = 2.0 * hi - x;
            vd = -vd;
        }
        if (x >= hi)
            x = nextafter(hi, lo);
        if (x < lo)
            x = lo;
    }
}

template <int D>
__device__ __forceinline__ void gather_f64(const Ctx &c, const BoxDev &b, bool in_tile, const int rel[3],
                                           const int ci[3], const double wx[3], const double wy[3],
                                           const double wz[3], const double2 *__restrict__ sF,
                                           double E[3], double Bf[3])
{
    E[0] = E[1] = E[2] = Bf[0] = Bf[1] = Bf[2] = 0.0;
    const int TX = c.tile[0], TY = c.tile[1];
    const double2 *__restrict__ gF = reinterpret_cast<const double2 *>(c.f64);
    int gx[3], gy[3], gz[3] = {0, 0, 0};
    if (!in_tile) {
        for (int a = 0; a < 3; ++a) {
            gx[a] = map_coord(ci[0] + a - 1, b.n[0], b.bc[0]);
            gy[a] = map_coord(ci[1] + a - 1, b.n[1], b.bc[1]);
            if (D == 3)
                gz[a] = map_coord(ci[2] + a - 1, b.n[2], b.bc[2]);
        }
    }
    int base = (rel[0] - 1) + TX * ((rel[1] - 1) + TY * (D == 3 ? rel[2] - 1 : 0));
    for (int cz = 0; cz < (D == 3 ? 3 : 1); ++cz)
        for (int cy = 0; cy < 3; ++cy)
            for (int cx = 0; cx < 3; ++cx) {
                double w = wx[cx] * wy[cy] * (D == 3 ? wz[cz] : 1.0);
                double2 a0, a1, a2;
                if (in_tile) {
                    int idx = base + cx + TX * (cy + TY * cz);
                    a0 = sF[3 * idx];
                    a1 = sF[3 * idx + 1];
                    a2 = sF[3 * idx + 2];
                } else {
                    int64_t g = b.cell0 + ((int64_t)gz[cz] * b.n[1] + gy[cy]) * b.n[0] + gx[cx];
                    a0 = __ldg(gF + 3 * g);
                    a1 = __ldg(gF + 3 * g + 1);
                    a2 = __ldg(gF + 3 * g + 2);
                }
                E[0] += w * a0.x;
                E[1] += w * a0.y;
                E[2] += w * a1.x;
                Bf[0] += w * a1.y;
                Bf[1] += w * a2.x;
                Bf[2] += w * a2.y;
            }
}

template <int D>
__device__ __forceinline__ void cell_of_f64(const BoxDev &b, const double x[3], int ci[3], double w[3][3])
{
    for (int d = 0; d < D; ++d) {
        double s = (x[d] - b.x0[d]) * b.inv_dx[d];
        double f = floor(s);
        ci[d] = (int)f;
        tsc_from_offset<double>(s - f, w[d]);
    }
}

template <int D, bool FULL>
__device__ __forceinline__ float push_one_f64(const Ctx &c, const BoxDev &b, const ItemGeom &gm,
                                             const F64Const &k, int64_t j, const double2 *sF,
                                             unsigned long long *sD, unsigned long long *mout)
{
    const int64_t np = c.np, nc = c.nc;
    const double C = k.C;
    double x[3] = {0.0, 0.0, 0.0}, v[3];
    for (int d = 0; d < D; ++d)
        x[d] = c.x[d * np + j];
    for (int d = 0; d < 3; ++d)
        v[d] = c.p64[d * np + j];

    double g0 = sqrt(C * C + (v[0] * v[0] + v[1] * v[1] + v[2] * v[2])) / C;
    for (int d = 0; d < D; ++d) {
        x[d] = x[d] + 0.5 * k.dt * (v[d] / g0);
        boundary_f64(b, d, x[d], v[d]);
    }

    int ci[3] = {0, 0, 0}, rel[3] = {0, 0, 0};
    double w[3][3] = {{0, 1, 0}, {0, 1, 0}, {0, 1, 0}};
    cell_of_f64<D>(b, x, ci, w);
    bool in_tile = true;
    for (int d = 0; d < D; ++d)
        in_tile &= tile_rel(c, b, gm, d, ci[d], rel[d]);

    double E[3], Bf[3];
    gather_f64<D>(c, b, in_tile, rel, ci, w[0], w[1], w[2], sF, E, Bf);
    double B2 = Bf[0] * Bf[0] + Bf[1] * Bf[1] + Bf[2] * Bf[2];
    if (B2 > 0.0) {
        double eb = (E[0] * Bf[0] + E[1] * Bf[1] + E[2] * Bf[2]) / B2;
        for (int d = 0; d < 3; ++d)
            E[d] -= eb * Bf[d];
    }

    const double h = k.h;
    double v0[3], v1[3], vn[3], bb[3], t[3], txb[3];
    for (int d = 0; d < 3; ++d)
        v0[d] = v[d] + 0.5 * h * E[d];
    double gam = sqrt(C * C + (v0[0] * v0[0] + v0[1] * v0[1] + v0[2] * v0[2])) / C;
    for (int d = 0; d < 3; ++d)
        bb[d] = 0.5 * h * Bf[d] / gam;
    t[0] = v0[1] * bb[2] - v0[2] * bb[1];
    t[1] = v0[2] * bb[0] - v0[0] * bb[2];
    t[2] = v0[0] * bb[1] - v0[1] * bb[0];
    for (int d = 0; d < 3; ++d)
        t[d] += v0[d];
    txb[0] = t[1] * bb[2] - t[2] * bb[1];
    txb[1] = t[2] * bb[0] - t[0] * bb[2];
    txb[2] = t[0] * bb[1] - t[1] * bb[0];
    double b2 = bb[0] * bb[0] + bb[1] * bb[1] + bb[2] * bb[2];
    for (int d = 0; d < 3; ++d)
        v1[d] = v0[d] + 2.0 * txb[d] / (1.0 + b2);
    for (int d = 0; d < 3; ++d)
        vn[d] = v1[d] + 0.5 * h * E[d];

    double g1 = sqrt(C * C + (vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2])) / C;
    double dv[3], sv[3];
    for (int d = 0; d < 3; ++d) {
        dv[d] = vn[d] - v[d];
        sv[d] = vn[d] + v[d];
    }
    double dEk = (dv[0] * sv[0] + dv[1] * sv[1] + dv[2] * sv[2]) / (g1 + g0);
    double qc[4] = {-k.m * dv[0] * k.scale[CH_MX], -k.m * dv[1] * k.scale[CH_MY],
                    -k.m * dv[2] * k.scale[CH_MZ], -k.m * dEk * k.scale[CH_E]};
    if (fabs(qc[0]) > k.vlim[CH_MX] || fabs(qc[1]) > k.vlim[CH_MY] || fabs(qc[2]) > k.vlim[CH_MZ] ||
        fabs(qc[3]) > k.vlim[CH_E])
        set_status(c.status, MHDPIC_ST_OVERFLOW);
    deposit4<D, double>(c, b, in_tile, rel, ci, w[0], w[1], w[2], qc, CH_MX, sD, c.corr, c.corr + nc,
                        c.corr + 2 * nc, c.corr + 3 * nc);

    for (int d = 0; d < D; ++d) {
        x[d] = x[d] + 0.5 * k.dt * (vn[d] / g1);
        boundary_f64(b, d, x[d], vn[d]);
    }
    if (FULL) {
        int ci2[3] = {0, 0, 0}, rel2[3] = {0, 0, 0};
        double w2[3][3] = {{0, 1, 0}, {0, 1, 0}, {0, 1, 0}};
        cell_of_f64<D>(b, x, ci2, w2);
        bool in2 = true;
        for (int d = 0; d < D; ++d)
            in2 &= tile_rel(c, b, gm, d, ci2[d], rel2[d]);
        double qm[4];
        qm[0] = k.qn * k.scale[CH_N];
        for (int d = 0; d < 3; ++d)
            qm[1 + d] = k.qn * (vn[d] / g1) * k.scale[CH_JX + d];
        deposit4<D, double>(c, b, in2, rel2, ci2, w2[0], w2[1], w2[2], qm, CH_N, sD, mout, mout + nc,
                            mout + 2 * nc, mout + 3 * nc);
    }
    if (!isfinite(vn[0] + vn[1] + vn[2]))
        set_status(c.status, MHDPIC_ST_NONFINITE);
    for (int d = 0; d < D; ++d)
        c.x[d * np + j] = x[d];
    for (int d = 0; d < 3; ++d)
        c.p64[d * np + j] = vn[d];
    return (float)(vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2]);
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------

template <int D, int PREC, bool FULL>
__global__ void __launch_bounds__(PUSH_THREADS) k_push(Ctx c, const WorkItem *__restrict__ items,
                                                      const int32_t *__restrict__ nitems,
                                                      int32_t *__restrict__ work_ctr, int cur_out,
                                                      double dt)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = c.tile_vol;
    unsigned long long *sD = reinterpret_cast<unsigned long long *>(smem);
    void *sFv = smem + sizeof(unsigned long long) * NCH * T;
    __shared__ int s_item;
    unsigned long long *mout = c.momdep[cur_out];
    const int nit = *nitems;
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

        // stage the tile's fields and clear its deposit accumulators
        for (int t = threadIdx.x; t < T; t += PUSH_THREADS) {
            int tx = t % c.tile[0];
            int r = t / c.tile[0];
            int ty = r % c.tile[1];
            int tz = r / c.tile[1];
            int gx = map_coord(gm.org[0] + tx, b.n[0], b.bc[0]);
            int gy = map_coord(gm.org[1] + ty, b.n[1], b.bc[1]);
            int gz = D == 3 ? map_coord(gm.org[2] + tz, b.n[2], b.bc[2]) : 0;
            int64_t g = b.cell0 + ((int64_t)gz * b.n[1] + gy) * b.n[0] + gx;
            if (PREC == MHDPIC_PREC_MIXED) {
                const float4 *gF = reinterpret_cast<const float4 *>(c.f32);
                float4 *sF = reinterpret_cast<float4 *>(sFv);
                sF[2 * t] = __ldg(gF + 2 * g);
                sF[2 * t + 1] = __ldg(gF + 2 * g + 1);
            } else {
                const double2 *gF = reinterpret_cast<const double2 *>(c.f64);
                double2 *sF = reinterpret_cast<double2 *>(sFv);
                sF[3 * t] = __ldg(gF + 3 * g);
                sF[3 * t + 1] = __ldg(gF + 3 * g + 1);
                sF[3 * t + 2] = __ldg(gF + 3 * g + 2);
            }
#pragma unroll
            for (int ch = 0; ch < NCH; ++ch)
                sD[ch * T + t] = 0ull;
        }
        __syncthreads();

        const int64_t cnt = it.p1 - it.p0;
        const int64_t Q = (cnt + 31) / 32;
        float vm2 = 0.f;   // largest |v|^2 pushed by this thread (sizes the next scales)
        if (PREC == MHDPIC_PREC_MIXED) {
            MixedConst k;
            for (int d = 0; d < 3; ++d)
                k.hdx[d] = (float)(0.5 * dt * b.inv_dx[d]);
            k.invC2 = (float)(1.0 / (b.C * b.C));
            k.hh = (float)(0.5 * b.qm_cr * dt);
            k.m = (float)b.m_cr;
            k.qn = (float)(b.qm_cr * b.m_cr * b.inv_dV);
            for (int ch = 0; ch < NCH; ++ch) {
                k.scale[ch] = (float)b.scale[ch];
                k.vlim[ch] = (float)(b.qmax[ch] * b.scale[ch]);
            }
            const float4 *sF = reinterpret_cast<const float4 *>(sFv);
            for (int64_t r = wid; r < Q; r += NW) {
                int64_t loc = lane * Q + r;
                if (loc < cnt)
                    vm2 = fmaxf(vm2, push_one_mixed<D, FULL>(c, b, gm, k, it.p0 + loc, sF, sD, mout));
            }
        } else {
            F64Const k;
            k.dt = dt;
            k.h = b.qm_cr * dt;
            k.C = b.C;
            k.m = b.m_cr;
            k.qn = b.qm_cr * b.m_cr * b.inv_dV;
            for (int ch = 0; ch < NCH; ++ch) {
                k.scale[ch] = b.scale[ch];
                k.vlim[ch] = b.qmax[ch] * b.scale[ch];
            }
            const double2 *sF = reinterpret_cast<const double2 *>(sFv);
            for (int64_t r = wid; r < Q; r += NW) {
                int64_t loc = lane * Q + r;
                if (loc < cnt)
                    vm2 = fmaxf(vm2, push_one_f64<D, FULL>(c, b, gm, k, it.p0 + loc, sF, sD, mout));
            }
        }
        {
            unsigned vb = __reduce_max_sync(0xffffffffu, __float_as_uint(sqrtf(vm2)));
            if (lane == 0 && vb)
                atomicMax(&c.stats[it.box].vmax, vb);
        }
        __syncthreads();

        // add the tile to the global accumulators
        for (int t = threadIdx.x; t < T; t += PUSH_THREADS) {
            int tx = t % c.tile[0];
            int r = t / c.tile[0];
            int ty = r % c.tile[1];
            int tz = r / c.tile[1];
            int gx = map_coord(gm.org[0] + tx, b.n[0], b.bc[0]);
            int gy = map_coord(gm.org[1] + ty, b.n[1], b.bc[1]);
            int gz = D == 3 ? map_coord(gm.org[2] + tz, b.n[2], b.bc[2]) : 0;
            int64_t g = b.cell0 + ((int64_t)gz * b.n[1] + gy) * b.n[0] + gx;
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
                unsigned long long a = sD[ch * T + t];
                if (a)
                    atomicAdd(c.corr + ch * c.nc + g, a);
            }
            if (FULL) {
#pragma unroll
                for (int ch = 0; ch < 4; ++ch) {
                    unsigned long long a = sD[(CH_N + ch) * T + t];
                    if (a)
                        atomicAdd(mout + ch * c.nc + g, a);
                }
            }
        }
        __syncthreads();
    }
}

// The opt-in limit is set to the largest tile any context may use, so
// contexts with different bricks can coexist in one process.
constexpr int PUSH_SMEM_LIMIT = 200 * 1024;

template <int D, int PREC, bool FULL>
int occupancy(size_t bytes)
{
    cudaFuncSetAttribute(k_push<D, PREC, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, PUSH_SMEM_LIMIT);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push<D, PREC, FULL>, PUSH_THREADS, bytes);
    return nb;
}

}  // namespace

size_t push_smem_bytes(const Ctx &c)
{
    size_t per_cell = sizeof(unsigned long long) * NCH + (c.prec == MHDPIC_PREC_MIXED ? 32 : 48);
    return per_cell * (size_t)c.tile_vol;
}

int push_blocks_per_sm(const Ctx &c)
{
    size_t bytes = push_smem_bytes(c);
    // every instantiation gets the opt-in limit once
    occupancy<3, MHDPIC_PREC_MIXED, false>(bytes);
    occupancy<2, MHDPIC_PREC_MIXED, false>(bytes);
    occupancy<3, MHDPIC_PREC_FP64, false>(bytes);
    occupancy<2, MHDPIC_PREC_FP64, false>(bytes);
    occupancy<3, MHDPIC_PREC_MIXED, true>(bytes);
    occupancy<2, MHDPIC_PREC_MIXED, true>(bytes);
    occupancy<3, MHDPIC_PREC_FP64, true>(bytes);
    occupancy<2, MHDPIC_PREC_FP64, true>(bytes);
    int nb;
    if (c.prec == MHDPIC_PREC_MIXED) {
        if (c.ndim == 3) {
            occupancy<3, MHDPIC_PREC_MIXED, false>(bytes);
            nb = occupancy<3, MHDPIC_PREC_MIXED, true>(bytes);
        } else {
            occupancy<2, MHDPIC_PREC_MIXED, false>(bytes);
            nb = occupancy<2, MHDPIC_PREC_MIXED, true>(bytes);
        }
    } else {
        if (c.ndim == 3) {
            occupancy<3, MHDPIC_PREC_FP64, false>(bytes);
            nb = occupancy<3, MHDPIC_PREC_FP64, true>(bytes);
        } else {
            occupancy<2, MHDPIC_PREC_FP64, false>(bytes);
            nb = occupancy<2, MHDPIC_PREC_FP64, true>(bytes);
        }
    }
    return nb < 1 ? 1 : nb;
}

int launch_push(const Ctx &c, const SortScratch &s, int32_t *work_ctr, int cur_out, int full, double dt,
                int grid_blocks, cudaStream_t st)
{
    size_t bytes = push_smem_bytes(c);
    cudaMemsetAsync(work_ctr, 0, sizeof(int32_t), st);
#define MHDPIC_LAUNCH(DD, PP, FF) \
    k_push<DD, PP, FF><<<grid_blocks, PUSH_THREADS, bytes, st>>>(c, s.items, s.nitems, work_ctr, cur_out, dt)
    if (c.prec == MHDPIC_PREC_MIXED) {
        if (c.ndim == 3) {
            if (full) MHDPIC_LAUNCH(3, MHDPIC_PREC_MIXED, true);
            else MHDPIC_LAUNCH(3, MHDPIC_PREC_MIXED, false);
        } else {
            if (full) MHDPIC_LAUNCH(2, MHDPIC_PREC_MIXED, true);
            else MHDPIC_LAUNCH(2, MHDPIC_PREC_MIXED, false);
        }
    } else {
        if (c.ndim == 3) {
            if (full) MHDPIC_LAUNCH(3, MHDPIC_PREC_FP64, true);
            else MHDPIC_LAUNCH(3, MHDPIC_PREC_FP64, false);
        } else {
            if (full) MHDPIC_LAUNCH(2, MHDPIC_PREC_FP64, true);
            else MHDPIC_LAUNCH(2, MHDPIC_PREC_FP64, false);
        }
    }
#undef MHDPIC_LAUNCH
    return 1;
}

}  // namespace mhdpic
