// Helpers shared by the mixed-precision and FP64 push kernels: tile geometry
// of a work item and the particle boundary in both position representations.
#pragma once

#include "device_common.cuh"

namespace mhdpic {

// Early-particle removal (Sec. 4.1): a particle injected at t_i < t_early
// is removed at t = 2 t_i, i.e. at the end of the first step whose end time
// (clock[0], already advanced) reaches 2 t_i.  It has taken part in that
// step (its corrector deposit stands) and, like a particle that left through
// an open face, deposits no moments at the new position.
__device__ __forceinline__ bool removed_early(const Ctx &c, int64_t j)
{
    if (!c.tinj)
        return false;
    const double ti = c.tinj[j];
    return ti < c.clock[1] && c.clock[0] >= 2.0 * ti;
}

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
#pragma unroll
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
// brick centre).  True when the whole 3-point stencil is inside the tile.
__device__ __forceinline__ bool tile_rel(const Ctx &c, const BoxDev &b, const ItemGeom &g, int d, int ci,
                                         int &rel)
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

// Slot of tile cell (tx, ty, tz) and the global cell it maps to.
__device__ __forceinline__ int tile_slot(const Ctx &c, int tx, int ty, int tz)
{
    return tx + c.ts[1] * ty + c.ts[2] * tz;
}

__device__ __forceinline__ int64_t tile_global(const Ctx &c, const BoxDev &b, const ItemGeom &gm, int tx,
                                               int ty, int tz, int D)
{
    int gx = map_coord(gm.org[0] + tx, b.n[0], b.bc[0]);
    int gy = map_coord(gm.org[1] + ty, b.n[1], b.bc[1]);
    int gz = D == 3 ? map_coord(gm.org[2] + tz, b.n[2], b.bc[2]) : 0;
    return b.cell0 + ((int64_t)gz * b.n[1] + gy) * b.n[0] + gx;
}

// Mixed representation: move the offset back into [0,1), carrying whole
// cells, then apply the particle boundary (periodic wrap, or specular
// reflection, which flips v[d]).  At an open face the particle is held just
// inside it and the call returns true (the particle is leaving the box).
__device__ __forceinline__ bool renorm_mixed(const BoxDev &b, int d, int &ci, float &o, float &vd,
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
        return false;
    if (b.bc[d] == MHDPIC_BC_PERIODIC) {
        ci = map_coord(ci, n, MHDPIC_BC_PERIODIC);
        return false;
    }
    if (b.bc[d] == MHDPIC_BC_WALL_OPEN && ci >= n) {
        ci = n - 1;
        o = 0x1.fffffep-1f;
        return true;
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
    return false;
}

// FP64 representation: the oracle's boundary rule on absolute positions;
// true when the particle reached an open face (it is held just inside).
__device__ __forceinline__ bool boundary_f64(const BoxDev &b, int d, double &x, double &vd)
{
    double lo = b.x0[d];
    double L = b.n[d] * b.dx[d];
    double hi = lo + L;
    if (b.bc[d] == MHDPIC_BC_WALL_OPEN && x >= hi) {
        x = nextafter(hi, lo);
        return true;
    }
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
    return false;
}

// Neighbour cells of a stencil along each dimension (global path).
template <int D>
__device__ __forceinline__ void stencil_coords(const BoxDev &b, const int ci[3], int gx[3], int gy[3], int gz[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        gx[a] = map_coord(ci[0] + a - 1, b.n[0], b.bc[0]);
        gy[a] = map_coord(ci[1] + a - 1, b.n[1], b.bc[1]);
        gz[a] = D == 3 ? map_coord(ci[2] + a - 1, b.n[2], b.bc[2]) : 0;
    }
}

// Split of an item's particles over the block's warps: with halves, warps
// 0..NW/2-1 take [p0, pm) and the rest [pm, p1); lane l works through the
// l-th 1/32 of its range, the warps of a group interleaving inside it.  The
// range's k-th particle sits at position base + k * step (k * step stays
// below 2^31: an item holds at most ITEM_MAX_PARTICLES).
struct LaneRange {
    int64_t base, cnt, q;
    int32_t step;
    int first, stride;
};

__device__ __forceinline__ LaneRange lane_range(const WorkItem &it, int wid, int nw)
{
    LaneRange r;
    if (it.pm >= 0) {
        int half = nw / 2;
        bool hi = wid >= half;
        r.base = hi ? it.pm : it.p0;
        r.cnt = hi ? it.p1 - it.pm : it.pm - it.p0;
        r.first = hi ? wid - half : wid;
        r.stride = half;
        r.step = 1;
    } else {
        r.base = it.p0;
        r.step = it.step;
        r.cnt = it.count;
        r.first = wid;
        r.stride = nw;
    }
    r.q = (r.cnt + 31) / 32;
    return r;
}

}  // namespace mhdpic
