// Plain FP64 particle step (the reference GPU path): drift, TSC gather,
// E-parallel cleaning, relativistic Boris kick-rotate-kick, drift, corrector
// deposit at x^(n+1/2) and moments deposit at x^(n+1) (App. A.1-A.3 of
// arXiv:1412.1087), in the oracle's arithmetic order.
//
// Same work decomposition as the mixed kernel (k_push_mixed.cu): persistent
// CTAs take brick items from an atomic counter, stage the brick's fields plus
// a halo in shared memory and accumulate the deposits in a shared int64
// fixed-point tile that is added to the global accumulators at the end; a
// particle whose stencil leaves the tile uses global memory directly.
#include "push_common.cuh"

namespace mhdpic {

namespace {

struct F64Const {
    double dt, h, C, m, qn;
    double scale[NCH];
    double vlim[NCH];
};

template <int D>
__device__ __forceinline__ void gather_f64(const Ctx &c, const BoxDev &b, bool in_tile, const int rel[3],
                                           const int ci[3], const double wx[3], const double wy[3],
                                           const double wz[3], const double2 *__restrict__ sF,
                                           double E[3], double Bf[3])
{
    E[0] = E[1] = E[2] = Bf[0] = Bf[1] = Bf[2] = 0.0;
    const double2 *__restrict__ gF = reinterpret_cast<const double2 *>(c.f64);
    int gx[3], gy[3], gz[3];
    stencil_coords<D>(b, ci, gx, gy, gz);
    int base = (rel[0] - 1) + c.ts[1] * (rel[1] - 1) + c.ts[2] * (D == 3 ? rel[2] - 1 : 0);
    for (int cz = 0; cz < (D == 3 ? 3 : 1); ++cz)
        for (int cy = 0; cy < 3; ++cy)
            for (int cx = 0; cx < 3; ++cx) {
                double w = wx[cx] * wy[cy] * (D == 3 ? wz[cz] : 1.0);
                double2 a0, a1, a2;
                if (in_tile) {
                    int s = base + cx + c.ts[1] * cy + c.ts[2] * cz;
                    a0 = sF[3 * s];
                    a1 = sF[3 * s + 1];
                    a2 = sF[3 * s + 2];
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

// Deposit 4 pre-scaled quantities (channels ch0..ch0+3) with TSC weights.
template <int D>
__device__ __forceinline__ void deposit4_f64(const Ctx &c, const BoxDev &b, bool in_tile, const int rel[3],
                                             const int ci[3], const double wx[3], const double wy[3],
                                             const double wz[3], const double q[4], int ch0,
                                             unsigned long long *__restrict__ sD,
                                             unsigned long long *__restrict__ gdst)
{
    const int S = c.tile_slots;
    const int64_t nc = c.nc;
    int gx[3], gy[3], gz[3];
    stencil_coords<D>(b, ci, gx, gy, gz);
    int base = (rel[0] - 1) + c.ts[1] * (rel[1] - 1) + c.ts[2] * (D == 3 ? rel[2] - 1 : 0);
    for (int cz = 0; cz < (D == 3 ? 3 : 1); ++cz)
        for (int cy = 0; cy < 3; ++cy)
            for (int cx = 0; cx < 3; ++cx) {
                double w = wx[cx] * wy[cy] * (D == 3 ? wz[cz] : 1.0);
                if (in_tile) {
                    int s = base + cx + c.ts[1] * cy + c.ts[2] * cz;
                    for (int k = 0; k < 4; ++k)
                        red_add(sD + (ch0 + k) * S + s, to_fixed(q[k] * w));
                } else {
                    int64_t g = b.cell0 + ((int64_t)gz[cz] * b.n[1] + gy[cy]) * b.n[0] + gx[cx];
                    for (int k = 0; k < 4; ++k)
                        red_add(gdst + k * nc + g, to_fixed(q[k] * w));
                }
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
    const int64_t np = c.np;
    const double C = k.C;
    const int64_t src = c.perm_src ? (int64_t)c.perm_src[j] : j;
    double x[3] = {0.0, 0.0, 0.0}, v[3];
    for (int d = 0; d < D; ++d)
        x[d] = c.src_x[d * np + src];
    for (int d = 0; d < 3; ++d)
        v[d] = c.src_p64[d * np + src];
    if (isnan(x[0])) {   // left the box earlier (kept until the next sort)
        for (int d = 0; d < D; ++d)
            c.x[d * np + j] = x[d];
        for (int d = 0; d < 3; ++d)
            c.p64[d * np + j] = 0.0;
        return 0.f;
    }

    // a particle at an open face is held just inside it, deposits its
    // corrector and then leaves
    double g0 = sqrt(C * C + (v[0] * v[0] + v[1] * v[1] + v[2] * v[2])) / C;
    bool leaving = false;
    for (int d = 0; d < D; ++d) {
        x[d] = x[d] + 0.5 * k.dt * (v[d] / g0);
        leaving |= boundary_f64(b, d, x[d], v[d]);
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

    // dE_k: the rotation keeps |v|, so the energy change is that of the two
    // half kicks, E_k(a) - E_k(b) = (a-b).(a+b)/(gamma_a+gamma_b), a-b = (h/2)E
    double g1 = sqrt(C * C + (vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2])) / C;
    double dv[3], e[3], s1[3], s0[3];
    for (int d = 0; d < 3; ++d) {
        dv[d] = vn[d] - v[d];
        e[d] = 0.5 * h * E[d];
        s1[d] = vn[d] + v1[d];
        s0[d] = v0[d] + v[d];
    }
    double dEk = (e[0] * s1[0] + e[1] * s1[1] + e[2] * s1[2]) / (g1 + gam) +
                 (e[0] * s0[0] + e[1] * s0[1] + e[2] * s0[2]) / (gam + g0);
    double qc[4] = {-k.m * dv[0] * k.scale[CH_MX], -k.m * dv[1] * k.scale[CH_MY],
                    -k.m * dv[2] * k.scale[CH_MZ], -k.m * dEk * k.scale[CH_E]};
    if (fabs(qc[0]) > k.vlim[CH_MX] || fabs(qc[1]) > k.vlim[CH_MY] || fabs(qc[2]) > k.vlim[CH_MZ] ||
        fabs(qc[3]) > k.vlim[CH_E])
        set_status(c.status, MHDPIC_ST_OVERFLOW);
    deposit4_f64<D>(c, b, in_tile, rel, ci, w[0], w[1], w[2], qc, CH_MX, sD, c.corr);

    for (int d = 0; d < D; ++d) {
        x[d] = x[d] + 0.5 * k.dt * (vn[d] / g1);
        leaving |= boundary_f64(b, d, x[d], vn[d]);
    }
    leaving |= removed_early(c, j);
    if (leaving) {   // removed: no moments deposit; the next sort drops it
        c.x[j] = __longlong_as_double(0x7ff8000000000000ll);
        for (int d = 1; d < D; ++d)
            c.x[d * np + j] = x[d];
        for (int d = 0; d < 3; ++d)
            c.p64[d * np + j] = 0.0;
        return 0.f;
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
        deposit4_f64<D>(c, b, in2, rel2, ci2, w2[0], w2[1], w2[2], qm, CH_N, sD, mout);
    }
    if (!isfinite(vn[0] + vn[1] + vn[2]))
        set_status(c.status, MHDPIC_ST_NONFINITE);
    for (int d = 0; d < D; ++d)
        c.x[d * np + j] = x[d];
    for (int d = 0; d < 3; ++d)
        c.p64[d * np + j] = vn[d];
    return (float)(vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2]);
}

template <int D, bool FULL>
__global__ void __launch_bounds__(PUSH_THREADS) k_push_f64(Ctx c, const WorkItem *__restrict__ items,
                                                          const int32_t *__restrict__ nitems,
                                                          int32_t *__restrict__ work_ctr, int cur_out,
                                                          double dt)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int S = c.tile_slots;
    unsigned long long *sD = reinterpret_cast<unsigned long long *>(smem);
    double2 *sF = reinterpret_cast<double2 *>(smem + sizeof(unsigned long long) * NCH * S);
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

        for (int s = threadIdx.x; s < NCH * S; s += PUSH_THREADS)
            sD[s] = 0ull;
        const double2 *gF = reinterpret_cast<const double2 *>(c.f64);
        for (int t = threadIdx.x; t < c.tile_vol; t += PUSH_THREADS) {
            int tx = t % c.tile[0], r = t / c.tile[0];
            int ty = r % c.tile[1], tz = r / c.tile[1];
            int64_t g = tile_global(c, b, gm, tx, ty, tz, D);
            int s = tile_slot(c, tx, ty, tz);
            sF[3 * s] = __ldg(gF + 3 * g);
            sF[3 * s + 1] = __ldg(gF + 3 * g + 1);
            sF[3 * s + 2] = __ldg(gF + 3 * g + 2);
        }
        __syncthreads();

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
        const LaneRange lr = lane_range(it, wid, NW);
        float vm2 = 0.f;
        for (int64_t r = lr.first; r < lr.q; r += lr.stride) {
            int64_t loc = lane * lr.q + r;
            if (loc < lr.cnt)
                vm2 = fmaxf(vm2, push_one_f64<D, FULL>(c, b, gm, k, lr.base + (int32_t)loc * lr.step, sF, sD, mout));
        }
        unsigned vb = __reduce_max_sync(0xffffffffu, __float_as_uint(sqrtf(vm2)));
        if (lane == 0 && vb)
            atomicMax(&c.stats[it.box].vmax, vb);
        __syncthreads();

        for (int t = threadIdx.x; t < c.tile_vol; t += PUSH_THREADS) {
            int tx = t % c.tile[0], r = t / c.tile[0];
            int ty = r % c.tile[1], tz = r / c.tile[1];
            int64_t g = tile_global(c, b, gm, tx, ty, tz, D);
            int s = tile_slot(c, tx, ty, tz);
            for (int ch = 0; ch < 4; ++ch) {
                unsigned long long a = sD[ch * S + s];
                if (a)
                    atomicAdd(c.corr + ch * c.nc + g, a);
            }
            if (FULL)
                for (int ch = 0; ch < 4; ++ch) {
                    unsigned long long a = sD[(CH_N + ch) * S + s];
                    if (a)
                        atomicAdd(mout + ch * c.nc + g, a);
                }
        }
        __syncthreads();
    }
}

constexpr int PUSH_SMEM_LIMIT = 200 * 1024;

template <int D, bool FULL>
int occupancy_f64(size_t bytes)
{
    cudaFuncSetAttribute(k_push_f64<D, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, PUSH_SMEM_LIMIT);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push_f64<D, FULL>, PUSH_THREADS, bytes);
    return nb;
}

}  // namespace

size_t push_smem_bytes_f64(const Ctx &c)
{
    return (sizeof(unsigned long long) * NCH + 48) * (size_t)c.tile_slots;
}

int push_blocks_per_sm_f64(const Ctx &c)
{
    size_t bytes = push_smem_bytes_f64(c);
    occupancy_f64<3, false>(bytes);
    occupancy_f64<2, false>(bytes);
    occupancy_f64<3, true>(bytes);
    occupancy_f64<2, true>(bytes);
    int nb = c.ndim == 3 ? occupancy_f64<3, true>(bytes) : occupancy_f64<2, true>(bytes);
    return nb < 1 ? 1 : nb;
}

int launch_push_f64(const Ctx &c, const SortScratch &s, int32_t *work_ctr, int cur_out, int full, double dt,
                    int grid_blocks, cudaStream_t st)
{
    size_t bytes = push_smem_bytes_f64(c);
    cudaMemsetAsync(work_ctr, 0, sizeof(int32_t), st);
    if (c.ndim == 3) {
        if (full)
            k_push_f64<3, true><<<grid_blocks, PUSH_THREADS, bytes, st>>>(c, s.items, s.nitems, work_ctr, cur_out, dt);
        else
            k_push_f64<3, false><<<grid_blocks, PUSH_THREADS, bytes, st>>>(c, s.items, s.nitems, work_ctr, cur_out, dt);
    } else {
        if (full)
            k_push_f64<2, true><<<grid_blocks, PUSH_THREADS, bytes, st>>>(c, s.items, s.nitems, work_ctr, cur_out, dt);
        else
            k_push_f64<2, false><<<grid_blocks, PUSH_THREADS, bytes, st>>>(c, s.items, s.nitems, work_ctr, cur_out, dt);
    }
    return 1;
}

}  // namespace mhdpic
