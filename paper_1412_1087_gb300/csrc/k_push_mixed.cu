// Mixed-precision particle step: int32 cell + f32 offset positions, f32
// Boris push, fixed-point deposits (App. A.1-A.3 of arXiv:1412.1087).
//
// A persistent CTA of 8 warps takes brick items from an atomic counter.  Per
// item it stages the brick's E, B plus a halo of HALO cells in shared memory
// and accumulates both deposits in a shared int32 fixed-point tile, which is
// shifted exactly into the int64 global accumulators at the end.
//
//  * Lane <-> cell: a 64-cell brick is two 32-cell halves; warps 0-3 work on
//    one half and warps 4-7 on the other, and lane l works through the
//    particles of the l-th cell of its half, so the 32 lanes of an instruction
//    sit in 32 different cells.  The tile strides are padded (3-D: y 12, z 112
//    slots; 2-D: y 24) so those 32 cells fall on 32 different banks for the
//    32-bit deposit atomics and on distinct bank groups for the 128-bit and
//    64-bit field loads.
//  * Fixed point: the tile scale of each channel is a power of two chosen per
//    item so that no tile cell can overflow int32 whatever the particles do
//    (item size x largest single-cell TSC weight x the channel's per-particle
//    bound < 2^31), and every contribution stays below 2^21 so one FFMA with
//    1.5*2^23 rounds it to an integer.  The tile scale divides the global
//    int64 scale by 2^k; the flush shifts by k, so the sums remain exact and
//    independent of the order of the additions.
//  * A particle whose stencil leaves the tile, or whose quantities exceed the
//    bound the scales were sized for, deposits straight into the int64 global
//    accumulators at the global scale.
#include "push_common.cuh"

namespace mhdpic {

namespace {

constexpr float MAGIC = 12582912.0f;  // 1.5 * 2^23: x + MAGIC has unit spacing for |x| < 2^22
constexpr int MAGIC_BITS = 0x4B400000;

// round(a * b) to the nearest integer (ties to even), for |a * b| < 2^22
__device__ __forceinline__ int round_fma(float a, float b)
{
    return __float_as_int(fmaf(a, b, MAGIC)) - MAGIC_BITS;
}

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
    float cap = fminf(2097152.f, 2147483648.f / ((float)cnt * wmax + 1.f));
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
        float Q = fmaxf((float)b.qbound[ch], 1e-30f);
        int eg = b.escale[ch];
        int et = ilogbf(cap / Q);     // 2^et * Q <= cap
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
__device__ __forceinline__ void gather_tile(const Ctx &c, int base, const float wx[3], const float wy[3],
                                            const float wz[3], const float4 *__restrict__ sFa,
                                            const float2 *__restrict__ sFb, float E[3], float Bf[3])
{
    E[0] = E[1] = E[2] = Bf[0] = Bf[1] = Bf[2] = 0.f;
    const int SY = c.ts[1], SZ = c.ts[2];
#pragma unroll
    for (int cz = 0; cz < (D == 3 ? 3 : 1); ++cz)
#pragma unroll
        for (int cy = 0; cy < 3; ++cy) {
            float wyz = D == 3 ? wy[cy] * wz[cz] : wy[cy];
#pragma unroll
            for (int cx = 0; cx < 3; ++cx) {
                float w = wx[cx] * wyz;
                int s = base + cx + SY * cy + SZ * cz;
                float4 a = sFa[s];
                float2 bb = sFb[s];
                E[0] = fmaf(w, a.x, E[0]);
                E[1] = fmaf(w, a.y, E[1]);
                E[2] = fmaf(w, a.z, E[2]);
                Bf[0] = fmaf(w, a.w, Bf[0]);
                Bf[1] = fmaf(w, bb.x, Bf[1]);
                Bf[2] = fmaf(w, bb.y, Bf[2]);
            }
        }
}

template <int D>
__device__ __noinline__ void gather_global(const Ctx &c, const BoxDev &b, const int ci[3], const float wx[3],
                                           const float wy[3], const float wz[3], float E[3], float Bf[3])
{
    E[0] = E[1] = E[2] = Bf[0] = Bf[1] = Bf[2] = 0.f;
    const float4 *__restrict__ gF = reinterpret_cast<const float4 *>(c.f32);
    int gx[3], gy[3], gz[3];
    stencil_coords<D>(b, ci, gx, gy, gz);
    for (int cz = 0; cz < (D == 3 ? 3 : 1); ++cz)
        for (int cy = 0; cy < 3; ++cy) {
            float wyz = D == 3 ? wy[cy] * wz[cz] : wy[cy];
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

// Four channels into the int32 tile; q already carries the tile scale.
template <int D>
__device__ __forceinline__ void deposit_tile(const Ctx &c, int base, const float wx[3], const float wy[3],
                                             const float wz[3], const float q[4], int *__restrict__ s0)
{
    const int S = c.tile_slots, SY = c.ts[1], SZ = c.ts[2];
    int *__restrict__ s1 = s0 + S;
    int *__restrict__ s2 = s0 + 2 * S;
    int *__restrict__ s3 = s0 + 3 * S;
#pragma unroll
    for (int cz = 0; cz < (D == 3 ? 3 : 1); ++cz)
#pragma unroll
        for (int cy = 0; cy < 3; ++cy) {
            float wyz = D == 3 ? wy[cy] * wz[cz] : wy[cy];
            float a0 = q[0] * wyz, a1 = q[1] * wyz, a2 = q[2] * wyz, a3 = q[3] * wyz;
#pragma unroll
            for (int cx = 0; cx < 3; ++cx) {
                int s = base + cx + SY * cy + SZ * cz;
                atomicAdd(s0 + s, round_fma(a0, wx[cx]));
                atomicAdd(s1 + s, round_fma(a1, wx[cx]));
                atomicAdd(s2 + s, round_fma(a2, wx[cx]));
                atomicAdd(s3 + s, round_fma(a3, wx[cx]));
            }
        }
}

// Four channels straight into the int64 global accumulators; q carries the
// global scale.
template <int D>
__device__ __noinline__ void deposit_global(const Ctx &c, const BoxDev &b, const int ci[3], const float wx[3],
                                            const float wy[3], const float wz[3], const float q[4],
                                            unsigned long long *__restrict__ g0)
{
    const int64_t nc = c.nc;
    int gx[3], gy[3], gz[3];
    stencil_coords<D>(b, ci, gx, gy, gz);
    for (int cz = 0; cz < (D == 3 ? 3 : 1); ++cz)
        for (int cy = 0; cy < 3; ++cy) {
            float wyz = D == 3 ? wy[cy] * wz[cz] : wy[cy];
            for (int cx = 0; cx < 3; ++cx) {
                float w = wx[cx] * wyz;
                int64_t g = b.cell0 + ((int64_t)gz[cz] * b.n[1] + gy[cy]) * b.n[0] + gx[cx];
                for (int k = 0; k < 4; ++k)
                    red_add(g0 + k * nc + g, __float2ll_rn(q[k] * w));
            }
        }
}

template <int D>
__device__ __forceinline__ bool within(const float q[4], const float *qb, int ch0)
{
    return fabsf(q[0]) <= qb[ch0] && fabsf(q[1]) <= qb[ch0 + 1] && fabsf(q[2]) <= qb[ch0 + 2] &&
           fabsf(q[3]) <= qb[ch0 + 3];
}

template <int D, bool FULL>
__device__ __forceinline__ float push_one(const Ctx &c, const BoxDev &b, const ItemGeom &gm, const MixedConst &k,
                                          int64_t j, const float4 *sFa, const float2 *sFb, int *sD,
                                          unsigned long long *mout)
{
    const int64_t np = c.np;
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

    float w[3][3] = {{0.f, 1.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 1.f, 0.f}};
    int rel[3] = {0, 0, 0};
    bool in_tile = true;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        tsc_from_offset<float>(o[d], w[d]);
        in_tile &= tile_rel(c, b, gm, d, ci[d], rel[d]);
    }
    const int base = (rel[0] - 1) + c.ts[1] * (rel[1] - 1) + (D == 3 ? c.ts[2] * (rel[2] - 1) : 0);

    float E[3], Bf[3];
    if (in_tile)
        gather_tile<D>(c, base, w[0], w[1], w[2], sFa, sFb, E, Bf);
    else
        gather_global<D>(c, b, ci, w[0], w[1], w[2], E, Bf);

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
    const float ig1 = rsqrtf(fmaf(v00 * v00 + v01 * v01 + v02 * v02, k.invC2, 1.f));
    const float hb = k.hh * ig1;
    const float b0 = hb * Bf[0], b1 = hb * Bf[1], b2 = hb * Bf[2];
    const float t0 = v00 + (v01 * b2 - v02 * b1), t1 = v01 + (v02 * b0 - v00 * b2),
                t2 = v02 + (v00 * b1 - v01 * b0);
    const float s2 = 2.f / (1.f + b0 * b0 + b1 * b1 + b2 * b2);
    const float r0 = s2 * (t1 * b2 - t2 * b1), r1 = s2 * (t2 * b0 - t0 * b2), r2 = s2 * (t0 * b1 - t1 * b0);
    const float v10 = v00 + r0, v11 = v01 + r1, v12 = v02 + r2;
    float vn[3] = {v10 + e0, v11 + e1, v12 + e2};

    // dv = h E + rot without cancellation; the rotation keeps |v|, so dE_k is
    // the change of the two half kicks, E_k(a) - E_k(b) = (a-b).(a+b)/(ga+gb)
    const float ig2 = rsqrtf(fmaf(vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2], k.invC2, 1.f));
    const float gn = 1.f / ign, g1 = 1.f / ig1, g2 = 1.f / ig2;
    const float dEk = (e0 * (vn[0] + v10) + e1 * (vn[1] + v11) + e2 * (vn[2] + v12)) / (g2 + g1) +
                      (e0 * (v00 + v[0]) + e1 * (v01 + v[1]) + e2 * (v02 + v[2])) / (g1 + gn);
    {
        const float qc[4] = {-k.m * (2.f * e0 + r0), -k.m * (2.f * e1 + r1), -k.m * (2.f * e2 + r2), -k.m * dEk};
        if (in_tile && within<D>(qc, k.qb, CH_MX)) {
            const float qs[4] = {qc[0] * k.st[0], qc[1] * k.st[1], qc[2] * k.st[2], qc[3] * k.st[3]};
            deposit_tile<D>(c, base, w[0], w[1], w[2], qs, sD);
        } else {
            const float qg[4] = {qc[0] * k.gs[0], qc[1] * k.gs[1], qc[2] * k.gs[2], qc[3] * k.gs[3]};
            deposit_global<D>(c, b, ci, w[0], w[1], w[2], qg, c.corr);
        }
    }

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
        const float qj = k.qn * ig2;
        const float qm[4] = {k.qn, qj * vn[0], qj * vn[1], qj * vn[2]};
        if (in2 && within<D>(qm, k.qb, CH_N)) {
            const int base2 = (rel2[0] - 1) + c.ts[1] * (rel2[1] - 1) + (D == 3 ? c.ts[2] * (rel2[2] - 1) : 0);
            const float qs[4] = {qm[0] * k.st[4], qm[1] * k.st[5], qm[2] * k.st[6], qm[3] * k.st[7]};
            deposit_tile<D>(c, base2, w2[0], w2[1], w2[2], qs, sD + CH_N * c.tile_slots);
        } else {
            const float qg[4] = {qm[0] * k.gs[4], qm[1] * k.gs[5], qm[2] * k.gs[6], qm[3] * k.gs[7]};
            deposit_global<D>(c, b, ci, w2[0], w2[1], w2[2], qg, mout);
        }
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

template <int D, bool FULL>
__global__ void __launch_bounds__(PUSH_THREADS, 2) k_push_mixed(Ctx c, const WorkItem *__restrict__ items,
                                                                 const int32_t *__restrict__ nitems,
                                                                 int32_t *__restrict__ work_ctr, int cur_out,
                                                                 float dt)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int S = c.tile_slots;
    int *sD = reinterpret_cast<int *>(smem);
    float4 *sFa = reinterpret_cast<float4 *>(smem + sizeof(int) * NCH * S);
    float2 *sFb = reinterpret_cast<float2 *>(smem + (sizeof(int) * NCH + sizeof(float4)) * S);
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

        // clear the deposit tile and stage the fields
        for (int s = threadIdx.x; s < NCH * S; s += PUSH_THREADS)
            sD[s] = 0;
        const float4 *gF = reinterpret_cast<const float4 *>(c.f32);
        for (int t = threadIdx.x; t < c.tile_vol; t += PUSH_THREADS) {
            int tx = t % c.tile[0], r = t / c.tile[0];
            int ty = r % c.tile[1], tz = r / c.tile[1];
            int64_t g = tile_global(c, b, gm, tx, ty, tz, D);
            int s = tile_slot(c, tx, ty, tz);
            float4 f1 = __ldg(gF + 2 * g), f2 = __ldg(gF + 2 * g + 1);
            sFa[s] = f1;
            sFb[s] = make_float2(f2.x, f2.y);
        }
        MixedConst k;
        item_const(b, dt, it.p1 - it.p0, D, k);
        __syncthreads();

        const LaneRange lr = lane_range(it, wid, NW);
        float vm2 = 0.f;
        for (int64_t r = lr.first; r < lr.q; r += lr.stride) {
            int64_t loc = lane * lr.q + r;
            if (loc < lr.cnt)
                vm2 = fmaxf(vm2, push_one<D, FULL>(c, b, gm, k, lr.base + loc, sFa, sFb, sD, mout));
        }
        unsigned vb = __reduce_max_sync(0xffffffffu, __float_as_uint(sqrtf(vm2)));
        if (lane == 0 && vb)
            atomicMax(&c.stats[it.box].vmax, vb);
        __syncthreads();

        // shift the tile into the global int64 accumulators
        for (int t = threadIdx.x; t < c.tile_vol; t += PUSH_THREADS) {
            int tx = t % c.tile[0], r = t / c.tile[0];
            int ty = r % c.tile[1], tz = r / c.tile[1];
            int64_t g = tile_global(c, b, gm, tx, ty, tz, D);
            int s = tile_slot(c, tx, ty, tz);
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
                int a = sD[ch * S + s];
                if (a)
                    atomicAdd(c.corr + ch * c.nc + g, (unsigned long long)(long long)a << k.ksh[ch]);
            }
            if (FULL) {
#pragma unroll
                for (int ch = 0; ch < 4; ++ch) {
                    int a = sD[(CH_N + ch) * S + s];
                    if (a)
                        atomicAdd(mout + ch * c.nc + g, (unsigned long long)(long long)a << k.ksh[CH_N + ch]);
                }
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

}  // namespace

size_t push_smem_bytes_mixed(const Ctx &c)
{
    return (sizeof(int) * NCH + sizeof(float4) + sizeof(float2)) * (size_t)c.tile_slots;
}

int push_blocks_per_sm_mixed(const Ctx &c)
{
    size_t bytes = push_smem_bytes_mixed(c);
    occupancy_mixed<3, false>(bytes);
    occupancy_mixed<2, false>(bytes);
    occupancy_mixed<3, true>(bytes);
    occupancy_mixed<2, true>(bytes);
    int nb = c.ndim == 3 ? occupancy_mixed<3, true>(bytes) : occupancy_mixed<2, true>(bytes);
    return nb < 1 ? 1 : nb;
}

int launch_push_mixed(const Ctx &c, const SortScratch &s, int32_t *work_ctr, int cur_out, int full, double dt,
                      int grid_blocks, cudaStream_t st)
{
    size_t bytes = push_smem_bytes_mixed(c);
    cudaMemsetAsync(work_ctr, 0, sizeof(int32_t), st);
    float fdt = (float)dt;
    if (c.ndim == 3) {
        if (full)
            k_push_mixed<3, true><<<grid_blocks, PUSH_THREADS, bytes, st>>>(c, s.items, s.nitems, work_ctr, cur_out, fdt);
        else
            k_push_mixed<3, false><<<grid_blocks, PUSH_THREADS, bytes, st>>>(c, s.items, s.nitems, work_ctr, cur_out, fdt);
    } else {
        if (full)
            k_push_mixed<2, true><<<grid_blocks, PUSH_THREADS, bytes, st>>>(c, s.items, s.nitems, work_ctr, cur_out, fdt);
        else
            k_push_mixed<2, false><<<grid_blocks, PUSH_THREADS, bytes, st>>>(c, s.items, s.nitems, work_ctr, cur_out, fdt);
    }
    return 1;
}

}  // namespace mhdpic
