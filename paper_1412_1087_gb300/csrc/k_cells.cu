// Per-cell kernels: feedback to the gas fused with the staging of the
// cell-centred fields; the standalone charge/current deposit; FP64 totals;
// read-back conversions.
#include "cells_common.cuh"

namespace mhdpic {

namespace {

// One pass over the cells of all boxes (prep_cells).
template <int PREC>
__global__ void k_prep(Ctx c, int cur, int apply)
{
    prep_cells<PREC>(c, cur, apply);
}

__global__ void k_scales(Ctx c, double dt)
{
    int bx = blockIdx.x * blockDim.x + threadIdx.x;
    if (bx < c.nbox)
        scales_box(c, bx, dt);
}
// Charge and current densities at the current positions (App. A.1, eq:nJCR):
// n = qm m W / dV, J = qm m u W / dV, straight into the global accumulators.
template <int PREC, int D>
__global__ void k_moments(Ctx c, int cur)
{
    unsigned long long *__restrict__ md = c.momdep[cur];
    const int64_t nc = c.nc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.np;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (particle_dead<PREC>(c, i))   // left the box
            continue;
        int bx = find_box(c.box_part_start, c.nbox, i);
        const BoxDev &b = c.boxes[bx];
        int ci[3] = {0, 0, 0};
        double w[3][3] = {{0, 1, 0}, {0, 1, 0}, {0, 1, 0}};
        double v[3];
        if (PREC == MHDPIC_PREC_MIXED) {
            const int4 ps = c.pos[i];
            const float4 vs = c.vel[i];
            const float o[3] = {__int_as_float(ps.y), __int_as_float(ps.z), __int_as_float(ps.w)};
            decode_cell(b, ps.x, ci);
            for (int d = 0; d < D; ++d)
                tsc_from_offset<double>((double)o[d], w[d]);
            for (int d = 0; d < 3; ++d)
                v[d] = vel_f64(vs, d);
        } else {
            for (int d = 0; d < D; ++d) {
                double s = (c.x[(int64_t)d * c.np + i] - b.x0[d]) * b.inv_dx[d];
                double f = floor(s);
                ci[d] = (int)f;
                tsc_from_offset<double>(s - f, w[d]);
            }
            for (int d = 0; d < 3; ++d)
                v[d] = c.p64[(int64_t)d * c.np + i];
        }
        double C = b.C;
        double gam = sqrt(C * C + v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / C;
        double q[4];
        q[0] = b.qm_cr * b.m_cr * b.inv_dV;
        for (int d = 0; d < 3; ++d)
            q[1 + d] = q[0] * (v[d] / gam);
        for (int k = 0; k < 4; ++k)
            q[k] *= b.scale[CH_N + k];
        int gx[3], gy[3], gz[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a) {
            gx[a] = map_coord(ci[0] + a - 1, b.n[0], b.bc[0]);
            gy[a] = map_coord(ci[1] + a - 1, b.n[1], b.bc[1]);
            if (D == 3)
                gz[a] = map_coord(ci[2] + a - 1, b.n[2], b.bc[2]);
        }
        for (int cz = 0; cz < (D == 3 ? 3 : 1); ++cz)
            for (int cy = 0; cy < 3; ++cy)
                for (int cxx = 0; cxx < 3; ++cxx) {
                    double ww = w[0][cxx] * w[1][cy] * (D == 3 ? w[2][cz] : 1.0);
                    int64_t gc = b.cell0 + ((int64_t)gz[cz] * b.n[1] + gy[cy]) * b.n[0] + gx[cxx];
                    for (int k = 0; k < 4; ++k)
                        red_add(md + k * nc + gc, to_fixed(q[k] * ww));
                }
    }
}

// Deterministic FP64 totals per box: block (chunk, box) reduces a fixed slice
// of the box's cells and particles in a fixed order; a second kernel adds the
// chunks in order.  out per box: P_gas(3), E_gas, P_CR(3), E_CR.
template <int PREC>
__global__ void __launch_bounds__(256) k_totals_partial(Ctx c, int nchunks, int64_t per_chunk, double *partials)
{
    const int bx = blockIdx.y, chunk = blockIdx.x;
    const BoxDev &b = c.boxes[bx];
    const int64_t nc = c.nc;
    // each box takes as many of the nchunks slices as its size asks for;
    // the others add zeros
    const int nbc = box_chunks(b, per_chunk, nchunks);
    if (chunk >= nbc) {
        if (threadIdx.x < 8)
            partials[((int64_t)bx * nchunks + chunk) * 8 + threadIdx.x] = 0.0;
        return;
    }
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int64_t cs = (b.ncell + nbc - 1) / nbc;
    int64_t c0 = b.cell0 + chunk * cs, c1 = min(b.cell0 + b.ncell, c0 + cs);
    for (int64_t g = c0 + threadIdx.x; g < c1; g += blockDim.x) {
        for (int d = 0; d < 3; ++d)
            acc[d] += c.mom[d * nc + g] * b.dV;
        acc[3] += c.egas[g] * b.dV;
    }
    int64_t npb = b.part1 - b.part0;
    int64_t ps = (npb + nbc - 1) / nbc;
    int64_t p0 = b.part0 + chunk * ps, p1 = min(b.part1, p0 + ps);
    for (int64_t i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
        double v[3];
        if (PREC == MHDPIC_PREC_MIXED) {
            const float4 vs = c.vel[i];   // the exact value of the two-word four-velocity
            for (int d = 0; d < 3; ++d)
                v[d] = vel_f64(vs, d);
        } else {
            for (int d = 0; d < 3; ++d)
                v[d] = c.p64[(int64_t)d * c.np + i];
        }
        double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        double gam = sqrt(b.C * b.C + v2) / b.C;
        for (int d = 0; d < 3; ++d)
            acc[4 + d] += b.m_cr * v[d];
        acc[7] += b.m_cr * (v2 / (gam + 1.0));
    }
    __shared__ double red[8][256];
    for (int q = 0; q < 8; ++q)
        red[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int q = 0; q < 8; ++q)
                red[q][threadIdx.x] += red[q][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 8)
        partials[((int64_t)bx * nchunks + chunk) * 8 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void k_totals_final(int nbox, int nchunks, const double *partials, double *out)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nbox * 8)
        return;
    int bx = t / 8, q = t % 8;
    double s = 0.0;
    for (int k = 0; k < nchunks; ++k)
        s += partials[((int64_t)bx * nchunks + k) * 8 + q];
    out[t] = s;
}

__global__ void k_fixed_to_double(Ctx c, const unsigned long long *__restrict__ src, int ch0,
                                  double *__restrict__ out)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < c.nc;
         g += (int64_t)gridDim.x * blockDim.x) {
        const BoxDev &b = c.boxes[find_box(c.box_cell_start, c.nbox, g)];
        for (int q = 0; q < 4; ++q)
            out[q * c.nc + g] = from_fixed(src[q * c.nc + g], b.inv_scale[ch0 + q]);
    }
}

__global__ void k_fields_to_double(Ctx c, double *__restrict__ out)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < c.nc;
         g += (int64_t)gridDim.x * blockDim.x) {
        if (c.prec == MHDPIC_PREC_MIXED) {
            const int bx = find_box(c.box_cell_start, c.nbox, g);
            const BoxDev &b = c.boxes[bx];
            int ci[3];
            decode_cell(b, (int32_t)(g - b.cell0), ci);
            const int64_t f = fidx(b, ci[0], ci[1], ci[2]);
            const float4 a = c.fa[f];
            const float2 bb = c.fb[f];
            const float v[6] = {a.x, a.y, a.z, a.w, bb.x, bb.y};
            for (int q = 0; q < 6; ++q)
                out[q * c.nc + g] = (double)v[q];
        } else {
            for (int q = 0; q < 6; ++q)
                out[q * c.nc + g] = c.f64[g * 6 + q];
        }
    }
}

// The current four-velocities as double, plane-major: the exact value of each
// two-word record in mixed precision, a copy in FP64.
__global__ void k_velocities_to_double(Ctx c, double *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.np;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (c.prec == MHDPIC_PREC_MIXED) {
            const float4 vs = c.vel[i];
            for (int d = 0; d < 3; ++d)
                out[d * c.np + i] = vel_f64(vs, d);
        } else {
            for (int d = 0; d < 3; ++d)
                out[d * c.np + i] = c.p64[d * c.np + i];
        }
    }
}

// Largest |v| per box (for the fixed-point scales): a running maximum per
// thread while its particles stay in one box, one atomic per box and warp.
template <int PREC>
__global__ void k_vmax(Ctx c)
{
    float acc = 0.f;
    int bacc = -1;
    auto flush = [&](int bx, float vm) {
        const unsigned active = __activemask();
        const unsigned peers = __match_any_sync(active, bx);
        const unsigned m = __reduce_max_sync(peers, __float_as_uint(vm));
        if (bx >= 0 && m && (threadIdx.x & 31) == __ffs(peers) - 1)
            atomicMax(&c.stats[bx].vmax, m);
    };
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.np;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int bx = find_box(c.box_part_start, c.nbox, i);
        float vm;
        if (PREC == MHDPIC_PREC_MIXED) {
            const float4 vs = c.vel[i];
            const float v[3] = {vs.x, vs.y, vs.z};
            vm = sqrtf(vsq3(v));
        } else {
            double v2 = 0.0;
            for (int d = 0; d < 3; ++d) {
                const double v = c.p64[(int64_t)d * c.np + i];
                v2 += v * v;
            }
            vm = (float)sqrt(v2);
        }
        if (!(vm <= 1.0e37f))
            vm = 1.0e37f;
        if (bx != bacc) {   // rare: a thread's particles cross into the next box
            if (bacc >= 0 && acc > 0.f)
                atomicMax(&c.stats[bacc].vmax, __float_as_uint(acc));
            bacc = bx;
            acc = 0.f;
        }
        acc = fmaxf(acc, vm);
    }
    flush(bacc, acc);
}

int grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1)
        b = 1;
    if (b > 152 * 32)
        b = 152 * 32;
    return (int)b;
}

}  // namespace

int launch_prep(const Ctx &c, int cur, int apply, cudaStream_t st)
{
    if (c.prec == MHDPIC_PREC_MIXED)
        k_prep<MHDPIC_PREC_MIXED><<<grid_for(c.nc, 256), 256, 0, st>>>(c, cur, apply);
    else
        k_prep<MHDPIC_PREC_FP64><<<grid_for(c.nc, 256), 256, 0, st>>>(c, cur, apply);
    return 1;
}

int launch_moments(const Ctx &c, int cur, cudaStream_t st)
{
    cudaMemsetAsync(c.momdep[cur], 0, sizeof(unsigned long long) * 4 * c.nc, st);
    if (c.np == 0)
        return 0;
    int g = grid_for(c.np, 256);
    if (c.prec == MHDPIC_PREC_MIXED) {
        if (c.ndim == 3)
            k_moments<MHDPIC_PREC_MIXED, 3><<<g, 256, 0, st>>>(c, cur);
        else
            k_moments<MHDPIC_PREC_MIXED, 2><<<g, 256, 0, st>>>(c, cur);
    } else {
        if (c.ndim == 3)
            k_moments<MHDPIC_PREC_FP64, 3><<<g, 256, 0, st>>>(c, cur);
        else
            k_moments<MHDPIC_PREC_FP64, 2><<<g, 256, 0, st>>>(c, cur);
    }
    return 1;
}

int launch_totals(const Ctx &c, double *partials, int nchunks, int64_t per_chunk, double *out, cudaStream_t st)
{
    dim3 grid(nchunks, c.nbox);
    if (c.prec == MHDPIC_PREC_MIXED)
        k_totals_partial<MHDPIC_PREC_MIXED><<<grid, 256, 0, st>>>(c, nchunks, per_chunk, partials);
    else
        k_totals_partial<MHDPIC_PREC_FP64><<<grid, 256, 0, st>>>(c, nchunks, per_chunk, partials);
    k_totals_final<<<(c.nbox * 8 + 255) / 256, 256, 0, st>>>(c.nbox, nchunks, partials, out);
    return 2;
}

int launch_fixed_to_double(const Ctx &c, const unsigned long long *src, int ch0, double *out,
                           cudaStream_t st)
{
    k_fixed_to_double<<<grid_for(c.nc, 256), 256, 0, st>>>(c, src, ch0, out);
    return 1;
}

int launch_fields_to_double(const Ctx &c, double *out, cudaStream_t st)
{
    k_fields_to_double<<<grid_for(c.nc, 256), 256, 0, st>>>(c, out);
    return 1;
}

int launch_velocities_to_double(const Ctx &c, double *out, cudaStream_t st)
{
    if (c.np == 0)
        return 0;
    k_velocities_to_double<<<grid_for(c.np, 256), 256, 0, st>>>(c, out);
    return 1;
}

int launch_vmax(const Ctx &c, cudaStream_t st)
{
    if (c.np == 0)
        return 0;
    if (c.prec == MHDPIC_PREC_MIXED)
        k_vmax<MHDPIC_PREC_MIXED><<<grid_for(c.np, 256), 256, 0, st>>>(c);
    else
        k_vmax<MHDPIC_PREC_FP64><<<grid_for(c.np, 256), 256, 0, st>>>(c);
    return 1;
}

int launch_scales(const Ctx &c, double dt, cudaStream_t st)
{
    k_scales<<<(c.nbox + 127) / 128, 128, 0, st>>>(c, dt);
    return 1;
}

}  // namespace mhdpic
