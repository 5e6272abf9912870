// Per-cell kernels: feedback to the gas fused with the staging of the
// cell-centred fields; the standalone charge/current deposit; FP64 totals;
// read-back conversions.
#include "device_common.cuh"

namespace mhdpic {

namespace {

constexpr double FIXED_LIMIT = 4611686018427387904.0;  // 2^62: accumulator headroom


// One pass over the cells of all boxes:
//   apply:  rho v += dM / dV, egas += dE / dV (Section 2.1 Newton's third law,
//           App. A.3 corrector), accumulators zeroed;
//   stage:  E0 = -v_g x B (eq:emf0); with the CR-Hall term
//           n_g = qm_gas rho (eq:ng), R = n/(n_g + n) (eq:defR),
//           F = (1-R)(n E0 + J x B) (eq:lorentz2), E = E0 - F/n_g (eq:emfcr2),
//           n, J being the moments in buffer `cur`;
//   clear:  moments buffer cur^1, which the next push fills.
template <int PREC>
__global__ void k_prep(Ctx c, int cur, int apply)
{
    const unsigned long long *__restrict__ md = c.momdep[cur];
    unsigned long long *__restrict__ mnext = c.momdep[cur ^ 1];
    const int64_t nc = c.nc;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nc;
         g += (int64_t)gridDim.x * blockDim.x) {
        int bx = find_box(c.box_cell_start, c.nbox, g);
        const BoxDev &b = c.boxes[bx];
        double rho = c.rho[g];
        double m[3] = {c.mom[g], c.mom[nc + g], c.mom[2 * nc + g]};
        if (apply) {
            bool over = false;
            for (int d = 0; d < 3; ++d) {
                unsigned long long a = c.corr[d * nc + g];
                over |= fabs((double)(long long)a) >= FIXED_LIMIT;
                m[d] += from_fixed(a, b.inv_scale[CH_MX + d]) * b.inv_dV;
                c.mom[d * nc + g] = m[d];
                c.corr[d * nc + g] = 0ull;
            }
            unsigned long long a = c.corr[3 * nc + g];
            over |= fabs((double)(long long)a) >= FIXED_LIMIT;
            c.egas[g] += from_fixed(a, b.inv_scale[CH_E]) * b.inv_dV;
            c.corr[3 * nc + g] = 0ull;
            if (over)
                set_status(c.status, MHDPIC_ST_OVERFLOW);
        }
        double Bc[3] = {c.B[g], c.B[nc + g], c.B[2 * nc + g]};
        double v[3] = {m[0] / rho, m[1] / rho, m[2] / rho};
        double E0[3] = {-(v[1] * Bc[2] - v[2] * Bc[1]), -(v[2] * Bc[0] - v[0] * Bc[2]),
                        -(v[0] * Bc[1] - v[1] * Bc[0])};
        double E[3] = {E0[0], E0[1], E0[2]};
        if (b.hall) {
            double ng = b.qm_gas * rho;
            double n = from_fixed(md[g], b.inv_scale[CH_N]);
            double J[3] = {from_fixed(md[nc + g], b.inv_scale[CH_JX]), from_fixed(md[2 * nc + g], b.inv_scale[CH_JY]),
                           from_fixed(md[3 * nc + g], b.inv_scale[CH_JZ])};
            double R = n / (ng + n);
            double JxB[3] = {J[1] * Bc[2] - J[2] * Bc[1], J[2] * Bc[0] - J[0] * Bc[2],
                             J[0] * Bc[1] - J[1] * Bc[0]};
            for (int d = 0; d < 3; ++d) {
                double F = (1.0 - R) * (n * E0[d] + JxB[d]);
                E[d] = E0[d] - F / ng;
            }
        }
        if (PREC == MHDPIC_PREC_MIXED) {
            float4 a = make_float4((float)E[0], (float)E[1], (float)E[2], (float)Bc[0]);
            float4 bb = make_float4((float)Bc[1], (float)Bc[2], 0.f, 0.f);
            reinterpret_cast<float4 *>(c.f32)[2 * g] = a;
            reinterpret_cast<float4 *>(c.f32)[2 * g + 1] = bb;
        } else {
            double2 *f = reinterpret_cast<double2 *>(c.f64) + 3 * g;
            f[0] = make_double2(E[0], E[1]);
            f[1] = make_double2(E[2], Bc[0]);
            f[2] = make_double2(Bc[1], Bc[2]);
        }
        for (int q = 0; q < 4; ++q)
            mnext[q * nc + g] = 0ull;
        // per-box maxima of |E| and |B| for the corrector scales
        float em = (float)sqrt(E[0] * E[0] + E[1] * E[1] + E[2] * E[2]);
        float bm = (float)sqrt(Bc[0] * Bc[0] + Bc[1] * Bc[1] + Bc[2] * Bc[2]);
        unsigned peers = __match_any_sync(__activemask(), bx);
        unsigned eb = __reduce_max_sync(peers, __float_as_uint(em));
        unsigned bb2 = __reduce_max_sync(peers, __float_as_uint(bm));
        if ((threadIdx.x & 31) == __ffs(peers) - 1) {
            atomicMax(&c.stats[bx].emax, eb);
            atomicMax(&c.stats[bx].bmax, bb2);
        }
    }
    if (apply && blockIdx.x == 0)
        for (int bx = threadIdx.x; bx < c.nbox; bx += blockDim.x)
            c.stats[bx].corr_dirty = 0;
}

// Size the corrector scales of every box for a push of step dt, unless the
// accumulators already hold data (then the scales stay as they are).
// Bounds, with hh = |q/mc| dt / 2 and u = v/gamma (|u| < C):
//   |v^0| <= vmax + hh Emax;
//   rotation |v^1 - v^0| = 2|v^0| sin(theta/2) <= 2 |v^0| |b| = 2 hh |B| |u^0|;
//   |dv| <= 2 hh Emax + 2 hh Bmax min(|v^0|, C)                       (x2 margin)
//   the rotation keeps |v|, so dE_k is the energy change of the two half
//   kicks, each (hh E).(a+b)/(gamma_a+gamma_b) with |a+b|/(gamma_a+gamma_b) <
//   min(C, max|a|, |b|):  |dE_k| <= 2 hh Emax min(C, |v^0| + hh Emax)  (x2 margin).
// With H = 3^D (4 maxcount + 64) contributions per cell at most, the scale is
// the power of two with Q H S <= 2^62.
__global__ void k_scales(Ctx c, double dt)
{
    int bx = blockIdx.x * blockDim.x + threadIdx.x;
    if (bx >= c.nbox)
        return;
    BoxStats &st = c.stats[bx];
    if (st.corr_dirty)
        return;
    BoxDev &b = c.boxes_rw[bx];
    double hh = 0.5 * fabs(b.qm_cr) * dt;
    // no staging since the last choice (e.g. a push right after the coupled
    // step's corrector): the staged fields are the ones measured then
    uint32_t eb = st.emax, bb = st.bmax;
    if (eb == 0u && bb == 0u) {
        eb = st.emax_used;
        bb = st.bmax_used;
    }
    st.emax_used = eb;
    st.bmax_used = bb;
    double vmax = (double)__uint_as_float(st.vmax);
    double emax = (double)__uint_as_float(eb);
    double bmax = (double)__uint_as_float(bb);
    double H = (c.ndim == 3 ? 27.0 : 9.0) * (4.0 * st.maxcount + 64.0);
    double vb = vmax + hh * emax;
    double qdv = 2.0 * (2.0 * hh * emax + 2.0 * hh * bmax * fmin(vb, b.C));
    double q[4];
    q[0] = q[1] = q[2] = fabs(b.m_cr) * qdv;
    q[3] = fabs(b.m_cr) * 2.0 * (2.0 * hh * emax * fmin(b.C, vb + hh * emax));
    for (int ch = 0; ch < 4; ++ch) {
        double Q = fmax(q[ch], 1e-30);
        int e;
        frexp(FIXED_LIMIT / (Q * H), &e);   // 2^(e-1) <= 2^62/(Q H) < 2^e
        e -= 1;
        if (e > SCALE_EXP_MAX)
            e = SCALE_EXP_MAX;
        b.escale[ch] = e;
        b.scale[ch] = ldexp(1.0, e);
        b.inv_scale[ch] = ldexp(1.0, -e);
        b.qbound[ch] = Q;
        b.qmax[ch] = 4.0 * Q;   // a particle quantity beyond this raises the overflow flag
    }
    st.corr_dirty = 1;
    st.vmax = 0u;
    st.emax = 0u;
    st.bmax = 0u;
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
        for (int q = 0; q < 6; ++q)
            out[q * c.nc + g] = c.prec == MHDPIC_PREC_MIXED ? (double)c.f32[g * 8 + q] : c.f64[g * 6 + q];
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
