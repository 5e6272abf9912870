// Shock front tracking and CR injection (Section 5 of arXiv:1412.1087) for a
// single box with a conducting wall at x = 0 and an open inflow face at
// x = L_x (MHDPIC_BC_WALL_OPEN along x).
//
//   front     the transverse average of v_x = (rho v_x)/rho per x cell,
//             smoothed with a Gaussian kernel of standard deviation 4 cells
//             (truncated at 3 standard deviations and at the box ends,
//             renormalised); v_up is the smoothed value of the last (inflow)
//             cell; the front x_s is where, coming from upstream, |v_x| first
//             falls to 0.6 |v_up| (linear interpolation between centres); the
//             tail x_t is the centre of the first cell at or below the front
//             cell whose smoothed pressure reaches 2/3 of P1 = r/(r-1) rho_up
//             v_up^2 (eq:rh), x0 if none;
//   inject    eta of the gas mass swept in the step, rho_up (|v_up| + max(V,0))
//             dt A with V the front speed since the previous call, as CRs of
//             mass m_CR (the fraction carried to the next call), at x = x_s,
//             uniform across the box, isotropic in the front frame with
//             E_k = energy_factor v_up^2/2, boosted by V along x; random
//             numbers from Philox4x32-10 with counter (k, call, 0, 0);
//   compensation  the gas gives the injected mass, momentum and energy evenly
//             from the cells with centres in [x_t, x_s) (the front's cell
//             column when there are none).
// New particles go into the free slots past the live particles of the last
// sort, which puts the particles that left the box after all others: with
// that sort still pending, slot live + k of the sorted order is particle
// perm[live + k] of the current set; once a push (or a gather) has applied
// it, the slots live + k of the current set are free themselves.  Particles
// that left since that sort are collected by the next one.
#include "device_common.cuh"

namespace mhdpic {

// Device-resident state of the injection (one per context).
struct InjState {
    double xs, xt, rup, vup;   // front
    double xs_prev;            // front of the previous call (NaN: none)
    double carry;              // fraction of a particle carried to the next call
    double V;                  // front speed
    double Pin[3], Ein;        // injected momentum and energy
    int64_t n;                 // particles injected by this call
    int64_t live;              // live particles before injection
    int64_t i0, i1;            // compensation columns
    int32_t capped;
};


namespace {

constexpr int FRONT_THREADS = 1024;
constexpr int FRONT_CHUNKS = 16;    // row chunks of the column averages
constexpr int SMOOTH_HALF = 12;     // 3 standard deviations of 4 cells
constexpr int INJ_THREADS = 256;
constexpr int INJ_BLOCKS = 152 * 4;

__device__ __forceinline__ void philox4x32(uint32_t x[4], uint32_t k0, uint32_t k1)
{
    for (int r = 0; r < 10; ++r) {
        const uint32_t h0 = __umulhi(0xD2511F53u, x[0]), l0 = 0xD2511F53u * x[0];
        const uint32_t h1 = __umulhi(0xCD9E8D57u, x[2]), l1 = 0xCD9E8D57u * x[2];
        const uint32_t y0 = h1 ^ x[1] ^ k0, y2 = h0 ^ x[3] ^ k1;
        x[0] = y0;
        x[1] = l1;
        x[2] = y2;
        x[3] = l0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

__device__ __forceinline__ double unit_open(uint32_t u)
{
    return ((double)u + 0.5) * (1.0 / 4294967296.0);
}

// Column sums per x cell over one chunk of the rows: v_x, rho and pressure
// (part[chunk][3][nx]); k_front_reduce adds the chunks in order.
__global__ void k_front_profile(Ctx c, double gamma_gas, double *__restrict__ part)
{
    const BoxDev &b = c.boxes[0];
    const int64_t nx = b.n[0], nt = (int64_t)b.n[1] * b.n[2], nc = c.nc;
    const int64_t chunk = blockIdx.y;
    const int64_t t0 = nt * chunk / FRONT_CHUNKS, t1 = nt * (chunk + 1) / FRONT_CHUNKS;
    double *prof = part + chunk * 3 * nx;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nx; i += (int64_t)gridDim.x * blockDim.x) {
        double sv = 0.0, sr = 0.0, sp = 0.0;
        for (int64_t t = t0; t < t1; ++t) {
            const int64_t g = t * nx + i;
            const double r = c.rho[g];
            const double m0 = c.mom[g], m1 = c.mom[nc + g], m2 = c.mom[2 * nc + g];
            const double b0 = c.B[g], b1 = c.B[nc + g], b2 = c.B[2 * nc + g];
            sv += m0 / r;
            sr += r;
            const double mm = __dadd_rn(__dadd_rn(__dmul_rn(m0, m0), __dmul_rn(m1, m1)), __dmul_rn(m2, m2));
            const double bb = __dadd_rn(__dadd_rn(__dmul_rn(b0, b0), __dmul_rn(b1, b1)), __dmul_rn(b2, b2));
            sp += (gamma_gas - 1.0) * (c.egas[g] - 0.5 * mm / r - 0.5 * bb);
        }
        prof[i] = sv;
        prof[nx + i] = sr;
        prof[2 * nx + i] = sp;
    }
}

// Column averages: the chunks' sums in chunk order, over the rows.
__global__ void k_front_reduce(Ctx c, const double *__restrict__ part, double *__restrict__ prof)
{
    const BoxDev &b = c.boxes[0];
    const int64_t nx = b.n[0], nt = (int64_t)b.n[1] * b.n[2];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 3 * nx; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < FRONT_CHUNKS; ++k)
            s += part[k * 3 * nx + e];
        prof[e] = s / (double)nt;
    }
}

// Gaussian smoothing (standard deviation 4 cells, truncated at 3 standard
// deviations and at the box ends, renormalised) of the three profiles.
__global__ void k_front_smooth(Ctx c, const double *__restrict__ prof, double *__restrict__ smooth)
{
    __shared__ double w[2 * SMOOTH_HALF + 1];
    const BoxDev &b = c.boxes[0];
    const int64_t nx = b.n[0];
    const double sig = 4.0;
    if (threadIdx.x <= 2 * SMOOTH_HALF) {
        const int k = (int)threadIdx.x - SMOOTH_HALF;
        w[threadIdx.x] = exp(-0.5 * (double)(k * k) / (sig * sig));
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nx; i += (int64_t)gridDim.x * blockDim.x) {
        double ws = 0.0, a = 0.0, r = 0.0, p = 0.0;
        for (int k = -SMOOTH_HALF; k <= SMOOTH_HALF; ++k) {
            const int64_t j = i + k;
            if (j < 0 || j >= nx)
                continue;
            const double wk = w[k + SMOOTH_HALF];
            ws += wk;
            a += wk * prof[j];
            r += wk * prof[nx + j];
            p += wk * prof[2 * nx + j];
        }
        smooth[i] = a / ws;
        smooth[nx + i] = r / ws;
        smooth[2 * nx + i] = p / ws;
    }
}

__device__ __forceinline__ int64_t block_min(int64_t v, int64_t *red)
{
    for (int o = 16; o > 0; o >>= 1)
        v = min(v, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = v;
    __syncthreads();
    int64_t r = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        r = min(r, red[w]);
    return r;
}

__device__ __forceinline__ int64_t block_max(int64_t v, int64_t *red)
{
    for (int o = 16; o > 0; o >>= 1)
        v = max(v, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = v;
    __syncthreads();
    int64_t r = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        r = max(r, red[w]);
    return r;
}

// One block: the front and the tail, the injected count and the
// compensation columns.
__global__ void __launch_bounds__(FRONT_THREADS) k_front_scan(Ctx c, const double *__restrict__ smooth,
                                                              double gamma_gas, double dt, double eta, InjState *st,
                                                              const int32_t *__restrict__ offset)
{
    __shared__ int64_t red[32];
    const BoxDev &b = c.boxes[0];
    const int64_t nx = b.n[0];
    const double vup = smooth[nx - 1], rup = smooth[2 * nx - 1];
    const double thr = 0.6 * fabs(vup);
    int64_t best = -1;
    if (vup != 0.0)
        for (int64_t i = threadIdx.x; i <= nx - 2; i += blockDim.x)
            if (fabs(smooth[i]) <= thr)
                best = max(best, i);
    const int64_t is = block_max(best, red);
    double xs = __longlong_as_double(0x7ff8000000000000ll);
    if (is >= 0) {
        const double a = fabs(smooth[is]), bb = fabs(smooth[is + 1]);
        const double f = (thr - a) / (bb - a);
        xs = b.x0[0] + ((double)is + 0.5 + f) * b.dx[0];
    }
    int64_t it = -1;
    if (is >= 0) {
        const double r = (gamma_gas + 1.0) / (gamma_gas - 1.0);
        const double P1 = r / (r - 1.0) * rup * vup * vup;
        for (int64_t i = threadIdx.x; i <= is; i += blockDim.x)
            if (smooth[2 * nx + i] >= (2.0 / 3.0) * P1)
                it = max(it, i);
    }
    it = block_max(it, red);
    const double xt = it >= 0 ? b.x0[0] + ((double)it + 0.5) * b.dx[0] : b.x0[0];
    // compensation columns: centres in [x_t, x_s)
    int64_t lo = INT64_MAX, hi = -1;
    if (is >= 0)
        for (int64_t i = threadIdx.x; i < nx; i += blockDim.x) {
            const double xc = b.x0[0] + ((double)i + 0.5) * b.dx[0];
            if (xc >= xt && xc < xs) {
                lo = min(lo, i);
                hi = max(hi, i);
            }
        }
    lo = block_min(lo, red);
    hi = block_max(hi, red);
    if (threadIdx.x == 0) {
        st->xs = xs;
        st->xt = xt;
        st->rup = rup;
        st->vup = vup;
        st->live = offset[c.nkeys];
        st->n = 0;
        st->capped = 0;
        st->V = 0.0;
        if (!isnan(xs)) {
            const double V = isnan(st->xs_prev) ? 0.0 : (xs - st->xs_prev) / dt;
            double A = 1.0;
            for (int d = 1; d < 3; ++d)
                A *= d < c.ndim ? b.n[d] * b.dx[d] : b.dx[d];
            const double M = rup * (fabs(vup) + (V > 0.0 ? V : 0.0)) * dt * A;
            const double want = eta * M / b.m_cr + st->carry;
            int64_t n = (int64_t)floor(want);
            st->carry = want - (double)n;
            const int64_t freeslots = c.np - st->live;
            if (n > freeslots) {
                n = freeslots;
                st->capped = 1;
                set_status(c.status, MHDPIC_ST_INJECT_CAP);
            }
            st->n = n;
            st->V = V;
            int64_t i0 = hi >= 0 ? lo : -1, i1 = hi;
            if (i0 < 0) {
                i0 = (int64_t)floor((xs - b.x0[0]) / b.dx[0]);
                if (i0 >= nx)
                    i0 = nx - 1;
                i1 = i0;
            }
            st->i0 = i0;
            st->i1 = i1;
        }
        st->xs_prev = xs;
    }
}

// New particles k < n into the free slots; per-block sums of m v and m E_k of
// what was stored (in a fixed order) into partials[block][4].
template <int PREC>
__global__ void __launch_bounds__(INJ_THREADS) k_inject_particles(Ctx c, const int32_t *__restrict__ perm,
                                                                  const InjState *__restrict__ st, double fE,
                                                                  uint64_t seed, uint32_t call, int use_perm,
                                                                  double *__restrict__ partials)
{
    __shared__ double red[4][INJ_THREADS];
    const BoxDev &b = c.boxes[0];
    const int64_t n = st->n, live = st->live;
    const double xs = st->xs, V = st->V, vup = st->vup;
    const double C = b.C;
    const double Ek = fE * 0.5 * vup * vup;
    const double gp = 1.0 + Ek / (C * C);
    const double vmag = C * sqrt(gp * gp - 1.0);
    const double Gam = 1.0 / sqrt(1.0 - V * V / (C * C));
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    // block b takes the contiguous range [b q, (b+1) q)
    const int64_t q = (n + gridDim.x - 1) / gridDim.x;
    const int64_t a0 = blockIdx.x * q, a1 = min(n, a0 + q);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    float vm = 0.f;   // largest |v| injected, for the next corrector scale
    for (int64_t k = a0 + threadIdx.x; k < a1; k += blockDim.x) {
        uint32_t x[4] = {(uint32_t)k, call, 0u, 0u};
        philox4x32(x, k0, k1);
        double pos[3] = {xs, 0.0, 0.0};
        if (c.ndim >= 2)
            pos[1] = b.x0[1] + unit_open(x[0]) * b.n[1] * b.dx[1];
        if (c.ndim == 3)
            pos[2] = b.x0[2] + unit_open(x[1]) * b.n[2] * b.dx[2];
        const double mu = 2.0 * unit_open(x[2]) - 1.0;
        const double ph = 6.283185307179586 * unit_open(x[3]);
        const double s = sqrt(1.0 - mu * mu);
        double v[3] = {vmag * mu, vmag * s * cos(ph), vmag * s * sin(ph)};
        v[0] = Gam * (v[0] + V * gp);
        const int64_t j = use_perm ? (int64_t)perm[live + k] : live + k;
        if (PREC == MHDPIC_PREC_MIXED) {
            int ci[3] = {0, 0, 0};
            float off[3] = {0.f, 0.f, 0.f};
            for (int d = 0; d < c.ndim; ++d) {
                const double sd = (pos[d] - b.x0[d]) / b.dx[d];
                double f = floor(sd);
                int i = (int)f;
                float o = (float)(sd - f);
                if (o >= 1.f) {
                    o = 0.f;
                    ++i;
                }
                i = i < 0 ? 0 : (i >= b.n[d] ? b.n[d] - 1 : i);
                ci[d] = i;
                off[d] = o;
            }
            c.pos[j] = make_int4((int32_t)(((int64_t)ci[2] * b.n[1] + ci[1]) * b.n[0] + ci[0]),
                                 __float_as_int(off[0]), __float_as_int(off[1]), __float_as_int(off[2]));
            float vf[3];
            for (int d = 0; d < 3; ++d) {
                vf[d] = (float)v[d];
                v[d] = (double)vf[d];   // the sums below are of what is stored (no residual)
            }
            c.vel[j] = make_float4(vf[0], vf[1], vf[2], 0.f);
        } else {
            for (int d = 0; d < c.ndim; ++d)
                c.x[(int64_t)d * c.np + j] = pos[d];
            for (int d = 0; d < 3; ++d)
                c.p64[(int64_t)d * c.np + j] = v[d];
        }
        if (c.tinj)   // injected now: t_i is the clock
            c.tinj[j] = c.clock[0];
        const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        const double g = sqrt(C * C + v2) / C;
        for (int d = 0; d < 3; ++d)
            acc[d] += b.m_cr * v[d];
        acc[3] += b.m_cr * (v2 / (g + 1.0));
        vm = fmaxf(vm, (float)sqrt(v2));
    }
    const unsigned vb = __reduce_max_sync(0xffffffffu, __float_as_uint(vm));
    if ((threadIdx.x & 31) == 0 && vb)
        atomicMax(&c.stats[0].vmax, vb);
    for (int q2 = 0; q2 < 4; ++q2)
        red[q2][threadIdx.x] = acc[q2];
    __syncthreads();
    for (int s2 = INJ_THREADS / 2; s2 > 0; s2 >>= 1) {
        if (threadIdx.x < s2)
            for (int q2 = 0; q2 < 4; ++q2)
                red[q2][threadIdx.x] += red[q2][threadIdx.x + s2];
        __syncthreads();
    }
    if (threadIdx.x < 4)
        partials[blockIdx.x * 4 + threadIdx.x] = red[threadIdx.x][0];
}

// One warp: lane l adds blocks l, l+32, ... in order, then a fixed tree.
__global__ void k_inject_totals(const double *__restrict__ partials, int nblocks, InjState *st)
{
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += 32)
        for (int q = 0; q < 4; ++q)
            s[q] += partials[b * 4 + q];
    for (int o = 16; o > 0; o >>= 1)
        for (int q = 0; q < 4; ++q)
            s[q] += __shfl_down_sync(0xffffffffu, s[q], o);
    if (threadIdx.x == 0) {
        st->Pin[0] = s[0];
        st->Pin[1] = s[1];
        st->Pin[2] = s[2];
        st->Ein = s[3];
    }
}

// The gas of the compensation columns gives the injected mass, momentum and energy.
__global__ void k_compensate(Ctx c, const InjState *__restrict__ st)
{
    if (st->n <= 0)
        return;
    const BoxDev &b = c.boxes[0];
    const int64_t nx = b.n[0], nt = (int64_t)b.n[1] * b.n[2], nc = c.nc;
    const int64_t i0 = st->i0, i1 = st->i1, w = i1 - i0 + 1;
    const double Vreg = (double)(w * nt) * b.dV;
    const double Min = (double)st->n * b.m_cr;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < w * nt; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = e / w, i = i0 + e % w;
        const int64_t g = t * nx + i;
        c.rho[g] -= Min / Vreg;
        for (int d = 0; d < 3; ++d)
            c.mom[d * nc + g] -= st->Pin[d] / Vreg;
        c.egas[g] -= st->Ein / Vreg;
    }
}

int grid_of(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

}  // namespace

size_t inject_state_bytes()
{
    return sizeof(InjState);
}

void init_inject_state(void *st_host)
{
    InjState *s = reinterpret_cast<InjState *>(st_host);
    *s = InjState{};
    s->xs_prev = __builtin_nan("");
}

void inject_outputs(const void *st_host, double front[2], int64_t *n, int *capped)
{
    const InjState *s = reinterpret_cast<const InjState *>(st_host);
    front[0] = s->xs;
    front[1] = s->xt;
    *n = s->n;
    *capped = s->capped;
}

int launch_inject(const Ctx &c, const SortScratch &s, void *state, double *scratch, int64_t nx, double dt,
                  double eta, double energy_factor, double gamma_gas, uint64_t seed, uint32_t call, int use_perm,
                  cudaStream_t st)
{
    InjState *is = reinterpret_cast<InjState *>(state);
    double *prof = scratch, *smooth = scratch + 3 * nx, *partials = scratch + 6 * nx;
    double *part = partials + 4 * INJ_BLOCKS;
    k_front_profile<<<dim3(grid_of(nx, 128), FRONT_CHUNKS), 128, 0, st>>>(c, gamma_gas, part);
    k_front_reduce<<<grid_of(3 * nx, 256), 256, 0, st>>>(c, part, prof);
    k_front_smooth<<<grid_of(nx, 128), 128, 0, st>>>(c, prof, smooth);
    k_front_scan<<<1, FRONT_THREADS, 0, st>>>(c, smooth, gamma_gas, dt, eta, is, s.offset);
    if (c.prec == MHDPIC_PREC_MIXED)
        k_inject_particles<MHDPIC_PREC_MIXED><<<INJ_BLOCKS, INJ_THREADS, 0, st>>>(c, s.perm, is, energy_factor, seed,
                                                                                  call, use_perm, partials);
    else
        k_inject_particles<MHDPIC_PREC_FP64><<<INJ_BLOCKS, INJ_THREADS, 0, st>>>(c, s.perm, is, energy_factor, seed,
                                                                                 call, use_perm, partials);
    k_inject_totals<<<1, 32, 0, st>>>(partials, INJ_BLOCKS, is);
    k_compensate<<<grid_of(c.nc, 256), 256, 0, st>>>(c, is);
    return 7;
}

size_t inject_scratch_doubles(int64_t nx)
{
    return (size_t)(6 * nx + 4 * INJ_BLOCKS + 3 * FRONT_CHUNKS * nx);
}

}  // namespace mhdpic
