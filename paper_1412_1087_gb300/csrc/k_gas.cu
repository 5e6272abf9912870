// Gas kernels of the coupled step, the predictor-corrector of App. A.3
// (eq:scheme of arXiv:1412.1087):
//
//   predictor  g^(n+1/2) = g^n + G(f^n, g^n) dt/2, with the CR sources of the
//              moments n, J deposited at x^n, fused with the staging of the
//              half-step cell fields the push reads;
//   corrector  g^(n+1) = g^n + G((f^n + f^(n+1))/2, g^(n+1/2)) dt, the CR part
//              being the corrector deposit of the push (momentum and energy
//              handed to the gas over the step).
//
// G has a CR part and a gas part.  CR sources (eq:gasmotion, eq:engeq):
// momentum -F_CR, F_CR = (1-R)(n E0 + J x B) (eq:lorentz2), energy
// -(1-R) J.E0, R = n/(n_g + n) with the CR-Hall term and 0 without it.  Gas
// part, by model:
//   MHDPIC_GAS_SOURCES   nothing else: B stays as it is;
//   MHDPIC_GAS_LINEAR_X  plane-parallel linear MHD along x (rho and B_x
//                        uniform, v_x = 0 to first order):
//                          d(rho v_y,z)/dt = B_x dB_y,z/dx,
//                          dB_y,z/dt = B_x dv_y,z/dx,
//                        plus the curl of the CR-Hall field -F_CR/n_g
//                        (eq:emfcr2 in eq:induction):
//                          dB_y/dt += -d(F_z/n_g)/dx, dB_z/dt += d(F_y/n_g)/dx;
//                        centred differences, x periodic.  In the corrector
//                        the CR-Hall field takes the force the corrector
//                        deposit implies, F_CR = -dM/(dV dt).
// The gas energy takes only the CR sources (the paper's linear test gas is
// isothermal, App. B.2).  All gas arithmetic is FP64.
#include "device_common.cuh"

namespace mhdpic {

namespace {

constexpr double FIXED_LIMIT_G = 4611686018427387904.0;  // 2^62

__device__ __forceinline__ void cross(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// Neighbour along x (s = -1 or +1) of global cell g inside box b, x periodic.
__device__ __forceinline__ int64_t x_neighbour(const BoxDev &b, int64_t g, int s)
{
    const uint32_t loc = (uint32_t)(g - b.cell0);   // a box has < 2^31 cells
    const int nx = b.n[0];
    const int i = (int)(loc - fdiv(loc, b.div_nx) * (uint32_t)nx);
    const int j = i + s < 0 ? nx - 1 : (i + s >= nx ? 0 : i + s);
    return g - i + j;
}

// n and J of the moments buffer md at cell g.
__device__ __forceinline__ void moments_at(const Ctx &c, const BoxDev &b, const unsigned long long *md, int64_t g,
                                           double &n, double J[3])
{
    const int64_t nc = c.nc;
    n = from_fixed(md[g], b.inv_scale[CH_N]);
    J[0] = from_fixed(md[nc + g], b.inv_scale[CH_JX]);
    J[1] = from_fixed(md[2 * nc + g], b.inv_scale[CH_JY]);
    J[2] = from_fixed(md[3 * nc + g], b.inv_scale[CH_JZ]);
}

// F_CR (eq:lorentz2) and (1-R) J.E0 (eq:engeq) of one cell.
__device__ __forceinline__ void cr_force(const BoxDev &b, double rho, const double m[3], const double B[3], double n,
                                         const double J[3], double F[3], double &P)
{
    // FP64 divisions are slow on this GPU: one reciprocal per cell
    const double ir = 1.0 / rho;
    const double vg[3] = {m[0] * ir, m[1] * ir, m[2] * ir};
    double vxb[3], JxB[3];
    cross(vg, B, vxb);
    const double E0[3] = {-vxb[0], -vxb[1], -vxb[2]};
    const double R = b.hall ? n / (b.qm_gas * rho + n) : 0.0;
    cross(J, B, JxB);
    for (int d = 0; d < 3; ++d)
        F[d] = (1.0 - R) * (n * E0[d] + JxB[d]);
    P = (1.0 - R) * (J[0] * E0[0] + J[1] * E0[1] + J[2] * E0[2]);
}

// CR-Hall field F_CR / n_g at cell g of the state (rho, mom, B) with moments md.
__device__ __forceinline__ void hall_field(const Ctx &c, const BoxDev &b, const unsigned long long *md,
                                           const double *rho, const double *mom, const double *B, int64_t g,
                                           double H[3])
{
    const int64_t nc = c.nc;
    double n, J[3], F[3], P;
    moments_at(c, b, md, g, n, J);
    const double m[3] = {mom[g], mom[nc + g], mom[2 * nc + g]};
    const double Bc[3] = {B[g], B[nc + g], B[2 * nc + g]};
    cr_force(b, rho[g], m, Bc, n, J, F, P);
    const double ng = b.qm_gas * rho[g];
    for (int d = 0; d < 3; ++d)
        H[d] = F[d] / ng;
}

// Gas-model part of G at cell g of the state (rho, mom, B): dmom and dB
// (without the CR-Hall curl, which the callers add).
__device__ __forceinline__ void linear_x(const Ctx &c, const BoxDev &b, const double *rho, const double *mom,
                                         const double *B, int64_t g, int64_t l, int64_t r, double dmom[3],
                                         double dB[3])
{
    const int64_t nc = c.nc;
    const double h = 0.5 * b.inv_dx[0];
    const double Bx = B[g];
    const double irr = 1.0 / rho[r], irl = 1.0 / rho[l];
    dmom[0] = dB[0] = 0.0;
    for (int d = 1; d < 3; ++d) {
        dmom[d] = Bx * (B[d * nc + r] - B[d * nc + l]) * h;
        dB[d] = Bx * (mom[d * nc + r] * irr - mom[d * nc + l] * irl) * h;
    }
}

// Predictor: half state into `half` (planes rho, mom x3, egas, B x3) and the
// cell fields of the half state (as the stage kernel: E0 = -v x B, with the
// CR-Hall term E = E0 - F/n_g from the moments at x^n) for the push; clears
// the moments buffer the next push fills; records max |E|, |B|.
template <int PREC>
__global__ void k_gas_predict(Ctx c, int cur, double dt, int model, double *__restrict__ half)
{
    const unsigned long long *__restrict__ md = c.momdep[cur];
    unsigned long long *__restrict__ mnext = c.momdep[cur ^ 1];
    const int64_t nc = c.nc;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nc;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int bx = find_box(c.box_cell_start, c.nbox, g);
        const BoxDev &b = c.boxes[bx];
        const double rho = c.rho[g];
        const double m[3] = {c.mom[g], c.mom[nc + g], c.mom[2 * nc + g]};
        const double Bc[3] = {c.B[g], c.B[nc + g], c.B[2 * nc + g]};
        double n, J[3], F[3], P;
        moments_at(c, b, md, g, n, J);
        cr_force(b, rho, m, Bc, n, J, F, P);
        double dmom[3] = {0.0, 0.0, 0.0}, dB[3] = {0.0, 0.0, 0.0};
        if (model == MHDPIC_GAS_LINEAR_X) {
            const int64_t l = x_neighbour(b, g, -1), r = x_neighbour(b, g, 1);
            linear_x(c, b, c.rho, c.mom, c.B, g, l, r, dmom, dB);
            if (b.hall) {
                double Hl[3], Hr[3];
                hall_field(c, b, md, c.rho, c.mom, c.B, l, Hl);
                hall_field(c, b, md, c.rho, c.mom, c.B, r, Hr);
                const double h = 1.0 / (2.0 * b.dx[0]);
                dB[1] -= (Hr[2] - Hl[2]) * h;
                dB[2] += (Hr[1] - Hl[1]) * h;
            }
        }
        double mh[3], Bh[3];
        for (int d = 0; d < 3; ++d) {
            mh[d] = m[d] + 0.5 * dt * (dmom[d] - F[d]);
            Bh[d] = Bc[d] + 0.5 * dt * dB[d];
        }
        const double egh = c.egas[g] - 0.5 * dt * P;
        half[g] = rho;
        half[nc + g] = mh[0];
        half[2 * nc + g] = mh[1];
        half[3 * nc + g] = mh[2];
        half[4 * nc + g] = egh;
        half[5 * nc + g] = Bh[0];
        half[6 * nc + g] = Bh[1];
        half[7 * nc + g] = Bh[2];

        // cell fields of the half state
        const double irho = 1.0 / rho;
        const double v[3] = {mh[0] * irho, mh[1] * irho, mh[2] * irho};
        const double E0[3] = {-(v[1] * Bh[2] - v[2] * Bh[1]), -(v[2] * Bh[0] - v[0] * Bh[2]),
                              -(v[0] * Bh[1] - v[1] * Bh[0])};
        double E[3] = {E0[0], E0[1], E0[2]};
        if (b.hall) {
            const double ng = b.qm_gas * rho;
            const double R = n / (ng + n);
            double JxB[3];
            cross(J, Bh, JxB);
            for (int d = 0; d < 3; ++d) {
                const double Fh = (1.0 - R) * (n * E0[d] + JxB[d]);
                E[d] = E0[d] - Fh / ng;
            }
        }
        if (PREC == MHDPIC_PREC_MIXED) {
            int ci[3];
            decode_cell(b, (int32_t)(g - b.cell0), ci);
            store_fields_mixed(c.fa, c.fb, b, ci[0], ci[1], ci[2],
                               make_float4((float)E[0], (float)E[1], (float)E[2], (float)Bh[0]),
                               make_float2((float)Bh[1], (float)Bh[2]));
        } else {
            double2 *f = reinterpret_cast<double2 *>(c.f64) + 3 * g;
            f[0] = make_double2(E[0], E[1]);
            f[1] = make_double2(E[2], Bh[0]);
            f[2] = make_double2(Bh[1], Bh[2]);
        }
        for (int q = 0; q < 4; ++q)
            mnext[q * nc + g] = 0ull;
        const float em = (float)sqrt(E[0] * E[0] + E[1] * E[1] + E[2] * E[2]);
        const float bm = (float)sqrt(Bh[0] * Bh[0] + Bh[1] * Bh[1] + Bh[2] * Bh[2]);
        const unsigned peers = __match_any_sync(__activemask(), bx);
        const unsigned eb = __reduce_max_sync(peers, __float_as_uint(em));
        const unsigned bb = __reduce_max_sync(peers, __float_as_uint(bm));
        if ((threadIdx.x & 31) == __ffs(peers) - 1) {
            atomicMax(&c.stats[bx].emax, eb);
            atomicMax(&c.stats[bx].bmax, bb);
        }
    }
}

// Corrector: the caller's gas (c.mom, c.egas, c.B) advances from g^n to
// g^(n+1) in place; rho does not change.  Reads the half state and the
// corrector accumulators of this cell and its x neighbours; the accumulators
// are cleared by the caller after the kernel.
__global__ void k_gas_correct(Ctx c, double dt, int model, const double *__restrict__ half)
{
    const int64_t nc = c.nc;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nc;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int bx = find_box(c.box_cell_start, c.nbox, g);
        const BoxDev &b = c.boxes[bx];
        bool over = false;
        double dM[3];
        for (int d = 0; d < 3; ++d) {
            const unsigned long long a = c.corr[d * nc + g];
            over |= fabs((double)(long long)a) >= FIXED_LIMIT_G;
            dM[d] = from_fixed(a, b.inv_scale[CH_MX + d]);
        }
        const unsigned long long ae = c.corr[3 * nc + g];
        over |= fabs((double)(long long)ae) >= FIXED_LIMIT_G;
        const double dE = from_fixed(ae, b.inv_scale[CH_E]);
        double dmom[3] = {0.0, 0.0, 0.0}, dB[3] = {0.0, 0.0, 0.0};
        if (model == MHDPIC_GAS_LINEAR_X) {
            const int64_t l = x_neighbour(b, g, -1), r = x_neighbour(b, g, 1);
            const double *rho_h = half, *mom_h = half + nc, *B_h = half + 5 * nc;
            linear_x(c, b, rho_h, mom_h, B_h, g, l, r, dmom, dB);
            if (b.hall) {
                // F_CR = -dM / (dV dt), H = F_CR / n_g of the half state
                double Hl[3], Hr[3];
                for (int d = 0; d < 3; ++d) {
                    Hl[d] = (-from_fixed(c.corr[d * nc + l], b.inv_scale[CH_MX + d]) / (b.dV * dt)) /
                            (b.qm_gas * rho_h[l]);
                    Hr[d] = (-from_fixed(c.corr[d * nc + r], b.inv_scale[CH_MX + d]) / (b.dV * dt)) /
                            (b.qm_gas * rho_h[r]);
                }
                const double h = 1.0 / (2.0 * b.dx[0]);
                dB[1] -= (Hr[2] - Hl[2]) * h;
                dB[2] += (Hr[1] - Hl[1]) * h;
            }
        }
        for (int d = 0; d < 3; ++d) {
            c.mom[d * nc + g] += dt * dmom[d] + dM[d] * b.inv_dV;
            c.B[d * nc + g] += dt * dB[d];
        }
        c.egas[g] += dE * b.inv_dV;
        if (over)
            set_status(c.status, MHDPIC_ST_OVERFLOW);
    }
    if (blockIdx.x == 0)
        for (int q = threadIdx.x; q < c.nbox; q += blockDim.x)
            c.stats[q].corr_dirty = 0;
}

int cell_grid(int64_t nc)
{
    int64_t g = (nc + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

}  // namespace

int launch_gas_predict(const Ctx &c, int cur, double dt, int model, double *half, cudaStream_t st)
{
    if (c.prec == MHDPIC_PREC_MIXED)
        k_gas_predict<MHDPIC_PREC_MIXED><<<cell_grid(c.nc), 256, 0, st>>>(c, cur, dt, model, half);
    else
        k_gas_predict<MHDPIC_PREC_FP64><<<cell_grid(c.nc), 256, 0, st>>>(c, cur, dt, model, half);
    return 1;
}

int launch_gas_correct(const Ctx &c, double dt, int model, const double *half, cudaStream_t st)
{
    k_gas_correct<<<cell_grid(c.nc), 256, 0, st>>>(c, dt, model, half);
    cudaMemsetAsync(c.corr, 0, sizeof(unsigned long long) * 4 * (size_t)c.nc, st);
    return 1;
}

}  // namespace mhdpic
