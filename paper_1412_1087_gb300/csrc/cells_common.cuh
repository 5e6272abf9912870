// Per-cell device code shared by the cell kernels and the fused step kernel:
// the feedback to the gas fused with the field staging (prep_cells) and the
// choice of the corrector's fixed-point scales (scales_box).
#pragma once

#include "device_common.cuh"

namespace mhdpic {

constexpr double FIXED_LIMIT = 4611686018427387904.0;  // 2^62: accumulator headroom


// One pass over the cells of all boxes:
//   apply:  rho v += dM / dV, egas += dE / dV (Section 2.1 Newton's third law,
//           App. A.3 corrector), accumulators zeroed;
//   stage:  E0 = -v_g x B (eq:emf0); with the CR-Hall term
//           n_g = qm_gas rho (eq:ng), R = n/(n_g + n) (eq:defR),
//           F = (1-R)(n E0 + J x B) (eq:lorentz2), E = E0 - F/n_g (eq:emfcr2),
//           n, J being the moments in buffer `cur`;
//   clear:  moments buffer cur^1, which the next push fills.
// The loop runs over the whole grid of the calling kernel (grid-stride).
template <int PREC>
__device__ __forceinline__ void prep_cells(const Ctx &c, int cur, int apply)
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
        // FP64 divisions are slow on this GPU: the mixed path, whose fields
        // are staged in FP32, divides once by rho (and once by n_g) and
        // multiplies; the FP64 path keeps the oracle's divisions
        double v[3];
        if (PREC == MHDPIC_PREC_MIXED) {
            const double ir = 1.0 / rho;
            v[0] = m[0] * ir;
            v[1] = m[1] * ir;
            v[2] = m[2] * ir;
        } else {
            v[0] = m[0] / rho;
            v[1] = m[1] / rho;
            v[2] = m[2] / rho;
        }
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
            const double ing = PREC == MHDPIC_PREC_MIXED ? 1.0 / ng : 0.0;
            for (int d = 0; d < 3; ++d) {
                double F = (1.0 - R) * (n * E0[d] + JxB[d]);
                E[d] = PREC == MHDPIC_PREC_MIXED ? E0[d] - F * ing : E0[d] - F / ng;
            }
        }
        float em, bm;   // |E| and |B| for the per-box maxima
        if (PREC == MHDPIC_PREC_MIXED) {
            int ci[3];
            decode_cell(b, (int32_t)(g - b.cell0), ci);
            const float4 fa = make_float4((float)E[0], (float)E[1], (float)E[2], (float)Bc[0]);
            const float2 fb = make_float2((float)Bc[1], (float)Bc[2]);
            store_fields_mixed(c.fa, c.fb, b, ci[0], ci[1], ci[2], fa, fb);
            em = sqrtf(fa.x * fa.x + fa.y * fa.y + fa.z * fa.z);
            bm = sqrtf(fa.w * fa.w + fb.x * fb.x + fb.y * fb.y);
        } else {
            double2 *f = reinterpret_cast<double2 *>(c.f64) + 3 * g;
            f[0] = make_double2(E[0], E[1]);
            f[1] = make_double2(E[2], Bc[0]);
            f[2] = make_double2(Bc[1], Bc[2]);
            em = (float)sqrt(E[0] * E[0] + E[1] * E[1] + E[2] * E[2]);
            bm = (float)sqrt(Bc[0] * Bc[0] + Bc[1] * Bc[1] + Bc[2] * Bc[2]);
        }
        for (int q = 0; q < 4; ++q)
            mnext[q * nc + g] = 0ull;
        // per-box maxima of |E| and |B| for the corrector scales
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
__device__ __forceinline__ void scales_box(const Ctx &c, int bx, double dt)
{
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

}  // namespace mhdpic
