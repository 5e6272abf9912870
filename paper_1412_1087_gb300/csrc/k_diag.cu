// Diagnostics of arXiv:1412.1087: particle spectra and E_max (Section 4.3,
// eq:dpdE, eq:emax) and the CR-Hall parameter map Lambda (Section 2.2,
// eq:defR, eq:lambda).
//
// The spectrum bins a per-particle quantity (E_k = v^2/(gamma+1) or |v|)
// against caller-given edges.  Every value that decides a bin or the region
// test is computed with explicitly rounded IEEE double operations in a fixed
// order (no contraction into FMAs), so the decision is reproducible exactly
// on any IEEE machine.  Counts are integers; the moment sums are reduced in a
// fixed order (per block of a fixed particle slice, then the slices in
// order), so repeated calls on the same state give identical results.
#include "device_common.cuh"

namespace mhdpic {

namespace {

constexpr int SPEC_THREADS = 256;

template <int PREC>
__global__ void __launch_bounds__(SPEC_THREADS) k_spectrum_partial(Ctx c, SpecArgs a, int nchunks, int64_t per_chunk,
                                                                    unsigned long long *__restrict__ counts,
                                                                    double *__restrict__ partials)
{
    __shared__ unsigned int hist[MHDPIC_SPEC_MAX_BINS];
    __shared__ double edges[MHDPIC_SPEC_MAX_BINS + 1];
    __shared__ double red[2][SPEC_THREADS];
    const int bx = blockIdx.y, chunk = blockIdx.x;
    const BoxDev &b = c.boxes[bx];
    const int nb = a.nbins;
    // each box takes as many of the nchunks slices as its size asks for;
    // the others add zeros
    const int nbc = box_chunks(b, per_chunk, nchunks);
    if (chunk >= nbc) {
        if (threadIdx.x < 2)
            partials[((int64_t)bx * nchunks + chunk) * 2 + threadIdx.x] = 0.0;
        return;
    }
    for (int i = threadIdx.x; i < nb; i += SPEC_THREADS)
        hist[i] = 0u;
    for (int i = threadIdx.x; i <= nb; i += SPEC_THREADS)
        edges[i] = a.edges[i];
    __syncthreads();

    const int64_t npb = b.part1 - b.part0;
    const int64_t ps = (npb + nbc - 1) / nbc;
    const int64_t p0 = b.part0 + chunk * ps, p1 = min(b.part1, p0 + ps);
    double s1 = 0.0, s0 = 0.0;
    for (int64_t i = p0 + threadIdx.x; i < p1; i += SPEC_THREADS) {
        if (particle_dead<PREC>(c, i))   // left the box
            continue;
        if (a.has_region) {
            bool inside = true;
            if (PREC == MHDPIC_PREC_MIXED) {
                int ci[3];
                const int4 ps = c.pos[i];
                const float o[3] = {__int_as_float(ps.y), __int_as_float(ps.z), __int_as_float(ps.w)};
                decode_cell(b, ps.x, ci);
                for (int d = 0; d < c.ndim; ++d) {
                    const double s = __dadd_rn((double)ci[d], (double)o[d]);
                    const double xd = __dadd_rn(b.x0[d], __dmul_rn(s, b.dx[d]));
                    inside &= xd >= a.region[2 * d] && xd < a.region[2 * d + 1];
                }
            } else {
                for (int d = 0; d < c.ndim; ++d) {
                    const double xd = c.x[(int64_t)d * c.np + i];
                    inside &= xd >= a.region[2 * d] && xd < a.region[2 * d + 1];
                }
            }
            if (!inside)
                continue;
        }
        double v[3];
        if (PREC == MHDPIC_PREC_MIXED) {
            const float4 vs = c.vel[i];   // the exact value of the two-word four-velocity
            for (int d = 0; d < 3; ++d)
                v[d] = vel_f64(vs, d);
        } else {
            for (int d = 0; d < 3; ++d)
                v[d] = c.p64[(int64_t)d * c.np + i];
        }
        double v2 = __dadd_rn(__dmul_rn(v[0], v[0]), __dmul_rn(v[1], v[1]));
        v2 = __dadd_rn(v2, __dmul_rn(v[2], v[2]));
        double q;
        if (a.kind == MHDPIC_SPEC_ENERGY) {
            const double gam = __ddiv_rn(__dsqrt_rn(__dadd_rn(__dmul_rn(b.C, b.C), v2)), b.C);
            q = __ddiv_rn(v2, __dadd_rn(gam, 1.0));
        } else {
            q = __dsqrt_rn(v2);
        }
        if (!(q >= edges[0] && q < edges[nb]))
            continue;
        // largest bin whose lower edge is <= q
        int lo = 0, hi = nb - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (edges[mid] <= q)
                lo = mid;
            else
                hi = mid - 1;
        }
        atomicAdd(&hist[lo], 1u);
        double qn = 1.0;
        for (int k = 0; k < a.n_moment; ++k)
            qn = __dmul_rn(qn, q);
        s1 += __dmul_rn(qn, q);
        s0 += qn;
    }
    red[0][threadIdx.x] = s1;
    red[1][threadIdx.x] = s0;
    __syncthreads();
    for (int s = SPEC_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x < 2)
        partials[((int64_t)bx * nchunks + chunk) * 2 + threadIdx.x] = red[threadIdx.x][0];
    for (int i = threadIdx.x; i < nb; i += SPEC_THREADS)
        if (hist[i])
            atomicAdd(counts + (int64_t)bx * nb + i, (unsigned long long)hist[i]);
}

__global__ void k_spectrum_final(int nbox, int nchunks, const double *__restrict__ partials,
                                 double *__restrict__ sums)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nbox * 2)
        return;
    const int bx = t / 2, q = t % 2;
    double s = 0.0;
    for (int k = 0; k < nchunks; ++k)
        s += partials[((int64_t)bx * nchunks + k) * 2 + q];
    sums[t] = s;
}

// Lambda = (J - n v_g) / ((n_g + n) v_A) per cell, from the latest charge and
// current deposit (moments buffer cur) and the gas.
__global__ void k_lambda(Ctx c, int cur, double *__restrict__ out)
{
    const unsigned long long *md = c.momdep[cur];
    const int64_t nc = c.nc;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nc;
         g += (int64_t)gridDim.x * blockDim.x) {
        const BoxDev &b = c.boxes[find_box(c.box_cell_start, c.nbox, g)];
        const double rho = c.rho[g];
        const double Bx = c.B[g], By = c.B[nc + g], Bz = c.B[2 * nc + g];
        const double vA = sqrt(Bx * Bx + By * By + Bz * Bz) / sqrt(rho);
        const double n = from_fixed(md[g], b.inv_scale[CH_N]);
        const double ng = b.qm_gas * rho;
        for (int d = 0; d < 3; ++d) {
            const double vg = c.mom[d * nc + g] / rho;
            const double J = from_fixed(md[(1 + d) * nc + g], b.inv_scale[CH_N + 1 + d]);
            out[d * nc + g] = vA > 0.0 ? (J - n * vg) / ((ng + n) * vA) : 0.0;
        }
    }
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

int launch_spectrum(const Ctx &c, const SpecArgs &a, int nchunks, int64_t per_chunk, unsigned long long *counts,
                    double *partials,
                    double *sums, cudaStream_t st)
{
    cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * (size_t)c.nbox * a.nbins, st);
    dim3 grid(nchunks, c.nbox);
    if (c.prec == MHDPIC_PREC_MIXED)
        k_spectrum_partial<MHDPIC_PREC_MIXED><<<grid, SPEC_THREADS, 0, st>>>(c, a, nchunks, per_chunk, counts, partials);
    else
        k_spectrum_partial<MHDPIC_PREC_FP64><<<grid, SPEC_THREADS, 0, st>>>(c, a, nchunks, per_chunk, counts, partials);
    k_spectrum_final<<<(c.nbox * 2 + 255) / 256, 256, 0, st>>>(c.nbox, nchunks, partials, sums);
    return 2;
}

int launch_lambda(const Ctx &c, int cur, double *out, cudaStream_t st)
{
    k_lambda<<<grid_for(c.nc, 256), 256, 0, st>>>(c, cur, out);
    return 1;
}

}  // namespace mhdpic
