// Allocation-free charge and current deposit (mhdpic_deposit_moments_noalloc).
//
// Some callers cannot allocate device memory once they are running: codes
// with a fixed device-memory budget reserved at start-up, allocation-free hot
// loops in a host code's time stepper, or call sites where the implicit device
// synchronisation of cudaMalloc/cudaFree is not acceptable.  This entry point
// does the same TSC deposit of n_CR and J_CR as mhdpic_deposit but needs no
// context and no cudaMalloc: its int64 fixed-point accumulators, per-cell
// counts and scales live in one file-scope device array (about 9 MiB for
// MHDPIC_NOALLOC_MAX_CELLS cells) that every GPU loading the library holds
// until the process exits.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include "device_common.cuh"

namespace {

constexpr int MAX_DEVICES = 64;

// The shared scratch, one array: four planes of int64 fixed-point sums, then
// the per-cell particle counts (int32), the densest-cell count and the four
// scales with their inverses (double).  In host code the name below is only a
// host-side stand-in; the kernels receive the device address obtained once per
// device with cudaGetSymbolAddress.
constexpr int64_t ACC_WORDS = 4ll * MHDPIC_NOALLOC_MAX_CELLS;
constexpr int64_t COUNT_WORDS = MHDPIC_NOALLOC_MAX_CELLS / 2;   // int32 counts, two per word
constexpr int64_t MISC_WORDS = 16;                              // maxcount, 4 scales, 4 inverses
static __device__ __align__(256) unsigned long long g_noalloc_scratch[ACC_WORDS + COUNT_WORDS + MISC_WORDS];

struct ScratchView {
    unsigned long long *acc;
    int32_t *count;
    int32_t *maxcount;
    double *scale;      // [4], then the inverses [4]
};

__host__ __device__ inline ScratchView view_of(unsigned long long *base)
{
    ScratchView v;
    v.acc = base;
    v.count = reinterpret_cast<int32_t *>(base + ACC_WORDS);
    v.maxcount = reinterpret_cast<int32_t *>(base + ACC_WORDS + COUNT_WORDS);
    v.scale = reinterpret_cast<double *>(base + ACC_WORDS + COUNT_WORDS + 2);
    return v;
}

std::mutex g_setup_mutex;
std::atomic<unsigned long long *> g_acc_ptr[MAX_DEVICES];

// The message goes to the library's per-thread last-error string.
int noalloc_fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    mhdpic::set_last_error(buf);
    return code;
}

struct NoallocBox {
    int n[3], bc[3], ndim;
    double x0[3], inv_dx[3];
    double qn, C;
    mhdpic::FastDiv div_nx, div_nxy;
};

// Cell of a particle (box coordinates), or false when it lies outside the box.
template <int PREC, int D>
__device__ __forceinline__ bool particle_cell(const NoallocBox &b, int64_t np, int64_t i, const int4 *pos,
                                              const double *x, int ci[3], int64_t ncell)
{
    if (PREC == MHDPIC_PREC_MIXED) {
        int32_t cl = __ldg(&pos[i].x);
        if (cl < 0 || cl >= ncell)
            return false;
        uint32_t uc = (uint32_t)cl;
        uint32_t k = mhdpic::fdiv(uc, b.div_nxy);
        uint32_t r = uc - k * b.div_nxy.d;
        uint32_t j = mhdpic::fdiv(r, b.div_nx);
        ci[0] = (int)(r - j * b.div_nx.d);
        ci[1] = (int)j;
        ci[2] = (int)k;
    } else {
        if (isnan(x[i]))   // left the box through an open face
            return false;
        for (int d = 0; d < D; ++d)
            ci[d] = (int)floor((x[(int64_t)d * np + i] - b.x0[d]) * b.inv_dx[d]);
    }
    return true;
}

// particles per cell (cells outside the box are folded in like the stencil)
template <int PREC, int D>
__global__ void k_noalloc_count(NoallocBox b, int64_t np, const int4 *__restrict__ pos,
                                const double *__restrict__ x, ScratchView v, int64_t ncell)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        int ci[3] = {0, 0, 0};
        if (!particle_cell<PREC, D>(b, np, i, pos, x, ci, ncell))
            continue;
        int gx = mhdpic::map_coord(ci[0], b.n[0], b.bc[0]);
        int gy = mhdpic::map_coord(ci[1], b.n[1], b.bc[1]);
        int gz = D == 3 ? mhdpic::map_coord(ci[2], b.n[2], b.bc[2]) : 0;
        atomicAdd(v.count + ((int64_t)gz * b.n[1] + gy) * b.n[0] + gx, 1);
    }
}

__global__ void k_noalloc_maxcount(ScratchView v, int64_t ncell)
{
    int mx = 0;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ncell; g += (int64_t)gridDim.x * blockDim.x)
        mx = max(mx, v.count[g]);
    for (int o = 16; o > 0; o >>= 1)
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(v.maxcount, mx);
}

// Scales sized from the densest cell: a cell receives at most 3^D x maxcount
// contributions, each |n| <= |qn| and |J| <= |qn| C; sums stay below 2^62.
__global__ void k_noalloc_scales(NoallocBox b, ScratchView v)
{
    double H = (b.ndim == 3 ? 27.0 : 9.0) * (double)max(*v.maxcount, 1);
    double qb[4] = {fabs(b.qn), fabs(b.qn) * b.C, fabs(b.qn) * b.C, fabs(b.qn) * b.C};
    for (int k = 0; k < 4; ++k) {
        int e;
        frexp(4611686018427387904.0 / (fmax(qb[k], 1e-30) * H), &e);
        e -= 1;
        if (e > mhdpic::SCALE_EXP_MAX)
            e = mhdpic::SCALE_EXP_MAX;
        v.scale[k] = ldexp(1.0, e);
        v.scale[4 + k] = ldexp(1.0, -e);
    }
}

// n = qm m W / dV, J = qm m u W / dV (App. A.1, eq:nJCR), into int64 fixed point
template <int PREC, int D>
__global__ void k_noalloc_deposit(NoallocBox b, int64_t np, const int4 *__restrict__ pos,
                                  const float4 *__restrict__ vel, const double *__restrict__ x,
                                  const double *__restrict__ p64, ScratchView sv, int64_t ncell)
{
    unsigned long long *__restrict__ acc = sv.acc;
    const double sc[4] = {sv.scale[0], sv.scale[1], sv.scale[2], sv.scale[3]};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        int ci[3] = {0, 0, 0};
        double w[3][3] = {{0, 1, 0}, {0, 1, 0}, {0, 1, 0}};
        double v[3];
        if (PREC == MHDPIC_PREC_MIXED) {
            if (!particle_cell<PREC, D>(b, np, i, pos, x, ci, ncell))
                continue;   // outside the box: contributes nothing
            const int4 ps = pos[i];
            const float o[3] = {__int_as_float(ps.y), __int_as_float(ps.z), __int_as_float(ps.w)};
            const float4 vs = vel[i];
            for (int d = 0; d < D; ++d)
                mhdpic::tsc_from_offset<double>((double)o[d], w[d]);
            for (int d = 0; d < 3; ++d)
                v[d] = mhdpic::vel_f64(vs, d);
        } else {
            if (isnan(x[i]))   // left the box through an open face
                continue;
            for (int d = 0; d < D; ++d) {
                double s = (x[(int64_t)d * np + i] - b.x0[d]) * b.inv_dx[d];
                double f = floor(s);
                ci[d] = (int)f;
                mhdpic::tsc_from_offset<double>(s - f, w[d]);
            }
            for (int d = 0; d < 3; ++d)
                v[d] = p64[(int64_t)d * np + i];
        }
        double gam = sqrt(b.C * b.C + v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / b.C;
        double q[4] = {b.qn, b.qn * (v[0] / gam), b.qn * (v[1] / gam), b.qn * (v[2] / gam)};
        for (int k = 0; k < 4; ++k)
            q[k] *= sc[k];
        int gx[3], gy[3], gz[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a) {
            gx[a] = mhdpic::map_coord(ci[0] + a - 1, b.n[0], b.bc[0]);
            gy[a] = mhdpic::map_coord(ci[1] + a - 1, b.n[1], b.bc[1]);
            if (D == 3)
                gz[a] = mhdpic::map_coord(ci[2] + a - 1, b.n[2], b.bc[2]);
        }
        for (int cz = 0; cz < (D == 3 ? 3 : 1); ++cz)
            for (int cy = 0; cy < 3; ++cy)
                for (int cx = 0; cx < 3; ++cx) {
                    double ww = w[0][cx] * w[1][cy] * (D == 3 ? w[2][cz] : 1.0);
                    int64_t g = ((int64_t)gz[cz] * b.n[1] + gy[cy]) * b.n[0] + gx[cx];
                    for (int k = 0; k < 4; ++k)
                        mhdpic::red_add(acc + k * ncell + g, mhdpic::to_fixed(q[k] * ww));
                }
    }
}

__global__ void k_noalloc_to_double(ScratchView sv, int64_t ncell, double *__restrict__ out)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < 4 * ncell;
         g += (int64_t)gridDim.x * blockDim.x)
        out[g] = (double)(long long)sv.acc[g] * sv.scale[4 + g / ncell];
}

// The device address of the scratch array on the current device.  Outside a
// stream capture it is looked up again on every call (cheap), so that a
// device reset, which reloads the module, cannot leave a stale address; a
// call made while `st` is capturing uses the address of the last call on
// this device, since the lookup may load the module, which a capture does
// not allow.
int scratch_on_current_device(cudaStream_t st, unsigned long long **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return noalloc_fail(MHDPIC_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES)
        return noalloc_fail(MHDPIC_E_CAPACITY, "device %d beyond the %d devices supported", dev, MAX_DEVICES);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess)
        return noalloc_fail(MHDPIC_E_CUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(e));
    if (cap != cudaStreamCaptureStatusNone) {
        unsigned long long *ptr = g_acc_ptr[dev].load();
        if (!ptr)
            return noalloc_fail(MHDPIC_E_STATE, "the first call on a device must come before any stream capture");
        *out = ptr;
        return MHDPIC_OK;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    void *addr = nullptr;
    e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
    if (e != cudaSuccess || !addr)
        return noalloc_fail(MHDPIC_E_CUDA, "cudaGetSymbolAddress of the scratch array: %s", cudaGetErrorString(e));
    g_acc_ptr[dev].store((unsigned long long *)addr);
    *out = (unsigned long long *)addr;
    return MHDPIC_OK;
}

}  // namespace

extern "C" {

int mhdpic_deposit_moments_noalloc(const mhdpic_grid *grid, const mhdpic_params *params, int32_t precision,
                                   int64_t np, const mhdpic_pos *pos_in, const mhdpic_vel *vel_in,
                                   const double *x, const double *p64, double *out, void *stream)
{
    if (!grid || !params || !out)
        return noalloc_fail(MHDPIC_E_ARG, "grid, params and out must be non-NULL");
    if (grid->ndim != 2 && grid->ndim != 3)
        return noalloc_fail(MHDPIC_E_ARG, "ndim must be 2 or 3 (got %d)", grid->ndim);
    if (precision != MHDPIC_PREC_MIXED && precision != MHDPIC_PREC_FP64)
        return noalloc_fail(MHDPIC_E_ARG, "unknown precision %d", precision);
    for (int d = 0; d < 3; ++d) {
        if (grid->n[d] < 1 || !(grid->dx[d] > 0.0))
            return noalloc_fail(MHDPIC_E_ARG, "n[%d] must be >= 1 and dx[%d] > 0", d, d);
        if (grid->bc[d] != MHDPIC_BC_PERIODIC && grid->bc[d] != MHDPIC_BC_REFLECT &&
            grid->bc[d] != MHDPIC_BC_WALL_OPEN)
            return noalloc_fail(MHDPIC_E_ARG, "unknown boundary %d", grid->bc[d]);
        // each side on its own first, so that the product below cannot overflow
        if (grid->n[d] > MHDPIC_NOALLOC_MAX_CELLS)
            return noalloc_fail(MHDPIC_E_CAPACITY,
                                "grid side n[%d] = %d exceeds the allocation-free limit of %d cells", d,
                                grid->n[d], MHDPIC_NOALLOC_MAX_CELLS);
    }
    if (grid->ndim == 2 && grid->n[2] != 1)
        return noalloc_fail(MHDPIC_E_ARG, "a 2-D grid must have n[2] == 1");
    const int64_t ncell = (int64_t)grid->n[0] * grid->n[1] * grid->n[2];   // < 2^54: no overflow
    if (ncell > MHDPIC_NOALLOC_MAX_CELLS)
        return noalloc_fail(MHDPIC_E_CAPACITY,
                            "grid of %lld cells exceeds the allocation-free limit of %d cells",
                            (long long)ncell, MHDPIC_NOALLOC_MAX_CELLS);
    if (np < 0 || np > 0x7fffffffLL)
        return noalloc_fail(MHDPIC_E_CAPACITY, "particle count %lld outside [0, 2^31)", (long long)np);
    if (np > 0 && (precision == MHDPIC_PREC_MIXED ? (!pos_in || !vel_in) : (!x || !p64)))
        return noalloc_fail(MHDPIC_E_ARG, "particle arrays of the chosen precision must be non-NULL");
    if (precision == MHDPIC_PREC_MIXED && (((uintptr_t)pos_in | (uintptr_t)vel_in) & 15u))
        return noalloc_fail(MHDPIC_E_ARG, "pos and vel must be 16-byte aligned");
    const int4 *pos = reinterpret_cast<const int4 *>(pos_in);
    const float4 *vel = reinterpret_cast<const float4 *>(vel_in);
    if (!(params->C > 0.0) || !std::isfinite(params->qm_cr) || !std::isfinite(params->m_cr))
        return noalloc_fail(MHDPIC_E_ARG, "C must be > 0, qm_cr and m_cr finite");

    unsigned long long *acc = nullptr;
    int rc = scratch_on_current_device((cudaStream_t)stream, &acc);
    if (rc)
        return rc;

    NoallocBox b{};
    b.ndim = grid->ndim;
    for (int d = 0; d < 3; ++d) {
        b.n[d] = grid->n[d];
        b.bc[d] = grid->bc[d];
        b.x0[d] = grid->x0[d];
        b.inv_dx[d] = 1.0 / grid->dx[d];
    }
    b.C = params->C;
    const double dV = grid->dx[0] * grid->dx[1] * grid->dx[2];
    b.qn = params->qm_cr * params->m_cr / dV;
    b.div_nx = mhdpic::make_fastdiv((uint32_t)grid->n[0]);
    b.div_nxy = mhdpic::make_fastdiv((uint32_t)(grid->n[0] * grid->n[1]));
    cudaStream_t st = (cudaStream_t)stream;
    const ScratchView sv = view_of(acc);
    // clear what must start at zero: the sums, the counts and the densest-cell count
    cudaError_t e = cudaMemsetAsync(sv.acc, 0, sizeof(unsigned long long) * 4 * ncell, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(sv.count, 0, sizeof(int32_t) * ncell, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(sv.maxcount, 0, sizeof(int32_t), st);
    if (e != cudaSuccess)
        return noalloc_fail(MHDPIC_E_CUDA, "clearing the scratch: %s", cudaGetErrorString(e));
    const int64_t blocks = (np + 255) / 256;
    const int pg = (int)(blocks < 1 ? 1 : (blocks < 152 * 32 ? blocks : 152 * 32));
    const int64_t cb = (ncell + 255) / 256;
    const int cg = (int)(cb < 152 * 32 ? cb : 152 * 32);
#define MHDPIC_NOALLOC_DISPATCH(KERNEL, ...)                                              \
    do {                                                                                  \
        if (precision == MHDPIC_PREC_MIXED) {                                             \
            if (grid->ndim == 3)                                                          \
                KERNEL<MHDPIC_PREC_MIXED, 3><<<pg, 256, 0, st>>>(__VA_ARGS__);            \
            else                                                                          \
                KERNEL<MHDPIC_PREC_MIXED, 2><<<pg, 256, 0, st>>>(__VA_ARGS__);            \
        } else {                                                                          \
            if (grid->ndim == 3)                                                          \
                KERNEL<MHDPIC_PREC_FP64, 3><<<pg, 256, 0, st>>>(__VA_ARGS__);             \
            else                                                                          \
                KERNEL<MHDPIC_PREC_FP64, 2><<<pg, 256, 0, st>>>(__VA_ARGS__);             \
        }                                                                                 \
    } while (0)
    if (np > 0)
        MHDPIC_NOALLOC_DISPATCH(k_noalloc_count, b, np, pos, x, sv, ncell);
    k_noalloc_maxcount<<<cg, 256, 0, st>>>(sv, ncell);
    k_noalloc_scales<<<1, 1, 0, st>>>(b, sv);
    if (np > 0)
        MHDPIC_NOALLOC_DISPATCH(k_noalloc_deposit, b, np, pos, vel, x, p64, sv, ncell);
#undef MHDPIC_NOALLOC_DISPATCH
    const int64_t ob = (4 * ncell + 255) / 256;
    k_noalloc_to_double<<<(int)(ob < 152 * 32 ? ob : 152 * 32), 256, 0, st>>>(sv, ncell, out);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return noalloc_fail(MHDPIC_E_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    return MHDPIC_OK;
}

}  // extern "C"
