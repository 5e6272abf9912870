// C ABI of the sm_103a MHD-PIC cosmic-ray particle library (include/mhdpic.h).
//
// Host-side only: argument validation, the box table, scratch allocation,
// host<->device staging of caller buffers in MEM_HOST mode, and the order of
// the kernel launches of each entry point.  All arithmetic runs in the
// kernels of k_push.cu, k_cells.cu and k_sort.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "mhdpic_internal.cuh"

using namespace mhdpic;

namespace {

// default wait limit of the kernels' tensor copies (one second)
constexpr int64_t COPY_LIMIT_DEFAULT_NS = 1000000000ll;

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *where)
{
    return fail(MHDPIC_E_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess)                     \
            return cuda_fail(e_, #call);           \
    } while (0)

}  // namespace

void mhdpic::set_last_error(const char *msg)
{
    g_last_error = msg;
}

struct mhdpic_ctx {
    Ctx k{};
    SortScratch s{};
    cudaStream_t stream = nullptr;
    int nbox = 0;
    int mem = MHDPIC_MEM_DEVICE;
    int cur = 0;              // moments buffer holding the latest deposit
    bool next_clear = false;  // buffer cur^1 is known to be zero (the stage kernel clears it)
    int grid_blocks = 0;      // persistent push grid
    int nchunks = 0;          // totals reduction slices per box, at most
    int64_t chunk_work = 1;   // particles + cells per slice (chunked reductions)
    int32_t *work_ctr = nullptr;
    double *partials = nullptr;
    double *totals_dev = nullptr;
    unsigned long long *spec_counts = nullptr;   // [nbox][MHDPIC_SPEC_MAX_BINS]
    int spec_chunks = 0;                         // particle slices per box of the spectrum
    double *spec_partials = nullptr;             // [nbox][spec_chunks][2]
    double *spec_edges = nullptr;                // [MHDPIC_SPEC_MAX_BINS + 1]
    int64_t launches = 0;
    int64_t fail_countdown = 0;   // mhdpic_debug_fail_launch: launch checks left before a reported failure
    // one-launch steps of mhdpic_run (mixed precision): the grid barrier, its
    // wait limit, the co-resident grid, and whether they are used
    GridBarrier *bar = nullptr;
    long long bar_limit_ns = 1000000000ll;
    int step_grid = 0;
    bool fuse = true;
    // staged mixed-precision fields: padded planes, their tensor maps
    int64_t fcells = 0;
    unsigned char *tmaps = nullptr;   // device, 2 CUtensorMap (128 B) per box
    bool tma_ok = false;              // the maps could be encoded for this layout
    // look-ahead sort: per box {t/dx, t/dy, t/dz, 1/C^2} in FP32 (device copy
    // in k.sort_k) for the look-ahead in use, k.sort_ahead; the caller's
    // look-ahead per sort (mhdpic_sort), scaled by the cadence in mhdpic_run
    std::vector<float4> sort_k_host;
    float4 *sort_k = nullptr;
    double ahead_user = 0.0;
    std::vector<BoxDev> boxes;
    std::vector<int64_t> part_start, cell_start, brick_start;
    std::vector<void *> allocs;
    // particle sets: 0 = the caller's buffers (their device mirrors in
    // MEM_HOST mode), 1 = the library's second set; k's particle pointers
    // are sets[cur_set]'s.  A sort only computes the permutation (pending);
    // the next push reads through it from the current set and writes the
    // other one, which then becomes current.
    PSet sets[2]{};
    int cur_set = 0;
    bool pending = false;
    int sub_sort_every = 0;   // interp_push re-sorts every this many sub-steps (0: never)
    // caller's host buffers in MEM_HOST mode
    mhdpic_particles hp{};
    mhdpic_gas hg{};
    bool valid = false;
    // mhdpic_run: captured step cycle and sort cadence
    cudaGraphExec_t graph = nullptr;
    double graph_dt = 0.0;
    int graph_k = 0;
    int graph_cur = -1;
    int graph_set = -1;
    bool graph_pending = false;
    int64_t graph_launches = 0;   // kernel launches inside one replay
    int step_in_cycle = 0;        // steps since the last sort done by mhdpic_run
    int tuned_k = 0;
    bool has_open = false;   // a box has an open face: particles can leave
    void *inj_state = nullptr;      // device injection state
    double *inj_scratch = nullptr;
    uint32_t inj_calls = 0;
    unsigned long long *live_dev = nullptr;
    // early-particle removal: injection times in both sets, clock {t, t_early}
    bool track_tinj = false;
    double *clock = nullptr;
    // coupled step: half state of the last mhdpic_gas_predict
    double *gas_half = nullptr;
    bool half_valid = false;
    // the gas changed since the fields were last staged (mhdpic_gas_correct,
    // mhdpic_inject): the next push stages them from the current gas first
    bool fields_stale = false;
    double half_dt = 0.0;
    int half_model = -1;
    // MEM_HOST_GAS: a feedback right after a push uploads the gas on
    // copy_stream while the push runs (the push reads only the staged
    // fields): copy_stream waits for ev_push, recorded before the push, and
    // the stream waits for ev_h2d before the feedback
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_push = nullptr, ev_h2d = nullptr;
    // MEM_DEVICE, a sort every step: the feedback runs on side_stream beside
    // the sort that follows the push (ev_fork after the push, ev_join after
    // the feedback)
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool push_marked = false;       // ev_push marks the work before the last push
    uint64_t gas_copies = 0;        // gas copies enqueued so far
    uint64_t gas_copies_push = 0;   // ... when the last push was enqueued
    int64_t launches_push = 0;      // kernel launches when the last push was enqueued

    template <typename T>
    int alloc(T **p, size_t count)
    {
        *p = nullptr;
        if (count == 0)
            count = 1;
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, sizeof(T) * count);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(MHDPIC_E_NOMEM, "cudaMalloc of %zu bytes failed: %s", sizeof(T) * count,
                        cudaGetErrorString(e));
        }
        allocs.push_back(q);
        *p = (T *)q;
        return MHDPIC_OK;
    }

    size_t particle_bytes() const
    {
        return k.prec == MHDPIC_PREC_MIXED ? (size_t)(sizeof(int4) + sizeof(float4)) : (size_t)(8 * k.ndim + 24);
    }
};

namespace {

int check_launch(mhdpic_ctx *c, int n)
{
    c->launches += n;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e, "kernel launch");
    if (c->fail_countdown > 0 && --c->fail_countdown == 0)
        return fail(MHDPIC_E_CUDA, "kernel launch: failure injected by mhdpic_debug_fail_launch");
    return MHDPIC_OK;
}

int copy_particles(mhdpic_ctx *c, bool to_device)
{
    if (c->mem != MHDPIC_MEM_HOST || c->k.np == 0)
        return MHDPIC_OK;
    const int64_t np = c->k.np;
    cudaMemcpyKind kind = to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
    auto cp = [&](void *dev, void *host, size_t bytes) {
        return to_device ? cudaMemcpyAsync(dev, host, bytes, kind, c->stream)
                         : cudaMemcpyAsync(host, dev, bytes, kind, c->stream);
    };
    if (c->k.prec == MHDPIC_PREC_MIXED) {
        CK(cp(c->k.pos, c->hp.pos, sizeof(int4) * np));
        CK(cp(c->k.vel, c->hp.vel, sizeof(float4) * np));
    } else {
        CK(cp(c->k.x, c->hp.x, sizeof(double) * c->k.ndim * np));
        CK(cp(c->k.p64, c->hp.p64, sizeof(double) * 3 * np));
    }
    return MHDPIC_OK;
}

// all: rho, mom, egas, B; otherwise only the arrays the feedback changes
int copy_gas(mhdpic_ctx *c, bool to_device, bool all, cudaStream_t st)
{
    if (c->mem == MHDPIC_MEM_DEVICE)
        return MHDPIC_OK;
    ++c->gas_copies;
    const int64_t nc = c->k.nc;
    if (to_device) {
        if (all) {
            CK(cudaMemcpyAsync(c->k.rho, c->hg.rho, sizeof(double) * nc, cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(c->k.B, c->hg.B, sizeof(double) * 3 * nc, cudaMemcpyHostToDevice, st));
        }
        CK(cudaMemcpyAsync(c->k.mom, c->hg.mom, sizeof(double) * 3 * nc, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(c->k.egas, c->hg.egas, sizeof(double) * nc, cudaMemcpyHostToDevice, st));
    } else {
        CK(cudaMemcpyAsync(c->hg.mom, c->k.mom, sizeof(double) * 3 * nc, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(c->hg.egas, c->k.egas, sizeof(double) * nc, cudaMemcpyDeviceToHost, st));
    }
    return MHDPIC_OK;
}

int copy_gas(mhdpic_ctx *c, bool to_device, bool all)
{
    return copy_gas(c, to_device, all, c->stream);
}

// The gas upload of a feedback, for the feedback enqueued next on stream
// `waiter`.  Right after a push (nothing launched and no gas copied since it
// was enqueued) in MEM_HOST_GAS mode it runs on copy_stream, after the work
// enqueued before the push and beside the push itself, which reads only the
// staged fields; `waiter` then waits for it.  Otherwise it is enqueued on
// `waiter`.
int upload_gas_for_feedback(mhdpic_ctx *c, cudaStream_t waiter)
{
    const bool beside = c->mem == MHDPIC_MEM_HOST_GAS && c->copy_stream && c->push_marked &&
                        c->launches == c->launches_push && c->gas_copies == c->gas_copies_push;
    c->push_marked = false;
    if (!beside)
        return copy_gas(c, true, true, waiter);
    CK(cudaStreamWaitEvent(c->copy_stream, c->ev_push, 0));
    int rc = copy_gas(c, true, true, c->copy_stream);
    if (rc)
        return rc;
    CK(cudaEventRecord(c->ev_h2d, c->copy_stream));
    CK(cudaStreamWaitEvent(waiter, c->ev_h2d, 0));
    return MHDPIC_OK;
}

void use_set(mhdpic_ctx *c, int set)
{
    c->cur_set = set;
    const PSet &q = c->sets[set];
    Ctx &k = c->k;
    k.pos = q.pos;
    k.vel = q.vel;
    k.x = q.x;
    k.p64 = q.p64;
    k.tinj = q.tinj;
    k.perm_src = nullptr;
    k.src_pos = q.pos;
    k.src_vel = q.vel;
    k.src_x = q.x;
    k.src_p64 = q.p64;
}

// Apply a pending sort to the particle arrays (gather into the other set).
int materialize(mhdpic_ctx *c)
{
    if (!c->pending)
        return MHDPIC_OK;
    int rc = check_launch(c, launch_gather(c->k, c->s.perm, c->sets[c->cur_set], c->sets[c->cur_set ^ 1], c->stream));
    if (rc)
        return rc;
    use_set(c, c->cur_set ^ 1);
    c->pending = false;
    return MHDPIC_OK;
}

// Materialize, then make the caller's buffers the current set.
int sync_to_caller(mhdpic_ctx *c)
{
    int rc;
    if ((rc = materialize(c)))
        return rc;
    if (c->cur_set == 0 || c->k.np == 0) {
        use_set(c, 0);
        return MHDPIC_OK;
    }
    const int64_t np = c->k.np;
    const PSet &a = c->sets[1], &b = c->sets[0];
    if (c->k.prec == MHDPIC_PREC_MIXED) {
        CK(cudaMemcpyAsync(b.pos, a.pos, sizeof(int4) * np, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(b.vel, a.vel, sizeof(float4) * np, cudaMemcpyDeviceToDevice, c->stream));
    } else {
        CK(cudaMemcpyAsync(b.x, a.x, sizeof(double) * c->k.ndim * np, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(b.p64, a.p64, sizeof(double) * 3 * np, cudaMemcpyDeviceToDevice, c->stream));
    }
    if (c->track_tinj)
        CK(cudaMemcpyAsync(b.tinj, a.tinj, sizeof(double) * np, cudaMemcpyDeviceToDevice, c->stream));
    use_set(c, 0);
    return MHDPIC_OK;
}

// Static scales of the charge / current channels: |n| <= |qm| m / dV and
// |J| <= |qm| m C / dV per particle, H = 3^D (4 maxcount + 64) per cell.
void moment_scales(mhdpic_ctx *c, int maxcount)
{
    const double H = (c->k.ndim == 3 ? 27.0 : 9.0) * (4.0 * maxcount + 64.0);
    for (auto &b : c->boxes) {
        double qn = std::fabs(b.qm_cr) * std::fabs(b.m_cr) * b.inv_dV;
        double q[4] = {qn, qn * b.C, qn * b.C, qn * b.C};
        for (int k = 0; k < 4; ++k) {
            double Q = std::fmax(q[k], 1e-30);
            int e;
            std::frexp(4611686018427387904.0 / (Q * H), &e);
            e -= 1;
            if (e > SCALE_EXP_MAX)
                e = SCALE_EXP_MAX;
            b.escale[CH_N + k] = e;
            b.scale[CH_N + k] = std::ldexp(1.0, e);
            b.inv_scale[CH_N + k] = std::ldexp(1.0, -e);
            b.qbound[CH_N + k] = Q;
            b.qmax[CH_N + k] = 4.0 * Q;
        }
        for (int k = 0; k < 4; ++k) {   // corrector: sized by the first push
            b.escale[k] = 0;
            b.scale[k] = 1.0;
            b.inv_scale[k] = 1.0;
            b.qbound[k] = 0.0;
            b.qmax[k] = 1e300;
        }
    }
}

int validate(int32_t nbox, const mhdpic_grid *grids, const mhdpic_params *params,
             const mhdpic_options *opt, const mhdpic_particles *parts, const mhdpic_gas *gas)
{
    if (nbox < 1)
        return fail(MHDPIC_E_ARG, "nbox must be >= 1 (got %d)", nbox);
    if (!grids || !params || !opt || !parts || !gas)
        return fail(MHDPIC_E_ARG, "grids, params, options, particles and gas must be non-NULL");
    if (opt->precision != MHDPIC_PREC_MIXED && opt->precision != MHDPIC_PREC_FP64)
        return fail(MHDPIC_E_ARG, "unknown precision %d", opt->precision);
    if (opt->memory != MHDPIC_MEM_DEVICE && opt->memory != MHDPIC_MEM_HOST && opt->memory != MHDPIC_MEM_HOST_GAS)
        return fail(MHDPIC_E_ARG, "unknown memory kind %d", opt->memory);
    if (!parts->box_start)
        return fail(MHDPIC_E_ARG, "particles.box_start must be a host array of nbox+1 offsets");
    if (parts->np < 0 || parts->np > 0x7fffffffLL)
        return fail(MHDPIC_E_CAPACITY, "particle count %lld outside [0, 2^31)", (long long)parts->np);
    if (parts->box_start[0] != 0 || parts->box_start[nbox] != parts->np)
        return fail(MHDPIC_E_ARG, "box_start must run from 0 to np");
    const int ndim = grids[0].ndim;
    int64_t nc = 0;
    for (int b = 0; b < nbox; ++b) {
        const mhdpic_grid &g = grids[b];
        const mhdpic_params &p = params[b];
        if (parts->box_start[b + 1] < parts->box_start[b])
            return fail(MHDPIC_E_ARG, "box_start must be non-decreasing (box %d)", b);
        if (g.ndim != ndim || (ndim != 2 && ndim != 3))
            return fail(MHDPIC_E_ARG, "box %d: ndim must be 2 or 3 and equal for all boxes", b);
        for (int d = 0; d < 3; ++d) {
            if (g.n[d] < 1)
                return fail(MHDPIC_E_ARG, "box %d: n[%d] must be >= 1", b, d);
            if (!(g.dx[d] > 0.0) || !std::isfinite(g.dx[d]) || !std::isfinite(g.x0[d]))
                return fail(MHDPIC_E_ARG, "box %d: dx[%d] must be finite and > 0", b, d);
            if (g.bc[d] != MHDPIC_BC_PERIODIC && g.bc[d] != MHDPIC_BC_REFLECT && g.bc[d] != MHDPIC_BC_WALL_OPEN)
                return fail(MHDPIC_E_ARG, "box %d: unknown boundary %d", b, g.bc[d]);
            if (g.bc[d] == MHDPIC_BC_WALL_OPEN && nbox != 1)
                return fail(MHDPIC_E_ARG, "MHDPIC_BC_WALL_OPEN needs a single-box context");
        }
        if (ndim == 2 && g.n[2] != 1)
            return fail(MHDPIC_E_ARG, "box %d: a 2-D box must have n[2] == 1", b);
        int64_t ncb = (int64_t)g.n[0] * g.n[1] * g.n[2];
        if (ncb > 0x7fffffffLL)
            return fail(MHDPIC_E_CAPACITY, "box %d: %lld cells exceed 2^31", b, (long long)ncb);
        nc += ncb;
        if (p.shape != MHDPIC_SHAPE_TSC)
            return fail(MHDPIC_E_ARG, "box %d: only MHDPIC_SHAPE_TSC is supported", b);
        if (!(p.C > 0.0) || !std::isfinite(p.C))
            return fail(MHDPIC_E_ARG, "box %d: C must be finite and > 0", b);
        if (!std::isfinite(p.qm_cr) || !std::isfinite(p.m_cr) || p.m_cr < 0.0)
            return fail(MHDPIC_E_ARG, "box %d: qm_cr must be finite and m_cr finite and >= 0", b);
        if (p.hall && !(p.qm_gas > 0.0))
            return fail(MHDPIC_E_ARG, "box %d: the CR-Hall term needs qm_gas > 0", b);
    }
    if (nc > 0x7fffffffLL)
        return fail(MHDPIC_E_CAPACITY, "%lld cells in total exceed 2^31", (long long)nc);
    if (opt->precision == MHDPIC_PREC_MIXED) {
        if (parts->np > 0 && (!parts->pos || !parts->vel))
            return fail(MHDPIC_E_ARG, "mixed precision needs particles.pos and .vel");
        if (((uintptr_t)parts->pos | (uintptr_t)parts->vel) & 15u)
            return fail(MHDPIC_E_ARG, "particles.pos and .vel must be 16-byte aligned");
    } else if (parts->np > 0 && (!parts->x || !parts->p64)) {
        return fail(MHDPIC_E_ARG, "FP64 needs particles.x and .p64");
    }
    if (!gas->rho || !gas->mom || !gas->egas || !gas->B)
        return fail(MHDPIC_E_ARG, "gas.rho, .mom, .egas and .B must be non-NULL");
    for (int d = 0; d < 3; ++d)
        if (opt->brick[d] < 0 || opt->brick[d] > 64)
            return fail(MHDPIC_E_ARG, "options.brick[%d] must be in [0, 64]", d);
    return MHDPIC_OK;
}

int do_prep(mhdpic_ctx *c, int apply)
{
    int rc = check_launch(c, launch_prep(c->k, c->cur, apply, c->stream));
    if (rc == MHDPIC_OK) {
        c->next_clear = true;
        c->fields_stale = false;
    }
    return rc;
}

// Tensor maps of the field planes, two per box (plane fa: 4 floats per cell,
// plane fb: 2), each a (floats per row, rows, layers) tensor over the box's
// padded block whose copy box is the push's field tile: (ts[1] cells, tile y,
// tile z).  Tiles start on cell org + FGHOST = brick origin, so the copies are
// used only when the brick's x extent is even (the innermost coordinate of the
// fb copy is then a multiple of 16 bytes) and the tile fits the copy limits;
// otherwise, or when the driver entry point is missing, the threads stage the
// tile.  Returns an error only for allocation or copy failures.
int setup_tensor_maps(mhdpic_ctx *c)
{
    Ctx &k = c->k;
    k.tma = 0;
    k.tmaps = nullptr;
    const int fsy = k.fts[1];
    if (k.brick[0] % 2 || fsy % 2 || 4 * fsy > 256 || k.tile[1] > 256 || k.tile[2] > 256)
        return MHDPIC_OK;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return MHDPIC_OK;
    }
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    std::vector<CUtensorMap> maps(2 * (size_t)c->nbox);
    const cuuint32_t rank = k.ndim == 3 ? 3 : 2;
    for (int b = 0; b < c->nbox; ++b) {
        const BoxDev &bd = c->boxes[b];
        for (int plane = 0; plane < 2; ++plane) {
            const int per = plane == 0 ? 4 : 2;   // floats per cell
            void *base = plane == 0 ? (void *)(k.fa + bd.fcell0) : (void *)(k.fb + bd.fcell0);
            const cuuint64_t dim[3] = {(cuuint64_t)per * bd.pn[0], (cuuint64_t)bd.pn[1], (cuuint64_t)bd.pn[2]};
            const cuuint64_t stride[2] = {(cuuint64_t)per * 4 * bd.pn[0], (cuuint64_t)per * 4 * bd.pn[0] * bd.pn[1]};
            const cuuint32_t box[3] = {(cuuint32_t)(per * fsy), (cuuint32_t)k.tile[1], (cuuint32_t)k.tile[2]};
            const cuuint32_t estr[3] = {1, 1, 1};
            CUresult r = encode(&maps[2 * b + plane], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, base, dim, stride, box,
                                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS)
                return MHDPIC_OK;   // this layout is not expressible: the threads stage the tiles
        }
    }
    int rc;
    if ((rc = c->alloc(&c->tmaps, maps.size() * sizeof(CUtensorMap))))
        return rc;
    CK(cudaMemcpy(c->tmaps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    k.tmaps = c->tmaps;
    k.tma = 1;
    c->tma_ok = true;
    return MHDPIC_OK;
}

// Make t the look-ahead of the next sorts: the FP32 key constants of every
// box, each rounded once to FP32 from its exact double (t/dx) or from two
// correctly rounded FP32 operations (1/(C C)).  Not during a capture.
int apply_lookahead(mhdpic_ctx *c, double t)
{
    if (t == c->k.sort_ahead)
        return MHDPIC_OK;
    for (int b = 0; b < c->nbox; ++b) {
        const BoxDev &bd = c->boxes[b];
        const float C = (float)bd.C;
        const float C2 = C * C;
        c->sort_k_host[b] = make_float4((float)(t * bd.inv_dx[0]), (float)(t * bd.inv_dx[1]),
                                        (float)(t * bd.inv_dx[2]), 1.f / C2);
    }
    CK(cudaMemcpyAsync(c->sort_k, c->sort_k_host.data(), sizeof(float4) * c->nbox, cudaMemcpyHostToDevice,
                       c->stream));
    c->k.sort_ahead = t;
    return MHDPIC_OK;
}

// The sort (mhdpic_sort) with whatever look-ahead is in use.
int do_sort(mhdpic_ctx *c, int64_t *perm_out, int32_t *counts_out)
{
    int rc;
    if ((rc = copy_particles(c, true)))
        return rc;
    // a permutation asked for is relative to the order the caller sees
    if (perm_out && (rc = materialize(c)))
        return rc;
    if ((rc = check_launch(c, launch_sort(c->k, c->s, perm_out, counts_out, c->stream))))
        return rc;
    c->pending = true;
    // refresh the densest-cell count used by the corrector scales
    if ((rc = check_launch(c, launch_max_count(c->k, c->s, c->stream))))
        return rc;
    if (c->mem == MHDPIC_MEM_HOST && (rc = materialize(c)))
        return rc;
    return copy_particles(c, false);
}

// Charge/current deposit of the current particles into moments buffer cur.
// Mixed precision goes through the push's tile over the work list of a sort
// of the current particles: the list is current when `listed` (right after
// a sort that has been applied), else a pending sort is used or one is made
// (the next push applies it).  FP64 uses the direct global-memory deposit.
int deposit_current(mhdpic_ctx *c, bool listed)
{
    int rc;
    if (c->k.prec != MHDPIC_PREC_MIXED) {
        if ((rc = materialize(c)))
            return rc;
        return check_launch(c, launch_moments(c->k, c->cur, c->stream));
    }
    Ctx kk = c->k;
    if (!listed) {
        if (!c->pending) {
            if ((rc = check_launch(c, launch_sort(c->k, c->s, nullptr, nullptr, c->stream))) ||
                (rc = check_launch(c, launch_max_count(c->k, c->s, c->stream))))
                return rc;
            c->pending = true;
        }
        kk.perm_src = c->s.perm;   // read through the permutation, write nothing
    }
    CK(cudaMemsetAsync(c->k.momdep[c->cur], 0, sizeof(unsigned long long) * 4 * c->k.nc, c->stream));
    return check_launch(c, launch_deposit_mixed(kk, c->s, c->work_ctr, c->cur, c->grid_blocks, c->stream));
}

// Stage the fields of the current gas when a call changed it since.
int restage_if_stale(mhdpic_ctx *c)
{
    if (!c->fields_stale)
        return MHDPIC_OK;
    int rc;
    if ((rc = copy_gas(c, true, true)))
        return rc;
    return do_prep(c, 0);
}

}  // namespace

extern "C" {

const char *mhdpic_strerror(int code)
{
    switch (code) {
    case MHDPIC_OK: return "success";
    case MHDPIC_E_ARG: return "invalid argument";
    case MHDPIC_E_CUDA: return "CUDA runtime error";
    case MHDPIC_E_NOMEM: return "device allocation failed";
    case MHDPIC_E_STATUS: return "a device status flag is set";
    case MHDPIC_E_CAPACITY: return "a size limit of the library was exceeded";
    case MHDPIC_E_STATE: return "call made in the wrong state";
    default: return "unknown error";
    }
}

const char *mhdpic_last_error(void) { return g_last_error.c_str(); }

int mhdpic_destroy(mhdpic_ctx *c)
{
    if (!c)
        return MHDPIC_OK;
    if (c->stream || c->valid)
        cudaStreamSynchronize(c->stream);
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
    }
    if (c->ev_push)
        cudaEventDestroy(c->ev_push);
    if (c->ev_h2d)
        cudaEventDestroy(c->ev_h2d);
    if (c->side_stream) {
        cudaStreamSynchronize(c->side_stream);
        cudaStreamDestroy(c->side_stream);
    }
    if (c->ev_fork)
        cudaEventDestroy(c->ev_fork);
    if (c->ev_join)
        cudaEventDestroy(c->ev_join);
    if (c->graph)
        cudaGraphExecDestroy(c->graph);
    for (void *p : c->allocs)
        cudaFree(p);
    c->valid = false;
    delete c;
    return MHDPIC_OK;
}

int mhdpic_init(mhdpic_ctx **out, int32_t nbox, const mhdpic_grid *grids, const mhdpic_params *params,
                const mhdpic_options *opt, const mhdpic_particles *parts, const mhdpic_gas *gas,
                void *stream)
{
    if (!out)
        return fail(MHDPIC_E_ARG, "ctx out-pointer is NULL");
    *out = nullptr;
    int rc = validate(nbox, grids, params, opt, parts, gas);
    if (rc)
        return rc;
    mhdpic_ctx *c = new mhdpic_ctx();
    auto bail = [&](int code) {
        mhdpic_destroy(c);
        return code;
    };
    c->stream = (cudaStream_t)stream;
    c->nbox = nbox;
    c->mem = opt->memory;
    c->k.copy_limit_ns = COPY_LIMIT_DEFAULT_NS;
    if (c->mem == MHDPIC_MEM_HOST_GAS) {
        cudaError_t e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&c->ev_push, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&c->ev_h2d, cudaEventDisableTiming);
        if (e != cudaSuccess)
            return bail(cuda_fail(e, "copy stream"));
    }
    if (c->mem == MHDPIC_MEM_DEVICE || c->mem == MHDPIC_MEM_HOST_GAS) {
        cudaError_t e = cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
        if (e != cudaSuccess)
            return bail(cuda_fail(e, "side stream"));
    }
    Ctx &k = c->k;
    k.nbox = nbox;
    k.ndim = grids[0].ndim;
    k.prec = opt->precision;
    k.np = parts->np;
    for (int d = 0; d < 3; ++d) {
        int def = k.ndim == 3 ? 4 : (d < 2 ? 8 : 1);
        k.brick[d] = opt->brick[d] > 0 ? opt->brick[d] : def;
        if (d >= k.ndim)
            k.brick[d] = 1;
        k.tile[d] = d < k.ndim ? k.brick[d] + 2 * HALO : 1;
        k.brick_sh[d] = -1;
        for (int sh = 0; sh < 31; ++sh)
            if (k.brick[d] == (1 << sh))
                k.brick_sh[d] = sh;
    }
    k.tile_vol = k.tile[0] * k.tile[1] * k.tile[2];
    // Default 64-cell bricks are worked as two 32-cell halves, one lane per
    // cell; the tile strides are padded so those 32 cells hit 32 banks.
    k.halves = 0;
    k.ts[0] = 1;
    k.ts[1] = k.tile[0];
    k.ts[2] = k.tile[0] * k.tile[1];
    if (k.ndim == 3 && k.brick[0] == 4 && k.brick[1] == 4 && k.brick[2] == 4) {
        k.halves = 1;
        k.ts[1] = 12;    // (x + 12 y + 112 z) mod 32 is a bijection of a 4x4x2 half
        k.ts[2] = 112;
    } else if (k.ndim == 2 && k.brick[0] == 8 && k.brick[1] == 8) {
        k.halves = 1;
        k.ts[1] = 24;    // (x + 24 y) mod 32 is a bijection of an 8x4 half
        k.ts[2] = 24 * k.tile[1];
    }
    k.tile_slots = k.ndim == 3 ? k.ts[2] * k.tile[2] : k.ts[1] * k.tile[1];
    // the field tile: x stride 1, y stride ts[1] (the bank spread the
    // gathers need), z dense, as one tensor copy of a (ts[1], tile y, tile z)
    // box writes it
    k.fts[0] = 1;
    k.fts[1] = k.ts[1];
    k.fts[2] = k.ts[1] * k.tile[1];
    k.ftile_slots = k.fts[2] * k.tile[2];
    size_t smem = k.prec == MHDPIC_PREC_MIXED ? push_smem_bytes_mixed(k) : push_smem_bytes_f64(k);
    if (smem > 200 * 1024)
        return bail(fail(MHDPIC_E_CAPACITY, "brick %dx%dx%d needs %zu bytes of shared memory", k.brick[0],
                         k.brick[1], k.brick[2], smem));

    // box table
    c->part_start.assign(parts->box_start, parts->box_start + nbox + 1);
    c->cell_start.assign(nbox + 1, 0);
    c->brick_start.assign(nbox + 1, 0);
    int64_t key0 = 0;
    for (int b = 0; b < nbox; ++b) {
        const mhdpic_grid &g = grids[b];
        const mhdpic_params &p = params[b];
        BoxDev bd{};
        for (int d = 0; d < 3; ++d) {
            bd.n[d] = g.n[d];
            bd.bc[d] = g.bc[d];
            bd.dx[d] = g.dx[d];
            bd.inv_dx[d] = 1.0 / g.dx[d];
            bd.x0[d] = g.x0[d];
            bd.nb[d] = (g.n[d] + k.brick[d] - 1) / k.brick[d];
        }
        bd.ndim = g.ndim;
        bd.hall = p.hall;
        bd.dV = g.dx[0] * g.dx[1] * g.dx[2];
        bd.inv_dV = 1.0 / bd.dV;
        bd.qm_cr = p.qm_cr;
        bd.qm_gas = p.qm_gas;
        bd.C = p.C;
        bd.m_cr = p.m_cr;
        bd.ncell = (int64_t)g.n[0] * g.n[1] * g.n[2];
        bd.cell0 = c->cell_start[b];
        c->cell_start[b + 1] = bd.cell0 + bd.ncell;
        bd.part0 = parts->box_start[b];
        bd.part1 = parts->box_start[b + 1];
        bd.nbricks = bd.nb[0] * bd.nb[1] * bd.nb[2];
        bd.brick0 = c->brick_start[b];
        c->brick_start[b + 1] = bd.brick0 + bd.nbricks;
        bd.key0 = key0;
        bd.nkeys = (int64_t)bd.nbricks * k.brick[0] * k.brick[1] * k.brick[2];
        key0 += bd.nkeys;
        bd.div_nx = make_fastdiv((uint32_t)g.n[0]);
        bd.div_nxy = make_fastdiv((uint32_t)(g.n[0] * g.n[1]));
        // padded staged-field planes: FGHOST ghosts below, and above up to
        // the brick grid's end plus FGHOST, so that every tile of the push
        // (bricks plus halo, periodic images included) lies inside; x rounded
        // up to even so that a row of the float2 plane is 16-byte aligned
        bd.pn[0] = (bd.nb[0] * k.brick[0] + 2 * FGHOST + 1) / 2 * 2;
        bd.pn[1] = bd.nb[1] * k.brick[1] + 2 * FGHOST;
        bd.pn[2] = g.ndim == 3 ? bd.nb[2] * k.brick[2] + 2 * FGHOST : 1;
        bd.fcell0 = c->fcells;
        c->fcells += (int64_t)bd.pn[0] * bd.pn[1] * bd.pn[2];
        c->boxes.push_back(bd);
    }
    k.nc = c->cell_start[nbox];
    k.nkeys = key0;
    k.nbricks_total = c->brick_start[nbox];
    if (k.nkeys >= 0x7fffffffLL)
        return bail(fail(MHDPIC_E_CAPACITY, "%lld sort keys exceed 2^31", (long long)k.nkeys));

    // device allocations
    const int64_t np = k.np, nc = k.nc;
    BoxDev *boxes_d;
    int64_t *ps_d, *cs_d;
    if ((rc = c->alloc(&boxes_d, nbox)) || (rc = c->alloc(&ps_d, nbox + 1)) || (rc = c->alloc(&cs_d, nbox + 1)) ||
        (rc = c->alloc(&c->s.brick_start, nbox + 1)) || (rc = c->alloc(&k.stats, nbox)))
        return bail(rc);
    k.boxes = boxes_d;
    k.boxes_rw = boxes_d;
    k.box_part_start = ps_d;
    k.box_cell_start = cs_d;
    if ((rc = c->alloc(&k.corr, 4 * nc)) || (rc = c->alloc(&k.momdep[0], 4 * nc)) ||
        (rc = c->alloc(&k.momdep[1], 4 * nc)) || (rc = c->alloc(&k.status, 1)))
        return bail(rc);
    if (k.prec == MHDPIC_PREC_MIXED) {
        if (!(rc = c->alloc(&k.fa, c->fcells)))
            rc = c->alloc(&k.fb, c->fcells);
    } else {
        rc = c->alloc(&k.f64, 6 * nc);
    }
    if (rc)
        return bail(rc);
    if (k.prec == MHDPIC_PREC_MIXED) {
        // zero the planes once: the columns added for alignment and tile cells
        // past a ragged box are never written by the staging but are copied
        if (cudaMemsetAsync(k.fa, 0, sizeof(float4) * c->fcells, c->stream) ||
            cudaMemsetAsync(k.fb, 0, sizeof(float2) * c->fcells, c->stream))
            return bail(cuda_fail(cudaGetLastError(), "init field planes"));
        if ((rc = setup_tensor_maps(c)))
            return bail(rc);
    }
    int64_t scan_n = std::max<int64_t>(k.nkeys, k.nbricks_total) / 4096 + 2;
    if ((rc = c->alloc(&c->s.count, k.nkeys + 2)) || (rc = c->alloc(&c->s.offset, k.nkeys + 2)) ||
        (rc = c->alloc(&c->s.pkey, np)) || (rc = c->alloc(&c->s.pslot, np)) || (rc = c->alloc(&c->s.perm, np)) ||
        (rc = c->alloc(&c->s.scan_tmp, scan_n)) || (rc = c->alloc(&c->s.big_list, k.nkeys + 1)) ||
        (rc = c->alloc(&c->s.big_count, 1)) ||
        (rc = c->alloc((char **)&c->s.tmp, (size_t)np * c->particle_bytes())) ||
        (rc = c->alloc(&c->s.brick_items, k.nbricks_total + 1)) ||
        (rc = c->alloc(&c->s.item_off, k.nbricks_total + 1)) ||
        // at most one item per brick, or per half of a crowded brick
        // ceil(n_half / ITEM_MAX_PARTICLES) <= n_half / ITEM_MAX_PARTICLES + 1
        (rc = c->alloc(&c->s.items, 2 * k.nbricks_total + np / ITEM_MAX_PARTICLES + 2)) ||
        (rc = c->alloc(&c->s.nitems, 1)) || (rc = c->alloc(&c->s.max_count, 1)) ||
        (rc = c->alloc(&c->work_ctr, 1)))
        return bail(rc);
    k.key_off = c->s.offset;
    // chunked reductions (totals, spectrum): about 8 blocks per SM over all
    // boxes, each box sliced in proportion to its particles and cells
    {
        int64_t work = 0, wmax = 0;
        for (int b = 0; b < nbox; ++b) {
            const int64_t w = (c->part_start[b + 1] - c->part_start[b]) + c->boxes[b].ncell;
            work += w;
            wmax = std::max(wmax, w);
        }
        c->chunk_work = std::max<int64_t>(1, (work + 1215) / 1216);
        c->nchunks = (int)std::max<int64_t>(1, std::min<int64_t>(1216, (wmax + c->chunk_work - 1) / c->chunk_work));
        c->spec_chunks = c->nchunks;
    }
    if ((rc = c->alloc(&c->sort_k, nbox)))
        return bail(rc);
    k.sort_k = c->sort_k;
    c->sort_k_host.assign(nbox, make_float4(0.f, 0.f, 0.f, 0.f));
    if ((rc = c->alloc(&c->partials, (size_t)nbox * c->nchunks * 8)) || (rc = c->alloc(&c->totals_dev, 8 * nbox)) ||
        (rc = c->alloc(&c->spec_counts, (size_t)nbox * MHDPIC_SPEC_MAX_BINS)) ||
        (rc = c->alloc(&c->spec_partials, (size_t)nbox * c->spec_chunks * 2)) ||
        (rc = c->alloc(&c->spec_edges, MHDPIC_SPEC_MAX_BINS + 1)))
        return bail(rc);

    // caller buffers (or device mirrors of host ones)
    PSet &s0 = c->sets[0], &s1 = c->sets[1];
    if (c->mem == MHDPIC_MEM_HOST) {
        c->hp = *parts;
        if (k.prec == MHDPIC_PREC_MIXED) {
            if ((rc = c->alloc(&s0.pos, np)) || (rc = c->alloc(&s0.vel, np)))
                return bail(rc);
        } else if ((rc = c->alloc(&s0.x, k.ndim * np)) || (rc = c->alloc(&s0.p64, 3 * np))) {
            return bail(rc);
        }
    } else {
        s0.pos = reinterpret_cast<int4 *>(parts->pos);
        s0.vel = reinterpret_cast<float4 *>(parts->vel);
        s0.x = parts->x;
        s0.p64 = parts->p64;
    }
    // the second set lives in the particle staging scratch
    {
        char *t = (char *)c->s.tmp;
        if (k.prec == MHDPIC_PREC_MIXED) {
            s1.pos = (int4 *)t;
            s1.vel = (float4 *)(t + sizeof(int4) * np);
        } else {
            s1.x = (double *)t;
            s1.p64 = s1.x + (size_t)k.ndim * np;
        }
    }
    use_set(c, 0);
    if (c->mem != MHDPIC_MEM_DEVICE) {
        c->hg = *gas;
        if ((rc = c->alloc(&k.rho, nc)) || (rc = c->alloc(&k.mom, 3 * nc)) || (rc = c->alloc(&k.egas, nc)) ||
            (rc = c->alloc(&k.B, 3 * nc)))
            return bail(rc);
    } else {
        k.rho = gas->rho;
        k.mom = gas->mom;
        k.egas = gas->egas;
        k.B = gas->B;
    }
    cudaStream_t st = c->stream;
    if ((rc = copy_particles(c, true)) || (rc = copy_gas(c, true, true)))
        return bail(rc);
    if (cudaMemcpyAsync(ps_d, c->part_start.data(), sizeof(int64_t) * (nbox + 1), cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(cs_d, c->cell_start.data(), sizeof(int64_t) * (nbox + 1), cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(c->s.brick_start, c->brick_start.data(), sizeof(int64_t) * (nbox + 1),
                        cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(boxes_d, c->boxes.data(), sizeof(BoxDev) * nbox, cudaMemcpyHostToDevice, st) ||
        cudaMemsetAsync(k.corr, 0, sizeof(unsigned long long) * 4 * nc, st) ||
        cudaMemsetAsync(k.momdep[0], 0, sizeof(unsigned long long) * 4 * nc, st) ||
        cudaMemsetAsync(k.momdep[1], 0, sizeof(unsigned long long) * 4 * nc, st) ||
        cudaMemsetAsync(k.status, 0, sizeof(uint32_t), st) || cudaMemsetAsync(k.stats, 0, sizeof(BoxStats) * nbox, st) ||
        // the second particle set and the sort's per-particle arrays start as
        // valid values (cell 0, key 0, slot 0, index 0): a launch that gives
        // up part of its work (MHDPIC_ST_COPY_TIMEOUT, MHDPIC_ST_BARRIER)
        // leaves stale but in-range entries behind, never raw memory
        cudaMemsetAsync(c->s.tmp, 0, (size_t)np * c->particle_bytes(), st) ||
        cudaMemsetAsync(c->s.pkey, 0, sizeof(int32_t) * np, st) ||
        cudaMemsetAsync(c->s.pslot, 0, sizeof(int32_t) * np, st) ||
        cudaMemsetAsync(c->s.perm, 0, sizeof(int32_t) * np, st))
        return bail(cuda_fail(cudaGetLastError(), "init uploads"));

    // sort (into the caller's buffers), then size the charge/current scales
    // from the densest cell
    if ((rc = check_launch(c, launch_sort(k, c->s, nullptr, nullptr, st))) ||
        (rc = check_launch(c, launch_max_count(k, c->s, st))))
        return bail(rc);
    c->pending = true;
    if ((rc = sync_to_caller(c)))
        return bail(rc);
    int32_t maxcount = 0;
    if (cudaMemcpyAsync(&maxcount, c->s.max_count, sizeof(int32_t), cudaMemcpyDeviceToHost, st) ||
        cudaStreamSynchronize(st))
        return bail(cuda_fail(cudaGetLastError(), "init max count"));
    moment_scales(c, maxcount);
    if (cudaMemcpyAsync(boxes_d, c->boxes.data(), sizeof(BoxDev) * nbox, cudaMemcpyHostToDevice, st))
        return bail(cuda_fail(cudaGetLastError(), "init scales"));
    std::vector<BoxStats> stats(nbox);
    for (auto &s : stats) {
        memset(&s, 0, sizeof s);
        s.maxcount = maxcount;
    }
    if (cudaMemcpyAsync(k.stats, stats.data(), sizeof(BoxStats) * nbox, cudaMemcpyHostToDevice, st) ||
        cudaStreamSynchronize(st))
        return bail(cuda_fail(cudaGetLastError(), "init stats"));

    int bps = k.prec == MHDPIC_PREC_MIXED ? push_blocks_per_sm_mixed(k) : push_blocks_per_sm_f64(k);
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    c->grid_blocks = bps * (nsm > 0 ? nsm : 1);
    if (k.prec == MHDPIC_PREC_MIXED) {
        int coop = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        c->step_grid = coop ? step_blocks_per_sm_mixed(k) * (nsm > 0 ? nsm : 1) : 0;
        if ((rc = c->alloc(&c->bar, 1)))
            return bail(rc);
        if (cudaMemsetAsync(c->bar, 0, sizeof(GridBarrier), st))
            return bail(cuda_fail(cudaGetLastError(), "init barrier"));
    }

    // moments at the initial positions, maxima, staged fields
    c->cur = 0;
    if ((rc = deposit_current(c, true)) || (rc = check_launch(c, launch_vmax(k, st))) ||
        (rc = do_prep(c, 0)))
        return bail(rc);
    if ((rc = copy_particles(c, false)))
        return bail(rc);
    for (int b = 0; b < nbox; ++b)
        for (int d = 0; d < 3; ++d)
            c->has_open |= grids[b].bc[d] == MHDPIC_BC_WALL_OPEN;
    c->valid = true;
    *out = c;
    return MHDPIC_OK;
}

int mhdpic_sort(mhdpic_ctx *c, int64_t *perm_out, int32_t *counts_out)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    int rc;
    if ((rc = apply_lookahead(c, c->ahead_user)))
        return rc;
    return do_sort(c, perm_out, counts_out);
}

int mhdpic_interp_push(mhdpic_ctx *c, double dt, int32_t nsub)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    if (!(dt > 0.0) || !std::isfinite(dt))
        return fail(MHDPIC_E_ARG, "dt must be finite and > 0");
    if (nsub < 1)
        return fail(MHDPIC_E_ARG, "nsub must be >= 1");
    int rc;
    if ((rc = copy_particles(c, true)) || (rc = restage_if_stale(c)))
        return rc;
    if (c->copy_stream) {   // everything before the push (see upload_gas_for_feedback)
        CK(cudaEventRecord(c->ev_push, c->stream));
        c->push_marked = false;
    }
    if ((rc = check_launch(c, launch_scales(c->k, dt, c->stream))))
        return rc;
    if (!c->next_clear)   // two pushes with no staging in between
        CK(cudaMemsetAsync(c->k.momdep[c->cur ^ 1], 0, sizeof(unsigned long long) * 4 * c->k.nc, c->stream));
    for (int s = 0; s < nsub; ++s) {
        bool last = s == nsub - 1;
        // after a sort the first push reads the current set through the
        // permutation and writes the other set
        Ctx kk = c->k;
        const bool gather = c->pending;
        if (gather) {
            const PSet &src = c->sets[c->cur_set], &dst = c->sets[c->cur_set ^ 1];
            kk.pos = dst.pos;
            kk.vel = dst.vel;
            kk.x = dst.x;
            kk.p64 = dst.p64;
            kk.tinj = dst.tinj;
            kk.perm_src = c->s.perm;
            kk.src_pos = src.pos;
            kk.src_vel = src.vel;
            kk.src_x = src.x;
            kk.src_p64 = src.p64;
            // the injection times follow the permutation before the push reads them
            if (c->track_tinj &&
                (rc = check_launch(c, launch_gather_f64(c->k.np, c->s.perm, src.tinj, dst.tinj, c->stream))))
                return rc;
        }
        // the push removes early particles at the time it reaches
        if (c->track_tinj && (rc = check_launch(c, launch_clock_advance(c->clock, dt, c->stream))))
            return rc;
        int n = c->k.prec == MHDPIC_PREC_MIXED
                    ? launch_push_mixed(kk, c->s, c->work_ctr, c->cur ^ 1, last ? 1 : 0, dt, c->grid_blocks, c->stream)
                    : launch_push_f64(kk, c->s, c->work_ctr, c->cur ^ 1, last ? 1 : 0, dt, c->grid_blocks, c->stream);
        if ((rc = check_launch(c, n)))
            return rc;
        if (gather) {
            use_set(c, c->cur_set ^ 1);
            c->pending = false;
            if (c->has_open && (rc = check_launch(c, launch_mark_free(c->k, c->s, c->stream))))
                return rc;
        }
        // re-sort between sub-steps (the next sub-step applies it)
        if (!last && c->sub_sort_every > 0 && (s + 1) % c->sub_sort_every == 0) {
            if ((rc = check_launch(c, launch_sort(c->k, c->s, nullptr, nullptr, c->stream))) ||
                (rc = check_launch(c, launch_max_count(c->k, c->s, c->stream))))
                return rc;
            c->pending = true;
        }
    }
    c->cur ^= 1;
    c->next_clear = false;
    if (c->copy_stream) {
        c->push_marked = true;
        c->launches_push = c->launches;
        c->gas_copies_push = c->gas_copies;
    }
    return copy_particles(c, false);
}

int mhdpic_deposit(mhdpic_ctx *c)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    int rc;
    if ((rc = copy_particles(c, true)) || (rc = copy_gas(c, true, true)))
        return rc;
    // the stage kernel clears buffer cur^1, so deposit into cur and stage from it
    if ((rc = deposit_current(c, false)) || (rc = check_launch(c, launch_vmax(c->k, c->stream))) ||
        (rc = do_prep(c, 0)))
        return rc;
    return MHDPIC_OK;
}

int mhdpic_apply_feedback(mhdpic_ctx *c, double *totals_out)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    int rc;
    if ((rc = upload_gas_for_feedback(c, c->stream)))
        return rc;
    if ((rc = do_prep(c, 1)))
        return rc;
    if ((rc = copy_gas(c, false, false)))
        return rc;
    if (totals_out) {
        if ((rc = copy_particles(c, true)) || (rc = materialize(c)))
            return rc;
        if ((rc = check_launch(c, launch_totals(c->k, c->partials, c->nchunks, c->chunk_work, c->totals_dev, c->stream))))
            return rc;
        CK(cudaMemcpyAsync(totals_out, c->totals_dev, sizeof(double) * 8 * c->nbox, cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return MHDPIC_OK;
}

int mhdpic_inject(mhdpic_ctx *c, double dt, double eta, double energy_factor, double gamma_gas, uint64_t seed,
                  double *front_out, int64_t *ninj_out)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    if (c->nbox != 1 || c->boxes[0].bc[0] != MHDPIC_BC_WALL_OPEN)
        return fail(MHDPIC_E_ARG, "mhdpic_inject needs a single box with MHDPIC_BC_WALL_OPEN along x");
    if (!(dt > 0.0) || !std::isfinite(dt) || !(eta >= 0.0) || !std::isfinite(eta) || !(energy_factor > 0.0) ||
        !std::isfinite(energy_factor) || !(gamma_gas > 1.0) || !std::isfinite(gamma_gas))
        return fail(MHDPIC_E_ARG, "dt, eta, energy_factor and gamma_gas must be finite with dt > 0, eta >= 0, "
                                  "energy_factor > 0, gamma_gas > 1");
    int rc;
    const int64_t nx = c->boxes[0].n[0];
    if (!c->inj_state) {
        std::vector<unsigned char> img(inject_state_bytes());
        init_inject_state(img.data());
        if ((rc = c->alloc(reinterpret_cast<unsigned char **>(&c->inj_state), img.size())) ||
            (rc = c->alloc(&c->inj_scratch, inject_scratch_doubles(nx))))
            return rc;
        CK(cudaMemcpyAsync(c->inj_state, img.data(), img.size(), cudaMemcpyHostToDevice, c->stream));
    }
    if ((rc = copy_particles(c, true)) || (rc = copy_gas(c, true, true)))
        return rc;
    // the free slots are those past the live particles of the last sort:
    // through its permutation while it is pending, in place once applied
    if ((rc = check_launch(c, launch_inject(c->k, c->s, c->inj_state, c->inj_scratch, nx, dt, eta, energy_factor,
                                            gamma_gas, seed, c->inj_calls, c->pending ? 1 : 0, c->stream))))
        return rc;
    ++c->inj_calls;
    c->fields_stale = true;   // the compensation changed the gas
    // the new particles into their cells
    if ((rc = check_launch(c, launch_sort(c->k, c->s, nullptr, nullptr, c->stream))) ||
        (rc = check_launch(c, launch_max_count(c->k, c->s, c->stream))))
        return rc;
    std::vector<unsigned char> img(inject_state_bytes());
    CK(cudaMemcpyAsync(img.data(), c->inj_state, img.size(), cudaMemcpyDeviceToHost, c->stream));
    if (c->mem != MHDPIC_MEM_DEVICE) {
        CK(cudaMemcpyAsync(c->hg.rho, c->k.rho, sizeof(double) * c->k.nc, cudaMemcpyDeviceToHost, c->stream));
        if ((rc = copy_gas(c, false, false)))
            return rc;
    }
    if (c->mem == MHDPIC_MEM_HOST && ((rc = materialize(c)) || (rc = copy_particles(c, false))))
        return rc;
    CK(cudaStreamSynchronize(c->stream));
    double fr[2];
    int64_t n = 0;
    int capped = 0;
    inject_outputs(img.data(), fr, &n, &capped);
    (void)capped;   // also raised on the device as MHDPIC_ST_INJECT_CAP
    if (front_out) {
        front_out[0] = fr[0];
        front_out[1] = fr[1];
    }
    if (ninj_out)
        *ninj_out = n;
    return MHDPIC_OK;
}

int mhdpic_set_injection_times(mhdpic_ctx *c, const double *t_inj, double t_now, double t_early)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    if (!std::isfinite(t_now) || std::isnan(t_early))
        return fail(MHDPIC_E_ARG, "t_now must be finite and t_early not NaN");
    int rc;
    // the caller's order: the caller's buffers made current
    if ((rc = copy_particles(c, true)) || (rc = sync_to_caller(c)))
        return rc;
    const int64_t np = c->k.np;
    if (!c->track_tinj) {
        if ((rc = c->alloc(&c->sets[0].tinj, np)) || (rc = c->alloc(&c->sets[1].tinj, np)) ||
            (rc = c->alloc(&c->clock, 2)))
            return rc;
        c->k.clock = c->clock;
        c->track_tinj = true;
        use_set(c, c->cur_set);
        if (c->graph) {   // a captured cycle has no removal in it
            cudaGraphExecDestroy(c->graph);
            c->graph = nullptr;
        }
    }
    if (np > 0) {
        if (t_inj) {
            CK(cudaMemcpyAsync(c->k.tinj, t_inj, sizeof(double) * np, cudaMemcpyHostToDevice, c->stream));
        } else {
            std::vector<double> never((size_t)np, std::numeric_limits<double>::infinity());
            CK(cudaMemcpyAsync(c->k.tinj, never.data(), sizeof(double) * np, cudaMemcpyHostToDevice, c->stream));
            CK(cudaStreamSynchronize(c->stream));
        }
    }
    const double clk[2] = {t_now, t_early};
    CK(cudaMemcpyAsync(c->clock, clk, sizeof clk, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MHDPIC_OK;
}

int mhdpic_get_injection_times(mhdpic_ctx *c, double *t_inj, double *t_now)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    if (!c->track_tinj)
        return fail(MHDPIC_E_STATE, "injection times are not tracked (mhdpic_set_injection_times)");
    int rc;
    if ((rc = copy_particles(c, true)) || (rc = sync_to_caller(c)))
        return rc;
    if (t_inj && c->k.np > 0)
        CK(cudaMemcpyAsync(t_inj, c->k.tinj, sizeof(double) * c->k.np, cudaMemcpyDeviceToHost, c->stream));
    double clk[2];
    CK(cudaMemcpyAsync(clk, c->clock, sizeof clk, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (t_now)
        *t_now = clk[0];
    return MHDPIC_OK;
}

int mhdpic_live_particles(mhdpic_ctx *c, int64_t *live_out)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    if (!live_out)
        return fail(MHDPIC_E_ARG, "live_out must be non-NULL");
    int rc;
    if (!c->live_dev && (rc = c->alloc(&c->live_dev, 1)))
        return rc;
    if ((rc = copy_particles(c, true)))
        return rc;
    if ((rc = check_launch(c, launch_count_live(c->k, c->live_dev, c->stream))))
        return rc;
    unsigned long long n = 0;
    CK(cudaMemcpyAsync(&n, c->live_dev, sizeof(n), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *live_out = (int64_t)n;
    return MHDPIC_OK;
}

int mhdpic_gas_predict(mhdpic_ctx *c, double dt, int32_t model)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    if (!(dt > 0.0) || !std::isfinite(dt))
        return fail(MHDPIC_E_ARG, "dt must be finite and > 0");
    if (model != MHDPIC_GAS_SOURCES && model != MHDPIC_GAS_LINEAR_X)
        return fail(MHDPIC_E_ARG, "unknown gas model %d", model);
    if (model == MHDPIC_GAS_LINEAR_X)
        for (int b = 0; b < c->nbox; ++b)
            if (c->boxes[b].bc[0] != MHDPIC_BC_PERIODIC)
                return fail(MHDPIC_E_ARG, "MHDPIC_GAS_LINEAR_X needs x-periodic boxes (box %d)", b);
    int rc;
    if (!c->gas_half && (rc = c->alloc(&c->gas_half, (size_t)8 * c->k.nc)))
        return rc;
    if ((rc = copy_gas(c, true, true)))
        return rc;
    if ((rc = check_launch(c, launch_gas_predict(c->k, c->cur, dt, model, c->gas_half, c->stream))))
        return rc;
    c->next_clear = true;
    c->fields_stale = false;
    c->half_valid = true;
    c->half_dt = dt;
    c->half_model = model;
    return MHDPIC_OK;
}

int mhdpic_gas_correct(mhdpic_ctx *c, double dt, int32_t model, double *totals_out)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    if (!c->half_valid)
        return fail(MHDPIC_E_STATE, "mhdpic_gas_correct needs a mhdpic_gas_predict first");
    if (dt != c->half_dt || model != c->half_model)
        return fail(MHDPIC_E_ARG, "dt and model must be the predictor's (%g, %d)", c->half_dt, c->half_model);
    int rc;
    if ((rc = copy_gas(c, true, true)))
        return rc;
    if ((rc = check_launch(c, launch_gas_correct(c->k, dt, model, c->gas_half, c->stream))))
        return rc;
    c->half_valid = false;
    c->fields_stale = true;
    if ((rc = copy_gas(c, false, false)))
        return rc;
    if (c->mem != MHDPIC_MEM_DEVICE)
        CK(cudaMemcpyAsync(c->hg.B, c->k.B, sizeof(double) * 3 * c->k.nc, cudaMemcpyDeviceToHost, c->stream));
    if (totals_out) {
        if ((rc = copy_particles(c, true)) || (rc = materialize(c)))
            return rc;
        if ((rc = check_launch(c, launch_totals(c->k, c->partials, c->nchunks, c->chunk_work, c->totals_dev, c->stream))))
            return rc;
        CK(cudaMemcpyAsync(totals_out, c->totals_dev, sizeof(double) * 8 * c->nbox, cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return MHDPIC_OK;
}

int mhdpic_spectrum(mhdpic_ctx *c, int32_t kind, int32_t nbins, const double *edges, const double *region,
                    int32_t n_moment, int64_t *counts_out, double *sums_out)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    if (kind != MHDPIC_SPEC_ENERGY && kind != MHDPIC_SPEC_MOMENTUM)
        return fail(MHDPIC_E_ARG, "unknown spectrum kind %d", kind);
    if (nbins < 1 || nbins > MHDPIC_SPEC_MAX_BINS)
        return fail(MHDPIC_E_ARG, "nbins must be in [1, %d]", MHDPIC_SPEC_MAX_BINS);
    if (!edges || !counts_out)
        return fail(MHDPIC_E_ARG, "edges and counts_out must be non-NULL");
    if (n_moment < 0 || n_moment > 64)
        return fail(MHDPIC_E_ARG, "n_moment must be in [0, 64]");
    for (int b = 0; b <= nbins; ++b)
        if (!std::isfinite(edges[b]) || (b > 0 && !(edges[b] > edges[b - 1])))
            return fail(MHDPIC_E_ARG, "edges must be finite and strictly ascending");
    SpecArgs a{};
    a.kind = kind;
    a.nbins = nbins;
    a.n_moment = n_moment;
    a.has_region = region != nullptr;
    for (int q = 0; q < 6; ++q)
        a.region[q] = region ? region[q] : 0.0;
    if (region)
        for (int d = 0; d < c->k.ndim; ++d)
            if (std::isnan(region[2 * d]) || std::isnan(region[2 * d + 1]))
                return fail(MHDPIC_E_ARG, "region bounds must not be NaN");
    a.edges = c->spec_edges;
    int rc;
    if ((rc = copy_particles(c, true)))
        return rc;
    CK(cudaMemcpyAsync(c->spec_edges, edges, sizeof(double) * (nbins + 1), cudaMemcpyHostToDevice, c->stream));
    if ((rc = check_launch(c, launch_spectrum(c->k, a, c->spec_chunks, c->chunk_work, c->spec_counts, c->spec_partials,
                                              c->totals_dev, c->stream))))
        return rc;
    static_assert(sizeof(unsigned long long) == sizeof(int64_t), "count width");
    CK(cudaMemcpyAsync(counts_out, c->spec_counts, sizeof(int64_t) * (size_t)c->nbox * nbins,
                       cudaMemcpyDeviceToHost, c->stream));
    if (sums_out)
        CK(cudaMemcpyAsync(sums_out, c->totals_dev, sizeof(double) * 2 * c->nbox, cudaMemcpyDeviceToHost,
                           c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MHDPIC_OK;
}

int mhdpic_lambda_map(mhdpic_ctx *c, double *out)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    if (!out)
        return fail(MHDPIC_E_ARG, "out must be non-NULL");
    int rc;
    if ((rc = copy_gas(c, true, true)))
        return rc;
    return check_launch(c, launch_lambda(c->k, c->cur, out, c->stream));
}

int mhdpic_set_sort_lookahead(mhdpic_ctx *c, double t)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    if (!std::isfinite(t))
        return fail(MHDPIC_E_ARG, "the look-ahead time must be finite");
    c->ahead_user = t;
    if (c->graph) {   // a captured cycle holds the sorts' look-ahead
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return apply_lookahead(c, t);
}

int mhdpic_set_subcycle_sort(mhdpic_ctx *c, int32_t every)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    if (every < 0)
        return fail(MHDPIC_E_ARG, "every must be >= 0");
    c->sub_sort_every = every;
    return MHDPIC_OK;
}

int mhdpic_sync_particles(mhdpic_ctx *c)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    if (c->mem == MHDPIC_MEM_HOST)   // the host buffers are current after every call
        return MHDPIC_OK;
    return sync_to_caller(c);
}

int mhdpic_get_deposits(mhdpic_ctx *c, int32_t which, double *out)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    if (!out || (which != 0 && which != 1))
        return fail(MHDPIC_E_ARG, "which must be 0 or 1 and out non-NULL");
    const unsigned long long *src = which == 0 ? c->k.corr : c->k.momdep[c->cur];
    return check_launch(c, launch_fixed_to_double(c->k, src, which == 0 ? CH_MX : CH_N, out, c->stream));
}

int mhdpic_get_velocities(mhdpic_ctx *c, double *out)
{
    if (!c || !c->valid || !out)
        return fail(MHDPIC_E_ARG, "invalid context or output pointer");
    int rc;
    if ((rc = copy_particles(c, true)) || (rc = sync_to_caller(c)))
        return rc;
    return check_launch(c, launch_velocities_to_double(c->k, out, c->stream));
}

int mhdpic_get_fields(mhdpic_ctx *c, double *out)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    if (!out)
        return fail(MHDPIC_E_ARG, "out must be non-NULL");
    return check_launch(c, launch_fields_to_double(c->k, out, c->stream));
}

}  // extern "C"

namespace {

// The one-launch step applies where the step is exactly a push and a
// feedback on device buffers: mixed precision, no open face (whose push is
// followed by the marking of free slots), no injection times (their clock
// and permutation are extra launches).
bool fused_ok(const mhdpic_ctx *c)
{
    return c->fuse && c->step_grid > 0 && c->k.prec == MHDPIC_PREC_MIXED && c->mem == MHDPIC_MEM_DEVICE &&
           !c->has_open && !c->track_tinj && c->k.np > 0;
}

// mhdpic_interp_push(dt, 1) + mhdpic_apply_feedback(NULL) as one cooperative
// launch of k_step_mixed, with the same host bookkeeping.
int fused_step(mhdpic_ctx *c, double dt)
{
    int rc;
    if ((rc = restage_if_stale(c)))
        return rc;
    if (!c->next_clear)   // two pushes with no staging in between
        CK(cudaMemsetAsync(c->k.momdep[c->cur ^ 1], 0, sizeof(unsigned long long) * 4 * c->k.nc, c->stream));
    Ctx kk = c->k;
    const bool gather = c->pending;
    if (gather) {   // read through the permutation, write the other set
        const PSet &src = c->sets[c->cur_set], &dst = c->sets[c->cur_set ^ 1];
        kk.pos = dst.pos;
        kk.vel = dst.vel;
        kk.perm_src = c->s.perm;
        kk.src_pos = src.pos;
        kk.src_vel = src.vel;
    }
    const int n = launch_step_mixed(kk, c->s, c->work_ctr, c->cur, dt, c->step_grid, c->bar, c->bar_limit_ns,
                                    c->stream);
    if (n < 0)
        return fail(MHDPIC_E_CUDA, "cooperative launch of the one-launch step: %s",
                    cudaGetErrorString(cudaGetLastError()));
    if ((rc = check_launch(c, n)))
        return rc;
    if (gather) {
        use_set(c, c->cur_set ^ 1);
        c->pending = false;
    }
    c->cur ^= 1;
    c->next_clear = true;
    c->fields_stale = false;
    return MHDPIC_OK;
}

// One full step of mhdpic_run: push, feedback, and the sort at the end of a cycle.
int run_one_step(mhdpic_ctx *c, double dt, int k)
{
    int rc;
    if (k == 1 && c->side_stream && c->fuse) {
        // every step sorts: the push (with its scales), then the feedback
        // and staging on the second stream beside the sort (with the gas in
        // host memory, also the gas upload's wait and the download of the
        // result); they share no data (the feedback reads the deposits and
        // the gas and writes the gas and the staged fields, the sort reads
        // the particles and writes its scratch), and the stream waits for
        // both before the next step
        if ((rc = mhdpic_interp_push(c, dt, 1)))
            return rc;
        CK(cudaEventRecord(c->ev_fork, c->stream));
        CK(cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0));
        rc = upload_gas_for_feedback(c, c->side_stream);
        if (rc == MHDPIC_OK)
            rc = check_launch(c, launch_prep(c->k, c->cur, 1, c->side_stream));
        if (rc == MHDPIC_OK) {
            c->next_clear = true;
            c->fields_stale = false;
            rc = copy_gas(c, false, false, c->side_stream);
        }
        if (rc == MHDPIC_OK) {
            c->step_in_cycle = 0;
            rc = do_sort(c, nullptr, nullptr);
        }
        // joined on every way out (a capture needs the side stream back)
        const cudaError_t e1 = cudaEventRecord(c->ev_join, c->side_stream);
        const cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(c->stream, c->ev_join, 0) : e1;
        if (rc == MHDPIC_OK && e2 != cudaSuccess)
            return cuda_fail(e2, "joining the side stream");
        return rc;
    }
    if (fused_ok(c)) {
        if ((rc = fused_step(c, dt)))
            return rc;
    } else if ((rc = mhdpic_interp_push(c, dt, 1)) || (rc = mhdpic_apply_feedback(c, nullptr))) {
        return rc;
    }
    if (++c->step_in_cycle >= k) {
        c->step_in_cycle = 0;
        if ((rc = do_sort(c, nullptr, nullptr)))
            return rc;
    }
    return MHDPIC_OK;
}

// Sort cadence with the shortest measured time per step: after one untimed
// warm-up step, each candidate runs whole cycles of real steps (at least four
// steps), timed with events on the context's stream.
int tune_sort_cadence(mhdpic_ctx *c, double dt, int32_t *steps_left)
{
    static const int cands[] = {1, 2, 3, 4};
    int rc;
    if (*steps_left > 0) {
        if ((rc = run_one_step(c, dt, 1)))
            return rc;
        --*steps_left;
    }
    // the two events are destroyed on every way out
    struct Events {
        cudaEvent_t e[2] = {nullptr, nullptr};
        ~Events()
        {
            for (cudaEvent_t x : e)
                if (x)
                    cudaEventDestroy(x);
        }
    } ev;
    CK(cudaEventCreate(&ev.e[0]));
    CK(cudaEventCreate(&ev.e[1]));
    float best = 0.f;
    int best_k = 1;
    for (int k : cands) {
        const int reps = (4 + k - 1) / k;
        if (*steps_left < reps * k)
            break;
        // align to the start of a cycle of length k (sort now), the sorts
        // looking k times as far ahead
        if ((rc = apply_lookahead(c, c->ahead_user * k)) || (rc = do_sort(c, nullptr, nullptr)))
            return rc;
        c->step_in_cycle = 0;
        CK(cudaEventRecord(ev.e[0], c->stream));
        for (int s = 0; s < reps * k; ++s)
            if ((rc = run_one_step(c, dt, k)))
                return rc;
        CK(cudaEventRecord(ev.e[1], c->stream));
        CK(cudaEventSynchronize(ev.e[1]));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ev.e[0], ev.e[1]));
        *steps_left -= reps * k;
        if (best == 0.f || ms / (reps * k) < best) {
            best = ms / (reps * k);
            best_k = k;
        }
    }
    c->tuned_k = best_k;
    return MHDPIC_OK;
}

int capture_cycle(mhdpic_ctx *c, double dt, int k, int cycle)
{
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    const int64_t l0 = c->launches;
    const int cur0 = c->cur, set0 = c->cur_set, sic0 = c->step_in_cycle;
    const bool pend0 = c->pending, clear0 = c->next_clear;
    // nothing captured ever runs unless the graph is kept: put the host
    // bookkeeping back where the capture started
    auto restore = [&]() {
        c->cur = cur0;
        c->step_in_cycle = sic0;
        c->pending = pend0;
        c->next_clear = clear0;
        use_set(c, set0);
    };
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = MHDPIC_OK;
    for (int s = 0; s < cycle && rc == MHDPIC_OK; ++s)
        rc = run_one_step(c, dt, k);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    c->graph_launches = c->launches - l0;
    c->launches = l0;   // captured, not yet executed
    if (rc || e != cudaSuccess) {
        if (g)
            cudaGraphDestroy(g);
        restore();
        if (rc)
            return rc;
        return cuda_fail(e, "cudaStreamEndCapture");
    }
    // a replay must leave the state it starts from; otherwise nothing was
    // run, so restore the state and let the caller go on eagerly
    if (c->cur != cur0 || c->cur_set != set0 || c->step_in_cycle != sic0 || c->pending != pend0 ||
        c->next_clear != clear0) {
        cudaGraphDestroy(g);
        restore();
        return MHDPIC_OK;
    }
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->graph = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    c->graph_dt = dt;
    c->graph_k = k;
    c->graph_cur = c->cur;
    c->graph_set = c->cur_set;
    c->graph_pending = c->pending;
    return MHDPIC_OK;
}

}  // namespace

extern "C" {

int mhdpic_run(mhdpic_ctx *c, double dt, int32_t nsteps, int32_t sort_every)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    if (!(dt > 0.0) || !std::isfinite(dt))
        return fail(MHDPIC_E_ARG, "dt must be finite and > 0");
    if (nsteps < 0 || sort_every < 0)
        return fail(MHDPIC_E_ARG, "nsteps and sort_every must be >= 0");
    int rc;
    int32_t left = nsteps;
    if ((rc = restage_if_stale(c)))   // before any capture
        return rc;
    if (sort_every == 0 && !c->tuned_k)
        if ((rc = tune_sort_cadence(c, dt, &left)))
            return rc;
    const int k = sort_every ? sort_every : c->tuned_k;
    if (c->step_in_cycle >= k)
        c->step_in_cycle = 0;
    // the sorts of a k-step cycle look k times as far ahead: with a look-ahead
    // of dt/2, the mean half-step position of the cycle's pushes
    if ((rc = apply_lookahead(c, c->ahead_user * k)))
        return rc;
    // finish the current cycle eagerly (and a first step when the next
    // moments buffer has not been cleared by a staging pass yet), up to a
    // sort whose permutation the next push applies: the state every cycle
    // starts from
    while (left > 0 && (c->step_in_cycle != 0 || !c->next_clear || !c->pending)) {
        if ((rc = run_one_step(c, dt, k)))
            return rc;
        --left;
    }
    // whole cycles from a graph: two sorts and 2k pushes, so that the moments
    // buffers and the particle sets alternate back to where the capture
    // started; the legacy default stream and host buffers cannot be captured
    // and run eagerly
    const int cycle = 2 * k;
    const bool graphs = c->stream != nullptr && c->mem != MHDPIC_MEM_HOST && c->mem != MHDPIC_MEM_HOST_GAS;
    if (graphs && left >= cycle) {
        if (!c->graph || c->graph_dt != dt || c->graph_k != k || c->graph_cur != c->cur ||
            c->graph_set != c->cur_set || c->graph_pending != c->pending)
            if ((rc = capture_cycle(c, dt, k, cycle)))
                return rc;
        while (c->graph && left >= cycle) {
            CK(cudaGraphLaunch(c->graph, c->stream));
            c->launches += c->graph_launches;
            left -= cycle;
        }
    }
    while (left > 0) {
        if ((rc = run_one_step(c, dt, k)))
            return rc;
        --left;
    }
    return MHDPIC_OK;
}

int32_t mhdpic_sort_cadence(const mhdpic_ctx *c) { return c && c->valid ? c->tuned_k : -1; }

int64_t mhdpic_num_keys(const mhdpic_ctx *c) { return c && c->valid ? c->k.nkeys : -1; }

int64_t mhdpic_launch_count(const mhdpic_ctx *c) { return c && c->valid ? c->launches : -1; }

int mhdpic_get_status(mhdpic_ctx *c, uint32_t *flags)
{
    if (!c || !c->valid || !flags)
        return fail(MHDPIC_E_ARG, "invalid context or flags pointer");
    CK(cudaMemcpyAsync(flags, c->k.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MHDPIC_OK;
}

int mhdpic_debug_fail_launch(mhdpic_ctx *c, int64_t n)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    if (n < 0)
        return fail(MHDPIC_E_ARG, "n must be >= 0");
    c->fail_countdown = n;
    return MHDPIC_OK;
}

int mhdpic_set_step_fusion(mhdpic_ctx *c, int32_t enable)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    c->fuse = enable != 0;
    if (c->graph) {   // a captured cycle holds the other form of the step
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return MHDPIC_OK;
}

int32_t mhdpic_step_fusion(const mhdpic_ctx *c)
{
    return c && c->valid ? (fused_ok(c) ? 1 : 0) : -1;
}

int mhdpic_set_field_tma(mhdpic_ctx *c, int32_t enable)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    c->k.tma = enable && c->tma_ok ? 1 : 0;
    if (c->graph) {   // a captured cycle holds the other form of the staging
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return MHDPIC_OK;
}

int32_t mhdpic_field_tma(const mhdpic_ctx *c)
{
    return c && c->valid ? c->k.tma : -1;
}

int mhdpic_debug_set_barrier_limit(mhdpic_ctx *c, int64_t ns)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    c->bar_limit_ns = ns > 0 ? (long long)ns : 1000000000ll;
    if (c->graph) {   // the limit is a launch argument of the captured cycle
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return MHDPIC_OK;
}

int mhdpic_debug_set_copy_limit(mhdpic_ctx *c, int64_t ns)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    c->k.copy_limit_ns = ns > 0 ? ns : COPY_LIMIT_DEFAULT_NS;
    if (c->graph) {   // the limit is a launch argument of the captured cycle
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return MHDPIC_OK;
}

int mhdpic_clear_status(mhdpic_ctx *c)
{
    if (!c || !c->valid)
        return fail(MHDPIC_E_STATE, "invalid context");
    CK(cudaMemsetAsync(c->k.status, 0, sizeof(uint32_t), c->stream));
    if (c->bar)   // a barrier that timed out may have been left half counted
        CK(cudaMemsetAsync(c->bar, 0, sizeof(GridBarrier), c->stream));
    return MHDPIC_OK;
}

}  // extern "C"
