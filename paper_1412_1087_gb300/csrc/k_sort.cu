// Cell sort of the particles (the library's layout; the paper has no sort).
//
// Stable counting sort by key = brick number * brick volume + cell number in
// the brick (x fastest at both levels), per box, keys of later boxes after
// earlier ones.  Steps:
//   1. key of each particle, rank among equal keys by warp-aggregated atomics
//      (this rank is not yet the stable one);
//   2. exclusive scan of the per-key counts;
//   3. scatter of the particle indices to their key segment;
//   4. sort of each key segment by particle index, which makes the result the
//      stable order: the permutation equals a stable sort by key.
// The particle arrays are permuted later: by the next push, which reads its
// particles through the permutation, or by launch_gather.
//   5. the push work list: every brick's particle range cut into items of at
//      most ITEM_MAX_PARTICLES.
#include <climits>

#include "async_copy.cuh"
#include "device_common.cuh"

namespace mhdpic {

namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_PER_THREAD = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER_THREAD;
constexpr int WARP_SORT_MAX = 1024;     // per-warp shared-memory bitonic sort
constexpr int BLOCK_SORT_MAX = 8192;    // per-block shared-memory bitonic sort
constexpr int RANK_SORT_MAX = 1 << 20;  // quadratic ranking beyond that is refused

__device__ __forceinline__ int64_t brick_key(const BoxDev &b, const Ctx &c, int ci, int cj, int ck)
{
    int q[3], r[3];
    const int cc[3] = {ci, cj, ck};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (c.brick_sh[d] >= 0) {   // power-of-two bricks: shifts and masks
            q[d] = cc[d] >> c.brick_sh[d];
            r[d] = cc[d] & (c.brick[d] - 1);
        } else {
            q[d] = cc[d] / c.brick[d];
            r[d] = cc[d] - q[d] * c.brick[d];
        }
    }
    const int64_t bid = ((int64_t)q[2] * b.nb[1] + q[1]) * b.nb[0] + q[0];
    const int64_t in = ((int64_t)r[2] * c.brick[1] + r[1]) * c.brick[0] + r[0];
    return b.key0 + bid * ((int64_t)c.brick[0] * c.brick[1] * c.brick[2]) + in;
}

// Cells a particle moves along each of the first D dimensions in time t at
// its current four-velocity v (the sort's look-ahead), -1, 0 or +1: whether
// the position o + (t/dx) v/gamma leaves its cell through the lower or the
// upper face (a half step moves a particle well under one cell).  With the
// box's FP32 constants k = {t/dx, t/dy, t/dz, 1/C^2} (each rounded once, on
// the host), g2 = gamma^2 = 1 + v^2 k.w and a_d = k_d, the faces are tested on
// squares, so that no square root or division is needed:
//   +1 when v_d > 0 and (a_d v_d)^2 >= ((1 - o_d)(1 - o_d)) g2,
//   -1 when v_d < 0 and (a_d v_d)^2 >  (o_d o_d) g2,
// v^2 = (vx vx + vy vy) + vz vz, every operation a correctly rounded FP32 one
// in this order (no contraction), so the key can be recomputed exactly
// elsewhere.
__device__ __forceinline__ void ahead_cells(const float4 k, const float v[3], const float o[3], int D, int cells[3])
{
    const float v2 = __fadd_rn(__fadd_rn(__fmul_rn(v[0], v[0]), __fmul_rn(v[1], v[1])), __fmul_rn(v[2], v[2]));
    const float g2 = __fadd_rn(1.f, __fmul_rn(v2, k.w));
    const float ta[3] = {k.x, k.y, k.z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d >= D)
            break;
        const float av = __fmul_rn(ta[d], v[d]);
        const float l = __fmul_rn(av, av);
        const float up = __fsub_rn(1.f, o[d]);
        const float ru = __fmul_rn(__fmul_rn(up, up), g2);
        const float rl = __fmul_rn(__fmul_rn(o[d], o[d]), g2);
        cells[d] = (v[d] > 0.f && l >= ru) ? 1 : ((v[d] < 0.f && l > rl) ? -1 : 0);
    }
}

// Clamp or wrap a key cell into the box, and its brick-major key.
__device__ __forceinline__ int32_t key_of_cell(const Ctx &c, const BoxDev &b, int ci[3], bool ahead)
{
    if (ahead)
        for (int d = 0; d < c.ndim; ++d)
            ci[d] = b.bc[d] == MHDPIC_BC_PERIODIC ? map_coord(ci[d], b.n[d], MHDPIC_BC_PERIODIC)
                                                  : (ci[d] < 0 ? 0 : (ci[d] >= b.n[d] ? b.n[d] - 1 : ci[d]));
    for (int d = 0; d < 3; ++d)   // defensive: a key outside the box would index out of range
        ci[d] = ci[d] < 0 ? 0 : (ci[d] >= b.n[d] ? b.n[d] - 1 : ci[d]);
    return (int32_t)brick_key(b, c, ci[0], ci[1], ci[2]);
}

// What the mixed-precision key needs of a box, held in registers while a
// thread's particles stay in one box (reloaded when the box changes).
struct KeyBox {
    int box;
    int n[3], bc[3], nb[3];
    int32_t ncell;
    int32_t key0;   // keys are int32: the box's first key
    FastDiv dnx, dnxy;
    float4 sk;
};

__device__ __forceinline__ void load_keybox(const Ctx &c, int bx, KeyBox &kb)
{
    const BoxDev &b = c.boxes[bx];
    kb.box = bx;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        kb.n[d] = b.n[d];
        kb.bc[d] = b.bc[d];
        kb.nb[d] = b.nb[d];
    }
    kb.ncell = (int32_t)b.ncell;
    kb.key0 = (int32_t)b.key0;
    kb.dnx = b.div_nx;
    kb.dnxy = b.div_nxy;
    kb.sk = __ldg(c.sort_k + bx);
}

// Mixed precision: the key of a particle from its two records (loaded by
// the caller, so that the loads of several particles are in flight at once),
// as key_of_cell / brick_key compute it.
template <int D, bool AHEAD>
__device__ __forceinline__ int32_t key_mixed(const Ctx &c, const KeyBox &kb, const int4 ps, const float4 vs)
{
    int32_t cl = ps.x;
    if (cl == DEAD_CELL)   // particles that left the box share one key after all the others
        return (int32_t)c.nkeys;
    if (cl < 0 || cl >= kb.ncell) {
        set_status(c.status, MHDPIC_ST_CELL_RANGE);
        cl = cl < 0 ? 0 : kb.ncell - 1;
    }
    const uint32_t uc = (uint32_t)cl;
    const uint32_t kz = fdiv(uc, kb.dnxy);
    const uint32_t rr = uc - kz * kb.dnxy.d;
    const uint32_t jy = fdiv(rr, kb.dnx);
    int ci[3] = {(int)(rr - jy * kb.dnx.d), (int)jy, (int)kz};
    if (AHEAD) {
        const float v[3] = {vs.x, vs.y, vs.z};
        const float o[3] = {__int_as_float(ps.y), __int_as_float(ps.z), __int_as_float(ps.w)};
        int k[3] = {0, 0, 0};
        ahead_cells(kb.sk, v, o, D, k);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int g = ci[d] + k[d];
            ci[d] = kb.bc[d] == MHDPIC_BC_PERIODIC ? (g < 0 ? g + kb.n[d] : (g >= kb.n[d] ? g - kb.n[d] : g))
                                                   : (g < 0 ? 0 : (g >= kb.n[d] ? kb.n[d] - 1 : g));
        }
    }
    int q[3] = {0, 0, 0}, r[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < D; ++d) {
        if (c.brick_sh[d] >= 0) {
            q[d] = ci[d] >> c.brick_sh[d];
            r[d] = ci[d] & (c.brick[d] - 1);
        } else {
            q[d] = ci[d] / c.brick[d];
            r[d] = ci[d] - q[d] * c.brick[d];
        }
    }
    // int32 throughout: every key of the context is below nkeys < 2^31
    const int bid = (q[2] * kb.nb[1] + q[1]) * kb.nb[0] + q[0];
    const int in = (r[2] * c.brick[1] + r[1]) * c.brick[0] + r[0];
    return kb.key0 + bid * (c.brick[0] * c.brick[1] * c.brick[2]) + in;
}

// FP64 precision: the key of particle i of box b, from its absolute position.
__device__ __forceinline__ int32_t key_f64(const Ctx &c, const BoxDev &b, int bx, int64_t i)
{
    int ci[3] = {0, 0, 0};
    const bool ahead = c.sort_ahead != 0.0;
    if (isnan(c.x[i]))   // particles that left the box share one key after all the others
        return (int32_t)c.nkeys;
    float o[3] = {0.f, 0.f, 0.f};
    for (int d = 0; d < c.ndim; ++d) {
        double s = (c.x[(int64_t)d * c.np + i] - b.x0[d]) / b.dx[d];
        double f = floor(s);
        int v = f < 0.0 ? 0 : (f >= (double)b.n[d] ? b.n[d] - 1 : (int)f);
        if (!(f >= 0.0 && f < (double)b.n[d]))
            set_status(c.status, MHDPIC_ST_CELL_RANGE);
        ci[d] = v;
        o[d] = (float)(s - (double)v);
    }
    if (ahead) {
        const float v[3] = {(float)c.p64[i], (float)c.p64[c.np + i], (float)c.p64[2 * c.np + i]};
        int k[3] = {0, 0, 0};
        ahead_cells(__ldg(c.sort_k + bx), v, o, c.ndim, k);
        for (int d = 0; d < c.ndim; ++d)
            ci[d] += k[d];
    }
    return key_of_cell(c, b, ci, ahead);
}

// Particles handled per thread and loop pass by the streaming sort kernels:
// independent loads (and atomics) in flight hide their latency.
constexpr int SORT_ILP = 4;

// Runs of equal keys in consecutive lanes (the input is nearly sorted) take
// one atomic per run, made by the run's first lane; the rank inside the run
// is the lane offset.  Lanes outside `active` take no part; a negative key
// takes no atomic.
struct RunSlot {
    int start;   // first lane of the run
    int base;    // first slot of the run (at the first lane)
};

__device__ __forceinline__ RunSlot run_reserve(int32_t key, int lane, unsigned active, int32_t *count)
{
    const int prev = __shfl_up_sync(active, key, 1);
    const bool head = lane == 0 || !((active >> (lane - 1)) & 1u) || prev != key;
    const unsigned heads = __ballot_sync(active, head);
    RunSlot r;
    r.start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));    // last head at or below lane
    const unsigned after = heads & ~(0xffffffffu >> (31 - lane));  // heads above lane
    const int end = after ? __ffs(after) - 1 : 32;
    const unsigned tail = (end < 32 ? (1u << end) : 0u) - 1u;      // lanes below end
    const int len = __popc(active & tail & ~((1u << r.start) - 1u));
    r.base = 0;
    if (head && key >= 0)
        r.base = atomicAdd(count + key, len);
    return r;
}

__device__ __forceinline__ int32_t run_slot(const RunSlot &r, int lane, unsigned active)
{
    return __shfl_sync(active, r.base, r.start) + (lane - r.start);
}

// FP64 precision: the keys from the absolute positions, SORT_ILP particles
// per thread and pass.
__global__ void k_sort_keys_f64(Ctx c, int32_t *__restrict__ count, int32_t *__restrict__ pkey,
                                int32_t *__restrict__ pslot)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < c.np; i0 += SORT_ILP * stride) {
        // lanes past the end take keys no other lane has, so they form runs
        // of their own and take no atomic
        const unsigned active = __activemask();
        int32_t key[SORT_ILP];
#pragma unroll
        for (int u = 0; u < SORT_ILP; ++u) {
            const int64_t i = i0 + u * stride;
            int bx = 0;
            if (i < c.np)
                bx = find_box(c.box_part_start, c.nbox, i);
            key[u] = i < c.np ? key_f64(c, c.boxes[bx], bx, i) : -1 - lane;
        }
        RunSlot rs[SORT_ILP];
#pragma unroll
        for (int u = 0; u < SORT_ILP; ++u)
            rs[u] = run_reserve(key[u], lane, active, count);
#pragma unroll
        for (int u = 0; u < SORT_ILP; ++u) {
            const int32_t slot = run_slot(rs[u], lane, active);
            const int64_t i = i0 + u * stride;
            if (i < c.np) {
                pkey[i] = key[u];
                pslot[i] = slot;
            }
        }
    }
}

// Mixed precision, records staged: the particle records stream through a
// ring of KEY_STAGES shared-memory stages of KEY_CHUNK particles, each filled
// by one bulk copy per record array that the block's first thread issues
// KEY_STAGES chunks ahead, so the loads of later chunks are in flight while
// the keys and the atomics of this one are done.  (Two stages, 32 KB, let 5
// blocks share an SM; 3 and 4 stages measured slower at 128^3 x 32.)  A block takes the chunks
// blockIdx.x, blockIdx.x + gridDim.x, ...; each warp's 32 lanes take 32
// consecutive particles, as the run detection needs.
constexpr int KEY_THREADS = 256;
constexpr int KEY_PER_THREAD = 2;
constexpr int KEY_CHUNK = KEY_THREADS * KEY_PER_THREAD;
constexpr int KEY_STAGES = 2;
constexpr size_t KEY_SMEM = (size_t)KEY_STAGES * KEY_CHUNK * (sizeof(int4) + sizeof(float4));

// Thread 0: the copies of chunk `chunk` into one stage (the velocities only
// when the key looks ahead).
__device__ __forceinline__ void issue_records(const Ctx &c, int64_t chunk, int4 *dp, float4 *dv, bool ahead,
                                              uint64_t *bar)
{
    const int64_t p0 = chunk * KEY_CHUNK;
    const int64_t left = c.np - p0;
    const unsigned bytes = (unsigned)(left < KEY_CHUNK ? left : KEY_CHUNK) * 16u;
    mbar_expect_tx(bar, ahead ? 2u * bytes : bytes);
    bulk_copy(dp, c.pos + p0, bytes, bar);
    if (ahead)
        bulk_copy(dv, c.vel + p0, bytes, bar);
}

template <int D, bool AHEAD>
__global__ void __launch_bounds__(KEY_THREADS) k_sort_keys_staged(Ctx c, int32_t *__restrict__ count,
                                                                  int32_t *__restrict__ pkey,
                                                                  int32_t *__restrict__ pslot)
{
    extern __shared__ __align__(128) unsigned char smem[];
    int4 *sp = reinterpret_cast<int4 *>(smem);
    float4 *sv = reinterpret_cast<float4 *>(smem + (size_t)KEY_STAGES * KEY_CHUNK * sizeof(int4));
    __shared__ __align__(8) uint64_t full[KEY_STAGES];
    const int lane = threadIdx.x & 31;
    constexpr bool ahead = AHEAD;
    const int64_t nchunk = (c.np + KEY_CHUNK - 1) / KEY_CHUNK;
    const int64_t mine = (int64_t)blockIdx.x < nchunk ? (nchunk - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    if (threadIdx.x == 0) {
        for (int st = 0; st < KEY_STAGES; ++st)
            mbar_init(&full[st]);
        fence_proxy_async();
        for (int64_t k = 0; k < KEY_STAGES && k < mine; ++k)
            issue_records(c, blockIdx.x + k * gridDim.x, sp + k * KEY_CHUNK, sv + k * KEY_CHUNK, ahead, &full[k]);
    }
    __syncthreads();
    KeyBox kb;
    load_keybox(c, 0, kb);
    for (int64_t k = 0; k < mine; ++k) {
        const int st = (int)(k % KEY_STAGES);
        const bool ok = mbar_wait(&full[st], (unsigned)((k / KEY_STAGES) & 1), c.copy_limit_ns);
        if (__syncthreads_or(!ok)) {
            // give up the launch, after the copies in flight have had their time
            if (threadIdx.x == 0) {
                set_status(c.status, MHDPIC_ST_COPY_TIMEOUT);
                for (int64_t j = k; j < mine && j < k + KEY_STAGES; ++j)
                    mbar_wait(&full[j % KEY_STAGES], (unsigned)((j / KEY_STAGES) & 1), COPY_LIMIT_NS);
            }
            return;
        }
        const int64_t p0 = (blockIdx.x + k * gridDim.x) * (int64_t)KEY_CHUNK;
        const int n = (int)(c.np - p0 < KEY_CHUNK ? c.np - p0 : KEY_CHUNK);
        int cbox = 0;   // the chunk's box, or -1 when it spans several
        if (c.nbox > 1) {
            const int b0 = find_box(c.box_part_start, c.nbox, p0);
            cbox = b0 == find_box(c.box_part_start, c.nbox, p0 + n - 1) ? b0 : -1;
        }
        int32_t key[KEY_PER_THREAD];
#pragma unroll
        for (int u = 0; u < KEY_PER_THREAD; ++u) {
            const int p = u * KEY_THREADS + threadIdx.x;
            key[u] = -1 - lane;   // past the end: a run of its own, no atomic
            if (p < n) {
                const int bx = cbox >= 0 ? cbox : find_box(c.box_part_start, c.nbox, p0 + p);
                if (bx != kb.box)
                    load_keybox(c, bx, kb);
                const float4 vs = ahead ? sv[st * KEY_CHUNK + p] : make_float4(0.f, 0.f, 0.f, 0.f);
                key[u] = key_mixed<D, AHEAD>(c, kb, sp[st * KEY_CHUNK + p], vs);
            }
        }
        RunSlot rs[KEY_PER_THREAD];
#pragma unroll
        for (int u = 0; u < KEY_PER_THREAD; ++u)
            rs[u] = run_reserve(key[u], lane, 0xffffffffu, count);
#pragma unroll
        for (int u = 0; u < KEY_PER_THREAD; ++u) {
            const int32_t slot = run_slot(rs[u], lane, 0xffffffffu);
            const int p = u * KEY_THREADS + threadIdx.x;
            if (p < n) {
                pkey[p0 + p] = key[u];
                pslot[p0 + p] = slot;
            }
        }
        __syncthreads();   // every thread has read the stage
        if (threadIdx.x == 0 && k + KEY_STAGES < mine) {
            fence_proxy_async();
            issue_records(c, blockIdx.x + (k + KEY_STAGES) * gridDim.x, sp + st * KEY_CHUNK, sv + st * KEY_CHUNK,
                          ahead, &full[st]);
        }
    }
}

// --- exclusive scan of int32 (values and totals < 2^31) ---

__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_sums, int *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o)
            x += y;
    }
    if (lane == 31)
        warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        int s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o)
                s += y;
        }
        if (lane < nw)
            warp_sums[lane] = s;
    }
    __syncthreads();
    int pre = (wid > 0 ? warp_sums[wid - 1] : 0) + x - v;
    if (total)
        *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return pre;
}

__global__ void k_scan_tiles(const int32_t *__restrict__ in, int64_t n, int32_t *__restrict__ sums)
{
    __shared__ int ws[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_PER_THREAD;
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k)
        if (base + k < n)
            s += in[base + k];
    int tot;
    block_exclusive_scan(s, ws, &tot);
    if (threadIdx.x == 0)
        sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int32_t *sums, int nt)
{
    __shared__ int ws[32];
    int carry = 0;
    for (int start = 0; start < nt; start += blockDim.x) {
        int i = start + threadIdx.x;
        int v = i < nt ? sums[i] : 0;
        int tot;
        int pre = block_exclusive_scan(v, ws, &tot);
        if (i < nt)
            sums[i] = pre + carry;
        carry += tot;
    }
}

__global__ void k_scan_apply(const int32_t *__restrict__ in, int64_t n,
                             const int32_t *__restrict__ sums, int32_t *__restrict__ out)
{
    __shared__ int ws[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_PER_THREAD;
    int vals[SCAN_PER_THREAD];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        vals[k] = base + k < n ? in[base + k] : 0;
        s += vals[k];
    }
    int pre = block_exclusive_scan(s, ws, nullptr) + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        if (base + k < n)
            out[base + k] = pre;
        pre += vals[k];
    }
    // the thread holding the last element closes the array with the total
    if (base <= n - 1 && n - 1 < base + SCAN_PER_THREAD)
        out[n] = pre;
}

// out[0..n] = exclusive scan of in[0..n), out[n] = total.
int scan(const int32_t *in, int64_t n, int32_t *out, int32_t *tmp, cudaStream_t st)
{
    if (n <= 0) {
        cudaMemsetAsync(out, 0, sizeof(int32_t), st);
        return 0;
    }
    int nt = (int)((n + SCAN_TILE - 1) / SCAN_TILE);
    k_scan_tiles<<<nt, SCAN_THREADS, 0, st>>>(in, n, tmp);
    k_scan_sums<<<1, SCAN_THREADS, 0, st>>>(tmp, nt);
    k_scan_apply<<<nt, SCAN_THREADS, 0, st>>>(in, n, tmp, out);
    return 3;
}

// A key outside [0, nkeys] (only after a key pass that gave up part of its
// work) is flagged and its particle skipped.
__global__ void k_sort_scatter(int64_t np, int64_t nkeys, const int32_t *__restrict__ pkey,
                               const int32_t *__restrict__ pslot, const int32_t *__restrict__ offset,
                               int32_t *__restrict__ perm, uint32_t *status)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < np; i0 += SORT_ILP * stride) {
        int32_t key[SORT_ILP], slot[SORT_ILP];
#pragma unroll
        for (int u = 0; u < SORT_ILP; ++u) {
            const int64_t i = i0 + u * stride;
            key[u] = i < np ? pkey[i] : 0;
            slot[u] = i < np ? pslot[i] : 0;
            if (key[u] < 0 || key[u] > nkeys) {
                set_status(status, MHDPIC_ST_SORT_CAP);
                key[u] = 0;
                slot[u] = -1 - (int32_t)np;   // lands outside [0, np): not written
            }
        }
        int32_t off[SORT_ILP];
#pragma unroll
        for (int u = 0; u < SORT_ILP; ++u)
            off[u] = i0 + u * stride < np ? offset[key[u]] : 0;
#pragma unroll
        for (int u = 0; u < SORT_ILP; ++u) {
            const int64_t i = i0 + u * stride;
            if (i >= np)
                continue;
            const int64_t dst = (int64_t)off[u] + slot[u];
            if (dst >= 0 && dst < np)
                perm[dst] = (int32_t)i;
            else
                set_status(status, MHDPIC_ST_SORT_CAP);
        }
    }
}

// Ascending bitonic sort of the 32 E values a[e*32 + lane] = v[e] held by a
// warp: distances below 32 exchange through shuffles, larger ones between a
// lane's own registers.
template <int E>
__device__ __forceinline__ void warp_bitonic(int (&v)[E], int lane)
{
#pragma unroll
    for (int k = 2; k <= 32 * E; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int pe = e ^ (j >> 5);
                    if (pe > e) {
                        const bool up = ((e * 32 + lane) & k) == 0;
                        const int x = v[e], y = v[pe];
                        if ((x > y) == up) {
                            v[e] = y;
                            v[pe] = x;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int o = __shfl_xor_sync(0xffffffffu, v[e], j);
                    const bool up = ((e * 32 + lane) & k) == 0;
                    const bool lower = (lane & j) == 0;
                    v[e] = (lower == up) ? min(v[e], o) : max(v[e], o);
                }
            }
        }
    }
}

// Sort of one segment [s, s + n), n <= 32 E, in registers, read from src
// (perm + s itself, or a copy of it); a segment already in ascending order is
// left alone.
template <int E>
__device__ __forceinline__ void warp_sort_segment(const int32_t *src, int32_t *__restrict__ perm, int s, int n,
                                                  int lane)
{
    int v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = e * 32 + lane;
        v[e] = i < n ? src[i] : INT_MAX;
    }
    bool ok = true;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        int nxt = __shfl_down_sync(0xffffffffu, v[e], 1);
        if (e + 1 < E) {
            const int first = __shfl_sync(0xffffffffu, v[e + 1 < E ? e + 1 : e], 0);
            if (lane == 31)
                nxt = first;
        }
        const int i = e * 32 + lane;
        ok &= i >= n - 1 || v[e] < nxt;
    }
    if (__all_sync(0xffffffffu, ok))
        return;
    warp_bitonic<E>(v, lane);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = e * 32 + lane;
        if (i < n)
            perm[s + i] = v[e];
    }
}

// A segment of the scatter is made of runs: each warp of the key pass gives
// the lanes of a run of equal keys consecutive slots, so a run is an
// increasing interval of consecutive particle indices, and runs never
// overlap.  Sorting such a segment only sorts its runs by their first index.
constexpr int MERGE_RUNS = 128;   // runs a warp merges (4 per lane)

// Ascending bitonic sort of the 128 values v[e] (element e*32 + lane) of a warp.
__device__ __forceinline__ void warp_bitonic64(long long (&v)[4], int lane)
{
#pragma unroll
    for (int k = 2; k <= 128; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int pe = e ^ (j >> 5);
                    if (pe > e) {
                        const bool up = ((e * 32 + lane) & k) == 0;
                        const long long x = v[e], y = v[pe];
                        if ((x > y) == up) {
                            v[e] = y;
                            v[pe] = x;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const long long o = __shfl_xor_sync(0xffffffffu, v[e], j);
                    const bool up = ((e * 32 + lane) & k) == 0;
                    const bool lower = (lane & j) == 0;
                    v[e] = (lower == up) ? min(v[e], o) : max(v[e], o);
                }
            }
        }
    }
}

// Segment a[0, n) in the warp's shared memory, at most MERGE_RUNS runs: the
// sorted order into perm[s, s + n).  Returns false (nothing written) with more.
__device__ __forceinline__ bool warp_merge_runs(const int32_t *a, int n, int32_t *__restrict__ perm, int s,
                                                int lane, int *hpos)
{
    int nruns = 0;
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        const bool head = i < n && (i == 0 || a[i] != a[i - 1] + 1);
        const unsigned m = __ballot_sync(0xffffffffu, head);
        if (head) {
            const int pos = nruns + __popc(m & ((1u << lane) - 1u));
            if (pos < MERGE_RUNS)
                hpos[pos] = i;
        }
        nruns += __popc(m);
    }
    __syncwarp();
    if (nruns > MERGE_RUNS)
        return false;
    // (first index, run number) of each run, sorted across the warp
    long long v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int r = e * 32 + lane;
        v[e] = r < nruns ? ((long long)a[hpos[r]] << 8) | r : LLONG_MAX;
    }
    warp_bitonic64(v, lane);
    int carry = 0;   // elements of the sorted runs before this group of 32
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int rr = e * 32 + lane;
        int st = 0, len = 0;
        if (rr < nruns) {
            const int r = (int)(v[e] & 0xff);
            st = hpos[r];
            len = (r + 1 < nruns ? hpos[r + 1] : n) - st;
        }
        int incl = len;   // inclusive scan of the lengths in sorted order
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o)
                incl += y;
        }
        const int dst = carry + incl - len;
        for (int q = 0; q < len; ++q)
            perm[s + dst + q] = a[st + q];
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    return true;
}

// Segments of up to 128 are sorted in registers, up to WARP_SORT_MAX in the
// warp's shared memory (by their runs when they have at most MERGE_RUNS, else
// by a bitonic network); longer ones are listed for k_sort_big.  This sorts
// one key's segment [s, s + n), read from perm (the warp's buffer a is free).
__device__ __forceinline__ void sort_one_segment(int64_t k, int s, int n, int32_t *__restrict__ perm, int32_t *a,
                                                 int *hp, int32_t *__restrict__ big_list,
                                                 int32_t *__restrict__ big_count, int lane)
{
    if (n <= 1)
        return;
    if (n <= 32) {
        warp_sort_segment<1>(perm + s, perm, s, n, lane);
    } else if (n <= 64) {
        warp_sort_segment<2>(perm + s, perm, s, n, lane);
    } else if (n <= 128) {
        warp_sort_segment<4>(perm + s, perm, s, n, lane);
    } else if (n <= WARP_SORT_MAX) {
        int P = 64;
        while (P < n)
            P <<= 1;
        for (int i = lane; i < P; i += 32)
            a[i] = i < n ? perm[s + i] : INT_MAX;
        __syncwarp();
        if (warp_merge_runs(a, n, perm, s, lane, hp))
            return;
        for (int kk = 2; kk <= P; kk <<= 1) {
            for (int j = kk >> 1; j > 0; j >>= 1) {
                for (int i = lane; i < P; i += 32) {
                    int ixj = i ^ j;
                    if (ixj > i) {
                        int x = a[i], y = a[ixj];
                        bool asc = (i & kk) == 0;
                        if ((x > y) == asc) {
                            a[i] = y;
                            a[ixj] = x;
                        }
                    }
                }
                __syncwarp();
            }
        }
        for (int i = lane; i < n; i += 32)
            perm[s + i] = a[i];
        __syncwarp();
    } else if (lane == 0) {
        int slot = atomicAdd(big_count, 1);
        big_list[slot] = (int32_t)k;
    }
}

// A warp takes SEG_GROUP consecutive keys at a time: their offsets in one
// load (one per lane), and, when the group's particles fit the warp's buffer,
// all of them in one coalesced pass, so that the loads of a whole group are in
// flight together; each segment of up to 128 is then sorted from the buffer.
// Longer segments, and groups that do not fit, go through sort_one_segment.
constexpr int SEG_GROUP = 31;

__global__ void __launch_bounds__(256) k_sort_segments(int64_t nkeys, const int32_t *__restrict__ offset,
                                                       int32_t *__restrict__ perm,
                                                       int32_t *__restrict__ big_list,
                                                       int32_t *__restrict__ big_count)
{
    __shared__ int32_t buf[8][WARP_SORT_MAX];
    __shared__ int hp[8][MERGE_RUNS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t *a = buf[wid];
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + wid) * SEG_GROUP; k0 < nkeys;
         k0 += nwarps * SEG_GROUP) {
        const int nk = (int)(nkeys - k0 < SEG_GROUP ? nkeys - k0 : SEG_GROUP);
        const int o = lane <= nk ? offset[k0 + lane] : 0;   // offsets of keys k0 .. k0 + nk
        const int gs = __shfl_sync(0xffffffffu, o, 0), ge = __shfl_sync(0xffffffffu, o, nk);
        if (ge - gs > WARP_SORT_MAX) {
            for (int j = 0; j < nk; ++j) {
                const int s = __shfl_sync(0xffffffffu, o, j), e = __shfl_sync(0xffffffffu, o, j + 1);
                sort_one_segment(k0 + j, s, e - s, perm, a, hp[wid], big_list, big_count, lane);
            }
            continue;
        }
        for (int i = lane; i < ge - gs; i += 32)
            a[i] = perm[gs + i];
        __syncwarp();
        unsigned longer = 0u;   // keys of the group with segments over 128
        for (int j = 0; j < nk; ++j) {
            const int s = __shfl_sync(0xffffffffu, o, j), e = __shfl_sync(0xffffffffu, o, j + 1);
            const int n = e - s;
            if (n <= 1)
                continue;
            if (n <= 32)
                warp_sort_segment<1>(a + (s - gs), perm, s, n, lane);
            else if (n <= 64)
                warp_sort_segment<2>(a + (s - gs), perm, s, n, lane);
            else if (n <= 128)
                warp_sort_segment<4>(a + (s - gs), perm, s, n, lane);
            else
                longer |= 1u << j;
        }
        __syncwarp();   // the buffer is free again
        while (longer) {
            const int j = __ffs(longer) - 1;
            longer &= longer - 1u;
            const int s = __shfl_sync(0xffffffffu, o, j), e = __shfl_sync(0xffffffffu, o, j + 1);
            sort_one_segment(k0 + j, s, e - s, perm, a, hp[wid], big_list, big_count, lane);
        }
    }
}

// Long segments: block bitonic sort in shared memory, or a quadratic ranking
// (elements are distinct particle indices) through `scratch` beyond that.
__global__ void __launch_bounds__(1024) k_sort_big(const int32_t *__restrict__ offset,
                                                   int32_t *__restrict__ perm,
                                                   const int32_t *__restrict__ big_list,
                                                   const int32_t *__restrict__ big_count,
                                                   int32_t *__restrict__ scratch, uint32_t *status)
{
    __shared__ int32_t a[BLOCK_SORT_MAX];
    const int nb = *big_count;
    for (int q = blockIdx.x; q < nb; q += gridDim.x) {
        int64_t k = big_list[q];
        int s = offset[k], e = offset[k + 1];
        int n = e - s;
        if (n <= BLOCK_SORT_MAX) {
            int P = 64;
            while (P < n)
                P <<= 1;
            for (int i = threadIdx.x; i < P; i += blockDim.x)
                a[i] = i < n ? perm[s + i] : INT_MAX;
            __syncthreads();
            for (int kk = 2; kk <= P; kk <<= 1) {
                for (int j = kk >> 1; j > 0; j >>= 1) {
                    for (int i = threadIdx.x; i < P; i += blockDim.x) {
                        int ixj = i ^ j;
                        if (ixj > i) {
                            int x = a[i], y = a[ixj];
                            bool asc = (i & kk) == 0;
                            if ((x > y) == asc) {
                                a[i] = y;
                                a[ixj] = x;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            for (int i = threadIdx.x; i < n; i += blockDim.x)
                perm[s + i] = a[i];
            __syncthreads();
        } else if (n <= RANK_SORT_MAX) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                int v = perm[s + i];
                int r = 0;
                for (int j = 0; j < n; ++j)
                    r += perm[s + j] < v;
                scratch[s + r] = v;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += blockDim.x)
                perm[s + i] = scratch[s + i];
            __syncthreads();
        } else if (threadIdx.x == 0) {
            set_status(status, MHDPIC_ST_SORT_CAP);
        }
    }
}

// All particle arrays gathered through the permutation in one pass: every
// plane q of element size esz[q] (4 or 8 bytes) is read at perm[r] and written
// at r.
struct Planes {
    const void *src[8];
    void *dst[8];
    int esz[8];
    int n;
};

__global__ void k_gather_all(int64_t np, const int32_t *__restrict__ perm, Planes pl)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < np;
         r += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = perm[r];
        if (i < 0 || i >= np)   // never taken for a valid permutation
            i = r;
        for (int q = 0; q < pl.n; ++q) {
            if (pl.esz[q] == 16)
                reinterpret_cast<int4 *>(pl.dst[q])[r] = __ldg(reinterpret_cast<const int4 *>(pl.src[q]) + i);
            else if (pl.esz[q] == 8)
                reinterpret_cast<unsigned long long *>(pl.dst[q])[r] =
                    __ldg(reinterpret_cast<const unsigned long long *>(pl.src[q]) + i);
            else
                reinterpret_cast<unsigned int *>(pl.dst[q])[r] =
                    __ldg(reinterpret_cast<const unsigned int *>(pl.src[q]) + i);
        }
    }
}

__global__ void k_perm_out(int64_t np, const int32_t *__restrict__ perm, int64_t *__restrict__ out)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < np;
         r += (int64_t)gridDim.x * blockDim.x)
        out[r] = perm[r];
}

// Items per brick: ceil(count / ITEM_MAX_PARTICLES) near-equal pieces.
__global__ void k_brick_items(Ctx c, const int64_t *__restrict__ brick_start,
                              const int32_t *__restrict__ offset, int32_t *__restrict__ nitems_of)
{
    int64_t nbt = c.nbricks_total;
    int vol = c.brick[0] * c.brick[1] * c.brick[2];
    for (int64_t gb = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gb < nbt;
         gb += (int64_t)gridDim.x * blockDim.x) {
        int bx = find_box(brick_start, c.nbox, gb);
        const BoxDev &b = c.boxes[bx];
        int64_t k0 = b.key0 + (gb - b.brick0) * vol;
        const int cnt = offset[k0 + vol] - offset[k0];
        if (cnt <= ITEM_MAX_PARTICLES) {
            nitems_of[gb] = cnt > 0 ? 1 : 0;
        } else if (c.halves) {
            const int na = offset[k0 + vol / 2] - offset[k0];
            nitems_of[gb] = (na + ITEM_MAX_PARTICLES - 1) / ITEM_MAX_PARTICLES +
                            (cnt - na + ITEM_MAX_PARTICLES - 1) / ITEM_MAX_PARTICLES;
        } else {
            nitems_of[gb] = (cnt + ITEM_MAX_PARTICLES - 1) / ITEM_MAX_PARTICLES;
        }
    }
}

__global__ void k_write_items(Ctx c, const int64_t *__restrict__ brick_start,
                              const int32_t *__restrict__ offset, const int32_t *__restrict__ nitems_of,
                              const int32_t *__restrict__ item_off, WorkItem *__restrict__ items,
                              int32_t *__restrict__ nitems)
{
    int64_t nbt = c.nbricks_total;
    int vol = c.brick[0] * c.brick[1] * c.brick[2];
    for (int64_t gb = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gb < nbt;
         gb += (int64_t)gridDim.x * blockDim.x) {
        int bx = find_box(brick_start, c.nbox, gb);
        const BoxDev &b = c.boxes[bx];
        int64_t k0 = b.key0 + (gb - b.brick0) * vol;
        const int64_t p0 = offset[k0], p1 = offset[k0 + vol];
        const int m = nitems_of[gb];
        if (m == 0)
            continue;
        int64_t o = item_off[gb];
        WorkItem w;
        w.box = bx;
        w.brick = (int32_t)(gb - b.brick0);
        if (p1 - p0 <= ITEM_MAX_PARTICLES) {
            // one item; a whole 64-cell brick splits at its 32nd cell (the
            // start of the second half)
            w.p0 = p0;
            w.p1 = p1;
            w.pm = c.halves ? (int64_t)offset[k0 + vol / 2] : -1;
            w.step = 1;
            w.count = (int32_t)(p1 - p0);
            items[o] = w;
        } else {
            // crowded: each part (the two halves, or the whole brick) into
            // m_p interleaved items, item t taking positions t, t + m_p, ...
            const int64_t pm = c.halves ? (int64_t)offset[k0 + vol / 2] : p1;
            const int64_t lo[2] = {p0, pm}, hi[2] = {pm, p1};
            for (int part = 0; part < 2; ++part) {
                const int64_t n = hi[part] - lo[part];
                const int mp = (int)((n + ITEM_MAX_PARTICLES - 1) / ITEM_MAX_PARTICLES);
                for (int t = 0; t < mp; ++t) {
                    w.p0 = lo[part] + t;
                    w.p1 = hi[part];
                    w.pm = -1;
                    w.step = mp;
                    w.count = (int32_t)((n - t + mp - 1) / mp);
                    items[o++] = w;
                }
            }
        }
        if (gb == nbt - 1)
            *nitems = item_off[nbt];
    }
}

__global__ void k_max_count(int64_t n, const int32_t *__restrict__ count, int32_t *out)
{
    int m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, count[i]);
    for (int o = 16; o > 0; o >>= 1)
        m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(out, m);
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

// Persistent grid of the staged key pass: as many blocks as fit on the
// device at once, at most one per chunk.
int key_grid(int64_t np)
{
    static int resident = 0;   // blocks of k_sort_keys_staged the device holds at once
    if (resident == 0) {
        int dev = 0, nsm = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_sort_keys_staged<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)KEY_SMEM);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sort_keys_staged<3, true>, KEY_THREADS, KEY_SMEM);
        resident = (per < 1 ? 1 : per) * (nsm < 1 ? 1 : nsm);
    }
    const int64_t chunks = (np + KEY_CHUNK - 1) / KEY_CHUNK;
    return (int)(chunks < resident ? (chunks < 1 ? 1 : chunks) : resident);
}

template <int D, bool AHEAD>
void launch_keys(const Ctx &c, const SortScratch &s, cudaStream_t st)
{
    cudaFuncSetAttribute(k_sort_keys_staged<D, AHEAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)KEY_SMEM);
    k_sort_keys_staged<D, AHEAD><<<key_grid(c.np), KEY_THREADS, KEY_SMEM, st>>>(c, s.count, s.pkey, s.pslot);
}

}  // namespace

int launch_sort(const Ctx &c, const SortScratch &s, int64_t *perm_out, int32_t *counts_out,
                cudaStream_t st)
{
    int launches = 0;
    cudaMemsetAsync(s.count, 0, sizeof(int32_t) * (c.nkeys + 2), st);
    if (c.np > 0) {
        if (c.prec == MHDPIC_PREC_MIXED) {
            const bool ahead = c.sort_ahead != 0.0;
            if (c.ndim == 3 && ahead)
                launch_keys<3, true>(c, s, st);
            else if (c.ndim == 3)
                launch_keys<3, false>(c, s, st);
            else if (ahead)
                launch_keys<2, true>(c, s, st);
            else
                launch_keys<2, false>(c, s, st);
        } else
            k_sort_keys_f64<<<grid_for(c.np, 256), 256, 0, st>>>(c, s.count, s.pkey, s.pslot);
        ++launches;
    }
    // key nkeys holds the particles that left the box: offset[nkeys] is the
    // number of live particles
    launches += scan(s.count, c.nkeys + 1, s.offset, s.scan_tmp, st);
    if (c.np > 0) {
        cudaMemsetAsync(s.perm, 0, sizeof(int32_t) * c.np, st);
        k_sort_scatter<<<grid_for(c.np, 256), 256, 0, st>>>(c.np, c.nkeys, s.pkey, s.pslot, s.offset, s.perm,
                                                           c.status);
        cudaMemsetAsync(s.big_count, 0, sizeof(int32_t), st);
        const int64_t nw = (c.nkeys + 8 * SEG_GROUP - 1) / (8 * SEG_GROUP);   // blocks of 8 warps
        int gb = (int)(nw < 152 * 16 ? (nw < 1 ? 1 : nw) : 152 * 16);
        k_sort_segments<<<gb, 256, 0, st>>>(c.nkeys, s.offset, s.perm, s.big_list, s.big_count);
        k_sort_big<<<152, 1024, 0, st>>>(s.offset, s.perm, s.big_list, s.big_count, s.pkey, c.status);
        launches += 3;
        if (perm_out) {
            k_perm_out<<<grid_for(c.np, 256), 256, 0, st>>>(c.np, s.perm, perm_out);
            ++launches;
        }
    }
    if (counts_out)
        cudaMemcpyAsync(counts_out, s.count, sizeof(int32_t) * c.nkeys, cudaMemcpyDeviceToDevice, st);
    // work list
    const int64_t *brick_start = s.brick_start;
    int32_t *nitems_of = s.brick_items;
    int32_t *item_off = s.item_off;
    int gb = grid_for(c.nbricks_total, 256);
    k_brick_items<<<gb, 256, 0, st>>>(c, brick_start, s.offset, nitems_of);
    launches += 1 + scan(nitems_of, c.nbricks_total, item_off, s.scan_tmp, st);
    cudaMemsetAsync(s.nitems, 0, sizeof(int32_t), st);
    k_write_items<<<gb, 256, 0, st>>>(c, brick_start, s.offset, nitems_of, item_off, s.items, s.nitems);
    ++launches;
    return launches;
}

int launch_gather(const Ctx &c, const int32_t *perm, const PSet &src, const PSet &dst, cudaStream_t st)
{
    if (c.np <= 0)
        return 0;
    Planes pl{};
    auto add = [&](const void *sp, void *dp, int esz, int ncomp) {
        for (int q = 0; q < ncomp; ++q) {
            pl.src[pl.n] = (const char *)sp + (size_t)q * c.np * esz;
            pl.dst[pl.n] = (char *)dp + (size_t)q * c.np * esz;
            pl.esz[pl.n] = esz;
            ++pl.n;
        }
    };
    if (c.prec == MHDPIC_PREC_MIXED) {
        add(src.pos, dst.pos, 16, 1);
        add(src.vel, dst.vel, 16, 1);
    } else {
        add(src.x, dst.x, 8, c.ndim);
        add(src.p64, dst.p64, 8, 3);
    }
    if (src.tinj && dst.tinj)
        add(src.tinj, dst.tinj, 8, 1);
    k_gather_all<<<grid_for(c.np, 256), 256, 0, st>>>(c.np, perm, pl);
    return 1;
}

int launch_gather_f64(int64_t np, const int32_t *perm, const double *src, double *dst, cudaStream_t st)
{
    if (np <= 0)
        return 0;
    Planes pl{};
    pl.src[0] = src;
    pl.dst[0] = dst;
    pl.esz[0] = 8;
    pl.n = 1;
    k_gather_all<<<grid_for(np, 256), 256, 0, st>>>(np, perm, pl);
    return 1;
}

namespace {
__global__ void k_clock_advance(double *clock, double dt) { clock[0] = clock[0] + dt; }
}  // namespace

int launch_clock_advance(double *clock, double dt, cudaStream_t st)
{
    k_clock_advance<<<1, 1, 0, st>>>(clock, dt);
    return 1;
}

namespace {

// Mark the slots [offset[nkeys], np) of the current set as free: after a push
// that applied a sort they still hold the states of an older step.
template <int PREC>
__global__ void k_mark_free(Ctx c, const int32_t *__restrict__ offset)
{
    const int64_t live = offset[c.nkeys];
    for (int64_t j = live + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < c.np;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (PREC == MHDPIC_PREC_MIXED) {
            c.pos[j] = make_int4(DEAD_CELL, 0, 0, 0);
            c.vel[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            c.x[j] = __longlong_as_double(0x7ff8000000000000ll);
            for (int d = 0; d < 3; ++d)
                c.p64[(int64_t)d * c.np + j] = 0.0;
        }
    }
}

__global__ void k_count_live(Ctx c, int prec, unsigned long long *out)
{
    unsigned long long n = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.np;
         i += (int64_t)gridDim.x * blockDim.x)
        n += prec == MHDPIC_PREC_MIXED ? (c.pos[i].x != DEAD_CELL) : !isnan(c.x[i]);
    for (int o = 16; o > 0; o >>= 1)
        n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0 && n)
        atomicAdd(out, n);
}

}  // namespace

int launch_mark_free(const Ctx &c, const SortScratch &s, cudaStream_t st)
{
    if (c.np <= 0)
        return 0;
    if (c.prec == MHDPIC_PREC_MIXED)
        k_mark_free<MHDPIC_PREC_MIXED><<<grid_for(c.np, 256), 256, 0, st>>>(c, s.offset);
    else
        k_mark_free<MHDPIC_PREC_FP64><<<grid_for(c.np, 256), 256, 0, st>>>(c, s.offset);
    return 1;
}

int launch_count_live(const Ctx &c, unsigned long long *out, cudaStream_t st)
{
    cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
    if (c.np <= 0)
        return 0;
    k_count_live<<<grid_for(c.np, 256), 256, 0, st>>>(c, c.prec, out);
    return 1;
}

int launch_max_count(const Ctx &c, const SortScratch &s, cudaStream_t st)
{
    cudaMemsetAsync(s.max_count, 0, sizeof(int32_t), st);
    k_max_count<<<grid_for(c.nkeys, 256), 256, 0, st>>>(c.nkeys, s.count, s.max_count);
    return 1;
}

}  // namespace mhdpic
