// lvb_broad.cu -- the local Verlet buffer broad phase on sm_103a and its C-ABI.
//
// One step (lvb_step) is one cooperative launch of the step kernel k_step
// (lvb_step.cuh): displacement check and updates of the flagged particles,
// partial rebuild of the rows that change, re-layout of the row store when
// a row outgrew its slack, separated by grid-wide barriers.  This file holds
// the context (device memory, init, store growth, export) and the C-ABI.
#include "lvb_step.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

using namespace lvb;

namespace {

constexpr int kNumSMs = 152;
constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// Full-build kernels (init and store growth).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_full_update(const float4 *__restrict__ pos, const float4 *__restrict__ vel, DevState s,
              int gate)
{
    const int items = gated_items(s, gate);
    if (!items) return;
    count_kernel(s);
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < items; i += gridDim.x * kThreads) {
        const float4 p = pos[i];
        const float4 v = vel ? vel[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const SceneGeom &g = geom_of(s, i);
        const float sk = skin_of(s.skin_kind, s.skin_value, s.skin_dt, g.H, s.rad[i], v, 0.0f);
        s.ref[i] = make_float4(p.x, p.y, p.z, sk);
        s.cell_of[i] = cell_key(g, p.x, p.y, p.z);
    }
}

// Init with the learned policy: the network needs a whole warp, so one
// warp per particle; the list does not exist yet, so partners, age, the
// old-skin ratio and the cell occupancy enter as 0.
__global__ void __launch_bounds__(kThreads)
k_full_update_learned(const float4 *__restrict__ pos, const float4 *__restrict__ vel,
                      const float4 *__restrict__ acc, DevState s)
{
    count_kernel(s);
    const int lane = threadIdx.x & 31;
    for (int i = (blockIdx.x * kThreads + threadIdx.x) >> 5; i < s.n;
         i += (gridDim.x * kThreads) >> 5) {
        const float4 p = pos[i];
        const float4 v = vel ? vel[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 a = acc ? acc[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float r = s.rad[i];
        const SceneGeom &g = geom_of(s, i);
        float f[LVB_MLP_IN];
        skin_features(s, p, v, a, r, g, make_float4(0.f, 0.f, 0.f, 0.f), 0, 0, 0, f);
        const float sk = warp_skin(s, g, r, v, f);
        if (lane == 0) {
            s.ref[i] = make_float4(p.x, p.y, p.z, sk);
            s.cell_of[i] = cell_key(g, p.x, p.y, p.z);
        }
    }
}

// Resume: take a saved reference state (xref, skin) instead of fresh ones.
// A skin that is negative, non-finite or above the cap is reported.
__global__ void __launch_bounds__(kThreads)
k_load_ref(const float4 *__restrict__ ref4, DevState s, unsigned *bad)
{
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < s.n; i += gridDim.x * kThreads) {
        const float4 q = ref4[i];
        const SceneGeom &g = geom_of(s, i);
        float capv = __fsub_rn(g.H, s.rad[i]);
        if (!(capv > 0.0f)) capv = 0.0f;
        const bool ok = isfinite(q.x) && isfinite(q.y) && isfinite(q.z) && q.w >= 0.0f &&
                        q.w <= capv;
        if (!ok) atomicOr(bad, 1u);
        s.ref[i] = q;
        s.cell_of[i] = cell_key(g, q.x, q.y, q.z);
    }
}

__global__ void __launch_bounds__(kThreads)
k_cells_clear(DevState s, int gate)
{
    if (gated_items(s, gate) == 0) return;
    count_kernel(s);
    for (long long c = blockIdx.x * kThreads + threadIdx.x; c < s.ncells;
         c += (long long)gridDim.x * kThreads) {
        s.cell_cnt[c] = 0;
        s.cell_live[c] = 0;
        s.cell_rmax[c] = 0;
    }
}

// count_only: occupancy histogram (init, before the slot capacity is known)
__global__ void __launch_bounds__(kThreads)
k_cells_insert(DevState s, int gate, int count_only)
{
    const int items = gated_items(s, gate);
    if (!items) return;
    count_kernel(s);
    const int ccap = s.ccap;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < items; i += gridDim.x * kThreads) {
        const int c = s.cell_of[i];
        const int sl = atomicAdd(&s.cell_cnt[c], 1);
        if (count_only) continue;
        atomicAdd(&s.cell_live[c], 1);
        if (sl < ccap) {
            const float4 q = s.ref[i];
            const float R = __fadd_rn(s.rad[i], q.w);
            s.cell_id[(long long)c * ccap + sl] = i;
            s.cell_ref[(long long)c * ccap + sl] = make_float4(q.x, q.y, q.z, R);
            atomicMax(&s.cell_rmax[c], __float_as_int(R));
            s.slot_of[i] = sl;
        } else {
            atomicOr(&s.cnt->err, DERR_CELL);
        }
    }
}

// Rows of every particle from the cells (init, store growth): fill = 0
// counts only, 1 also writes.
__global__ void __launch_bounds__(kThreads, 4)
k_rows(DevState s, int gate, int fill, int carry = 0)
{
    const int nitems = gated_items(s, gate);
    if (!nitems) return;
    count_kernel(s);
    tr_enter(s, TR_ROWS);
    ph_rows(s, nitems, fill, (blockIdx.x * kThreads + threadIdx.x) >> 5,
            (gridDim.x * kThreads) >> 5, &s.cnt->row_overflow, carry != 0);
    tr_exit(s, TR_ROWS);
}

// Contact history: the rows copied aside before the host re-lays them out
// (store or cell growth), for k_rows to carry each entry's record.
__global__ void __launch_bounds__(kThreads) k_save_rows(DevState s)
{
    count_kernel(s);
    save_rows_pass(s);
}

// ---------------------------------------------------------------------------
// Exclusive scan of per-row sizes into offsets (three kernels: block sums,
// one-block scan of the sums, block scan + offset).  Used to lay out the row
// store (size = row_capacity(row_len)) and the exported CSR (size = count).
// ---------------------------------------------------------------------------
constexpr int kScanPer = 8;
constexpr int kScanBlock = kThreads * kScanPer;

struct ScanArgs {
    const int *len;      // n sizes (before the transform)
    int *off;            // n (+1 if total_slot) offsets out
    int *cap;            // optional: transformed sizes out
    int slack;           // 1: size = row_capacity(len); 0: size = len
    int n;
    long long *blk;      // ceil(n / kScanBlock) partials
    long long limit;     // total must not exceed this (else DERR_STORE)
    int write_total;     // write the total to off[n]
};

__device__ __forceinline__ int scan_size(const ScanArgs &a, int i)
{
    if (i >= a.n) return 0;
    const int l = a.len[i];
    return a.slack ? row_capacity(l) : l;
}

__device__ long long block_excl_scan(long long v, long long *total)
{
    __shared__ long long ws[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long y = lane < kThreads / 32 ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long t = __shfl_up_sync(FULL, y, o);
            if (lane >= o) y += t;
        }
        if (lane < kThreads / 32) ws[lane] = y;
    }
    __syncthreads();
    const long long before = warp ? ws[warp - 1] : 0;
    *total = ws[kThreads / 32 - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kThreads)
k_scan_reduce(ScanArgs a, DevState s, int gate)
{
    if (gated_items(s, gate) == 0) return;
    count_kernel(s);
    const int b = blockIdx.x;
    long long sum = 0;
    for (int k = 0; k < kScanPer; ++k) sum += scan_size(a, b * kScanBlock + k * kThreads + threadIdx.x);
    long long tot;
    block_excl_scan(sum, &tot);
    if (threadIdx.x == 0) a.blk[b] = tot;
}

__global__ void __launch_bounds__(kThreads)
k_scan_top(ScanArgs a, DevState s, int gate, int nb)
{
    if (gated_items(s, gate) == 0) return;
    count_kernel(s);
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += kThreads) {
        const int b = b0 + threadIdx.x;
        const long long v = b < nb ? a.blk[b] : 0;
        long long tot;
        const long long ex = block_excl_scan(v, &tot);
        if (b < nb) a.blk[b] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (a.write_total) a.off[a.n] = (int)min(carry, (long long)INT32_MAX);
        if (a.slack) {
            s.cnt->store_needed = carry;
            if (carry > a.limit) atomicOr(&s.cnt->err, DERR_STORE);
        }
    }
}

__global__ void __launch_bounds__(kThreads)
k_scan_down(ScanArgs a, DevState s, int gate)
{
    if (gated_items(s, gate) == 0) return;
    count_kernel(s);
    const int b = blockIdx.x;
    long long run = a.blk[b];
    for (int k = 0; k < kScanPer; ++k) {
        const int i = b * kScanBlock + k * kThreads + threadIdx.x;
        const int v = scan_size(a, i);
        long long tot;
        const long long ex = block_excl_scan(v, &tot);
        if (i < a.n) {
            const long long o = run + ex;
            a.off[i] = (int)min(o, (long long)INT32_MAX);
            if (a.cap) a.cap[i] = v;
        }
        run += tot;
    }
}

// ---------------------------------------------------------------------------
// Init helpers.
// ---------------------------------------------------------------------------
// out[0] = min radius bits, out[1] = bad input, out[2 + s] = max radius
// bits of scene s (positive floats order like their bit patterns);
// *r3sum += the sum of r^3 (binary64, for the mean particle volume)
__global__ void k_radius_scan(const float4 *__restrict__ pos, int n, const int *scene_of,
                              unsigned *out, double *r3sum)
{
    double r3 = 0.0;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        const float4 p = pos[i];
        const bool ok = isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w) &&
                        p.w > 0.0f;
        if (!ok) { atomicOr(&out[1], 1u); continue; }
        atomicMin(&out[0], __float_as_uint(p.w));
        atomicMax(&out[2 + (scene_of ? scene_of[i] : 0)], __float_as_uint(p.w));
        r3 += (double)p.w * (double)p.w * (double)p.w;
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) r3 += __shfl_xor_sync(FULL, r3, o);
    if ((threadIdx.x & 31) == 0 && r3 != 0.0) atomicAdd(r3sum, r3);
}

__global__ void k_radius_store(const float4 *__restrict__ pos, int n, float *rad)
{
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads)
        rad[i] = pos[i].w;
}

__global__ void k_max_int(const int *v, long long n, int *out)
{
    int m = 0;
    for (long long c = blockIdx.x * kThreads + threadIdx.x; c < n; c += (long long)gridDim.x * kThreads)
        m = max(m, v[c]);
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(FULL, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Live entries of the list (rows hold -1 where a pair was removed).
__global__ void k_count_live(DevState s, unsigned long long *out)
{
    unsigned long long m = 0;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < s.n; i += gridDim.x * kThreads) {
        const int off = s.row_off[i], len = min(s.row_len[i], s.row_cap[i]);
        for (int e = 0; e < len; ++e) m += s.col[off + e] >= 0 ? 1u : 0u;
    }
    for (int o = 16; o; o >>= 1) m += __shfl_xor_sync(FULL, m, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, m);
}

// ---------------------------------------------------------------------------
// Export kernels.  mode 0: symmetric rows; 1: upper pairs j > i;
// 2: contacts j > i with delta > 0 (Eq. delta) at positions pos.
// Rows are emitted in ascending j by ranking each entry within its row.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool ex_keep(const DevState &s, int mode, int i, int j,
                                        const float4 *pos, float4 pi, float *dl)
{
    if (j < 0) return false;   // a removed pair's slot
    if (mode == 0) return true;
    if (j <= i) return false;
    if (mode == 1) return true;
    const float4 pj = pos[j];
    const float d = overlap_rn(make_float4(pi.x, pi.y, pi.z, s.rad[i]),
                               make_float4(pj.x, pj.y, pj.z, s.rad[j]));
    *dl = d;
    return d > 0.0f;
}

__global__ void __launch_bounds__(kThreads)
k_ex_count(DevState s, int mode, const float4 *__restrict__ pos, int *cnt)
{
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < s.n; i += gridDim.x * kThreads) {
        const int off = s.row_off[i], len = min(s.row_len[i], s.row_cap[i]);
        const float4 pi = pos ? pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        int c = 0;
        for (int e = 0; e < len; ++e) {
            float d;
            c += ex_keep(s, mode, i, s.col[off + e], pos, pi, &d) ? 1 : 0;
        }
        cnt[i] = c;
    }
}

__global__ void __launch_bounds__(kThreads)
k_ex_write(DevState s, int mode, const float4 *__restrict__ pos, const int *out_off,
           int *out_i, int *out_j, float *out_d)
{
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < s.n; i += gridDim.x * kThreads) {
        const int off = s.row_off[i], len = min(s.row_len[i], s.row_cap[i]);
        const float4 pi = pos ? pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int o = out_off[i];
        for (int e = 0; e < len; ++e) {
            const int j = s.col[off + e];
            float d = 0.0f;
            if (!ex_keep(s, mode, i, j, pos, pi, &d)) continue;
            int rank = 0;
            for (int e2 = 0; e2 < len; ++e2) {
                const int j2 = s.col[off + e2];
                float d2;
                if (j2 < j && ex_keep(s, mode, i, j2, pos, pi, &d2)) ++rank;
            }
            if (out_i) out_i[o + rank] = i;
            out_j[o + rank] = j;
            if (out_d) out_d[o + rank] = d;
        }
    }
}

// Pairs i < j whose squared reference distance (the fixed binary32 formula
// of the list) lies within rel of their squared cutoff (binary32), compared
// in binary64: one thread per particle over the 27 cells around its cell.
// write = 0 counts into cnt[i]; 1 writes at off[i], ... (cell order).
__global__ void __launch_bounds__(kThreads)
k_near(DevState s, double rel, int write, int *cnt, const int *off, int *out_i, int *out_j)
{
    const int ccap = s.ccap;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < s.n; i += gridDim.x * kThreads) {
        const SceneGeom &g = geom_of(s, i);
        const int d0 = g.dim[0], d1 = g.dim[1], d2 = g.dim[2];
        const int ci = s.cell_of[i] - g.cell_base;
        const int cx = ci % d0, cy = (ci / d0) % d1, cz = ci / (d0 * d1);
        const float4 q = s.ref[i];
        const float Ri = __fadd_rn(s.rad[i], q.w);
        int k = 0, o = write ? off[i] : 0;
        for (int t = 0; t < 27; ++t) {
            const int x = cx + t % 3 - 1, y = cy + (t / 3) % 3 - 1, z = cz + t / 9 - 1;
            if (x < 0 || x >= d0 || y < 0 || y >= d1 || z < 0 || z >= d2) continue;
            const long long base = (long long)(g.cell_base + (z * d1 + y) * d0 + x) * ccap;
            const int m = min(s.cell_cnt[g.cell_base + (z * d1 + y) * d0 + x], ccap);
            for (int e = 0; e < m; ++e) {
                const int j = s.cell_id[base + e];
                if (j <= i) continue;
                const float4 rj = s.cell_ref[base + e];
                const float dd = sqdist_rn(q.x, q.y, q.z, rj.x, rj.y, rj.z);
                const float c = __fadd_rn(Ri, rj.w);
                const float c2 = __fmul_rn(c, c);
                if (fabs((double)dd - (double)c2) <= rel * (double)c2) {
                    if (write) {
                        out_i[o + k] = i;
                        out_j[o + k] = j;
                    }
                    ++k;
                }
            }
        }
        if (!write) cnt[i] = k;
    }
}

}  // namespace

// ===========================================================================
// Host side
// ===========================================================================
struct lvb_ctx {
    int64_t n = 0;
    int nwords = 0;
    int trigger = 0;
    lvb_skin_policy skin{};
    int nscenes = 0;
    std::vector<SceneGeom> sg;      // host copy of the per-scene geometry
    SceneGeom *sg_d = nullptr;
    int *scene_of_d = nullptr;
    int ccap = 0;
    long long ncells = 0;
    cudaStream_t stream = nullptr;
    DevState s{};
    DevCounters *cnt_h = nullptr;   // pinned mirror
    long long nblk = 0;
    // export scratch
    int *ex_cnt = nullptr, *ex_off = nullptr;
    int *ex_i = nullptr, *ex_j = nullptr;
    float *ex_d = nullptr;
    long long ex_cap = 0;
    unsigned *scratch = nullptr;    // small device scratch (init reductions)
    unsigned long long *sum64 = nullptr;
    // launch shape of the step kernel: block size, and the blocks that fit
    // on the device at once (cooperative launch) for that size
    int block_threads = kStepMaxThreads;
    int step_blocks = 0;
    int version = 0;                // bumped whenever the step kernel's arguments change
    HostFlags *hflags = nullptr;    // mapped pinned host memory
    long long grows = 0;            // store or cell-slot growths done
    int grow = 1;                   // 0: requests to grow are ignored (LVB_OPT_GROW)
    bool history = false;           // contact history on (LVB_OPT_HISTORY)
    int ccap_want = 0;              // slots per cell asked for (LVB_OPT_CELL_CAPACITY)
    long long col_alloc = 0;        // entries allocated for the row store (s.col_cap,
                                    // the usable part, may be set lower: LVB_OPT_STORE_LIMIT)
    // lvb_step_host: two staging slots, each with device buffers for the
    // inputs (pos, vel, acc) and the outputs (flag words, flagged count);
    // the inputs come in on one copy stream and the outputs go out on
    // another, so both copies overlap the neighbouring steps' kernels
    struct {
        float4 *buf[2][3] = {};
        uint32_t *flags[2] = {};
        int *nf[2] = {};
        cudaStream_t in = nullptr, out = nullptr;
        cudaEvent_t copied[2] = {}, done[2] = {}, drained[2] = {};
        int slot = 0;
        bool ready = false;
    } hs;
};

namespace {

int grid_for(long long items, int per_block, int max_blocks)
{
    long long b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

template <class T>
cudaError_t dalloc(T **p, long long count)
{
    *p = nullptr;
    if (count <= 0) count = 1;
    return cudaMalloc((void **)p, sizeof(T) * (size_t)count);
}

void free_all(lvb_ctx *c)
{
    DevState &s = c->s;
    if (s.ubits && s.ubits != s.bits) cudaFree(s.ubits);
    void *ptrs[] = {s.ref, s.rad, s.cell_of, s.slot_of, s.fref, s.oref, s.bits, s.fid, s.sc_cnt,
                    s.sfid, s.sfref, s.fsc, s.row_off,
                    s.row_len, s.row_cap, s.col, s.cell_cnt, s.cell_id,
                    s.cell_ref, s.cnt, s.blk, c->ex_cnt, c->ex_off, c->ex_i, c->ex_j, c->ex_d,
                    c->scratch, c->sum64, c->sg_d, c->scene_of_d, s.born, s.cell_live,
                    s.cell_rmax,
                    s.lg_feat, s.lg_x, s.lg_t, s.lg_m, s.log_buf,
                    s.hist, s.pold, s.old_off, s.old_len, s.old_col, s.old_hist};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->cnt_h) cudaFreeHost(c->cnt_h);
    if (c->hflags) cudaFreeHost(c->hflags);
    for (auto &slot : c->hs.buf)
        for (float4 *p : slot)
            if (p) cudaFree(p);
    for (int k = 0; k < 2; ++k) {
        if (c->hs.flags[k]) cudaFree(c->hs.flags[k]);
        if (c->hs.nf[k]) cudaFree(c->hs.nf[k]);
        if (c->hs.copied[k]) cudaEventDestroy(c->hs.copied[k]);
        if (c->hs.done[k]) cudaEventDestroy(c->hs.done[k]);
        if (c->hs.drained[k]) cudaEventDestroy(c->hs.drained[k]);
    }
    if (c->hs.in) cudaStreamDestroy(c->hs.in);
    if (c->hs.out) cudaStreamDestroy(c->hs.out);
}

int from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return LVB_OK;
    if (e == cudaErrorMemoryAllocation) return LVB_ENOMEM;
    return LVB_EDEVICE;
}

int from_derr(unsigned e)
{
    if (e & DERR_SYNC) return LVB_ETIMEOUT;
    if (e & DERR_NAN) return LVB_ENAN;
    if (e & (DERR_CELL | DERR_STORE)) return LVB_EOVERFLOW;
    return LVB_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }


// Row-store scan of ctx rows (size = row_capacity(row_len)), gated.
ScanArgs layout_args(lvb_ctx *c);

void launch_layout_scan(lvb_ctx *c, int gate)
{
    const ScanArgs a = layout_args(c);
    const int nb = (int)c->nblk;
    k_scan_reduce<<<nb, kThreads, 0, c->stream>>>(a, c->s, gate);
    k_scan_top<<<1, kThreads, 0, c->stream>>>(a, c->s, gate, nb);
    k_scan_down<<<nb, kThreads, 0, c->stream>>>(a, c->s, gate);
}

int rows_grid(lvb_ctx *c) { return grid_for(c->n, kThreads / 32, 16 * kNumSMs); }
int items_grid(lvb_ctx *c) { return grid_for(c->n, kThreads, 4 * kNumSMs); }

ScanArgs layout_args(lvb_ctx *c)
{
    ScanArgs a{};
    a.len = c->s.row_len;
    a.off = c->s.row_off;
    a.cap = c->s.row_cap;
    a.slack = 1;
    a.n = (int)c->n;
    a.blk = c->s.blk;
    a.limit = c->s.col_cap;
    a.write_total = 0;
    return a;
}

// Blocks of the step kernel for the context's block size: as many as are
// resident at once (every block must be, the step's barriers wait for all),
// but no more than the check pass can use.
int size_step(lvb_ctx *c)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int smem = check_smem_bytes(c->block_threads);
    // the attribute belongs to the kernel, for every context of the process:
    // always the largest any block size needs
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_step<false, NoTail>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 check_smem_bytes(kStepMaxThreads));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step<false, NoTail>,
                                                          c->block_threads, smem);
    if (e != cudaSuccess) return from_cuda(e);
    if (per_sm < 1) return LVB_EDEVICE;
    const long long want = (c->n + (long long)c->block_threads * kCheckUnroll - 1) /
                           ((long long)c->block_threads * kCheckUnroll);
    c->step_blocks = (int)std::max<long long>(1, std::min<long long>(want, (long long)per_sm * sms));
    return LVB_OK;
}

int sync_counters(lvb_ctx *c)
{
    if (c->hs.ready) {   // outputs of lvb_step_host still on their way
        const cudaError_t eo = cudaStreamSynchronize(c->hs.out);
        if (eo != cudaSuccess) return from_cuda(eo);
    }
    cudaError_t e = cudaMemcpyAsync(c->cnt_h, c->s.cnt, sizeof(DevCounters),
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return from_cuda(e);
    return from_derr(c->cnt_h->err);
}

// Grows the row store and/or the cell slots when a kernel asked for it
// (over 75% full), then rebuilds the cells and rows from the current
// reference state -- the list is a function of that state alone, so the
// rebuilt list is the one the steps would have produced.  Synchronises;
// runs only on the rare steps that need it.
int grow_if_asked(lvb_ctx *c)
{
    volatile HostFlags *h = c->hflags;
    if (!c->grow || (!h->grow_store && !h->grow_cells)) return LVB_OK;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return from_cuda(e);
    DevState &s = c->s;
    const cudaStream_t st = c->stream;
    const bool cells = h->grow_cells != 0;
    if (c->history)   // the rows as they are, for carrying each entry's history
        k_save_rows<<<rows_grid(c), kThreads, 0, st>>>(s);
    if (cells && s.ccap < (1 << 16)) {
        const int ccap = std::min(std::max(2 * s.ccap, c->ccap_want), 1 << 16);
        cudaFree(s.cell_id);
        cudaFree(s.cell_ref);
        s.cell_id = nullptr;
        s.cell_ref = nullptr;
        e = dalloc(&s.cell_id, c->ncells * (long long)ccap);
        if (e == cudaSuccess) e = dalloc(&s.cell_ref, c->ncells * (long long)ccap);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(s.cell_id, 0xff, sizeof(int) * (size_t)c->ncells * ccap, st);
        if (e != cudaSuccess) return from_cuda(e);
        s.ccap = ccap;
        c->ccap = ccap;
        k_cells_clear<<<grid_for(c->ncells, kThreads, 4 * kNumSMs), kThreads, 0, st>>>(
            s, GATE_ALWAYS);
        k_cells_insert<<<items_grid(c), kThreads, 0, st>>>(s, GATE_ALWAYS, 0);
    }
    // rows: count, then a store with room to grow, then fill
    k_rows<<<rows_grid(c), kThreads, 0, st>>>(s, GATE_ALWAYS, 0);
    const long long cap0 = s.col_cap;
    s.col_cap = 1LL << 62;
    launch_layout_scan(c, GATE_ALWAYS);
    int rc = sync_counters(c);
    s.col_cap = cap0;
    if (rc) return rc;
    const long long need = c->cnt_h->store_needed;
    bool grown = false;
    if (need * 5 > s.col_cap * 3) {   // over 60%: grow
        const long long cap = std::min<long long>(2 * need + 8 * c->n + 1024, INT32_MAX);
        if (need > cap) return LVB_ENOMEM;
        cudaFree(s.col);
        s.col = nullptr;
        e = dalloc(&s.col, cap);
        if (e == cudaSuccess && c->history) {
            cudaFree(s.hist);
            s.hist = nullptr;
            e = dalloc(&s.hist, cap);
        }
        if (e != cudaSuccess) return from_cuda(e);
        s.col_cap = cap;
        c->col_alloc = cap;
        grown = true;
    }
    k_rows<<<rows_grid(c), kThreads, 0, st>>>(s, GATE_ALWAYS, 1, c->history ? 1 : 0);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return from_cuda(e);
    if (grown && c->history) {   // the copy-aside store follows the store's size
        cudaFree(s.old_col);
        cudaFree(s.old_hist);
        s.old_col = nullptr;
        s.old_hist = nullptr;
        e = dalloc(&s.old_col, c->col_alloc);
        if (e == cudaSuccess) e = dalloc(&s.old_hist, c->col_alloc);
        if (e != cudaSuccess) return from_cuda(e);
    }
    h->grow_store = 0;
    h->grow_cells = 0;
    c->grows += 1;
    c->version += 1;
    return sync_counters(c);
}

int ensure_export(lvb_ctx *c, long long need)
{
    cudaError_t e = cudaSuccess;
    if (!c->ex_cnt) e = dalloc(&c->ex_cnt, c->n);
    if (e == cudaSuccess && !c->ex_off) e = dalloc(&c->ex_off, c->n + 1);
    if (e != cudaSuccess) return from_cuda(e);
    if (need > c->ex_cap) {
        cudaStreamSynchronize(c->stream);
        if (c->ex_i) cudaFree(c->ex_i);
        if (c->ex_j) cudaFree(c->ex_j);
        if (c->ex_d) cudaFree(c->ex_d);
        c->ex_i = c->ex_j = nullptr;
        c->ex_d = nullptr;
        c->ex_cap = 0;
        long long cap = std::max(need, 1024LL);
        e = dalloc(&c->ex_i, cap);
        if (e == cudaSuccess) e = dalloc(&c->ex_j, cap);
        if (e == cudaSuccess) e = dalloc(&c->ex_d, cap);
        if (e != cudaSuccess) return from_cuda(e);
        c->ex_cap = cap;
    }
    return LVB_OK;
}

// Count + scan the export of `mode`; returns the total through *total.
int export_scan(lvb_ctx *c, long long *total);

int export_layout(lvb_ctx *c, int mode, const float4 *pos, long long *total)
{
    int rc = ensure_export(c, 0);
    if (rc) return rc;
    const int gi = items_grid(c);
    k_ex_count<<<gi, kThreads, 0, c->stream>>>(c->s, mode, pos, c->ex_cnt);
    return export_scan(c, total);
}

// Exclusive scan of the per-particle counts ex_cnt into ex_off (n + 1
// entries, the total last); waits for the total.
int export_scan(lvb_ctx *c, long long *total)
{
    ScanArgs a{};
    a.len = c->ex_cnt;
    a.off = c->ex_off;
    a.cap = nullptr;
    a.slack = 0;
    a.n = (int)c->n;
    a.blk = c->s.blk;
    a.limit = 0;
    a.write_total = 1;
    const int nb = (int)c->nblk;
    k_scan_reduce<<<nb, kThreads, 0, c->stream>>>(a, c->s, GATE_ALWAYS);
    k_scan_top<<<1, kThreads, 0, c->stream>>>(a, c->s, GATE_ALWAYS, nb);
    k_scan_down<<<nb, kThreads, 0, c->stream>>>(a, c->s, GATE_ALWAYS);
    int tot = 0;
    cudaError_t e = cudaMemcpyAsync(&tot, c->ex_off + c->n, sizeof(int), cudaMemcpyDeviceToHost,
                                    c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return from_cuda(e);
    *total = tot;
    return LVB_OK;
}

int copy_out(lvb_ctx *c, void *dst, const void *src, size_t bytes)
{
    if (!bytes) return LVB_OK;
    return from_cuda(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream));
}

}  // namespace

extern "C" {

const char *lvb_strerror(int status)
{
    switch (status) {
    case LVB_OK: return "ok";
    case LVB_EINVAL: return "invalid argument";
    case LVB_ENOMEM: return "device allocation failed";
    case LVB_ECAPACITY: return "output buffer too small";
    case LVB_EDEVICE: return "CUDA error";
    case LVB_ENAN: return "non-finite position or radius";
    case LVB_EOVERFLOW: return "internal store overflow (cell slots or pair store)";
    case LVB_ESTATE: return "invalid call for the context state";
    case LVB_ELIMIT: return "input exceeds the entry point's fixed maximum size";
    case LVB_ETIMEOUT: return "a grid-wide barrier of the step kernel timed out";
    default: return "unknown status";
    }
}

static int init_impl(lvb_ctx **out, int nscenes, const int64_t *offsets, int64_t n,
                     const float *pos_r, const float *ref4, const lvb_box *boxes,
                     const lvb_skin_policy *skin, int32_t trigger, float cell_factor,
                     const float *vel, const float *acc, void *stream)
{
    if (!out) return LVB_EINVAL;
    *out = nullptr;
    if (!pos_r || !boxes || !skin || n < 1 || n > INT32_MAX - 64 || nscenes < 1) return LVB_EINVAL;
    if (!aligned16(pos_r) || (vel && !aligned16(vel)) || (ref4 && !aligned16(ref4)))
        return LVB_EINVAL;
    if (trigger < LVB_TRIGGER_PARTIAL || trigger > LVB_TRIGGER_ALWAYS) return LVB_EINVAL;
    if (trigger == LVB_TRIGGER_GLOBAL && nscenes > 1) return LVB_EINVAL;
    if (skin->kind < LVB_SKIN_GLOBAL || skin->kind > LVB_SKIN_LEARNED) return LVB_EINVAL;
    if (skin->kind == LVB_SKIN_LEARNED &&
        (!skin->mlp || !aligned16(skin->mlp) || !vel || !acc ||
         trigger != LVB_TRIGGER_PARTIAL || !(skin->dt > 0.0f)))
        return LVB_EINVAL;
    if (acc && !aligned16(acc)) return LVB_EINVAL;
    if (!(skin->value >= 0.0f) || !std::isfinite(skin->value)) return LVB_EINVAL;
    if (skin->kind == LVB_SKIN_PAPER_KVDT && (!vel || !(skin->dt > 0.0f))) return LVB_EINVAL;
    if (!(cell_factor >= 1.0f) || !std::isfinite(cell_factor)) return LVB_EINVAL;
    if (offsets) {
        if (offsets[0] != 0 || offsets[nscenes] != n) return LVB_EINVAL;
        for (int q = 0; q < nscenes; ++q)
            if (!(offsets[q + 1] > offsets[q])) return LVB_EINVAL;
    } else if (nscenes != 1) {
        return LVB_EINVAL;
    }
    for (int q = 0; q < nscenes; ++q)
        for (int k = 0; k < 3; ++k)
            if (!(boxes[q].hi[k] > boxes[q].lo[k]) || !std::isfinite(boxes[q].lo[k]) ||
                !std::isfinite(boxes[q].hi[k]))
                return LVB_EINVAL;

    cudaGetLastError();   // clear a stale error of an unrelated earlier call
    lvb_ctx *c = new (std::nothrow) lvb_ctx();
    if (!c) return LVB_ENOMEM;
    c->n = n;
    c->nwords = (int)((n + 31) / 32);
    c->trigger = trigger;
    c->skin = *skin;
    c->nscenes = nscenes;
    c->stream = (cudaStream_t)stream;
    DevState &s = c->s;
    const cudaStream_t st = c->stream;
    cudaError_t e = cudaSuccess;
    int rc = LVB_OK;
    auto fail = [&](int code) {
        cudaStreamSynchronize(st);
        free_all(c);
        delete c;
        return code;
    };

    // scene of every particle (only stored when there is more than one)
    if (nscenes > 1) {
        std::vector<int> so((size_t)n);
        for (int q = 0; q < nscenes; ++q)
            for (int64_t i = offsets[q]; i < offsets[q + 1]; ++i) so[(size_t)i] = q;
        e = dalloc(&c->scene_of_d, n);
        if (e == cudaSuccess)
            e = cudaMemcpy(c->scene_of_d, so.data(), sizeof(int) * (size_t)n,
                           cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(from_cuda(e));
    }

    // radii: range per scene and validity
    e = dalloc(&c->scratch, 2 + nscenes + 8);
    if (e == cudaSuccess) e = dalloc(&c->sum64, 1);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->cnt_h, sizeof(DevCounters));
    if (e == cudaSuccess)
        e = cudaHostAlloc((void **)&c->hflags, sizeof(HostFlags), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        memset(c->hflags, 0, sizeof(HostFlags));
        e = cudaHostGetDevicePointer((void **)&s.hflags, c->hflags, 0);
    }
    if (e != cudaSuccess) return fail(from_cuda(e));
    std::vector<unsigned> rs((size_t)nscenes + 2, 0u);
    rs[0] = 0x7f800000u;
    e = cudaMemcpyAsync(c->scratch, rs.data(), sizeof(unsigned) * rs.size(),
                        cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(from_cuda(e));
    cudaMemsetAsync(c->sum64, 0, sizeof(double), st);
    k_radius_scan<<<grid_for(n, kThreads, 4 * kNumSMs), kThreads, 0, st>>>(
        (const float4 *)pos_r, (int)n, c->scene_of_d, c->scratch, (double *)c->sum64);
    double r3sum = 0.0;
    e = cudaMemcpyAsync(rs.data(), c->scratch, sizeof(unsigned) * rs.size(),
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&r3sum, c->sum64, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(from_cuda(e));
    if (rs[1]) return fail(LVB_ENAN);
    const double r3mean = r3sum / (double)n;

    // per-scene geometry: cell edge, cap H, grid (at most 2048 cells per axis)
    c->sg.resize((size_t)nscenes);
    long long ncells = 0;
    double Lmax = 0.0;
    for (int q = 0; q < nscenes; ++q) {
        SceneGeom &g = c->sg[(size_t)q];
        memset(&g, 0, sizeof(g));
        float rmax;
        memcpy(&rmax, &rs[(size_t)q + 2], 4);
        double L = (double)cell_factor * 2.0 * (double)rmax * (1.0 + 1.0 / 128.0);
        const lvb_box &box = boxes[q];
        double ext = 0.0;
        for (int k = 0; k < 3; ++k) ext = std::max(ext, (double)box.hi[k] - (double)box.lo[k]);
        if (ext / L > 2048.0) L = ext / 2048.0;
        long long nc = 1;
        for (int k = 0; k < 3; ++k) {
            long long d = (long long)std::ceil(((double)box.hi[k] - (double)box.lo[k]) / L);
            d = std::max(1LL, std::min(d, 2048LL));
            g.dim[k] = (int)d;
            g.lo[k] = box.lo[k];
            g.hi[k] = box.hi[k];
            nc *= d;
        }
        g.cell_base = (int)ncells;
        ncells += nc;
        if (ncells > (1LL << 28)) return fail(LVB_EINVAL);
        g.L = (float)L;
        g.H = (float)(0.5 * L * (1.0 - 1.0 / 256.0));
        g.invL = (float)(1.0 / L);
        g.first = offsets ? (int)offsets[q] : 0;
        g.count = offsets ? (int)(offsets[q + 1] - offsets[q]) : (int)n;
        if (!(rmax <= g.H)) return fail(LVB_EINVAL);
        Lmax = std::max(Lmax, L);
    }
    c->ncells = ncells;
    e = dalloc(&c->sg_d, nscenes);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->sg_d, c->sg.data(), sizeof(SceneGeom) * (size_t)nscenes,
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(from_cuda(e));

    c->nblk = (n + kScanBlock - 1) / kScanBlock;
    e = dalloc(&s.ref, n);
    if (e == cudaSuccess) e = dalloc(&s.rad, n);
    if (e == cudaSuccess) e = dalloc(&s.cell_of, n);
    if (e == cudaSuccess) e = dalloc(&s.slot_of, n);
    if (e == cudaSuccess) e = dalloc(&s.fref, n);
    if (e == cudaSuccess) e = dalloc(&s.oref, n);
    if (e == cudaSuccess) e = dalloc(&s.bits, c->nwords);
    if (e == cudaSuccess) e = dalloc(&s.fid, n);
    if (nscenes > 1) {
        if (e == cudaSuccess) e = dalloc(&s.sc_cnt, 2LL * nscenes);
        if (e == cudaSuccess) e = dalloc(&s.sfid, n);
        if (e == cudaSuccess) e = dalloc(&s.sfref, n);
        if (e == cudaSuccess) e = dalloc(&s.fsc, n);
        if (e == cudaSuccess) e = cudaMemsetAsync(s.sc_cnt, 0, sizeof(int) * 2 * nscenes, st);
    }
    if (e == cudaSuccess) e = dalloc(&s.row_off, n);
    if (e == cudaSuccess) e = dalloc(&s.row_len, n);
    if (e == cudaSuccess) e = dalloc(&s.row_cap, n);
    if (e == cudaSuccess) e = dalloc(&s.cell_cnt, ncells);
    if (e == cudaSuccess) e = dalloc(&s.cell_live, ncells);
    if (e == cudaSuccess) e = dalloc(&s.cell_rmax, ncells);
    if (e == cudaSuccess) e = dalloc(&s.born, n);
    if (e == cudaSuccess) e = dalloc(&s.cnt, 1);
    // scan partials: the init/export scans use nblk, the step kernel's
    // re-layout one per block (at most 4 per SM)
    if (e == cudaSuccess) e = dalloc(&s.blk, std::max<long long>(c->nblk + 1, 4096));
    if (e != cudaSuccess) return fail(from_cuda(e));
    cudaMemsetAsync(s.born, 0, sizeof(int) * n, st);
    cudaMemsetAsync(s.cell_live, 0, sizeof(int) * ncells, st);
    cudaMemsetAsync(s.cell_rmax, 0, sizeof(int) * ncells, st);
    cudaMemsetAsync(s.cnt, 0, sizeof(DevCounters), st);
    cudaMemsetAsync(&s.cnt->tr_start, 0xff, sizeof(s.cnt->tr_start), st);
    cudaMemsetAsync(s.bits, 0, sizeof(uint32_t) * c->nwords, st);

    s.n = (int)n;
    s.bar_spins = kBarrierSpins;
    s.direct_max = kFlaggedDirectMax;
    s.reach = 2;
    s.check_regs = 1;
    s.ubits = s.bits;
    s.early_beta = 1.0f;
    s.nwords = c->nwords;
    s.trigger = trigger;
    s.skin_kind = skin->kind;
    s.skin_value = skin->value;
    s.skin_dt = skin->dt;
    s.mlp = (const lvb_mlp_weights *)skin->mlp;
    s.nscenes = nscenes;
    s.sg = c->sg_d;
    s.scene_of = c->scene_of_d;
    s.ncells = ncells;

    const float4 *pos = (const float4 *)pos_r;
    const float4 *v4 = (const float4 *)vel;
    const int gi = items_grid(c);
    k_radius_store<<<gi, kThreads, 0, st>>>(pos, (int)n, s.rad);
    if (ref4) {
        cudaMemsetAsync(c->scratch, 0, sizeof(unsigned), st);
        k_load_ref<<<gi, kThreads, 0, st>>>((const float4 *)ref4, s, c->scratch);
        unsigned bad = 0;
        e = cudaMemcpyAsync(&bad, c->scratch, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(from_cuda(e));
        if (bad) return fail(LVB_EINVAL);
    } else if (skin->kind == LVB_SKIN_LEARNED) {
        k_full_update_learned<<<grid_for(n, kThreads / 32, 16 * kNumSMs), kThreads, 0, st>>>(
            pos, v4, (const float4 *)acc, s);
    } else {
        k_full_update<<<gi, kThreads, 0, st>>>(pos, v4, s, GATE_ALWAYS);
    }

    // slot capacity from the initial occupancy (twice the fullest cell,
    // and room for a dense packing of mean-volume particles)
    cudaMemsetAsync(s.cell_cnt, 0, sizeof(int) * ncells, st);
    k_cells_insert<<<gi, kThreads, 0, st>>>(s, GATE_ALWAYS, 1);
    cudaMemsetAsync(c->scratch, 0, sizeof(int), st);
    k_max_int<<<grid_for(ncells, kThreads, 4 * kNumSMs), kThreads, 0, st>>>(s.cell_cnt, ncells,
                                                                           (int *)c->scratch);
    int maxocc = 0;
    e = cudaMemcpyAsync(&maxocc, c->scratch, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(from_cuda(e));
    {
        const double vmean = 4.0 / 3.0 * M_PI * r3mean;
        const double dense = 0.74 * Lmax * Lmax * Lmax / std::max(vmean, 1e-30);
        long long cap = std::max<long long>(2LL * maxocc + 8, 32);
        cap = std::max<long long>(cap, (long long)std::min(dense * 0.5, 4096.0));
        cap = (cap + 31) / 32 * 32;
        cap = std::min<long long>(cap, 1 << 16);
        c->ccap = (int)cap;
        s.ccap = (int)cap;
    }
    e = dalloc(&s.cell_id, ncells * (long long)c->ccap);
    if (e == cudaSuccess) e = dalloc(&s.cell_ref, ncells * (long long)c->ccap);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(s.cell_id, 0xff, sizeof(int) * (size_t)ncells * c->ccap, st);
    if (e != cudaSuccess) return fail(from_cuda(e));
    cudaMemsetAsync(s.cell_cnt, 0, sizeof(int) * ncells, st);
    k_cells_insert<<<gi, kThreads, 0, st>>>(s, GATE_ALWAYS, 0);

    // rows: count, lay out with slack, allocate the store, fill
    k_rows<<<rows_grid(c), kThreads, 0, st>>>(s, GATE_ALWAYS, 0);
    s.col_cap = (1LL << 62);
    c->s = s;
    launch_layout_scan(c, GATE_ALWAYS);
    rc = sync_counters(c);
    if (rc) return fail(rc);
    const long long needed = c->cnt_h->store_needed;
    long long col_cap = std::max<long long>(2 * needed + 8 * n + 1024, 4096);
    if (col_cap > INT32_MAX) col_cap = INT32_MAX;
    if (needed > col_cap) return fail(LVB_ENOMEM);
    e = dalloc(&s.col, col_cap);
    if (e != cudaSuccess) return fail(from_cuda(e));
    s.col_cap = col_cap;
    c->col_alloc = col_cap;
    c->s = s;
    k_rows<<<rows_grid(c), kThreads, 0, st>>>(s, GATE_ALWAYS, 1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(from_cuda(e));
    rc = sync_counters(c);
    if (rc) return fail(rc);
    rc = size_step(c);
    if (rc) return fail(rc);
    *out = c;
    return LVB_OK;
}

int lvb_init(lvb_ctx **out, int64_t n, const float *pos_r, const lvb_box *box,
             const lvb_skin_policy *skin, int32_t trigger, float cell_factor,
             const float *vel, const float *acc, void *stream)
{
    return init_impl(out, 1, nullptr, n, pos_r, nullptr, box, skin, trigger, cell_factor, vel,
                     acc, stream);
}

int lvb_batch_init(lvb_ctx **out, int32_t n_scenes, const int64_t *offsets, const float *pos_r,
                   const lvb_box *boxes, const lvb_skin_policy *skin, int32_t trigger,
                   float cell_factor, const float *vel, const float *acc, void *stream)
{
    if (!offsets || n_scenes < 1) return LVB_EINVAL;
    return init_impl(out, n_scenes, offsets, offsets[n_scenes], pos_r, nullptr, boxes, skin,
                     trigger, cell_factor, vel, acc, stream);
}

int lvb_scene_info(lvb_ctx *c, int32_t scene, lvb_scene_info_t *o)
{
    if (!c || !o || scene < 0 || scene >= c->nscenes) return LVB_EINVAL;
    const SceneGeom &g = c->sg[(size_t)scene];
    memset(o, 0, sizeof(*o));
    o->first = g.first;
    o->count = g.count;
    o->cell_edge = g.L;
    o->rnl_max = g.H;
    for (int k = 0; k < 3; ++k) o->grid[k] = g.dim[k];
    return LVB_OK;
}

int lvb_init_resume(lvb_ctx **out, int64_t n, const float *pos_r, const float *ref4,
                    const lvb_box *box, const lvb_skin_policy *skin, int32_t trigger,
                    float cell_factor, const float *vel, const float *acc, void *stream)
{
    if (!ref4) return LVB_EINVAL;
    return init_impl(out, 1, nullptr, n, pos_r, ref4, box, skin, trigger, cell_factor, vel, acc,
                     stream);
}

int lvb_batch_init_resume(lvb_ctx **out, int32_t n_scenes, const int64_t *offsets,
                          const float *pos_r, const float *ref4, const lvb_box *boxes,
                          const lvb_skin_policy *skin, int32_t trigger, float cell_factor,
                          const float *vel, const float *acc, void *stream)
{
    if (!offsets || !ref4 || n_scenes < 1) return LVB_EINVAL;
    return init_impl(out, n_scenes, offsets, offsets[n_scenes], pos_r, ref4, boxes, skin,
                     trigger, cell_factor, vel, acc, stream);
}

int lvb_step(lvb_ctx *c, const float *pos_r, const float *vel, const float *acc)
{
    if (!c || !pos_r || !aligned16(pos_r) || (vel && !aligned16(vel)) || (acc && !aligned16(acc)))
        return LVB_EINVAL;
    if (c->skin.kind == LVB_SKIN_PAPER_KVDT && !vel) return LVB_EINVAL;
    if (c->skin.kind == LVB_SKIN_LEARNED && (!vel || !acc)) return LVB_EINVAL;
    const float4 *a4 = (const float4 *)acc;
    cudaGetLastError();   // clear a stale error of an unrelated earlier call
    {
        const int rc = grow_if_asked(c);
        if (rc) return rc;
    }
    const cudaError_t e =
        launch_coop(k_step<false, NoTail>, dim3(c->step_blocks), dim3(c->block_threads),
                    c->s.check_regs ? (size_t)0 : (size_t)check_smem_bytes(c->block_threads),
                    c->stream,
                    (const float4 *)pos_r, (const float4 *)vel, a4, c->s, IntegrateArgs{},
                    NoTail{});
    return from_cuda(e);
}

int lvb_step_host(lvb_ctx *c, const float *pos_r, const float *vel, const float *acc,
                  uint32_t *bits, int32_t *n_flagged)
{
    if (!c || !pos_r) return LVB_EINVAL;
    if (c->skin.kind == LVB_SKIN_PAPER_KVDT && !vel) return LVB_EINVAL;
    if (c->skin.kind == LVB_SKIN_LEARNED && (!vel || !acc)) return LVB_EINVAL;
    auto &hs = c->hs;
    const size_t bytes = sizeof(float4) * (size_t)c->n;
    const size_t fbytes = sizeof(uint32_t) * (size_t)c->nwords;
    cudaError_t e = cudaSuccess;
    if (!hs.ready) {
        e = cudaStreamCreateWithFlags(&hs.in, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hs.out, cudaStreamNonBlocking);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
            e = cudaEventCreateWithFlags(&hs.copied[k], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hs.done[k], cudaEventDisableTiming);
            if (e == cudaSuccess)
                e = cudaEventCreateWithFlags(&hs.drained[k], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaMalloc(&hs.flags[k], fbytes);
            if (e == cudaSuccess) e = cudaMalloc(&hs.nf[k], sizeof(int));
        }
        if (e != cudaSuccess) return from_cuda(e);
        hs.ready = true;
    }
    const float *src[3] = {pos_r, vel, acc};
    const int k = hs.slot;
    for (int a = 0; a < 3; ++a)
        if (src[a] && !hs.buf[k][a]) {
            e = cudaMalloc(&hs.buf[k][a], bytes);
            if (e != cudaSuccess) {
                hs.buf[k][a] = nullptr;
                return from_cuda(e);
            }
        }
    // inputs: after the slot's previous step has read them
    e = cudaStreamWaitEvent(hs.in, hs.done[k], 0);
    for (int a = 0; a < 3 && e == cudaSuccess; ++a)
        if (src[a])
            e = cudaMemcpyAsync(hs.buf[k][a], src[a], bytes, cudaMemcpyHostToDevice, hs.in);
    if (e == cudaSuccess) e = cudaEventRecord(hs.copied[k], hs.in);
    // the step: after its inputs, and after the slot's previous outputs left
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, hs.copied[k], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, hs.drained[k], 0);
    if (e != cudaSuccess) return from_cuda(e);
    hs.slot ^= 1;
    const bool outs = bits || n_flagged;
    c->s.bits_out = outs ? hs.flags[k] : nullptr;
    c->s.nf_out = outs ? hs.nf[k] : nullptr;
    const int rc = lvb_step(c, (const float *)hs.buf[k][0],
                            vel ? (const float *)hs.buf[k][1] : nullptr,
                            acc ? (const float *)hs.buf[k][2] : nullptr);
    c->s.bits_out = nullptr;
    c->s.nf_out = nullptr;
    if (rc) return rc;
    e = cudaEventRecord(hs.done[k], c->stream);
    // outputs: copied out while the next step runs
    if (e == cudaSuccess && outs) {
        e = cudaStreamWaitEvent(hs.out, hs.done[k], 0);
        if (e == cudaSuccess && bits)
            e = cudaMemcpyAsync(bits, hs.flags[k], fbytes, cudaMemcpyDeviceToHost, hs.out);
        if (e == cudaSuccess && n_flagged)
            e = cudaMemcpyAsync(n_flagged, hs.nf[k], sizeof(int32_t), cudaMemcpyDeviceToHost,
                                hs.out);
        if (e == cudaSuccess) e = cudaEventRecord(hs.drained[k], hs.out);
    }
    return from_cuda(e);
}

int lvb_set_option(lvb_ctx *c, int32_t option, int64_t value)
{
    if (!c) return LVB_EINVAL;
    if (option == LVB_OPT_TRACE) {
        c->s.trace = value != 0;
    } else if (option == LVB_OPT_BLOCK_THREADS) {
        if (value != 256 && value != 512 && value != 1024) return LVB_EINVAL;
        const int old = c->block_threads;
        c->block_threads = (int)value;
        const int rc = size_step(c);
        if (rc) {
            c->block_threads = old;
            size_step(c);
            return rc;
        }
    } else if (option == LVB_OPT_COMPACT) {
        if (value != LVB_COMPACT_WARP && value != LVB_COMPACT_BLOCK) return LVB_EINVAL;
        c->s.compact_block = value == LVB_COMPACT_BLOCK;
    } else if (option == LVB_OPT_BARRIER_EXTRA) {
        if (value != 0 && value != 1) return LVB_EINVAL;
        c->s.bar_extra = (unsigned)value;
    } else if (option == LVB_OPT_BARRIER_SPINS) {
        if (value < 1 || value > kBarrierSpins) return LVB_EINVAL;
        c->s.bar_spins = (unsigned)value;
    } else if (option == LVB_OPT_DIRECT_MAX) {
        if (value < 0 || value > (1 << 20)) return LVB_EINVAL;
        c->s.direct_max = (int)value;
    } else if (option == LVB_OPT_EARLY) {
        if (value < 1 || value > 1000) return LVB_EINVAL;
        if (value < 1000 && (c->trigger != LVB_TRIGGER_PARTIAL || c->nscenes != 1))
            return LVB_EINVAL;
        DevState &s = c->s;
        if (value < 1000 && s.ubits == s.bits) {
            const cudaError_t e = dalloc(&s.ubits, c->nwords);
            if (e != cudaSuccess) {
                s.ubits = s.bits;
                return from_cuda(e);
            }
        }
        s.early_beta = (float)((double)value / 1000.0);
    } else if (option == LVB_OPT_CHECK_LOADS) {
        if (value != LVB_CHECK_REGS && value != LVB_CHECK_RING) return LVB_EINVAL;
        c->s.check_regs = value == LVB_CHECK_REGS;
    } else if (option == LVB_OPT_STENCIL_REACH) {
        if (value < 0 || value > 2) return LVB_EINVAL;
        c->s.reach = (int)value;
    } else if (option == LVB_OPT_CELL_CAPACITY) {
        if (value < 1 || value > (1 << 16)) return LVB_EINVAL;
        const int want = (int)((value + 31) / 32 * 32);
        if (want > c->ccap) {
            c->ccap_want = want;
            c->hflags->grow_cells = 1;   // grown before the next step
        }
    } else if (option == LVB_OPT_HISTORY) {
        if (value != 0 && value != 1) return LVB_EINVAL;
        if (value && c->trigger != LVB_TRIGGER_PARTIAL) return LVB_EINVAL;
        const cudaError_t ee = cudaStreamSynchronize(c->stream);
        if (ee != cudaSuccess) return from_cuda(ee);
        DevState &s = c->s;
        void *ptrs[] = {s.hist, s.pold, s.old_off, s.old_len, s.old_col, s.old_hist};
        for (void *q : ptrs)
            if (q) cudaFree(q);
        s.hist = s.pold = s.old_hist = nullptr;
        s.old_off = s.old_len = s.old_col = nullptr;
        c->history = false;
        if (value) {
            cudaError_t e = dalloc(&s.hist, c->col_alloc);
            if (e == cudaSuccess) e = dalloc(&s.pold, c->n);
            if (e == cudaSuccess) e = dalloc(&s.old_off, c->n);
            if (e == cudaSuccess) e = dalloc(&s.old_len, c->n);
            if (e == cudaSuccess) e = dalloc(&s.old_col, c->col_alloc);
            if (e == cudaSuccess) e = dalloc(&s.old_hist, c->col_alloc);
            if (e == cudaSuccess)
                e = cudaMemsetAsync(s.hist, 0, sizeof(float4) * (size_t)c->col_alloc, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) {
                void *qs[] = {s.hist, s.pold, s.old_off, s.old_len, s.old_col, s.old_hist};
                for (void *q : qs)
                    if (q) cudaFree(q);
                s.hist = s.pold = s.old_hist = nullptr;
                s.old_off = s.old_len = s.old_col = nullptr;
                return from_cuda(e);
            }
            c->history = true;
        }
    } else if (option == LVB_OPT_FORCE_RELAYOUT) {
        if (value != 1) return LVB_EINVAL;
        const int one = 1;
        const cudaError_t e = cudaMemcpyAsync(&c->s.cnt->force_relayout, &one, sizeof(one),
                                              cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) return from_cuda(cudaStreamSynchronize(c->stream));
        return from_cuda(e);
    } else if (option == LVB_OPT_GROW) {
        if (value != 0 && value != 1) return LVB_EINVAL;
        c->grow = (int)value;
    } else if (option == LVB_OPT_STORE_LIMIT) {
        if (value < 0) return LVB_EINVAL;
        c->s.col_cap = value == 0 ? c->col_alloc : std::min<long long>(value, c->col_alloc);
    } else {
        return LVB_EINVAL;
    }
    c->version += 1;
    return LVB_OK;
}

int lvb_trace(lvb_ctx *c, uint64_t *sum_ns, uint64_t *count)
{
    if (!c || !sum_ns || !count) return LVB_EINVAL;
    int rc = sync_counters(c);
    if (rc) return rc;
    for (int k = 0; k < kTraceSlots; ++k) {
        sum_ns[k] = c->cnt_h->tr_sum[k];
        count[k] = c->cnt_h->tr_cnt[k];
    }
    return LVB_OK;
}

int lvb_log_enable(lvb_ctx *c, int32_t horizon, int64_t capacity)
{
    if (!c || horizon < 1 || capacity < 1 || c->trigger != LVB_TRIGGER_PARTIAL) return LVB_EINVAL;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    DevState &s = c->s;
    if (e == cudaSuccess && !s.lg_feat) {
        e = dalloc(&s.lg_feat, c->n * (long long)LVB_MLP_IN);
        if (e == cudaSuccess) e = dalloc(&s.lg_x, c->n);
        if (e == cudaSuccess) e = dalloc(&s.lg_t, c->n);
        if (e == cudaSuccess) e = dalloc(&s.lg_m, c->n);
        if (e == cudaSuccess) e = cudaMemset(s.lg_t, 0xff, sizeof(int) * (size_t)c->n);
    }
    if (e == cudaSuccess && s.log_cap != capacity) {
        if (s.log_buf) cudaFree(s.log_buf);
        s.log_buf = nullptr;
        e = dalloc(&s.log_buf, capacity * (long long)(LVB_MLP_IN + 1));
    }
    if (e != cudaSuccess) return from_cuda(e);
    s.log_on = 1;
    s.log_horizon = horizon;
    s.log_cap = capacity;
    e = cudaMemsetAsync(&s.cnt->log_n, 0, sizeof(long long), c->stream);
    c->version += 1;
    return from_cuda(e);
}

int lvb_log_read(lvb_ctx *c, float *samples, int64_t cap, int64_t *n_samples)
{
    if (!c || !n_samples || cap < 0) return LVB_EINVAL;
    if (!c->s.log_on) return LVB_ESTATE;
    int rc = sync_counters(c);
    if (rc) return rc;
    const long long n = std::min<long long>(c->cnt_h->log_n, c->s.log_cap);
    *n_samples = n;
    if (n > cap || (n > 0 && !samples)) return LVB_ECAPACITY;
    rc = copy_out(c, samples, c->s.log_buf, sizeof(float) * (size_t)n * (LVB_MLP_IN + 1));
    if (rc) return rc;
    return from_cuda(cudaStreamSynchronize(c->stream));
}

int lvb_sync(lvb_ctx *c)
{
    if (!c) return LVB_EINVAL;
    return sync_counters(c);
}

int lvb_get_pairs(lvb_ctx *c, int32_t *row_ptr, int32_t *col, int64_t cap, int64_t *n_entries)
{
    if (!c || !row_ptr || !n_entries || cap < 0) return LVB_EINVAL;
    int rc = sync_counters(c);
    if (rc) return rc;
    long long total = 0;
    rc = export_layout(c, 0, nullptr, &total);
    if (rc) return rc;
    *n_entries = total;
    rc = copy_out(c, row_ptr, c->ex_off, sizeof(int) * (size_t)(c->n + 1));
    if (rc) return rc;
    if (total > cap || (total > 0 && !col)) {
        cudaStreamSynchronize(c->stream);
        return LVB_ECAPACITY;
    }
    rc = ensure_export(c, total);
    if (rc) return rc;
    k_ex_write<<<items_grid(c), kThreads, 0, c->stream>>>(c->s, 0, nullptr, c->ex_off, nullptr,
                                                          c->ex_j, nullptr);
    rc = copy_out(c, col, c->ex_j, sizeof(int) * (size_t)total);
    if (rc) return rc;
    return from_cuda(cudaStreamSynchronize(c->stream));
}

int lvb_get_pairs_ij(lvb_ctx *c, int32_t *pi, int32_t *pj, int64_t cap, int64_t *n_pairs)
{
    if (!c || !n_pairs || cap < 0) return LVB_EINVAL;
    int rc = sync_counters(c);
    if (rc) return rc;
    long long total = 0;
    rc = export_layout(c, 1, nullptr, &total);
    if (rc) return rc;
    *n_pairs = total;
    if (total > cap || (total > 0 && (!pi || !pj))) return LVB_ECAPACITY;
    rc = ensure_export(c, total);
    if (rc) return rc;
    k_ex_write<<<items_grid(c), kThreads, 0, c->stream>>>(c->s, 1, nullptr, c->ex_off, c->ex_i,
                                                          c->ex_j, nullptr);
    rc = copy_out(c, pi, c->ex_i, sizeof(int) * (size_t)total);
    if (!rc) rc = copy_out(c, pj, c->ex_j, sizeof(int) * (size_t)total);
    if (rc) return rc;
    return from_cuda(cudaStreamSynchronize(c->stream));
}

int lvb_get_near_cutoff(lvb_ctx *c, double rel, int32_t *pi, int32_t *pj, int64_t cap,
                        int64_t *n_pairs)
{
    // the 27 cells hold every pair up to the cell edge L >= 2H / (1 - 2^-8),
    // so up to rel = 2^-8 no pair near its cutoff lies outside them
    if (!c || !n_pairs || cap < 0 || !(rel >= 0.0) || !(rel <= 1.0 / 256.0)) return LVB_EINVAL;
    int rc = sync_counters(c);
    if (rc) return rc;
    rc = ensure_export(c, 0);
    if (rc) return rc;
    k_near<<<items_grid(c), kThreads, 0, c->stream>>>(c->s, rel, 0, c->ex_cnt, nullptr, nullptr,
                                                      nullptr);
    long long total = 0;
    rc = export_scan(c, &total);
    if (rc) return rc;
    *n_pairs = total;
    if (total > cap || (total > 0 && (!pi || !pj))) return LVB_ECAPACITY;
    rc = ensure_export(c, total);
    if (rc) return rc;
    k_near<<<items_grid(c), kThreads, 0, c->stream>>>(c->s, rel, 1, nullptr, c->ex_off, c->ex_i,
                                                      c->ex_j);
    rc = copy_out(c, pi, c->ex_i, sizeof(int) * (size_t)total);
    if (!rc) rc = copy_out(c, pj, c->ex_j, sizeof(int) * (size_t)total);
    if (rc) return rc;
    return from_cuda(cudaStreamSynchronize(c->stream));
}

int lvb_get_contacts(lvb_ctx *c, const float *pos_r, int32_t *ci, int32_t *cj, float *delta,
                     int64_t cap, int64_t *n_contacts)
{
    if (!c || !pos_r || !aligned16(pos_r) || !n_contacts || cap < 0) return LVB_EINVAL;
    int rc = sync_counters(c);
    if (rc) return rc;
    long long total = 0;
    rc = export_layout(c, 2, (const float4 *)pos_r, &total);
    if (rc) return rc;
    *n_contacts = total;
    if (total > cap || (total > 0 && (!ci || !cj))) return LVB_ECAPACITY;
    rc = ensure_export(c, total);
    if (rc) return rc;
    k_ex_write<<<items_grid(c), kThreads, 0, c->stream>>>(c->s, 2, (const float4 *)pos_r,
                                                          c->ex_off, c->ex_i, c->ex_j, c->ex_d);
    rc = copy_out(c, ci, c->ex_i, sizeof(int) * (size_t)total);
    if (!rc) rc = copy_out(c, cj, c->ex_j, sizeof(int) * (size_t)total);
    if (!rc && delta) rc = copy_out(c, delta, c->ex_d, sizeof(float) * (size_t)total);
    if (rc) return rc;
    return from_cuda(cudaStreamSynchronize(c->stream));
}

int lvb_get_flags(lvb_ctx *c, uint32_t *bits, int64_t *n_flagged)
{
    if (!c || !bits) return LVB_EINVAL;
    int rc = sync_counters(c);
    if (rc) return rc;
    if (n_flagged) *n_flagged = c->cnt_h->last_flagged;
    rc = copy_out(c, bits, c->s.bits, sizeof(uint32_t) * (size_t)c->nwords);
    if (rc) return rc;
    return from_cuda(cudaStreamSynchronize(c->stream));
}

int lvb_get_ref(lvb_ctx *c, float *ref4)
{
    if (!c || !ref4) return LVB_EINVAL;
    int rc = sync_counters(c);
    if (rc) return rc;
    rc = copy_out(c, ref4, c->s.ref, sizeof(float4) * (size_t)c->n);
    if (rc) return rc;
    return from_cuda(cudaStreamSynchronize(c->stream));
}

int lvb_stats(lvb_ctx *c, lvb_stats_t *o)
{
    if (!c || !o) return LVB_EINVAL;
    int rc = sync_counters(c);
    if (rc) return rc;
    cudaMemsetAsync(c->sum64, 0, sizeof(unsigned long long), c->stream);
    k_count_live<<<items_grid(c), kThreads, 0, c->stream>>>(c->s, c->sum64);
    unsigned long long entries = 0;
    cudaError_t e = cudaMemcpyAsync(&entries, c->sum64, sizeof(entries), cudaMemcpyDeviceToHost,
                                    c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return from_cuda(e);
    memset(o, 0, sizeof(*o));
    const DevCounters &h = *c->cnt_h;
    o->n = c->n;
    o->steps = h.steps;
    o->rebuild_steps = h.rebuild_steps;
    o->flagged_total = h.flagged_total;
    o->updated_total = h.updated_total;
    o->last_flagged = h.last_flagged;
    o->entries = (int64_t)entries;
    o->pairs = (int64_t)(entries / 2);
    o->relayouts = h.relayouts;
    o->grows = c->grows;
    o->cell_capacity = c->ccap;
    o->row_store_capacity = c->s.col_cap;
    o->kernels_executed = (int64_t)h.kernels;
    o->barriers = (int64_t)h.barriers;
    o->step_blocks = c->step_blocks;
    o->block_threads = c->block_threads;
    o->compaction = c->s.compact_block ? LVB_COMPACT_BLOCK : LVB_COMPACT_WARP;
    o->n_scenes = c->nscenes;
    o->rebuild_candidates = (int64_t)h.alg_cand;
    o->rebuild_direct = (int64_t)h.alg_direct;
    o->rebuild_edits = (int64_t)h.alg_edits;
    o->cell_edge = c->sg[0].L;
    o->rnl_max = c->sg[0].H;
    for (int k = 0; k < 3; ++k) o->grid[k] = c->sg[0].dim[k];
    return LVB_OK;
}

int lvb_set_stream(lvb_ctx *c, void *stream)
{
    if (!c) return LVB_EINVAL;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    c->stream = (cudaStream_t)stream;
    return from_cuda(e);
}

int lvb_destroy(lvb_ctx *c)
{
    if (!c) return LVB_EINVAL;
    if (c->hs.ready) {   // host-buffer copies still in flight land first
        cudaStreamSynchronize(c->hs.in);
        cudaStreamSynchronize(c->hs.out);
    }
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
    return LVB_OK;
}

}  // extern "C"

namespace lvb {
RowsView rows_view(lvb_ctx *c)
{
    RowsView v;
    v.row_off = c->s.row_off;
    v.row_len = c->s.row_len;
    v.row_cap = c->s.row_cap;
    v.col = c->s.col;
    v.hist = c->s.hist;
    v.rad = c->s.rad;
    v.kernels = &c->s.cnt->kernels;
    v.cnt = c->s.cnt;
    v.trace = &c->s.trace;
    v.sg = c->sg_d;
    v.scene_of = c->scene_of_d;
    v.nscenes = c->nscenes;
    v.n = (int)c->n;
    return v;
}

DevState step_state(lvb_ctx *c)
{
    return c->s;
}

void step_shape(lvb_ctx *c, int *blocks, int *threads)
{
    *blocks = c->step_blocks;
    *threads = c->block_threads;
}

cudaStream_t step_stream(lvb_ctx *c)
{
    return c->stream;
}

void small_scratch(lvb_ctx *c, unsigned **u32, unsigned long long **u64)
{
    *u32 = c->scratch;
    *u64 = c->sum64;
}

int grow_stores_if_asked(lvb_ctx *c)
{
    return grow_if_asked(c);
}

int graph_version(lvb_ctx *c)
{
    return c->version;
}
}  // namespace lvb
