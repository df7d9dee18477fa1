// lvb_broad.cu -- the local Verlet buffer broad phase on sm_103a and its C-ABI.
//
// One step (lvb_step) is, in launch order:
//   k_check        displacement check of every particle (Eq. update), ballot
//                  + block-scan compaction of the flagged ids
//   PARTIAL trigger (local buffer, only flagged particles change):
//   k_p_update     new reference position and skin of each flagged particle
//                  (Eq. skin_formulus1 or another policy, capped per Eq.
//                  skin_formulus_mincell); marks the cells it leaves and the
//                  unflagged rows that list it
//   k_p_compact    drops flagged entries from those rows and the leavers
//                  from those cells
//   k_p_insert     moves the leavers into their new cells
//   k_rows         27-cell stencil search (Algorithm 1 on the extended
//                  spheres of Eq. bounding_sphere) for each flagged row
//   k_p_append     adds each flagged particle to its unflagged partners' rows
//   GLOBAL / ALWAYS trigger (Def. autoverlet / no buffer):
//   k_full_update, k_cells_clear, k_cells_insert, k_rows over all particles
//   then, only if a row outgrew its slack: k_rows (count), scan, k_rows (fill)
//   k_step_end     counters
// Every kernel after k_check is launched unconditionally and returns at once
// when the device-side counts say it has nothing to do, so a step needs no
// host round trip.
#include "lvb_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

using namespace lvb;

namespace {

constexpr int kNumSMs = 152;
constexpr int kThreads = 256;

struct DevState {
    int n, nwords, trigger, skin_kind;
    float skin_value, skin_dt, H, pad;
    GridGeom g;
    long long ncells;
    float4 *ref;
    float *rad;
    int *cell_of, *slot_of, *newcell;
    uint32_t *bits;
    int *fid;
    int *row_off, *row_len, *row_cap, *col;
    long long col_cap;
    int *trow, *trow_mark;
    int *cell_cnt, *cell_id;
    float4 *cell_ref;
    int *tcell, *tcell_mark;
    DevCounters *cnt;
    long long *blk;
    cudaGraphConditionalHandle h_path;      // which rebuild body runs
    cudaGraphConditionalHandle h_relayout;  // whether the re-layout body runs
    int use_cond;     // 1 inside a graph that owns the handles
    int small_max;    // flagged counts up to this use the one-block rebuild
};

// rebuild paths chosen by the check (values of h_path)
enum Path { PATH_SMALL = 0, PATH_BIG = 1, PATH_NONE = 2 };
// gate modes of the kernels
enum Gate { GATE_FLAGGED_BIG = 0, GATE_OVERFLOW = 1, GATE_ANY_FLAG = 2, GATE_ALWAYS = 3 };

__device__ __forceinline__ bool store_failed(const DevState &s)
{
    return (s.cnt->err & DERR_STORE) != 0;
}

// flagged count when the multi-kernel (big) partial path applies, else 0
__device__ __forceinline__ int big_nF(const DevState &s)
{
    const int nF = s.cnt->nF;
    return (store_failed(s) || nF <= s.small_max) ? 0 : nF;
}

// After a failed re-layout (DERR_STORE) the row offsets no longer fit the
// store, so every kernel that touches rows or cells stands down.
__device__ __forceinline__ int gated_items(const DevState &s, int gate)
{
    if (store_failed(s)) return 0;
    if (gate == GATE_FLAGGED_BIG) return big_nF(s);
    if (gate == GATE_OVERFLOW) return s.cnt->row_overflow ? s.n : 0;
    if (gate == GATE_ANY_FLAG) return s.cnt->nF ? s.n : 0;
    return s.n;
}

__device__ __forceinline__ void count_kernel(const DevState &s)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&s.cnt->kernels, 1ULL);
}

// ---------------------------------------------------------------------------
// a1: displacement check (Eq. update) and compaction of the flagged ids.
// One particle per thread: 32 B of coalesced loads (pos, ref); one ballot
// word per warp; one atomic per block.  The last block to finish publishes
// the step's flagged count, resets the per-step counters, keeps the
// statistics and, inside a graph, selects the rebuild body to run.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_check(const float4 *__restrict__ pos, DevState s)
{
    __shared__ int wcount[kThreads / 32];
    __shared__ int base;
    __shared__ bool last;
    count_kernel(s);
    const int i = blockIdx.x * kThreads + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool f = false;
    if (i < s.n) {
        float4 p = __ldg(pos + i);
        float4 q = s.ref[i];
        f = violates(p, q);
        if (!(isfinite(p.x) && isfinite(p.y) && isfinite(p.z))) atomicOr(&s.cnt->err, DERR_NAN);
    }
    const unsigned b = __ballot_sync(FULL, f);
    const int word = i >> 5;
    if (lane == 0) {
        if (word < s.nwords) s.bits[word] = b;
        wcount[warp] = __popc(b);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            int c = wcount[w];
            wcount[w] = tot;
            tot += c;
        }
        base = tot ? atomicAdd(&s.cnt->nF_accum, tot) : 0;
    }
    __syncthreads();
    if (f) s.fid[base + wcount[warp] + __popc(b & lanemask_lt())] = i;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&s.cnt->done_blocks, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    DevCounters *c = s.cnt;
    const int nF = atomicExch(&c->nF_accum, 0);
    c->done_blocks = 0;
    c->nF = nF;
    c->ntrow = 0;
    c->ntcell = 0;
    c->row_overflow = 0;
    int upd;
    if (s.trigger == LVB_TRIGGER_PARTIAL) upd = nF;
    else if (s.trigger == LVB_TRIGGER_GLOBAL) upd = nF ? s.n : 0;
    else upd = s.n;
    c->steps += 1;
    c->flagged_total += nF;
    c->updated_total += upd;
    if (upd) c->rebuild_steps += 1;
    c->last_flagged = nF;
    c->last_updated = upd;
    const bool ok = !(c->err & DERR_STORE);
    if (s.trigger == LVB_TRIGGER_PARTIAL && ok && nF > 0 && nF <= s.small_max)
        c->small_steps += 1;
    if (s.use_cond) {
        unsigned path;
        if (s.trigger == LVB_TRIGGER_PARTIAL)
            path = (!ok || nF == 0) ? PATH_NONE : (nF <= s.small_max ? PATH_SMALL : PATH_BIG);
        else
            path = (ok && upd) ? 1u : 0u;
        cudaGraphSetConditional(s.h_path, path);
    }
}

// ---------------------------------------------------------------------------
// Partial rebuild phases (PARTIAL trigger).  Each is a loop over its work
// items from k0 with stride `stride`, so that the same code runs as a
// grid-wide kernel (many flagged particles) or inside one block (few).
// ---------------------------------------------------------------------------

// a2 (+ bookkeeping for a3/a5): new reference position and skin of each
// flagged particle; marks the cell it leaves and every unflagged row that
// lists it.
__device__ __forceinline__ void ph_update(const DevState &s, const float4 *__restrict__ pos,
                                          const float4 *__restrict__ vel, int nF, int k0,
                                          int stride)
{
    for (int k = k0; k < nF; k += stride) {
        const int i = s.fid[k];
        const float4 p = pos[i];
        const float r = s.rad[i];
        const float4 v = vel ? vel[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float sk = skin_of(s.skin_kind, s.skin_value, s.skin_dt, s.H, r, v, 0.0f);
        s.ref[i] = make_float4(p.x, p.y, p.z, sk);
        const int nc = cell_key(s.g, p.x, p.y, p.z);
        const int oc = s.cell_of[i];
        s.newcell[i] = nc;
        if (nc != oc && atomicExch(&s.tcell_mark[oc], 1) == 0)
            s.tcell[atomicAdd(&s.cnt->ntcell, 1)] = oc;
        const int off = s.row_off[i], len = min(s.row_len[i], s.row_cap[i]);
        for (int e = 0; e < len; ++e) {
            const int j = s.col[off + e];
            if (!bit_of(s.bits, j) && atomicExch(&s.trow_mark[j], 1) == 0)
                s.trow[atomicAdd(&s.cnt->ntrow, 1)] = j;
        }
    }
}

// a5 (removal) and a3 (leavers): one item per touched row or cell.
__device__ __forceinline__ void ph_compact(const DevState &s, int k0, int stride)
{
    const int ntrow = s.cnt->ntrow, ntcell = s.cnt->ntcell;
    const int ccap = s.g.ccap;
    for (int k = k0; k < ntrow + ntcell; k += stride) {
        if (k < ntrow) {
            const int j = s.trow[k];
            const int off = s.row_off[j], len = min(s.row_len[j], s.row_cap[j]);
            int w = 0;
            for (int e = 0; e < len; ++e) {
                const int c = s.col[off + e];
                if (!bit_of(s.bits, c)) s.col[off + w++] = c;
            }
            s.row_len[j] = w;
            s.trow_mark[j] = 0;
        } else {
            const int c = s.tcell[k - ntrow];
            const long long base = (long long)c * ccap;
            const int cn = min(s.cell_cnt[c], ccap);
            int w = 0;
            for (int sl = 0; sl < cn; ++sl) {
                const int id = s.cell_id[base + sl];
                if (bit_of(s.bits, id) && s.newcell[id] != c) continue;   // left
                const float4 q = s.ref[id];
                s.cell_id[base + w] = id;
                s.cell_ref[base + w] = make_float4(q.x, q.y, q.z, __fadd_rn(s.rad[id], q.w));
                s.slot_of[id] = w;
                ++w;
            }
            s.cell_cnt[c] = w;
            s.tcell_mark[c] = 0;
        }
    }
}

// a3 (arrivals): leavers take a slot in their new cell; flagged particles
// that stay refresh their slot's copy of the reference state.
__device__ __forceinline__ void ph_insert(const DevState &s, int nF, int k0, int stride)
{
    const int ccap = s.g.ccap;
    for (int k = k0; k < nF; k += stride) {
        const int i = s.fid[k];
        const int nc = s.newcell[i];
        const float4 q = s.ref[i];
        const float4 cr = make_float4(q.x, q.y, q.z, __fadd_rn(s.rad[i], q.w));
        if (nc != s.cell_of[i]) {
            const int sl = atomicAdd(&s.cell_cnt[nc], 1);
            if (sl < ccap) {
                s.cell_id[(long long)nc * ccap + sl] = i;
                s.cell_ref[(long long)nc * ccap + sl] = cr;
                s.slot_of[i] = sl;
            } else {
                atomicOr(&s.cnt->err, DERR_CELL);
            }
            s.cell_of[i] = nc;
        } else {
            s.cell_ref[(long long)nc * ccap + s.slot_of[i]] = cr;
        }
    }
}

// a4: rows by the 27-cell stencil, one warp per row.  Lanes 0..26 each own
// one neighbour cell; a warp scan of their occupancies flattens the
// candidates, and every lane finds its candidate's cell with a 5-step
// shuffle binary search, so lanes stay busy across cell boundaries.
// fill = 0 counts only (row_len = count); fill = 1 also writes up to the
// row's capacity and raises row_overflow if the row does not fit.
// Items are fid[w] when `from_list`, else particle w.
__device__ __forceinline__ void ph_rows(const DevState &s, int nitems, bool from_list, int fill,
                                        int w0, int wstride)
{
    const int lane = threadIdx.x & 31;
    const int ccap = s.g.ccap;
    const int d0 = s.g.dim[0], d1 = s.g.dim[1], d2 = s.g.dim[2];
    for (int w = w0; w < nitems; w += wstride) {
        const int i = from_list ? s.fid[w] : w;
        const float4 q = s.ref[i];
        const float4 qi = make_float4(q.x, q.y, q.z, __fadd_rn(s.rad[i], q.w));
        const int ci = s.cell_of[i];
        const int cx = ci % d0, cy = (ci / d0) % d1, cz = ci / (d0 * d1);
        int cnt_l = 0, cid = 0;
        if (lane < 27) {
            const int x = cx + lane % 3 - 1, y = cy + (lane / 3) % 3 - 1, z = cz + lane / 9 - 1;
            if (x >= 0 && x < d0 && y >= 0 && y < d1 && z >= 0 && z < d2) {
                cid = (z * d1 + y) * d0 + x;
                cnt_l = min(s.cell_cnt[cid], ccap);
            }
        }
        const int incl = warp_incl_scan(cnt_l);
        const int excl = incl - cnt_l;
        const int total = __shfl_sync(FULL, incl, 31);
        const int off = fill ? s.row_off[i] : 0;
        const int cap = fill ? s.row_cap[i] : 0;
        int found = 0;
        for (int b0 = 0; b0 < total; b0 += 32) {
            const int k = b0 + lane;
            int c = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1)
                c += (__shfl_sync(FULL, incl, c + step - 1) <= k) ? step : 0;
            const int cc = __shfl_sync(FULL, cid, c);
            const int ex = __shfl_sync(FULL, excl, c);
            bool hit = false;
            int j = -1;
            if (k < total) {
                const long long idx = (long long)cc * ccap + (k - ex);
                j = s.cell_id[idx];
                if (j != i) hit = pair_hit(qi, s.cell_ref[idx]);
            }
            const unsigned m = __ballot_sync(FULL, hit);
            if (fill && hit) {
                const int p = found + __popc(m & lanemask_lt());
                if (p < cap) s.col[off + p] = j;
            }
            found += __popc(m);
        }
        if (lane == 0) {
            s.row_len[i] = found;
            if (fill && found > cap) atomicExch(&s.cnt->row_overflow, 1);
        }
    }
}

// a5 (insertion): flagged i joins the row of each unflagged partner.
__device__ __forceinline__ void ph_append(const DevState &s, int nF, int k0, int stride)
{
    for (int k = k0; k < nF; k += stride) {
        const int i = s.fid[k];
        const int len = s.row_len[i];
        if (len > s.row_cap[i]) continue;     // re-layout rebuilds everything
        const int off = s.row_off[i];
        for (int e = 0; e < len; ++e) {
            const int j = s.col[off + e];
            if (bit_of(s.bits, j)) continue;  // j's own new row lists i
            const int p = atomicAdd(&s.row_len[j], 1);
            if (p < s.row_cap[j]) s.col[s.row_off[j] + p] = i;
            else atomicExch(&s.cnt->row_overflow, 1);
        }
    }
}

__device__ __forceinline__ void set_relayout_cond(const DevState &s)
{
    if (s.use_cond)
        cudaGraphSetConditional(s.h_relayout,
                                (s.cnt->row_overflow && !store_failed(s)) ? 1u : 0u);
}

// The whole partial rebuild in one block, for steps with few flagged
// particles: five phases separated by block barriers instead of five
// launches.
constexpr int kFusedThreads = 1024;

__global__ void __launch_bounds__(kFusedThreads)
k_p_fused(const float4 *__restrict__ pos, const float4 *__restrict__ vel, DevState s)
{
    const int nF = s.cnt->nF;
    if (store_failed(s) || nF == 0 || nF > s.small_max) return;
    count_kernel(s);
    const int t = threadIdx.x;
    ph_update(s, pos, vel, nF, t, kFusedThreads);
    __syncthreads();
    ph_compact(s, t, kFusedThreads);
    __syncthreads();
    ph_insert(s, nF, t, kFusedThreads);
    __syncthreads();
    ph_rows(s, nF, true, 1, t >> 5, kFusedThreads / 32);
    __syncthreads();
    ph_append(s, nF, t, kFusedThreads);
    __syncthreads();
    if (t == 0) set_relayout_cond(s);
}

// Multi-kernel partial path, for steps with many flagged particles.
__global__ void __launch_bounds__(kThreads)
k_p_update(const float4 *__restrict__ pos, const float4 *__restrict__ vel, DevState s)
{
    const int nF = big_nF(s);
    if (!nF) return;
    count_kernel(s);
    ph_update(s, pos, vel, nF, blockIdx.x * kThreads + threadIdx.x, gridDim.x * kThreads);
}

__global__ void __launch_bounds__(kThreads)
k_p_compact(DevState s)
{
    if (!big_nF(s)) return;
    count_kernel(s);
    ph_compact(s, blockIdx.x * kThreads + threadIdx.x, gridDim.x * kThreads);
}

__global__ void __launch_bounds__(kThreads)
k_p_insert(DevState s)
{
    const int nF = big_nF(s);
    if (!nF) return;
    count_kernel(s);
    ph_insert(s, nF, blockIdx.x * kThreads + threadIdx.x, gridDim.x * kThreads);
}

__global__ void __launch_bounds__(kThreads, 4)
k_rows(DevState s, int gate, int fill)
{
    const int nitems = gated_items(s, gate);
    if (!nitems) return;
    count_kernel(s);
    ph_rows(s, nitems, gate == GATE_FLAGGED_BIG, fill, (blockIdx.x * kThreads + threadIdx.x) >> 5,
            (gridDim.x * kThreads) >> 5);
}

__global__ void __launch_bounds__(kThreads)
k_p_append(DevState s)
{
    const int nF = big_nF(s);
    if (!nF) return;
    count_kernel(s);
    ph_append(s, nF, blockIdx.x * kThreads + threadIdx.x, gridDim.x * kThreads);
}

// end of a rebuild body inside a graph: arm the re-layout body if needed
__global__ void k_set_relayout(DevState s)
{
    count_kernel(s);
    set_relayout_cond(s);
}

// end of the re-layout body
__global__ void k_relayout_done(DevState s)
{
    if (!s.cnt->row_overflow || store_failed(s)) return;
    count_kernel(s);
    s.cnt->relayouts += 1;
    s.cnt->row_overflow = 0;
}

// ---------------------------------------------------------------------------
// Full-build kernels (init, GLOBAL and ALWAYS triggers).
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
        const float sk = skin_of(s.skin_kind, s.skin_value, s.skin_dt, s.H, s.rad[i], v, 0.0f);
        s.ref[i] = make_float4(p.x, p.y, p.z, sk);
        s.cell_of[i] = cell_key(s.g, p.x, p.y, p.z);
    }
}

// Resume: take a saved reference state (xref, skin) instead of fresh ones.
// A skin that is negative, non-finite or above the cap is reported.
__global__ void __launch_bounds__(kThreads)
k_load_ref(const float4 *__restrict__ ref4, DevState s, unsigned *bad)
{
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < s.n; i += gridDim.x * kThreads) {
        const float4 q = ref4[i];
        float capv = __fsub_rn(s.H, s.rad[i]);
        if (!(capv > 0.0f)) capv = 0.0f;
        const bool ok = isfinite(q.x) && isfinite(q.y) && isfinite(q.z) && q.w >= 0.0f &&
                        q.w <= capv;
        if (!ok) atomicOr(bad, 1u);
        s.ref[i] = q;
        s.cell_of[i] = cell_key(s.g, q.x, q.y, q.z);
    }
}

__global__ void __launch_bounds__(kThreads)
k_cells_clear(DevState s, int gate)
{
    if (gated_items(s, gate) == 0) return;
    count_kernel(s);
    for (long long c = blockIdx.x * kThreads + threadIdx.x; c < s.ncells;
         c += (long long)gridDim.x * kThreads)
        s.cell_cnt[c] = 0;
}

// count_only: occupancy histogram (init, before the slot capacity is known)
__global__ void __launch_bounds__(kThreads)
k_cells_insert(DevState s, int gate, int count_only)
{
    const int items = gated_items(s, gate);
    if (!items) return;
    count_kernel(s);
    const int ccap = s.g.ccap;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < items; i += gridDim.x * kThreads) {
        const int c = s.cell_of[i];
        const int sl = atomicAdd(&s.cell_cnt[c], 1);
        if (count_only) continue;
        if (sl < ccap) {
            const float4 q = s.ref[i];
            s.cell_id[(long long)c * ccap + sl] = i;
            s.cell_ref[(long long)c * ccap + sl] =
                make_float4(q.x, q.y, q.z, __fadd_rn(s.rad[i], q.w));
            s.slot_of[i] = sl;
        } else {
            atomicOr(&s.cnt->err, DERR_CELL);
        }
    }
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
__global__ void k_radius_scan(const float4 *__restrict__ pos, int n, unsigned *out)
{
    // out[0] = max radius bits, out[1] = min radius bits, out[2] = bad input
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        const float4 p = pos[i];
        const bool ok = isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w) &&
                        p.w > 0.0f;
        if (!ok) { atomicOr(&out[2], 1u); continue; }
        atomicMax(&out[0], __float_as_uint(p.w));
        atomicMin(&out[1], __float_as_uint(p.w));
    }
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

__global__ void k_sum_int(const int *v, int n, unsigned long long *out)
{
    unsigned long long m = 0;
    for (int c = blockIdx.x * kThreads + threadIdx.x; c < n; c += gridDim.x * kThreads)
        m += (unsigned)v[c];
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

}  // namespace

// ===========================================================================
// Host side
// ===========================================================================
struct lvb_ctx {
    int64_t n = 0;
    int nwords = 0;
    int trigger = 0;
    lvb_skin_policy skin{};
    float L = 0, H = 0;
    GridGeom g{};
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
    // cached graph of one step, for the last (pos, vel) pointers seen
    bool use_graph = true;
    cudaGraphExec_t gexec = nullptr;
    const void *g_pos = nullptr, *g_vel = nullptr;
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
    void *ptrs[] = {s.ref, s.rad, s.cell_of, s.slot_of, s.newcell, s.bits, s.fid, s.row_off,
                    s.row_len, s.row_cap, s.col, s.trow, s.trow_mark, s.cell_cnt, s.cell_id,
                    s.cell_ref, s.tcell, s.tcell_mark, s.cnt, s.blk, c->ex_cnt, c->ex_off,
                    c->ex_i, c->ex_j, c->ex_d, c->scratch, c->sum64};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->cnt_h) cudaFreeHost(c->cnt_h);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
}

int from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return LVB_OK;
    if (e == cudaErrorMemoryAllocation) return LVB_ENOMEM;
    return LVB_EDEVICE;
}

int from_derr(unsigned e)
{
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

constexpr int kPerFlaggedGrid = 2 * kNumSMs;   // grid of the per-flagged kernels
constexpr int kDefaultSmallMax = 128;

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

void launch_relayout(lvb_ctx *c)
{
    k_rows<<<rows_grid(c), kThreads, 0, c->stream>>>(c->s, GATE_OVERFLOW, 0);
    launch_layout_scan(c, GATE_OVERFLOW);
    k_rows<<<rows_grid(c), kThreads, 0, c->stream>>>(c->s, GATE_OVERFLOW, 1);
    k_relayout_done<<<1, 1, 0, c->stream>>>(c->s);
}

// One step as direct launches (used while the caller's stream is being
// captured, or when graphs are switched off): every kernel is launched and
// the ones with nothing to do return at once.
void launch_step_direct(lvb_ctx *c, const float4 *pos, const float4 *v4)
{
    const cudaStream_t st = c->stream;
    DevState s = c->s;
    s.use_cond = 0;
    k_check<<<grid_for(c->n, kThreads, 1 << 30), kThreads, 0, st>>>(pos, s);
    if (c->trigger == LVB_TRIGGER_PARTIAL) {
        const int gp = kPerFlaggedGrid;
        k_p_fused<<<1, kFusedThreads, 0, st>>>(pos, v4, s);
        k_p_update<<<gp, kThreads, 0, st>>>(pos, v4, s);
        k_p_compact<<<gp, kThreads, 0, st>>>(s);
        k_p_insert<<<gp, kThreads, 0, st>>>(s);
        k_rows<<<rows_grid(c), kThreads, 0, st>>>(s, GATE_FLAGGED_BIG, 1);
        k_p_append<<<gp, kThreads, 0, st>>>(s);
    } else {
        const int gate = c->trigger == LVB_TRIGGER_GLOBAL ? GATE_ANY_FLAG : GATE_ALWAYS;
        const int gi = items_grid(c);
        k_full_update<<<gi, kThreads, 0, st>>>(pos, v4, s, gate);
        k_cells_clear<<<grid_for(c->ncells, kThreads, 4 * kNumSMs), kThreads, 0, st>>>(s, gate);
        k_cells_insert<<<gi, kThreads, 0, st>>>(s, gate, 0);
        k_rows<<<rows_grid(c), kThreads, 0, st>>>(s, gate, 1);
    }
    launch_relayout(c);
}

#define GK(x)                                  \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) return e_;      \
    } while (0)

cudaGraph_t add_cond(cudaGraphNode_t *out, cudaGraph_t g, cudaGraphNode_t dep,
                     cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                     unsigned size, cudaGraph_t *bodies, cudaError_t *err)
{
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = type;
    cp.conditional.size = size;
    *err = cudaGraphAddNode(out, g, &dep, nullptr, 1, &cp);
    if (*err != cudaSuccess) return nullptr;
    for (unsigned k = 0; k < size; ++k) bodies[k] = cp.conditional.phGraph_out[k];
    return bodies[0];
}

// The step as graph nodes: k_check, then a SWITCH (PARTIAL: body 0 = the
// one-block rebuild, body 1 = the multi-kernel rebuild, no body when
// nothing is flagged) or an IF (GLOBAL/ALWAYS: the full rebuild), then an
// IF for the row-store re-layout.  The check's last block and the end of
// each rebuild body set the conditions on the device.
cudaError_t build_step_nodes(lvb_ctx *c, cudaGraph_t g, cudaGraphNode_t *dep, const float4 *pos,
                             const float4 *v4)
{
    DevState s = c->s;
    cudaGraphConditionalHandle hp, hr;
    const bool partial = c->trigger == LVB_TRIGGER_PARTIAL;
    GK(cudaGraphConditionalHandleCreate(&hp, g, partial ? PATH_NONE : 0u,
                                        cudaGraphCondAssignDefault));
    GK(cudaGraphConditionalHandleCreate(&hr, g, 0u, cudaGraphCondAssignDefault));
    s.h_path = hp;
    s.h_relayout = hr;
    s.use_cond = 1;
    cudaGraphNode_t n = dep ? *dep : nullptr;
    GK(add_kernel(&n, g, &n, k_check, dim3(grid_for(c->n, kThreads, 1 << 30)), dim3(kThreads),
                  pos, s));
    cudaGraph_t bodies[2] = {nullptr, nullptr};
    cudaGraphNode_t cn = nullptr;
    cudaError_t err = cudaSuccess;
    const int gp = kPerFlaggedGrid;
    if (partial) {
        add_cond(&cn, g, n, hp, cudaGraphCondTypeSwitch, 2, bodies, &err);
        GK(err);
        cudaGraphNode_t b = nullptr;
        GK(add_kernel(&b, bodies[PATH_SMALL], &b, k_p_fused, dim3(1), dim3(kFusedThreads), pos,
                      v4, s));
        b = nullptr;
        cudaGraph_t big = bodies[PATH_BIG];
        GK(add_kernel(&b, big, &b, k_p_update, dim3(gp), dim3(kThreads), pos, v4, s));
        GK(add_kernel(&b, big, &b, k_p_compact, dim3(gp), dim3(kThreads), s));
        GK(add_kernel(&b, big, &b, k_p_insert, dim3(gp), dim3(kThreads), s));
        GK(add_kernel(&b, big, &b, k_rows, dim3(rows_grid(c)), dim3(kThreads), s,
                      (int)GATE_FLAGGED_BIG, 1));
        GK(add_kernel(&b, big, &b, k_p_append, dim3(gp), dim3(kThreads), s));
        GK(add_kernel(&b, big, &b, k_set_relayout, dim3(1), dim3(1), s));
    } else {
        add_cond(&cn, g, n, hp, cudaGraphCondTypeIf, 1, bodies, &err);
        GK(err);
        const int gate = c->trigger == LVB_TRIGGER_GLOBAL ? GATE_ANY_FLAG : GATE_ALWAYS;
        const int gi = items_grid(c);
        cudaGraph_t full = bodies[0];
        cudaGraphNode_t b = nullptr;
        GK(add_kernel(&b, full, &b, k_full_update, dim3(gi), dim3(kThreads), pos, v4, s, gate));
        GK(add_kernel(&b, full, &b, k_cells_clear,
                      dim3(grid_for(c->ncells, kThreads, 4 * kNumSMs)), dim3(kThreads), s, gate));
        GK(add_kernel(&b, full, &b, k_cells_insert, dim3(gi), dim3(kThreads), s, gate, 0));
        GK(add_kernel(&b, full, &b, k_rows, dim3(rows_grid(c)), dim3(kThreads), s, gate, 1));
        GK(add_kernel(&b, full, &b, k_set_relayout, dim3(1), dim3(1), s));
    }
    cudaGraph_t rl[1] = {nullptr};
    cudaGraphNode_t rn = nullptr;
    add_cond(&rn, g, cn, hr, cudaGraphCondTypeIf, 1, rl, &err);
    GK(err);
    cudaGraphNode_t b = nullptr;
    const ScanArgs a = layout_args(c);
    const int nb = (int)c->nblk;
    GK(add_kernel(&b, rl[0], &b, k_rows, dim3(rows_grid(c)), dim3(kThreads), s,
                  (int)GATE_OVERFLOW, 0));
    GK(add_kernel(&b, rl[0], &b, k_scan_reduce, dim3(nb), dim3(kThreads), a, s,
                  (int)GATE_OVERFLOW));
    GK(add_kernel(&b, rl[0], &b, k_scan_top, dim3(1), dim3(kThreads), a, s, (int)GATE_OVERFLOW,
                  nb));
    GK(add_kernel(&b, rl[0], &b, k_scan_down, dim3(nb), dim3(kThreads), a, s,
                  (int)GATE_OVERFLOW));
    GK(add_kernel(&b, rl[0], &b, k_rows, dim3(rows_grid(c)), dim3(kThreads), s,
                  (int)GATE_OVERFLOW, 1));
    GK(add_kernel(&b, rl[0], &b, k_relayout_done, dim3(1), dim3(1), s));
    if (dep) *dep = rn;
    return cudaSuccess;
}

int sync_counters(lvb_ctx *c)
{
    cudaError_t e = cudaMemcpyAsync(c->cnt_h, c->s.cnt, sizeof(DevCounters),
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return from_cuda(e);
    return from_derr(c->cnt_h->err);
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
int export_layout(lvb_ctx *c, int mode, const float4 *pos, long long *total)
{
    int rc = ensure_export(c, 0);
    if (rc) return rc;
    const int gi = items_grid(c);
    k_ex_count<<<gi, kThreads, 0, c->stream>>>(c->s, mode, pos, c->ex_cnt);
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
    default: return "unknown status";
    }
}

static int init_impl(lvb_ctx **out, int64_t n, const float *pos_r, const float *ref4,
                     const lvb_box *box, const lvb_skin_policy *skin, int32_t trigger,
                     float cell_factor, const float *vel, const float *acc, void *stream)
{
    (void)acc;
    if (!out) return LVB_EINVAL;
    *out = nullptr;
    if (!pos_r || !box || !skin || n < 1 || n > INT32_MAX - 64) return LVB_EINVAL;
    if (!aligned16(pos_r) || (vel && !aligned16(vel)) || (ref4 && !aligned16(ref4)))
        return LVB_EINVAL;
    if (trigger < LVB_TRIGGER_PARTIAL || trigger > LVB_TRIGGER_ALWAYS) return LVB_EINVAL;
    if (skin->kind < LVB_SKIN_GLOBAL || skin->kind > LVB_SKIN_PAPER_KVDT) return LVB_EINVAL;
    if (!(skin->value >= 0.0f) || !std::isfinite(skin->value)) return LVB_EINVAL;
    if (skin->kind == LVB_SKIN_PAPER_KVDT && (!vel || !(skin->dt > 0.0f))) return LVB_EINVAL;
    if (!(cell_factor >= 1.0f) || !std::isfinite(cell_factor)) return LVB_EINVAL;
    for (int k = 0; k < 3; ++k)
        if (!(box->hi[k] > box->lo[k]) || !std::isfinite(box->lo[k]) || !std::isfinite(box->hi[k]))
            return LVB_EINVAL;

    cudaGetLastError();   // clear a stale error of an unrelated earlier call
    lvb_ctx *c = new (std::nothrow) lvb_ctx();
    if (!c) return LVB_ENOMEM;
    c->n = n;
    c->nwords = (int)((n + 31) / 32);
    c->trigger = trigger;
    c->skin = *skin;
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

    // radii: range and validity
    e = dalloc(&c->scratch, 8);
    if (e == cudaSuccess) e = dalloc(&c->sum64, 1);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->cnt_h, sizeof(DevCounters));
    if (e != cudaSuccess) return fail(from_cuda(e));
    unsigned init_h[3] = {0u, 0x7f800000u, 0u};
    e = cudaMemcpyAsync(c->scratch, init_h, sizeof(init_h), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(from_cuda(e));
    k_radius_scan<<<grid_for(n, kThreads, 4 * kNumSMs), kThreads, 0, st>>>(
        (const float4 *)pos_r, (int)n, c->scratch);
    unsigned rs[3];
    e = cudaMemcpyAsync(rs, c->scratch, sizeof(rs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(from_cuda(e));
    if (rs[2]) return fail(LVB_ENAN);
    float rmax, rmin;
    memcpy(&rmax, &rs[0], 4);
    memcpy(&rmin, &rs[1], 4);

    // geometry: cell edge, cap H, grid (at most 2048 cells per axis)
    double L = (double)cell_factor * 2.0 * (double)rmax * (1.0 + 1.0 / 128.0);
    double ext = 0.0;
    for (int k = 0; k < 3; ++k) ext = std::max(ext, (double)box->hi[k] - (double)box->lo[k]);
    if (ext / L > 2048.0) L = ext / 2048.0;
    long long ncells = 1;
    for (int k = 0; k < 3; ++k) {
        long long d = (long long)std::ceil(((double)box->hi[k] - (double)box->lo[k]) / L);
        d = std::max(1LL, std::min(d, 2048LL));
        c->g.dim[k] = (int)d;
        c->g.lo[k] = box->lo[k];
        ncells *= d;
    }
    if (ncells > (1LL << 28)) return fail(LVB_EINVAL);
    c->ncells = ncells;
    c->L = (float)L;
    c->H = (float)(0.5 * L * (1.0 - 1.0 / 256.0));
    c->g.invL = (float)(1.0 / L);
    if (!(rmax <= c->H)) return fail(LVB_EINVAL);

    c->nblk = (n + kScanBlock - 1) / kScanBlock;
    e = dalloc(&s.ref, n);
    if (e == cudaSuccess) e = dalloc(&s.rad, n);
    if (e == cudaSuccess) e = dalloc(&s.cell_of, n);
    if (e == cudaSuccess) e = dalloc(&s.slot_of, n);
    if (e == cudaSuccess) e = dalloc(&s.newcell, n);
    if (e == cudaSuccess) e = dalloc(&s.bits, c->nwords);
    if (e == cudaSuccess) e = dalloc(&s.fid, n);
    if (e == cudaSuccess) e = dalloc(&s.row_off, n);
    if (e == cudaSuccess) e = dalloc(&s.row_len, n);
    if (e == cudaSuccess) e = dalloc(&s.row_cap, n);
    if (e == cudaSuccess) e = dalloc(&s.trow, n);
    if (e == cudaSuccess) e = dalloc(&s.trow_mark, n);
    if (e == cudaSuccess) e = dalloc(&s.cell_cnt, ncells);
    if (e == cudaSuccess) e = dalloc(&s.tcell, ncells);
    if (e == cudaSuccess) e = dalloc(&s.tcell_mark, ncells);
    if (e == cudaSuccess) e = dalloc(&s.cnt, 1);
    if (e == cudaSuccess) e = dalloc(&s.blk, c->nblk + 1);
    if (e != cudaSuccess) return fail(from_cuda(e));
    cudaMemsetAsync(s.trow_mark, 0, sizeof(int) * n, st);
    cudaMemsetAsync(s.tcell_mark, 0, sizeof(int) * ncells, st);
    cudaMemsetAsync(s.cnt, 0, sizeof(DevCounters), st);
    cudaMemsetAsync(s.bits, 0, sizeof(uint32_t) * c->nwords, st);

    s.n = (int)n;
    s.small_max = kDefaultSmallMax;
    s.nwords = c->nwords;
    s.trigger = trigger;
    s.skin_kind = skin->kind;
    s.skin_value = skin->value;
    s.skin_dt = skin->dt;
    s.H = c->H;
    s.g = c->g;
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
        const double vmean = 4.0 / 3.0 * M_PI * (double)rmin * rmin * rmin;
        const double dense = 0.74 * L * L * L / std::max(vmean, 1e-30);
        long long cap = std::max<long long>(2LL * maxocc + 8, 32);
        cap = std::max<long long>(cap, (long long)std::min(dense * 0.5, 4096.0));
        cap = (cap + 31) / 32 * 32;
        cap = std::min<long long>(cap, 1 << 16);
        c->g.ccap = (int)cap;
        s.g.ccap = (int)cap;
    }
    e = dalloc(&s.cell_id, ncells * (long long)c->g.ccap);
    if (e == cudaSuccess) e = dalloc(&s.cell_ref, ncells * (long long)c->g.ccap);
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
    long long col_cap = std::max<long long>(needed + needed / 2 + 1024, 4096);
    if (col_cap > INT32_MAX) col_cap = INT32_MAX;
    if (needed > col_cap) return fail(LVB_ENOMEM);
    e = dalloc(&s.col, col_cap);
    if (e != cudaSuccess) return fail(from_cuda(e));
    s.col_cap = col_cap;
    c->s = s;
    k_rows<<<rows_grid(c), kThreads, 0, st>>>(s, GATE_ALWAYS, 1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(from_cuda(e));
    rc = sync_counters(c);
    if (rc) return fail(rc);
    *out = c;
    return LVB_OK;
}

int lvb_init(lvb_ctx **out, int64_t n, const float *pos_r, const lvb_box *box,
             const lvb_skin_policy *skin, int32_t trigger, float cell_factor,
             const float *vel, const float *acc, void *stream)
{
    return init_impl(out, n, pos_r, nullptr, box, skin, trigger, cell_factor, vel, acc, stream);
}

int lvb_init_resume(lvb_ctx **out, int64_t n, const float *pos_r, const float *ref4,
                    const lvb_box *box, const lvb_skin_policy *skin, int32_t trigger,
                    float cell_factor, const float *vel, const float *acc, void *stream)
{
    if (!ref4) return LVB_EINVAL;
    return init_impl(out, n, pos_r, ref4, box, skin, trigger, cell_factor, vel, acc, stream);
}

int lvb_step(lvb_ctx *c, const float *pos_r, const float *vel, const float *acc)
{
    (void)acc;
    if (!c || !pos_r || !aligned16(pos_r) || (vel && !aligned16(vel))) return LVB_EINVAL;
    if (c->skin.kind == LVB_SKIN_PAPER_KVDT && !vel) return LVB_EINVAL;
    cudaGetLastError();   // clear a stale error of an unrelated earlier call
    const cudaStream_t st = c->stream;
    const float4 *pos = (const float4 *)pos_r;
    const float4 *v4 = (const float4 *)vel;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return from_cuda(e);
    if (!c->use_graph || cs != cudaStreamCaptureStatusNone) {
        launch_step_direct(c, pos, v4);
        return from_cuda(cudaGetLastError());
    }
    if (!c->gexec || c->g_pos != pos_r || c->g_vel != vel) {
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        cudaGraph_t g = nullptr;
        e = cudaGraphCreate(&g, 0);
        if (e == cudaSuccess) e = build_step_nodes(c, g, nullptr, pos, v4);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gexec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->gexec = nullptr;
            return from_cuda(e);
        }
        c->g_pos = pos_r;
        c->g_vel = vel;
    }
    return from_cuda(cudaGraphLaunch(c->gexec, st));
}

int lvb_set_option(lvb_ctx *c, int32_t option, int64_t value)
{
    if (!c) return LVB_EINVAL;
    if (option == LVB_OPT_GRAPH) {
        c->use_graph = value != 0;
    } else if (option == LVB_OPT_SMALL_MAX) {
        if (value < 0 || value > INT32_MAX) return LVB_EINVAL;
        c->s.small_max = (int)value;
    } else {
        return LVB_EINVAL;
    }
    if (c->gexec) {   // rebuilt with the new setting on the next step
        cudaStreamSynchronize(c->stream);
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return LVB_OK;
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
    k_sum_int<<<items_grid(c), kThreads, 0, c->stream>>>(c->s.row_len, (int)c->n, c->sum64);
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
    o->cell_capacity = c->g.ccap;
    o->row_store_capacity = c->s.col_cap;
    o->kernels_executed = (int64_t)h.kernels;
    o->small_path_steps = h.small_steps;
    o->small_max = c->s.small_max;
    o->graphs = c->use_graph ? 1 : 0;
    o->cell_edge = c->L;
    o->rnl_max = c->H;
    for (int k = 0; k < 3; ++k) o->grid[k] = c->g.dim[k];
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
    v.rad = c->s.rad;
    v.kernels = &c->s.cnt->kernels;
    v.n = (int)c->n;
    return v;
}

int append_step_nodes(lvb_ctx *c, cudaGraph_t g, cudaGraphNode_t *dep, const float *pos_r,
                      const float *vel)
{
    return from_cuda(build_step_nodes(c, g, dep, (const float4 *)pos_r, (const float4 *)vel));
}
}  // namespace lvb
