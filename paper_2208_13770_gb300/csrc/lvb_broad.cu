// lvb_broad.cu -- the local Verlet buffer broad phase on sm_103a and its C-ABI.
//
// One step (lvb_step) is, in launch order:
//   k_check        displacement check of every particle (Eq. update), ballot
//                  + block-scan compaction of the flagged ids; with the
//                  PARTIAL trigger (local buffer) each block then gives the
//                  particles it flagged their new reference position and
//                  skin (Eq. skin_formulus1 or another policy, capped per
//                  Eq. skin_formulus_mincell), moves them to their new cell
//                  slots and queues the rows that listed them.  Its last
//                  block finishes small rebuilds itself:
//   k_inc_rows     27-cell stencil search (Algorithm 1 on the extended
//                  spheres of Eq. bounding_sphere) for each flagged row, and
//                  removal of the flagged entries from the queued rows
//   k_inc_append   adds each flagged particle to its unflagged partners' rows
//   GLOBAL / ALWAYS trigger (Def. autoverlet / no buffer):
//   k_full_update, k_cells_clear, k_cells_insert, k_rows over all particles
//   then, only if a row outgrew its slack: k_rows (count), scan, k_rows (fill)
// Inside a graph the check selects, on the device, which of these run
// (conditional nodes); launched directly, every kernel after k_check runs
// and returns at once when the device-side counts say it has nothing to do,
// so a step needs no host round trip either way.
#include "lvb_internal.cuh"

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

// Written by kernels straight into mapped host memory: requests to grow a
// store before it fills (read by the host before every step, no sync).
struct HostFlags {
    int grow_store;
    int grow_cells;
    long long store_needed;
};

struct DevState {
    int n, nwords, trigger, skin_kind;
    float skin_value, skin_dt;
    int nscenes, ccap;
    const SceneGeom *sg;    // per-scene geometry
    const int *scene_of;    // scene of each particle (null when one scene)
    long long ncells;
    float4 *ref;
    float *rad;
    int *cell_of, *slot_of;
    int *prevcell;    // cell of each flagged particle before its update
    uint32_t *bits;
    int *fid;
    int *row_off, *row_len, *row_cap, *col;
    long long col_cap;
    int *trow, *trow_mark;
    int *cell_cnt, *cell_id;
    float4 *cell_ref;
    DevCounters *cnt;
    long long *blk;
    const lvb_mlp_weights *mlp;   // skin network (LVB_SKIN_LEARNED)
    int *born;        // step of each particle's last update
    int *cell_live;   // particles whose reference position lies in each cell
    // rebuild log (training samples of the skin network)
    int log_on, log_horizon;
    long long log_cap;
    float *lg_feat;   // n x 8 features of the open record
    float4 *lg_x;     // position at which the record opened
    int *lg_t;        // step the record opened (-1: none)
    float *lg_m;      // largest squared displacement since
    float *log_buf;   // log_cap x 9 samples
    HostFlags *hflags;    // device view of the mapped host flags
    int trace;            // record per-kernel device time (LVB_OPT_TRACE)
    cudaGraphConditionalHandle h_path;      // which rebuild body runs
    int use_cond;     // 1 inside a graph that owns the handles
    int small_max;    // flagged counts up to this use the one-block rebuild
    int medium_max;   // ... above it the grid-wide passes with the medium grid, then the big one
};

// bodies of the step's SWITCH, chosen by the check (values of h_path); when
// the check's last block finishes the rebuild itself no body runs
enum Path { PATH_MEDIUM = 0, PATH_BIG = 1, PATH_RELAYOUT = 2, PATH_NONE = 3 };
// gate modes of the kernels
enum Gate { GATE_OVERFLOW = 1, GATE_ANY_FLAG = 2, GATE_ALWAYS = 3 };

__device__ __forceinline__ const SceneGeom &geom_of(const DevState &s, int i)
{
    return s.sg[s.nscenes == 1 ? 0 : s.scene_of[i]];
}

__device__ __forceinline__ bool store_failed(const DevState &s)
{
    return (s.cnt->err & DERR_STORE) != 0;
}

// flagged count when the grid-wide passes of a partial rebuild run (more
// flagged than the check's last block takes), else 0
__device__ __forceinline__ int grid_nF(const DevState &s)
{
    const int nF = s.cnt->nF;
    return (s.trigger != LVB_TRIGGER_PARTIAL || store_failed(s) || nF <= s.small_max) ? 0 : nF;
}

// After a failed re-layout (DERR_STORE) the row offsets no longer fit the
// store, so every kernel that touches rows or cells stands down.
__device__ __forceinline__ int gated_items(const DevState &s, int gate)
{
    if (store_failed(s)) return 0;
    if (gate == GATE_OVERFLOW) return s.cnt->row_overflow ? s.n : 0;
    if (gate == GATE_ANY_FLAG) return s.cnt->nF ? s.n : 0;
    return s.n;
}

__device__ __forceinline__ void count_kernel(const DevState &s)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&s.cnt->kernels, 1ULL);
}

// per-kernel trace: first entry and last exit over the kernel's blocks
__device__ __forceinline__ void tr_enter(const DevState &s, int slot)
{
    if (s.trace && threadIdx.x == 0) atomicMin(&s.cnt->tr_start[slot], global_ns());
}

__device__ __forceinline__ void tr_exit(const DevState &s, int slot)
{
    if (s.trace && (threadIdx.x & 31) == 0) atomicMax(&s.cnt->tr_end[slot], global_ns());
}

// ---------------------------------------------------------------------------
// Partial rebuild phases (PARTIAL trigger).  Each is a loop over its work
// items from k0 with stride `stride`, so that the same code runs as a
// grid-wide kernel (many flagged particles) or inside one block (few).
// ---------------------------------------------------------------------------

// Phases that walk a row or a cell run one warp per item (w0/wstride count
// warps): the lanes take the entries, so a step costs a few memory
// latencies however long the rows are, and atomics are warp-aggregated.

// Features of the skin network (lvb_mlp.h) from the state before the
// particle's update; q_old is its old reference state.
__device__ __forceinline__ void skin_features(const DevState &s, float4 p, float4 v, float4 a,
                                              float r, const SceneGeom &g, float4 q_old,
                                              int nrow, int age, int occ, float f[LVB_MLP_IN])
{
    const float d = __fmul_rn(2.0f, r);
    const float vm = __fsqrt_rn(sqdist_rn(v.x, v.y, v.z, 0.f, 0.f, 0.f));
    const float am = __fsqrt_rn(sqdist_rn(a.x, a.y, a.z, 0.f, 0.f, 0.f));
    f[0] = __fdiv_rn(__fmul_rn(vm, s.skin_dt), d);
    f[1] = __fdiv_rn(__fmul_rn(__fmul_rn(am, s.skin_dt), s.skin_dt), d);
    f[2] = __fdiv_rn(r, g.H);
    f[3] = (float)nrow;
    f[4] = (float)age;
    f[5] = q_old.w > 0.0f
               ? __fdiv_rn(__fsqrt_rn(sqdist_rn(p.x, p.y, p.z, q_old.x, q_old.y, q_old.z)), q_old.w)
               : 0.0f;
    f[6] = (float)occ;
    float w = __fsub_rn(__fsub_rn(p.x, g.lo[0]), r);
    w = fminf(w, __fsub_rn(__fsub_rn(g.hi[0], p.x), r));
    w = fminf(w, __fsub_rn(__fsub_rn(p.y, g.lo[1]), r));
    w = fminf(w, __fsub_rn(__fsub_rn(g.hi[1], p.y), r));
    w = fminf(w, __fsub_rn(__fsub_rn(p.z, g.lo[2]), r));
    w = fminf(w, __fsub_rn(__fsub_rn(g.hi[2], p.z), r));
    f[7] = __fdiv_rn(w, d);
}

// Skin of particle i by the context's policy; the learned policy needs the
// whole warp (all lanes compute the same value).
__device__ __forceinline__ float warp_skin(const DevState &s, const SceneGeom &g, float r,
                                           float4 v, const float f[LVB_MLP_IN])
{
    float prop = 0.0f;
    if (s.skin_kind == LVB_SKIN_LEARNED) {
        const float y = mlp_y_warp(s.mlp, f);
        prop = __fmul_rn(__fmul_rn(2.0f, r), relu(y));
    }
    return skin_of(s.skin_kind, s.skin_value, s.skin_dt, g.H, r, v, prop);
}

// a2 + a3 for one flagged particle i, run by one warp inside the check
// kernel (PARTIAL trigger), right after the block that checked i found it
// flagged:
//   * new reference position and skin (the policy's features come from the
//     state before the update; `step` is the number of the step being taken);
//   * its cell slot: a stayer refreshes the slot's copy of the reference
//     state; a leaver leaves a tombstone (-1) in its old slot and takes a
//     tombstone slot of its new cell (claimed with compare-and-swap) or a
//     fresh one at the end.  Slots of unflagged particles never change, so
//     after the check every cell holds the step's final reference states;
//   * every partner j of its old row is queued (once) for the removal of
//     the flagged entries; whether j is flagged itself is only known after
//     the check, so the removal pass skips flagged rows;
//   * the occupancy counts of the cells (a feature of the skin network) are
//     left as they were before the step: the rows pass moves the counts
//     after the check, from the old cell kept in prevcell[i].
// (pos and vel may have been written earlier in the same kernel by the DEM
// position half-step, so they are read through plain coherent loads.)
// Not inlined: it runs only for flagged particles, and as a call it keeps
// the check loop's registers free of its working set.
__device__ __noinline__ void update_move_warp(const DevState &s, int i, const float4 *pos,
                                                 const float4 *vel, const float4 *acc, int step)
{
    const int lane = threadIdx.x & 31;
    const int ccap = s.ccap;
    const float4 p = pos[i];
    const float r = s.rad[i];
    const float4 v = vel ? vel[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const SceneGeom &g = geom_of(s, i);
    const int nc = cell_key(g, p.x, p.y, p.z);
    const int oc = s.cell_of[i], so = s.slot_of[i];
    const int off = s.row_off[i], len = min(s.row_len[i], s.row_cap[i]);
    float f[LVB_MLP_IN];
    if (s.skin_kind == LVB_SKIN_LEARNED || s.log_on) {
        const float4 a = acc ? acc[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        skin_features(s, p, v, a, r, g, s.ref[i], len, step - s.born[i], s.cell_live[nc], f);
    }
    const float sk = warp_skin(s, g, r, v, f);
    const float4 cr = make_float4(p.x, p.y, p.z, __fadd_rn(r, sk));
    if (lane == 0) {
        s.ref[i] = make_float4(p.x, p.y, p.z, sk);
        s.born[i] = step;
        s.prevcell[i] = oc;
        if (s.log_on && s.lg_t[i] < 0) {
            s.lg_t[i] = step;
            s.lg_x[i] = p;
            s.lg_m[i] = 0.0f;
#pragma unroll
            for (int q = 0; q < LVB_MLP_IN; ++q) s.lg_feat[(long long)i * LVB_MLP_IN + q] = f[q];
        }
    }
    // old partners: queue their rows for the removal pass
    for (int e0 = 0; e0 < len; e0 += 32) {
        const int e = e0 + lane;
        int j = 0;
        bool push = false;
        if (e < len) {
            j = s.col[off + e];
            push = atomicExch(&s.trow_mark[j], 1) == 0;
        }
        const unsigned m = __ballot_sync(FULL, push);
        if (m) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&s.cnt->ntrow, __popc(m));
            base = __shfl_sync(FULL, base, 0);
            if (push) s.trow[base + __popc(m & lanemask_lt())] = j;
        }
    }
    // cell slot
    if (nc == oc) {
        if (lane == 0) s.cell_ref[(long long)oc * ccap + so] = cr;
        return;
    }
    if (lane == 0) s.cell_id[(long long)oc * ccap + so] = -1;
    const long long base = (long long)nc * ccap;
    const int cn = min(s.cell_cnt[nc], ccap);
    int slot = -1;
    for (int e0 = 0; e0 < cn && slot < 0; e0 += 32) {
        const int sl = e0 + lane;
        unsigned m = __ballot_sync(FULL, sl < cn && s.cell_id[base + sl] < 0);
        while (m && slot < 0) {
            const int src = __ffs(m) - 1;
            int won = 0;
            if (lane == src) won = atomicCAS(&s.cell_id[base + sl], -1, i) == -1;
            won = __shfl_sync(FULL, won, src);
            if (won) slot = e0 + src;
            m &= m - 1;
        }
    }
    if (lane == 0) {
        if (slot < 0) {
            slot = atomicAdd(&s.cell_cnt[nc], 1);
            if (slot * 4 >= ccap * 3) s.hflags->grow_cells = 1;
            if (slot < ccap) s.cell_id[base + slot] = i;
            else atomicOr(&s.cnt->err, DERR_CELL);
        }
        if (slot < ccap) {
            s.cell_ref[base + slot] = cr;
            s.slot_of[i] = slot;
        }
        s.cell_of[i] = nc;
    }
}

// Occupancy counts of the cells a flagged particle left and entered.
__device__ __forceinline__ void move_live_count(const DevState &s, int i)
{
    const int oc = s.prevcell[i], nc = s.cell_of[i];
    if (oc != nc) {
        atomicSub(&s.cell_live[oc], 1);
        atomicAdd(&s.cell_live[nc], 1);
    }
}

// a5 (removal): each queued unflagged row drops its flagged entries.  Rows
// are short, so a warp takes four rows at a time, eight lanes each (stable
// in-place compaction: every lane reads its entry before the ballot, and an
// entry only moves to a lower index).  A queued row that is flagged itself
// is rebuilt by the rows pass and only loses its queue mark here.  `w0` and
// `wstride` count warps.
__device__ __forceinline__ void compact_rows(const DevState &s, int w0, int wstride)
{
    const int lane = threadIdx.x & 31, sub = lane >> 3, l8 = lane & 7;
    const unsigned below = lanemask_lt() & (0xFFu << (sub * 8));
    const int ntrow = s.cnt->ntrow;
    for (int k0 = w0 * 4; k0 < ntrow; k0 += wstride * 4) {
        const int k = k0 + sub;
        int j = -1, off = 0, len = 0;
        bool act = k < ntrow;
        if (act) {
            j = s.trow[k];
            if (bit_of(s.bits, j)) {
                act = false;
                if (l8 == 0) s.trow_mark[j] = 0;
            } else {
                off = s.row_off[j];
                len = min(s.row_len[j], s.row_cap[j]);
            }
        }
        int mx = len;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) mx = max(mx, __shfl_xor_sync(FULL, mx, o));
        int w = 0;
        for (int e0 = 0; e0 < mx; e0 += 8) {
            const int e = e0 + l8;
            int c = 0;
            bool keep = false;
            if (act && e < len) {
                c = s.col[off + e];
                keep = !bit_of(s.bits, c);
            }
            const unsigned m = __ballot_sync(FULL, keep);
            if (keep) s.col[off + w + __popc(m & below)] = c;
            w += __popc((m >> (sub * 8)) & 0xFFu);
        }
        if (act && l8 == 0) {
            s.row_len[j] = w;
            s.trow_mark[j] = 0;
        }
    }
}

// a4: rows by the 27-cell stencil, one warp per row.  Lanes 0..26 each own
// one neighbour cell; a warp scan of their occupancies flattens the
// candidates, and every lane finds its candidate's cell with a 5-step
// shuffle binary search, so lanes stay busy across cell boundaries.
// fill = 0 counts only (row_len = count); fill = 1 also writes up to the
// row's capacity and raises row_overflow if the row does not fit.
// Items are fid[w] when `from_list`, else particle w.  Cell slots holding a
// tombstone (id < 0) are skipped.  The cells must hold the step's final
// reference states (after the check kernel's moves, or a full re-bin).
__device__ __forceinline__ void ph_rows(const DevState &s, int nitems, bool from_list, int fill,
                                        int w0, int wstride)
{
    const int lane = threadIdx.x & 31;
    const int ccap = s.ccap;
    const unsigned lt = lanemask_lt();
    for (int w = w0; w < nitems; w += wstride) {
        const int i = from_list ? s.fid[w] : w;
        const SceneGeom &g = geom_of(s, i);
        const int d0 = g.dim[0], d1 = g.dim[1], d2 = g.dim[2];
        const float4 q = s.ref[i];
        const float4 qi = make_float4(q.x, q.y, q.z, __fadd_rn(s.rad[i], q.w));
        const int ci = s.cell_of[i] - g.cell_base;
        const int cx = ci % d0, cy = (ci / d0) % d1, cz = ci / (d0 * d1);
        int cnt_l = 0, cid = 0;
        if (lane < 27) {
            const int x = cx + lane % 3 - 1, y = cy + (lane / 3) % 3 - 1, z = cz + lane / 9 - 1;
            if (x >= 0 && x < d0 && y >= 0 && y < d1 && z >= 0 && z < d2) {
                cid = g.cell_base + (z * d1 + y) * d0 + x;
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
                if (j >= 0 && j != i) hit = pair_hit(qi, s.cell_ref[idx]);
            }
            const unsigned m = __ballot_sync(FULL, hit);
            if (fill && hit) {
                const int p = found + __popc(m & lt);
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

// a5 (insertion): flagged i joins the row of each unflagged partner; one
// warp per flagged particle, one lane per partner.  Runs after the removal
// pass, so a pair that survives the update is removed and re-added once.
__device__ __forceinline__ void ph_append(const DevState &s, int nF, int w0, int wstride)
{
    const int lane = threadIdx.x & 31;
    for (int k = w0; k < nF; k += wstride) {
        const int i = s.fid[k];
        const int len = s.row_len[i];
        if (len > s.row_cap[i]) continue;     // re-layout rebuilds everything
        const int off = s.row_off[i];
        for (int e = lane; e < len; e += 32) {
            const int j = s.col[off + e];
            if (bit_of(s.bits, j)) continue;  // j's own new row lists i
            const int p = atomicAdd(&s.row_len[j], 1);
            if (p < s.row_cap[j]) s.col[s.row_off[j] + p] = i;
            else atomicExch(&s.cnt->row_overflow, 1);
        }
    }
}

__device__ __forceinline__ void set_relayout_cond(const DevState &s,
                                                  cudaGraphConditionalHandle h)
{
    if (s.use_cond)
        cudaGraphSetConditional(h, (s.cnt->row_overflow && !store_failed(s)) ? 1u : 0u);
}

constexpr int kCheckMaxThreads = 1024;   // largest check block (LVB_OPT_CHECK_THREADS)
constexpr int kCheckUnroll = 2;          // 32-particle chunks a warp has in flight
constexpr int kFusedMax = 1024;          // flagged particles the one-block form takes

// The rest of a partial rebuild, for steps with few flagged particles, in
// the last block of the check kernel: the flagged rows by the stencil and
// the removal pass together (they touch different rows), then, after a
// block barrier, the insertion pass.
__device__ __forceinline__ void last_block_rebuild(const DevState &s, int nF)
{
    const int t = threadIdx.x, nt = blockDim.x, wid = t >> 5, nw = nt >> 5;
    const long long c0 = clock64();
    ph_rows(s, nF, true, 1, wid, nw);
    compact_rows(s, wid, nw);
    for (int k = t; k < nF; k += nt) move_live_count(s, s.fid[k]);
    __syncthreads();
    const long long c1 = clock64();
    ph_append(s, nF, wid, nw);
    __syncthreads();
    if (t == 0) {
        s.cnt->ntrow = 0;   // the queue was filled by the check, used above
        atomicAdd(&s.cnt->fused_cycles[0], (unsigned long long)(c1 - c0));
        atomicAdd(&s.cnt->fused_cycles[1], (unsigned long long)(clock64() - c1));
    }
}

// ---------------------------------------------------------------------------
// a1: displacement check (Eq. update) and compaction of the flagged ids, for
// every particle; with `ia.active` each thread first performs the DEM
// driver's position half-step of its particle.  Each warp takes chunks of 32
// consecutive particles (kCheckUnroll of them in flight), writes one ballot
// word per chunk, and a chunk with flags costs the warp one atomic on the
// flagged count (warp-level compaction: no block barrier in the loop).  With
// the PARTIAL trigger the warp then updates the particles it flagged (a2,
// a3: update_move_warp), one after the other.  The grid holds one block per
// SM at 1024 threads (more, smaller blocks at 512 or 256).  The last block to
// finish publishes the step's flagged count, resets the per-step counters,
// keeps the statistics, runs the rest of the rebuild itself when few
// particles are flagged, and inside a graph selects the SWITCH body that
// still has to run.  kFused selects the form with the DEM half-step
// (ia.active), compiled apart so the plain form keeps its registers.
// ---------------------------------------------------------------------------
template <bool kFused>
__global__ void __launch_bounds__(kCheckMaxThreads, 1)
k_check(const float4 *__restrict__ pos_in, const float4 *vel, const float4 *acc, DevState s,
        IntegrateArgs ia)
{
    __shared__ bool last, s_inc;
    __shared__ int s_nF, s_small, s_step;
    count_kernel(s);
    tr_enter(s, TR_CHECK);
    const float4 *pos = kFused ? ia.pos : pos_in;
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    if (threadIdx.x == 0) {
        // updates in the check: PARTIAL trigger, row store intact (after a
        // failed re-layout the list stays invalid and nothing is touched)
        s_inc = s.trigger == LVB_TRIGGER_PARTIAL && !store_failed(s);
        s_step = (int)s.cnt->steps + 1;
    }
    __syncthreads();
    const bool inc = s_inc;
    const int step = s_step;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int stride = nwarps * 32;
    for (int c0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; c0 < s.n;
         c0 += stride * kCheckUnroll) {
        float4 p[kCheckUnroll], q[kCheckUnroll];
#pragma unroll
        for (int u = 0; u < kCheckUnroll; ++u) {
            const int i = c0 + u * stride + lane;
            if (i < s.n) {
                p[u] = kFused ? integrate_one(ia, geom_of(s, i), i) : __ldg(pos_in + i);
                q[u] = s.ref[i];
            }
        }
#pragma unroll
        for (int u = 0; u < kCheckUnroll; ++u) {
            const int cu = c0 + u * stride;   // chunk start, a multiple of 32
            if (cu >= s.n) break;             // uniform over the warp
            const int i = cu + lane;
            bool f = false;
            if (i < s.n) {
                f = violates(p[u], q[u]);
                if (!(isfinite(p[u].x) && isfinite(p[u].y) && isfinite(p[u].z)))
                    atomicOr(&s.cnt->err, DERR_NAN);
            }
            const unsigned b = __ballot_sync(FULL, f);
            if (lane == 0) s.bits[cu >> 5] = b;
            if (b) {
                int k0 = 0;
                if (lane == 0) k0 = atomicAdd(&s.cnt->nF_accum, __popc(b));
                k0 = __shfl_sync(FULL, k0, 0);
                if (f) s.fid[k0 + __popc(b & lt)] = i;
                if (inc) {
                    // the new positions of this chunk were written by the
                    // warp's own lanes (DEM form): make them visible to all
                    __syncwarp();
                    for (unsigned m = b; m; m &= m - 1)
                        update_move_warp(s, cu + __ffs(m) - 1, pos, vel, acc, step);
                }
            }
        }
    }
    __threadfence();   // flags, ids, updates and new positions visible to the last block
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&s.cnt->done_blocks, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    DevCounters *c = s.cnt;
    if (threadIdx.x == 0) {
        __threadfence();
        if (s.trace) {   // fold the kernels of the previous step
            for (int k = 1; k < kTraceSlots; ++k) {
                const unsigned long long a = c->tr_start[k], bb = c->tr_end[k];
                if (bb != 0 && bb >= a) {
                    c->tr_sum[k] += bb - a;
                    c->tr_cnt[k] += 1;
                }
                c->tr_start[k] = ~0ULL;
                c->tr_end[k] = 0;
            }
        }
        const int nF = atomicExch(&c->nF_accum, 0);
        c->done_blocks = 0;
        c->nF = nF;
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
        const bool small = inc && nF > 0 && nF <= s.small_max && nF <= kFusedMax;
        if (small) c->small_steps += 1;
        s_nF = nF;
        s_small = small;
    }
    __syncthreads();
    if (s_small) last_block_rebuild(s, s_nF);
    if (threadIdx.x == 0) {
        const int nF = s_nF;
        if (s.use_cond) {
            unsigned path;
            if (s.trigger == LVB_TRIGGER_PARTIAL) {
                if (!inc || nF == 0) path = PATH_NONE;
                else if (s_small) path = c->row_overflow ? PATH_RELAYOUT : PATH_NONE;
                else path = nF <= s.medium_max ? PATH_MEDIUM : PATH_BIG;
            } else {
                path = (!store_failed(s) && c->last_updated) ? 1u : 0u;
            }
            cudaGraphSetConditional(s.h_path, path);
        }
        if (s.trace) {
            c->tr_sum[TR_CHECK] += global_ns() - c->tr_start[TR_CHECK];
            c->tr_cnt[TR_CHECK] += 1;
            c->tr_start[TR_CHECK] = ~0ULL;
        }
    }
}

// The rest of a partial rebuild when more particles are flagged than the
// check's last block takes: the same two passes as grid-wide kernels (the
// SWITCH bodies PATH_MEDIUM and PATH_BIG differ only in grid size).
__global__ void __launch_bounds__(kThreads, 4)
k_inc_rows(DevState s)
{
    const int nF = grid_nF(s);
    if (!nF) return;
    count_kernel(s);
    tr_enter(s, TR_INC_ROWS);
    const int w0 = (blockIdx.x * kThreads + threadIdx.x) >> 5, nw = (gridDim.x * kThreads) >> 5;
    ph_rows(s, nF, true, 1, w0, nw);
    compact_rows(s, w0, nw);
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < nF; k += gridDim.x * kThreads)
        move_live_count(s, s.fid[k]);
    tr_exit(s, TR_INC_ROWS);
}

__global__ void __launch_bounds__(kThreads)
k_inc_append(DevState s)
{
    const int nF = grid_nF(s);
    if (!nF) return;
    count_kernel(s);
    tr_enter(s, TR_INC_APPEND);
    if (blockIdx.x == 0 && threadIdx.x == 0) s.cnt->ntrow = 0;   // used by k_inc_rows
    ph_append(s, nF, (blockIdx.x * kThreads + threadIdx.x) >> 5, (gridDim.x * kThreads) >> 5);
    tr_exit(s, TR_INC_APPEND);
}

__global__ void __launch_bounds__(kThreads, 4)
k_rows(DevState s, int gate, int fill)
{
    const int nitems = gated_items(s, gate);
    if (!nitems) return;
    count_kernel(s);
    const int slot = gate == GATE_OVERFLOW ? TR_RELAYOUT : TR_ROWS;
    tr_enter(s, slot);
    ph_rows(s, nitems, false, fill, (blockIdx.x * kThreads + threadIdx.x) >> 5,
            (gridDim.x * kThreads) >> 5);
    tr_exit(s, slot);
}

// end of a rebuild body inside a graph: arm its re-layout body if needed
__global__ void k_set_relayout(DevState s, cudaGraphConditionalHandle h)
{
    count_kernel(s);
    set_relayout_cond(s, h);
}

// end of the re-layout body
__global__ void k_relayout_done(DevState s)
{
    if (!s.cnt->row_overflow || store_failed(s)) return;
    count_kernel(s);
    s.cnt->relayouts += 1;
    s.cnt->row_overflow = 0;
    const long long need = s.cnt->store_needed;
    if (need * 4 > s.col_cap * 3) {        // over 75% of the store: grow it
        s.hflags->store_needed = need;
        s.hflags->grow_store = 1;
    }
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

// Rebuild log: every open record tracks the particle's largest displacement
// since it opened, and closes `horizon` steps later with label
// sqrt(max |x - x_open|^2) / d.
__global__ void __launch_bounds__(kThreads)
k_log_step(const float4 *__restrict__ pos, DevState s)
{
    count_kernel(s);
    const int step = (int)s.cnt->steps;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < s.n; i += gridDim.x * kThreads) {
        const int t = s.lg_t[i];
        if (t < 0) continue;
        const float4 p = pos[i];
        const float4 x0 = s.lg_x[i];
        const float m = fmaxf(s.lg_m[i], sqdist_rn(p.x, p.y, p.z, x0.x, x0.y, x0.z));
        if (step - t >= s.log_horizon) {
            const long long idx =
                (long long)atomicAdd((unsigned long long *)&s.cnt->log_n, 1ULL);
            if (idx < s.log_cap) {
                float *o = s.log_buf + idx * (LVB_MLP_IN + 1);
#pragma unroll
                for (int q = 0; q < LVB_MLP_IN; ++q) o[q] = s.lg_feat[(long long)i * LVB_MLP_IN + q];
                o[LVB_MLP_IN] = __fdiv_rn(__fsqrt_rn(m), __fmul_rn(2.0f, s.rad[i]));
            }
            s.lg_t[i] = -1;
        } else {
            s.lg_m[i] = m;
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
// out[0] = min radius bits, out[1] = bad input, out[2 + s] = max radius
// bits of scene s (positive floats order like their bit patterns)
__global__ void k_radius_scan(const float4 *__restrict__ pos, int n, const int *scene_of,
                              unsigned *out)
{
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        const float4 p = pos[i];
        const bool ok = isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w) &&
                        p.w > 0.0f;
        if (!ok) { atomicOr(&out[1], 1u); continue; }
        atomicMin(&out[0], __float_as_uint(p.w));
        atomicMax(&out[2 + (scene_of ? scene_of[i] : 0)], __float_as_uint(p.w));
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
    // cached graph of one step, for the last (pos, vel) pointers seen
    bool use_graph = true;
    int check_threads = kCheckMaxThreads;   // block size of the check kernel
    cudaGraphExec_t gexec = nullptr;
    const void *g_pos = nullptr, *g_vel = nullptr, *g_acc = nullptr;
    int version = 0;                // bumped whenever the step's graph changes
    HostFlags *hflags = nullptr;    // mapped pinned host memory
    long long grows = 0;            // store or cell-slot growths done
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
    void *ptrs[] = {s.ref, s.rad, s.cell_of, s.slot_of, s.prevcell, s.bits, s.fid, s.row_off,
                    s.row_len, s.row_cap, s.col, s.trow, s.trow_mark, s.cell_cnt, s.cell_id,
                    s.cell_ref, s.cnt, s.blk, c->ex_cnt, c->ex_off, c->ex_i, c->ex_j, c->ex_d,
                    c->scratch, c->sum64, c->sg_d, c->scene_of_d, s.born, s.cell_live,
                    s.lg_feat, s.lg_x, s.lg_t, s.lg_m, s.log_buf};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->cnt_h) cudaFreeHost(c->cnt_h);
    if (c->hflags) cudaFreeHost(c->hflags);
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

constexpr int kBigGrid = 4 * kNumSMs;   // grid of the partial passes above medium_max flagged
constexpr int kDefaultSmallMax = 32;
constexpr int kDefaultMediumMax = 2048;

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

// 1024 check threads per SM (the kernel's register budget), in blocks of
// check_threads; each thread takes kCheckUnroll particles per pass
int check_grid(lvb_ctx *c)
{
    return grid_for((c->n + kCheckUnroll - 1) / kCheckUnroll, c->check_threads,
                    kNumSMs * (kCheckMaxThreads / c->check_threads));
}
int medium_grid(lvb_ctx *c)
{
    return grid_for(std::min<long long>(c->s.medium_max, c->n), kThreads / 32, kNumSMs);
}

// One step as direct launches (used while the caller's stream is being
// captured, or when graphs are switched off): every kernel is launched and
// the ones with nothing to do return at once.
void launch_step_direct(lvb_ctx *c, const float4 *pos, const float4 *v4, const float4 *a4,
                        const IntegrateArgs &ia)
{
    const cudaStream_t st = c->stream;
    DevState s = c->s;
    s.use_cond = 0;
    if (ia.active)
        k_check<true><<<check_grid(c), c->check_threads, 0, st>>>(pos, v4, a4, s, ia);
    else
        k_check<false><<<check_grid(c), c->check_threads, 0, st>>>(pos, v4, a4, s, ia);
    const float4 *p = ia.active ? ia.pos : pos;
    if (c->trigger == LVB_TRIGGER_PARTIAL) {
        const int gm = medium_grid(c);
        k_inc_rows<<<gm, kThreads, 0, st>>>(s);
        k_inc_append<<<gm, kThreads, 0, st>>>(s);
    } else {
        const int gate = c->trigger == LVB_TRIGGER_GLOBAL ? GATE_ANY_FLAG : GATE_ALWAYS;
        const int gi = items_grid(c);
        k_full_update<<<gi, kThreads, 0, st>>>(p, v4, s, gate);
        k_cells_clear<<<grid_for(c->ncells, kThreads, 4 * kNumSMs), kThreads, 0, st>>>(s, gate);
        k_cells_insert<<<gi, kThreads, 0, st>>>(s, gate, 0);
        k_rows<<<rows_grid(c), kThreads, 0, st>>>(s, gate, 1);
    }
    launch_relayout(c);
    if (s.log_on) k_log_step<<<items_grid(c), kThreads, 0, st>>>(p, s);
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

// The re-layout body (count, scan, fill) appended to graph g after *dep.
cudaError_t add_relayout_nodes(lvb_ctx *c, cudaGraph_t g, cudaGraphNode_t *dep, const DevState &s)
{
    const ScanArgs a = layout_args(c);
    const int nb = (int)c->nblk;
    GK(add_kernel(dep, g, dep, k_rows, dim3(rows_grid(c)), dim3(kThreads), s, (int)GATE_OVERFLOW,
                  0));
    GK(add_kernel(dep, g, dep, k_scan_reduce, dim3(nb), dim3(kThreads), a, s, (int)GATE_OVERFLOW));
    GK(add_kernel(dep, g, dep, k_scan_top, dim3(1), dim3(kThreads), a, s, (int)GATE_OVERFLOW, nb));
    GK(add_kernel(dep, g, dep, k_scan_down, dim3(nb), dim3(kThreads), a, s, (int)GATE_OVERFLOW));
    GK(add_kernel(dep, g, dep, k_rows, dim3(rows_grid(c)), dim3(kThreads), s, (int)GATE_OVERFLOW,
                  1));
    GK(add_kernel(dep, g, dep, k_relayout_done, dim3(1), dim3(1), s));
    return cudaSuccess;
}

// Ends a rebuild body: a kernel arms an IF whose body is the re-layout.
cudaError_t add_relayout_if(lvb_ctx *c, cudaGraph_t body, cudaGraphNode_t *dep, const DevState &s)
{
    cudaGraphConditionalHandle h;
    GK(cudaGraphConditionalHandleCreate(&h, body, 0u, cudaGraphCondAssignDefault));
    GK(add_kernel(dep, body, dep, k_set_relayout, dim3(1), dim3(1), s, h));
    cudaGraph_t rl[1] = {nullptr};
    cudaGraphNode_t n = nullptr;
    cudaError_t err = cudaSuccess;
    add_cond(&n, body, *dep, h, cudaGraphCondTypeIf, 1, rl, &err);
    GK(err);
    cudaGraphNode_t b = nullptr;
    GK(add_relayout_nodes(c, rl[0], &b, s));
    *dep = n;
    return cudaSuccess;
}

// The step as graph nodes: k_check (which also updates the flagged
// particles and, when few are flagged, finishes the rebuild in its last
// block), then for the PARTIAL trigger a SWITCH whose bodies are the two
// grid-wide passes on a medium grid, the same on a big grid, and the
// re-layout alone (no body when the check did all the work); the two
// rebuild bodies end in an IF around the re-layout.  GLOBAL / ALWAYS use an
// IF around the full rebuild.  Conditions are set on the device.
cudaError_t build_step_nodes(lvb_ctx *c, cudaGraph_t g, cudaGraphNode_t *dep, const float4 *pos,
                             const float4 *v4, const float4 *a4, const IntegrateArgs &ia)
{
    DevState s = c->s;
    cudaGraphConditionalHandle hp;
    const bool partial = c->trigger == LVB_TRIGGER_PARTIAL;
    GK(cudaGraphConditionalHandleCreate(&hp, g, partial ? PATH_NONE : 0u,
                                        cudaGraphCondAssignDefault));
    s.h_path = hp;
    s.use_cond = 1;
    cudaGraphNode_t n = dep ? *dep : nullptr;
    GK(add_kernel(&n, g, &n, ia.active ? k_check<true> : k_check<false>, dim3(check_grid(c)),
                  dim3(c->check_threads), pos, v4, a4, s,
                  ia));
    const float4 *p = ia.active ? ia.pos : pos;
    cudaGraphNode_t cn = nullptr;
    cudaError_t err = cudaSuccess;
    if (partial) {
        cudaGraph_t b3[3] = {nullptr, nullptr, nullptr};
        add_cond(&cn, g, n, hp, cudaGraphCondTypeSwitch, 3, b3, &err);
        GK(err);
        const int grids[2] = {medium_grid(c), kBigGrid};
        for (int q = PATH_MEDIUM; q <= PATH_BIG; ++q) {
            cudaGraphNode_t b = nullptr;
            const dim3 gq(grids[q]);
            GK(add_kernel(&b, b3[q], &b, k_inc_rows, gq, dim3(kThreads), s));
            GK(add_kernel(&b, b3[q], &b, k_inc_append, gq, dim3(kThreads), s));
            GK(add_relayout_if(c, b3[q], &b, s));
        }
        cudaGraphNode_t b = nullptr;
        GK(add_relayout_nodes(c, b3[PATH_RELAYOUT], &b, s));
    } else {
        cudaGraph_t body[1] = {nullptr};
        add_cond(&cn, g, n, hp, cudaGraphCondTypeIf, 1, body, &err);
        GK(err);
        const int gate = c->trigger == LVB_TRIGGER_GLOBAL ? GATE_ANY_FLAG : GATE_ALWAYS;
        const int gi = items_grid(c);
        cudaGraphNode_t b = nullptr;
        GK(add_kernel(&b, body[0], &b, k_full_update, dim3(gi), dim3(kThreads), p, v4, s, gate));
        GK(add_kernel(&b, body[0], &b, k_cells_clear,
                      dim3(grid_for(c->ncells, kThreads, 4 * kNumSMs)), dim3(kThreads), s, gate));
        GK(add_kernel(&b, body[0], &b, k_cells_insert, dim3(gi), dim3(kThreads), s, gate, 0));
        GK(add_kernel(&b, body[0], &b, k_rows, dim3(rows_grid(c)), dim3(kThreads), s, gate, 1));
        GK(add_relayout_if(c, body[0], &b, s));
    }
    if (s.log_on) GK(add_kernel(&cn, g, &cn, k_log_step, dim3(items_grid(c)), dim3(kThreads), p, s));
    if (dep) *dep = cn;
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

// Grows the row store and/or the cell slots when a kernel asked for it
// (over 75% full), then rebuilds the cells and rows from the current
// reference state -- the list is a function of that state alone, so the
// rebuilt list is the one the steps would have produced.  Synchronises;
// runs only on the rare steps that need it.
int grow_if_asked(lvb_ctx *c)
{
    volatile HostFlags *h = c->hflags;
    if (!h->grow_store && !h->grow_cells) return LVB_OK;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return from_cuda(e);
    DevState &s = c->s;
    const cudaStream_t st = c->stream;
    const bool cells = h->grow_cells != 0;
    if (cells && s.ccap < (1 << 16)) {
        const int ccap = std::min(2 * s.ccap, 1 << 16);
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
    if (need * 4 > s.col_cap * 3) {
        const long long cap = std::min<long long>(2 * need + 8 * c->n + 1024, INT32_MAX);
        if (need > cap) return LVB_ENOMEM;
        cudaFree(s.col);
        s.col = nullptr;
        e = dalloc(&s.col, cap);
        if (e != cudaSuccess) return from_cuda(e);
        s.col_cap = cap;
    }
    k_rows<<<rows_grid(c), kThreads, 0, st>>>(s, GATE_ALWAYS, 1);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return from_cuda(e);
    h->grow_store = 0;
    h->grow_cells = 0;
    c->grows += 1;
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
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
    case LVB_ELIMIT: return "input exceeds the entry point's fixed maximum size";
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
        (!skin->mlp || !vel || !acc || trigger != LVB_TRIGGER_PARTIAL || !(skin->dt > 0.0f)))
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
    k_radius_scan<<<grid_for(n, kThreads, 4 * kNumSMs), kThreads, 0, st>>>(
        (const float4 *)pos_r, (int)n, c->scene_of_d, c->scratch);
    e = cudaMemcpyAsync(rs.data(), c->scratch, sizeof(unsigned) * rs.size(),
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(from_cuda(e));
    if (rs[1]) return fail(LVB_ENAN);
    float rmin;
    memcpy(&rmin, &rs[0], 4);

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
    if (e == cudaSuccess) e = dalloc(&s.prevcell, n);
    if (e == cudaSuccess) e = dalloc(&s.bits, c->nwords);
    if (e == cudaSuccess) e = dalloc(&s.fid, n);
    if (e == cudaSuccess) e = dalloc(&s.row_off, n);
    if (e == cudaSuccess) e = dalloc(&s.row_len, n);
    if (e == cudaSuccess) e = dalloc(&s.row_cap, n);
    if (e == cudaSuccess) e = dalloc(&s.trow, n);
    if (e == cudaSuccess) e = dalloc(&s.trow_mark, n);
    if (e == cudaSuccess) e = dalloc(&s.cell_cnt, ncells);
    if (e == cudaSuccess) e = dalloc(&s.cell_live, ncells);
    if (e == cudaSuccess) e = dalloc(&s.born, n);
    if (e == cudaSuccess) e = dalloc(&s.cnt, 1);
    if (e == cudaSuccess) e = dalloc(&s.blk, c->nblk + 1);
    if (e != cudaSuccess) return fail(from_cuda(e));
    cudaMemsetAsync(s.trow_mark, 0, sizeof(int) * n, st);
    cudaMemsetAsync(s.born, 0, sizeof(int) * n, st);
    cudaMemsetAsync(s.cell_live, 0, sizeof(int) * ncells, st);
    cudaMemsetAsync(s.cnt, 0, sizeof(DevCounters), st);
    cudaMemsetAsync(&s.cnt->tr_start, 0xff, sizeof(s.cnt->tr_start), st);
    cudaMemsetAsync(s.bits, 0, sizeof(uint32_t) * c->nwords, st);

    s.n = (int)n;
    s.small_max = kDefaultSmallMax;
    s.medium_max = (int)std::min<int64_t>(kDefaultMediumMax, n);
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
        const double vmean = 4.0 / 3.0 * M_PI * (double)rmin * rmin * rmin;
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
    const cudaStream_t st = c->stream;
    const float4 *pos = (const float4 *)pos_r;
    const float4 *v4 = (const float4 *)vel;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return from_cuda(e);
    if (!c->use_graph || cs != cudaStreamCaptureStatusNone) {
        launch_step_direct(c, pos, v4, a4, IntegrateArgs{});
        return from_cuda(cudaGetLastError());
    }
    if (!c->gexec || c->g_pos != pos_r || c->g_vel != vel || c->g_acc != acc) {
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        cudaGraph_t g = nullptr;
        e = cudaGraphCreate(&g, 0);
        if (e == cudaSuccess) e = build_step_nodes(c, g, nullptr, pos, v4, a4, IntegrateArgs{});
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gexec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->gexec = nullptr;
            return from_cuda(e);
        }
        c->g_pos = pos_r;
        c->g_vel = vel;
        c->g_acc = acc;
    }
    return from_cuda(cudaGraphLaunch(c->gexec, st));
}

int lvb_set_option(lvb_ctx *c, int32_t option, int64_t value)
{
    if (!c) return LVB_EINVAL;
    if (option == LVB_OPT_GRAPH) {
        c->use_graph = value != 0;
    } else if (option == LVB_OPT_SMALL_MAX) {
        if (value < 0) return LVB_EINVAL;
        c->s.small_max = (int)std::min<int64_t>(value, kFusedMax);
        c->s.medium_max = std::max(c->s.medium_max, c->s.small_max);
    } else if (option == LVB_OPT_TRACE) {
        c->s.trace = value != 0;
    } else if (option == LVB_OPT_MEDIUM_MAX) {
        if (value < 0) return LVB_EINVAL;
        c->s.medium_max = (int)std::max<int64_t>(std::min<int64_t>(value, c->n),
                                                 c->s.small_max);
    } else if (option == LVB_OPT_CHECK_THREADS) {
        if (value != 256 && value != 512 && value != 1024) return LVB_EINVAL;
        c->check_threads = (int)value;
    } else {
        return LVB_EINVAL;
    }
    if (c->gexec) {   // rebuilt with the new setting on the next step
        cudaStreamSynchronize(c->stream);
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
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
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
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
    o->grows = c->grows;
    o->cell_capacity = c->ccap;
    o->row_store_capacity = c->s.col_cap;
    o->kernels_executed = (int64_t)h.kernels;
    for (int k = 0; k < 4; ++k) o->fused_phase_cycles[k] = (int64_t)h.fused_cycles[k];
    o->small_path_steps = h.small_steps;
    o->small_max = c->s.small_max;
    o->medium_max = c->s.medium_max;
    o->graphs = c->use_graph ? 1 : 0;
    o->n_scenes = c->nscenes;
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
    v.cnt = c->s.cnt;
    v.trace = &c->s.trace;
    v.sg = c->sg_d;
    v.scene_of = c->scene_of_d;
    v.nscenes = c->nscenes;
    v.n = (int)c->n;
    return v;
}

int append_step_nodes(lvb_ctx *c, cudaGraph_t g, cudaGraphNode_t *dep, const float *pos_r,
                      const float *vel, const float *acc, const IntegrateArgs *integ)
{
    return from_cuda(build_step_nodes(c, g, dep, (const float4 *)pos_r, (const float4 *)vel,
                                      (const float4 *)acc, integ ? *integ : IntegrateArgs{}));
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
