// lvb_step.cuh -- device state of a broad-phase context and the step kernel.
//
// One step of the local Verlet buffer is one cooperative kernel, k_step,
// whose phases are separated by grid-wide barriers (all its blocks are
// co-resident: cooperative launch, grid sized by occupancy):
//   check      every particle: displacement check (Eq. update), ballot
//              words, compaction of the flagged ids; with the PARTIAL
//              trigger the warp that flags a particle also computes its new
//              reference state and skin (Eq. skin_formulus1 or another
//              policy, capped per Eq. skin_formulus_mincell)
//   -- barrier --
//   rebuild    PARTIAL: each flagged particle moves to its new cell slot,
//              gets its new row by the 27-cell stencil (Algorithm 1 on the
//              extended spheres, Eq. bounding_sphere) plus a direct test
//              against the other flagged particles of its scene, and
//              patches the rows of its unflagged partners in place (removed
//              pairs become -1, new pairs take a -1 slot or the row's end)
//              -- one phase, no barrier (many flagged particles: moves
//              first, then a barrier)
//              GLOBAL / ALWAYS (Def. autoverlet / no buffer): new reference
//              states, cells and rows of every particle
//   -- barrier --
//   re-layout  only if a row overflowed in the rebuild
//   tail       the DEM driver's forces (k_step instantiated by lvb_dem.cu)
// A step with nothing flagged is the check and one barrier.  The kernel is
// included by lvb_broad.cu (the broad phase alone) and lvb_dem.cu (a whole
// DEM step per launch).
#pragma once

#include "lvb_internal.cuh"

namespace lvb {

constexpr int kStepMaxThreads = 1024;     // block size limit of k_step (one block per SM)
constexpr int kCheckUnroll = 2;           // 32-particle chunks a warp has in flight
constexpr int kFlaggedDirectMax = 4096;   // default of DevState::direct_max
constexpr int kDirectUnroll = 4;          // flagged reference states per lane in flight
constexpr unsigned kBarrierSpins = 1u << 22;   // ~1-3 s of polling (L2 round trips) before a barrier gives up

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
    uint32_t *bits;
    int *fid;         // flagged ids of the step, in compaction order
    float4 *fref;     // their new (xref, R_NL), same order
    float4 *oref;     // their old (xref, R_NL), same order
    // many scenes: the flagged particles of scene q also sit in its own
    // segment [first_q, first_q + sc_cnt[par][q]) of sfid / sfref, so the
    // direct flagged test scans only its scene (null with one scene)
    int *sc_cnt;      // 2 x nscenes counters (by step parity)
    int *sfid;
    float4 *sfref;
    int *fsc;         // scene of each flagged particle, same order as fid
                      // (saves the rebuild a dependent load; null with one scene)
    // rows: row i is col[row_off[i], row_off[i] + row_cap[i]); entries below
    // row_len[i] are partners or -1 (a removed pair), entries at or above
    // it are -1; row_len[i] > row_cap[i] means the row overflowed
    int *row_off, *row_len, *row_cap, *col;
    long long col_cap;
    int *cell_cnt, *cell_id;
    float4 *cell_ref;
    DevCounters *cnt;
    long long *blk;   // scan partials (one per block of the widest scan)
    const lvb_mlp_weights *mlp;   // skin network (LVB_SKIN_LEARNED)
    int *born;        // step of each particle's last update
    int *cell_live;   // particles whose reference position lies in each cell
    int *cell_rmax;   // per cell, an upper bound on the R_NL of its particles
                      // (binary32 bits; raised by every insert, reset only
                      // when the cells are rebuilt)
    // rebuild log (training samples of the skin network)
    int log_on, log_horizon;
    long long log_cap;
    float *lg_feat;   // n x 8 features of the open record
    float4 *lg_x;     // position at which the record opened
    int *lg_t;        // step the record opened (-1: none)
    float *lg_m;      // largest squared displacement since
    float *log_buf;   // log_cap x 9 samples
    HostFlags *hflags;    // device view of the mapped host flags
    int trace;            // record per-phase device time (LVB_OPT_TRACE)
    int compact_block;    // flag compaction: 0 one atomic per warp chunk,
                          // 1 one per block tile (LVB_OPT_COMPACT)
    unsigned bar_extra;   // arrivals a barrier waits for beyond the grid's
                          // blocks: 0, or 1 to make every wait run out (the
                          // failure test, LVB_OPT_BARRIER_EXTRA)
    unsigned bar_spins;   // polls before a barrier gives up
    int direct_max;       // largest flagged count rebuilt in one phase with
                          // the direct flagged-pair test (LVB_OPT_DIRECT_MAX)
    int check_regs;       // check pass of the broad phase alone: 1 register loads,
                          // 0 the bulk-copy ring (LVB_OPT_CHECK_LOADS)
    int reach;            // stencil cells skipped by distance (LVB_OPT_STENCIL_REACH):
                          // 0 none, 1 by the cap H, 2 by H and the cell's own bound
    // second destination of this step's flag words and flagged count
    // (lvb_step_host: a staging slot copied out while the next step runs),
    // or null
    uint32_t *bits_out;
    int *nf_out;
    // the particles updated at this step, one bit each: the flag words
    // (bits) unless the early trigger is on (LVB_OPT_EARLY), which adds
    // particles past beta * skin on steps with a flag; the rebuild reads this
    uint32_t *ubits;
    float early_beta;     // 1: off; < 1: the early trigger's fraction of the skin
    // contact history (LVB_OPT_HISTORY): one record per row entry, hist[e]
    // beside col[e], kept with its entry through partial rebuilds,
    // re-layouts and store growth; null when off
    float4 *hist;
    float4 *pold;     // per particle: the old (xref, R_NL) of a particle
                      // updated at this step (written by its update)
    // the rows as they were before a re-layout, for carrying history
    int *old_off, *old_len, *old_col;
    float4 *old_hist;
};

// gate modes of the separate full-build kernels (init, store growth)
enum Gate { GATE_OVERFLOW = 1, GATE_ANY_FLAG = 2, GATE_ALWAYS = 3 };

__device__ __forceinline__ const SceneGeom &geom_of(const DevState &s, int i)
{
    return s.sg[s.nscenes == 1 ? 0 : s.scene_of[i]];
}

// geometry and scene of flagged list entry k (particle fid[k])
__device__ __forceinline__ int flagged_scene(const DevState &s, int k)
{
    return s.nscenes == 1 ? 0 : s.fsc[k];
}

__device__ __forceinline__ bool store_failed(const DevState &s)
{
    return (s.cnt->err & DERR_STORE) != 0;
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

// per-kernel trace of the separate kernels: first entry and last exit over
// the kernel's blocks (folded into the sums by the next step)
__device__ __forceinline__ void tr_enter(const DevState &s, int slot)
{
    if (s.trace && threadIdx.x == 0) atomicMin(&s.cnt->tr_start[slot], global_ns());
}

__device__ __forceinline__ void tr_exit(const DevState &s, int slot)
{
    if (s.trace && (threadIdx.x & 31) == 0) atomicMax(&s.cnt->tr_end[slot], global_ns());
}

// ---------------------------------------------------------------------------
// Phases that walk a row or a cell run one warp per item (w0/wstride count
// warps): the lanes take the entries, so a phase costs a few memory
// latencies however long the rows are, and atomics are warp-aggregated.
// ---------------------------------------------------------------------------

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
        prop = mlp_skin(s.mlp, y, __fmul_rn(2.0f, r), f[0]);
    }
    return skin_of(s.skin_kind, s.skin_value, s.skin_dt, g.H, r, v, prop);
}


// The network's weights in shared memory for the step: copied
// asynchronously (16-byte cp.async pieces) when the kernel starts, so the
// copy runs under the check pass; the issuing threads wait for their pieces
// before the first grid barrier, whose block barrier then publishes them.
static_assert(sizeof(lvb_mlp_weights) % 16 == 0, "weights are copied in 16-byte pieces");

__device__ __forceinline__ void weights_copy_async(lvb_mlp_weights *dst,
                                                   const lvb_mlp_weights *src)
{
    const char *g = reinterpret_cast<const char *>(src);
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    for (int t = threadIdx.x; t < (int)(sizeof(lvb_mlp_weights) / 16); t += blockDim.x)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + 16u * t),
                     "l"(g + 16 * t)
                     : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void weights_copy_wait()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Live partners of row i (entries >= 0), counted by one lane: eight
// entries loaded at a time, so a short row costs one memory latency.
__device__ __forceinline__ int row_live_lane(const DevState &s, int i)
{
    const int off = s.row_off[i], len = min(s.row_len[i], s.row_cap[i]);
    int c = 0;
    for (int e = 0; e < len; e += 8) {
        int v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = e + u < len ? s.col[off + e + u] : -1;
#pragma unroll
        for (int u = 0; u < 8; ++u) c += v[u] >= 0;
    }
    return c;
}

// a2 for the m <= 32 flagged particles at list indices k0 .. k0 + m - 1,
// after the check pass (PARTIAL trigger, deferred_update): lane t takes
// particle fid[k0 + t] -- its loads and features (from the state before
// the update: rows and cells change only in the rebuild that follows;
// `step` is the number of the step being taken) in flight with the other
// lanes' -- and the warp evaluates the network for the m particles one
// after another; each lane then writes its particle's new reference
// position and skin, kept with the old state at its list index.  (pos and
// vel may have been written earlier in the same kernel by the DEM position
// half-step, so they are read through plain coherent loads.)
__device__ __forceinline__ void update_group(const DevState &s, const lvb_mlp_weights *W, int k0,
                                             int m, const float4 *pos, const float4 *vel,
                                             const float4 *acc, int step)
{
    const int lane = threadIdx.x & 31;
    const bool act = lane < m;
    const int i = act ? s.fid[k0 + lane] : 0;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    float f[LVB_MLP_IN];
#pragma unroll
    for (int t = 0; t < LVB_MLP_IN; ++t) f[t] = 0.0f;
    if (act && (s.skin_kind == LVB_SKIN_LEARNED || s.log_on)) {
        const float4 p = pos[i];
        const SceneGeom &g = geom_of(s, i);
        const int nc = cell_key(g, p.x, p.y, p.z);
        skin_features(s, p, vel ? vel[i] : zero, acc ? acc[i] : zero, s.rad[i], g, s.ref[i],
                      row_live_lane(s, i), step - s.born[i], s.cell_live[nc], f);
    }
    float y = 0.0f;
    if (s.skin_kind == LVB_SKIN_LEARNED) {
        for (int t = 0; t < m; ++t) {
            float ft[LVB_MLP_IN];
#pragma unroll
            for (int k = 0; k < LVB_MLP_IN; ++k) ft[k] = __shfl_sync(FULL, f[k], t);
            const float yt = mlp_y_warp(W, ft);
            if (lane == t) y = yt;
        }
    }
    if (!act) return;
    // the particle's state again (cached): fewer registers held across the
    // network's evaluation
    const int k = k0 + lane;
    const float4 p = pos[i];
    const float r = s.rad[i];
    const float4 v = vel ? vel[i] : zero;
    const float4 q = s.ref[i];
    const SceneGeom &g = geom_of(s, i);
    const float prop =
        s.skin_kind == LVB_SKIN_LEARNED ? mlp_skin(W, y, __fmul_rn(2.0f, r), f[0]) : 0.0f;
    const float sk = skin_of(s.skin_kind, s.skin_value, s.skin_dt, g.H, r, v, prop);
    const float4 qn = make_float4(p.x, p.y, p.z, __fadd_rn(r, sk));
    s.ref[i] = make_float4(p.x, p.y, p.z, sk);
    s.born[i] = step;
    s.fref[k] = qn;
    s.oref[k] = make_float4(q.x, q.y, q.z, __fadd_rn(r, q.w));
    if (s.pold) s.pold[i] = s.oref[k];
    if (s.sc_cnt) {
        const int sc = s.scene_of[i];
        s.fsc[k] = sc;
        const int slot = g.first + atomicAdd(&s.sc_cnt[(step & 1) * s.nscenes + sc], 1);
        s.sfid[slot] = i;
        s.sfref[slot] = qn;
    }
    if (s.log_on && s.lg_t[i] < 0) {
        s.lg_t[i] = step;
        s.lg_x[i] = p;
        s.lg_m[i] = 0.0f;
#pragma unroll
        for (int t = 0; t < LVB_MLP_IN; ++t) s.lg_feat[(long long)i * LVB_MLP_IN + t] = f[t];
    }
}

// a2 for up to 32 flagged particles at once, one per lane (lane t takes
// particle id[t], list index k0 + t, t < m), inside the check pass: the same
// update as update_group for the policies that need neither the network
// nor the rebuild log.
static __device__ __noinline__ void update_lanes(const DevState &s, const int *id, int k0, int m,
                                                 const float4 *pos, const float4 *vel, int step)
{
    const int lane = threadIdx.x & 31;
    if (lane >= m) return;
    const int i = id[lane], k = k0 + lane;
    const float4 p = pos[i];
    const float r = s.rad[i];
    const float4 v = vel ? vel[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 q = s.ref[i];
    const SceneGeom &g = geom_of(s, i);
    const float sk = skin_of(s.skin_kind, s.skin_value, s.skin_dt, g.H, r, v, 0.0f);
    const float4 qn = make_float4(p.x, p.y, p.z, __fadd_rn(r, sk));
    s.ref[i] = make_float4(p.x, p.y, p.z, sk);
    s.born[i] = step;
    s.fref[k] = qn;
    const float4 qo = make_float4(q.x, q.y, q.z, __fadd_rn(r, q.w));
    s.oref[k] = qo;
    if (s.pold) s.pold[i] = qo;
    if (s.sc_cnt) {
        const int sc = s.scene_of[i];
        s.fsc[k] = sc;
        const int slot = g.first + atomicAdd(&s.sc_cnt[(step & 1) * s.nscenes + sc], 1);
        s.sfid[slot] = i;
        s.sfref[slot] = qn;
    }
}

// a3 for flagged particle i (warp), qn its new (xref, R_NL): a stayer
// refreshes its slot's copy of the reference state; a leaver leaves a
// tombstone (-1) in its old slot and takes a tombstone slot of its new cell
// (compare-and-swap) or a fresh one at the end; the cells' live counts
// follow, and the new cell's R_NL bound is raised to qn.w if below.  Slots
// of unflagged particles never change.
__device__ __forceinline__ void move_warp(const DevState &s, int i, float4 qn, int sc)
{
    const int lane = threadIdx.x & 31;
    const int ccap = s.ccap;
    const SceneGeom &g = s.sg[sc];
    const int nc = cell_key(g, qn.x, qn.y, qn.z);
    const int oc = s.cell_of[i], so = s.slot_of[i];
    if (lane == 0) atomicMax(&s.cell_rmax[nc], __float_as_int(qn.w));
    if (nc == oc) {
        if (lane == 0) s.cell_ref[(long long)oc * ccap + so] = qn;
        return;
    }
    if (lane == 0) {
        s.cell_id[(long long)oc * ccap + so] = -1;
        atomicSub(&s.cell_live[oc], 1);
        atomicAdd(&s.cell_live[nc], 1);
    }
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
        // a fresh slot at the end, also claimed by compare-and-swap: once
        // the count covers it, another mover's tombstone search may see it
        // still holding -1 and take it first; then the next one is taken
        for (int t = 0; slot < 0 && t <= ccap; ++t) {
            const int sl = atomicAdd(&s.cell_cnt[nc], 1);
            if (sl * 4 >= ccap * 3) s.hflags->grow_cells = 1;
            if (sl >= ccap) {
                atomicOr(&s.cnt->err, DERR_CELL);
                break;
            }
            if (atomicCAS(&s.cell_id[base + sl], -1, i) == -1) slot = sl;
        }
        if (slot >= 0) {
            s.cell_ref[base + slot] = qn;
            s.slot_of[i] = slot;
        }
        s.cell_of[i] = nc;
    }
    __syncwarp();
}

// Squared distance from a particle's reference position q to the box of
// stencil cell (x, y, z) of scene g.  A partner j lies within R_NL,i +
// R_NL,j of it, and R_NL,j is at most H (the cap of Eq.
// skin_formulus_mincell) and at most the cell's own bound cell_rmax, so a
// cell whose box is farther away than R_NL,i plus either bound holds no
// partner (within_reach).  The box is widened by L/1024 on every side --
// far more than the rounding of the binned coordinates -- and open outward
// at the grid's border (where particles outside the box are binned), and
// the reach is rounded up: a cell with a partner is never skipped.  With
// polydisperse radii most of the 27 cells are out of reach of a small
// particle.
__device__ __forceinline__ float cell_dist2(const SceneGeom &g, int x, int y, int z, float4 q)
{
    const float slack = g.L * (1.0f / 1024.0f);
    const int c[3] = {x, y, z};
    const float p[3] = {q.x, q.y, q.z};
    float d2 = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lo = g.lo[k] + (float)c[k] * g.L - slack;
        const float hi = g.lo[k] + (float)(c[k] + 1) * g.L + slack;
        float d = 0.0f;
        if (c[k] > 0 && p[k] < lo) d = lo - p[k];
        if (c[k] < g.dim[k] - 1 && p[k] > hi) d = p[k] - hi;
        d2 += d * d;
    }
    return d2;
}

// d2 from cell_dist2 against R_NL,i (q.w) plus a bound on the partners'
// R_NL (H, or the cell's own bound), with the reach rounded up
__device__ __forceinline__ bool within_reach(const SceneGeom &g, float d2, float q_w, float r_bound)
{
    const float reach = (q_w + r_bound) * 1.001f + g.L * (1.0f / 1024.0f);
    return d2 <= reach * reach;
}

// Removes partner i from unflagged row j (one lane): its entry becomes -1.
// Rows are short; four entries are loaded at a time.
__device__ __forceinline__ void lane_remove(const DevState &s, int j, int i)
{
    const int off = s.row_off[j], len = min(s.row_len[j], s.row_cap[j]);
    for (int e = 0; e < len; e += 4) {
        int v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = e + u < len ? s.col[off + e + u] : -2;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (v[u] == i) {
                s.col[off + e + u] = -1;
                return;
            }
    }
}

// Adds partner i to unflagged row j (one lane): a -1 entry below row_len,
// claimed with compare-and-swap, else the next slot at the end (also by
// compare-and-swap: a slot past row_len holds -1 and another warp's search
// may claim it first).  A full row raises *ovf (the re-layout rebuilds it).
__device__ __forceinline__ void lane_insert(const DevState &s, int j, int i, int *ovf)
{
    const int off = s.row_off[j], cap = s.row_cap[j], len = min(s.row_len[j], cap);
    for (int e = 0; e < len; e += 4) {
        int v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = e + u < len ? s.col[off + e + u] : 0;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (v[u] < 0 && atomicCAS(&s.col[off + e + u], -1, i) == -1) {
                if (s.hist) s.hist[off + e + u] = make_float4(0.f, 0.f, 0.f, 0.f);
                return;
            }
    }
    for (int t = 0; t <= cap; ++t) {
        const int p = atomicAdd(&s.row_len[j], 1);
        if (p >= cap) {
            atomicExch(ovf, 1);
            return;
        }
        if (atomicCAS(&s.col[off + p], -1, i) == -1) {
            if (s.hist) s.hist[off + p] = make_float4(0.f, 0.f, 0.f, 0.f);
            return;
        }
    }
}

// One removal (partner i leaves row jr) and one insertion (partner i joins
// row ji) by one lane, their loads interleaved so that both edits take the
// latency of one: the two rows' bounds together, then four entries of each
// at a time.  jr or ji < 0: no such edit.  Same rules as lane_remove and
// lane_insert (the two rows differ: a removed pair is not a new one).
__device__ __forceinline__ void lane_edit(const DevState &s, int jr, int ji, int i, int *ovf)
{
    int offr = 0, lenr = 0, offi = 0, capi = 0, leni = 0;
    if (jr >= 0) {
        offr = s.row_off[jr];
        lenr = min(s.row_len[jr], s.row_cap[jr]);
    }
    if (ji >= 0) {
        offi = s.row_off[ji];
        capi = s.row_cap[ji];
        leni = min(s.row_len[ji], capi);
    }
    bool dr = jr < 0 || lenr == 0, di = ji < 0;
    for (int e = 0; !dr || (!di && e < leni); e += 4) {
        int vr[4], vi[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            vr[u] = !dr && e + u < lenr ? s.col[offr + e + u] : -2;
            vi[u] = !di && e + u < leni ? s.col[offi + e + u] : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (!dr && vr[u] == i) {
                s.col[offr + e + u] = -1;
                dr = true;
            }
            if (!di && vi[u] < 0 && atomicCAS(&s.col[offi + e + u], -1, i) == -1) {
                di = true;
                if (s.hist) s.hist[offi + e + u] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        if (e + 4 >= lenr) dr = true;
    }
    if (di) return;
    for (int t = 0; t <= capi; ++t) {
        const int p = atomicAdd(&s.row_len[ji], 1);
        if (p >= capi) {
            atomicExch(ovf, 1);
            return;
        }
        if (atomicCAS(&s.col[offi + p], -1, i) == -1) {
            if (s.hist) s.hist[offi + p] = make_float4(0.f, 0.f, 0.f, 0.f);
            return;
        }
    }
}

// a4 + a5 for flagged particle k of the list (warp), i = fid[k]:
//   1. each old partner j that is unflagged and no longer a pair (test on
//      i's new reference state) loses i from its row;
//   2. the new row of i: the 27-cell stencil around its new cell over the
//      cells' reference states.  direct: the moves of the flagged particles
//      run at the same time, so flagged particles found in the cells are
//      skipped and the flagged partners come from a direct test against the
//      flagged list; otherwise the cells are final and hold everyone;
//   3. each new partner j that is unflagged and was not a pair before (test
//      on i's old reference state) gets i in its row.
// A pair is a function of the two reference states (Def. verletlist) and an
// unflagged particle's state does not change, so these tests decide exactly
// which entries of the unflagged rows change; no other warp touches row i.
// The edits of other rows run one per lane, in parallel; the first 32 old
// partners and the first 32 stencil candidates are loaded together.
static __device__ __noinline__ void patch_warp(const DevState &s, int k, int nF, bool direct,
                                               int par, int *ovf, unsigned (&work)[3])
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const int ccap = s.ccap;
    const int i = s.fid[k];
    const float4 qn = s.fref[k], qo = s.oref[k];
    const int sc = flagged_scene(s, k);
    const int off = s.row_off[i], cap = s.row_cap[i], len0 = min(s.row_len[i], cap);
    const SceneGeom &g = s.sg[sc];
    // the direct test's count, loaded now (its latency under the stencil's)
    const bool own = s.sc_cnt != nullptr;
    const int m_dir = !direct ? 0 : own ? s.sc_cnt[par * s.nscenes + sc] : nF;
    const int d0 = g.dim[0], d1 = g.dim[1], d2 = g.dim[2];
    const int ci = cell_key(g, qn.x, qn.y, qn.z) - g.cell_base;
    const int cx = ci % d0, cy = (ci / d0) % d1, cz = ci / (d0 * d1);
    int cnt_l = 0, cid = 0;
    if (lane < 27) {
        const int x = cx + lane % 3 - 1, y = cy + (lane / 3) % 3 - 1, z = cz + lane / 9 - 1;
        if (x >= 0 && x < d0 && y >= 0 && y < d1 && z >= 0 && z < d2) {
            const float dd = s.reach ? cell_dist2(g, x, y, z, qn) : 0.0f;
            if (s.reach == 0 || within_reach(g, dd, qn.w, g.H)) {
                cid = g.cell_base + (z * d1 + y) * d0 + x;
                cnt_l = s.cell_cnt[cid];
                if (s.reach == 2 && !within_reach(g, dd, qn.w, __int_as_float(s.cell_rmax[cid])))
                    cnt_l = 0;
            }
        }
    }
    const int jo0 = lane < len0 ? s.col[off + lane] : -1;
    cnt_l = min(cnt_l, ccap);
    const int incl = warp_incl_scan(cnt_l);
    const int excl = incl - cnt_l;
    const int total = __shfl_sync(FULL, incl, 31);
    // candidate kk of the stencil: its cell by a 5-step shuffle search
    auto cand_idx = [&](int kk) {
        int c = 0;
#pragma unroll
        for (int st = 16; st >= 1; st >>= 1)
            c += (__shfl_sync(FULL, incl, c + st - 1) <= kk) ? st : 0;
        const int cc = __shfl_sync(FULL, cid, c);
        const int ex = __shfl_sync(FULL, excl, c);
        return (long long)cc * ccap + (kk - ex);
    };
    const long long idx0 = cand_idx(lane);
    const int jc0 = lane < total ? s.cell_id[idx0] : -1;
    const float4 rc0 = lane < total ? s.cell_ref[idx0] : make_float4(0.f, 0.f, 0.f, 0.f);
    // 1. removals.  An old row of up to 32 entries is held in registers
    // (jo0), so the new row may overwrite it at once: the removals of that
    // row are only decided here and made together with the first batch of
    // insertions (lane_edit); a longer row is done first, entry by entry.
    int jr0 = -1;
    for (int e0 = 0; e0 < len0; e0 += 32) {
        const int e = e0 + lane;
        const int j = e0 == 0 ? jo0 : (e < len0 ? s.col[off + e] : -1);
        bool rm = false;
        if (e < len0 && j >= 0) {
            // the partner's flag word, reference state and radius are
            // loaded together (one memory latency; none of them changes
            // during the rebuild), and only an unflagged partner's pair is
            // tested
            const uint32_t fw = s.ubits[j >> 5];
            const float4 rj = s.ref[j];
            const float rr = s.rad[j];
            if (!((fw >> (j & 31)) & 1u))
                rm = !pair_hit(qn, make_float4(rj.x, rj.y, rj.z, __fadd_rn(rr, rj.w)));
        }
        if (len0 <= 32) jr0 = rm ? j : -1;
        else if (rm) lane_remove(s, j, i);
        work[2] += __popc(__ballot_sync(FULL, rm));
    }
    work[0] += total;
    // 2. stencil (+ direct test) and 3. insertions
    int found = 0;
    if (total == 0 && jr0 >= 0) lane_remove(s, jr0, i);
    for (int b0 = 0; b0 < total; b0 += 32) {
        const int kk = b0 + lane;
        int j = -1;
        float4 rj = make_float4(0.f, 0.f, 0.f, 0.f);
        if (b0 == 0) {
            j = jc0;
            rj = rc0;
        } else {
            const long long idx = cand_idx(kk);
            if (kk < total) {
                j = s.cell_id[idx];
                rj = s.cell_ref[idx];
            }
        }
        bool hit = false, ins = false;
        if (kk < total && j >= 0 && j != i) {
            const bool fj = bit_of(s.ubits, j);
            if (!(direct && fj)) {
                hit = pair_hit(qn, rj);
                ins = hit && !fj && !pair_hit(qo, rj);
            }
        }
        const unsigned m = __ballot_sync(FULL, hit);
        if (hit) {
            const int p = found + __popc(m & lt);
            if (p < cap) s.col[off + p] = j;
        }
        found += __popc(m);
        work[2] += __popc(__ballot_sync(FULL, ins));
        if (b0 == 0) {
            lane_edit(s, jr0, ins ? j : -1, i, ovf);
        } else if (ins) {
            lane_insert(s, j, i, ovf);
        }
    }
    if (direct) {
        // kDirectUnroll reference states and ids per lane in flight (one
        // memory latency a batch).  Many scenes: the scene's own segment of
        // the flagged particles (scenes share one coordinate frame, so the
        // global list would also hold far-away twins)
        const float4 *lst = own ? s.sfref + g.first : s.fref;
        const int *ids = own ? s.sfid + g.first : s.fid;
        const int m = m_dir;
        work[1] += m;
        for (int b0 = 0; b0 < m; b0 += 32 * kDirectUnroll) {
            float4 rf[kDirectUnroll];
            int jf[kDirectUnroll];
#pragma unroll
            for (int u = 0; u < kDirectUnroll; ++u) {
                const int kk = b0 + u * 32 + lane;
                rf[u] = kk < m ? lst[kk] : make_float4(0.f, 0.f, 0.f, 0.f);
                jf[u] = kk < m ? ids[kk] : -1;
            }
#pragma unroll
            for (int u = 0; u < kDirectUnroll; ++u) {
                const int kk = b0 + u * 32 + lane;
                int j = -1;
                if (kk < m && pair_hit(qn, rf[u])) {
                    j = jf[u];
                    if (j == i || j < g.first || j >= g.first + g.count) j = -1;
                }
                const unsigned msk = __ballot_sync(FULL, j >= 0);
                if (j >= 0) {
                    const int p = found + __popc(msk & lt);
                    if (p < cap) s.col[off + p] = j;
                }
                found += __popc(msk);
            }
        }
    }
    for (int e = found + lane; e < len0; e += 32) s.col[off + e] = -1;
    if (lane == 0) {
        s.row_len[i] = found;
        if (found > cap) atomicExch(ovf, 1);
    }
}

// The reference record (xref, R_NL) of particle j as it was before this
// step's updates: its old record if it was updated at this step (history
// mode keeps it in pold), else its present one.
__device__ __forceinline__ float4 old_record(const DevState &s, int j)
{
    if (bit_of(s.ubits, j)) return s.pold[j];
    const float4 r = s.ref[j];
    return make_float4(r.x, r.y, r.z, __fadd_rn(s.rad[j], r.w));
}

// Appends the partners j of the lanes with `ins` to row i, which only this
// warp edits: first into the row's free slots among its first 32 entries
// (bits of *freemask), then at its end (*tail); each new entry's history
// starts at zero.  An entry past the row's capacity is dropped and the
// row's length records the overflow (the re-layout rebuilds the row).
__device__ __forceinline__ void own_row_insert(const DevState &s, int off, int cap, bool ins,
                                               int j, unsigned *freemask, int *tail)
{
    const unsigned m = __ballot_sync(FULL, ins);
    if (!m) return;
    const int cnt = __popc(m), nfree = __popc(*freemask);
    const int rank = __popc(m & lanemask_lt());
    if (ins) {
        const int slot = rank < nfree ? (int)__fns(*freemask, 0, rank + 1) : *tail + rank - nfree;
        if (slot < cap) {
            s.col[off + slot] = j;
            s.hist[off + slot] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    const int used = min(cnt, nfree);
    for (int t = 0; t < used; ++t) *freemask &= *freemask - 1;   // lowest bits taken
    *tail += cnt - used;
}

// a4 + a5 for flagged particle k with contact history (LVB_OPT_HISTORY):
// the same pair decisions as patch_warp, but row i is edited in place, as
// the unflagged rows are, so that a partner that stays a pair keeps its
// slot -- and its history -- through the rebuild:
//   1. each old entry j no longer a pair under the new reference states of
//      i and j (this step's updates are all written) becomes -1, and i
//      leaves row j if j is unflagged (a flagged j edits its own row);
//   2. each partner found by the stencil (+ the direct flagged test) that
//      is a pair now and was not one under the old states (the old record
//      of a flagged partner is kept in pold) joins row i with zero
//      history, and an unflagged partner gets i in its row.
static __device__ __noinline__ void patch_warp_hist(const DevState &s, int k, int nF, bool direct,
                                                    int par, int *ovf, unsigned (&work)[3])
{
    const int lane = threadIdx.x & 31;
    const int ccap = s.ccap;
    const int i = s.fid[k];
    const float4 qn = s.fref[k], qo = s.oref[k];
    const int sc = flagged_scene(s, k);
    const int off = s.row_off[i], cap = s.row_cap[i], len0 = min(s.row_len[i], cap);
    const SceneGeom &g = s.sg[sc];
    const int d0 = g.dim[0], d1 = g.dim[1], d2 = g.dim[2];
    const int ci = cell_key(g, qn.x, qn.y, qn.z) - g.cell_base;
    const int cx = ci % d0, cy = (ci / d0) % d1, cz = ci / (d0 * d1);
    int cnt_l = 0, cid = 0;
    if (lane < 27) {
        const int x = cx + lane % 3 - 1, y = cy + (lane / 3) % 3 - 1, z = cz + lane / 9 - 1;
        if (x >= 0 && x < d0 && y >= 0 && y < d1 && z >= 0 && z < d2) {
            const float dd = s.reach ? cell_dist2(g, x, y, z, qn) : 0.0f;
            if (s.reach == 0 || within_reach(g, dd, qn.w, g.H)) {
                cid = g.cell_base + (z * d1 + y) * d0 + x;
                cnt_l = s.cell_cnt[cid];
                if (s.reach == 2 && !within_reach(g, dd, qn.w, __int_as_float(s.cell_rmax[cid])))
                    cnt_l = 0;
            }
        }
    }
    cnt_l = min(cnt_l, ccap);
    const int incl = warp_incl_scan(cnt_l);
    const int excl = incl - cnt_l;
    const int total = __shfl_sync(FULL, incl, 31);
    work[0] += total;
    // 1. old entries
    unsigned freemask = 0u;
    for (int e0 = 0; e0 < len0; e0 += 32) {
        const int e = e0 + lane;
        const int j = e < len0 ? s.col[off + e] : -2;
        bool rm = false;
        if (j >= 0) {
            const float4 rj = s.ref[j];
            rm = !pair_hit(qn, make_float4(rj.x, rj.y, rj.z, __fadd_rn(s.rad[j], rj.w)));
            if (rm) {
                s.col[off + e] = -1;
                if (!bit_of(s.ubits, j)) lane_remove(s, j, i);
            }
        }
        const unsigned fm = __ballot_sync(FULL, e < len0 && (j == -1 || rm));
        if (e0 == 0) freemask = fm;
        work[2] += __popc(__ballot_sync(FULL, rm));
    }
    int tail = len0;
    // 2. stencil
    for (int b0 = 0; b0 < total; b0 += 32) {
        const int kk = b0 + lane;
        int c = 0;
#pragma unroll
        for (int st = 16; st >= 1; st >>= 1)
            c += (__shfl_sync(FULL, incl, c + st - 1) <= kk) ? st : 0;
        const int cc = __shfl_sync(FULL, cid, c);
        const int ex = __shfl_sync(FULL, excl, c);
        int j = -1;
        float4 rj = make_float4(0.f, 0.f, 0.f, 0.f);
        if (kk < total) {
            const long long idx = (long long)cc * ccap + (kk - ex);
            j = s.cell_id[idx];
            rj = s.cell_ref[idx];
        }
        bool ins = false, fj = false;
        if (kk < total && j >= 0 && j != i) {
            fj = bit_of(s.ubits, j);
            if (!(direct && fj) && pair_hit(qn, rj))
                ins = !pair_hit(qo, fj ? s.pold[j] : rj);
        }
        own_row_insert(s, off, cap, ins, j, &freemask, &tail);
        work[2] += __popc(__ballot_sync(FULL, ins && !fj));
        if (ins && !fj) lane_insert(s, j, i, ovf);
    }
    if (direct) {
        const bool own = s.sc_cnt != nullptr;
        const float4 *lst = own ? s.sfref + g.first : s.fref;
        const int *ids = own ? s.sfid + g.first : s.fid;
        const int m = own ? s.sc_cnt[par * s.nscenes + sc] : nF;
        work[1] += m;
        for (int b0 = 0; b0 < m; b0 += 32) {
            const int kk = b0 + lane;
            int j = -1;
            if (kk < m && pair_hit(qn, lst[kk])) {
                j = ids[kk];
                if (j == i || j < g.first || j >= g.first + g.count) j = -1;
            }
            const bool ins = j >= 0 && !pair_hit(qo, s.pold[j]);
            own_row_insert(s, off, cap, ins, j, &freemask, &tail);
        }
    }
    if (lane == 0) {
        s.row_len[i] = tail;
        if (tail > cap) atomicExch(ovf, 1);
    }
}

// a4: rows of every particle by the 27-cell stencil, one warp per row
// (init, store growth, re-layout, GLOBAL / ALWAYS).  Lanes 0..26 each own
// one neighbour cell; a warp scan of their occupancies flattens the
// candidates, and every lane finds its candidate's cell with a 5-step
// shuffle binary search, so lanes stay busy across cell boundaries.
// fill = 0 counts only (row_len = count); fill = 1 also writes up to the
// row's capacity, clears the rest of the row to -1 and raises *ovf if the
// row does not fit.  The cells must hold the final reference states.  With
// contact history each written entry's record is zero, or, with carry, the
// record of the same partner in the particle's row as it was before
// (old_off / old_len / old_col / old_hist; zero if not there).
__device__ __forceinline__ float4 carried_history(const DevState &s, int i, int j)
{
    const int o = s.old_off[i], l = s.old_len[i];
    for (int e = 0; e < l; ++e)
        if (s.old_col[o + e] == j) return s.old_hist[o + e];
    return make_float4(0.f, 0.f, 0.f, 0.f);
}

__device__ __forceinline__ void ph_rows(const DevState &s, int nitems, int fill, int w0,
                                        int wstride, int *ovf, bool carry = false)
{
    const int lane = threadIdx.x & 31;
    const int ccap = s.ccap;
    const unsigned lt = lanemask_lt();
    for (int i = w0; i < nitems; i += wstride) {
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
                const float dd = s.reach ? cell_dist2(g, x, y, z, qi) : 0.0f;
                if (s.reach == 0 || within_reach(g, dd, qi.w, g.H)) {
                    cid = g.cell_base + (z * d1 + y) * d0 + x;
                    cnt_l = min(s.cell_cnt[cid], ccap);
                    if (s.reach == 2 &&
                        !within_reach(g, dd, qi.w, __int_as_float(s.cell_rmax[cid])))
                        cnt_l = 0;
                }
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
            for (int st = 16; st >= 1; st >>= 1)
                c += (__shfl_sync(FULL, incl, c + st - 1) <= k) ? st : 0;
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
                if (p < cap) {
                    s.col[off + p] = j;
                    if (s.hist)
                        s.hist[off + p] = carry ? carried_history(s, i, j)
                                                : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            found += __popc(m);
        }
        if (fill)
            for (int e = found + lane; e < cap; e += 32) s.col[off + e] = -1;
        if (lane == 0) {
            s.row_len[i] = found;
            if (fill && found > cap) atomicExch(ovf, 1);
        }
    }
}

// ---------------------------------------------------------------------------
// Grid-wide barrier of the step kernel (all blocks co-resident).  A 64-bit
// arrival counter per step parity: the kernel of a step counts on
// bar_cnt[parity] (which starts at zero) and clears the other one for the
// next step.  Thread 0 of each block arrives with a release add (no
// return value to wait for) and polls with acquire loads until the counter
// holds the arrivals of this barrier and of all earlier ones in the kernel.
// Polling is bounded: after s.bar_spins polls (kBarrierSpins unless a test
// lowers it) the block records DERR_SYNC and leaves; every block then
// returns, and later steps do nothing (the context reports LVB_ETIMEOUT).
// Returns false when the step must be abandoned.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void red_add_release(unsigned long long *p, unsigned long long v)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// the barrier state of this block (used by its thread 0 only)
static __shared__ unsigned long long s_bar_need;   // arrivals up to the last barrier
static __shared__ int s_bar_par;                   // parity of the step
// the block's share of the partial rebuild's work counts (DevCounters
// alg_*), gathered by its warps with shared-memory atomics and added to the
// context's counters by thread 0 once per step
static __shared__ unsigned long long s_work[3];
// the block's rebuild work items when traced: first start, last end,
// longest item (item_start / item_stop)
static __shared__ unsigned long long s_items[3];
static __shared__ unsigned long long s_item_t0[kStepMaxThreads / 32];

// Called by every thread at the start of the step kernel, before any barrier.
__device__ __forceinline__ void grid_barrier_begin(const DevState &s, int par)
{
    if (threadIdx.x == 0) {
        s_bar_need = 0;
        s_bar_par = par;
        s_work[0] = s_work[1] = s_work[2] = 0ULL;
        s_items[0] = ~0ULL;
        s_items[1] = s_items[2] = 0ULL;
        if (blockIdx.x == 0) s.cnt->bar_cnt[par ^ 1] = 0;
    }
}

__device__ __forceinline__ bool grid_barrier(const DevState &s)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        DevCounters *c = s.cnt;
        unsigned long long *w = &c->bar_cnt[s_bar_par];
        const unsigned long long need = s_bar_need + gridDim.x + s.bar_extra;
        s_bar_need = need;
        red_add_release(w, 1ULL);
        int ok = 1;
        unsigned it = 0;
        while (ld_acquire(w) < need) {
            if (++it > s.bar_spins) {
                atomicOr(&c->err, DERR_SYNC);
                ok = 0;
                break;
            }
        }
        if (ok && blockIdx.x == 0) atomicAdd(&c->barriers, 1ULL);
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Exclusive scan over the block (any block size up to 1024); *total gets
// the block's sum.  Contains block barriers.
__device__ __forceinline__ long long block_scan_any(long long v, long long *total)
{
    __shared__ long long ws[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long y = lane < nw ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(FULL, y, o);
            if (lane >= o) y += t;
        }
        if (lane < nw) ws[lane] = y;
    }
    __syncthreads();
    const long long before = warp ? ws[warp - 1] : 0;
    *total = ws[nw - 1];
    __syncthreads();
    return before + x - v;
}

// ---------------------------------------------------------------------------
// Flagged particles a warp found in the check and has not yet entered in
// the flagged list: their ids, in shared memory (per warp).  The list
// indices are taken when the pending list is flushed (when it fills, and at
// the end of the pass), so no atomic round trip holds up the block's stream
// of tiles, and the updates' dependent loads run after the warp's tiles.
constexpr int kPending = 32;

struct Pending {
    int *id;    // kPending entries of this warp
    int n;      // warp-uniform count
};

// a2 of the learned policy, and of any policy while the rebuild log is on,
// waits until the check pass has ended: then every warp of the grid takes
// at most a few flagged particles (update_pass) instead of the warps that
// flagged them taking all of theirs one after another inside the check.
__device__ __forceinline__ bool deferred_update(const DevState &s)
{
    return s.skin_kind == LVB_SKIN_LEARNED || s.log_on;
}

// Enters the warp's pending particles in the flagged list at k0, k0 + 1, ...
// (fid) and, with inc, updates them one per lane (update_lanes) unless the
// update is deferred; empties the list.  New positions written earlier in this kernel by the warp's own
// lanes (DEM form) are made visible to the whole warp first.
__device__ __forceinline__ void enter_pending(const DevState &s, Pending &pd, int k0,
                                              const float4 *pos, const float4 *vel,
                                              const float4 *acc, bool inc, int step)
{
    const int lane = threadIdx.x & 31;
    __syncwarp();
    if (lane < pd.n) s.fid[k0 + lane] = pd.id[lane];
    if (inc && !deferred_update(s)) update_lanes(s, pd.id, k0, pd.n, pos, vel, step);
    __syncwarp();
    pd.n = 0;
}

// The same with list indices from one atomic of this warp.
__device__ __forceinline__ void flush_pending(const DevState &s, Pending &pd, const float4 *pos,
                                              const float4 *vel, const float4 *acc, bool inc,
                                              int step, int *nF_acc)
{
    int k0 = 0;
    if ((threadIdx.x & 31) == 0) k0 = atomicAdd(nF_acc, pd.n);
    k0 = __shfl_sync(FULL, k0, 0);
    enter_pending(s, pd, k0, pos, vel, acc, inc, step);
}

// End of the check pass, every thread of the block: the pending particles
// of all warps enter the list -- with one atomic per warp (warp scheme) or
// one per block after a scan of the warps' counts (block scheme).
__device__ __forceinline__ void flush_pending_final(const DevState &s, Pending &pd,
                                                    const float4 *pos, const float4 *vel,
                                                    const float4 *acc, bool inc, int step,
                                                    int *nF_acc)
{
    if (!s.compact_block) {
        if (pd.n) flush_pending(s, pd, pos, vel, acc, inc, step, nF_acc);
        return;
    }
    __shared__ int s_cnt[32];
    __shared__ int s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (!__syncthreads_or(pd.n)) return;
    if (lane == 0) s_cnt[warp] = pd.n;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const int v = s_cnt[w];
            s_cnt[w] = run;
            run += v;
        }
        s_base = atomicAdd(nF_acc, run);
    }
    __syncthreads();
    if (pd.n) enter_pending(s, pd, s_base + s_cnt[warp], pos, vel, acc, inc, step);
}

// a1 for U chunks of 32 consecutive particles held by one warp (chunk u
// starts at cu[u], a multiple of 32; f[u] is this lane's flag in it): one
// ballot word per chunk; the flagged particles join the warp's pending list
// (entered in the flagged list, and updated with the PARTIAL trigger, when
// it fills and at the end of the pass).
template <int U>
__device__ __forceinline__ void flag_chunks(const DevState &s, const int (&cu)[U],
                                            const bool (&f)[U], const float4 *pos,
                                            const float4 *vel, const float4 *acc, bool inc,
                                            int step, int *nF_acc, Pending &pd)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const unsigned b = __ballot_sync(FULL, f[u]);
        if (lane == 0 && cu[u] < s.n) {
            s.bits[cu[u] >> 5] = b;
            if (s.bits_out) s.bits_out[cu[u] >> 5] = b;
        }
        if (!b) continue;
        if (pd.n + __popc(b) > kPending) flush_pending(s, pd, pos, vel, acc, inc, step, nF_acc);
        if (b >> lane & 1u) pd.id[pd.n + __popc(b & lt)] = cu[u] + lane;
        pd.n += __popc(b);
    }
}

// The check pass of the DEM form: each thread first performs the driver's
// position half-step of its particles (integrate_one), so the positions are
// produced here and read back from registers.  Block b takes tiles b,
// b + grid, ... of blockDim * kCheckUnroll particles; in a tile each warp
// checks kCheckUnroll chunks of 32 (loads of all chunks first).
__device__ __forceinline__ void check_pass_fused(const DevState &s, const float4 *vel,
                                                 const float4 *acc, const IntegrateArgs &ia,
                                                 bool inc, int step, int *nF_acc)
{
    __shared__ int pend_id[kStepMaxThreads / 32][kPending];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Pending pd{pend_id[warp], 0};
    const int tile = blockDim.x * kCheckUnroll;
    for (int t0 = blockIdx.x * tile; t0 < s.n; t0 += gridDim.x * tile) {
        float4 p[kCheckUnroll], q[kCheckUnroll];
        int cu[kCheckUnroll];
        bool f[kCheckUnroll];
#pragma unroll
        for (int u = 0; u < kCheckUnroll; ++u) {
            cu[u] = t0 + u * blockDim.x + warp * 32;
            const int i = cu[u] + lane;
            if (i < s.n) {
                p[u] = integrate_one(ia, geom_of(s, i), i);
                q[u] = s.ref[i];
            }
        }
#pragma unroll
        for (int u = 0; u < kCheckUnroll; ++u) {
            const int i = cu[u] + lane;
            f[u] = false;
            if (i < s.n) {
                f[u] = violates(p[u], q[u]);
                if (!(isfinite(p[u].x) && isfinite(p[u].y) && isfinite(p[u].z)))
                    atomicOr(&s.cnt->err, DERR_NAN);
            }
        }
        flag_chunks<kCheckUnroll>(s, cu, f, ia.pos, vel, acc, inc, step, nF_acc, pd);
    }
    flush_pending_final(s, pd, ia.pos, vel, acc, inc, step, nF_acc);
}

// The check pass of the broad phase alone, register form
// (LVB_OPT_CHECK_LOADS = LVB_CHECK_REGS): block b takes tiles b, b + grid,
// ... of blockDim * kCheckRegsUnroll particles; each warp loads its
// kCheckRegsUnroll chunks of 32 consecutive particles' pos and ref at once
// (streaming loads: read once, evict first), so every warp keeps 16 loads
// of 16 bytes in flight with no block barrier in the loop.
constexpr int kCheckRegsUnroll = 4;

__device__ __forceinline__ void check_pass_regs(const DevState &s, const float4 *__restrict__ pos,
                                                const float4 *vel, const float4 *acc, bool inc,
                                                int step, int *nF_acc)
{
    constexpr int U = kCheckRegsUnroll;
    __shared__ int pend_id[kStepMaxThreads / 32][kPending];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Pending pd{pend_id[warp], 0};
    const int tile = blockDim.x * U;
    for (int t0 = blockIdx.x * tile; t0 < s.n; t0 += gridDim.x * tile) {
        float4 p[U], q[U];
        int cu[U];
        bool f[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            cu[u] = t0 + u * blockDim.x + warp * 32;
            const int i = cu[u] + lane;
            if (i < s.n) {
                p[u] = __ldcs(pos + i);
                q[u] = __ldcs(s.ref + i);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = cu[u] + lane;
            f[u] = false;
            if (i < s.n) {
                f[u] = violates(p[u], q[u]);
                if (!(isfinite(p[u].x) && isfinite(p[u].y) && isfinite(p[u].z)))
                    atomicOr(&s.cnt->err, DERR_NAN);
            }
        }
        flag_chunks<U>(s, cu, f, pos, vel, acc, inc, step, nF_acc, pd);
    }
    flush_pending_final(s, pd, pos, vel, acc, inc, step, nF_acc);
}

// ---------------------------------------------------------------------------
// Bulk copies into shared memory (cp.async.bulk, completion counted by an
// mbarrier), for the check pass of the broad phase alone.
// ---------------------------------------------------------------------------
constexpr int kStages = 4;                 // tiles in flight per block
constexpr unsigned kStageWaitSpins = 1u << 22;

__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Global -> shared bulk copy of `bytes` (a multiple of 16, both addresses
// 16-byte aligned) that completes `bytes` transactions on *bar.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    unsigned long long g;
    asm volatile("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(src));
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(g), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Bounded wait for a stage: true when its copies have landed.
__device__ __forceinline__ bool stage_wait(uint64_t *bar, unsigned parity)
{
    for (unsigned it = 0; it < kStageWaitSpins; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Dynamic shared memory of the check pass for a block of `threads`.
__host__ __device__ constexpr int check_smem_bytes(int threads)
{
    return kStages * threads * 2 * (int)sizeof(float4);
}

// The check pass of the broad phase alone.  Block b takes tiles b, b + grid,
// ... of blockDim particles; thread 0 keeps kStages tiles of pos and ref in
// flight as bulk copies into a ring of shared-memory stages, every thread
// checks its particle from shared memory, and the stage is refilled once
// the whole block is done with it.  A stage whose copies do not land within
// kStageWaitSpins polls is reported (DERR_SYNC) and skipped, never waited
// for indefinitely.
__device__ __forceinline__ void check_pass_stream(const DevState &s, const float4 *__restrict__ pos,
                                                  const float4 *vel, const float4 *acc, bool inc,
                                                  int step, int *nF_acc)
{
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ __align__(8) uint64_t bar[kStages];
    __shared__ int pend_id[kStepMaxThreads / 32][kPending];
    const int T = blockDim.x, tid = threadIdx.x, warp = tid >> 5;
    Pending pd{pend_id[warp], 0};
    float4 *spos = reinterpret_cast<float4 *>(dsm);
    float4 *sref = spos + kStages * T;
    const int ntiles = (s.n + T - 1) / T;
    const int mine = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) mbar_init(&bar[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](int j) {   // thread 0 only
        const int t0 = (blockIdx.x + j * gridDim.x) * T;
        const unsigned bytes = (unsigned)min(T, s.n - t0) * (unsigned)sizeof(float4);
        const int st = j % kStages;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bar[st], 2u * bytes);
        bulk_load(spos + st * T, pos + t0, bytes, &bar[st]);
        bulk_load(sref + st * T, s.ref + t0, bytes, &bar[st]);
    };
    int issued = 0;   // meaningful in thread 0
    if (tid == 0)
        for (; issued < min(kStages, mine); ++issued) issue(issued);
    bool failed = false;
    int j = 0;
    for (; j < mine; ++j) {
        const int st = j % kStages;
        const bool landed = stage_wait(&bar[st], (unsigned)(j / kStages) & 1u);
        if (__syncthreads_or(!landed)) {
            if (tid == 0) atomicOr(&s.cnt->err, DERR_SYNC);
            failed = true;
            break;
        }
        const int t0 = (blockIdx.x + j * gridDim.x) * T;
        const int i = t0 + tid;
        const int cu[1] = {t0 + warp * 32};
        bool f[1] = {false};
        if (i < s.n) {
            const float4 p = spos[st * T + tid];
            f[0] = violates(p, sref[st * T + tid]);
            if (!(isfinite(p.x) && isfinite(p.y) && isfinite(p.z)))
                atomicOr(&s.cnt->err, DERR_NAN);
        }
        flag_chunks<1>(s, cu, f, pos, vel, acc, inc, step, nF_acc, pd);
        __syncthreads();   // the block is done with this stage
        if (tid == 0 && j + kStages < mine) issue(issued++);
    }
    if (failed && tid == 0) {
        // copies still in flight land before the block leaves.  The wait is
        // bounded like every wait here; a copy of in-bounds memory lands in
        // microseconds, so one that outlasts it would mean the device is
        // already failing.  The context is marked failed (DERR_SYNC): no
        // later step on it launches work that uses this block's stages.
        for (int k = j; k < issued; ++k)
            stage_wait(&bar[k % kStages], (unsigned)(k / kStages) & 1u);
    }
    flush_pending_final(s, pd, pos, vel, acc, inc, step, nF_acc);
}

static __device__ __noinline__ void full_update_pass(const DevState &s, const float4 *pos,
                                              const float4 *vel)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    for (int i = t; i < s.n; i += nt) {
        const float4 p = pos[i];
        const float4 v = vel ? vel[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const SceneGeom &g = geom_of(s, i);
        const float sk = skin_of(s.skin_kind, s.skin_value, s.skin_dt, g.H, s.rad[i], v, 0.0f);
        s.ref[i] = make_float4(p.x, p.y, p.z, sk);
        s.cell_of[i] = cell_key(g, p.x, p.y, p.z);
    }
    for (long long c = t; c < s.ncells; c += nt) {
        s.cell_cnt[c] = 0;
        s.cell_live[c] = 0;
        s.cell_rmax[c] = 0;
    }
}

static __device__ __noinline__ void full_insert_pass(const DevState &s)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    const int ccap = s.ccap;
    for (int i = t; i < s.n; i += nt) {
        const int c = s.cell_of[i];
        const int sl = atomicAdd(&s.cell_cnt[c], 1);
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
        if (sl * 4 >= ccap * 3) s.hflags->grow_cells = 1;
    }
}

static __device__ __noinline__ void all_rows_pass(const DevState &s, int fill, int *ovf,
                                                  bool carry = false)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    ph_rows(s, s.n, fill, t >> 5, nt >> 5, ovf, carry);
}

// Contact history: the rows as they stand (offsets, lengths, entries and
// records up to the extent of the last layout) copied aside before a
// re-layout, so that the new rows can carry each entry's history.
static __device__ __noinline__ void save_rows_pass(const DevState &s)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nt = (long long)gridDim.x * blockDim.x;
    for (long long i = t; i < s.n; i += nt) {
        s.old_off[i] = s.row_off[i];
        s.old_len[i] = min(s.row_len[i], s.row_cap[i]);
    }
    const long long ext = min(*(volatile long long *)&s.cnt->store_needed, s.col_cap);
    for (long long e = t; e < ext; e += nt) {
        s.old_col[e] = s.col[e];
        s.old_hist[e] = s.hist[e];
    }
}

// Offsets of the row store by a grid-wide exclusive scan of the row sizes
// (row_capacity(len), or len itself when tight), block b owning rows
// [b * per, (b + 1) * per); block 0 scans the block sums and writes the
// total to store_needed.  Every block returns the total (read after a
// barrier).  Returns -1 when the step must be abandoned.
static __device__ long long layout_scan(const DevState &s, bool tight)
{
    DevCounters *c = s.cnt;
    const long long per = ((long long)s.n + gridDim.x - 1) / gridDim.x;
    const int lo = (int)min((long long)s.n, blockIdx.x * per);
    const int hi = (int)min((long long)s.n, lo + per);
    long long sum = 0, tot;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x)
        sum += tight ? s.row_len[i] : row_capacity(s.row_len[i]);
    block_scan_any(sum, &tot);
    if (threadIdx.x == 0) s.blk[blockIdx.x] = tot;
    if (!grid_barrier(s)) return -1;
    if (blockIdx.x == 0) {
        __shared__ long long carry;
        if (threadIdx.x == 0) carry = 0;
        __syncthreads();
        for (int b0 = 0; b0 < (int)gridDim.x; b0 += blockDim.x) {
            const int b = b0 + threadIdx.x;
            const long long v = b < (int)gridDim.x ? s.blk[b] : 0;
            const long long ex = block_scan_any(v, &tot);
            if (b < (int)gridDim.x) s.blk[b] = carry + ex;
            __syncthreads();
            if (threadIdx.x == 0) carry += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0) c->store_needed = carry;
    }
    if (!grid_barrier(s)) return -1;
    long long run = s.blk[blockIdx.x];
    for (int i0 = lo; i0 < hi; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const int v = i < hi ? (tight ? s.row_len[i] : row_capacity(s.row_len[i])) : 0;
        const long long ex = block_scan_any(v, &tot);
        if (i < hi) {
            s.row_off[i] = (int)min(run + ex, (long long)INT32_MAX);
            s.row_cap[i] = v;
        }
        run += tot;
    }
    return *(volatile long long *)&c->store_needed;
}

// Re-layout of the row store after a row outgrew its slack: rows counted
// from the (final) cells, offsets with slack, rows filled.  When the rows
// with slack do not fit the store they are laid out tight (no slack; the
// next edits re-lay out again) and, if even that does not fit, the store
// has failed (DERR_STORE).  A layout above 60% of the store asks the host
// to grow it before the next step.  Returns false when the step must be
// abandoned.
static __device__ __noinline__ bool relayout_pass(const DevState &s)
{
    DevCounters *c = s.cnt;
    if (s.hist) {
        save_rows_pass(s);
        if (!grid_barrier(s)) return false;
    }
    all_rows_pass(s, 0, nullptr);
    if (!grid_barrier(s)) return false;
    const long long need = layout_scan(s, false);
    if (need < 0) return false;
    long long used = need;
    if (need > s.col_cap) {
        if (!grid_barrier(s)) return false;   // everyone has read the slack total
        used = layout_scan(s, true);
        if (used < 0) return false;
        if (used > s.col_cap && blockIdx.x == 0 && threadIdx.x == 0)
            atomicOr(&c->err, DERR_STORE);
    }
    if (!grid_barrier(s)) return false;
    if (!store_failed(s)) {
        int unused = 0;
        all_rows_pass(s, 1, &unused, s.hist != nullptr);
    }
    if (!grid_barrier(s)) return false;
    if (blockIdx.x == 0 && threadIdx.x == 0 && !store_failed(s)) {
        c->force_relayout = 0;
        c->relayouts += 1;
        c->store_needed = need;
        if (need * 5 > s.col_cap * 3) {        // over 60% of the store: grow it
            s.hflags->store_needed = need;
            s.hflags->grow_store = 1;
        }
    }
    (void)used;
    return true;
}

// Rebuild log: every open record tracks the particle's largest displacement
// since it opened, and closes `horizon` steps later with label
// sqrt(max |x - x_open|^2) / d.
static __device__ __noinline__ void log_pass(const DevState &s, const float4 *pos, int step)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    for (int i = t; i < s.n; i += nt) {
        const int t0 = s.lg_t[i];
        if (t0 < 0) continue;
        const float4 p = pos[i];
        const float4 x0 = s.lg_x[i];
        const float m = fmaxf(s.lg_m[i], sqdist_rn(p.x, p.y, p.z, x0.x, x0.y, x0.z));
        if (step - t0 >= s.log_horizon) {
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

// The early trigger (LVB_OPT_EARLY), on a step where some particle
// violates Eq. update: every other particle whose displacement exceeds
// beta times its skin, |x - xref|^2 > (beta skin)^2 in the fixed binary32
// formula, is updated too, so that the next violation comes later (a
// reading of Def. autoverlet's trigger between its per-particle and global
// forms: the pair set stays the function of (xref, skin) it always is).
// One warp per 32 consecutive particles: the updated-set word ubits = the
// flag word | the early ones; the early ones join the flagged list (one
// atomic per warp) and, unless the update is deferred, are updated here.
static __device__ __noinline__ void early_pass(const DevState &s, const float4 *pos,
                                               const float4 *vel, int step, int *nF_acc)
{
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    __shared__ int ids_sh[kStepMaxThreads / 32][32];
    int *ids = ids_sh[threadIdx.x >> 5];
    for (int w = w0; w < s.nwords; w += nw) {
        const int i = w * 32 + lane;
        const uint32_t fw = s.bits[w];
        bool e = false;
        if (i < s.n && !((fw >> lane) & 1u)) {
            const float4 p = pos[i];
            const float4 q = s.ref[i];
            const float t = __fmul_rn(s.early_beta, q.w);
            e = sqdist_rn(p.x, p.y, p.z, q.x, q.y, q.z) > __fmul_rn(t, t);
        }
        const unsigned m = __ballot_sync(FULL, e);
        if (lane == 0) s.ubits[w] = fw | m;
        if (!m) continue;
        int k0 = 0;
        if (lane == 0) k0 = atomicAdd(nF_acc, __popc(m));
        k0 = __shfl_sync(FULL, k0, 0);
        const int r = __popc(m & lanemask_lt());
        if (e) {
            ids[r] = i;
            s.fid[k0 + r] = i;
        }
        __syncwarp();
        if (!deferred_update(s)) update_lanes(s, ids, k0, __popc(m), pos, vel, step);
        __syncwarp();
    }
}

// Tail of a step that only does the broad phase.
struct NoTail {
    static constexpr bool kActive = false;
    __device__ void operator()(int, int) const {}
};

__device__ __forceinline__ void trace_add(DevCounters *c, int slot, unsigned long long a,
                                          unsigned long long b)
{
    c->tr_sum[slot] += b - a;
    c->tr_cnt[slot] += 1;
}

// The deferred a2 (deferred_update) for the nF flagged particles of the
// step: each warp takes groups of c = ceil(nF / warps) <= 32 consecutive
// list entries (update_group), the groups spread over the blocks first as
// in partial_pass.
static __device__ __noinline__ void update_pass(const DevState &s, const lvb_mlp_weights *W,
                                                int nF, const float4 *pos, const float4 *vel,
                                                const float4 *acc, int step)
{
    const int w0 = (int)(threadIdx.x >> 5) * (int)gridDim.x + (int)blockIdx.x;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int c = min(32, (nF + nw - 1) / nw);
    for (long long k0 = (long long)w0 * c; k0 < nF; k0 += (long long)nw * c)
        update_group(s, W, (int)k0, min(c, nF - (int)k0), pos, vel, acc, step);
}

// Trace of the rebuild's work items (LVB_OPT_TRACE; lane 0 of each warp):
// each item's start is kept in shared memory (nothing held in registers
// across the item), and the block's first start, last end and longest item
// gather in s_items by shared-memory atomics; items_flush adds them to the
// context's trace slots TR_ITEMS / TR_ITEM_MAX before the step's last
// barrier.
__device__ __forceinline__ void item_start(const DevState &s)
{
    if (s.trace && (threadIdx.x & 31) == 0) s_item_t0[threadIdx.x >> 5] = global_ns();
}

__device__ __forceinline__ void item_stop(const DevState &s)
{
    if (s.trace && (threadIdx.x & 31) == 0) {
        const unsigned long long tb = global_ns(), ta = s_item_t0[threadIdx.x >> 5];
        atomicMin(&s_items[0], ta);
        atomicMax(&s_items[1], tb);
        atomicMax(&s_items[2], tb - ta);
    }
}

__device__ __forceinline__ void items_flush(const DevState &s)
{
    __syncthreads();
    if (threadIdx.x == 0 && s_items[1] != 0) {
        DevCounters *c = s.cnt;
        atomicMin(&c->tr_start[TR_ITEMS], s_items[0]);
        atomicMax(&c->tr_end[TR_ITEMS], s_items[1]);
        atomicMin(&c->tr_start[TR_ITEM_MAX], 0ULL);
        atomicMax(&c->tr_end[TR_ITEM_MAX], s_items[2]);
    }
}

// The rebuild of a partial step (nF flagged).  Up to s.direct_max
// flagged particles: moves and patches in one phase, on different warps
// (work items 0..nF-1 patch rows, nF..2nF-1 move cell slots; the patches
// skip the flagged particles in the cells and test them directly); more:
// the moves first and a barrier, then the patches on final cells.  Returns
// false when the step must be abandoned.
static __device__ __noinline__ bool partial_pass(const DevState &s, int nF, int par, int *ovf)
{
    // work items go round the blocks first (item w to block w % grid), so
    // that a few flagged particles spread over all SMs instead of filling
    // the warps of the first blocks
    const int w0 = (int)(threadIdx.x >> 5) * (int)gridDim.x + (int)blockIdx.x;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const bool direct = nF <= s.direct_max;
    unsigned work[3] = {0u, 0u, 0u};
    if (!direct) {
        for (int k = w0; k < nF; k += nw) {
            item_start(s);
            move_warp(s, s.fid[k], s.fref[k], flagged_scene(s, k));
            item_stop(s);
        }
        if (!grid_barrier(s)) return false;
        for (int k = w0; k < nF; k += nw) {
            item_start(s);
            if (s.hist) patch_warp_hist(s, k, nF, false, par, ovf, work);
            else patch_warp(s, k, nF, false, par, ovf, work);
            item_stop(s);
        }
    } else {
        for (int w = w0; w < 2 * nF; w += nw) {
            item_start(s);
            if (w < nF) {
                if (s.hist) patch_warp_hist(s, w, nF, true, par, ovf, work);
                else patch_warp(s, w, nF, true, par, ovf, work);
            } else {
                move_warp(s, s.fid[w - nF], s.fref[w - nF], flagged_scene(s, w - nF));
            }
            item_stop(s);
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (work[q]) atomicAdd(&s_work[q], (unsigned long long)work[q]);
    }
    return true;
}

// Adds the block's rebuild work counts to the context's (thread 0, after a
// block barrier that follows partial_pass).
__device__ __forceinline__ void flush_work(const DevState &s)
{
    if (threadIdx.x == 0) {
        DevCounters *c = s.cnt;
        if (s_work[0]) atomicAdd(&c->alg_cand, s_work[0]);
        if (s_work[1]) atomicAdd(&c->alg_direct, s_work[1]);
        if (s_work[2]) atomicAdd(&c->alg_edits, s_work[2]);
    }
}

// ---------------------------------------------------------------------------
// One step.  pos_in / vel / acc: the caller's positions, velocities (policy
// input) and accelerations; with kFused the positions come from the DEM
// half-step (ia) instead.  Launched cooperatively with every block resident.
// Per-step counts live in two slots chosen by the step's parity, so that the
// slots of the next step can be cleared while this one is read.  The list
// is final when the kernel ends (and before the tail).
// ---------------------------------------------------------------------------
template <bool kFused, class Tail>
__global__ void __launch_bounds__(kStepMaxThreads, 1)
k_step(const float4 *__restrict__ pos_in, const float4 *vel, const float4 *acc,
       const __grid_constant__ DevState sp,
       IntegrateArgs ia, Tail tail)
{
    // the context's state read in place from the parameter space (uniform
    // reads through the constant cache; no copy at the start)
    const DevState &s = sp;
    DevCounters *c = s.cnt;
    // the step's bookkeeping (counters, trace) runs on the last warp of
    // block 0, whose rebuild work items come last
    const bool lead = blockIdx.x == 0 && threadIdx.x == blockDim.x - 32;
    const unsigned long long t0 = (s.trace && lead) ? global_ns() : 0ULL;
    // every thread reads the counters it needs (one broadcast load each, no
    // block barrier before the check's loads); they are stable while the
    // check runs
    const unsigned err = c->err;
    if (err & DERR_SYNC) return;   // a barrier failed earlier: the context is unusable
    const bool inc = s.trigger == LVB_TRIGGER_PARTIAL && !(err & DERR_STORE);
    const int step = (int)c->steps + 1, par = step & 1;
    __shared__ __align__(16) lvb_mlp_weights w_sh;
    const bool net = s.skin_kind == LVB_SKIN_LEARNED;
    if (net) weights_copy_async(&w_sh, s.mlp);
    grid_barrier_begin(s, par);
    const float4 *pos = kFused ? ia.pos : pos_in;
    int *ovf = &c->ovf[par];

    if constexpr (kFused)
        check_pass_fused(s, vel, acc, ia, inc, step, &c->nF_acc[par]);
    else if (s.check_regs)
        check_pass_regs(s, pos_in, vel, acc, inc, step, &c->nF_acc[par]);
    else
        check_pass_stream(s, pos_in, vel, acc, inc, step, &c->nF_acc[par]);
    if (net) weights_copy_wait();
    if (!grid_barrier(s)) return;
    const int nV = *(volatile int *)&c->nF_acc[par];   // violations of Eq. update
    int nF = nV;                                        // particles updated
    if (inc && nV > 0 && s.early_beta < 1.0f) {
        early_pass(s, pos, vel, step, &c->nF_acc[par]);
        if (!grid_barrier(s)) return;
        nF = *(volatile int *)&c->nF_acc[par];
    }
    if (s.sc_cnt && blockIdx.x == 0)   // the next step's scene counters
        for (int q = threadIdx.x; q < s.nscenes; q += blockDim.x)
            s.sc_cnt[(par ^ 1) * s.nscenes + q] = 0;
    int upd;
    if (s.trigger == LVB_TRIGGER_PARTIAL) upd = nF;
    else if (s.trigger == LVB_TRIGGER_GLOBAL) upd = nV ? s.n : 0;
    else upd = s.n;
    unsigned long long t1 = 0;
    if (lead) {
        // stores and reductions only: no load on the step's last path
        c->nF_acc[par ^ 1] = 0;
        c->ovf[par ^ 1] = 0;
        c->nF = nV;
        if (s.nf_out) *s.nf_out = nV;
        c->last_flagged = nV;
        c->last_updated = upd;
        atomicAdd((unsigned long long *)&c->steps, 1ULL);
        atomicAdd((unsigned long long *)&c->flagged_total, (unsigned long long)nV);
        atomicAdd((unsigned long long *)&c->updated_total, (unsigned long long)upd);
        if (upd) atomicAdd((unsigned long long *)&c->rebuild_steps, 1ULL);
        atomicAdd(&c->kernels, 1ULL);
        if (s.trace) {
            t1 = global_ns();
            trace_add(c, TR_CHECK, t0, t1);
            // separate kernels (DEM phases, full-build rows) since the last step
            for (int k = TR_INTEGRATE; k <= TR_ROWS; ++k) {
                const unsigned long long a = c->tr_start[k], b = c->tr_end[k];
                if (b != 0 && b >= a) trace_add(c, k, a, b);
                c->tr_start[k] = ~0ULL;
                c->tr_end[k] = 0;
            }
        }
    }
    bool changed = false;
    if (inc) {
        if (nF > 0) {
            if (deferred_update(s)) {
                update_pass(s, &w_sh, nF, pos, vel, acc, step);
                if (!grid_barrier(s)) return;
            }
            if (!partial_pass(s, nF, par, ovf)) return;
            if (s.trace) items_flush(s);
            changed = true;
        }
    } else if (upd > 0 && !store_failed(s)) {
        full_update_pass(s, pos, vel);
        if (!grid_barrier(s)) return;
        full_insert_pass(s);
        if (!grid_barrier(s)) return;
        all_rows_pass(s, 1, ovf);
        changed = true;
    }
    if (changed) {
        if (!grid_barrier(s)) return;
        flush_work(s);
        unsigned long long t2 = 0;
        if (s.trace && lead) {
            t2 = global_ns();
            trace_add(c, TR_REBUILD, t1, t2);
            for (int k = TR_ITEMS; k <= TR_ITEM_MAX; ++k) {
                const unsigned long long a = c->tr_start[k], b = c->tr_end[k];
                if (b != 0 && b >= a) trace_add(c, k, a, b);
                c->tr_start[k] = ~0ULL;
                c->tr_end[k] = 0;
            }
        }
        if ((*(volatile int *)ovf || *(volatile int *)&c->force_relayout) && !store_failed(s)) {
            if (!relayout_pass(s)) return;
            if (s.trace && lead) trace_add(c, TR_RELAYOUT, t2, global_ns());
        }
    }
    if (s.log_on) log_pass(s, pos, step);
    if (Tail::kActive) {
        const unsigned long long t3 = (s.trace && lead) ? global_ns() : 0ULL;
        tail(blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
        if (s.trace) {
            if (!grid_barrier(s)) return;
            if (lead) trace_add(c, TR_TAIL, t3, global_ns());
        }
    }
}

}  // namespace lvb
