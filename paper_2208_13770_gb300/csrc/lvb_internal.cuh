// lvb_internal.cuh -- device-side definitions shared by the liblvb sources.
//
// Data layout in device memory (all structure-of-arrays, 16-byte records):
//   ref[i]      float4 (xref, yref, zref, skin)   reference state of i
//   rad[i]      float                             radius (fixed at init)
//   cell_of[i]  int    cell of xref_i;  slot_of[i]  its slot in that cell
//   cells       fixed-capacity slots, cell c owns slots [c*ccap, (c+1)*ccap):
//               cell_id (int) and cell_ref (float4 xref, yref, zref, R_NL)
//               -- a copy of the reference state in cell order, so that the
//               27-cell stencil reads contiguous, coalesced runs
//   rows        one row per particle in a slack CSR: entries
//               col[row_off[i] .. row_off[i] + row_len[i]), capacity
//               row_cap[i] >= row_len[i]; a row that outgrows its capacity
//               triggers a re-layout of the whole row store on the device
//   flag_bits   bit i%32 of word i/32 = flag of i at the current step
//   fid         compacted ids of the flagged particles (nF of them)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <tuple>

#include "lvb.h"
#include "lvb_mlp.h"

#include <cuda_bf16.h>

namespace lvb {

// sticky device error bits
enum : unsigned { DERR_NAN = 1u, DERR_CELL = 2u, DERR_STORE = 4u, DERR_SYNC = 8u };

// slots of the trace: phases of the step kernel, then separate kernels
enum TraceSlot {
    TR_CHECK = 0, TR_REBUILD, TR_RELAYOUT, TR_TAIL, TR_INTEGRATE, TR_FORCES, TR_ROWS,
    TR_ITEMS, TR_ITEM_MAX,
    kTraceSlots = 16
};

struct DevCounters {
    int nF;            // flagged at the last step (final)
    int nF_acc[2];     // flagged count while the check runs (slot: step parity)
    int ovf[2];        // a row outgrew its capacity (slot: step parity)
    int row_overflow;  // same, for the separate full-build kernels
    int force_relayout;  // the next step that rebuilds rows re-lays them out (test hook)
    unsigned err;      // sticky DERR_* bits
    int last_flagged;
    int last_updated;
    unsigned long long bar_cnt[2];  // grid-barrier arrivals in the step kernel, by step parity
    long long steps;
    long long rebuild_steps;
    long long flagged_total;
    long long updated_total;
    long long relayouts;
    long long store_needed;  // entries the row store needed at the last layout
    unsigned long long kernels;  // kernels of this library executed (device count)
    unsigned long long barriers; // grid barriers passed by step kernels
    long long log_n;         // rebuild-log samples closed so far
    // work of the partial rebuilds so far (for the algorithmic byte count):
    // stencil candidates read, flagged-list records read by the direct
    // test, and edits (removals + insertions) of unflagged partners' rows
    unsigned long long alg_cand, alg_direct, alg_edits;
    // per-phase / per-kernel device time (LVB_OPT_TRACE): sums over steps;
    // separate kernels record first block entry / last block exit first
    unsigned long long tr_start[kTraceSlots], tr_end[kTraceSlots];
    unsigned long long tr_sum[kTraceSlots], tr_cnt[kTraceSlots];
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Geometry of one scene (a context holds one or many independent scenes,
// each a contiguous range of particles with its own box and cell grid).
struct SceneGeom {
    float lo[3];    // box lower corner (origin of the cell grid)
    float invL;     // 1 / L, rounded to binary32
    float hi[3];    // box upper corner
    float H;        // cap on R_NL = r + skin (just under L/2)
    int dim[3];     // cells per axis
    int cell_base;  // first global cell index of the scene
    float L;        // cell edge
    int first;      // first particle
    int count;      // particles
    int pad;
};

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// The fixed binary32 formula.  Explicit _rn intrinsics: nvcc never fuses them
// into FMAs, so every product and sum rounds exactly as written.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float sqdist_rn(float ax, float ay, float az,
                                           float bx, float by, float bz)
{
    float dx = __fsub_rn(ax, bx);
    float dy = __fsub_rn(ay, by);
    float dz = __fsub_rn(az, bz);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// Eq. update: |x - xref|^2 > skin^2
__device__ __forceinline__ bool violates(float4 p, float4 q)
{
    float d2 = sqdist_rn(p.x, p.y, p.z, q.x, q.y, q.z);
    return d2 > __fmul_rn(q.w, q.w);
}

// Def. verletlist on reference positions; a.w, b.w hold R_NL = r + skin.
__device__ __forceinline__ bool pair_hit(float4 a, float4 b)
{
    float c = __fadd_rn(a.w, b.w);
    float d2 = sqdist_rn(a.x, a.y, a.z, b.x, b.y, b.z);
    return d2 <= __fmul_rn(c, c);
}

// Eq. delta in binary32 with the correctly rounded square root.
__device__ __forceinline__ float overlap_rn(float4 a, float4 b)
{
    float R = __fadd_rn(a.w, b.w);
    float d2 = sqdist_rn(a.x, a.y, a.z, b.x, b.y, b.z);
    return __fsub_rn(R, __fsqrt_rn(d2));
}

// Skin policy, then the cap r + skin <= H (Eq. skin_formulus_mincell as
// R_NL bounded by half a cell).  kind: LVB_SKIN_*.
__device__ __forceinline__ float skin_of(int kind, float value, float dt, float H, float r,
                                         float4 v, float proposal)
{
    float s;
    if (kind == LVB_SKIN_GLOBAL) {
        s = value;
    } else if (kind == LVB_SKIN_DIAMETER_FACTOR) {
        s = __fmul_rn(value, __fmul_rn(2.0f, r));
    } else if (kind == LVB_SKIN_PAPER_KVDT) {
        float v2 = __fadd_rn(__fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y)),
                             __fmul_rn(v.z, v.z));
        s = __fmul_rn(__fmul_rn(value, __fsqrt_rn(v2)), dt);
    } else {
        s = proposal;
    }
    float capv = __fsub_rn(H, r);
    if (!(capv > 0.0f)) capv = 0.0f;
    if (!(s >= 0.0f)) s = 0.0f;
    if (s > capv) s = capv;
    return s;
}

__device__ __forceinline__ int cell_coord(float x, float lo, float invL, int dim)
{
    float u = __fmul_rn(__fsub_rn(x, lo), invL);
    u = fminf(fmaxf(u, -1.0f), (float)dim);   // NaN -> -1 (NaN is reported apart)
    int c = (int)floorf(u);
    return min(max(c, 0), dim - 1);
}

// global cell index of a point in scene g
__device__ __forceinline__ int cell_key(const SceneGeom &g, float x, float y, float z)
{
    int cx = cell_coord(x, g.lo[0], g.invL, g.dim[0]);
    int cy = cell_coord(y, g.lo[1], g.invL, g.dim[1]);
    int cz = cell_coord(z, g.lo[2], g.invL, g.dim[2]);
    return g.cell_base + (cz * g.dim[1] + cy) * g.dim[0] + cx;
}

__device__ __forceinline__ bool bit_of(const uint32_t *bits, int i)
{
    return (bits[i >> 5] >> (i & 31)) & 1u;
}

__device__ __forceinline__ int warp_incl_scan(int v)
{
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------------------
// The skin network (lvb_mlp.h), one warp per particle: lane o computes hidden
// unit o of each layer (its weights of input k are one coalesced line for
// the warp, the layout being input-major); every sum runs in index order
// from its bias, so the result is the same on every lane and equal to the
// CPU evaluation.  The weights hold bfloat16 values, so fmaf(w, x, acc) =
// acc + w*x rounded once.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float bf16_rn(float x)
{
    return __bfloat162float(__float2bfloat16_rn(x));
}

__device__ __forceinline__ float relu(float x) { return x > 0.0f ? x : 0.0f; }

__device__ __forceinline__ float mlp_y_warp(const lvb_mlp_weights *__restrict__ W,
                                            const float f[LVB_MLP_IN])
{
    const int lane = threadIdx.x & 31;
    float z[LVB_MLP_IN];
#pragma unroll
    for (int k = 0; k < LVB_MLP_IN; ++k)
        z[k] = bf16_rn(__fmul_rn(__fsub_rn(f[k], W->mu[k]), W->isd[k]));
    float acc = W->b1[lane];
#pragma unroll
    for (int k = 0; k < LVB_MLP_IN; ++k) acc = fmaf(W->W1[k * LVB_MLP_HIDDEN + lane], z[k], acc);
    const float h1 = bf16_rn(relu(acc));
    // unrolled by 8 only: enough loads in flight, and few registers held
    // (the step kernel's callers run at 64 registers a thread)
    float acc2 = W->b2[lane];
#pragma unroll 8
    for (int k = 0; k < LVB_MLP_HIDDEN; ++k)
        acc2 = fmaf(W->W2[k * LVB_MLP_HIDDEN + lane], __shfl_sync(FULL, h1, k), acc2);
    const float h2 = bf16_rn(relu(acc2));
    float y = W->b3;
#pragma unroll 8
    for (int k = 0; k < LVB_MLP_HIDDEN; ++k) y = fmaf(W->w3[k], __shfl_sync(FULL, h2, k), y);
    return y;
}

// The network's skin proposal from its output y for a particle of diameter
// d with travel feature f0 (lvb_mlp.h): diameter form (y_steps = 0) or
// travel form, each product rounded once in the header's order.
__device__ __forceinline__ float mlp_skin(const lvb_mlp_weights *__restrict__ W, float y, float d,
                                          float f0)
{
    const float yc = fminf(fmaxf(y, W->y_lo), W->y_hi);
    const float u = W->y_steps > 0.0f ? __fmul_rn(f0, __fmul_rn(yc, W->y_steps)) : yc;
    return __fmul_rn(d, u);
}

// Slack rule of the row store: capacity for a row of `len` entries (room
// for the row to grow by half, and by 8 however short it is, before the
// store is re-laid out).
__host__ __device__ __forceinline__ int row_capacity(int len)
{
    return len + 8 + (len >> 1);
}

}  // namespace lvb

// Library-internal view of a broad-phase context's rows (used by the DEM
// driver in the same library; not part of the C-ABI).
namespace lvb {
// Velocity-Verlet position half-step of the DEM driver, shared by its own
// integrate kernel and by the check kernel that fuses it (identical
// arithmetic either way: explicit roundings, no compiler-chosen fusion):
//   x' = x + (v dt + a dt^2/2),  v* = v + a dt   (v*.w keeps 1/m)
// with specular reflection at the scene box when `specular` (x mirrored, v
// and v* negated per axis).
struct IntegrateArgs {
    float4 *pos, *vel, *acc, *vstar;
    float4 *omega, *alpha, *wstar;   // rotation (friction), or null
    float dt, half_dt2;
    int specular;
    int active;     // 0: the check reads positions as they are
};

// kStream (the integrator as a kernel of its own): the old state is read
// with streaming loads (evict first), so that the L2 keeps the new
// positions this kernel writes for the broad phase that follows; inside the
// fused step (kStream false) the forces tail reads v and a again.
template <bool kStream = false>
__device__ __forceinline__ float4 integrate_one(const IntegrateArgs &a, const SceneGeom &g, int i)
{
    float4 x = kStream ? __ldcs(a.pos + i) : a.pos[i];
    float4 v = kStream ? __ldcs(a.vel + i) : a.vel[i];
    const float4 ac = kStream ? __ldcs(a.acc + i) : a.acc[i];
    const float im = v.w;   // the driver keeps 1 / m in v.w (and v*.w)
    x.x = __fadd_rn(x.x, fmaf(ac.x, a.half_dt2, __fmul_rn(v.x, a.dt)));
    x.y = __fadd_rn(x.y, fmaf(ac.y, a.half_dt2, __fmul_rn(v.y, a.dt)));
    x.z = __fadd_rn(x.z, fmaf(ac.z, a.half_dt2, __fmul_rn(v.z, a.dt)));
    float4 vs = make_float4(fmaf(ac.x, a.dt, v.x), fmaf(ac.y, a.dt, v.y), fmaf(ac.z, a.dt, v.z), im);
    if (a.specular) {
        const float r = x.w;
        float lo = __fadd_rn(g.lo[0], r), hi = __fsub_rn(g.hi[0], r);
        if (x.x < lo || x.x > hi) {
            x.x = __fsub_rn(__fmul_rn(2.0f, x.x < lo ? lo : hi), x.x); v.x = -v.x; vs.x = -vs.x;
        }
        lo = __fadd_rn(g.lo[1], r); hi = __fsub_rn(g.hi[1], r);
        if (x.y < lo || x.y > hi) {
            x.y = __fsub_rn(__fmul_rn(2.0f, x.y < lo ? lo : hi), x.y); v.y = -v.y; vs.y = -vs.y;
        }
        lo = __fadd_rn(g.lo[2], r); hi = __fsub_rn(g.hi[2], r);
        if (x.z < lo || x.z > hi) {
            x.z = __fsub_rn(__fmul_rn(2.0f, x.z < lo ? lo : hi), x.z); v.z = -v.z; vs.z = -vs.z;
        }
        a.vel[i] = v;
    }
    a.pos[i] = x;
    a.vstar[i] = vs;
    if (a.omega) {   // w* = w + al dt (w*.w keeps 1/I)
        const float4 w = a.omega[i], al = a.alpha[i];
        a.wstar[i] = make_float4(fmaf(al.x, a.dt, w.x), fmaf(al.y, a.dt, w.y),
                                 fmaf(al.z, a.dt, w.z), w.w);
    }
    return x;
}

struct DevState;

struct RowsView {
    const int *row_off;
    const int *row_len;
    const int *row_cap;
    const int *col;
    float4 *hist;                  // contact history beside col, or null
    const float *rad;
    unsigned long long *kernels;   // device kernel counter of the context
    DevCounters *cnt;              // counters (trace slots)
    const int *trace;              // host address of the trace switch
    const SceneGeom *sg;           // per-scene geometry (device)
    const int *scene_of;           // scene of each particle (null: one scene)
    int nscenes;
    int n;
};
RowsView rows_view(lvb_ctx *c);

// The device state a step kernel takes by value, and the launch shape of
// the step kernel (blocks: all co-resident; threads per block).
DevState step_state(lvb_ctx *c);
void step_shape(lvb_ctx *c, int *blocks, int *threads);
cudaStream_t step_stream(lvb_ctx *c);
// The context's small device scratch (at least 8 words and one 64-bit
// word), used on its stream by calls that synchronise before returning.
void small_scratch(lvb_ctx *c, unsigned **u32, unsigned long long **u64);

// Changes whenever the step kernel's arguments change (options, logging,
// store growth), so that a caller holding a graph of steps knows to rebuild
// it.
int graph_version(lvb_ctx *c);

// Grows the row store / cell slots if a kernel asked for it (see lvb_step).
int grow_stores_if_asked(lvb_ctx *c);

// Adds a kernel node running fn(args...) after the given dependency (none
// when dep or *dep is null); the argument values are copied into the node.
// add_coop_kernel adds a cooperative one (all blocks resident at once).
template <typename... P, typename... A>
cudaError_t add_kernel(cudaGraphNode_t *out, cudaGraph_t g, const cudaGraphNode_t *dep,
                       void (*fn)(P...), dim3 grid, dim3 block, A... args);

template <typename... P, typename... A>
cudaError_t add_coop_kernel(cudaGraphNode_t *out, cudaGraph_t g, const cudaGraphNode_t *dep,
                            void (*fn)(P...), dim3 grid, dim3 block, A... args)
{
    cudaError_t e = add_kernel(out, g, dep, fn, grid, block, args...);
    if (e != cudaSuccess) return e;
    cudaLaunchAttributeValue v = {};
    v.cooperative = 1;
    return cudaGraphKernelNodeSetAttribute(*out, cudaLaunchAttributeCooperative, &v);
}

// Launches fn(args...) cooperatively on `stream` with `smem` bytes of
// dynamic shared memory.
template <typename... P, typename... A>
cudaError_t launch_coop(void (*fn)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                        A... args)
{
    static_assert(sizeof...(P) == sizeof...(A), "argument count");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, static_cast<P>(args)...);
}

template <typename... P, typename... A>
cudaError_t add_kernel(cudaGraphNode_t *out, cudaGraph_t g, const cudaGraphNode_t *dep,
                       void (*fn)(P...), dim3 grid, dim3 block, A... args)
{
    static_assert(sizeof...(P) == sizeof...(A), "argument count");
    std::tuple<P...> vals(args...);
    void *ptrs[sizeof...(P) > 0 ? sizeof...(P) : 1];
    std::apply([&](auto &...v) {
        int k = 0;
        ((ptrs[k++] = (void *)&v), ...);
    }, vals);
    cudaKernelNodeParams p = {};
    p.func = (void *)fn;
    p.gridDim = grid;
    p.blockDim = block;
    p.sharedMemBytes = 0;
    p.kernelParams = ptrs;
    p.extra = nullptr;
    return cudaGraphAddKernelNode(out, g, dep && *dep ? dep : nullptr, dep && *dep ? 1 : 0, &p);
}
}  // namespace lvb
