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

namespace lvb {

// sticky device error bits
enum : unsigned { DERR_NAN = 1u, DERR_CELL = 2u, DERR_STORE = 4u };

struct DevCounters {
    int nF;            // flagged at this step (final, set by the check's last block)
    int ntrow;         // rows touched by removals this step
    int ntcell;        // cells touched by removals this step
    int row_overflow;  // some row exceeded its capacity this step
    unsigned err;      // sticky DERR_* bits
    int last_flagged;
    int last_updated;
    int nF_accum;      // running count while the check kernel's blocks compact
    unsigned done_blocks;  // check blocks finished (last-block detection)
    int pad0;
    long long steps;
    long long rebuild_steps;
    long long flagged_total;
    long long updated_total;
    long long relayouts;
    long long store_needed;  // entries the row store needed at the last layout
    unsigned long long kernels;  // kernels of this library executed (device count)
    long long small_steps;   // steps whose rebuild ran in the one-block kernel
};

struct GridGeom {
    float lo[3];
    float invL;     // 1 / L, rounded to binary32
    int dim[3];     // cells per axis
    int ccap;       // slots per cell
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

__device__ __forceinline__ int cell_key(const GridGeom &g, float x, float y, float z)
{
    int cx = cell_coord(x, g.lo[0], g.invL, g.dim[0]);
    int cy = cell_coord(y, g.lo[1], g.invL, g.dim[1]);
    int cz = cell_coord(z, g.lo[2], g.invL, g.dim[2]);
    return (cz * g.dim[1] + cy) * g.dim[0] + cx;
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

// Slack rule of the row store: capacity for a row of `len` entries.
__host__ __device__ __forceinline__ int row_capacity(int len)
{
    return len + 4 + (len >> 2);
}

}  // namespace lvb

// Library-internal view of a broad-phase context's rows (used by the DEM
// driver in the same library; not part of the C-ABI).
namespace lvb {
struct RowsView {
    const int *row_off;
    const int *row_len;
    const int *row_cap;
    const int *col;
    const float *rad;
    unsigned long long *kernels;   // device kernel counter of the context
    int n;
};
RowsView rows_view(lvb_ctx *c);

// Appends the nodes of one lvb_step (check, conditional rebuild, conditional
// re-layout) to graph g after *dep (may be null); *dep receives the last node.
int append_step_nodes(lvb_ctx *c, cudaGraph_t g, cudaGraphNode_t *dep, const float *pos_r,
                      const float *vel);

// Adds a kernel node running fn(args...) after the given dependency (none
// when dep or *dep is null); the argument values are copied into the node.
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
