// noalloc.cu -- lvb_pairs_noalloc: the neighbour list of one reference
// state (Def. verletlist), built without allocating any memory.
//
// Which callers cannot allocate, and why: code that runs inside another
// framework's memory budget (a caching allocator that owns the device heap
// and would be bypassed or fragmented by a cudaMalloc), a plug-in or
// callback that must not change the process's memory footprint, or a
// long-running loop where an allocation may neither fail nor stall half-way
// through.  Such a caller brings only its input and output buffers.  The
// working memory -- cell counts and offsets, and the particles' reference
// records sorted by cell -- lives in one file-scope device array of fixed
// size (about 1.6 MB), which the library's module holds on every device it
// is loaded on until the process exits.  A context (lvb_init) does the same
// job without these limits and keeps its list up to date step by step; this
// call is one-shot.
//
// The list equals the one a context holds for the same reference state: the
// same fixed binary32 test (|xref_i - xref_j|^2 <= (R_NL,i + R_NL,j)^2 with
// R_NL = r + skin), the same pair set, in no particular order.
#include "lvb_internal.cuh"
#include "lvb_noalloc.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>

using namespace lvb;

namespace {

constexpr int kNaMaxN = 1 << 16;       // particles one call takes (LVB_NOALLOC_MAX_N)
constexpr int kNaMaxCells = 1 << 15;   // cells of the grid; coarser cells if needed
constexpr int kNaThreads = 256;
constexpr int kNaBlocks = 4 * 152;     // grid-stride launches: 4 blocks per SM

enum : unsigned { NA_BAD_NONFINITE = 1u, NA_BAD_NEGATIVE = 2u };

struct NaScratch {
    int cell_cnt[kNaMaxCells];         // particles per cell, then fill cursors
    int cell_start[kNaMaxCells + 1];   // exclusive prefix sums of the counts
    int ids[kNaMaxN];                  // particle ids in cell order
    float4 sref[kNaMaxN];              // (xref, yref, zref, R_NL) in cell order
    unsigned long long npairs;         // pairs found, including any beyond cap
    unsigned rnl_max_bits;             // largest R_NL (bits of a float >= 0)
    unsigned bad;                      // NA_BAD_* seen in the input
};

// The scratch: one per device, shared by every call on that device.  Its
// counters and cell counts are zeroed by each call before use, so no state
// carries from one call to the next.
static __device__ __align__(256) NaScratch g_na_scratch;

struct NaGrid {
    float lo[3];
    float invL;
    int dim[3];
    int ncells;
};

__device__ __forceinline__ int na_key(const NaGrid &g, float x, float y, float z)
{
    const int cx = cell_coord(x, g.lo[0], g.invL, g.dim[0]);
    const int cy = cell_coord(y, g.lo[1], g.invL, g.dim[1]);
    const int cz = cell_coord(z, g.lo[2], g.invL, g.dim[2]);
    return (cz * g.dim[1] + cy) * g.dim[0] + cx;
}

__device__ __forceinline__ float na_rnl(const float4 *pos4, const float4 &q, int i)
{
    return __fadd_rn(pos4[i].w, q.w);
}

__global__ void k_na_reset(NaScratch *sc)
{
    sc->npairs = 0ULL;
    sc->rnl_max_bits = 0u;
    sc->bad = 0u;
}

// Largest R_NL (sizes the cells) and input checks.
__global__ void __launch_bounds__(kNaThreads)
k_na_extent(NaScratch *sc, const float4 *__restrict__ ref4, const float4 *__restrict__ pos4, int n)
{
    unsigned bad = 0u, mx = 0u;
    for (int i = blockIdx.x * kNaThreads + threadIdx.x; i < n; i += gridDim.x * kNaThreads) {
        const float4 q = ref4[i];
        const float r = pos4[i].w;
        const float rnl = __fadd_rn(r, q.w);
        if (!(isfinite(q.x) && isfinite(q.y) && isfinite(q.z) && isfinite(r) && isfinite(q.w) &&
              isfinite(rnl)))
            bad |= NA_BAD_NONFINITE;
        else if (!(r > 0.0f) || !(q.w >= 0.0f))
            bad |= NA_BAD_NEGATIVE;
        else
            mx = max(mx, __float_as_uint(rnl));   // rnl > 0: bit order is value order
    }
    if (bad) atomicOr(&sc->bad, bad);
    if (mx) atomicMax(&sc->rnl_max_bits, mx);
}

__global__ void __launch_bounds__(kNaThreads) k_na_clear(NaScratch *sc, int ncells)
{
    for (int c = blockIdx.x * kNaThreads + threadIdx.x; c < ncells; c += gridDim.x * kNaThreads)
        sc->cell_cnt[c] = 0;
}

__global__ void __launch_bounds__(kNaThreads)
k_na_count(NaScratch *sc, const float4 *__restrict__ ref4, int n, NaGrid g)
{
    for (int i = blockIdx.x * kNaThreads + threadIdx.x; i < n; i += gridDim.x * kNaThreads) {
        const float4 q = ref4[i];
        atomicAdd(&sc->cell_cnt[na_key(g, q.x, q.y, q.z)], 1);
    }
}

// One block: exclusive scan of the counts into cell_start (each thread owns
// a contiguous run of cells); the counts become zeroed fill cursors.
__global__ void __launch_bounds__(kNaThreads) k_na_scan(NaScratch *sc, int ncells)
{
    __shared__ int part[kNaThreads];
    const int t = threadIdx.x;
    const int per = (ncells + kNaThreads - 1) / kNaThreads;
    const int a = min(t * per, ncells), b = min(a + per, ncells);
    int sum = 0;
    for (int c = a; c < b; ++c) sum += sc->cell_cnt[c];
    part[t] = sum;
    __syncthreads();
    if (t == 0) {
        int run = 0;
        for (int k = 0; k < kNaThreads; ++k) {
            const int v = part[k];
            part[k] = run;
            run += v;
        }
        sc->cell_start[ncells] = run;
    }
    __syncthreads();
    int run = part[t];
    for (int c = a; c < b; ++c) {
        sc->cell_start[c] = run;
        run += sc->cell_cnt[c];
        sc->cell_cnt[c] = 0;
    }
}

__global__ void __launch_bounds__(kNaThreads)
k_na_fill(NaScratch *sc, const float4 *__restrict__ ref4, const float4 *__restrict__ pos4, int n,
          NaGrid g)
{
    for (int i = blockIdx.x * kNaThreads + threadIdx.x; i < n; i += gridDim.x * kNaThreads) {
        const float4 q = ref4[i];
        const int c = na_key(g, q.x, q.y, q.z);
        const int k = sc->cell_start[c] + atomicAdd(&sc->cell_cnt[c], 1);
        sc->ids[k] = i;
        sc->sref[k] = make_float4(q.x, q.y, q.z, na_rnl(pos4, q, i));
    }
}

// One warp per particle i: lane c < 27 owns one cell of the 3x3x3 stencil
// around i's cell; the warp walks the concatenated cell runs 32 candidates at
// a time and keeps the partners j > i that pass the test of Def. verletlist.
__global__ void __launch_bounds__(kNaThreads)
k_na_pairs(NaScratch *sc, const float4 *__restrict__ ref4, const float4 *__restrict__ pos4, int n,
           NaGrid g, int *__restrict__ pi, int *__restrict__ pj, long long cap)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const int nw = (gridDim.x * kNaThreads) >> 5;
    for (int i = (blockIdx.x * kNaThreads + threadIdx.x) >> 5; i < n; i += nw) {
        const float4 q = ref4[i];
        const float4 qi = make_float4(q.x, q.y, q.z, na_rnl(pos4, q, i));
        const int cx = cell_coord(q.x, g.lo[0], g.invL, g.dim[0]);
        const int cy = cell_coord(q.y, g.lo[1], g.invL, g.dim[1]);
        const int cz = cell_coord(q.z, g.lo[2], g.invL, g.dim[2]);
        int cnt = 0, first = 0;
        if (lane < 27) {
            const int x = cx + lane % 3 - 1, y = cy + (lane / 3) % 3 - 1, z = cz + lane / 9 - 1;
            if (x >= 0 && x < g.dim[0] && y >= 0 && y < g.dim[1] && z >= 0 && z < g.dim[2]) {
                const int c = (z * g.dim[1] + y) * g.dim[0] + x;
                first = sc->cell_start[c];
                cnt = sc->cell_start[c + 1] - first;
            }
        }
        const int incl = warp_incl_scan(cnt);
        const int excl = incl - cnt;
        const int total = __shfl_sync(FULL, incl, 31);
        for (int b0 = 0; b0 < total; b0 += 32) {
            const int k = b0 + lane;
            // stencil cell of candidate k: the number of cells whose
            // inclusive end is <= k (binary search over the 32 lanes)
            int c = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1)
                c += (__shfl_sync(FULL, incl, c + step - 1) <= k) ? step : 0;
            const int f = __shfl_sync(FULL, first, c & 31);
            const int ex = __shfl_sync(FULL, excl, c & 31);
            bool hit = false;
            int j = -1;
            if (k < total) {
                const int slot = f + (k - ex);
                j = sc->ids[slot];
                hit = j > i && pair_hit(qi, sc->sref[slot]);
            }
            const unsigned m = __ballot_sync(FULL, hit);
            if (m) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(&sc->npairs, (unsigned long long)__popc(m));
                base = __shfl_sync(FULL, base, 0);
                if (hit) {
                    const unsigned long long o = base + __popc(m & lt);
                    if (o < (unsigned long long)cap) {
                        pi[o] = i;
                        pj[o] = j;
                    }
                }
            }
        }
    }
}

// Launches fn<<<grid, threads, 0, st>>>(args...) and returns the launch's
// own status (cudaLaunchKernelEx reports it directly), so that no call here
// needs cudaGetLastError -- which would also read and clear an error of the
// caller's own earlier work that the caller has not yet collected.
template <typename... P, typename... A>
cudaError_t na_launch(void (*fn)(P...), int grid, int threads, cudaStream_t st, A... args)
{
    static_assert(sizeof...(P) == sizeof...(A), "argument count");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = nullptr;
    cfg.numAttrs = 0;
    return cudaLaunchKernelEx(&cfg, fn, static_cast<P>(args)...);
}

// Device address of the scratch, looked up once per device (with that
// device current) and kept for the life of the process.
constexpr int kNaMaxDevices = 64;
std::atomic<NaScratch *> g_na_addr[kNaMaxDevices];

int na_scratch(NaScratch **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return LVB_EDEVICE;
    NaScratch *p = g_na_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        void *a = nullptr;
        if (cudaGetSymbolAddress(&a, g_na_scratch) != cudaSuccess || !a) return LVB_EDEVICE;
        p = (NaScratch *)a;
        g_na_addr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return LVB_OK;
}

// Cell edge and grid: edges of at least 2 max R_NL (1 + 2^-7), so that any
// pair lies in neighbouring cells even after the binary32 rounding of a cell
// coordinate; widened by 1.25x until the grid has at most kNaMaxCells cells.
// Out-of-grid coordinates clamp to the border cells, which keeps neighbours
// neighbours.
NaGrid na_grid(const lvb_box &box, float rnl_max)
{
    NaGrid g;
    double L = 2.0 * (double)rnl_max * (1.0 + 1.0 / 128.0);
    double ext_max = 0.0;
    for (int k = 0; k < 3; ++k) ext_max = std::max(ext_max, (double)box.hi[k] - (double)box.lo[k]);
    L = std::max(L, ext_max / 2048.0);
    for (;;) {
        long long cells = 1;
        for (int k = 0; k < 3; ++k) {
            const double e = (double)box.hi[k] - (double)box.lo[k];
            g.dim[k] = (int)std::min(std::max(std::ceil(e / L), 1.0), 2048.0);
            cells *= g.dim[k];
        }
        if (cells <= kNaMaxCells) {
            g.ncells = (int)cells;
            break;
        }
        L *= 1.25;
    }
    for (int k = 0; k < 3; ++k) g.lo[k] = box.lo[k];
    g.invL = (float)(1.0 / L);
    return g;
}

}  // namespace

extern "C" {

int lvb_pairs_noalloc(int64_t n, const float *pos4, const float *ref4, const lvb_box *box,
                      int32_t *pi, int32_t *pj, int64_t cap, int64_t *n_pairs, void *stream)
{
    if (n_pairs) *n_pairs = 0;
    if (!pos4 || !ref4 || !box || !n_pairs || n < 1 || cap < 0 || (cap > 0 && (!pi || !pj)))
        return LVB_EINVAL;
    if (((uintptr_t)pos4 & 15u) || ((uintptr_t)ref4 & 15u)) return LVB_EINVAL;
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(box->lo[k]) || !std::isfinite(box->hi[k]) || !(box->hi[k] > box->lo[k]))
            return LVB_EINVAL;
    if (n > kNaMaxN) return LVB_ELIMIT;
    const cudaStream_t st = (cudaStream_t)stream;
    // the call synchronises its stream and reads results to the host, so
    // it cannot be captured into a graph: refuse before any launch
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return LVB_EINVAL;

    NaScratch *sc = nullptr;
    if (int rc = na_scratch(&sc)) return rc;
    const float4 *p4 = (const float4 *)pos4;
    const float4 *r4 = (const float4 *)ref4;
    const int nn = (int)n;
    const int grid = std::min((nn + kNaThreads - 1) / kNaThreads, kNaBlocks);

    cudaError_t e = na_launch(k_na_reset, 1, 1, st, sc);
    if (e == cudaSuccess) e = na_launch(k_na_extent, grid, kNaThreads, st, sc, r4, p4, nn);
    unsigned ext[2] = {0u, 0u};   // rnl_max_bits, bad (adjacent in NaScratch)
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ext, &sc->rnl_max_bits, sizeof(ext), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return LVB_EDEVICE;
    if (ext[1] & NA_BAD_NONFINITE) return LVB_ENAN;
    if (ext[1] & NA_BAD_NEGATIVE) return LVB_EINVAL;
    float rnl_max;
    memcpy(&rnl_max, &ext[0], sizeof(float));

    const NaGrid g = na_grid(*box, rnl_max);
    const int gc = std::min((g.ncells + kNaThreads - 1) / kNaThreads, kNaBlocks);
    const int gw = std::min((nn + 7) / 8, 4 * kNaBlocks);   // 8 warps (particles) per block
    e = na_launch(k_na_clear, gc, kNaThreads, st, sc, g.ncells);
    if (e == cudaSuccess) e = na_launch(k_na_count, grid, kNaThreads, st, sc, r4, nn, g);
    if (e == cudaSuccess) e = na_launch(k_na_scan, 1, kNaThreads, st, sc, g.ncells);
    if (e == cudaSuccess) e = na_launch(k_na_fill, grid, kNaThreads, st, sc, r4, p4, nn, g);
    if (e == cudaSuccess)
        e = na_launch(k_na_pairs, gw, kNaThreads, st, sc, r4, p4, nn, g, pi, pj, cap);
    unsigned long long np = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&np, &sc->npairs, sizeof(np), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return LVB_EDEVICE;
    *n_pairs = (int64_t)np;
    return (int64_t)np > cap ? LVB_ECAPACITY : LVB_OK;
}

}  // extern "C"
