// clumps.cu -- narrow phase of multi-sphere clumps on the list
// (include/lvb_clump.h): the broad phase runs on the clumps' bounding
// spheres, and every clump pair of its list is resolved into the contacts
// of their sub-spheres, each at its world position x_i + R(q_i) b_a.
#include "lvb_internal.cuh"
#include "lvb_clump.h"

#include <algorithm>
#include <cmath>

using namespace lvb;

namespace {

constexpr int kThreads = 256;
constexpr int kMaxSub = 64;

enum : unsigned { CL_BAD_QUAT = 1u, CL_BAD_BOUND = 2u, CL_BAD_OFFSETS = 4u, CL_BAD_VALUE = 8u };

// The rotation matrix of a unit quaternion (w, x, y, z), each entry in
// binary32 with the roundings of lvb_clump.h.
__device__ __forceinline__ void rotmat(float4 q, float R[9])
{
    const float w = q.x, x = q.y, y = q.z, z = q.w;
    R[0] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(__fmul_rn(y, y), __fmul_rn(z, z))));
    R[1] = __fmul_rn(2.0f, __fsub_rn(__fmul_rn(x, y), __fmul_rn(w, z)));
    R[2] = __fmul_rn(2.0f, __fadd_rn(__fmul_rn(x, z), __fmul_rn(w, y)));
    R[3] = __fmul_rn(2.0f, __fadd_rn(__fmul_rn(x, y), __fmul_rn(w, z)));
    R[4] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(__fmul_rn(x, x), __fmul_rn(z, z))));
    R[5] = __fmul_rn(2.0f, __fsub_rn(__fmul_rn(y, z), __fmul_rn(w, x)));
    R[6] = __fmul_rn(2.0f, __fsub_rn(__fmul_rn(x, z), __fmul_rn(w, y)));
    R[7] = __fmul_rn(2.0f, __fadd_rn(__fmul_rn(y, z), __fmul_rn(w, x)));
    R[8] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y))));
}

// World position and radius of a sub-sphere (b: body offset and radius).
__device__ __forceinline__ float4 world(float4 c, const float R[9], float4 b)
{
    float4 o;
    o.x = __fadd_rn(c.x, __fadd_rn(__fadd_rn(__fmul_rn(R[0], b.x), __fmul_rn(R[1], b.y)),
                                   __fmul_rn(R[2], b.z)));
    o.y = __fadd_rn(c.y, __fadd_rn(__fadd_rn(__fmul_rn(R[3], b.x), __fmul_rn(R[4], b.y)),
                                   __fmul_rn(R[5], b.z)));
    o.z = __fadd_rn(c.z, __fadd_rn(__fadd_rn(__fmul_rn(R[6], b.x), __fmul_rn(R[7], b.y)),
                                   __fmul_rn(R[8], b.z)));
    o.w = b.w;
    return o;
}

// Input checks, one thread per clump.
__global__ void __launch_bounds__(kThreads)
k_clump_check(int n, const float4 *__restrict__ pos, const float4 *__restrict__ quat,
              const int *__restrict__ off, const float4 *__restrict__ sub, unsigned *bad)
{
    unsigned b = 0;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        const float4 q = quat[i];
        const double qq = (double)q.x * q.x + (double)q.y * q.y + (double)q.z * q.z +
                          (double)q.w * q.w;
        if (!(fabs(qq - 1.0) <= 1.0 / 524288.0)) b |= CL_BAD_QUAT;
        const int a0 = off[i], a1 = off[i + 1];
        if (a0 < 0 || !(a1 > a0) || a1 - a0 > kMaxSub) {
            b |= CL_BAD_OFFSETS;
            continue;
        }
        const double R = pos[i].w;
        if (!(R > 0.0) || !isfinite(pos[i].x) || !isfinite(pos[i].y) || !isfinite(pos[i].z))
            b |= CL_BAD_VALUE;
        for (int a = a0; a < a1; ++a) {
            const float4 s = sub[a];
            if (!(s.w > 0.0f) || !isfinite(s.x) || !isfinite(s.y) || !isfinite(s.z)) {
                b |= CL_BAD_VALUE;
                continue;
            }
            const double nb = sqrt((double)s.x * s.x + (double)s.y * s.y + (double)s.z * s.z);
            if (!(nb + (double)s.w <= R * (1.0 - 1.0 / 4096.0))) b |= CL_BAD_BOUND;
        }
    }
    if (b) atomicOr(bad, b);
}

// One thread per clump i: every partner j > i of its row, every pair of
// their sub-spheres.
__global__ void __launch_bounds__(kThreads)
k_clump_contacts(RowsView rv, const float4 *__restrict__ pos, const float4 *__restrict__ quat,
                 const int *__restrict__ off, const float4 *__restrict__ sub,
                 unsigned long long *cnt, long long cap, int *ci, int *ca, int *cj, int *cb,
                 float *delta)
{
    const int i = blockIdx.x * kThreads + threadIdx.x;
    if (i == 0) atomicAdd(rv.kernels, 1ULL);
    if (i >= rv.n) return;
    float Ri[9], Rj[9];
    const float4 xi = pos[i];
    rotmat(quat[i], Ri);
    const int i0 = off[i], i1 = off[i + 1];
    const int roff = rv.row_off[i], rlen = min(rv.row_len[i], rv.row_cap[i]);
    for (int e = 0; e < rlen; ++e) {
        const int j = rv.col[roff + e];
        if (j <= i) continue;      // a removed pair's slot, or the pair from j's row
        const float4 xj = pos[j];
        rotmat(quat[j], Rj);
        const int j0 = off[j], j1 = off[j + 1];
        for (int a = i0; a < i1; ++a) {
            const float4 wa = world(xi, Ri, sub[a]);
            for (int b = j0; b < j1; ++b) {
                const float4 wb = world(xj, Rj, sub[b]);
                const float dl = overlap_rn(wa, wb);
                if (!(dl > 0.0f)) continue;
                const unsigned long long k = atomicAdd(cnt, 1ULL);
                if (k < (unsigned long long)cap) {
                    ci[k] = i;
                    ca[k] = a - i0;
                    cj[k] = j;
                    cb[k] = b - j0;
                    delta[k] = dl;
                }
            }
        }
    }
}

int from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return LVB_OK;
    if (e == cudaErrorMemoryAllocation) return LVB_ENOMEM;
    return LVB_EDEVICE;
}

bool on_device(const void *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // an unknown pointer: host memory
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int lvb_clump_contacts(lvb_ctx *ctx, const float *pos_r, const float *quat,
                                  const int32_t *sub_off, const float *sub, int32_t *ci,
                                  int32_t *ca, int32_t *cj, int32_t *cb, float *delta,
                                  int64_t cap, int64_t *n_contacts)
{
    if (!ctx || !pos_r || !quat || !sub_off || !sub || !n_contacts || cap < 0 ||
        (cap > 0 && (!ci || !ca || !cj || !cb || !delta)))
        return LVB_EINVAL;
    if (((uintptr_t)pos_r & 15u) || ((uintptr_t)quat & 15u) || ((uintptr_t)sub & 15u))
        return LVB_EINVAL;
    *n_contacts = 0;
    int rc = lvb_sync(ctx);       // the list must be valid (sticky errors)
    if (rc) return rc;
    const RowsView rv = rows_view(ctx);
    const cudaStream_t st = step_stream(ctx);
    const int n = rv.n;
    unsigned *bad = nullptr;
    unsigned long long *cnt = nullptr;
    small_scratch(ctx, &bad, &cnt);
    // outputs in device memory are written by the kernel in place; any
    // output in host memory sends all five through device temporaries
    bool direct = true;
    if (cap > 0) {
        const void *outs[5] = {ci, ca, cj, cb, delta};
        for (const void *p : outs) direct = direct && on_device(p);
    }
    const long long cp = std::max<long long>(cap, 1);
    int *di = nullptr, *da = nullptr, *dj = nullptr, *db = nullptr;
    float *dd = nullptr;
    auto done = [&](int code) {
        cudaStreamSynchronize(st);
        if (!direct) {
            cudaFree(di);
            cudaFree(da);
            cudaFree(dj);
            cudaFree(db);
            cudaFree(dd);
        }
        return code;
    };
    cudaError_t e = cudaSuccess;
    if (direct) {
        di = ci;
        da = ca;
        dj = cj;
        db = cb;
        dd = delta;
    } else {
        e = cudaMalloc((void **)&di, sizeof(int) * cp);
        if (e == cudaSuccess) e = cudaMalloc((void **)&da, sizeof(int) * cp);
        if (e == cudaSuccess) e = cudaMalloc((void **)&dj, sizeof(int) * cp);
        if (e == cudaSuccess) e = cudaMalloc((void **)&db, sizeof(int) * cp);
        if (e == cudaSuccess) e = cudaMalloc((void **)&dd, sizeof(float) * cp);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return done(from_cuda(e));
    const int grid = std::min((n + kThreads - 1) / kThreads, 4 * 152);
    k_clump_check<<<grid, kThreads, 0, st>>>(n, (const float4 *)pos_r, (const float4 *)quat,
                                             sub_off, (const float4 *)sub, bad);
    unsigned hbad = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return done(from_cuda(e));
    if (hbad) return done(LVB_EINVAL);
    k_clump_contacts<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(
        rv, (const float4 *)pos_r, (const float4 *)quat, sub_off, (const float4 *)sub, cnt, cap,
        di, da, dj, db, dd);
    unsigned long long total = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&total, cnt, sizeof(total), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return done(from_cuda(e));
    const long long m = std::min<long long>((long long)total, cap);
    if (!direct && m > 0) {
        int32_t *outs[4] = {ci, ca, cj, cb};
        int *srcs[4] = {di, da, dj, db};
        for (int k = 0; k < 4 && e == cudaSuccess; ++k)
            e = cudaMemcpyAsync(outs[k], srcs[k], sizeof(int) * m, cudaMemcpyDefault, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(delta, dd, sizeof(float) * m, cudaMemcpyDefault, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return done(from_cuda(e));
    }
    *n_contacts = (int64_t)total;
    return done((long long)total > cap ? LVB_ECAPACITY : LVB_OK);
}
