// lvb_dem.cu -- DEM driver on the local Verlet buffer list (include/lvb_dem.h).
//
// Per step: position half-step (x', v*), the broad-phase step at x'
// (displacement check and partial rebuild), forces (narrow phase on the
// list rows, linear spring-dashpot, walls, a', v').  dem_advance runs each
// step as one cooperative launch of the broad phase's step kernel with the
// half-step fused into its check pass and the forces as its tail phase;
// dem_phase runs the three parts as separate launches (k_integrate,
// lvb_step, k_forces), with identical results.  Forces are accumulated per row of the
// symmetric list, so each pair is evaluated once from each side and no
// atomics are needed; both evaluations give exactly opposite forces.
//
// The overlap delta = r_i + r_j - |x_i - x_j| is a small difference of large
// numbers: at 0.3 m coordinates a binary32 position carries ~3e-8 m of
// rounding while a resting overlap under k_n = 1e4 N/m is ~1e-8 m.  So the
// distance is evaluated exactly-rounded-ish in compensated binary32
// (error-free TwoSum / TwoProduct transformations, Knuth and Dekker), which
// brings its error to ~1e-16 m at the cost of ~30 FP32 operations per
// contact -- far cheaper on this part than binary64.
#include "lvb_step.cuh"
#include "lvb_dem.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

using namespace lvb;

namespace {

constexpr int kThreads = 256;
constexpr int kNumSMs = 152;

struct DemDev {
    int n;
    float dt, half_dt, half_dt2;
    float kn, two_zeta, g[3];
    int wall_kind, clamp_tensile, contacts_on;
    float drum_cx, drum_cz, drum_R;
    float4 *pos, *vel, *acc, *vstar;   // vel.w = vstar.w = 1 / m (the integrator
                                       // reads it with v, not from vstar)
    // friction (mu > 0): rotation and the tangential law; omega.w = 1 / I
    float mu, kt, gt_ratio;
    float4 *omega, *alpha, *wstar;     // null without friction
    RowsView rows;
    int trace;                         // per-kernel trace (copied at launch)
};

__device__ __forceinline__ void dtr_enter(const DemDev &d, int slot)
{
    if (d.trace && threadIdx.x == 0) atomicMin(&d.rows.cnt->tr_start[slot], global_ns());
}

__device__ __forceinline__ void dtr_exit(const DemDev &d, int slot)
{
    if (d.trace && (threadIdx.x & 31) == 0) atomicMax(&d.rows.cnt->tr_end[slot], global_ns());
}

// exact a - b = s + e (TwoSum on a and -b)
__device__ __forceinline__ void two_diff(float a, float b, float &s, float &e)
{
    s = __fsub_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fsub_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fadd_rn(b, bb));
}

// exact a + b = s + e
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// |h + l| for a 3-vector given as high + low parts: returns s0 (rounded
// sqrt of the leading sum) and corr with |h + l| = s0 + corr to ~2^-46.
__device__ __forceinline__ void norm_dd(const float h[3], const float l[3], float &s0, float &corr)
{
    float p0 = __fmul_rn(h[0], h[0]), p1 = __fmul_rn(h[1], h[1]), p2 = __fmul_rn(h[2], h[2]);
    float e0 = fmaf(h[0], h[0], -p0), e1 = fmaf(h[1], h[1], -p1), e2 = fmaf(h[2], h[2], -p2);
    float s, t, u, w;
    two_sum(p0, p1, s, t);
    two_sum(s, p2, u, w);
    float lo = t + w + (e0 + e1 + e2) +
               2.0f * (h[0] * l[0] + h[1] * l[1] + h[2] * l[2]);
    s0 = __fsqrt_rn(u);
    const float rem = fmaf(-s0, s0, u) + lo;     // fma remainder is exact
    corr = s0 > 0.0f ? rem / (2.0f * s0) : 0.0f;
}

__device__ __forceinline__ float lsd(const DemDev &d, float dl, float vn, float meff)
{
    const float gam = d.two_zeta * sqrtf(meff * d.kn);
    float f = d.kn * dl - gam * vn;
    if (d.clamp_tensile && f < 0.0f) f = 0.0f;
    return f;
}

__host__ __device__ __forceinline__ IntegrateArgs integrate_args(const DemDev &d)
{
    IntegrateArgs a;
    a.pos = d.pos;
    a.vel = d.vel;
    a.acc = d.acc;
    a.vstar = d.vstar;
    a.omega = d.omega;
    a.alpha = d.alpha;
    a.wstar = d.wstar;
    a.dt = d.dt;
    a.half_dt2 = d.half_dt2;
    a.specular = d.wall_kind == DEM_WALL_SPECULAR;
    a.active = 1;
    return a;
}

__global__ void __launch_bounds__(kThreads)
k_integrate(DemDev d)
{
    const int i = blockIdx.x * kThreads + threadIdx.x;
    if (i == 0) atomicAdd(d.rows.kernels, 1ULL);
    dtr_enter(d, TR_INTEGRATE);
    // the scene's geometry only for the specular walls (no load otherwise)
    if (i < d.n)
        integrate_one<true>(integrate_args(d),
                      d.rows.sg[d.rows.nscenes == 1 || d.wall_kind != DEM_WALL_SPECULAR
                                    ? 0
                                    : d.rows.scene_of[i]],
                      i);
    dtr_exit(d, TR_INTEGRATE);
}

// Wall planes normal to one axis: x in [lo, hi], velocity component v.
__device__ __forceinline__ float plane_force(const DemDev &d, float x, float v, float r, float lo,
                                             float hi, float m)
{
    float F = 0.0f, hh, ll;
    two_diff(x, lo, hh, ll);                       // x - lo
    const float dlo = __fsub_rn(r, hh) - ll;
    if (dlo > 0.0f) F += lsd(d, dlo, v, m);
    two_diff(hi, x, hh, ll);                       // hi - x
    const float dhi = __fsub_rn(r, hh) - ll;
    if (dhi > 0.0f) F -= lsd(d, dhi, -v, m);
    return F;
}

// One contact of the narrow phase (Eq. delta) and its force: particle i at
// xi with v* and 1/m in vi, against partner j of its row.  Returns false
// when the two do not overlap (delta <= 0); else the overlap dl (compensated
// binary32), the unit normal n (from j to i) and the normal force f on i
// along n (linear spring-dashpot, damping on the normal component of
// v*_i - v*_j).
__device__ __forceinline__ bool contact_pair(const DemDev &d, float4 xi, float4 vi, int j,
                                             float &dl, float n[3], float &f)
{
    const float4 xj = d.pos[j];
    float h[3], l[3];
    two_diff(xi.x, xj.x, h[0], l[0]);
    two_diff(xi.y, xj.y, h[1], l[1]);
    two_diff(xi.z, xj.z, h[2], l[2]);
    // cheap reject before the compensated distance
    const float Rr = xi.w + xj.w;
    const float d2 = h[0] * h[0] + h[1] * h[1] + h[2] * h[2];
    if (d2 > Rr * Rr * 1.0001f) return false;
    float s0, corr;
    norm_dd(h, l, s0, corr);
    float Rh, Rl;
    two_sum(xi.w, xj.w, Rh, Rl);
    dl = __fsub_rn(Rh, s0) + (Rl - corr);
    if (!(dl > 0.0f) || !(s0 > 0.0f)) return false;
    const float inv = 1.0f / (s0 + corr);
    n[0] = (h[0] + l[0]) * inv;
    n[1] = (h[1] + l[1]) * inv;
    n[2] = (h[2] + l[2]) * inv;
    const float4 vj = d.vstar[j];
    const float vn = (vi.x - vj.x) * n[0] + (vi.y - vj.y) * n[1] + (vi.z - vj.z) * n[2];
    const float meff = 1.0f / (vi.w + vj.w);
    f = lsd(d, dl, vn, meff);
    return true;
}

__device__ __forceinline__ float dot_rn(float ax, float ay, float az, const float n[3])
{
    return __fadd_rn(__fadd_rn(__fmul_rn(ax, n[0]), __fmul_rn(ay, n[1])), __fmul_rn(az, n[2]));
}

// The tangential law of one contact (friction), from particle i's side:
// updates the spring xi kept in h (row i's history record of partner j)
// and returns the tangential force on i.  Every operation is rounded
// explicitly (no contraction), in an order that is exactly sign-symmetric
// under exchanging i and j (n -> -n), so that j's record stays exactly -h.
__device__ __forceinline__ float3 tangential(const DemDev &d, float ri, float4 vi, float4 wi,
                                             int j, const float n[3], float fn, float meff,
                                             float4 &h)
{
    const float4 vj = d.vstar[j], wj = d.wstar[j];
    const float rj = d.pos[j].w;
    // s = r_i w_i + r_j w_j, c = s x n: the contact point's rotational velocity
    const float sx = __fadd_rn(__fmul_rn(ri, wi.x), __fmul_rn(rj, wj.x));
    const float sy = __fadd_rn(__fmul_rn(ri, wi.y), __fmul_rn(rj, wj.y));
    const float sz = __fadd_rn(__fmul_rn(ri, wi.z), __fmul_rn(rj, wj.z));
    const float cx = __fsub_rn(__fmul_rn(sy, n[2]), __fmul_rn(sz, n[1]));
    const float cy = __fsub_rn(__fmul_rn(sz, n[0]), __fmul_rn(sx, n[2]));
    const float cz = __fsub_rn(__fmul_rn(sx, n[1]), __fmul_rn(sy, n[0]));
    const float ux = __fsub_rn(__fsub_rn(vi.x, vj.x), cx);
    const float uy = __fsub_rn(__fsub_rn(vi.y, vj.y), cy);
    const float uz = __fsub_rn(__fsub_rn(vi.z, vj.z), cz);
    const float un = dot_rn(ux, uy, uz, n);
    const float tx = __fsub_rn(ux, __fmul_rn(un, n[0]));
    const float ty = __fsub_rn(uy, __fmul_rn(un, n[1]));
    const float tz = __fsub_rn(uz, __fmul_rn(un, n[2]));
    // the spring kept in the tangent plane, then stretched by v_t dt
    const float hn = dot_rn(h.x, h.y, h.z, n);
    float hx = __fadd_rn(__fsub_rn(h.x, __fmul_rn(hn, n[0])), __fmul_rn(tx, d.dt));
    float hy = __fadd_rn(__fsub_rn(h.y, __fmul_rn(hn, n[1])), __fmul_rn(ty, d.dt));
    float hz = __fadd_rn(__fsub_rn(h.z, __fmul_rn(hn, n[2])), __fmul_rn(tz, d.dt));
    const float gt = __fmul_rn(d.gt_ratio, __fmul_rn(d.two_zeta, __fsqrt_rn(__fmul_rn(meff, d.kn))));
    float Fx = -__fadd_rn(__fmul_rn(d.kt, hx), __fmul_rn(gt, tx));
    float Fy = -__fadd_rn(__fmul_rn(d.kt, hy), __fmul_rn(gt, ty));
    float Fz = -__fadd_rn(__fmul_rn(d.kt, hz), __fmul_rn(gt, tz));
    const float Fm = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(Fx, Fx), __fmul_rn(Fy, Fy)),
                                          __fmul_rn(Fz, Fz)));
    const float lim = __fmul_rn(d.mu, fmaxf(fn, 0.0f));
    if (Fm > lim) {   // sliding: the force at the Coulomb limit, the spring to match it
        const float sc = __fdiv_rn(lim, Fm);
        Fx = __fmul_rn(Fx, sc);
        Fy = __fmul_rn(Fy, sc);
        Fz = __fmul_rn(Fz, sc);
        hx = -__fdiv_rn(__fadd_rn(Fx, __fmul_rn(gt, tx)), d.kt);
        hy = -__fdiv_rn(__fadd_rn(Fy, __fmul_rn(gt, ty)), d.kt);
        hz = -__fdiv_rn(__fadd_rn(Fz, __fmul_rn(gt, tz)), d.kt);
    }
    h = make_float4(hx, hy, hz, 0.0f);
    return make_float3(Fx, Fy, Fz);
}

// Narrow phase on the row of particle i + walls + velocity finish; the
// friction form (fric) also the tangential law, torques and rotation.
// kEarly (the forces as a kernel of their own, 32 registers): the row
// bounds and the scene of i are loaded with the particle's own state, not
// after the error word and the row walk; the fused tail keeps the late
// loads (fewer registers held across the walk).
template <bool fric, bool kEarly = false>
__device__ __forceinline__ void forces_body(const DemDev &d, int i)
{
    const float4 xi = d.pos[i];
    const float4 vi = d.vstar[i];
    const float4 a = d.acc[i];
    float4 v = d.vel[i];
    const float im_i = vi.w;
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
    float Tx = 0.f, Ty = 0.f, Tz = 0.f;
    const float4 wi = fric ? d.wstar[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const bool walls = d.wall_kind == DEM_WALL_BOX || d.wall_kind == DEM_WALL_DRUM;
    int sc_i = 0, off = 0, len = 0;
    if (kEarly) {   // in range either way; used only as below
        sc_i = walls && d.rows.nscenes > 1 ? d.rows.scene_of[i] : 0;
        off = d.rows.row_off[i];
        len = min(d.rows.row_len[i], d.rows.row_cap[i]);
    }
    // after a row store that failed even a tight re-layout (LVB_EOVERFLOW)
    // the row offsets no longer fit the store: the rows are not read
    if (d.contacts_on && !(d.rows.cnt->err & DERR_STORE)) {
        if (!kEarly) {
            off = d.rows.row_off[i];
            len = min(d.rows.row_len[i], d.rows.row_cap[i]);
        }
        for (int e = 0; e < len; ++e) {
            const int j = d.rows.col[off + e];
            if (j < 0) continue;            // a removed pair's slot
            float dl, n[3], f;
            if (!contact_pair(d, xi, vi, j, dl, n, f)) {
                if (fric) d.rows.hist[off + e] = make_float4(0.f, 0.f, 0.f, 0.f);
                continue;
            }
            Fx += f * n[0];
            Fy += f * n[1];
            Fz += f * n[2];
            if (fric) {
                float4 h = d.rows.hist[off + e];
                const float meff = 1.0f / (im_i + d.vstar[j].w);
                const float3 Ft = tangential(d, xi.w, vi, wi, j, n, f, meff, h);
                d.rows.hist[off + e] = h;
                Fx += Ft.x;
                Fy += Ft.y;
                Fz += Ft.z;
                // torque -r_i n x F_t
                Tx -= xi.w * (n[1] * Ft.z - n[2] * Ft.y);
                Ty -= xi.w * (n[2] * Ft.x - n[0] * Ft.z);
                Tz -= xi.w * (n[0] * Ft.y - n[1] * Ft.x);
            }
        }
    }
    const float r = xi.w;
    if (walls) {
        if (!kEarly && d.rows.nscenes > 1) sc_i = d.rows.scene_of[i];
        const SceneGeom &g = d.rows.sg[sc_i];
        const float m = 1.0f / im_i;
        if (d.wall_kind == DEM_WALL_BOX) {
            Fx += plane_force(d, xi.x, vi.x, r, g.lo[0], g.hi[0], m);
            Fz += plane_force(d, xi.z, vi.z, r, g.lo[2], g.hi[2], m);
        }
        Fy += plane_force(d, xi.y, vi.y, r, g.lo[1], g.hi[1], m);   // box side / drum caps
        if (d.wall_kind == DEM_WALL_DRUM) {
            float h[3], l[3];
            two_diff(xi.x, d.drum_cx, h[0], l[0]);
            h[1] = 0.0f;
            l[1] = 0.0f;
            two_diff(xi.z, d.drum_cz, h[2], l[2]);
            float s0, corr;
            norm_dd(h, l, s0, corr);
            // delta = r + rho - R, rho = s0 + corr; (s0 - R) is exact near the wall
            const float t = __fsub_rn(s0, d.drum_R);
            const float dl = __fadd_rn(t, r) + corr;
            if (dl > 0.0f && s0 > 0.0f) {
                const float inv = 1.0f / s0;
                const float nx = -(h[0] + l[0]) * inv, nz = -(h[2] + l[2]) * inv;
                const float vn = vi.x * nx + vi.z * nz;
                const float f = lsd(d, dl, vn, m);
                Fx += f * nx;
                Fz += f * nz;
            }
        }
    }
    const float4 an = make_float4(Fx * im_i + d.g[0], Fy * im_i + d.g[1], Fz * im_i + d.g[2],
                                  0.0f);
    v.x += (a.x + an.x) * d.half_dt;
    v.y += (a.y + an.y) * d.half_dt;
    v.z += (a.z + an.z) * d.half_dt;
    d.vel[i] = v;
    d.acc[i] = an;
    if (fric) {   // al' = T / I, w' = w + (al + al') dt / 2
        float4 w = d.omega[i];
        const float4 al = d.alpha[i];
        const float4 aln = make_float4(Tx * w.w, Ty * w.w, Tz * w.w, 0.0f);
        w.x += (al.x + aln.x) * d.half_dt;
        w.y += (al.y + aln.y) * d.half_dt;
        w.z += (al.z + aln.z) * d.half_dt;
        d.omega[i] = w;
        d.alpha[i] = aln;
    }
}

// The friction form is a separate function, so that its registers do not
// weigh on the kernels that run without it.
static __device__ __noinline__ void forces_one_fric(const DemDev &d, int i)
{
    forces_body<true>(d, i);
}

template <bool kEarly = false>
__device__ __forceinline__ void forces_one(const DemDev &d, int i)
{
    if (d.omega) forces_one_fric(d, i);
    else forces_body<false, kEarly>(d, i);
}

// Forces as a separate kernel, one thread per particle.  Eight blocks per
// SM (32 registers, a few spilled): the row walks are dependent loads, and
// full occupancy hides them better (-10% on the batched workload).
__global__ void __launch_bounds__(kThreads, 8)
k_forces(DemDev d)
{
    const int i = blockIdx.x * kThreads + threadIdx.x;
    if (i == 0) atomicAdd(d.rows.kernels, 1ULL);
    dtr_enter(d, TR_FORCES);
    if (i < d.n) forces_one<true>(d, i);
    dtr_exit(d, TR_FORCES);
}

// Forces as the tail phase of the fused step kernel (grid-stride).
struct DemTail {
    static constexpr bool kActive = true;
    DemDev d;
    __device__ void operator()(int t, int nt) const
    {
        for (int i = t; i < d.n; i += nt) forces_one(d, i);
    }
};

// The contacts of the current state, each pair once (i < j from row i),
// with the force on i and the overlap; positions in the output from one
// atomic counter, so in no particular order.
__global__ void __launch_bounds__(kThreads)
k_contact_list(DemDev d, unsigned long long *cnt, long long cap, int *ci, int *cj, float *f3,
               float *delta, float *xi3, int both)
{
    const int i = blockIdx.x * kThreads + threadIdx.x;
    if (i == 0) atomicAdd(d.rows.kernels, 1ULL);
    if (i >= d.n || !d.contacts_on || (d.rows.cnt->err & DERR_STORE)) return;
    const float4 xi = d.pos[i];
    const float4 vi = d.vstar[i];
    const bool fric = d.omega != nullptr;
    const int off = d.rows.row_off[i];
    const int len = min(d.rows.row_len[i], d.rows.row_cap[i]);
    for (int e = 0; e < len; ++e) {
        const int j = d.rows.col[off + e];
        // a removed pair's slot, or (one side only) the pair from j's row
        if (j < 0 || (!both && j <= i)) continue;
        float dl, n[3], f;
        if (!contact_pair(d, xi, vi, j, dl, n, f)) continue;
        float Ft[3] = {0.f, 0.f, 0.f}, h[3] = {0.f, 0.f, 0.f};
        if (fric) {
            // F_t = -k_t xi - gamma_t v_t from the spring as the step left it
            const float4 r = d.rows.hist[off + e];
            h[0] = r.x;
            h[1] = r.y;
            h[2] = r.z;
            const float4 vj = d.vstar[j], wi = d.wstar[i], wj = d.wstar[j];
            const float ri = xi.w, rj = d.pos[j].w;
            const float sx = __fadd_rn(__fmul_rn(ri, wi.x), __fmul_rn(rj, wj.x));
            const float sy = __fadd_rn(__fmul_rn(ri, wi.y), __fmul_rn(rj, wj.y));
            const float sz = __fadd_rn(__fmul_rn(ri, wi.z), __fmul_rn(rj, wj.z));
            const float u[3] = {
                __fsub_rn(__fsub_rn(vi.x, vj.x), __fsub_rn(__fmul_rn(sy, n[2]), __fmul_rn(sz, n[1]))),
                __fsub_rn(__fsub_rn(vi.y, vj.y), __fsub_rn(__fmul_rn(sz, n[0]), __fmul_rn(sx, n[2]))),
                __fsub_rn(__fsub_rn(vi.z, vj.z), __fsub_rn(__fmul_rn(sx, n[1]), __fmul_rn(sy, n[0])))};
            const float un = dot_rn(u[0], u[1], u[2], n);
            const float meff = 1.0f / (vi.w + vj.w);
            const float gt =
                __fmul_rn(d.gt_ratio, __fmul_rn(d.two_zeta, __fsqrt_rn(__fmul_rn(meff, d.kn))));
            for (int c = 0; c < 3; ++c)
                Ft[c] = -__fadd_rn(__fmul_rn(d.kt, h[c]),
                                   __fmul_rn(gt, __fsub_rn(u[c], __fmul_rn(un, n[c]))));
        }
        const unsigned long long k = atomicAdd(cnt, 1ULL);
        if (k < (unsigned long long)cap) {
            ci[k] = i;
            cj[k] = j;
            f3[3 * k + 0] = f * n[0] + Ft[0];
            f3[3 * k + 1] = f * n[1] + Ft[1];
            f3[3 * k + 2] = f * n[2] + Ft[2];
            delta[k] = dl;
            if (xi3) {
                xi3[3 * k + 0] = h[0];
                xi3[3 * k + 1] = h[1];
                xi3[3 * k + 2] = h[2];
            }
        }
    }
}

__global__ void k_dem_setup(DemDev d, const float4 *__restrict__ pos, const float4 *__restrict__ vel,
                            float rho)
{
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < d.n; i += gridDim.x * kThreads) {
        const float4 p = pos[i];
        const float4 v = vel[i];
        const double r = p.w;
        const double m = (double)rho * (4.0 / 3.0) * 3.14159265358979323846 * r * r * r;
        d.pos[i] = p;
        const float im = (float)(1.0 / m);
        d.vel[i] = make_float4(v.x, v.y, v.z, im);
        d.vstar[i] = make_float4(v.x, v.y, v.z, im);
        d.acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (d.omega) {   // at rest, I = 2/5 m r^2
            const float iI = (float)(1.0 / (0.4 * m * r * r));
            d.omega[i] = make_float4(0.f, 0.f, 0.f, iI);
            d.wstar[i] = make_float4(0.f, 0.f, 0.f, iI);
            d.alpha[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

// After the caller overwrote v: 1 / m back into v.w (from v*.w).
__global__ void k_restore_im(DemDev d)
{
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < d.n; i += gridDim.x * kThreads)
        d.vel[i].w = d.vstar[i].w;
}

// initial a0 = F(x0, v0)/m + g: the force kernel with a = 0 and dt = 0
// leaves v unchanged and writes a0.
}  // namespace

struct dem_ctx {
    DemDev d{};
    dem_params prm{};
    lvb_ctx *bp = nullptr;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    int64_t graph_steps = 0;
    int graph_version = 0;
};

namespace {

int from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return LVB_OK;
    if (e == cudaErrorMemoryAllocation) return LVB_ENOMEM;
    return LVB_EDEVICE;
}

int grid_n(int n) { return (n + kThreads - 1) / kThreads; }

void dem_free(dem_ctx *c)
{
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->bp) lvb_destroy(c->bp);
    float4 *ptrs[] = {c->d.pos, c->d.vel, c->d.acc, c->d.vstar, c->d.omega, c->d.alpha,
                      c->d.wstar};
    for (float4 *p : ptrs)
        if (p) cudaFree(p);
}

// The driver's copy of the row-store addresses follows the broad phase's
// (a grown store moves), and the trace switch follows its option.
void refresh(dem_ctx *c)
{
    c->d.rows = rows_view(c->bp);
    c->d.trace = *c->d.rows.trace;
}

int launch_phase(dem_ctx *c, int phase)
{
    refresh(c);
    if (phase == DEM_PHASE_INTEGRATE) {
        k_integrate<<<grid_n(c->d.n), kThreads, 0, c->stream>>>(c->d);
    } else if (phase == DEM_PHASE_BROAD) {
        int rc = lvb_step(c->bp, (const float *)c->d.pos, (const float *)c->d.vstar,
                          (const float *)c->d.acc);
        if (rc) return rc;
    } else if (phase == DEM_PHASE_FORCES) {
        k_forces<<<grid_n(c->d.n), kThreads, 0, c->stream>>>(c->d);
    } else {
        return LVB_EINVAL;
    }
    return from_cuda(cudaGetLastError());
}

// Launch shape of the fused step: the broad phase's block size, and no more
// blocks than fit on the device at once for this kernel.
int fused_shape(dem_ctx *c, dim3 *grid, dim3 *block)
{
    int blocks = 0, threads = 0, dev = 0, sms = 0, per_sm = 0;
    step_shape(c->bp, &blocks, &threads);
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step<true, DemTail>, threads,
                                                          0);
    if (e != cudaSuccess) return from_cuda(e);
    if (per_sm < 1) return LVB_EDEVICE;
    *grid = dim3(std::min(blocks, per_sm * sms));
    *block = dim3(threads);
    return LVB_OK;
}

// One whole step (half-step, broad phase, forces) as one cooperative launch.
int launch_fused(dem_ctx *c)
{
    int rc = grow_stores_if_asked(c->bp);
    if (rc) return rc;
    refresh(c);
    dim3 grid, block;
    rc = fused_shape(c, &grid, &block);
    if (rc) return rc;
    const DemDev &d = c->d;
    return from_cuda(launch_coop(k_step<true, DemTail>, grid, block, 0, c->stream,
                                 (const float4 *)d.pos, (const float4 *)d.vstar,
                                 (const float4 *)d.acc, step_state(c->bp), integrate_args(d),
                                 DemTail{d}));
}

}  // namespace

extern "C" {

static int dem_init_impl(dem_ctx **out, int32_t n_scenes, const int64_t *offsets, int64_t n,
                         const float *pos_r, const float *vel, const dem_params *prm, float dt,
                         const lvb_box *box, const lvb_skin_policy *skin, int32_t trigger,
                         float cell_factor, void *stream)
{
    if (!out) return LVB_EINVAL;
    *out = nullptr;
    if (!pos_r || !vel || !prm || !box || !skin || n < 1 || n > INT32_MAX - 64) return LVB_EINVAL;
    if (!(dt > 0.0f) || !(prm->kn >= 0.0f) || !(prm->rho > 0.0f) ||
        !(prm->restitution > 0.0f && prm->restitution <= 1.0f))
        return LVB_EINVAL;
    if (prm->wall_kind < DEM_WALL_NONE || prm->wall_kind > DEM_WALL_SPECULAR) return LVB_EINVAL;
    if (!(prm->mu >= 0.0f) || !std::isfinite(prm->mu)) return LVB_EINVAL;
    if (prm->mu > 0.0f && (!(prm->kt_ratio > 0.0f) || !std::isfinite(prm->kt_ratio) ||
                           !(prm->gt_ratio >= 0.0f) || !std::isfinite(prm->gt_ratio) ||
                           trigger != LVB_TRIGGER_PARTIAL))
        return LVB_EINVAL;
    if (((uintptr_t)pos_r & 15u) || ((uintptr_t)vel & 15u)) return LVB_EINVAL;
    cudaGetLastError();   // clear a stale error of an unrelated earlier call
    dem_ctx *c = new (std::nothrow) dem_ctx();
    if (!c) return LVB_ENOMEM;
    c->prm = *prm;
    c->stream = (cudaStream_t)stream;
    DemDev &d = c->d;
    d.n = (int)n;
    d.dt = dt;
    d.half_dt = 0.5f * dt;
    d.half_dt2 = (float)(0.5 * (double)dt * (double)dt);
    d.kn = prm->kn;
    const double le = std::log((double)prm->restitution);
    d.two_zeta = (float)(2.0 * (-le / std::sqrt(M_PI * M_PI + le * le)));
    for (int k = 0; k < 3; ++k) d.g[k] = prm->g[k];
    d.wall_kind = prm->wall_kind;
    d.clamp_tensile = prm->clamp_tensile;
    d.contacts_on = prm->contacts_on;
    d.drum_cx = prm->drum_cx;
    d.drum_cz = prm->drum_cz;
    d.drum_R = prm->drum_R;
    d.mu = prm->mu;
    d.kt = prm->kt_ratio * prm->kn;
    d.gt_ratio = prm->gt_ratio;
    cudaError_t e = cudaMalloc((void **)&d.pos, sizeof(float4) * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.vel, sizeof(float4) * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.acc, sizeof(float4) * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.vstar, sizeof(float4) * n);
    if (prm->mu > 0.0f) {
        if (e == cudaSuccess) e = cudaMalloc((void **)&d.omega, sizeof(float4) * n);
        if (e == cudaSuccess) e = cudaMalloc((void **)&d.alpha, sizeof(float4) * n);
        if (e == cudaSuccess) e = cudaMalloc((void **)&d.wstar, sizeof(float4) * n);
    }
    if (e != cudaSuccess) {
        dem_free(c);
        delete c;
        return from_cuda(e);
    }
    k_dem_setup<<<std::min(grid_n((int)n), 4 * kNumSMs), kThreads, 0, c->stream>>>(
        d, (const float4 *)pos_r, (const float4 *)vel, prm->rho);
    int rc = offsets ? lvb_batch_init(&c->bp, n_scenes, offsets, (const float *)d.pos, box, skin,
                                      trigger, cell_factor, (const float *)d.vstar,
                                      (const float *)d.acc, stream)
                     : lvb_init(&c->bp, n, (const float *)d.pos, box, skin, trigger, cell_factor,
                                (const float *)d.vstar, (const float *)d.acc, stream);
    if (rc) {
        c->bp = nullptr;
        dem_free(c);
        delete c;
        return rc;
    }
    if (prm->mu > 0.0f) {   // the tangential springs live in the contact history
        rc = lvb_set_option(c->bp, LVB_OPT_HISTORY, 1);
        if (rc) {
            dem_free(c);
            delete c;
            return rc;
        }
    }
    d.rows = rows_view(c->bp);
    // a0 from the forces at (x0, v0): one force pass with a = 0, dt = 0
    // (the tangential springs start at zero: this pass leaves them alone,
    // and al0 = 0)
    DemDev d0 = d;
    d0.half_dt = 0.0f;
    d0.omega = d0.alpha = d0.wstar = nullptr;
    k_forces<<<grid_n(d.n), kThreads, 0, c->stream>>>(d0);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        dem_free(c);
        delete c;
        return from_cuda(e);
    }
    *out = c;
    return LVB_OK;
}

int dem_init(dem_ctx **out, int64_t n, const float *pos_r, const float *vel,
             const dem_params *prm, float dt, const lvb_box *box, const lvb_skin_policy *skin,
             int32_t trigger, float cell_factor, void *stream)
{
    return dem_init_impl(out, 1, nullptr, n, pos_r, vel, prm, dt, box, skin, trigger,
                         cell_factor, stream);
}

int dem_batch_init(dem_ctx **out, int32_t n_scenes, const int64_t *offsets, const float *pos_r,
                   const float *vel, const dem_params *prm, float dt, const lvb_box *boxes,
                   const lvb_skin_policy *skin, int32_t trigger, float cell_factor, void *stream)
{
    if (!offsets || n_scenes < 1) return LVB_EINVAL;
    return dem_init_impl(out, n_scenes, offsets, offsets[n_scenes], pos_r, vel, prm, dt, boxes,
                         skin, trigger, cell_factor, stream);
}

int dem_phase(dem_ctx *c, int32_t phase)
{
    if (!c) return LVB_EINVAL;
    cudaGetLastError();
    // the row store may have been re-laid out; pointers stay the same
    return launch_phase(c, phase);
}

int dem_advance(dem_ctx *c, int64_t steps)
{
    if (!c || steps < 0) return LVB_EINVAL;
    cudaGetLastError();   // clear a stale error of an unrelated earlier call
    const int64_t chunk = DEM_GRAPH_STEPS;
    int64_t done = 0;
    while (steps - done >= chunk) {
        // a store asked to grow: grow it (the graph holds the old store's
        // addresses, so it is rebuilt below)
        int rc = grow_stores_if_asked(c->bp);
        if (rc) return rc;
        if (c->graph && c->graph_version != graph_version(c->bp)) {
            cudaGraphExecDestroy(c->graph);
            c->graph = nullptr;
        }
        if (!c->graph) {
            // one graph of `chunk` cooperative step kernels, built node by
            // node (no stream capture, so any stream works, the legacy
            // default one included)
            refresh(c);
            dim3 grid, block;
            rc = fused_shape(c, &grid, &block);
            if (rc) return rc;
            const DemDev &d = c->d;
            const DevState st = step_state(c->bp);
            const IntegrateArgs ia = integrate_args(d);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaGraphCreate(&g, 0);
            cudaGraphNode_t dep = nullptr;
            for (int64_t k = 0; k < chunk && e == cudaSuccess; ++k)
                e = add_coop_kernel(&dep, g, &dep, k_step<true, DemTail>, grid, block,
                                    (const float4 *)d.pos, (const float4 *)d.vstar,
                                    (const float4 *)d.acc, st, ia, DemTail{d});
            if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                c->graph = nullptr;
                return from_cuda(e);
            }
            c->graph_steps = chunk;
            c->graph_version = graph_version(c->bp);
        }
        const cudaError_t e = cudaGraphLaunch(c->graph, c->stream);
        if (e != cudaSuccess) return from_cuda(e);
        done += chunk;
    }
    for (; done < steps; ++done) {
        const int rc = launch_fused(c);
        if (rc) return rc;
    }
    return LVB_OK;
}

static int contact_list(dem_ctx *c, int both, int32_t *ci, int32_t *cj, float *force3,
                        float *delta, float *xi3, int64_t cap, int64_t *n_contacts);

int dem_get_contact_forces(dem_ctx *c, int32_t *ci, int32_t *cj, float *force3, float *delta,
                           int64_t cap, int64_t *n_contacts)
{
    return contact_list(c, 0, ci, cj, force3, delta, nullptr, cap, n_contacts);
}

int dem_get_contact_history(dem_ctx *c, int32_t sides, int32_t *ci, int32_t *cj, float *force3,
                            float *delta, float *xi3, int64_t cap, int64_t *n_contacts)
{
    if (sides != 1 && sides != 2) return LVB_EINVAL;
    return contact_list(c, sides == 2, ci, cj, force3, delta, xi3, cap, n_contacts);
}

int dem_get_rot_state(dem_ctx *c, float *omega, float *alpha, float *omega_star)
{
    if (!c) return LVB_EINVAL;
    const size_t b = sizeof(float4) * (size_t)c->d.n;
    cudaError_t e = cudaSuccess;
    float *outs[3] = {omega, alpha, omega_star};
    const float4 *srcs[3] = {c->d.omega, c->d.alpha, c->d.wstar};
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        if (!outs[k]) continue;
        if (srcs[k]) e = cudaMemcpyAsync(outs[k], srcs[k], b, cudaMemcpyDefault, c->stream);
        else e = cudaMemsetAsync(outs[k], 0, b, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return from_cuda(e);
}

static int contact_list(dem_ctx *c, int both, int32_t *ci, int32_t *cj, float *force3,
                        float *delta, float *xi3, int64_t cap, int64_t *n_contacts)
{
    if (!c || !n_contacts || cap < 0 || (cap > 0 && (!ci || !cj || !force3 || !delta)))
        return LVB_EINVAL;
    *n_contacts = 0;
    refresh(c);
    const long long cp = std::max<long long>(cap, 1);
    int *di = nullptr, *dj = nullptr;
    float *df = nullptr, *dd = nullptr, *dx = nullptr;
    unsigned long long *cnt = nullptr;
    cudaError_t e = cudaMalloc((void **)&cnt, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void **)&di, sizeof(int) * cp);
    if (e == cudaSuccess) e = cudaMalloc((void **)&dj, sizeof(int) * cp);
    if (e == cudaSuccess) e = cudaMalloc((void **)&df, sizeof(float) * 3 * cp);
    if (e == cudaSuccess) e = cudaMalloc((void **)&dd, sizeof(float) * cp);
    if (e == cudaSuccess && xi3) e = cudaMalloc((void **)&dx, sizeof(float) * 3 * cp);
    unsigned long long total = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(total), c->stream);
    if (e == cudaSuccess) {
        k_contact_list<<<grid_n(c->d.n), kThreads, 0, c->stream>>>(c->d, cnt, cap, di, dj, df,
                                                                     dd, dx, both);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&total, cnt, sizeof(total), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    const long long m = std::min<long long>((long long)total, cap);
    if (e == cudaSuccess && m > 0) {
        e = cudaMemcpyAsync(ci, di, sizeof(int) * m, cudaMemcpyDefault, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(cj, dj, sizeof(int) * m, cudaMemcpyDefault, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(force3, df, sizeof(float) * 3 * m, cudaMemcpyDefault, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(delta, dd, sizeof(float) * m, cudaMemcpyDefault, c->stream);
        if (e == cudaSuccess && xi3)
            e = cudaMemcpyAsync(xi3, dx, sizeof(float) * 3 * m, cudaMemcpyDefault, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    cudaFree(cnt);
    cudaFree(di);
    cudaFree(dj);
    cudaFree(df);
    cudaFree(dd);
    if (dx) cudaFree(dx);
    if (e != cudaSuccess) return from_cuda(e);
    *n_contacts = (int64_t)total;
    const int rc = lvb_sync(c->bp);
    if (rc) return rc;
    return (long long)total > cap ? LVB_ECAPACITY : LVB_OK;
}

int dem_get_state(dem_ctx *c, float *pos_r, float *vel, float *acc, float *vstar)
{
    if (!c) return LVB_EINVAL;
    const size_t b = sizeof(float4) * (size_t)c->d.n;
    cudaError_t e = cudaSuccess;
    if (pos_r) e = cudaMemcpyAsync(pos_r, c->d.pos, b, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess && vel) e = cudaMemcpyAsync(vel, c->d.vel, b, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess && acc) e = cudaMemcpyAsync(acc, c->d.acc, b, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess && vstar)
        e = cudaMemcpyAsync(vstar, c->d.vstar, b, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return from_cuda(e);
}

int dem_set_state(dem_ctx *c, const float *pos_r, const float *vel, const float *acc)
{
    if (!c) return LVB_EINVAL;
    const size_t b = sizeof(float4) * (size_t)c->d.n;
    cudaError_t e = cudaSuccess;
    if (pos_r) e = cudaMemcpyAsync(c->d.pos, pos_r, b, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess && vel) e = cudaMemcpyAsync(c->d.vel, vel, b, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess && vel) {
        const int grid = std::min(grid_n((int)c->d.n), 4 * kNumSMs);
        k_restore_im<<<grid, kThreads, 0, c->stream>>>(c->d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && acc) e = cudaMemcpyAsync(c->d.acc, acc, b, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return from_cuda(e);
}

int dem_lvb(dem_ctx *c, lvb_ctx **out)
{
    if (!c || !out) return LVB_EINVAL;
    *out = c->bp;
    return LVB_OK;
}

int dem_device_state(dem_ctx *c, float **pos_r, float **vel, float **acc, float **vstar)
{
    if (!c) return LVB_EINVAL;
    if (pos_r) *pos_r = (float *)c->d.pos;
    if (vel) *vel = (float *)c->d.vel;
    if (acc) *acc = (float *)c->d.acc;
    if (vstar) *vstar = (float *)c->d.vstar;
    return LVB_OK;
}

int dem_sync(dem_ctx *c)
{
    if (!c) return LVB_EINVAL;
    return lvb_sync(c->bp);
}

int dem_destroy(dem_ctx *c)
{
    if (!c) return LVB_EINVAL;
    cudaStreamSynchronize(c->stream);
    dem_free(c);
    delete c;
    return LVB_OK;
}

}  // extern "C"
