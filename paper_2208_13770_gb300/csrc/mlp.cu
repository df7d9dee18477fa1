// mlp.cu -- the skin network's inference, gradient and training on the GPU
// (include/lvb_mlp.h).  bfloat16 weights and activations, binary32
// accumulation; no tensor cores: the whole network is 1,377 parameters and
// ~2.6 kFLOP per sample, far below what a contraction would need to pay.
//
// Training: one thread per sample runs the forward pass (the exact inference
// formula) and the backward pass (straight-through the bfloat16 roundings);
// a block of kTB samples stages its activations in shared memory and reduces
// its share of every weight gradient into its own row of partial sums; the
// rows are then added in block order (no atomics), so training is bitwise
// repeatable.  Adam updates the binary32 master parameters.
#include "lvb_internal.cuh"
#include "lvb_mlp.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

using namespace lvb;

namespace {

constexpr int NI = LVB_MLP_IN, NH = LVB_MLP_HIDDEN, NP = LVB_MLP_PARAMS;
constexpr int OFF_W1 = 0, OFF_B1 = NH * NI, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH;
constexpr int kTB = 64;   // samples per training block
constexpr int kSamp = NI + 1;

__host__ __device__ inline float bf16_host_rn(float x)
{
    unsigned u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x7fffffu)) return x;   // NaN
    u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

__global__ void k_mlp_infer(const float *__restrict__ feats, const float *__restrict__ diam,
                            int64_t n, const lvb_mlp_weights *__restrict__ W, float *skin,
                            float *yout)
{
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = wid; i < n; i += nw) {
        float f[NI];
#pragma unroll
        for (int k = 0; k < NI; ++k) f[k] = feats[i * NI + k];
        const float y = mlp_y_warp(W, f);
        if ((threadIdx.x & 31) == 0) {
            skin[i] = mlp_skin(W, y, diam[i], f[0]);
            if (yout) yout[i] = y;
        }
    }
}

// Per-column sum and sum of squares (binary64) of the samples: the eight
// features (normalisation) and the label (output range).
// Per-warp sums of every column and of its squares (binary64), written to
// the warp's row of part (2 x kSamp values); the host adds the rows in warp
// order, so the statistics do not depend on scheduling.
constexpr int kStatBlocks = 152 * 4, kStatThreads = 256;
constexpr int kStatWarps = kStatBlocks * kStatThreads / 32;

__global__ void k_feature_stats(const float *__restrict__ samples, int64_t n, double *part)
{
    double s[kSamp] = {0}, q[kSamp] = {0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < kSamp; ++k) {
            const double v = samples[i * kSamp + k];
            s[k] += v;
            q[k] += v * v;
        }
    }
#pragma unroll
    for (int k = 0; k < kSamp; ++k) {
        for (int o = 16; o; o >>= 1) {
            s[k] += __shfl_xor_sync(FULL, s[k], o);
            q[k] += __shfl_xor_sync(FULL, q[k], o);
        }
        if ((threadIdx.x & 31) == 0) {
            const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
            part[(size_t)w * 2 * kSamp + k] = s[k];
            part[(size_t)w * 2 * kSamp + kSamp + k] = q[k];
        }
    }
}

struct TrainArgs {
    const float *samples;   // n x 9
    const int *order;       // sample index of each position (null: identity)
    int64_t first, count;   // positions [first, first + count) form the batch
    const float *params;    // master parameters
    const float *mu, *isd;
    float *part;            // per-block partial gradients (blocks x NP)
    double *loss;           // accumulated sum of (weighted) squared errors
    float dy_scale;         // 2 / batch size
    float rel_floor;        // > 0: relative error, (y - t) / max(t, rel_floor)
};

__global__ void __launch_bounds__(kTB)
k_mlp_batch(TrainArgs a)
{
    __shared__ float sW1[NH * NI], sb1[NH], sW2[NH * NH], sb2[NH], sw3[NH];
    __shared__ float sz[kTB][NI], sh1[kTB][NH], sh2[kTB][NH], sd2[kTB][NH], sd1[kTB][NH];
    __shared__ float sdy[kTB];
    const int t = threadIdx.x;
    for (int k = t; k < NH * NI; k += kTB) sW1[k] = bf16_host_rn(a.params[OFF_W1 + k]);
    for (int k = t; k < NH * NH; k += kTB) sW2[k] = bf16_host_rn(a.params[OFF_W2 + k]);
    for (int k = t; k < NH; k += kTB) {
        sb1[k] = a.params[OFF_B1 + k];
        sb2[k] = a.params[OFF_B2 + k];
        sw3[k] = bf16_host_rn(a.params[OFF_W3 + k]);
    }
    __syncthreads();
    const float b3 = a.params[OFF_B3];
    const int64_t pos = a.first + (int64_t)blockIdx.x * kTB + t;
    const bool live = pos < a.first + a.count;
    float dy = 0.0f;
    if (live) {
        const int64_t si = a.order ? a.order[pos] : pos;
        const float *smp = a.samples + si * kSamp;
#pragma unroll
        for (int k = 0; k < NI; ++k)
            sz[t][k] = bf16_rn(__fmul_rn(__fsub_rn(smp[k], a.mu[k]), a.isd[k]));
        for (int o = 0; o < NH; ++o) {
            float acc = sb1[o];
#pragma unroll
            for (int k = 0; k < NI; ++k) acc = fmaf(sW1[o * NI + k], sz[t][k], acc);
            sh1[t][o] = acc > 0.0f ? bf16_rn(acc) : 0.0f;   // h1 > 0 marks the active units
        }
        for (int o = 0; o < NH; ++o) {
            float acc = sb2[o];
            for (int k = 0; k < NH; ++k) acc = fmaf(sW2[o * NH + k], sh1[t][k], acc);
            sh2[t][o] = acc > 0.0f ? bf16_rn(acc) : 0.0f;   // > 0 marks the active units
        }
        float y = b3;
        for (int k = 0; k < NH; ++k) y = fmaf(sw3[k], sh2[t][k], y);
        const float lab = smp[NI];
        float r = y - lab;
        float w = 1.0f;   // d(loss)/d(r^2)
        if (a.rel_floor > 0.0f) {
            const float den = fmaxf(lab, a.rel_floor);
            w = 1.0f / (den * den);
        }
        dy = a.dy_scale * w * r;
        atomicAdd(a.loss, (double)w * (double)r * (double)r);
        for (int o = 0; o < NH; ++o) sd2[t][o] = sh2[t][o] > 0.0f ? dy * sw3[o] : 0.0f;
        for (int k = 0; k < NH; ++k) {
            float g = 0.0f;
            for (int o = 0; o < NH; ++o) g = fmaf(sd2[t][o], sW2[o * NH + k], g);
            sd1[t][k] = sh1[t][k] > 0.0f ? g : 0.0f;
        }
    } else {
#pragma unroll
        for (int k = 0; k < NI; ++k) sz[t][k] = 0.0f;
        for (int o = 0; o < NH; ++o) sh1[t][o] = sh2[t][o] = sd2[t][o] = sd1[t][o] = 0.0f;
    }
    sdy[t] = dy;
    __syncthreads();
    // this block's share of every parameter's gradient
    for (int p = t; p < NP; p += kTB) {
        float g = 0.0f;
        if (p < OFF_B1) {
            const int o = p / NI, k = p % NI;
            for (int q = 0; q < kTB; ++q) g = fmaf(sd1[q][o], sz[q][k], g);
        } else if (p < OFF_W2) {
            const int o = p - OFF_B1;
            for (int q = 0; q < kTB; ++q) g += sd1[q][o];
        } else if (p < OFF_B2) {
            const int o = (p - OFF_W2) / NH, k = (p - OFF_W2) % NH;
            for (int q = 0; q < kTB; ++q) g = fmaf(sd2[q][o], sh1[q][k], g);
        } else if (p < OFF_W3) {
            const int o = p - OFF_B2;
            for (int q = 0; q < kTB; ++q) g += sd2[q][o];
        } else if (p < OFF_B3) {
            const int k = p - OFF_W3;
            for (int q = 0; q < kTB; ++q) g = fmaf(sdy[q], sh2[q][k], g);
        } else {
            for (int q = 0; q < kTB; ++q) g += sdy[q];
        }
        a.part[(size_t)blockIdx.x * NP + p] = g;
    }
}

// grad[i] += the nb blocks' partial sums of parameter i, in block order.
__global__ void k_fold_parts(const float *part, int nb, float *grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    float g = grad[i];
    for (int b = 0; b < nb; ++b) g += part[(size_t)b * NP + i];
    grad[i] = g;
}

// One Adam step; the gradient is the sum of the nb blocks' partials, added
// in block order.
__global__ void k_adam(float *p, const float *part, int nb, float *m, float *v, int n, float lr,
                       float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = 0.0f;
    for (int b = 0; b < nb; ++b) gi += part[(size_t)b * NP + i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

int from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return LVB_OK;
    if (e == cudaErrorMemoryAllocation) return LVB_ENOMEM;
    return LVB_EDEVICE;
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf()
    {
        if (p) cudaFree(p);
    }
};

template <class T>
cudaError_t dnew(DevBuf &b, size_t count)
{
    return cudaMalloc(&b.p, sizeof(T) * std::max<size_t>(count, 1));
}

// one pass of k_mlp_batch over positions [first, first + count) of a mean
// over `total` samples; returns the number of blocks (rows of part)
int launch_batch(const float *samples, const int *order, int64_t first, int64_t count,
                 int64_t total, const float *params, const float *mu, const float *isd,
                 float *part, double *loss, float rel_floor, cudaStream_t st)
{
    TrainArgs a;
    a.samples = samples;
    a.order = order;
    a.first = first;
    a.count = count;
    a.params = params;
    a.mu = mu;
    a.isd = isd;
    a.part = part;
    a.loss = loss;
    a.dy_scale = 2.0f / (float)total;
    a.rel_floor = rel_floor;
    const int64_t blocks = (count + kTB - 1) / kTB;
    k_mlp_batch<<<(unsigned)blocks, kTB, 0, st>>>(a);
    return (int)blocks;
}

constexpr int64_t kGradChunk = 1024 * kTB;   // samples per pass of lvb_mlp_grad

}  // namespace

extern "C" {

int lvb_mlp_pack(const float *params, const float *mu, const float *isd, const float *y_range,
                 float y_steps, lvb_mlp_weights *out)
{
    if (!params || !mu || !isd || !out) return LVB_EINVAL;
    if (y_range && !(y_range[0] <= y_range[1])) return LVB_EINVAL;
    if (!(y_steps >= 0.0f) || !std::isfinite(y_steps)) return LVB_EINVAL;
    lvb_mlp_weights w;
    memset(&w, 0, sizeof(w));
    w.y_lo = y_range ? y_range[0] : 0.0f;
    w.y_hi = y_range ? y_range[1] : INFINITY;
    w.y_steps = y_steps;
    // input-major device layout (lvb_mlp.h) from the [out][in] master form
    for (int o = 0; o < NH; ++o)
        for (int k = 0; k < NI; ++k) w.W1[k * NH + o] = bf16_host_rn(params[OFF_W1 + o * NI + k]);
    for (int k = 0; k < NH; ++k) w.b1[k] = params[OFF_B1 + k];
    for (int o = 0; o < NH; ++o)
        for (int k = 0; k < NH; ++k) w.W2[k * NH + o] = bf16_host_rn(params[OFF_W2 + o * NH + k]);
    for (int k = 0; k < NH; ++k) w.b2[k] = params[OFF_B2 + k];
    for (int k = 0; k < NH; ++k) w.w3[k] = bf16_host_rn(params[OFF_W3 + k]);
    w.b3 = params[OFF_B3];
    for (int k = 0; k < NI; ++k) {
        w.mu[k] = mu[k];
        w.isd[k] = isd[k];
    }
    return from_cuda(cudaMemcpy(out, &w, sizeof(w), cudaMemcpyDefault));
}

int lvb_mlp_infer(const float *feats, const float *diam, int64_t n, const lvb_mlp_weights *w,
                  float *skin, float *y, void *stream)
{
    if (!feats || !diam || !w || !skin || n < 0) return LVB_EINVAL;
    if (n == 0) return LVB_OK;
    cudaGetLastError();
    const int64_t blocks = std::min<int64_t>((n * 32 + 255) / 256, 152 * 16);
    k_mlp_infer<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(feats, diam, n, w, skin, y);
    return from_cuda(cudaGetLastError());
}

int lvb_mlp_grad(const float *samples, int64_t n, const float *params, const float *mu,
                 const float *isd, float rel_floor, float *grad, double *loss, void *stream)
{
    if (!samples || n < 1 || !params || !mu || !isd || !grad || !loss) return LVB_EINVAL;
    if (!(rel_floor >= 0.0f)) return LVB_EINVAL;
    cudaGetLastError();
    const cudaStream_t st = (cudaStream_t)stream;
    DevBuf dp, dmu, disd, dg, dl, dpart;
    cudaError_t e = dnew<float>(dp, NP);
    if (e == cudaSuccess) e = dnew<float>(dmu, NI);
    if (e == cudaSuccess) e = dnew<float>(disd, NI);
    if (e == cudaSuccess) e = dnew<float>(dg, NP);
    if (e == cudaSuccess) e = dnew<double>(dl, 1);
    if (e == cudaSuccess)
        e = dnew<float>(dpart, (size_t)((std::min(n, kGradChunk) + kTB - 1) / kTB) * NP);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp.p, params, NP * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dmu.p, mu, NI * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(disd.p, isd, NI * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dg.p, 0, NP * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dl.p, 0, 8, st);
    if (e != cudaSuccess) return from_cuda(e);
    for (int64_t first = 0; first < n; first += kGradChunk) {
        const int nb = launch_batch(samples, nullptr, first, std::min(kGradChunk, n - first), n,
                                    (const float *)dp.p, (const float *)dmu.p,
                                    (const float *)disd.p, (float *)dpart.p, (double *)dl.p,
                                    rel_floor, st);
        k_fold_parts<<<(NP + 255) / 256, 256, 0, st>>>((const float *)dpart.p, nb, (float *)dg.p);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(grad, dg.p, NP * 4, cudaMemcpyDeviceToHost, st);
    double sse = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sse, dl.p, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return from_cuda(e);
    *loss = sse / (double)n;
    return LVB_OK;
}

int lvb_mlp_train(const float *samples, int64_t n, int32_t epochs, int32_t batch, float lr,
                  uint64_t seed, int32_t loss_kind, float *params, float *mu, float *isd,
                  float *y_range, float *losses, void *stream)
{
    if (!samples || n < 1 || epochs < 1 || batch < 1 || !(lr > 0.0f) || !params || !mu || !isd ||
        !y_range)
        return LVB_EINVAL;
    if (loss_kind != LVB_MLP_LOSS_SQUARED && loss_kind != LVB_MLP_LOSS_RELATIVE)
        return LVB_EINVAL;
    if (n > INT32_MAX) return LVB_EINVAL;
    cudaGetLastError();
    const cudaStream_t st = (cudaStream_t)stream;
    // feature normalisation from the samples (mean, 1/std), label range
    DevBuf dstat;
    cudaError_t e = dnew<double>(dstat, (size_t)kStatWarps * 2 * kSamp);
    if (e != cudaSuccess) return from_cuda(e);
    k_feature_stats<<<kStatBlocks, kStatThreads, 0, st>>>(samples, n, (double *)dstat.p);
    std::vector<double> parts((size_t)kStatWarps * 2 * kSamp);
    e = cudaMemcpyAsync(parts.data(), dstat.p, sizeof(double) * parts.size(),
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return from_cuda(e);
    double stat[2 * kSamp] = {0};
    for (int w = 0; w < kStatWarps; ++w)
        for (int k = 0; k < 2 * kSamp; ++k) stat[k] += parts[(size_t)w * 2 * kSamp + k];
    for (int k = 0; k < NI; ++k) {
        const double m = stat[k] / (double)n;
        const double var = std::max(stat[kSamp + k] / (double)n - m * m, 0.0);
        mu[k] = (float)m;
        isd[k] = var > 1e-30 ? (float)(1.0 / std::sqrt(var)) : 1.0f;
    }
    {
        const double m = stat[NI] / (double)n;
        const double sd = std::sqrt(std::max(stat[kSamp + NI] / (double)n - m * m, 0.0));
        y_range[0] = (float)(m / 16.0);
        y_range[1] = (float)(m + 4.0 * sd);
    }
    // relative error: labels below the output range's floor count as the floor
    const float rel_floor = loss_kind == LVB_MLP_LOSS_RELATIVE ? std::max(y_range[0], 1e-30f)
                                                               : 0.0f;
    DevBuf dp, dmu, disd, dg, dm, dv, dl, dord;
    e = dnew<float>(dp, NP);
    if (e == cudaSuccess) e = dnew<float>(dmu, NI);
    if (e == cudaSuccess) e = dnew<float>(disd, NI);
    if (e == cudaSuccess) e = dnew<float>(dg, (size_t)((batch + kTB - 1) / kTB) * NP);
    if (e == cudaSuccess) e = dnew<float>(dm, NP);
    if (e == cudaSuccess) e = dnew<float>(dv, NP);
    if (e == cudaSuccess) e = dnew<double>(dl, 1);
    if (e == cudaSuccess) e = dnew<int>(dord, (size_t)n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp.p, params, NP * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dmu.p, mu, NI * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(disd.p, isd, NI * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dm.p, 0, NP * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dv.p, 0, NP * 4, st);
    if (e != cudaSuccess) return from_cuda(e);
    std::vector<int> order((size_t)n);
    for (int64_t i = 0; i < n; ++i) order[(size_t)i] = (int)i;
    std::mt19937_64 rng(seed);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    int64_t t = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(order.begin(), order.end(), rng);
        e = cudaMemcpyAsync(dord.p, order.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice,
                            st);
        if (e == cudaSuccess) e = cudaMemsetAsync(dl.p, 0, 8, st);
        if (e != cudaSuccess) return from_cuda(e);
        for (int64_t first = 0; first < n; first += batch) {
            const int64_t cnt = std::min<int64_t>(batch, n - first);
            const int nb = launch_batch(samples, (const int *)dord.p, first, cnt, cnt,
                                        (const float *)dp.p, (const float *)dmu.p,
                                        (const float *)disd.p, (float *)dg.p, (double *)dl.p,
                                        rel_floor, st);
            ++t;
            const float c1 = 1.0f - std::pow(b1, (float)t), c2 = 1.0f - std::pow(b2, (float)t);
            k_adam<<<(NP + 255) / 256, 256, 0, st>>>((float *)dp.p, (const float *)dg.p, nb,
                                                     (float *)dm.p, (float *)dv.p, NP, lr, b1, b2,
                                                     eps, c1, c2);
        }
        double sse = 0.0;
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&sse, dl.p, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return from_cuda(e);
        if (losses) losses[ep] = (float)(sse / (double)n);
    }
    e = cudaMemcpyAsync(params, dp.p, NP * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return from_cuda(e);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Travel-form labels (lvb_mlp_travel_labels): samples with f0 > 0 kept in
// their order (chunked stable compaction: block b owns a contiguous chunk
// and writes its kept samples after those of the blocks before it), label
// t -> (t * margin) / (f0 * horizon), then clipped at an order statistic
// found by bisection over the binary32 bit patterns (non-negative values
// order like their bits).
// ---------------------------------------------------------------------------
namespace {

constexpr int kTlThreads = 256;
constexpr int kTlBlocks = 256;

__device__ __forceinline__ bool tl_keep(const float *s) { return s[0] > 0.0f; }

__global__ void __launch_bounds__(kTlThreads)
k_tl_count(const float *__restrict__ smp, int64_t n, int64_t chunk, int *blk_cnt)
{
    const int64_t a = (int64_t)blockIdx.x * chunk, b = min(n, a + chunk);
    int c = 0;
    for (int64_t i = a + threadIdx.x; i < b; i += kTlThreads) c += tl_keep(smp + i * kSamp);
    __shared__ int ws[kTlThreads / 32];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kTlThreads / 32; ++w) t += ws[w];
        blk_cnt[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kTlThreads)
k_tl_scatter(const float *__restrict__ smp, int64_t n, int64_t chunk, const int *blk_cnt,
             int horizon, float margin, float *__restrict__ out)
{
    __shared__ int ws[kTlThreads / 32];
    __shared__ int s_base;
    if (threadIdx.x == 0) {
        int base = 0;
        for (int q = 0; q < (int)blockIdx.x; ++q) base += blk_cnt[q];
        s_base = base;
    }
    __syncthreads();
    int base = s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t a = (int64_t)blockIdx.x * chunk, b = min(n, a + chunk);
    const float hz = (float)horizon;
    for (int64_t t0 = a; t0 < b; t0 += kTlThreads) {
        const int64_t i = t0 + threadIdx.x;
        const bool keep = i < b && tl_keep(smp + i * kSamp);
        const unsigned m = __ballot_sync(FULL, keep);
        if (lane == 0) ws[warp] = __popc(m);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < kTlThreads / 32; ++w) {
            before += w < warp ? ws[w] : 0;
            total += ws[w];
        }
        if (keep) {
            const float *s = smp + i * kSamp;
            float *o = out + (int64_t)(base + before + __popc(m & lanemask_lt())) * kSamp;
#pragma unroll
            for (int k = 0; k < NI; ++k) o[k] = s[k];
            o[NI] = __fdiv_rn(__fmul_rn(s[NI], margin), __fmul_rn(s[0], hz));
        }
        base += total;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kTlThreads)
k_tl_count_le(const float *__restrict__ out, int64_t m, unsigned t, unsigned long long *cnt)
{
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * kTlThreads + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * kTlThreads)
        c += __float_as_uint(out[i * kSamp + NI]) <= t;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

__global__ void __launch_bounds__(kTlThreads)
k_tl_clip(float *out, int64_t m, float c)
{
    for (int64_t i = (int64_t)blockIdx.x * kTlThreads + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * kTlThreads)
        out[i * kSamp + NI] = fminf(out[i * kSamp + NI], c);
}

}  // namespace

extern "C" int lvb_mlp_travel_labels(const float *samples, int64_t n, int32_t horizon,
                                     float margin, float clip_q, float *out, int64_t *n_out,
                                     void *stream)
{
    if (n_out) *n_out = 0;
    if (!samples || !out || !n_out || n < 0 || horizon < 1 || samples == out) return LVB_EINVAL;
    if (!(margin > 0.0f) || !std::isfinite(margin) || !(clip_q > 0.0f) || !(clip_q <= 1.0f))
        return LVB_EINVAL;
    if (n == 0) return LVB_OK;
    const cudaStream_t st = (cudaStream_t)stream;
    const int64_t chunk = (n + kTlBlocks - 1) / kTlBlocks;
    int *blk = nullptr;
    unsigned long long *cnt = nullptr;
    cudaError_t e = cudaMalloc((void **)&blk, sizeof(int) * kTlBlocks);
    if (e == cudaSuccess) e = cudaMalloc((void **)&cnt, sizeof(unsigned long long));
    auto done = [&](int rc) {
        cudaStreamSynchronize(st);
        if (blk) cudaFree(blk);
        if (cnt) cudaFree(cnt);
        return rc;
    };
    if (e != cudaSuccess) return done(e == cudaErrorMemoryAllocation ? LVB_ENOMEM : LVB_EDEVICE);
    k_tl_count<<<kTlBlocks, kTlThreads, 0, st>>>(samples, n, chunk, blk);
    k_tl_scatter<<<kTlBlocks, kTlThreads, 0, st>>>(samples, n, chunk, blk, horizon, margin, out);
    std::vector<int> bc(kTlBlocks);
    e = cudaMemcpyAsync(bc.data(), blk, sizeof(int) * kTlBlocks, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return done(LVB_EDEVICE);
    int64_t m = 0;
    for (int v : bc) m += v;
    if (m > 0) {
        // order statistic k (0-based, ascending): the smallest bit pattern
        // t with at least k + 1 labels <= t
        const int64_t k = (int64_t)std::floor((double)clip_q * (double)(m - 1));
        const int g = (int)std::min<int64_t>((m + kTlThreads - 1) / kTlThreads, 4 * 152);
        unsigned lo = 0u, hi = 0x7fffffffu;
        while (lo < hi && e == cudaSuccess) {
            const unsigned mid = lo + (hi - lo) / 2;
            unsigned long long c = 0;
            e = cudaMemsetAsync(cnt, 0, sizeof(c), st);
            if (e == cudaSuccess) {
                k_tl_count_le<<<g, kTlThreads, 0, st>>>(out, m, mid, cnt);
                e = cudaMemcpyAsync(&c, cnt, sizeof(c), cudaMemcpyDeviceToHost, st);
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if ((int64_t)c >= k + 1) hi = mid;
            else lo = mid + 1;
        }
        if (e != cudaSuccess) return done(LVB_EDEVICE);
        float c;
        memcpy(&c, &lo, sizeof(c));
        k_tl_clip<<<g, kTlThreads, 0, st>>>(out, m, c);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return done(LVB_EDEVICE);
    *n_out = m;
    return done(LVB_OK);
}
