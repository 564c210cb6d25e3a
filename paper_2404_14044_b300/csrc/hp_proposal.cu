// Learned depth-interval proposal (an extension beyond the paper, in the
// spirit of the learned samplers it cites as related work): a 16 -> 32 -> 32
// -> 2 MLP maps a ray's depth histogram -- camera depths of the points in the
// 3 x 3 buckets around its pixel, 16 bins over [t_near, t_far], log(1 + n) --
// to an interval [t0, t1] that should hold the ray's primary-surface samples.
//
// k_prop_infer   one thread per ray: histogram from the table, MLP with BF16
//                weights and FP32 accumulation, interval out; a ray with no
//                point around its pixel gets the full [t_near, t_far].
// k_prop_train   one thread per ray of a training batch: the same forward in
//                FP32 (master weights), an asymmetric interval loss against the
//                first / last sample depth the plain search found, backward;
//                weight gradients are summed per warp with shuffles and added
//                to a global gradient buffer.
// k_prop_adam    Adam step on the FP32 master weights, refreshes the BF16 copy
//                and clears the gradient.
#include <cuda_bf16.h>

#include "hp_kernels.cuh"
#include "hp_proposal.cuh"

namespace hp {

namespace {

using namespace prop;

// Loss shape: softplus hinges (sharpness kKappa) that push t0 below the first
// sample and t1 above the last by kMargin (fractions of t_far - t_near), plus
// kLambda times the interval width.
constexpr float kKappa = 200.0f, kMargin = 0.01f, kLambda = 0.05f;

__device__ __forceinline__ int ray_pixel(const PropArgs &a, int64_t r) { return a.rays ? a.rays[r] : (int)r; }

}  // namespace

__global__ void __launch_bounds__(256, 4) k_prop_infer(const PropArgs a)
{
    grid_dep_wait();
    grid_dep_trigger();
    __shared__ __align__(16) float w[kImage];
    load_weights(a.weights_bf16, w);
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.R) return;
    const int pix = ray_pixel(a, r);
    const int64_t npix = (int64_t)a.cam.width * a.cam.height;
    if (pix < 0 || pix >= npix) {
        a.interval[r] = make_float2(a.cam.t_near, a.cam.t_far);
        return;
    }
    const int pv = pix / a.cam.width, pu = pix - pv * a.cam.width;
    float x[kIn];
    histogram(a.cam, a.start, a.spts, a.h, a.Wp, a.Hp, pu, pv, x);
    a.interval[r] = interval(w, x, a.cam);
}

__global__ void __launch_bounds__(256) k_prop_train(const PropArgs a)
{
    grid_dep_wait();
    grid_dep_trigger();
    __shared__ float w[kNP];
    for (int e = threadIdx.x; e < kNP; e += blockDim.x) w[e] = a.params[e];
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool active = r < a.R;
    float x[kIn], h1[kHid], h2[kHid];
    float s0 = 0.f, s1 = 0.f;
    if (active) {
        const int pix = ray_pixel(a, r);
        const int n = a.n_s[r];
        active = n > 0 && pix >= 0 && pix < a.cam.width * a.cam.height;
        if (active) {
            const int64_t o = a.sample_offset[r];
            s0 = a.t[o];
            s1 = a.t[o + n - 1];
            const int pv = pix / a.cam.width, pu = pix - pv * a.cam.width;
            histogram(a.cam, a.start, a.spts, a.h, a.Wp, a.Hp, pu, pv, x);
#pragma unroll
            for (int b = 0; b < kIn; ++b) x[b] = log1pf(x[b]);
        }
    }
    float g[kNP];   // per-thread gradient (registers / local)
    float loss = 0.0f;
    if (active) {
        for (int o = 0; o < kHid; ++o) {
            float z = w[oB0 + o];
            for (int i = 0; i < kIn; ++i) z = fmaf(w[oW0 + o * kIn + i], x[i], z);
            h1[o] = fmaxf(z, 0.0f);
        }
        for (int o = 0; o < kHid; ++o) {
            float z = w[oB1 + o];
            for (int i = 0; i < kHid; ++i) z = fmaf(w[oW1 + o * kHid + i], h1[i], z);
            h2[o] = fmaxf(z, 0.0f);
        }
        float o0 = w[oB2], o1 = w[oB2 + 1];
        for (int i = 0; i < kHid; ++i) {
            o0 = fmaf(w[oW2 + i], h2[i], o0);
            o1 = fmaf(w[oW2 + kHid + i], h2[i], o1);
        }
        const float span = a.cam.t_far - a.cam.t_near;
        const float u0 = sigm(o0), u1 = sigm(o1);
        const float t0n = u0, t1n = u0 + (1.0f - u0) * u1;
        const float s0n = (s0 - a.cam.t_near) / span, s1n = (s1 - a.cam.t_near) / span;
        const float e0 = kKappa * (t0n - s0n + kMargin), e1 = kKappa * (s1n - t1n + kMargin);
        loss = (log1pf(expf(-fabsf(e0))) + fmaxf(e0, 0.0f) + log1pf(expf(-fabsf(e1))) + fmaxf(e1, 0.0f)) / kKappa +
               kLambda * (t1n - t0n);
        const float gt0 = sigm(e0) - kLambda, gt1 = -sigm(e1) + kLambda;
        const float gu0 = gt0 + gt1 * (1.0f - u1), gu1 = gt1 * (1.0f - u0);
        const float go0 = gu0 * u0 * (1.0f - u0), go1 = gu1 * u1 * (1.0f - u1);
        float gh2[kHid], gh1[kHid];
        g[oB2] = go0;
        g[oB2 + 1] = go1;
        for (int i = 0; i < kHid; ++i) {
            g[oW2 + i] = go0 * h2[i];
            g[oW2 + kHid + i] = go1 * h2[i];
            gh2[i] = h2[i] > 0.0f ? (w[oW2 + i] * go0 + w[oW2 + kHid + i] * go1) : 0.0f;
        }
        for (int i = 0; i < kHid; ++i) gh1[i] = 0.0f;
        for (int o = 0; o < kHid; ++o) {
            g[oB1 + o] = gh2[o];
            for (int i = 0; i < kHid; ++i) {
                g[oW1 + o * kHid + i] = gh2[o] * h1[i];
                gh1[i] = fmaf(w[oW1 + o * kHid + i], gh2[o], gh1[i]);
            }
        }
        for (int o = 0; o < kHid; ++o) {
            const float gz = h1[o] > 0.0f ? gh1[o] : 0.0f;
            g[oB0 + o] = gz;
            for (int i = 0; i < kIn; ++i) g[oW0 + o * kIn + i] = gz * x[i];
        }
    } else {
        for (int e = 0; e < kNP; ++e) g[e] = 0.0f;
    }
    // warp sums, one atomic per weight per warp
    for (int e = 0; e < kNP; ++e) {
        float v = g[e];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0 && v != 0.0f) atomicAdd(a.grad + e, v);
    }
    for (int off = 16; off > 0; off >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, off);
    int cnt = active ? 1 : 0;
    for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
    if (lane == 0 && a.loss) {
        atomicAdd(a.loss, loss);
        atomicAdd(a.loss + 1, (float)cnt);
    }
}

// Adam (Kingma & Ba 2015) on the FP32 master weights; gradient = sum / count.
__global__ void k_prop_adam(float *params, float *grad, float *m, float *v, uint16_t *bf16, const float *loss_cnt,
                            int step, float lr)
{
    grid_dep_wait();
    grid_dep_trigger();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kNP) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float n = loss_cnt ? fmaxf(loss_cnt[1], 1.0f) : 1.0f;
    const float gr = grad[e] / n;
    const float mm = b1 * m[e] + (1.0f - b1) * gr;
    const float vv = b2 * v[e] + (1.0f - b2) * gr * gr;
    m[e] = mm;
    v[e] = vv;
    const float mh = mm / (1.0f - powf(b1, (float)step)), vh = vv / (1.0f - powf(b2, (float)step));
    const float p = params[e] - lr * mh / (sqrtf(vh) + eps);
    params[e] = p;
    const __nv_bfloat16 b = __float2bfloat16_rn(p);
    bf16[e] = *reinterpret_cast<const uint16_t *>(&b);
    grad[e] = 0.0f;
}

cudaError_t launch_prop_infer(const PropArgs &a, cudaStream_t st, Prof *prof)
{
    if (a.R <= 0) return cudaSuccess;
    prof_begin(prof, st, KID_PROP_INFER);
    launch_chained(k_prop_infer, (unsigned)div_up(a.R, 256), 256, 0, st, a);
    prof_end(prof, st);
    return cudaGetLastError();
}

cudaError_t launch_prop_train(const PropArgs &a, float *m, float *v, int step, float lr, cudaStream_t st)
{
    cudaError_t e;
    if (a.loss && (e = cudaMemsetAsync(a.loss, 0, 2 * sizeof(float), st)) != cudaSuccess) return e;
    if (a.R > 0) {
        launch_chained(k_prop_train, (unsigned)div_up(a.R, 256), 256, 0, st, a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    launch_chained(k_prop_adam, (unsigned)div_up(kNP, 256), 256, 0, st, a.params, a.grad, m, v, a.weights_out, a.loss, step, lr);
    return cudaGetLastError();
}

}  // namespace hp
