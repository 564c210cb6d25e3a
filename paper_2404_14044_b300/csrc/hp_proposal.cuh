// Learned depth-interval proposal: the per-ray histogram input and the
// network's forward pass, shared by the inference kernel and the fused
// learned search so that both produce identical intervals.
//
// Input: camera depths of the points in the 3 x 3 buckets around the ray's
// pixel, 16 bins over [t_near, t_far], x_b = log(1 + n_b).  Network
// 16 -> 32 -> 32 -> 2 (ReLU); t0 = t_near + (t_far - t_near) sigmoid(o0),
// t1 = t0 + (t_far - t0) sigmoid(o1).  A ray with no point around its pixel
// gets [t_near, t_far].  This component is not in the paper: it extends the
// method towards the learned ray samplers the paper cites as related work.
#pragma once

#include "hp_common.cuh"

namespace hp {
namespace prop {

constexpr int kIn = HP_PROP_BINS, kHid = 32;
constexpr int oW0 = 0, oB0 = oW0 + kHid * kIn, oW1 = oB0 + kHid, oB1 = oW1 + kHid * kHid, oW2 = oB1 + kHid,
              oB2 = oW2 + 2 * kHid, kNP = oB2 + 2;
static_assert(kNP == HP_PROP_PARAMS, "parameter count");

// Depth histogram of the 3 x 3 buckets around padded pixel (pu + h, pv + h).
__device__ __forceinline__ void histogram(const Cam &cam, const uint32_t *start, const float4 *spts, int h, int Wp,
                                          int Hp, int pu, int pv, float (&x)[kIn])
{
#pragma unroll
    for (int b = 0; b < kIn; ++b) x[b] = 0.0f;
    const float scale = (float)kIn / (cam.t_far - cam.t_near);
    uint32_t lo[3], hi[3];
    const int c0 = max(pu + h - 1, 0), c1 = min(pu + h + 1, Wp - 1);
#pragma unroll
    for (int q = 0; q < 3; ++q) {                      // the three row runs, loads issued together
        const int row = pv + h + q - 1;
        lo[q] = hi[q] = 0;
        if (row >= 0 && row < Hp) {
            const int64_t k0 = (int64_t)row * Wp;
            lo[q] = __ldg(start + k0 + c0);
            hi[q] = __ldg(start + k0 + c1 + 1);
        }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
#pragma unroll 4
        for (uint32_t i = lo[q]; i < hi[q]; ++i) {
            const float z = __ldg(&spts[i].z);
            int b = (int)floorf((z - cam.t_near) * scale);
            b = b < 0 ? 0 : (b >= kIn ? kIn - 1 : b);
            // registers need static indices: accumulate through a compare chain
#pragma unroll
            for (int r = 0; r < kIn; ++r) x[r] += (r == b) ? 1.0f : 0.0f;
        }
    }
#pragma unroll
    for (int b = 0; b < kIn; ++b) x[b] = log1pf(x[b]);
}

__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + expf(-x)); }

// Interval from the histogram features x; w: the network's weights as FP32
// in shared memory (rows of W are multiples of 4 floats, 16-byte aligned).
__device__ __forceinline__ float2 interval(const float *w, const float (&x)[kIn], const Cam &cam)
{
    float any = 0.0f;
#pragma unroll
    for (int b = 0; b < kIn; ++b) any += x[b];
    if (any == 0.0f) return make_float2(cam.t_near, cam.t_far);   // no point around the pixel
    const float4 *w4 = reinterpret_cast<const float4 *>(w);
    float h1[kHid];
#pragma unroll
    for (int o = 0; o < kHid; ++o) {
        float z = w[oB0 + o];
#pragma unroll
        for (int i = 0; i < kIn; i += 4) {
            const float4 q = w4[(oW0 + o * kIn + i) / 4];
            z = fmaf(q.x, x[i], z);
            z = fmaf(q.y, x[i + 1], z);
            z = fmaf(q.z, x[i + 2], z);
            z = fmaf(q.w, x[i + 3], z);
        }
        h1[o] = fmaxf(z, 0.0f);
    }
    // second hidden layer and output layer together: each h2 value is used
    // as soon as it is formed (no h2 array)
    float o0 = w[oB2], o1 = w[oB2 + 1];
#pragma unroll 4
    for (int o = 0; o < kHid; ++o) {
        float z = w[oB1 + o];
#pragma unroll
        for (int i = 0; i < kHid; i += 4) {
            const float4 q = w4[(oW1 + o * kHid + i) / 4];
            z = fmaf(q.x, h1[i], z);
            z = fmaf(q.y, h1[i + 1], z);
            z = fmaf(q.z, h1[i + 2], z);
            z = fmaf(q.w, h1[i + 3], z);
        }
        const float h2 = fmaxf(z, 0.0f);
        o0 = fmaf(w[oW2 + o], h2, o0);
        o1 = fmaf(w[oW2 + kHid + o], h2, o1);
    }
    const float u0 = sigm(o0), u1 = sigm(o1);
    const float span = cam.t_far - cam.t_near;
    const float t0 = cam.t_near + span * u0;
    const float t1 = t0 + (cam.t_far - t0) * u1;
    return make_float2(t0, t1);
}

// BF16 weights (global) -> FP32 in shared memory, by the whole block.
__device__ __forceinline__ void load_weights(const uint16_t *w_bf16, float *w)
{
    for (int e = threadIdx.x; e < kNP; e += blockDim.x)
        w[e] = __uint_as_float((uint32_t)__ldg(w_bf16 + e) << 16);
}

}  // namespace prop
}  // namespace hp
