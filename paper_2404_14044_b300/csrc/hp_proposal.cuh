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
#include "hp_tc.cuh"

namespace hp {
namespace prop {

constexpr int kIn = HP_PROP_BINS, kHid = 32;
constexpr int oW0 = 0, oB0 = oW0 + kHid * kIn, oW1 = oB0 + kHid, oB1 = oW1 + kHid * kHid, oW2 = oB1 + kHid,
              oB2 = oW2 + 2 * kHid, kNP = oB2 + 2;
static_assert(kNP == HP_PROP_PARAMS, "parameter count");
// Counts below kLogTab take log(1 + n) from a table (log1pf of each count,
// written once per block next to the weights); larger counts call log1pf.
constexpr int kLogTab = 256;
// Floats of the inference's shared-memory image: the weights (rearranged,
// see load_weights), then the log table.
constexpr int kImage = kNP + kLogTab;

// Depth histogram of the 3 x 3 buckets around padded pixel (pu + h, pv + h):
// the count of each bin (the network's input is log(1 + count)).
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
}

// x_b = log(1 + n_b), from the table for small counts (the same log1pf
// values the function gives for them).
__device__ __forceinline__ void log_counts(const float *logtab, float (&x)[kIn])
{
#pragma unroll
    for (int b = 0; b < kIn; ++b) x[b] = x[b] < (float)kLogTab ? logtab[(int)x[b]] : log1pf(x[b]);
}

__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + expf(-x)); }

// Interval from the histogram counts x (turned into log(1 + n) here); w:
// the inference image in shared memory (load_weights).  Each unit's sum runs
// over its inputs in order with one FMA per input, two units per packed
// FP32-pair FMA (`fma.rn.f32x2`, each lane rounding as the scalar FMA): the
// same arithmetic as a scalar loop over the units.
__device__ __forceinline__ float2 interval(const float *w, float (&x)[kIn], const Cam &cam)
{
    float any = 0.0f;
#pragma unroll
    for (int b = 0; b < kIn; ++b) any += x[b];
    if (any == 0.0f) return make_float2(cam.t_near, cam.t_far);   // no point around the pixel
    log_counts(w + kNP, x);
    const float4 *w4 = reinterpret_cast<const float4 *>(w);
    // layer 1: W0 transposed ([input][unit]), units in pairs
    uint64_t z1[kHid / 2];
#pragma unroll
    for (int p = 0; p < kHid / 2; ++p) z1[p] = tc::f32x2(w[oB0 + 2 * p], w[oB0 + 2 * p + 1]);
#pragma unroll
    for (int i = 0; i < kIn; ++i) {
        const uint64_t xx = tc::f32x2(x[i], x[i]);
#pragma unroll
        for (int q = 0; q < kHid / 4; ++q) {
            const float4 c = w4[(oW0 + i * kHid) / 4 + q];
            z1[2 * q] = tc::fma_f32x2(tc::f32x2(c.x, c.y), xx, z1[2 * q]);
            z1[2 * q + 1] = tc::fma_f32x2(tc::f32x2(c.z, c.w), xx, z1[2 * q + 1]);
        }
    }
    float h1[kHid];
#pragma unroll
    for (int p = 0; p < kHid / 2; ++p) {
        const float2 v = tc::f32x2_unpack(z1[p]);
        h1[2 * p] = fmaxf(v.x, 0.0f);
        h1[2 * p + 1] = fmaxf(v.y, 0.0f);
    }
    // layer 2 (W1 transposed) in blocks of 8 units, each block's h2 values
    // going straight into the output layer (W2 as (unit 0, unit 1) pairs per
    // input), inputs of the output layer in order
    uint64_t o01 = tc::f32x2(w[oB2], w[oB2 + 1]);
#pragma unroll 1
    for (int ob = 0; ob < kHid; ob += 8) {
        uint64_t z2[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) z2[p] = tc::f32x2(w[oB1 + ob + 2 * p], w[oB1 + ob + 2 * p + 1]);
#pragma unroll
        for (int i = 0; i < kHid; ++i) {
            const uint64_t hh = tc::f32x2(h1[i], h1[i]);
            const float4 c0 = w4[(oW1 + i * kHid + ob) / 4], c1 = w4[(oW1 + i * kHid + ob) / 4 + 1];
            z2[0] = tc::fma_f32x2(tc::f32x2(c0.x, c0.y), hh, z2[0]);
            z2[1] = tc::fma_f32x2(tc::f32x2(c0.z, c0.w), hh, z2[1]);
            z2[2] = tc::fma_f32x2(tc::f32x2(c1.x, c1.y), hh, z2[2]);
            z2[3] = tc::fma_f32x2(tc::f32x2(c1.z, c1.w), hh, z2[3]);
        }
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const float2 v = tc::f32x2_unpack(z2[p]);
            const float2 wa = reinterpret_cast<const float2 *>(w + oW2)[ob + 2 * p];
            const float2 wb = reinterpret_cast<const float2 *>(w + oW2)[ob + 2 * p + 1];
            const float ha = fmaxf(v.x, 0.0f), hb = fmaxf(v.y, 0.0f);
            o01 = tc::fma_f32x2(tc::f32x2(wa.x, wa.y), tc::f32x2(ha, ha), o01);
            o01 = tc::fma_f32x2(tc::f32x2(wb.x, wb.y), tc::f32x2(hb, hb), o01);
        }
    }
    const float2 o = tc::f32x2_unpack(o01);
    const float u0 = sigm(o.x), u1 = sigm(o.y);
    const float span = cam.t_far - cam.t_near;
    const float t0 = cam.t_near + span * u0;
    const float t1 = t0 + (cam.t_far - t0) * u1;
    return make_float2(t0, t1);
}

// The inference image, written by the whole block: the BF16 weights (global,
// in the parameter order W0 [unit][input], b0, W1, b1, W2 [2][unit], b2) as
// FP32 with W0 and W1 transposed to [input][unit] and W2 as one (unit 0,
// unit 1) pair per input, the biases in place; then log1pf(n) for the
// counts n < kLogTab.
__device__ __forceinline__ void load_weights(const uint16_t *w_bf16, float *w)
{
    for (int e = threadIdx.x; e < kNP; e += blockDim.x) {
        const float v = __uint_as_float((uint32_t)__ldg(w_bf16 + e) << 16);
        int d = e;
        if (e < oB0) {
            const int o = (e - oW0) / kIn, i = (e - oW0) - o * kIn;
            d = oW0 + i * kHid + o;
        } else if (e >= oW1 && e < oB1) {
            const int o = (e - oW1) / kHid, i = (e - oW1) - o * kHid;
            d = oW1 + i * kHid + o;
        } else if (e >= oW2 && e < oB2) {
            const int o = (e - oW2) / kHid, i = (e - oW2) - o * kHid;
            d = oW2 + 2 * i + o;
        }
        w[d] = v;
    }
    for (int n = threadIdx.x; n < kLogTab; n += blockDim.x) w[kNP + n] = log1pf((float)n);
}

}  // namespace prop
}  // namespace hp
