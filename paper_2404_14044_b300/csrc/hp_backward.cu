// Backward of the integration stage (Sec. 3.4, Eq. 2) with respect to the
// point features and the point positions, the discrete structure (neighbour
// sets, samples) held fixed.
//
// K9a k_composite_bwd (one thread per ray): from dL/dc and dL/dW of the ray
//     and the forward's per-sample (sigma, colour) and Delta, the gradients of
//     Eq. 2: with E_j = exp(-sigma_j Delta_j), tau_j, w'_j = tau_j (1 - E_j) and
//     g_j = dL/dw'_j, dL/dsigma_j = Delta_j (g_j tau_j E_j - sum_{k>j} g_k w'_k)
//     and dL/dDelta_j likewise with sigma_j; writes dL/d(MLP output) per
//     sample and the part of dL/dt_j that comes through the Delta's.
// K9b k_decode_bwd (persistent, 32-sample tiles, lane = sample): recomputes
//     the IDW features and the hidden pre-activation signs (warp ballots),
//     back-propagates through the MLP (FP32), then scatters
//     dL/df_i = (w_ij / W_j) dL/df_j and, through the inverse-distance
//     weights and t_j (x_j = t_j d, t_j = <P_src, d>), the position gradients
//     (camera space, turned to world space with R^T) with atomic adds.
#include "hp_kernels.cuh"

namespace hp {

namespace {

constexpr int kBwdTile = 32;
constexpr int kBwdThreads = 128;

struct BwdLayout {
    int woff[HP_MLP_MAX_LAYERS], boff[HP_MLP_MAX_LAYERS];
    int n_params, maxw;
    size_t feat, h, dz, dh, mask, wsum, total;
};

BwdLayout bwd_layout(const BwdArgs &a)
{
    BwdLayout L{};
    int o = 0, maxw = a.F;
    for (int l = 0; l < a.n_layers; ++l) {
        L.woff[l] = o;
        o += a.dims[l] * a.dims[l + 1];
        L.boff[l] = o;
        o += a.dims[l + 1];
        maxw = maxw > a.dims[l] ? maxw : a.dims[l];
    }
    L.n_params = o;
    L.maxw = maxw;
    size_t b = ((size_t)o * 4 + 15) & ~size_t(15);
    L.feat = b;  b += (size_t)a.F * kBwdTile * 4;
    L.h = b;     b += (size_t)maxw * kBwdTile * 4;
    L.dz = b;    b += (size_t)maxw * kBwdTile * 4;
    L.dh = b;    b += (size_t)maxw * kBwdTile * 4;
    L.mask = b;  b += (size_t)HP_MLP_MAX_LAYERS * 128 * 4;
    L.wsum = b;  b += kBwdTile * 4;
    L.total = b;
    return L;
}

__device__ __forceinline__ void add_world(float *gp, int id, const Cam &cam, float gx, float gy, float gz)
{
    // dL/dp_world = R^T dL/dP_camera
    atomicAdd(gp + 3 * (int64_t)id + 0, cam.R[0] * gx + cam.R[3] * gy + cam.R[6] * gz);
    atomicAdd(gp + 3 * (int64_t)id + 1, cam.R[1] * gx + cam.R[4] * gy + cam.R[7] * gz);
    atomicAdd(gp + 3 * (int64_t)id + 2, cam.R[2] * gx + cam.R[5] * gy + cam.R[8] * gz);
}

}  // namespace

__global__ void __launch_bounds__(256) k_composite_bwd(const BwdArgs a)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.R) return;
    const int64_t o = __ldg(a.sample_offset + r);
    int n = __ldg(a.n_s + r);
    if (o + n > a.capacity) n = (int)(a.capacity > o ? a.capacity - o : 0);
    if (n == 0) return;
    const float bg = a.bg_mode == 1 ? 1.0f : 0.0f;
    const float g0 = a.grad_rgb[3 * r], g1 = a.grad_rgb[3 * r + 1], g2 = a.grad_rgb[3 * r + 2];
    const float gW = a.grad_wsum ? a.grad_wsum[r] : 0.0f;
    float sig[kMaxSamples], dl[kMaxSamples], E[kMaxSamples], tau[kMaxSamples], wp[kMaxSamples], gw[kMaxSamples];
    float4 so[kMaxSamples];
    float T = 1.0f;
    for (int j = 0; j < n; ++j) {
        so[j] = a.sample_out[o + j];
        sig[j] = so[j].x;
        dl[j] = a.delta[o + j];
        E[j] = expf(-sig[j] * dl[j]);
        tau[j] = T;
        wp[j] = T * -expm1f(-sig[j] * dl[j]);
        gw[j] = g0 * (so[j].y - bg) + g1 * (so[j].z - bg) + g2 * (so[j].w - bg) + gW;
        T *= E[j];
    }
    // cone coefficient of this ray (for Delta_last = 2 t c)
    float cone = 0.0f;
    if (a.mode != HP_RADIUS_FIXED) {
        const int pix = a.rays ? a.rays[r] : (int)r;
        cone = a.raytab[pix].w;
    }
    float suffix = 0.0f, gdel[kMaxSamples];
    for (int j = n - 1; j >= 0; --j) {
        const float bracket = gw[j] * tau[j] * E[j] - suffix;      // suffix = sum_{k>j} g_k w'_k
        const float gsig = bracket * dl[j];
        gdel[j] = bracket * sig[j];
        suffix += gw[j] * wp[j];
        // softplus' = sigmoid(logit) = 1 - exp(-sigma); sigmoid' = c (1 - c)
        const float sp = -expm1f(-sig[j]);
        a.go[o + j] = make_float4(gsig * sp, g0 * wp[j] * so[j].y * (1.0f - so[j].y),
                                  g1 * wp[j] * so[j].z * (1.0f - so[j].z), g2 * wp[j] * so[j].w * (1.0f - so[j].w));
    }
    // Delta_j = t_{j+1} - t_j, Delta_last = 2 r (fixed) or 2 t c (cone)
    for (int j = 0; j < n; ++j) {
        float gt = j > 0 ? gdel[j - 1] : 0.0f;
        if (j + 1 < n) gt -= gdel[j];
        else if (a.mode != HP_RADIUS_FIXED) gt += gdel[j] * 2.0f * cone;
        a.gt[o + j] = gt;
    }
}

__global__ void __launch_bounds__(kBwdThreads) k_decode_bwd(const BwdArgs a, const BwdLayout L)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float *prm = reinterpret_cast<float *>(smem);              // W^T [in][out] per layer, then biases
    float *feat = reinterpret_cast<float *>(smem + L.feat);    // [F][32]
    float *hb = reinterpret_cast<float *>(smem + L.h);         // [w][32]
    float *dz = reinterpret_cast<float *>(smem + L.dz);
    float *dh = reinterpret_cast<float *>(smem + L.dh);
    uint32_t *mask = reinterpret_cast<uint32_t *>(smem + L.mask);   // [layer][128] sample bits
    float *Wsum = reinterpret_cast<float *>(smem + L.wsum);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        int g = 0;
        for (int l = 0; l < a.n_layers; ++l) {
            const int fi = a.dims[l], fo = a.dims[l + 1], nw = fi * fo;
            for (int e = tid; e < nw; e += blockDim.x) {
                const int oo = e / fi, ii = e - oo * fi;
                prm[L.woff[l] + ii * fo + oo] = __ldg(a.mlp + g + e);
            }
            g += nw;
            for (int e = tid; e < fo; e += blockDim.x) prm[L.boff[l] + e] = __ldg(a.mlp + g + e);
            g += fo;
        }
    }
    __syncthreads();
    const int64_t S_all = __ldg(a.sample_offset + a.R);
    const int64_t S = S_all < a.capacity ? S_all : a.capacity;
    const int F = a.F, K = a.K, NL = a.n_layers;
    const int nwarps = kBwdThreads / 32;

    for (int64_t base = (int64_t)blockIdx.x * kBwdTile; base < S; base += (int64_t)gridDim.x * kBwdTile) {
        // ---- IDW features [F][32] (warp w: samples w, w+4, ...; lanes over features)
        for (int s = warp; s < kBwdTile; s += nwarps) {
            const int64_t g = base + s;
            for (int k = lane; k < F; k += 32) {
                float acc = 0.0f, W = 0.0f;
                if (g < S) {
                    for (int m = 0; m < K; ++m) {
                        const int id = __ldg(a.nbr + g * K + m);
                        if (id < 0) continue;
                        const float w = 1.0f / fmaxf(__ldg(a.nbr_dist + g * K + m), a.eps_d);
                        acc = fmaf(w, __ldg(a.feats + (int64_t)id * F + k), acc);
                        W += w;
                    }
                }
                feat[k * kBwdTile + s] = g < S ? acc / W : 0.0f;
                if (k == 0) Wsum[s] = W;
            }
        }
        __syncthreads();
        // ---- forward through the hidden layers for the ReLU masks (lane = sample)
        const float *in = feat;
        for (int l = 0; l + 1 < NL; ++l) {
            const int fi = a.dims[l], fo = a.dims[l + 1];
            const float *Wt = prm + L.woff[l];
            for (int oo = warp; oo < fo; oo += nwarps) {
                float z = prm[L.boff[l] + oo];
                for (int i = 0; i < fi; ++i) z = fmaf(Wt[i * fo + oo], in[i * kBwdTile + lane], z);
                const unsigned bits = __ballot_sync(0xffffffffu, z > 0.0f);
                if (lane == 0) mask[l * 128 + oo] = bits;
                hb[oo * kBwdTile + lane] = fmaxf(z, 0.0f);
            }
            __syncthreads();
            // next layer's input: copy h into dz scratch so hb can be rewritten
            for (int e = tid; e < fo * kBwdTile; e += blockDim.x) dh[e] = hb[e];
            __syncthreads();
            in = dh;
        }
        // ---- backward: dz of the output layer = dL/do
        for (int e = tid; e < 4 * kBwdTile; e += blockDim.x) {
            const int c = e / kBwdTile, s = e - c * kBwdTile;
            const int64_t g = base + s;
            float v = 0.0f;
            if (g < S) {
                const float4 go = a.go[g];
                v = c == 0 ? go.x : c == 1 ? go.y : c == 2 ? go.z : go.w;
            }
            dz[c * kBwdTile + s] = v;
        }
        __syncthreads();
        for (int l = NL - 1; l >= 0; --l) {
            const int fi = a.dims[l], fo = a.dims[l + 1];
            const float *Wt = prm + L.woff[l];
            for (int i = warp; i < fi; i += nwarps) {
                float acc = 0.0f;
                for (int oo = 0; oo < fo; ++oo) acc = fmaf(Wt[i * fo + oo], dz[oo * kBwdTile + lane], acc);
                hb[i * kBwdTile + lane] = acc;
            }
            __syncthreads();
            if (l > 0) {
                for (int e = tid; e < fi * kBwdTile; e += blockDim.x) {
                    const int i = e / kBwdTile, s = e - i * kBwdTile;
                    dz[e] = ((mask[(l - 1) * 128 + i] >> s) & 1u) ? hb[e] : 0.0f;
                }
                __syncthreads();
            }
        }
        // hb[k][s] = dL/df_j.  IDW backward (warp per sample, lanes over features)
        for (int s = warp; s < kBwdTile; s += nwarps) {
            const int64_t g = base + s;
            if (g >= S) continue;
            const int ray = __ldg(a.ray + g);
            const int pix = a.rays ? __ldg(a.rays + ray) : ray;
            const float4 dd = __ldg(a.raytab + pix);
            const float tj = __ldg(a.t + g);
            const float W = Wsum[s];
            float gx0 = 0.0f, gx1 = 0.0f, gx2 = 0.0f;
            for (int m = 0; m < K; ++m) {
                const int id = __ldg(a.nbr + g * K + m);
                if (id < 0) continue;
                const float dist = __ldg(a.nbr_dist + g * K + m);
                const float w = 1.0f / fmaxf(dist, a.eps_d);
                float gw_part = 0.0f;
                for (int k = lane; k < F; k += 32) {
                    const float dfk = hb[k * kBwdTile + s];
                    if (a.grad_feats) atomicAdd(a.grad_feats + (int64_t)id * F + k, w / W * dfk);
                    gw_part = fmaf(dfk, __ldg(a.feats + (int64_t)id * F + k) - feat[k * kBwdTile + s], gw_part);
                }
                for (int off = 16; off > 0; off >>= 1) gw_part += __shfl_xor_sync(0xffffffffu, gw_part, off);
                if (dist > a.eps_d && a.grad_points && lane == 0) {
                    const float gdist = -(gw_part / W) / (dist * dist);
                    const float3 P = cam_point(a.cam, __ldg(a.points + 3 * (int64_t)id), __ldg(a.points + 3 * (int64_t)id + 1),
                                               __ldg(a.points + 3 * (int64_t)id + 2));
                    const float vx = fmaf(tj, dd.x, -P.x), vy = fmaf(tj, dd.y, -P.y), vz = fmaf(tj, dd.z, -P.z);
                    const float sc = gdist / dist;
                    add_world(a.grad_points, id, a.cam, -sc * vx, -sc * vy, -sc * vz);
                    gx0 = fmaf(sc, vx, gx0);
                    gx1 = fmaf(sc, vy, gx1);
                    gx2 = fmaf(sc, vz, gx2);
                }
            }
            if (a.grad_points && lane == 0) {
                const float gt = a.gt[g] + (gx0 * dd.x + gx1 * dd.y + gx2 * dd.z);
                add_world(a.grad_points, __ldg(a.src + g), a.cam, gt * dd.x, gt * dd.y, gt * dd.z);
            }
        }
        __syncthreads();
    }
}

size_t backward_smem_bytes(const BwdArgs &a) { return bwd_layout(a).total; }

cudaError_t launch_backward(const BwdArgs &a, cudaStream_t st, Prof *prof)
{
    cudaError_t e;
    if (a.R <= 0) return cudaSuccess;
    prof_begin(prof, st, KID_COMPOSITE_BWD);
    k_composite_bwd<<<(unsigned)div_up(a.R, 256), 256, 0, st>>>(a);
    prof_end(prof, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const BwdLayout L = bwd_layout(a);
    if ((e = cudaFuncSetAttribute(k_decode_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total)) !=
        cudaSuccess)
        return e;
    int64_t grid = (int64_t)a.num_sms * 2;
    const int64_t tiles = div_up(a.capacity > 0 ? a.capacity : 1, kBwdTile);
    if (grid > tiles) grid = tiles;
    prof_begin(prof, st, KID_DECODE_BWD);
    k_decode_bwd<<<(unsigned)grid, kBwdThreads, L.total, st>>>(a, L);
    prof_end(prof, st);
    return cudaGetLastError();
}

}  // namespace hp
