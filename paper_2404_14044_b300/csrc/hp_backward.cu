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

constexpr int kBwdTile = 32;         // samples per tile
constexpr int kBwdThreads = 256;     // 8 warps; matmul threads hold 4 samples x 4 units

struct BwdLayout {
    int woff[HP_MLP_MAX_LAYERS], boff[HP_MLP_MAX_LAYERS];   // float offsets of W_l, b_l in the packed parameters
    int maxw;
    size_t feat, act0, act1, dz, dx, mask, wsum, total;
};

// Shared memory: the tile's IDW features [F][32], two activation buffers and
// two gradient buffers [maxw][32] (unit-major, sample-minor), the hidden
// layers' ReLU masks [layer][maxw][32] (bytes) and the IDW weight sums.  The
// weights stay in global memory (read row-wise through L1).
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
        maxw = maxw > a.dims[l + 1] ? maxw : a.dims[l + 1];
    }
    L.maxw = maxw;
    const size_t buf = (size_t)maxw * kBwdTile * 4;
    size_t b = 0;
    L.feat = b;  b += (size_t)a.F * kBwdTile * 4;
    L.act0 = b;  b += buf;
    L.act1 = b;  b += buf;
    L.dz = b;    b += buf;
    L.dx = b;    b += buf;
    L.mask = b;  b += (size_t)(a.n_layers > 1 ? a.n_layers - 1 : 1) * maxw * kBwdTile;
    b = (b + 15) & ~size_t(15);
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
    grid_dep_wait();
    grid_dep_trigger();
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

// out[u][s] = sum_i W[u][i] in[i][s] (+ b[u]) for the tile's 32 samples, u <
// n_out, i < n_in; W row-major [n_out][n_in] in global memory.  Thread t
// holds samples 4 (t % 8) .. +3 and units 4 (t / 8) .. +3 (16 multiply-adds
// per summed index, each output's sum in index order).  When the widths are
// multiples of 4 the weights come as 16-byte loads: forward, four summed
// indices of a unit's row at a time; transposed (the backward through W,
// out[i][s] = sum_u W[u][i] in[u][s]), the four output units of a row.
template <bool kTransposed>
__device__ __forceinline__ void tile_matmul(const float *__restrict__ W, const float *__restrict__ bias, int n_out,
                                            int n_in, const float *in, float (&acc)[4][4], int sb, int ub)
{
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[s][q] = (!kTransposed && bias && 4 * ub + q < n_out) ? __ldg(bias + 4 * ub + q) : 0.0f;
    if (4 * ub >= n_out) return;
    auto fma16 = [&](const float (&w)[4], const float4 x) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            acc[0][q] = fmaf(w[q], x.x, acc[0][q]);
            acc[1][q] = fmaf(w[q], x.y, acc[1][q]);
            acc[2][q] = fmaf(w[q], x.z, acc[2][q]);
            acc[3][q] = fmaf(w[q], x.w, acc[3][q]);
        }
    };
    const bool vec = (n_in & 3) == 0 && (n_out & 3) == 0 && (reinterpret_cast<uintptr_t>(W) & 15) == 0;
    if (vec && kTransposed) {
        // W[k][4ub .. 4ub+3]: one 16-byte load per summed index (eight in flight)
#pragma unroll 8
        for (int k = 0; k < n_in; ++k) {
            const float4 x = *reinterpret_cast<const float4 *>(in + k * kBwdTile + 4 * sb);
            const float4 w4 = __ldg(reinterpret_cast<const float4 *>(W + (int64_t)k * n_out + 4 * ub));
            const float w[4] = {w4.x, w4.y, w4.z, w4.w};
            fma16(w, x);
        }
        return;
    }
    if (vec) {
        // W[4ub + q][k .. k+3]: four 16-byte loads per four summed indices
#pragma unroll 4
        for (int k0 = 0; k0 < n_in; k0 += 4) {
            float4 wr[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                wr[q] = __ldg(reinterpret_cast<const float4 *>(W + (int64_t)(4 * ub + q) * n_in + k0));
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const float4 x = *reinterpret_cast<const float4 *>(in + (k0 + kk) * kBwdTile + 4 * sb);
                float w[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    w[q] = kk == 0 ? wr[q].x : kk == 1 ? wr[q].y : kk == 2 ? wr[q].z : wr[q].w;
                fma16(w, x);
            }
        }
        return;
    }
#pragma unroll 4
    for (int k = 0; k < n_in; ++k) {
        const float4 x = *reinterpret_cast<const float4 *>(in + k * kBwdTile + 4 * sb);
        float w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int u = 4 * ub + q;
            // forward: W[u][k] (row u of n_in); transposed: W[k][u] (row k of n_out)
            w[q] = u < n_out ? __ldg(kTransposed ? W + (int64_t)k * n_out + u : W + (int64_t)u * n_in + k) : 0.0f;
        }
        fma16(w, x);
    }
}

__global__ void __launch_bounds__(kBwdThreads, 2) k_decode_bwd(const BwdArgs a, const BwdLayout L)
{
    grid_dep_wait();
    grid_dep_trigger();
    extern __shared__ __align__(16) unsigned char smem[];
    float *feat = reinterpret_cast<float *>(smem + L.feat);    // [F][32]
    float *act[2] = {reinterpret_cast<float *>(smem + L.act0), reinterpret_cast<float *>(smem + L.act1)};
    float *dzb = reinterpret_cast<float *>(smem + L.dz);
    float *dxb = reinterpret_cast<float *>(smem + L.dx);
    uint8_t *mask = reinterpret_cast<uint8_t *>(smem + L.mask);   // [layer][unit][sample]
    float *Wsum = reinterpret_cast<float *>(smem + L.wsum);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sb = tid & 7, ub = tid >> 3;
    const int64_t S_all = __ldg(a.sample_offset + a.R);
    const int64_t S = S_all < a.capacity ? S_all : a.capacity;
    const int F = a.F, K = a.K, NL = a.n_layers;
    constexpr int kWarps = kBwdThreads / 32;
    constexpr int kNb = 8;                     // neighbours whose loads are in flight together

    for (int64_t base = (int64_t)blockIdx.x * kBwdTile; base < S; base += (int64_t)gridDim.x * kBwdTile) {
        // ---- IDW features [F][32]: a warp per sample, lanes over features;
        // a sample's neighbour ids and distances are read by K lanes at once
        for (int s = warp; s < kBwdTile; s += kWarps) {
            const int64_t g = base + s;
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            float W = 0.0f;
            if (g < S) {
                for (int m0 = 0; m0 < K; m0 += 32) {
                    const int m = m0 + lane;
                    int id_l = m < K ? __ldg(a.nbr + g * K + m) : -1;
                    if (id_l >= 0 && !hp_check(id_l < a.n_points, a.err, id_l)) id_l = -1;
                    const float w_l = id_l >= 0 ? 1.0f / fmaxf(__ldg(a.nbr_dist + g * K + m), a.eps_d) : 0.0f;
                    const int mn = min(32, K - m0);
                    for (int c0 = 0; c0 < mn; c0 += kNb) {
                        float fv[kNb][4];
                        int idv[kNb];
                        float wv[kNb];
#pragma unroll
                        for (int q = 0; q < kNb; ++q) {
                            idv[q] = __shfl_sync(0xffffffffu, id_l, (c0 + q) & 31);
                            wv[q] = __shfl_sync(0xffffffffu, w_l, (c0 + q) & 31);
                            if (c0 + q >= mn) idv[q] = -1;
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const int k = lane + 32 * j;
                                fv[q][j] = (idv[q] >= 0 && k < F) ? __ldg(a.feats + (int64_t)idv[q] * F + k) : 0.0f;
                            }
                        }
#pragma unroll
                        for (int q = 0; q < kNb; ++q) {
                            if (idv[q] < 0) continue;
#pragma unroll
                            for (int j = 0; j < 4; ++j) acc[j] = fmaf(wv[q], fv[q][j], acc[j]);
                            W += wv[q];
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int k = lane + 32 * j;
                if (k < F) feat[k * kBwdTile + s] = g < S ? acc[j] / W : 0.0f;
            }
            if (lane == 0) Wsum[s] = W;
        }
        __syncthreads();
        // ---- forward through the hidden layers: ReLU masks
        const float *in = feat;
        for (int l = 0; l + 1 < NL; ++l) {
            const int fi = a.dims[l], fo = a.dims[l + 1];
            float z[4][4];
            tile_matmul<false>(a.mlp + L.woff[l], a.mlp + L.boff[l], fo, fi, in, z, sb, ub);
            float *out = act[l & 1];
            uint8_t *mk = mask + (size_t)l * L.maxw * kBwdTile;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int u = 4 * ub + q;
                if (u >= fo) break;
                *reinterpret_cast<float4 *>(out + u * kBwdTile + 4 * sb) =
                    make_float4(fmaxf(z[0][q], 0.f), fmaxf(z[1][q], 0.f), fmaxf(z[2][q], 0.f), fmaxf(z[3][q], 0.f));
                *reinterpret_cast<uchar4 *>(mk + u * kBwdTile + 4 * sb) =
                    make_uchar4(z[0][q] > 0.f, z[1][q] > 0.f, z[2][q] > 0.f, z[3][q] > 0.f);
            }
            __syncthreads();
            in = out;
        }
        // ---- backward: the output layer's dz = dL/do
        for (int e = tid; e < 4 * kBwdTile; e += blockDim.x) {
            const int c = e / kBwdTile, s = e - c * kBwdTile;
            const int64_t g = base + s;
            float v = 0.0f;
            if (g < S) {
                const float4 go = a.go[g];
                v = c == 0 ? go.x : c == 1 ? go.y : c == 2 ? go.z : go.w;
            }
            dzb[c * kBwdTile + s] = v;
        }
        __syncthreads();
        float *dz = dzb, *dx = dxb;
        for (int l = NL - 1; l >= 0; --l) {
            const int fi = a.dims[l], fo = a.dims[l + 1];
            float d[4][4];
            tile_matmul<true>(a.mlp + L.woff[l], nullptr, fi, fo, dz, d, sb, ub);
            const uint8_t *mk = l > 0 ? mask + (size_t)(l - 1) * L.maxw * kBwdTile : nullptr;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = 4 * ub + q;
                if (i >= fi) break;
                float4 v = make_float4(d[0][q], d[1][q], d[2][q], d[3][q]);
                if (mk) {
                    const uchar4 m4 = *reinterpret_cast<const uchar4 *>(mk + i * kBwdTile + 4 * sb);
                    v.x = m4.x ? v.x : 0.f;
                    v.y = m4.y ? v.y : 0.f;
                    v.z = m4.z ? v.z : 0.f;
                    v.w = m4.w ? v.w : 0.f;
                }
                *reinterpret_cast<float4 *>(dx + i * kBwdTile + 4 * sb) = v;
            }
            __syncthreads();
            float *tmp = dz;
            dz = dx;
            dx = tmp;
        }
        // dz[k][s] = dL/df_j.  IDW backward (warp per sample, lanes over
        // features, a sample's neighbours kNb at a time with their feature
        // loads in flight together)
        for (int s = warp; s < kBwdTile; s += kWarps) {
            const int64_t g = base + s;
            if (g >= S) continue;
            const int ray = __ldg(a.ray + g);
            const int pix = a.rays ? __ldg(a.rays + ray) : ray;
            const float4 dd = __ldg(a.raytab + pix);
            const float tj = __ldg(a.t + g);
            const float W = Wsum[s];
            float dfk[4], fj[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int k = lane + 32 * j;
                dfk[j] = k < F ? dz[k * kBwdTile + s] : 0.0f;
                fj[j] = k < F ? feat[k * kBwdTile + s] : 0.0f;
            }
            float gx0 = 0.0f, gx1 = 0.0f, gx2 = 0.0f;
            for (int m0 = 0; m0 < K; m0 += 32) {
                const int m = m0 + lane;
                int id_l = m < K ? __ldg(a.nbr + g * K + m) : -1;
                if (id_l >= 0 && !hp_check(id_l < a.n_points, a.err, id_l)) id_l = -1;
                const float d_l = id_l >= 0 ? __ldg(a.nbr_dist + g * K + m) : 1.0f;
                const int mn = min(32, K - m0);
                float sc_l = 0.0f;                   // lane m: dL/d|x_j - P_m| / |x_j - P_m|
                for (int c0 = 0; c0 < mn; c0 += kNb) {
                    float fv[kNb][4];
                    int idv[kNb];
                    float dv[kNb];
#pragma unroll
                    for (int q = 0; q < kNb; ++q) {
                        idv[q] = __shfl_sync(0xffffffffu, id_l, (c0 + q) & 31);
                        dv[q] = __shfl_sync(0xffffffffu, d_l, (c0 + q) & 31);
                        if (c0 + q >= mn) idv[q] = -1;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int k = lane + 32 * j;
                            fv[q][j] = (idv[q] >= 0 && k < F) ? __ldg(a.feats + (int64_t)idv[q] * F + k) : 0.0f;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < kNb; ++q) {
                        const int id = idv[q];
                        if (id < 0) continue;
                        const float dist = dv[q];
                        const float w = 1.0f / fmaxf(dist, a.eps_d);
                        float gw_part = 0.0f;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int k = lane + 32 * j;
                            if (k >= F) break;
                            if (a.grad_feats) atomicAdd(a.grad_feats + (int64_t)id * F + k, w / W * dfk[j]);
                            gw_part = fmaf(dfk[j], fv[q][j] - fj[j], gw_part);
                        }
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1) gw_part += __shfl_xor_sync(0xffffffffu, gw_part, off);
                        // the neighbour's lane keeps its distance gradient
                        if (lane == ((c0 + q) & 31) && dist > a.eps_d) sc_l = (-(gw_part / W) / (dist * dist)) / dist;
                    }
                }
                // position gradients: each lane its own neighbour, the point
                // loads of all lanes in flight together
                if (a.grad_points && m < K && id_l >= 0 && d_l > a.eps_d) {
                    const float3 P = cam_point(a.cam, __ldg(a.points + 3 * (int64_t)id_l),
                                               __ldg(a.points + 3 * (int64_t)id_l + 1),
                                               __ldg(a.points + 3 * (int64_t)id_l + 2));
                    const float vx = fmaf(tj, dd.x, -P.x), vy = fmaf(tj, dd.y, -P.y), vz = fmaf(tj, dd.z, -P.z);
                    add_world(a.grad_points, id_l, a.cam, -sc_l * vx, -sc_l * vy, -sc_l * vz);
                    gx0 = fmaf(sc_l, vx, gx0);
                    gx1 = fmaf(sc_l, vy, gx1);
                    gx2 = fmaf(sc_l, vz, gx2);
                }
            }
            if (a.grad_points) {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    gx0 += __shfl_xor_sync(0xffffffffu, gx0, off);
                    gx1 += __shfl_xor_sync(0xffffffffu, gx1, off);
                    gx2 += __shfl_xor_sync(0xffffffffu, gx2, off);
                }
                if (lane == 0) {
                    const float gt = a.gt[g] + (gx0 * dd.x + gx1 * dd.y + gx2 * dd.z);
                    const int src = __ldg(a.src + g);
                    if (hp_check(src >= 0 && src < a.n_points, a.err, src))
                        add_world(a.grad_points, src, a.cam, gt * dd.x, gt * dd.y, gt * dd.z);
                }
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
    launch_chained(k_composite_bwd, (unsigned)div_up(a.R, 256), 256, 0, st, a);
    prof_end(prof, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const BwdLayout L = bwd_layout(a);
    if ((e = cudaFuncSetAttribute(k_decode_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total)) !=
        cudaSuccess)
        return e;
    int64_t grid = (int64_t)a.num_sms * 2;   // two 256-thread blocks per SM
    const int64_t tiles = div_up(a.capacity > 0 ? a.capacity : 1, kBwdTile);
    if (grid > tiles) grid = tiles;
    prof_begin(prof, st, KID_DECODE_BWD);
    launch_chained(k_decode_bwd, (unsigned)grid, kBwdThreads, L.total, st, a, L);
    prof_end(prof, st);
    return cudaGetLastError();
}

}  // namespace hp
