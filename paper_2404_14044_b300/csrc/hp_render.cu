// Integration stage (Sec. 3.4): inverse-distance feature aggregation, the
// radiance MLP, and volume rendering (Eq. 2).
//
// K7a k_aggregate_decode (persistent, one block per SM): the MLP weights are
//     staged once per block in shared memory (transposed, W^T[in][out]).  The
//     block then walks 64-sample tiles: each warp gathers its samples'
//     neighbour feature rows with 16-byte loads (F/4 lanes per row, several
//     rows per load instruction), blends them with weights 1/max(dist, eps_d)
//     in registers and writes the aggregated features straight into the
//     shared activation tile -- aggregated features never go to HBM.  The MLP
//     runs tile-wide in FP32 (each thread 4 samples x OPT outputs), and the
//     block writes (sigma, r, g, b) per sample.
// K7b k_composite: one thread per ray, front-to-back Eq. 2 over its samples.
#include "hp_kernels.cuh"

namespace hp {

namespace {

constexpr int kTileS = 64;          // samples per tile
constexpr int kRenderThreads = 256;

struct RenderSmem {
    int woff[HP_MLP_MAX_LAYERS];
    int boff[HP_MLP_MAX_LAYERS];
    int n_params;                    // floats of the staged parameter block
    int maxw;
    size_t xa, xb, total;
};

inline RenderSmem render_layout(const RenderArgs &a)
{
    RenderSmem L;
    int o = 0, maxw = 0;
    for (int l = 0; l < a.n_layers; ++l) {
        const int fi = a.dims[l], fo = a.dims[l + 1];
        L.woff[l] = o;
        o += fi * fo;
        L.boff[l] = o;
        o += fo;
        maxw = maxw > fi ? maxw : fi;
    }
    L.n_params = o;
    L.maxw = maxw;
    L.xa = (size_t)o * 4;
    L.xa = (L.xa + 15) & ~size_t(15);
    L.xb = L.xa + (size_t)maxw * kTileS * 4;
    L.total = L.xb + (size_t)maxw * kTileS * 4;
    return L;
}

// Activation tiles are stored feature-major, X[f][s] with 64 samples per row;
// the 4-sample groups of a row are XOR-swizzled by the row index so that the
// per-layer stores of 16 output rows do not all land on one bank group.
__device__ __forceinline__ int swz(int row) { return ((row >> 3) & 7) << 2; }
__device__ __forceinline__ int xidx(int row, int s) { return row * kTileS + (((s & ~3) ^ swz(row)) | (s & 3)); }

struct LayerDesc {
    int fi, fo, woff, boff;
};

template <int OPT>
__device__ __forceinline__ void dense_relu(const float *__restrict__ prm, const LayerDesc &ld,
                                           const float *__restrict__ in, float *__restrict__ out, int tid)
{
    const int ty = tid >> 4, tx = tid & 15;
    const float *Wt = prm + ld.woff;
    const float *b = prm + ld.boff;
    float acc[4][OPT];
#pragma unroll
    for (int m = 0; m < OPT; ++m) {
        const float bb = b[tx * OPT + m];
#pragma unroll
        for (int s = 0; s < 4; ++s) acc[s][m] = bb;
    }
#pragma unroll 4
    for (int i = 0; i < ld.fi; ++i) {
        const float4 x = *reinterpret_cast<const float4 *>(in + i * kTileS + ((4 * ty) ^ swz(i)));
        float w[OPT];
        if constexpr (OPT >= 4) {
#pragma unroll
            for (int m = 0; m < OPT; m += 4) {
                const float4 w4 = *reinterpret_cast<const float4 *>(Wt + i * ld.fo + tx * OPT + m);
                w[m] = w4.x; w[m + 1] = w4.y; w[m + 2] = w4.z; w[m + 3] = w4.w;
            }
        } else {
#pragma unroll
            for (int m = 0; m < OPT; ++m) w[m] = Wt[i * ld.fo + tx * OPT + m];
        }
#pragma unroll
        for (int m = 0; m < OPT; ++m) {
            acc[0][m] = fmaf(x.x, w[m], acc[0][m]);
            acc[1][m] = fmaf(x.y, w[m], acc[1][m]);
            acc[2][m] = fmaf(x.z, w[m], acc[2][m]);
            acc[3][m] = fmaf(x.w, w[m], acc[3][m]);
        }
    }
#pragma unroll
    for (int m = 0; m < OPT; ++m) {
        const int o = tx * OPT + m;
        float4 v;
        v.x = fmaxf(acc[0][m], 0.0f);
        v.y = fmaxf(acc[1][m], 0.0f);
        v.z = fmaxf(acc[2][m], 0.0f);
        v.w = fmaxf(acc[3][m], 0.0f);
        *reinterpret_cast<float4 *>(out + o * kTileS + ((4 * ty) ^ swz(o))) = v;
    }
}

__device__ __forceinline__ float softplusf(float x) { return x > 0.0f ? x + log1pf(expf(-x)) : log1pf(expf(x)); }
__device__ __forceinline__ float sigmoidf(float x) { return 1.0f / (1.0f + expf(-x)); }

}  // namespace

__global__ void __launch_bounds__(kRenderThreads) k_aggregate_decode(const RenderArgs a, int n_params, int maxw,
                                                                     int xa_off, int xb_off)
{
    grid_dep_wait();
    grid_dep_trigger();
    extern __shared__ __align__(16) unsigned char smem[];
    float *prm = reinterpret_cast<float *>(smem);
    float *XA = reinterpret_cast<float *>(smem + xa_off);
    float *XB = reinterpret_cast<float *>(smem + xb_off);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // stage W^T and biases once per block
    LayerDesc lds[HP_MLP_MAX_LAYERS];
    {
        int o = 0;
        for (int l = 0; l < a.n_layers; ++l) {
            lds[l].fi = a.dims[l];
            lds[l].fo = a.dims[l + 1];
            lds[l].woff = o;
            o += lds[l].fi * lds[l].fo;
            lds[l].boff = o;
            o += lds[l].fo;
        }
    }
    {
        int g = 0;
        for (int l = 0; l < a.n_layers; ++l) {
            const int fi = lds[l].fi, fo = lds[l].fo, nw = fi * fo;
            for (int e = tid; e < nw; e += blockDim.x) {
                const int oo = e / fi, ii = e - oo * fi;           // global W is [out][in]
                prm[lds[l].woff + ii * fo + oo] = __ldg(a.mlp + g + e);
            }
            g += nw;
            for (int e = tid; e < fo; e += blockDim.x) prm[lds[l].boff + e] = __ldg(a.mlp + g + e);
            g += fo;
        }
    }
    __syncthreads();

    const int64_t S_all = __ldg(a.sample_offset + a.R);
    const int64_t S = S_all < a.capacity ? S_all : a.capacity;
    const int F = a.F, K = a.K;
    const int lpr = F >> 2;                    // lanes per feature row (one float4 each)
    const int rpp = 32 / lpr;                  // rows per warp load
    const int sub = lane / lpr, chunk = lane - sub * lpr;
    const float4 *feats4 = reinterpret_cast<const float4 *>(a.feats);

    for (int64_t base = (int64_t)blockIdx.x * kTileS; base < S; base += (int64_t)gridDim.x * kTileS) {
        // ---- gather + inverse-distance blend into XA[f][s]
        for (int sl = warp; sl < kTileS; sl += kRenderThreads / 32) {
            const int64_t g = base + sl;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            float wsum = 0.0f;
            if (g < S) {
                const int64_t row = list_row(a, g) * K;
                const int32_t *ids = list_ids(a) + row;
                const float *dists = list_dists(a) + row;
                for (int k0 = 0; k0 < K; k0 += rpp) {
                    const int k = k0 + sub;
                    if (k < K) {
                        const int id = __ldg(ids + k);
                        if (id >= 0 && hp_check(id < a.n_feats, a.err, id)) {
                            const float w = 1.0f / fmaxf(__ldg(dists + k), a.eps_d);
                            const float4 f = __ldg(feats4 + (int64_t)id * lpr + chunk);
                            acc.x = fmaf(w, f.x, acc.x);
                            acc.y = fmaf(w, f.y, acc.y);
                            acc.z = fmaf(w, f.z, acc.z);
                            acc.w = fmaf(w, f.w, acc.w);
                            wsum += w;
                        }
                    }
                }
                for (int o = lpr; o < 32; o <<= 1) {
                    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
                    acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
                    acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
                    wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
                }
            }
            if (sub == 0) {
                const float inv = g < S ? 1.0f / wsum : 0.0f;
                XA[xidx(4 * chunk + 0, sl)] = acc.x * inv;
                XA[xidx(4 * chunk + 1, sl)] = acc.y * inv;
                XA[xidx(4 * chunk + 2, sl)] = acc.z * inv;
                XA[xidx(4 * chunk + 3, sl)] = acc.w * inv;
            }
        }
        __syncthreads();

        // ---- hidden layers (ReLU), ping-pong XA <-> XB
        float *in = XA, *out = XB;
        for (int l = 0; l + 1 < a.n_layers; ++l) {
            const int opt = lds[l].fo >> 4;
            if (opt == 8) dense_relu<8>(prm, lds[l], in, out, tid);
            else if (opt == 4) dense_relu<4>(prm, lds[l], in, out, tid);
            else if (opt == 2) dense_relu<2>(prm, lds[l], in, out, tid);
            else dense_relu<1>(prm, lds[l], in, out, tid);
            __syncthreads();
            float *tmp = in;
            in = out;
            out = tmp;
        }

        // ---- output layer (4 channels): thread = (sample, channel)
        {
            const LayerDesc &ld = lds[a.n_layers - 1];
            const int s = tid >> 2, o = tid & 3;
            const float *Wt = prm + ld.woff;
            float acc = prm[ld.boff + o];
            for (int i = 0; i < ld.fi; ++i) acc = fmaf(in[xidx(i, s)], Wt[i * 4 + o], acc);
            const int gl = lane & ~3;
            const float o0 = __shfl_sync(0xffffffffu, acc, gl + 0);
            const float o1 = __shfl_sync(0xffffffffu, acc, gl + 1);
            const float o2 = __shfl_sync(0xffffffffu, acc, gl + 2);
            const float o3 = __shfl_sync(0xffffffffu, acc, gl + 3);
            const int64_t g = base + s;
            if (o == 0 && g < S) a.sample_out[g] = make_float4(softplusf(o0), sigmoidf(o1), sigmoidf(o2), sigmoidf(o3));
        }
        __syncthreads();
    }
}

// Eq. 2: tau_j = exp(-sum_{k<j} sigma_k Delta_k), weight tau_j (1 - exp(-sigma_j Delta_j)).
__global__ void __launch_bounds__(256) k_composite(const RenderArgs a)
{
    grid_dep_wait();
    grid_dep_trigger();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.R) return;
    int64_t o = __ldg(a.sample_offset + r);
    int64_t e = o + __ldg(a.n_s + r);
    if (e > a.capacity) e = a.capacity;
    float T = 1.0f, ws = 0.0f, c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;
    for (int64_t g = o; g < e; ++g) {
        const float4 v = a.sample_out[g];
        const float sd = v.x * __ldg(a.delta + g);
        const float w = T * (-expm1f(-sd));
        c0 = fmaf(w, v.y, c0);
        c1 = fmaf(w, v.z, c1);
        c2 = fmaf(w, v.w, c2);
        ws += w;
        T *= expf(-sd);
    }
    const float bg = a.bg_mode == 1 ? 1.0f - ws : 0.0f;
    a.rgb[3 * r + 0] = c0 + bg;
    a.rgb[3 * r + 1] = c1 + bg;
    a.rgb[3 * r + 2] = c2 + bg;
    a.wsum[r] = ws;
}

size_t render_smem_bytes(const RenderArgs &a) { return render_layout(a).total; }

cudaError_t launch_render(const RenderArgs &a, cudaStream_t st, Prof *prof)
{
    cudaError_t e;
    if (a.R <= 0) return cudaSuccess;
    const bool bf16 = a.decode == HP_DECODE_BF16;
    if (a.decode != HP_DECODE_FP32_SIMT && decode_tc_supported(a, bf16, nullptr)) {
        prof_begin(prof, st, KID_DECODE);
        int nk = 1;
        e = launch_decode_tc(a, bf16, st, &nk);
        prof_end(prof, st, nk);
        if (e != cudaSuccess) return e;
        prof_begin(prof, st, KID_COMPOSITE);
        launch_chained(k_composite, (unsigned)div_up(a.R, 256), 256, 0, st, a);
        prof_end(prof, st);
        return cudaGetLastError();
    }
    const RenderSmem L = render_layout(a);
    if ((e = cudaFuncSetAttribute(k_aggregate_decode, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total)) !=
        cudaSuccess)
        return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_aggregate_decode, kRenderThreads, L.total)) !=
        cudaSuccess)
        return e;
    if (per_sm < 1) per_sm = 1;
    // persistent grid: every resident slot, but no more blocks than tiles could need
    int64_t max_tiles = div_up(a.capacity, kTileS);
    int64_t grid = (int64_t)a.num_sms * per_sm;
    if (grid > max_tiles) grid = max_tiles;
    if (grid < 1) grid = 1;
    prof_begin(prof, st, KID_DECODE);
    launch_chained(k_aggregate_decode, (unsigned)grid, kRenderThreads, L.total, st, a, L.n_params, L.maxw, (int)L.xa, (int)L.xb);
    prof_end(prof, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    prof_begin(prof, st, KID_COMPOSITE);
    launch_chained(k_composite, (unsigned)div_up(a.R, 256), 256, 0, st, a);
    prof_end(prof, st);
    return cudaGetLastError();
}

}  // namespace hp
