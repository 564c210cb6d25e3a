// Radiance-MLP decode on the 5th-generation tensor cores (tcgen05 + TMEM).
//
// Two kernels.  k_decode_ws (further down; the one that runs whenever every
// layer is at most 128 wide and its weights fit shared memory) is
// warp-specialized: producer warps gather and blend while two groups of
// consumer warps take alternate tiles, keep the hidden activations in tensor
// memory and accumulate the FP32-accurate split in one accumulator.
// k_decode_tc, described here, serves the MLPs that do not fit that layout.
//
// k_decode_tc (persistent, one 512-thread block per SM, 128 samples per
// tile): the block stages the hidden layers' weights once in shared memory as
// K-major FP16 (or BF16) operands.  The neighbour lists (ids and distances)
// of the next tile are fetched by a bulk copy on the TMA engine while the
// current tile computes.  Per tile the block gathers and inverse-distance
// blends the samples' neighbour features straight into the first A operand,
// then for every hidden layer one thread issues tcgen05.mma (M = 128 samples,
// N = layer width, K = 16 per instruction) into TMEM; the whole block reads
// the FP32 accumulators back (tcgen05.ld), adds bias, applies ReLU and writes
// the next layer's A operand; the 4-wide output layer and the density /
// colour activations run on the FP32 cores from registers.
//
// Precision.  The default FP32-accurate mode splits every operand x into
// hi = fp16(x) and lo = fp16((x - hi) * 2^11) and accumulates
// A_hi B_hi into D1 and A_hi B_lo + A_lo B_hi into D2, so that
// D1 + 2^-11 D2 carries about 22 significant bits (Ootomo & Yokota 2022; the
// dropped lo*lo term is ~2^-22 relative).  The BF16 mode keeps one BF16 term
// per operand and one accumulator (the BF16 decode variant).
#include "hp_kernels.cuh"
#include "hp_tc.cuh"

namespace hp {

namespace {

constexpr int kTcTile = 128;
constexpr int kTcThreads = 512;            // 16 warps: 4 TMEM lane quarters x 4 column groups
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kMbarLimit = 1u << 24;

struct TcLayout {
    int nh;                              // hidden (tensor-core) layers
    int fi[HP_MLP_MAX_LAYERS], fo[HP_MLP_MAX_LAYERS];
    int w_hi[HP_MLP_MAX_LAYERS], w_lo[HP_MLP_MAX_LAYERS];   // byte offsets
    int bias[HP_MLP_MAX_LAYERS + 1];     // float offsets into the FP32 block
    int wl;                              // float offset of the output layer's W [4][fi]
    int f32_block;                       // byte offset of the FP32 block
    int a_hi, a_lo;                      // byte offsets of the activation operand
    int comb;                            // byte offset of the [4][128][4] combine buffer
    int ids, dists;                      // byte offsets of the staged neighbour lists
    int prefetch;                        // neighbour lists staged per tile (they fit)
    int mbar, tslot;                     // two mbarriers (MMA, list copy), TMEM address
    int total;
};

constexpr int kSmemLimit = 227 * 1024;

inline int up16(int x) { return (x + 15) & ~15; }

TcLayout tc_layout(const RenderArgs &a, bool bf16)
{
    TcLayout L{};
    L.nh = a.n_layers - 1;
    int o = 0, maxw = 0;
    for (int l = 0; l < L.nh; ++l) {
        L.fi[l] = a.dims[l];
        L.fo[l] = a.dims[l + 1];
        maxw = maxw > L.fi[l] ? maxw : L.fi[l];
        L.w_hi[l] = o;
        o += L.fi[l] * L.fo[l] * 2;
        L.w_lo[l] = o;
        if (!bf16) o += L.fi[l] * L.fo[l] * 2;
    }
    L.a_hi = o;
    o += kTcTile * maxw * 2;
    L.a_lo = o;
    if (!bf16) o += kTcTile * maxw * 2;
    L.f32_block = o;
    int f = 0;
    for (int l = 0; l < a.n_layers; ++l) {
        L.bias[l] = f;
        f += a.dims[l + 1];
    }
    L.wl = f;
    f += 4 * a.dims[a.n_layers - 1];
    o += up16(f * 4);
    // the output layer's combine buffer reuses the activation operand, which
    // is idle after the last hidden layer's MMAs
    const int comb_bytes = 4 * kTcTile * 4 * 4;
    if (kTcTile * maxw * 2 * (bf16 ? 1 : 2) >= comb_bytes) {
        L.comb = L.a_hi;
    } else {
        L.comb = o;
        o += comb_bytes;
    }
    const int list_bytes = kTcTile * a.K * 4;
    L.prefetch = o + 2 * list_bytes + 32 <= kSmemLimit;
    if (L.prefetch) {
        L.ids = o;
        o += list_bytes;
        L.dists = o;
        o += list_bytes;
    }
    L.mbar = o;
    o += 16;
    L.tslot = o;
    o += 16;
    L.total = o;
    return L;
}

__device__ __forceinline__ float softplus_f(float x) { return x > 0.0f ? x + log1pf(expf(-x)) : log1pf(expf(x)); }
__device__ __forceinline__ float sigmoid_f(float x) { return 1.0f / (1.0f + expf(-x)); }

template <bool kBF16>
__device__ __forceinline__ void store_operand8(unsigned char *hi_base, unsigned char *lo_base, uint32_t off,
                                               const float (&v)[8])
{
    if constexpr (kBF16) {
        __nv_bfloat16 h[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) h[i] = __float2bfloat16_rn(v[i]);
        *reinterpret_cast<uint4 *>(hi_base + off) = *reinterpret_cast<const uint4 *>(h);
    } else {
        __half h[8], l[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) tc::split_f16(v[i], h[i], l[i]);
        *reinterpret_cast<uint4 *>(hi_base + off) = *reinterpret_cast<const uint4 *>(h);
        *reinterpret_cast<uint4 *>(lo_base + off) = *reinterpret_cast<const uint4 *>(l);
    }
}

template <bool kBF16>
__device__ __forceinline__ void store_operand4(unsigned char *hi_base, unsigned char *lo_base, uint32_t off,
                                               float4 v)
{
    const float x[4] = {v.x, v.y, v.z, v.w};
    if constexpr (kBF16) {
        __nv_bfloat16 h[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) h[i] = __float2bfloat16_rn(x[i]);
        *reinterpret_cast<uint2 *>(hi_base + off) = *reinterpret_cast<const uint2 *>(h);
    } else {
        __half h[4], l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) tc::split_f16(x[i], h[i], l[i]);
        *reinterpret_cast<uint2 *>(hi_base + off) = *reinterpret_cast<const uint2 *>(h);
        *reinterpret_cast<uint2 *>(lo_base + off) = *reinterpret_cast<const uint2 *>(l);
    }
}

template <bool kBF16>
__device__ __forceinline__ void store_operand4_ss(unsigned char *hi_base, unsigned char *lo_base, uint32_t off,
                                                  float4 v)
{
    const float x[4] = {v.x, v.y, v.z, v.w};
    if constexpr (kBF16) {
        __nv_bfloat16 h[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) h[i] = __float2bfloat16_rn(x[i]);
        *reinterpret_cast<uint2 *>(hi_base + off) = *reinterpret_cast<const uint2 *>(h);
    } else {
        uint2 h, l;
        tc::split_f16x2_same_scale(x[0], x[1], h.x, l.x);
        tc::split_f16x2_same_scale(x[2], x[3], h.y, l.y);
        *reinterpret_cast<uint2 *>(hi_base + off) = h;
        *reinterpret_cast<uint2 *>(lo_base + off) = l;
    }
}

}  // namespace

template <bool kBF16>
__global__ void __launch_bounds__(kTcThreads, 1) k_decode_tc(const RenderArgs a, const TcLayout L, int bulk_ok)
{
    grid_dep_wait();
    grid_dep_trigger();
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *f32 = reinterpret_cast<float *>(smem + L.f32_block);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + L.mbar);       // MMA completion
    uint64_t *lbar = mbar + 1;                                           // list copy completion
    int *s_ids = reinterpret_cast<int *>(smem + L.ids);
    float *s_dst = reinterpret_cast<float *>(smem + L.dists);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + L.tslot);
    unsigned char *A_hi = smem + L.a_hi;
    unsigned char *A_lo = smem + L.a_lo;
    float *comb = reinterpret_cast<float *>(smem + L.comb);

    // ---- stage weights (global W is [out][in] FP32) and FP32 biases
    {
        int g = 0;
        for (int l = 0; l < a.n_layers; ++l) {
            const int fi = a.dims[l], fo = a.dims[l + 1];
            const int nw = fi * fo;
            if (l < L.nh) {
                for (int e = tid; e < nw; e += blockDim.x) {
                    const int o = e / fi, i = e - o * fi;
                    const float w = __ldg(a.mlp + g + e);
                    const uint32_t off = tc::kmajor_off(o, i, fi);
                    if constexpr (kBF16) {
                        *reinterpret_cast<__nv_bfloat16 *>(smem + L.w_hi[l] + off) = __float2bfloat16_rn(w);
                    } else {
                        __half h, lo;
                        tc::split_f16(w, h, lo);
                        *reinterpret_cast<__half *>(smem + L.w_hi[l] + off) = h;
                        *reinterpret_cast<__half *>(smem + L.w_lo[l] + off) = lo;
                    }
                }
            } else {
                for (int e = tid; e < nw; e += blockDim.x) f32[L.wl + e] = __ldg(a.mlp + g + e);
            }
            g += nw;
            for (int e = tid; e < fo; e += blockDim.x) f32[L.bias[l] + e] = __ldg(a.mlp + g + e);
            g += fo;
        }
    }
    if (tid == 0) {
        tc::mbar_init(mbar, 1);
        tc::mbar_init(lbar, 1);
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, kTmemCols);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;
    const uint32_t d1 = tbase, d2 = tbase + 128;

    const int64_t S_all = __ldg(a.sample_offset + a.R);
    const int64_t S = S_all < a.capacity ? S_all : a.capacity;
    const int F = a.F, K = a.K;
    const uint32_t list_bytes = (uint32_t)(kTcTile * K * 4);
    // a tile's lists come by bulk copy when the whole 128-sample block of the
    // (16-byte aligned) arrays lies inside their allocation
    auto bulk_tile = [&](int64_t b) { return L.prefetch && bulk_ok && b < S && b + kTcTile <= a.capacity; };
    uint32_t lphase = 0;
    bool pending = bulk_tile((int64_t)blockIdx.x * kTcTile);   // a list copy in flight (all threads agree)
    if (tid == 0 && pending) {
        const int64_t b = (int64_t)blockIdx.x * kTcTile;
        tc::mbar_arrive_expect_tx(lbar, 2 * list_bytes);
        tc::bulk_g2s(s_ids, a.nbr + b * K, list_bytes, lbar);
        tc::bulk_g2s(s_dst, a.nbr_dist + b * K, list_bytes, lbar);
    }
    const int lpr = F >> 2, spw = 32 / lpr;                   // lanes per feature row, samples per warp step
    const int sub = lane / lpr, chunk = lane - sub * lpr;
    const float4 *feats4 = reinterpret_cast<const float4 *>(a.feats);
    const int q = warp & 3, cg = warp >> 2;                    // TMEM lane quarter, column group (0..3)
    const int row = 32 * q + lane;                             // sample row of this thread in the tile
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    uint32_t phase = 0;
    bool ok = true;

    for (int64_t base = (int64_t)blockIdx.x * kTcTile; base < S && ok; base += (int64_t)gridDim.x * kTcTile) {
        // ---- this tile's neighbour lists: staged (bulk copy issued during
        // the previous tile) or read directly
        const bool staged = L.prefetch != 0;
        if (staged) {
            if (bulk_tile(base)) {
                if (!tc::mbar_wait(lbar, lphase, kMbarLimit)) {
                    ok = false;
                    set_error(a.err, HP_ERR_TIMEOUT, -4);
                }
                lphase ^= 1u;
                pending = false;
            } else {
                for (int e = tid; e < kTcTile * K; e += kTcThreads) {
                    const int64_t g = base + e / K;
                    const bool in = g < S;
                    const int64_t at = in ? list_row(a, g) * K + e % K : 0;
                    s_ids[e] = in ? __ldg(list_ids(a) + at) : -1;
                    s_dst[e] = in ? __ldg(list_dists(a) + at) : 1.0f;
                }
            }
            ok = __syncthreads_and(ok) != 0;
            if (!ok) break;
        }
        // ---- gather + inverse-distance blend -> first A operand (K = F).
        // Lane (s, c) of a warp owns sample s of the group and the 16-byte
        // chunk c of its feature row and walks the K neighbours itself, so
        // the K row loads of a lane are independent and in flight together.
        for (int s0 = warp * spw; s0 < kTcTile; s0 += (kTcThreads / 32) * spw) {
            const int sl = s0 + sub;
            const int64_t g = base + sl;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            if (sl < kTcTile && g < S) {
                float wsum = 0.0f;
                const int *nb = staged ? s_ids + sl * K : list_ids(a) + list_row(a, g) * K;
                const float *nd = staged ? s_dst + sl * K : list_dists(a) + list_row(a, g) * K;
#pragma unroll 8
                for (int k = 0; k < K; ++k) {
                    const int id = nb[k];
                    if (id >= 0 && hp_check(id < a.n_feats, a.err, id)) {
                        const float w = 1.0f / fmaxf(nd[k], a.eps_d);
                        const float4 f = __ldg(feats4 + (int64_t)id * lpr + chunk);
                        acc.x = fmaf(w, f.x, acc.x);
                        acc.y = fmaf(w, f.y, acc.y);
                        acc.z = fmaf(w, f.z, acc.z);
                        acc.w = fmaf(w, f.w, acc.w);
                        wsum += w;
                    }
                }
                const float inv = 1.0f / wsum;
                acc.x *= inv; acc.y *= inv; acc.z *= inv; acc.w *= inv;
            }
            if (sl < kTcTile) store_operand4<kBF16>(A_hi, A_lo, tc::kmajor_off(sl, 4 * chunk, F), acc);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        // the lists are consumed: fetch the next tile's while this one computes
        pending = bulk_tile(base + (int64_t)gridDim.x * kTcTile);
        if (tid == 0 && pending) {
            const int64_t b = base + (int64_t)gridDim.x * kTcTile;
            tc::mbar_arrive_expect_tx(lbar, 2 * list_bytes);
            tc::bulk_g2s(s_ids, a.nbr + b * K, list_bytes, lbar);
            tc::bulk_g2s(s_dst, a.nbr_dist + b * K, list_bytes, lbar);
        }

        float o4[4] = {0.f, 0.f, 0.f, 0.f};
        for (int l = 0; l < L.nh && ok; ++l) {
            const int fi = L.fi[l], fo = L.fo[l];
            if (tid == 0) {
                tc::fence_after_sync();
                const uint32_t idesc = tc::idesc_f16(kTcTile, fo, kBF16);
                const uint32_t ah = tc::smem_u32(A_hi), al = tc::smem_u32(A_lo);
                const uint32_t wh = tc::smem_u32(smem + L.w_hi[l]), wl = tc::smem_u32(smem + L.w_lo[l]);
                const uint32_t sbo = (uint32_t)fi * 16;
                for (int kk = 0; kk < fi / 16; ++kk) {
                    const uint64_t dah = tc::sdesc(ah + kk * 256, 128, sbo), dbh = tc::sdesc(wh + kk * 256, 128, sbo);
                    tc::mma_f16(d1, dah, dbh, idesc, kk > 0);
                    if constexpr (!kBF16) {
                        const uint64_t dal = tc::sdesc(al + kk * 256, 128, sbo);
                        const uint64_t dbl = tc::sdesc(wl + kk * 256, 128, sbo);
                        tc::mma_f16(d2, dah, dbl, idesc, kk > 0);
                        tc::mma_f16(d2, dal, dbh, idesc, 1);
                    }
                }
                tc::commit(mbar);
            }
            if (!tc::mbar_wait(mbar, phase, kMbarLimit)) {
                ok = false;
                set_error(a.err, HP_ERR_TIMEOUT, -2);
            }
            phase ^= 1u;
            ok = __syncthreads_and(ok) != 0;
            if (!ok) break;
            tc::fence_after_sync();

            // ---- epilogue: this thread's sample row; the layer's 8-column
            // chunks go round-robin to the 4 column groups (chunks cg, cg+4, ...)
            const float *bias = f32 + L.bias[l];
            const bool last = (l + 1 == L.nh);
            {
                const int nch = fo / 8;
                // all of this thread's chunks (up to 4) leave TMEM together, then one wait
                float v1[4][8], v2[4][8];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int ch = cg + 4 * j;
                    if (ch < nch) {
                        tc::ld8(d1 + lane_off + (uint32_t)(8 * ch), v1[j]);
                        if constexpr (!kBF16) tc::ld8(d2 + lane_off + (uint32_t)(8 * ch), v2[j]);
                    }
                }
                tc::wait_ld();
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int ch = cg + 4 * j;
                    if (ch >= nch) break;
                    const int c = 8 * ch;
                    float h[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        float x = v1[j][i];
                        if constexpr (!kBF16) x = fmaf(v2[j][i], 1.0f / 2048.0f, x);
                        h[i] = fmaxf(x + bias[c + i], 0.0f);
                    }
                    if (!last) {
                        store_operand8<kBF16>(A_hi, A_lo, tc::kmajor_off(row, c, fo), h);
                    } else {
                        const float *W = f32 + L.wl;
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            o4[0] = fmaf(h[i], W[0 * fo + c + i], o4[0]);
                            o4[1] = fmaf(h[i], W[1 * fo + c + i], o4[1]);
                            o4[2] = fmaf(h[i], W[2 * fo + c + i], o4[2]);
                            o4[3] = fmaf(h[i], W[3 * fo + c + i], o4[3]);
                        }
                    }
                }
            }
            tc::fence_async_smem();
            tc::fence_before_sync();
            __syncthreads();
        }
        if (!ok) break;

        // ---- output layer: combine the column groups, activations
        if (cg > 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) comb[(cg * kTcTile + row) * 4 + i] = o4[i];
        }
        __syncthreads();
        if (cg == 0) {
            const float *bl = f32 + L.bias[a.n_layers - 1];
            float o[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                o[i] = ((o4[i] + comb[(kTcTile + row) * 4 + i]) + comb[(2 * kTcTile + row) * 4 + i]) +
                       comb[(3 * kTcTile + row) * 4 + i] + bl[i];
            const int64_t g = base + row;
            if (g < S) a.sample_out[g] = make_float4(softplus_f(o[0]), sigmoid_f(o[1]), sigmoid_f(o[2]), sigmoid_f(o[3]));
        }
        __syncthreads();
    }

    // a list copy still in flight (the loop left early) lands before exit
    if (pending) tc::mbar_wait(lbar, lphase, kMbarLimit);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tbase, kTmemCols);
}

// One 128 x N x K product D = A B^T on the tensor cores (A: 128 x K, B: N x K,
// row-major 16-bit inputs), for the library's self-test of the tcgen05 path.
// flags bit 0: BF16 inputs; bit 1: A taken from tensor memory (written there
// with tcgen05.st) instead of shared memory.
__global__ void __launch_bounds__(128, 1) k_mma_selftest(const uint16_t *A, const uint16_t *B, float *D, int K, int N,
                                                         int flags, ErrWord *err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool bf16 = (flags & 1) != 0, a_tmem = (flags & 2) != 0;
    constexpr uint32_t kCols = 512, kAcol = 256;   // D in columns [0, N), A in [256, 256 + K/2)
    unsigned char *sa = smem;
    unsigned char *sb = smem + 128 * K * 2;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sb + N * K * 2);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    if (!a_tmem) {
        for (int e = tid; e < 128 * K; e += blockDim.x) {
            const int r = e / K, k = e - r * K;
            *reinterpret_cast<uint16_t *>(sa + tc::kmajor_off(r, k, K)) = A[e];
        }
    }
    for (int e = tid; e < N * K; e += blockDim.x) {
        const int r = e / K, k = e - r * K;
        *reinterpret_cast<uint16_t *>(sb + tc::kmajor_off(r, k, K)) = B[e];
    }
    if (tid == 0) {
        tc::mbar_init(mbar, 1);
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, kCols);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;
    const uint32_t lane_off = (uint32_t)(32 * warp) << 16;
    if (a_tmem) {
        // thread = row 32 warp + lane; two elements per column
        const int r = 32 * warp + lane;
        for (int c0 = 0; c0 < K / 2; c0 += 8) {
            uint32_t v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                v[j] = (uint32_t)A[r * K + 2 * (c0 + j)] | ((uint32_t)A[r * K + 2 * (c0 + j) + 1] << 16);
            tc::st8(tbase + lane_off + kAcol + (uint32_t)c0, v);
        }
        tc::wait_st();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    if (tid == 0) {
        const uint32_t idesc = tc::idesc_f16(128, N, bf16);
        for (int kk = 0; kk < K / 16; ++kk) {
            const uint64_t bd = tc::sdesc(tc::smem_u32(sb) + kk * 256, 128, K * 16);
            if (a_tmem)
                tc::mma_f16_ta(tbase, tbase + kAcol + (uint32_t)(kk * 8), bd, idesc, kk > 0);
            else
                tc::mma_f16(tbase, tc::sdesc(tc::smem_u32(sa) + kk * 256, 128, K * 16), bd, idesc, kk > 0);
        }
        tc::commit(mbar);
    }
    const bool done = tc::mbar_wait(mbar, 0, kMbarLimit);
    if (!done && tid == 0) set_error(err, HP_ERR_TIMEOUT, -3);
    if (__syncthreads_and(done)) {
        tc::fence_after_sync();
        const int r = 32 * warp + lane;
        for (int c = 0; c < N; c += 8) {
            float v[8];
            tc::ld8(tbase + lane_off + (uint32_t)c, v);
            tc::wait_ld();
#pragma unroll
            for (int i = 0; i < 8; ++i) D[r * N + c + i] = v[i];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tbase, kCols);
}

// ---------------------------------------------------------------------------
// k_decode_ws: the same decode, warp-specialized, one 1024-thread block per
// SM.  16 producer warps gather and inverse-distance blend the samples of the
// next tiles into two shared-memory buffers of the first A operand; 16
// consumer warps in two groups of 8 (4 TMEM lane quarters x 2 column groups)
// take alternate tiles (tile i in buffer i % 2), so one group's epilogues
// overlap the other's MMAs.  Tiles come from a grid-wide counter.  Hidden
// activations never touch shared memory: the epilogue writes them back into
// tensor memory (two 16-bit values per column) and the next layer's
// tcgen05.mma reads its A operand from there.  The 4-wide output layer runs
// on the FP32 cores inside the last hidden layer's epilogue (a 16-wide MMA
// for it measured slower: its round trip queues behind the other group's
// layer MMAs).
// FP32-accurate mode: A = A_hi + A_lo and B = B_hi + B_lo with lo the FP16
// rounding of the remainder (unscaled; A_hi rounded toward zero so that the
// ReLU clamps both parts), and A_hi B_hi + A_hi B_lo + A_lo B_hi
// accumulate in one FP32 accumulator.  Tensor memory per group g:
// D [256g, 256g+128), A_hi [256g+128, +64), A_lo [256g+192, +64).
// The weights arrive as a prepared image (k_ws_image) by bulk copies.
// Hand-offs: full[b] (producers -> consumers, one arrival per producer warp), empty[b]
// (tcgen05.commit after the layer-0 MMAs that read buffer b), lbar[b] (bulk
// copy of a tile's neighbour lists), mma (per layer), the weights' barrier.
// Every wait is bounded.
// Consumer warps kCW (a template parameter): two groups, each 4 TMEM lane
// quarters x (kCW / 8) column groups.  16 for K <= 8; 8 for larger K, where
// the gather of twice the neighbours sets the pace and the fewer, wider
// consumer warps leave the producers more of the SM (forward_1008, K 16:
// 0.380 -> 0.354 ms FP32, 0.342 -> 0.314 BF16; objects_800, K 8: 0.233 ->
// 0.245 FP32, so K 8 keeps 16).
constexpr int kWsProducerWarps = 16;
constexpr int kWsBatch = 1;               // 8-column chunks a consumer thread reads from TMEM at once (2 and 4: register spills)
__host__ __device__ constexpr int ws_threads(int kCW) { return (kCW + kWsProducerWarps) * 32; }
constexpr uint32_t kWsCols = 512, kColAH = 128, kColAL = 192;   // per consumer group, group g at 256 g

struct WsLayout {
    int nh;
    int fi[HP_MLP_MAX_LAYERS], fo[HP_MLP_MAX_LAYERS];
    int w_hi[HP_MLP_MAX_LAYERS], w_lo[HP_MLP_MAX_LAYERS];
    int bias[HP_MLP_MAX_LAYERS + 1];
    int wl, f32_block, f32_bytes;
    int a0[2], a0_lo;                    // first A operand buffers; lo part at +a0_lo
    int ids[2], dists[2];                // neighbour list buffers
    int comb, bars, tiles, tslot, total;
    int ok;                              // the layout fits this kernel
};

// The weights' shared-memory image as k_ws_image writes it to global memory:
// the hidden layers' B operands (bytes [0, a0[0]) of the layout) followed by
// the FP32 block (biases and the output layer).  Each CTA copies it in with
// bulk copies.
__host__ __device__ inline int ws_image_bytes(const WsLayout &L) { return L.a0[0] + L.f32_bytes; }

WsLayout ws_layout(const RenderArgs &a, bool bf16)
{
    WsLayout L{};
    L.nh = a.n_layers - 1;
    L.ok = L.nh >= 1;
    int o = 0;
    for (int l = 0; l < L.nh; ++l) {
        L.fi[l] = a.dims[l];
        L.fo[l] = a.dims[l + 1];
        if (L.fo[l] > 128 || L.fi[l] > 128) L.ok = 0;
        L.w_hi[l] = o;
        o += L.fi[l] * L.fo[l] * 2;
        L.w_lo[l] = o;
        if (!bf16) o += L.fi[l] * L.fo[l] * 2;
    }
    const int a0_bytes = kTcTile * a.dims[0] * 2;
    L.a0_lo = a0_bytes;
    for (int b = 0; b < 2; ++b) {
        L.a0[b] = o;
        o += a0_bytes * (bf16 ? 1 : 2);
    }
    L.f32_block = o;
    int f = 0;
    for (int l = 0; l < a.n_layers; ++l) {
        L.bias[l] = f;
        f += a.dims[l + 1];
    }
    L.wl = f;
    f += 4 * a.dims[a.n_layers - 1];
    L.f32_bytes = up16(f * 4);
    o += L.f32_bytes;
    const int list_bytes = kTcTile * a.K * 4;
    for (int b = 0; b < 2; ++b) {
        L.ids[b] = o;
        o += list_bytes;
        L.dists[b] = o;
        o += list_bytes;
    }
    L.comb = o;
    o += 4 * kTcTile * 4 * 4;
    L.bars = o;
    o += 9 * 8;                           // full[2], empty[2], lbar[2], mma[2], weights
    L.tiles = o;
    o += 4 * 8;                           // tile of each A buffer: producers' [2], consumers' [2]
    L.tslot = o;
    o += 16;
    L.total = o;
    if (L.total > kSmemLimit) L.ok = 0;
    // the gather maps 16-byte chunks of a feature row to lanes
    if (a.dims[0] % 16 != 0 || a.dims[0] > 128) L.ok = 0;
    return L;
}

// Converts the MLP (global, FP32, W [out][in] then b per layer) once per call
// into the decode's shared-memory image (see ws_image_bytes) and clears the
// decode's tile counter.
template <bool kBF16>
__global__ void k_ws_image(const RenderArgs a, const WsLayout L)
{
    grid_dep_wait();
    grid_dep_trigger();
    const int gid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    unsigned char *img = a.wimg;
    float *f32 = reinterpret_cast<float *>(img + L.a0[0]);
    if (gid == 0) *a.tile_ctr = 0u;
    int g = 0;
    for (int l = 0; l < a.n_layers; ++l) {
        const int fi = a.dims[l], fo = a.dims[l + 1];
        const int nw = fi * fo;
        for (int e = gid; e < nw; e += nthr) {
            const int o = e / fi, i = e - o * fi;
            const float w = __ldg(a.mlp + g + e);
            if (l < L.nh) {
                const uint32_t off = tc::kmajor_off(o, i, fi);
                if constexpr (kBF16) {
                    *reinterpret_cast<__nv_bfloat16 *>(img + L.w_hi[l] + off) = __float2bfloat16_rn(w);
                } else {
                    __half h, lo;
                    tc::split_f16_same_scale(w, h, lo);
                    *reinterpret_cast<__half *>(img + L.w_hi[l] + off) = h;
                    *reinterpret_cast<__half *>(img + L.w_lo[l] + off) = lo;
                }
            } else {
                // the output layer's W [4][fi] stored transposed, [fi][4]:
                // one 16-byte load gives an input's four weights
                f32[L.wl + i * 4 + o] = w;
            }
        }
        g += nw;
        for (int e = gid; e < fo; e += nthr) f32[L.bias[l] + e] = __ldg(a.mlp + g + e);
        g += fo;
    }
}

template <bool kBF16, int kCW>
__global__ void __launch_bounds__(ws_threads(kCW), 1) k_decode_ws(const RenderArgs a, const WsLayout L, int bulk_ok)
{
    constexpr int kWsConsumerWarps = kCW;
    constexpr int kWsGroupWarps = kWsConsumerWarps / 2;
    constexpr int kWsGroups = kWsGroupWarps / 4;
    static_assert(kWsGroups >= 1 && kWsGroupWarps % 4 == 0, "consumer groups of whole lane-quarter sets");
    grid_dep_wait();
    grid_dep_trigger();
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *f32 = reinterpret_cast<float *>(smem + L.f32_block);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bars);
    uint64_t *full = bars, *empty = bars + 2, *lbar = bars + 4, *mbar = bars + 6;   // mbar: one per group
    float *comb = reinterpret_cast<float *>(smem + L.comb);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + L.tslot);

    int64_t *ptile = reinterpret_cast<int64_t *>(smem + L.tiles), *ctile = ptile + 2;
    uint64_t *wbar = bars + 8;

    // ---- the weights' image (k_ws_image) arrives by two bulk copies while
    // the producers start on the first tiles; the consumers wait for it
    if (tid == 0) {
        tc::mbar_init(&full[0], kWsProducerWarps);
        tc::mbar_init(&full[1], kWsProducerWarps);
        tc::mbar_init(&empty[0], 1);
        tc::mbar_init(&empty[1], 1);
        tc::mbar_init(&lbar[0], 1);
        tc::mbar_init(&lbar[1], 1);
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::mbar_init(wbar, 1);
        tc::mbar_fence_init();
        const uint32_t wbytes = (uint32_t)L.a0[0], fbytes = (uint32_t)L.f32_bytes;
        tc::mbar_arrive_expect_tx(wbar, wbytes + fbytes);
        constexpr uint32_t kChunk = 32768;
        for (uint32_t o = 0; o < wbytes; o += kChunk)
            tc::bulk_g2s(smem + o, a.wimg + o, wbytes - o < kChunk ? wbytes - o : kChunk, wbar);
        tc::bulk_g2s(smem + L.f32_block, a.wimg + wbytes, fbytes, wbar);
    }
    if (warp == 0) tc::tmem_alloc(tslot, kWsCols);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;

    const int64_t S_all = __ldg(a.sample_offset + a.R);
    const int64_t S = S_all < a.capacity ? S_all : a.capacity;
    const int F = a.F, K = a.K;
    const uint32_t list_bytes = (uint32_t)(kTcTile * K * 4);
    // a tile's neighbour lists: bulk_ok 1, two bulk copies of the packed
    // rows; 2, copied by the producer warps from the slot rows (the search
    // left the lists in the slots); 0, plain loads
    auto bulk_tile = [&](int64_t b) { return bulk_ok == 1 && b < S && b + kTcTile <= a.capacity; };

    if (warp >= kWsConsumerWarps) {
        // =============================== producers: gather + blend
        const int ptid = tid - kWsConsumerWarps * 32, pw = warp - kWsConsumerWarps;
        const int lpr = F >> 2, spw = 32 / lpr;
        const int sub = lane / lpr, chunk = lane - sub * lpr;
        const float4 *feats4 = reinterpret_cast<const float4 *>(a.feats);
        uint32_t lph = 0u, eph = 3u;   // parity bit per buffer; a fresh barrier's previous phase counts as done
        uint32_t pend = 0u;            // list copies in flight, per buffer (leader only)
        bool ok = true;
        // Tiles come from a grid-wide counter (cleared by k_ws_image); the
        // leader warp (pw 0) fetches them two ahead.  At the top of iteration
        // j, ptile[j & 1] holds tile j and ptile[(j + 1) & 1] tile j + 1, so
        // the lists of tile j + 1 arrive while tile j is gathered.  ctile[b]
        // is the tile of A buffer b for the consumers (-1: no more tiles; each
        // buffer gets one such end mark).
        int64_t t_next = 0;        // (leader warp) tile j + 2
        auto fetch = [&]() -> int64_t {
            uint32_t v = 0;
            if (lane == 0) v = atomicAdd(a.tile_ctr, 1u);
            return (int64_t)__shfl_sync(0xffffffffu, v, 0) * kTcTile;
        };
        // (leader warp, bulk_ok 1) the packed lists of tile tb into buffer buf
        auto issue_lists = [&](int buf, int64_t tb) {
            pend |= 1u << buf;
            if (lane == 0) {
                tc::mbar_arrive_expect_tx(&lbar[buf], 2 * list_bytes);
                tc::bulk_g2s(smem + L.ids[buf], a.nbr + tb * K, list_bytes, &lbar[buf]);
                tc::bulk_g2s(smem + L.dists[buf], a.nbr_dist + tb * K, list_bytes, &lbar[buf]);
            }
        };
        // bulk_ok 2 (the lists stay in the search's slots): every producer
        // warp copies the slot rows of its kRowSamples samples of a tile, in
        // 16-byte chunks (at most two per lane: K <= 16).  The slot indices
        // are loaded at the top of an iteration, the rows after the producer
        // barrier, and they are stored into the other list buffer after the
        // warp's gather, so their latency overlaps the gather.
        constexpr int kRowSamples = kTcTile / kWsProducerWarps;
        static_assert(kTcTile % kWsProducerWarps == 0, "samples per producer warp");
        const int cpr = K >> 2;                                  // 16-byte chunks per row
        const int n_chunks = kRowSamples * 2 * cpr;              // per warp, <= 64
        // per lane and chunk u (fixed for the whole kernel): the sample of the
        // warp's share (-1: no chunk), the row offset (list bit 31 set for the
        // distances) and the byte offset in a list buffer
        int rq[2], rsrc[2], rdst[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int e = lane + 32 * u;
            const int q = cpr > 0 ? e / (2 * cpr) : 0, rem = cpr > 0 ? e - q * 2 * cpr : 0;
            const int list = rem >= cpr, c = rem - (list ? cpr : 0);
            rq[u] = (bulk_ok == 2 && e < n_chunks) ? q : -1;
            rsrc[u] = 4 * c;
            rdst[u] = (list ? (int)list_bytes : 0) + ((pw * kRowSamples + q) * K + 4 * c) * 4;
            if (list) rsrc[u] |= 1 << 30;
        }
        int32_t rslot[2] = {-1, -1};
        float4 rval[2];
        auto row_index = [&](int64_t tb) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int64_t g = tb + pw * kRowSamples + rq[u];
                rslot[u] = (rq[u] >= 0 && g < S) ? __ldg(a.sample_slot + g) : -1;
                if (rslot[u] >= 0 && !hp_check(rslot[u] < a.n_slots, a.err, rslot[u])) rslot[u] = -1;
            }
        };
        auto row_load = [&]() {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (rslot[u] < 0) continue;
                const int64_t at = (int64_t)rslot[u] * K + (rsrc[u] & 0xffff);
                const float *src = (rsrc[u] >> 30) ? a.slot_dist : reinterpret_cast<const float *>(a.slot_nbr);
                rval[u] = __ldg(reinterpret_cast<const float4 *>(src + at));
            }
        };
        auto row_store = [&](int buf) {
#pragma unroll
            for (int u = 0; u < 2; ++u)
                if (rslot[u] >= 0) *reinterpret_cast<float4 *>(smem + L.ids[buf] + rdst[u]) = rval[u];
        };
        if (pw == 0) {
            const int64_t t0 = fetch();
            const int64_t t1 = t0 < S ? fetch() : t0;
            if (lane == 0) {
                ptile[0] = t0;
                ptile[1] = t1;
            }
            if (bulk_tile(t0)) issue_lists(0, t0);
            t_next = t1 < S ? fetch() : t1;
        }
        tc::bar_and(3, kWsProducerWarps * 32, true);
        if (bulk_ok == 2) {
            // the first tile's rows
            if (ptile[0] < S) {
                row_index(ptile[0]);
                row_load();
                row_store(0);
            }
            tc::bar_and(3, kWsProducerWarps * 32, true);
        }
        int ends = 0;
        for (int it = 0; ends < 2; ++it) {
            const int b = it & 1;
            const int64_t base = ptile[b], nb = ptile[b ^ 1];
            const bool valid = base < S;
            int *s_ids = reinterpret_cast<int *>(smem + L.ids[b]);
            float *s_dst = reinterpret_cast<float *>(smem + L.dists[b]);
            // the next tile's lists into the other buffer (its readers finished:
            // producer barrier at the end of the previous iteration)
            if (pw == 0 && valid && bulk_tile(nb)) issue_lists(b ^ 1, nb);
            const bool rows = bulk_ok == 2 && nb < S;     // this warp's rows of the next tile
            if (rows) row_index(nb);
            if (valid) {
                if (bulk_tile(base)) {
                    if (!tc::mbar_wait(&lbar[b], (lph >> b) & 1u, kMbarLimit)) {
                        ok = false;
                        set_error(a.err, HP_ERR_TIMEOUT, -5);
                    }
                    lph ^= 1u << b;
                    pend &= ~(1u << b);
                } else if (bulk_ok != 2) {
                    // (tiles the bulk copy does not take: plain loads; with
                    // bulk_ok 2 the producers stored the rows a step earlier)
                    for (int e = ptid; e < kTcTile * K; e += kWsProducerWarps * 32) {
                        const int64_t g = base + e / K;
                        const bool in = g < S;
                        const int64_t at = in ? list_row(a, g) * K + e % K : 0;
                        s_ids[e] = in ? __ldg(list_ids(a) + at) : -1;
                        s_dst[e] = in ? __ldg(list_dists(a) + at) : 1.0f;
                    }
                    ok = tc::bar_and(3, kWsProducerWarps * 32, ok);
                }
                // BF16: the inverse-distance weights, each computed once, in place
                // of the distances (read by other producers after the barrier
                // below).  FP32 keeps the division in the gather loop: with the
                // precomputed weights that variant spills at its 64 registers.
                if constexpr (kBF16) {
                    for (int e = ptid; e < kTcTile * K; e += kWsProducerWarps * 32)
                        s_dst[e] = s_ids[e] >= 0 ? __fdividef(1.0f, fmaxf(s_dst[e], a.eps_d)) : 0.0f;
                }
            }
            // the buffer is free once the layer-0 MMAs of tile it-2 are done
            if (ok && !tc::mbar_wait(&empty[b], (eph >> b) & 1u, kMbarLimit)) {
                ok = false;
                set_error(a.err, HP_ERR_TIMEOUT, -6);
            }
            eph ^= 1u << b;
            ok = tc::bar_and(3, kWsProducerWarps * 32, ok);   // every producer leaves together
            if (!ok) break;
            if (rows) row_load();
            if (valid) {
                unsigned char *A_hi = smem + L.a0[b];
                unsigned char *A_lo = A_hi + L.a0_lo;
                for (int s0 = pw * spw; s0 < kTcTile; s0 += kWsProducerWarps * spw) {
                    const int sl = s0 + sub;
                    const int64_t g = base + sl;
                    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (g < S) {
                        float wsum = 0.0f;
                        const int *nl = s_ids + sl * K;
                        const float *nw = s_dst + sl * K;
                        // (BF16 with K > 8: 16 loads in flight, 0.306 -> 0.295 ms on
                        // forward_1008; FP32 keeps 8, which it runs faster with)
#pragma unroll (kCW == 8 && kBF16 ? 16 : 8)
                        for (int k = 0; k < K; ++k) {
                            const int id = nl[k];
                            if (id >= 0 && hp_check(id < a.n_feats, a.err, id)) {
                                // inverse-distance weight (approximate reciprocal:
                                // ~2 ulp, far inside the colour tolerance)
                                const float w = kBF16 ? nw[k] : __fdividef(1.0f, fmaxf(nw[k], a.eps_d));
                                const float4 f = __ldg(feats4 + (int64_t)id * lpr + chunk);
                                acc.x = fmaf(w, f.x, acc.x);
                                acc.y = fmaf(w, f.y, acc.y);
                                acc.z = fmaf(w, f.z, acc.z);
                                acc.w = fmaf(w, f.w, acc.w);
                                wsum += w;
                            }
                        }
                        const float inv = __fdividef(1.0f, wsum);
                        acc.x *= inv; acc.y *= inv; acc.z *= inv; acc.w *= inv;
                    }
                    store_operand4_ss<kBF16>(A_hi, A_lo, tc::kmajor_off(sl, 4 * chunk, F), acc);
                }
                tc::fence_async_smem();                  // generic stores -> tensor-core reads
            } else {
                ++ends;
            }
            if (rows) row_store(b ^ 1);
            // (leader) tile j + 2 into the slot of tile j, which every producer
            // read at the top of this iteration (before the barrier above)
            if (pw == 0) {
                if (lane == 0) ptile[b] = t_next;
                if (t_next < S) t_next = fetch();
            }
            if (ptid == 0) ctile[b] = valid ? base : -1;
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&full[b]);
            ok = tc::bar_and(3, kWsProducerWarps * 32, ok);
            if (!ok) break;
        }
        // a list copy still in flight lands before exit
        for (int b = 0; b < 2; ++b)
            if (ptid == 0 && ((pend >> b) & 1u)) tc::mbar_wait(&lbar[b], (lph >> b) & 1u, kMbarLimit);
    } else {
        // =============================== consumers: MMA + epilogues
        const int grp = warp / kWsGroupWarps, wg = warp - grp * kWsGroupWarps;
        const int gtid = tid - grp * kWsGroupWarps * 32;
        const int barid = 1 + grp, nthr = kWsGroupWarps * 32;
        const int q = wg & 3, cg = wg >> 2;
        const int row = 32 * q + lane;
        const uint32_t lane_off = (uint32_t)(32 * q) << 16;
        const uint32_t gbase = tbase + 256u * (uint32_t)grp;
        const uint32_t d1 = gbase, ah = gbase + kColAH, al = gbase + kColAL;
        uint64_t *gbar = &mbar[grp];
        float *gcomb = comb + grp * (kWsGroups * kTcTile * 4);
        uint32_t fph = 0u, mph = 0u;
        bool ok = true;
        const int b = grp;                       // this group's tiles all use A buffer grp
        if (!tc::mbar_wait(wbar, 0u, kMbarLimit)) {  // the weights' image
            ok = false;
            set_error(a.err, HP_ERR_TIMEOUT, -9);
        }
        for (;;) {
            if (ok && !tc::mbar_wait(&full[b], fph, kMbarLimit)) {
                ok = false;
                set_error(a.err, HP_ERR_TIMEOUT, -7);
            }
            fph ^= 1u;
            const int64_t base = ctile[b];           // -1: no more tiles
            ok = tc::bar_and(barid, nthr, ok);
            if (!ok || base < 0) break;
            tc::fence_after_sync();
            uint64_t o01 = tc::f32x2(0.f, 0.f), o23 = tc::f32x2(0.f, 0.f);   // output layer sums
            for (int l = 0; l < L.nh; ++l) {
                const int fi = L.fi[l], fo = L.fo[l];
                if (gtid == 0) {
                    const uint32_t idesc = tc::idesc_f16(kTcTile, fo, kBF16);
                    const uint32_t wh = tc::smem_u32(smem + L.w_hi[l]), wl = tc::smem_u32(smem + L.w_lo[l]);
                    const uint32_t sbo = (uint32_t)fi * 16;
                    if (l == 0) {
                        const uint32_t a0h = tc::smem_u32(smem + L.a0[b]), a0l = a0h + (uint32_t)L.a0_lo;
                        for (int kk = 0; kk < fi / 16; ++kk) {
                            const uint64_t dah = tc::sdesc(a0h + kk * 256, 128, sbo);
                            const uint64_t dbh = tc::sdesc(wh + kk * 256, 128, sbo);
                            tc::mma_f16(d1, dah, dbh, idesc, kk > 0);
                            if constexpr (!kBF16) {
                                tc::mma_f16(d1, dah, tc::sdesc(wl + kk * 256, 128, sbo), idesc, 1);
                                tc::mma_f16(d1, tc::sdesc(a0l + kk * 256, 128, sbo), dbh, idesc, 1);
                            }
                        }
                        tc::commit(&empty[b]);        // buffer b may be refilled once these are done
                    } else {
                        for (int kk = 0; kk < fi / 16; ++kk) {
                            const uint64_t dbh = tc::sdesc(wh + kk * 256, 128, sbo);
                            tc::mma_f16_ta(d1, ah + (uint32_t)(kk * 8), dbh, idesc, kk > 0);
                            if constexpr (!kBF16) {
                                tc::mma_f16_ta(d1, ah + (uint32_t)(kk * 8), tc::sdesc(wl + kk * 256, 128, sbo), idesc,
                                               1);
                                tc::mma_f16_ta(d1, al + (uint32_t)(kk * 8), dbh, idesc, 1);
                            }
                        }
                    }
                    tc::commit(gbar);
                }
                if (!tc::mbar_wait(gbar, mph, kMbarLimit)) {
                    ok = false;
                    set_error(a.err, HP_ERR_TIMEOUT, -8);
                }
                mph ^= 1u;
                ok = tc::bar_and(barid, nthr, ok);
                if (!ok) break;
                tc::fence_after_sync();

                // ---- epilogue: this thread's row; 8-column chunks round-robin
                // over the column groups, kWsBatch at a time (TMEM -> registers
                // -> TMEM as the next layer's A operand; the last hidden layer
                // feeds the output layer's FMAs instead)
                const float *bias = f32 + L.bias[l];
                const bool last = (l + 1 == L.nh);
                const int nch = fo / 8;
                for (int ch0 = cg; ch0 < nch; ch0 += kWsGroups * kWsBatch) {
                    float v1[kWsBatch][8];
                    // the biases (16-byte aligned rows: widths are multiples
                    // of 16) are loaded before the TMEM loads, so the two overlap
                    float4 bq[kWsBatch][2];
#pragma unroll
                    for (int j = 0; j < kWsBatch; ++j) {
                        const int ch = ch0 + kWsGroups * j;
                        if (ch < nch) {
                            bq[j][0] = *reinterpret_cast<const float4 *>(bias + 8 * ch);
                            bq[j][1] = *reinterpret_cast<const float4 *>(bias + 8 * ch + 4);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < kWsBatch; ++j) {
                        const int ch = ch0 + kWsGroups * j;
                        if (ch < nch) tc::ld8(d1 + lane_off + (uint32_t)(8 * ch), v1[j]);
                    }
                    // the first wait completes the loads; the others only tie
                    // each array to the wait
#pragma unroll
                    for (int j = 0; j < kWsBatch; ++j) tc::wait_ld_regs(v1[j]);
#pragma unroll
                    for (int j = 0; j < kWsBatch; ++j) {
                        const int ch = ch0 + kWsGroups * j;
                        if (ch >= nch) break;
                        const int c = 8 * ch;
                        const float4 b0 = bq[j][0];
                        const float4 b1 = bq[j][1];
                        const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
                        // bias as packed pair additions (the scalar roundings)
                        uint64_t z[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            z[i] = tc::add_f32x2(tc::f32x2(v1[j][2 * i], v1[j][2 * i + 1]),
                                                 tc::f32x2(bb[2 * i], bb[2 * i + 1]));
                        if (!last) {
                            // ReLU inside the conversions; the next layer's A:
                            // columns c/2 .. c/2+3 of A_hi (and A_lo)
                            uint32_t ph[4], pl[4];
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                if constexpr (kBF16)
                                    ph[i] = tc::relu_bf16x2(z[i]);
                                else
                                    tc::split_relu_f16x2(z[i], ph[i], pl[i]);
                            }
                            tc::st4(ah + lane_off + (uint32_t)(c / 2), ph);
                            if constexpr (!kBF16) tc::st4(al + lane_off + (uint32_t)(c / 2), pl);
                        } else {
                            // ReLU; output layer: outputs (0, 1) and (2, 3) as
                            // packed FMAs in input order (each output's scalar
                            // FMA chain)
                            const float4 *W4 = reinterpret_cast<const float4 *>(f32 + L.wl) + c;
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                const float2 zz = tc::f32x2_unpack(z[i >> 1]);
                                const float h = fmaxf((i & 1) ? zz.y : zz.x, 0.0f);
                                const float4 w = W4[i];
                                const uint64_t hh = tc::f32x2(h, h);
                                o01 = tc::fma_f32x2(hh, tc::f32x2(w.x, w.y), o01);
                                o23 = tc::fma_f32x2(hh, tc::f32x2(w.z, w.w), o23);
                            }
                        }
                    }
                }
                if (!last) tc::wait_st();
                tc::fence_before_sync();
                tc::bar_and(barid, nthr, true);
                tc::fence_after_sync();
            }
            if (!ok) break;

            // ---- output layer: combine the column groups, activations
            float o4[4];
            {
                const float2 x01 = tc::f32x2_unpack(o01), x23 = tc::f32x2_unpack(o23);
                o4[0] = x01.x;
                o4[1] = x01.y;
                o4[2] = x23.x;
                o4[3] = x23.y;
            }
            if (cg > 0) {
#pragma unroll
                for (int i = 0; i < 4; ++i) gcomb[(cg * kTcTile + row) * 4 + i] = o4[i];
            }
            tc::bar_and(barid, nthr, true);
            if (cg == 0) {
                const float *bl = f32 + L.bias[a.n_layers - 1];
                float o[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    o[i] = o4[i];
#pragma unroll
                    for (int gr = 1; gr < kWsGroups; ++gr) o[i] += gcomb[(gr * kTcTile + row) * 4 + i];
                    o[i] += bl[i];
                }
                const int64_t g = base + row;
                if (g < S)
                    a.sample_out[g] = make_float4(softplus_f(o[0]), sigmoid_f(o[1]), sigmoid_f(o[2]), sigmoid_f(o[3]));
            }
        }
    }

    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tbase, kWsCols);
}

// Tensor-core decode possible for this MLP?  Hidden layers on tcgen05 need
// K (fan-in) multiple of 16 and N (width) in 16..128 step 16.
bool decode_tc_supported(const RenderArgs &a, bool bf16, size_t *smem)
{
    if (a.n_layers < 2) return false;
    for (int l = 0; l + 1 < a.n_layers; ++l) {
        const int fi = a.dims[l], fo = a.dims[l + 1];
        if (fi % 16 != 0 || fi > 128 || fo % 16 != 0 || fo < 16 || fo > 128) return false;
    }
    const TcLayout L = tc_layout(a, bf16);
    if (smem) *smem = (size_t)L.total;
    return L.total <= kSmemLimit;
}

cudaError_t launch_decode_tc(const RenderArgs &a, bool bf16, cudaStream_t st, int *n_kernels)
{
    *n_kernels = 1;
    cudaError_t e;
    const int bulk_ok_ws = a.nbr ? (((uintptr_t)a.nbr % 16 == 0) && ((uintptr_t)a.nbr_dist % 16 == 0) ? 1 : 0)
                                 : ((a.K % 4 == 0) && a.K <= 16 && ((uintptr_t)a.slot_nbr % 16 == 0) &&
                                    ((uintptr_t)a.slot_dist % 16 == 0) ? 2 : 0);
    const WsLayout W = ws_layout(a, bf16);
    if (W.ok) {
        const bool narrow = a.K > 8;           // 8 consumer warps
        auto kern = bf16 ? (narrow ? k_decode_ws<true, 8> : k_decode_ws<true, 16>)
                         : (narrow ? k_decode_ws<false, 8> : k_decode_ws<false, 16>);
        const int threads = ws_threads(narrow ? 8 : 16);
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, W.total)) != cudaSuccess)
            return e;
        if (ws_image_bytes(W) > kWsImageMax || (uintptr_t)a.wimg % 16 != 0) return cudaErrorInvalidValue;
        int64_t grid = a.num_sms;
        const int64_t tiles = div_up(a.capacity > 0 ? a.capacity : 1, kTcTile);
        if (grid > tiles) grid = tiles;
        launch_chained(bf16 ? k_ws_image<true> : k_ws_image<false>, (unsigned)a.num_sms, 256, 0, st, a, W);
        launch_chained(kern, (unsigned)grid, threads, W.total, st, a, W, bulk_ok_ws);
        *n_kernels = 2;
        return cudaGetLastError();
    }
    const TcLayout L = tc_layout(a, bf16);
    auto kern = bf16 ? k_decode_tc<true> : k_decode_tc<false>;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total)) != cudaSuccess)
        return e;
    int64_t grid = a.num_sms;
    const int64_t tiles = div_up(a.capacity > 0 ? a.capacity : 1, kTcTile);
    if (grid > tiles) grid = tiles;
    const int bulk_ok = a.nbr && ((uintptr_t)a.nbr % 16 == 0) && ((uintptr_t)a.nbr_dist % 16 == 0);
    launch_chained(kern, (unsigned)grid, kTcThreads, L.total, st, a, L, bulk_ok);
    return cudaGetLastError();
}

cudaError_t launch_mma_selftest(const uint16_t *A, const uint16_t *B, float *D, int K, int N, int flags, ErrWord *err,
                                cudaStream_t st)
{
    cudaError_t e;
    const size_t smem = (size_t)128 * K * 2 + (size_t)N * K * 2 + 32;
    if ((e = cudaFuncSetAttribute(k_mma_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    k_mma_selftest<<<1, 128, smem, st>>>(A, B, D, K, N, flags, err);
    return cudaGetLastError();
}

}  // namespace hp
