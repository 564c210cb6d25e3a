// Table build (Sec. 3.2, "Accelerated structure construction"): every visible
// point is projected to its pixel; all points of a pixel are kept (no
// z-buffer); the point list is reordered so that each pixel's points are
// contiguous, and the table holds, per pixel key, the start of its run (the
// count is the difference of consecutive starts).
//
// K1 k_project_count  camera transform + key, one atomic count per point;
//                     the atomic's return value is the point's slot in its run
// K2 k_scan           exclusive prefix sum of the counts (decoupled look-back)
// K3 k_scatter        each point written to start[key] + slot as float4
//                     (camera x, y, z, id bits), with its bucket beside it
// K4 k_bucket_sort    each run ordered by (z, x, y, id), which makes the list
//                     independent of the atomics' order and of the input order:
//                     one thread per bucket sorts a small bucket in registers;
//                     k_bucket_sort_big ranks the points of larger buckets,
//                     one warp per bucket.  Nothing the search, the sampling or
//                     the proposal computes depends on the order inside a
//                     bucket (every walk tests all of a bucket's points and
//                     every selection orders candidates by (t, id)), so the
//                     frame leaves the scatter's order and the sort runs when
//                     the table is read out (hp_table_copy)
#include "hp_kernels.cuh"

namespace hp {

__global__ void __launch_bounds__(256) k_project_count(const float *__restrict__ pts, int64_t N, Cam cam, int h,
                                                       uint32_t *__restrict__ cnt, uint2 *__restrict__ keyrank,
                                                       uint32_t *__restrict__ zmin_enc)
{
    grid_dep_wait();
    grid_dep_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool in = i < N;
    uint32_t key = kNoKey;
    float X_z = 0.0f;
    if (in) {
        float3 X = cam_point(cam, __ldg(pts + 3 * i), __ldg(pts + 3 * i + 1), __ldg(pts + 3 * i + 2));
        key = pixel_key(cam, h, X);
        X_z = X.z;
    }
    const bool valid = in && key != kNoKey;
    // the smallest depth of a tabled point, encoded so that atomicMax takes
    // it (a depth <= 0, possible only with z_near < 0, counts as 0)
    __shared__ uint32_t s_ze;
    if (threadIdx.x == 0) s_ze = 0u;
    __syncthreads();
    const uint32_t ze = __reduce_max_sync(
        0xffffffffu, valid ? (X_z > 0.0f ? 0x7f800000u - (uint32_t)__float_as_int(X_z) : 0x7f800000u) : 0u);
    if (lane == 0 && ze != 0u) atomicMax(&s_ze, ze);
    __syncthreads();
    if (threadIdx.x == 0 && s_ze != 0u) atomicMax(zmin_enc, s_ze);   // one global atomic per block
    uint32_t rank = 0;
    // one atomic per point; its return value is the point's slot in its run
    if (valid) rank = atomicAdd(cnt + key, 1u);
    if (in) keyrank[i] = make_uint2(key, rank);
}

// Exclusive scan of n uint32 values; tile = kScanTile entries.
__global__ void __launch_bounds__(kScanThreads) k_scan(const uint32_t *__restrict__ in, uint32_t *__restrict__ out,
                                                      int64_t n, uint64_t *flags, uint32_t *ticket, ErrWord *err,
                                                      uint32_t spin_limit, int32_t skip_tile)
{
    grid_dep_wait();
    grid_dep_trigger();
    __shared__ int64_t s_tile;
    __shared__ int64_t s_prefix;
    __shared__ uint32_t s_warp[kScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * kScanTile + (int64_t)tid * kScanItems;
    uint32_t v[kScanItems];
    if (base + kScanItems <= n) {
        const uint4 a = *reinterpret_cast<const uint4 *>(in + base);
        const uint4 b = *reinterpret_cast<const uint4 *>(in + base + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) v[k] = (base + k < n) ? in[base + k] : 0u;
    }
    // tile arithmetic modulo 2^32 (the sums wrap like the uint32 result); the
    // tile aggregate is published zero-extended, so the look-back's 62-bit
    // sums of up to 2^26 / kScanTile aggregates never reach the state bits
    uint32_t tsum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) tsum += v[k];
    const uint32_t incl = warp_incl_scan_u32(tsum);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < kScanThreads / 32 ? s_warp[lane] : 0u;
        const uint32_t wi = warp_incl_scan_u32(w);
        if (lane < kScanThreads / 32) s_warp[lane] = wi - w;      // exclusive warp offsets
        const int64_t agg = (int64_t)__shfl_sync(0xffffffffu, wi, kScanThreads / 32 - 1);
        const int64_t pre = lookback_prefix_warp(flags, tile, agg, err, spin_limit, tile != skip_tile);
        if (lane == 0) s_prefix = pre;
    }
    __syncthreads();
    uint32_t run = (uint32_t)s_prefix + s_warp[warp] + (incl - tsum);
    uint32_t o[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        o[k] = run;
        run += v[k];
    }
    if (base + kScanItems <= n) {
        *reinterpret_cast<uint4 *>(out + base) = make_uint4(o[0], o[1], o[2], o[3]);
        *reinterpret_cast<uint4 *>(out + base + 4) = make_uint4(o[4], o[5], o[6], o[7]);
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k)
            if (base + k < n) out[base + k] = o[k];
    }
}

__global__ void __launch_bounds__(256) k_scatter(const float *__restrict__ pts, int64_t N, Cam cam,
                                                 const uint2 *__restrict__ keyrank,
                                                 const uint32_t *__restrict__ start, float4 *__restrict__ spts,
                                                 uint32_t *__restrict__ pcell, ErrWord *err)
{
    grid_dep_wait();
    grid_dep_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint2 kr = keyrank[i];
    if (kr.x == kNoKey) return;
    // the same float32 sequence as K1, so the stored position is the one keyed
    float3 X = cam_point(cam, __ldg(pts + 3 * i), __ldg(pts + 3 * i + 1), __ldg(pts + 3 * i + 2));
    const uint32_t slot = start[kr.x] + kr.y;
    if (!hp_check(slot < N, err, slot)) return;
    spts[slot] = make_float4(X.x, X.y, X.z, __int_as_float((int)i));
    pcell[slot] = kr.x;
}

__device__ __forceinline__ bool pt_less(const float4 &a, const float4 &b)
{
    if (a.z != b.z) return a.z < b.z;
    if (a.x != b.x) return a.x < b.x;
    if (a.y != b.y) return a.y < b.y;
    return __float_as_int(a.w) < __float_as_int(b.w);
}

// Buckets are ordered by (z, x, y, id) -- a strict total order, ids being
// distinct.  One thread per bucket sorts a bucket of up to kSmallBucket points
// in registers (consecutive threads read and write consecutive ranges); a
// larger bucket goes on a list that one warp per bucket ranks: each point's
// place is the number of the bucket's points before it.
constexpr int kSmallBucket = 8;
constexpr unsigned kBigSortBlocks = 888;   // warps loop over the large-bucket list (6 blocks per SM of 148)

__global__ void __launch_bounds__(256) k_bucket_sort(int64_t P, const uint32_t *__restrict__ start,
                                                     const float4 *__restrict__ tmp, float4 *__restrict__ spts,
                                                     uint32_t *__restrict__ big, uint32_t *__restrict__ n_big)
{
    grid_dep_wait();
    grid_dep_trigger();
    const int64_t bkt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (bkt >= P) return;
    const uint32_t a = __ldg(start + bkt), n = __ldg(start + bkt + 1) - a;
    if (n == 0) return;
    if (n > (uint32_t)kSmallBucket) {
        big[atomicAdd(n_big, 1u)] = (uint32_t)bkt;
        return;
    }
    float4 v[kSmallBucket];
#pragma unroll
    for (int i = 0; i < kSmallBucket; ++i)
        if (i < (int)n) v[i] = __ldg(tmp + a + i);
    // insertion sort with fixed register indices: v[i] sinks into the sorted prefix
#pragma unroll
    for (int i = 1; i < kSmallBucket; ++i) {
        if (i < (int)n) {
#pragma unroll
            for (int j = i; j > 0; --j) {
                if (pt_less(v[j], v[j - 1])) {
                    const float4 t = v[j];
                    v[j] = v[j - 1];
                    v[j - 1] = t;
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < kSmallBucket; ++i)
        if (i < (int)n) spts[a + i] = v[i];
}

constexpr int kBigStage = 128;   // points of a large bucket staged in shared memory per warp (larger ones: from global memory)

__global__ void __launch_bounds__(256) k_bucket_sort_big(const uint32_t *__restrict__ start,
                                                         const float4 *__restrict__ tmp, float4 *__restrict__ spts,
                                                         const uint32_t *__restrict__ big,
                                                         const uint32_t *__restrict__ n_big)
{
    grid_dep_wait();
    grid_dep_trigger();
    __shared__ float4 s_pts[8][kBigStage];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 *sp = s_pts[warp];
    const uint32_t nb = *n_big;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nb; w += (gridDim.x * blockDim.x) >> 5) {
        const uint32_t bkt = big[w];
        const uint32_t a = __ldg(start + bkt), b = __ldg(start + bkt + 1), n = b - a;
        if (n <= (uint32_t)kBigStage) {
            // the bucket in shared memory (coalesced), then ranks from broadcast reads
            for (uint32_t p = lane; p < n; p += 32) sp[p] = __ldg(tmp + a + p);
            __syncwarp();
            for (uint32_t p = lane; p < n; p += 32) {
                const float4 x = sp[p];
                uint32_t rank = 0;
                for (uint32_t j = 0; j < n; ++j) rank += pt_less(sp[j], x) ? 1u : 0u;
                spts[a + rank] = x;
            }
            __syncwarp();
        } else {
            for (uint32_t p = a + lane; p < b; p += 32) {
                const float4 x = __ldg(tmp + p);
                uint32_t rank = 0;
                for (uint32_t j = a; j < b; ++j) rank += pt_less(__ldg(tmp + j), x) ? 1u : 0u;
                spts[a + rank] = x;
            }
        }
    }
}

// Zeroes n 32-bit words: the tickets, look-back words and counts a pass
// starts from (a kernel, so that it chains with its neighbours).
__global__ void __launch_bounds__(256) k_clear(uint32_t *__restrict__ p, int64_t n)
{
    grid_dep_wait();
    grid_dep_trigger();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = 0u;
}

cudaError_t launch_clear(void *p, size_t bytes, cudaStream_t st, Prof *prof)
{
    if (bytes % 4 != 0 || reinterpret_cast<uintptr_t>(p) % 4 != 0) return cudaErrorInvalidValue;
    const int64_t n = (int64_t)(bytes / 4);
    if (n == 0) return cudaSuccess;
    const int64_t blocks = div_up(n, 256) < 4096 ? div_up(n, 256) : 4096;
    prof_begin(prof, st, KID_CLEAR);
    launch_chained(k_clear, (unsigned)blocks, 256, 0, st, static_cast<uint32_t *>(p), n);
    prof_end(prof, st);
    return cudaGetLastError();
}

cudaError_t launch_build(const BuildArgs &a, cudaStream_t st, Prof *prof)
{
    cudaError_t e;
    const int64_t n_scan = a.P + 1;
    const int64_t scan_tiles = div_up(n_scan, kScanTile);
    // the scan's ticket, the depth minimum (scan_ticket[1] == zmin_enc), the
    // large-bucket count of the sort (scan_ticket[2]), the look-back words and
    // the counts lie in this order, back to back: one memset clears them
    const char *z0 = reinterpret_cast<const char *>(a.scan_ticket);
    const char *zf = reinterpret_cast<const char *>(a.scan_flags);
    const char *zc = reinterpret_cast<const char *>(a.cnt);
    if (!(zf >= z0 + 3 * sizeof(uint32_t) && zc >= zf + sizeof(uint64_t) * (size_t)scan_tiles))
        return cudaErrorInvalidValue;
    if ((e = launch_clear(a.scan_ticket, (size_t)(zc - z0) + sizeof(uint32_t) * (size_t)n_scan, st, prof)) !=
        cudaSuccess)
        return e;
    if (a.N > 0) {
        prof_begin(prof, st, KID_PROJECT);
        launch_chained(k_project_count, (unsigned)div_up(a.N, 256), 256, 0, st, a.pts, a.N, a.cam, a.h, a.cnt, a.keyrank, a.zmin_enc);
        prof_end(prof, st);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    prof_begin(prof, st, KID_SCAN);
    launch_chained(k_scan, (unsigned)scan_tiles, kScanThreads, 0, st, a.cnt, a.start, n_scan, a.scan_flags, a.scan_ticket,
                                                          a.err, a.spin_limit, a.skip_tile);
    prof_end(prof, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (a.N > 0) {
        prof_begin(prof, st, KID_SCATTER);
        launch_chained(k_scatter, (unsigned)div_up(a.N, 256), 256, 0, st, a.pts, a.N, a.cam, a.keyrank, a.start, a.spts, a.pcell,
                       a.err);
        prof_end(prof, st);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_bucket_sort(int64_t P, const uint32_t *start, const float4 *list, float4 *out, uint32_t *big,
                               uint32_t *n_big, cudaStream_t st)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(n_big, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
    launch_chained(k_bucket_sort, (unsigned)div_up(P, 256), 256, 0, st, P, start, list, out, big, n_big);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    launch_chained(k_bucket_sort_big, kBigSortBlocks, 256, 0, st, start, list, out, big, n_big);
    return cudaGetLastError();
}

}  // namespace hp
