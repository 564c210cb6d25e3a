// Window search (Sec. 3.2 "Searching") and adaptive primary surface sampling
// (Sec. 3.3), fused in one kernel.
//
// A block owns a tile of kRaysPerCta consecutive rays (tile number from an
// atomic ticket) and its warps take rays one at a time.  For a ray through
// pixel (u, v) the s x s window of buckets is s rows of the padded table;
// the buckets of one row are adjacent keys, so each row's points are one
// contiguous run of the reordered list [start[k], start[k+s]).  A warp reads
// a run 32 points at a time (one coalesced 512-byte load), tests the radius
// predicate in every lane and appends the accepted points with a ballot
// prefix into its shared-memory candidate buffer.  The buffer is sorted by
// (t, id) with a warp bitonic sort; then, candidate by candidate in depth
// order, the warp finds the K nearest candidates within r(t_j) of the
// sample (warp min-reductions), forms d_j, alpha_j and w_j, and applies the
// primary-cluster rule, stopping as soon as the cluster ends.  Samples are
// staged in shared memory; the tile's sample count is turned into its global
// offset with a decoupled look-back, and the tile writes its samples packed,
// ray by ray, so the output order is independent of scheduling.
#include "hp_kernels.cuh"

namespace hp {

namespace {

constexpr unsigned kFull = 0xffffffffu;

struct SearchSmem {
    size_t cp, ck, st, ssrc, sdel, snbr, sdist, sns, soff, map, ci, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline SearchSmem search_layout(int K, int n_max)
{
    SearchSmem L;
    size_t o = 0;
    const size_t slots = (size_t)kRaysPerCta * n_max;
    L.cp = o;    o += sizeof(float4) * kCandCap * kSearchWarps;
    L.ck = o;    o += sizeof(uint64_t) * kCandCap * kSearchWarps;
    L.st = o;    o += align16(4 * slots);
    L.ssrc = o;  o += align16(4 * slots);
    L.sdel = o;  o += align16(4 * slots);
    L.snbr = o;  o += align16(4 * slots * K);
    L.sdist = o; o += align16(4 * slots * K);
    L.sns = o;   o += align16(4 * kRaysPerCta);
    L.soff = o;  o += align16(4 * (kRaysPerCta + 1));
    L.map = o;   o += align16(2 * slots);
    L.ci = o;    o += align16((size_t)kCandCap * kSearchWarps);
    L.total = o;
    return L;
}

// Radius test: t = (X dx + Y dy) + Z dz, e = P - t d (one rounding per axis),
// rho2 = (ex^2 + ey^2) + ez^2; accept iff t in [t_near, t_far] and rho2 <= r(t)^2.
__device__ __forceinline__ bool accept_point(const SearchArgs &a, const Ray &ray, const float4 &p, float &t)
{
    t = dadd(dadd(dmul(p.x, ray.dx), dmul(p.y, ray.dy)), dmul(p.z, ray.dz));
    if (!(t >= a.cam.t_near && t <= a.cam.t_far)) return false;
    const float ex = dfma(-t, ray.dx, p.x);
    const float ey = dfma(-t, ray.dy, p.y);
    const float ez = dfma(-t, ray.dz, p.z);
    const float rho2 = dadd(dadd(dmul(ex, ex), dmul(ey, ey)), dmul(ez, ez));
    const float rad = radius_at(a.mode, a.r, ray, t);
    return rho2 <= dmul(rad, rad);
}

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

}  // namespace

__global__ void __launch_bounds__(kSearchWarps * 32) k_search_select(const SearchArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t s_tile, s_prefix;
    __shared__ int s_next, s_total;
    const SearchSmem L = search_layout(a.K, a.n_max);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    if (tid == 0) {
        s_tile = atomicAdd(a.ticket, 1u);
        s_next = 0;
    }
    __syncthreads();
    const int64_t tile = s_tile;

    float4 *cp = reinterpret_cast<float4 *>(smem + L.cp) + warp * kCandCap;
    uint64_t *ck = reinterpret_cast<uint64_t *>(smem + L.ck) + warp * kCandCap;
    uint8_t *ci = reinterpret_cast<uint8_t *>(smem + L.ci) + warp * kCandCap;
    float *stg_t = reinterpret_cast<float *>(smem + L.st);
    int *stg_src = reinterpret_cast<int *>(smem + L.ssrc);
    float *stg_del = reinterpret_cast<float *>(smem + L.sdel);
    int *stg_nbr = reinterpret_cast<int *>(smem + L.snbr);
    float *stg_dist = reinterpret_cast<float *>(smem + L.sdist);
    int *s_ns = reinterpret_cast<int *>(smem + L.sns);
    int *s_off = reinterpret_cast<int *>(smem + L.soff);
    uint16_t *s_map = reinterpret_cast<uint16_t *>(smem + L.map);

    const int K = a.K, n_max = a.n_max, span = 2 * a.h + 1;
    const int64_t npix = (int64_t)a.cam.width * a.cam.height;

    for (;;) {
        int rl = 0;
        if (lane == 0) rl = atomicAdd(&s_next, 1);
        rl = __shfl_sync(kFull, rl, 0);
        if (rl >= kRaysPerCta) break;
        const int64_t ri = tile * kRaysPerCta + rl;
        if (ri >= a.R) {
            if (lane == 0) s_ns[rl] = 0;
            continue;
        }
        const int64_t pix = a.rays ? (int64_t)__ldg(a.rays + ri) : ri;
        if (pix < 0 || pix >= npix) {
            if (lane == 0) {
                set_error(a.err, HP_ERR_BAD_RAY, ri);
                a.n_s[ri] = 0;
                a.primary[ri] = -1;
                a.cand_count[ri] = 0;
                s_ns[rl] = 0;
            }
            continue;
        }
        const int pu = (int)(pix % a.cam.width), pv = (int)(pix / a.cam.width);
        const Ray ray = make_ray(a.cam, a.mode, a.rdd, pu, pv);

        // ---- window walk: s rows, each a contiguous run of the list
        int kept = 0, total = 0;
        for (int dy = 0; dy < span; ++dy) {
            const int64_t kb = (int64_t)(pv + dy) * a.Wp + pu;
            const uint32_t lo = __ldg(a.start + kb), hi = __ldg(a.start + kb + span);
            for (uint32_t b0 = lo; b0 < hi; b0 += 32) {
                const uint32_t i = b0 + lane;
                bool acc = false;
                float t = 0.0f;
                float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
                if (i < hi) {
                    p = __ldg(a.spts + i);
                    acc = accept_point(a, ray, p, t);
                }
                const unsigned m = __ballot_sync(kFull, acc);
                if (m == 0) continue;
                const int n = __popc(m);
                const uint64_t key = ((uint64_t)__float_as_uint(t) << 32) | (uint32_t)__float_as_int(p.w);
                if (kept + n <= a.cand_cap) {
                    if (acc) {
                        const int pos = kept + __popc(m & lt_mask);
                        ck[pos] = key;
                        cp[pos] = p;
                    }
                    kept += n;
                } else {
                    // buffer full: keep the cand_cap smallest (t, id), one insertion at a time
                    __syncwarp();
                    unsigned mm = m;
                    while (mm) {
                        const int sl = __ffs(mm) - 1;
                        mm &= mm - 1;
                        const uint64_t kk = __shfl_sync(kFull, key, sl);
                        float4 pp;
                        pp.x = __shfl_sync(kFull, p.x, sl);
                        pp.y = __shfl_sync(kFull, p.y, sl);
                        pp.z = __shfl_sync(kFull, p.z, sl);
                        pp.w = __shfl_sync(kFull, p.w, sl);
                        if (kept < a.cand_cap) {
                            if (lane == 0) {
                                ck[kept] = kk;
                                cp[kept] = pp;
                            }
                            ++kept;
                        } else {
                            uint64_t best = 0;
                            int bi = -1;
                            for (int e = lane; e < a.cand_cap; e += 32) {
                                const uint64_t v = ck[e];
                                if (bi < 0 || v > best) { best = v; bi = e; }
                            }
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1) {
                                const uint64_t ob = __shfl_xor_sync(kFull, best, o);
                                const int oi = __shfl_xor_sync(kFull, bi, o);
                                if (oi >= 0 && (bi < 0 || ob > best)) { best = ob; bi = oi; }
                            }
                            if (kk < best && lane == 0) {
                                ck[bi] = kk;
                                cp[bi] = pp;
                            }
                        }
                        __syncwarp();
                    }
                }
                total += n;
            }
        }
        __syncwarp();

        // ---- sort the candidates by (t, id): bitonic network in shared memory
        const int C = kept;
        if (C > 1) {
            int n2 = 2;
            while (n2 < C) n2 <<= 1;
            for (int e = C + lane; e < n2; e += 32) ck[e] = ~0ull;
            for (int e = lane; e < n2; e += 32) ci[e] = (uint8_t)e;
            __syncwarp();
            for (int k = 2; k <= n2; k <<= 1) {
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int e = lane; e < n2; e += 32) {
                        const int x = e ^ j;
                        if (x > e) {
                            const bool up = (e & k) == 0;
                            const uint64_t A = ck[e], B = ck[x];
                            if ((A > B) == up) {
                                ck[e] = B;
                                ck[x] = A;
                                const uint8_t t8 = ci[e];
                                ci[e] = ci[x];
                                ci[x] = t8;
                            }
                        }
                    }
                    __syncwarp();
                }
            }
        } else if (C == 1) {
            if (lane == 0) ci[0] = 0;
            __syncwarp();
        }

        float4 P[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int i = lane + 32 * m;
            P[m] = (i < C) ? cp[ci[i]] : make_float4(0.f, 0.f, 0.f, 0.f);
        }

        // ---- adaptive primary surface sampling
        float T = 1.0f, t_prev = 0.0f;
        int jstar = -1, ns = 0, prim = -1;
        const int slot0 = rl * n_max;
        for (int j = 0; j < C; ++j) {
            const uint64_t kj = ck[j];
            const float tj = __uint_as_float((uint32_t)(kj >> 32));
            if (jstar >= 0) {
                const float gap = dsub(tj, t_prev);
                if (!(gap <= dmul(a.gap_k, radius_at(a.mode, a.r, ray, t_prev)))) break;
            }
            const float rad = radius_at(a.mode, a.r, ray, tj);
            const float rad2 = dmul(rad, rad);
            uint64_t q[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                q[m] = ~0ull;
                if (lane + 32 * m < C) {
                    const float ax = dfma(tj, ray.dx, -P[m].x);
                    const float ay = dfma(tj, ray.dy, -P[m].y);
                    const float az = dfma(tj, ray.dz, -P[m].z);
                    const float d2 = dadd(dadd(dmul(ax, ax), dmul(ay, ay)), dmul(az, az));
                    if (d2 <= rad2) q[m] = ((uint64_t)__float_as_uint(d2) << 32) | (uint32_t)__float_as_int(P[m].w);
                }
            }
            float s = 0.0f;
            int kp = 0, my_id = -1;
            float my_d = 0.0f;
            for (int k = 0; k < K; ++k) {
                uint64_t mn = umin64(umin64(q[0], q[1]), umin64(q[2], q[3]));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) mn = umin64(mn, __shfl_xor_sync(kFull, mn, o));
                if (mn == ~0ull) break;
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    if (q[m] == mn) q[m] = ~0ull;
                const float dist = dsqrt(__uint_as_float((uint32_t)(mn >> 32)));
                s = dadd(s, dist);
                if (lane == k) {
                    my_id = (int)(uint32_t)mn;
                    my_d = dist;
                }
                ++kp;
            }
            const float dj = ddiv(s, (float)kp);
            const float alpha = dmul(a.gamma, exp32(-ddiv(dmul(dj, dj), a.beta2)));
            const float w = dmul(alpha, T);
            T = dmul(T, dsub(1.0f, alpha));
            if (w > a.eps_w) {
                if (jstar < 0) {
                    jstar = j;
                    const float4 pj = cp[ci[j]];
                    prim = (int)pixel_key(a.cam, a.h, make_float3(pj.x, pj.y, pj.z));
                }
                const int slot = slot0 + ns;
                if (lane < K) {
                    stg_nbr[slot * K + lane] = my_id;
                    stg_dist[slot * K + lane] = my_d;
                }
                if (lane == 0) {
                    stg_t[slot] = tj;
                    stg_src[slot] = (int)(uint32_t)kj;
                }
                if (++ns == n_max) break;
            }
            t_prev = tj;
        }
        __syncwarp();
        if (lane < ns) {
            const int slot = slot0 + lane;
            const float tm = stg_t[slot];
            stg_del[slot] = (lane + 1 < ns) ? stg_t[slot + 1] - tm : 2.0f * radius_at(a.mode, a.r, ray, tm);
        }
        if (lane == 0) {
            a.n_s[ri] = ns;
            a.primary[ri] = prim;
            a.cand_count[ri] = total;
            s_ns[rl] = ns;
        }
        __syncwarp();
    }
    __syncthreads();

    // ---- tile prefix: exclusive scan of the per-ray counts, then look-back
    if (warp == 0) {
        const int v0 = s_ns[lane], v1 = s_ns[lane + 32];
        const int i0 = warp_incl_scan(v0);
        const int t0 = __shfl_sync(kFull, i0, 31);
        const int i1 = warp_incl_scan(v1) + t0;
        s_off[lane] = i0 - v0;
        s_off[lane + 32] = i1 - v1;
        if (lane == 31) {
            s_off[kRaysPerCta] = i1;
            s_total = i1;
            s_prefix = lookback_prefix(a.flags, tile, i1, a.err, a.spin_limit, true);
        }
    }
    __syncthreads();
    const int total = s_total;
    const int64_t prefix = s_prefix;
    for (int rl = tid; rl < kRaysPerCta; rl += blockDim.x) {
        const int64_t ri = tile * kRaysPerCta + rl;
        if (ri < a.R) a.sample_offset[ri] = prefix + s_off[rl];
        if (ri == a.R - 1) a.sample_offset[a.R] = prefix + s_off[rl] + s_ns[rl];
    }
    for (int e = tid; e < kRaysPerCta * n_max; e += blockDim.x) {
        const int rl = e / n_max, m = e - rl * n_max;
        if (m < s_ns[rl]) s_map[s_off[rl] + m] = (uint16_t)e;
    }
    __syncthreads();
    if (tid == 0 && prefix + total > a.capacity) set_error(a.err, HP_ERR_OVERFLOW, prefix + total);
    for (int e = tid; e < total; e += blockDim.x) {
        const int64_t g = prefix + e;
        if (g >= a.capacity) break;
        const int slot = s_map[e];
        a.t[g] = stg_t[slot];
        a.ray[g] = (int)(tile * kRaysPerCta + slot / n_max);
        a.src[g] = stg_src[slot];
        a.delta[g] = stg_del[slot];
    }
    for (int e = tid; e < total * K; e += blockDim.x) {
        const int s = e / K, k = e - s * K;
        const int64_t g = prefix + s;
        if (g >= a.capacity) break;
        const int slot = s_map[s];
        a.nbr[g * K + k] = stg_nbr[slot * K + k];
        a.nbr_dist[g * K + k] = stg_dist[slot * K + k];
    }
}

size_t search_smem_bytes(int K, int n_max) { return search_layout(K, n_max).total; }

cudaError_t launch_search(const SearchArgs &a, cudaStream_t st, Prof *prof)
{
    cudaError_t e;
    const int64_t tiles = div_up(a.R, kRaysPerCta);
    if ((e = cudaMemsetAsync(a.flags, 0, sizeof(uint64_t) * (size_t)tiles, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.ticket, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
    const size_t smem = search_smem_bytes(a.K, a.n_max);
    if ((e = cudaFuncSetAttribute(k_search_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    prof_begin(prof, st, KID_SEARCH);
    k_search_select<<<(unsigned)tiles, kSearchWarps * 32, smem, st>>>(a);
    prof_end(prof, st);
    return cudaGetLastError();
}

}  // namespace hp
