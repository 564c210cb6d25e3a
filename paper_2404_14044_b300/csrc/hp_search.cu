// Window search (Sec. 3.2 "Searching") and adaptive primary surface sampling
// (Sec. 3.3), fused.
//
// k_search_splat (whole frames, plain search): one thread per tabled point
// tests it against the ray of every pixel whose window holds its bucket and
// appends the accepted depth and table index to that pixel's slots (two
// arrays; an atomic count per pixel; kPmCap slots), listing the pixels whose
// count passes the slots.  Rays then only select.
//
// k_search_select: one thread per ray.  A warp owns an 8 x 4 tile of pixels
// (whole frames) or 32 consecutive listed rays.  The lane gathers its ray's
// accepted points into its own column of a [cap][32] shared-memory array
// (conflict-free whatever the counts; cap kLaneCapShort for the point-major
// selection and the restricted walk, kLaneCap for the plain and learned
// walks): from the point-major slots, or
// by walking the s x s window itself (listed rays, restricted searches; a
// window row of s buckets is s adjacent keys, so one contiguous run of the
// reordered list).  The column stays unsorted: candidate j+1 is the smallest
// (t, id) above candidate j, found by a scan, and the selection visits only
// ~1.4 candidates a ray.  For candidate j the lane collects the K nearest
// candidates within r(t_j) of the sample (only those within that distance in
// t can qualify), forms d_j and alpha_j, applies the weight and the primary-
// cluster rule, and stops when the cluster ends, when n samples are kept or
// when gamma * T_j <= eps_w (no later weight can pass).  Whole frames: the
// column keeps only the prefix of the (t, id) order the selection can reach
// (prune_m), and the warps first search the overflowed pixels with the
// warp-per-ray code.  Rays with more candidates than a column holds are
// listed for k_search_select_wide.
//
// k_search_select_wide: one warp per listed ray.  The candidates come from
// the point-major slots, or from a walk that reads the concatenated runs 32
// points at a time and appends the accepted ones with a ballot prefix
// (keeping the cand_cap smallest (t, id)).  Lane l holds candidates l, l+32,
// l+64, l+96; candidates are taken in (t, id) order by warp minima and each
// one's K nearest are ranked in shared memory.
//
// Each ray writes its samples into n_samples slots of a scratch area (slot m
// of ray i at m R + i); K6 packs them ray by ray (scan + copy; the neighbour
// lists may stay in the slots, K6 then writing each sample's slot index), so
// the output order is independent of scheduling and blocks never wait on one
// another while they search.
#include <algorithm>
#include <type_traits>

#include "hp_kernels.cuh"
#include "hp_proposal.cuh"

namespace hp {

namespace {

constexpr unsigned kFull = 0xffffffffu;

struct SearchSmem {
    size_t cp, ck, total;
};

__host__ __device__ inline SearchSmem search_layout()
{
    SearchSmem L;
    size_t o = 0;
    L.cp = o; o += sizeof(float4) * kCandCap * kSearchWarps;
    L.ck = o; o += sizeof(uint64_t) * kCandCap * kSearchWarps;
    L.total = o;
    return L;
}

// Radius test: t = (X dx + Y dy) + Z dz, e = P - t d (one rounding per axis),
// rho2 = (ex^2 + ey^2) + ez^2; accept iff t in [t_near, t_far] and rho2 <= r(t)^2.
__device__ __forceinline__ bool accept_point(const SearchArgs &a, const Ray &ray, const float4 &p, float tn, float tf,
                                             float &t)
{
    t = dadd(dadd(dmul(p.x, ray.dx), dmul(p.y, ray.dy)), dmul(p.z, ray.dz));
    if (!(t >= tn && t <= tf)) return false;
    const float ex = dfma(-t, ray.dx, p.x);
    const float ey = dfma(-t, ray.dy, p.y);
    const float ez = dfma(-t, ray.dz, p.z);
    const float rho2 = dadd(dadd(dmul(ex, ex), dmul(ey, ey)), dmul(ez, ez));
    const float rad = radius_at(a.mode, a.r, ray, t);
    return rho2 <= dmul(rad, rad);
}

// Window half-width of the plain search.  An accepted point P lies within
// r(t) of the ray point X nearest to it; along the segment X-P the depth
// falls by at most r sin(theta_max) below P's own, so the projection offset
// of every accepted point obeys the window bound of the table (h, derived
// from t_near) and the same bound taken at the smallest depth of any tabled
// point minus r sin(theta_max): the smaller window finds the same points.
// Fixed radius only (the cone modes keep h).
__device__ __forceinline__ int plain_window(const SearchArgs &a)
{
    int h = a.h;
    if (a.mode == HP_RADIUS_FIXED && a.zmin_enc) {
        const uint32_t e = __ldg(a.zmin_enc);
        if (e != 0u) {
            const float zmin = __int_as_float((int)(0x7f800000u - e));
            const float zlo = fmaxf(dsub(zmin, dmul(a.r, a.sin_max)), a.cam.z_near);
            const float lim = dadd(dmul(ddiv(a.win_fx, zlo), 1.001f), 1e-3f);
            if (lim < (float)h) h = min(h, (int)floorf(dadd(lim, 0.5f)));
        }
    }
    return h;
}

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t u = __shfl_xor_sync(kFull, v, o);
        v = u < v ? u : v;
    }
    return v;
}

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t u = __shfl_xor_sync(kFull, v, o);
        v = u > v ? u : v;
    }
    return v;
}

// Point-major candidate pass (whole frames, plain search): one thread per
// tabled point tests it against the ray of every pixel whose window holds its
// bucket -- the (point, ray) pairs the ray-major walk tests, each once -- and
// appends the accepted ones, (t, table index), to that pixel's slots.  The
// points are read once, coalesced; the appends are in any order, and the
// selection takes candidates in (t, id) order whatever their order.
__global__ void __launch_bounds__(256) k_search_splat(const SearchArgs a)
{
    grid_dep_wait();
    grid_dep_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int Hp = a.cam.height + 2 * a.h;
    const int64_t nv = (int64_t)__ldg(a.start + (int64_t)a.Wp * Hp);
    if (i >= nv || i >= a.n_points) return;
    const float4 p = __ldg(a.spts + i);
    const uint32_t key = __ldg(a.pcell + i);
    const int kv = (int)(key / (uint32_t)a.Wp), ku = (int)(key - (uint32_t)kv * (uint32_t)a.Wp);
    // pixel (pu, pv) walks buckets pu + o .. pu + o + 2 hw (padded), o = h - hw
    const int hw = plain_window(a), o = a.h - hw;
    const int W = a.cam.width, H = a.cam.height;
    const int pu0 = max(ku - o - 2 * hw, 0), pu1 = min(ku - o, W - 1);
    const int pv0 = max(kv - o - 2 * hw, 0), pv1 = min(kv - o, H - 1);
    for (int pv = pv0; pv <= pv1; ++pv) {
        for (int pu = pu0; pu <= pu1; ++pu) {
            const int64_t pix = (int64_t)pv * W + pu;
            const float4 rt = __ldg(a.raytab + pix);
            Ray ray;
            ray.dx = rt.x;
            ray.dy = rt.y;
            ray.dz = rt.z;
            ray.c = rt.w;
            float t;
            if (!accept_point(a, ray, p, a.cam.t_near, a.cam.t_far, t)) continue;
            const uint32_t pos = atomicAdd(a.pm_cnt + pix, 1u);
            // the first append past the slots lists the pixel (once)
            if (pos == (uint32_t)kPmCap) a.ovf[atomicAdd(a.ovf_count, 1u)] = pix;
            if (pos < (uint32_t)kPmCap) {
                a.pm_t[pix * kPmCap + pos] = t;
                a.pm_i[pix * kPmCap + pos] = (uint32_t)i;
            }
        }
    }
}

// Keep the cand_cap smallest (t, id) of the accepted points: lanes whose
// point passed append it at a ballot prefix; once the buffer is full each
// further point replaces the current largest key if it is smaller.
__device__ __forceinline__ void append_candidates(bool acc, uint64_t key, float4 p, int lane, unsigned lt_mask,
                                                  int cap, uint64_t *ck, float4 *cp, int &kept, int &total)
{
    const unsigned m = __ballot_sync(kFull, acc);
    if (m == 0) return;
    const int n = __popc(m);
    if (kept + n <= cap) {
        if (acc) {
            const int pos = kept + __popc(m & lt_mask);
            ck[pos] = key;
            cp[pos] = p;
        }
        kept += n;
    } else {
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
            if (kept < cap) {
                if (lane == 0) {
                    ck[kept] = kk;
                    cp[kept] = pp;
                }
                ++kept;
            } else {
                uint64_t best = 0;
                int bi = -1;
                for (int e = lane; e < cap; e += 32) {
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

// Insert x into the ascending register array keys (the largest falls off);
// n counts the keys held (at most KB).  While fewer than 8 (or 16) are held
// the slots above are empty, so the insertion runs over the first 8 (or 16)
// only -- most neighbourhoods hold a few points.
template <int KB>
__device__ __forceinline__ void knn_insert_n(uint64_t (&keys)[KB], uint64_t x, int &n)
{
    auto ins = [&](auto width) {
        constexpr int kW = decltype(width)::value;
#pragma unroll
        for (int m = 0; m < kW; ++m) {
            const uint64_t k = keys[m];
            const bool lt = x < k;
            keys[m] = lt ? x : k;
            x = lt ? k : x;
        }
    };
    if (KB > 8 && n < 8)
        ins(std::integral_constant<int, (KB > 8 ? 8 : KB)>{});
    else if (KB > 16 && n < 16)
        ins(std::integral_constant<int, (KB > 16 ? 16 : KB)>{});
    else
        ins(std::integral_constant<int, KB>{});
    n += n < KB ? 1 : 0;
}

}  // namespace

// Per-pixel ray table: direction and cone coefficient of every pixel's ray
// (the decision contract's D3/D4 arithmetic).  Rays live in camera space, so
// the table depends only on the intrinsics and the radius mode and is reused
// by every frame whose intrinsics are unchanged.
__global__ void __launch_bounds__(256) k_ray_table(Cam cam, int mode, float rdd, float4 *__restrict__ tab)
{
    grid_dep_wait();
    grid_dep_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)cam.width * cam.height) return;
    const int pu = (int)(i % cam.width), pv = (int)(i / cam.width);
    const Ray r = make_ray(cam, mode, rdd, pu, pv);
    tab[i] = make_float4(r.dx, r.dy, r.dz, r.c);
}

// One ray on one warp (the warp-per-ray search); cp / ck: the warp's
// candidate buffers (kCandCap entries each).
template <int KB>
__device__ __forceinline__ void wide_ray(const SearchArgs &a, const float2 *interval, int64_t ri, float4 *cp,
                                         uint64_t *ck)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int K = a.K, n_max = a.n_max;
    const int64_t npix = (int64_t)a.cam.width * a.cam.height;
    const int pix = a.rays ? __ldg(a.rays + ri) : (int)ri;
    if (pix < 0 || pix >= npix) {
        if (lane == 0) {
            set_error(a.err, HP_ERR_BAD_RAY, ri);
            a.n_s[ri] = 0;
            a.primary[ri] = -1;
            a.cand_count[ri] = 0;
        }
        return;
    }
    const int pv = pix / a.cam.width, pu = pix - pv * a.cam.width;
    const float4 rt = __ldg(a.raytab + pix);
    Ray ray;
    ray.dx = rt.x;
    ray.dy = rt.y;
    ray.dz = rt.z;
    ray.c = rt.w;

    // depth range and window half-width of this ray: the plain search uses
    // [t_near, t_far] and h; the proposal-restricted search the ray's
    // interval and the (smaller) window bound that follows from its t0
    float tn = a.cam.t_near, tf = a.cam.t_far;
    const int hw = plain_window(a);           // the plain search's window
    int hr = hw;
    if (interval) {
        const float2 iv = __ldg(interval + ri);
        tn = fmaxf(tn, iv.x);
        tf = fminf(tf, iv.y);
        if (a.mode == HP_RADIUS_FIXED) {
            // window bound for t >= tn (contract step D12, written out with
            // single roundings so the CPU reference walks the same window)
            const float zlo = fmaxf(dsub(dmul(tn, a.cos_max), dmul(a.r, a.sin_max)), a.cam.z_near);
            const float lim = dadd(dmul(ddiv(a.win_fx, zlo), 1.001f), 1e-3f);
            if (lim < (float)a.h) hr = min(hr, (int)floorf(dadd(lim, 0.5f)));
        }
    }
    const int span = 2 * hr + 1, off = a.h - hr;
    // restricted search: does the full window hold any point at all?  If
    // not, the ray is empty for the plain search too and needs no fallback
    bool full_window_empty = false;
    if (interval) {
        const int fspan = 2 * a.h + 1;
        int flen = 0;
        for (int q = lane; q < fspan; q += 32) {
            const int64_t kb = (int64_t)(pv + q) * a.Wp + pu;
            flen += (int)(__ldg(a.start + kb + fspan) - __ldg(a.start + kb));
        }
        full_window_empty = __ballot_sync(kFull, flen != 0) == 0;
    }

    // whole frames, plain search: the point-major pass left the ray's
    // accepted points in its slots; the walk is needed only when they
    // overflowed the slots or exceed the candidate cap
    int kept = 0, total = 0;
    bool early_hit = false, late_hit = false;
    uint32_t n_slot = 0;
    bool from_slots = false;
    if (a.pm_cnt && !interval) {
        n_slot = __ldg(a.pm_cnt + pix);
        from_slots = n_slot <= (uint32_t)kPmCap && (int)n_slot <= a.cand_cap;
    }

    // ---- window walk.  The s rows' runs are concatenated into one index
    // space (lane q holds row q's [lo, lo+len) and its exclusive offset),
    // so every load instruction serves 32 points whatever the row lengths;
    // visit(p, v < tot) runs for every 32 points, all lanes together.
    auto walk = [&](auto &&visit) {
        for (int r0 = 0; r0 < span; r0 += 32) {
            const int nrows = min(32, span - r0);
            uint32_t lo = 0;
            int len = 0;
            if (lane < nrows) {
                const int64_t kb = (int64_t)(pv + off + r0 + lane) * a.Wp + pu + off;
                lo = __ldg(a.start + kb);
                len = (int)(__ldg(a.start + kb + span) - lo);
            }
            const int incl = warp_incl_scan(len);
            const int tot = __shfl_sync(kFull, incl, 31);
            const int excl = incl - len;
            // point v of the concatenated runs (v < tot); the load for the next
            // 32 points is issued before the current ones are tested
            auto fetch = [&](int v) {
                // row of v: the last row whose exclusive offset is <= v (binary search)
                int row = 0;
                for (int step = 16; step > 0; step >>= 1) {
                    const int cand = row + step;
                    const int ec = __shfl_sync(kFull, excl, cand < nrows ? cand : 31);
                    if (cand < nrows && v >= ec) row = cand;
                }
                const uint32_t rlo = __shfl_sync(kFull, lo, row);
                const int rex = __shfl_sync(kFull, excl, row);
                return v < tot ? __ldg(a.spts + rlo + (uint32_t)(v - rex)) : make_float4(0.f, 0.f, 0.f, 0.f);
            };
            float4 pn = tot > 0 ? fetch(lane) : make_float4(0.f, 0.f, 0.f, 0.f);
            for (int v0 = 0; v0 < tot; v0 += 32) {
                const float4 p = pn;
                if (v0 + 32 < tot) pn = fetch(v0 + 32 + lane);
                visit(p, v0 + lane < tot);
            }
        }
    };
    // Plain search, pruned (the lane kernel's argument): a first walk finds
    // the prune_m-th smallest accepted depth (each lane its own smallest,
    // then prune_m warp minima) and counts the accepted points; the second
    // appends only the reachable prefix of the (t, id) order, so the
    // candidate buffer never has to replace entries.
    float thr = __int_as_float(0x7f800000);
    int walk_total = -1;
    if (!from_slots && !interval && a.prune_m > 0) {
        float tm[kPruneMax];
#pragma unroll
        for (int q = 0; q < kPruneMax; ++q) tm[q] = thr;
        int n_acc = 0;
        walk([&](const float4 &p, bool in) {
            float t = 0.0f;
            if (in && accept_point(a, ray, p, tn, tf, t)) {
                ++n_acc;
                float x = t;
#pragma unroll
                for (int q = 0; q < kPruneMax; ++q) {
                    const float lo2 = fminf(tm[q], x);
                    x = fmaxf(tm[q], x);
                    tm[q] = lo2;
                }
            }
        });
        for (int o = 16; o > 0; o >>= 1) n_acc += __shfl_xor_sync(kFull, n_acc, o);
        if (n_acc > a.prune_m) {
            // the prune_m-th smallest over the warp: repeated warp minima of
            // the lanes' smallest unused depths (ties taken one lane at a time)
            int head = 0;
            float tl = thr;
            for (int r = 0; r < a.prune_m; ++r) {
                float mine = thr;
#pragma unroll
                for (int q = 0; q < kPruneMax; ++q)
                    if (q == head) mine = tm[q];
                float m = mine;
                for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(kFull, m, o));
                const unsigned who = __ballot_sync(kFull, mine == m);
                if (lane == __ffs(who) - 1) ++head;
                tl = m;
            }
            const float rl = radius_at(a.mode, a.r, ray, tl);
            thr = tl + (rl * 1.001f + 1e-5f * (1.0f + tl)) * 1.01f;
        }
        walk_total = n_acc;
    }
    if (!from_slots) {
        walk([&](const float4 &p, bool in) {
            bool acc = false;
            float t = 0.0f;
            if (in) {
                if (!interval) {
                    acc = accept_point(a, ray, p, tn, tf, t) && t <= thr;
                } else {
                    // restricted: points the plain search would accept outside
                    // [t0, t1] flag a possible miss (a surface in front, or
                    // the cluster running on behind t1)
                    const bool plain = accept_point(a, ray, p, a.cam.t_near, a.cam.t_far, t);
                    acc = plain && t >= tn && t <= tf;
                    if (plain && t < tn) early_hit = true;
                    if (plain && t > tf) late_hit = true;
                }
            }
            const uint64_t key = ((uint64_t)__float_as_uint(t) << 32) | (uint32_t)__float_as_int(p.w);
            append_candidates(acc, key, p, lane, lt_mask, a.cand_cap, ck, cp, kept, total);
        });
        if (walk_total >= 0) total = walk_total;   // the count is of every accepted point
    }
    __syncwarp();

    // ---- adaptive primary surface sampling, candidates taken lazily in
    // (t, id) order.  Lane l holds candidates l, l+32, l+64, l+96 in
    // registers; the next candidate is a warp minimum of the keys above the
    // last one, and candidate j's K nearest (d2, id) keys come out of its
    // neighbourhood (candidates within lim in depth) by K warp minima, in
    // ascending order -- so only the candidates the selection reaches are
    // ever ordered.
    static_assert(kCandCap <= 128 && kPmCap <= 128, "4 candidates per lane");
    const int C = from_slots ? (int)n_slot : kept;
    uint64_t ckey[4];
    float4 cpos[4];
    if (from_slots) {
        // depths and table indices from the slots, the positions from the table
        const float *st = a.pm_t + (int64_t)pix * kPmCap;
        const uint32_t *si = a.pm_i + (int64_t)pix * kPmCap;
        float et[4];
        uint32_t ei[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int e = lane + 32 * m;
            et[m] = e < C ? __ldg(st + e) : 0.0f;
            ei[m] = e < C ? __ldg(si + e) : 0u;
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int e = lane + 32 * m;
            cpos[m] = e < C && hp_check(ei[m] < (uint64_t)a.n_points, a.err, ei[m]) ? __ldg(a.spts + ei[m])
                                                                                     : make_float4(0.f, 0.f, 0.f, 0.f);
            ckey[m] = e < C ? ((uint64_t)__float_as_uint(et[m]) << 32) | (uint32_t)__float_as_int(cpos[m].w) : ~0ull;
        }
        total = C;
    } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int e = lane + 32 * m;
            ckey[m] = e < C ? ck[e] : ~0ull;
            cpos[m] = e < C ? cp[e] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    __syncwarp();                              // the buffers are scratch from here on
    float T = 1.0f, t_prev = 0.0f, t_sel = 0.0f;
    int jstar = -1, ns = 0, prim = -1;
    // slot m of ray ri at m R + ri: sample-major planes, so the rays of a
    // tile write (and the pack reads) their first samples side by side
    auto slot_at = [&](int m) { return (int64_t)m * a.R + ri; };
    bool done = false;
    early_hit = __any_sync(kFull, early_hit);
    late_hit = __any_sync(kFull, late_hit);
    uint64_t prev = 0;
    for (int j = 0; j < C; ++j) {
        uint64_t lm = ~0ull;
#pragma unroll
        for (int m = 0; m < 4; ++m)
            if (ckey[m] != ~0ull && (j == 0 || ckey[m] > prev) && ckey[m] < lm) lm = ckey[m];
        const uint64_t mk = warp_min_u64(lm);
        prev = mk;
        const float tj = __uint_as_float((uint32_t)(mk >> 32));
        const int idj = (int)(uint32_t)mk;
        if (jstar >= 0 && a.gap_k > 0.0f) {
            const float gap = dsub(tj, t_prev);
            if (!(gap <= dmul(a.gap_k, radius_at(a.mode, a.r, ray, t_prev)))) {
                done = true;
                break;
            }
        }
        const float rad = radius_at(a.mode, a.r, ray, tj);
        const float rad2 = dmul(rad, rad);
        // |x_j - P_i| >= |t_j - t_i| up to float32 rounding (~1e-6 (1 + t)),
        // far inside the margin, so only candidates within lim in depth qualify
        const float lim = rad * 1.001f + 1e-5f * (1.0f + tj);
        uint64_t nk[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            nk[m] = ~0ull;
            if (ckey[m] != ~0ull && !(fabsf(__uint_as_float((uint32_t)(ckey[m] >> 32)) - tj) > lim)) {
                const float4 Pi = cpos[m];
                const float ax = dfma(tj, ray.dx, -Pi.x);
                const float ay = dfma(tj, ray.dy, -Pi.y);
                const float az = dfma(tj, ray.dz, -Pi.z);
                const float d2 = dadd(dadd(dmul(ax, ax), dmul(ay, ay)), dmul(az, az));
                if (d2 <= rad2) nk[m] = ((uint64_t)__float_as_uint(d2) << 32) | (uint32_t)ckey[m];
            }
        }
        // the K nearest, ascending: the neighbourhood's keys are compacted
        // into shared memory (the candidate buffers are free once in
        // registers), each ranked against all of them, the first K placed by
        // rank; lane k keeps the k-th
        uint64_t *nb_keys = ck;                                   // up to kCandCap
        uint64_t *nb_sorted = reinterpret_cast<uint64_t *>(cp);   // the first K by rank
        int n_nb = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const unsigned bm = __ballot_sync(kFull, nk[m] != ~0ull);
            if (nk[m] != ~0ull) nb_keys[n_nb + __popc(bm & lt_mask)] = nk[m];
            n_nb += __popc(bm);
        }
        __syncwarp();
        for (int i = lane; i < n_nb; i += 32) {
            const uint64_t x = nb_keys[i];
            int rank = 0;
            for (int jn = 0; jn < n_nb; ++jn) rank += nb_keys[jn] < x ? 1 : 0;
            if (rank < K) nb_sorted[rank] = x;
        }
        __syncwarp();
        const int kp = n_nb < K ? n_nb : K;
        const uint64_t mine = lane < kp ? nb_sorted[lane] : ~0ull;
        float s = 0.0f;
        for (int k = 0; k < kp; ++k) s = dadd(s, dsqrt(__uint_as_float((uint32_t)(nb_sorted[k] >> 32))));
        __syncwarp();                                             // buffers reused next candidate
        const float dj = ddiv(s, (float)kp);
        const float alpha = dmul(a.gamma, exp32(-ddiv(dmul(dj, dj), a.beta2)));
        const float w = dmul(alpha, T);
        T = dmul(T, dsub(1.0f, alpha));
        if (w > a.eps_w) {
            if (jstar < 0) {
                jstar = j;
                // the candidate's position, from the lane that holds it
                int src = -1, sm = 0;
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    if (ckey[m] == mk) {
                        src = lane;
                        sm = m;
                    }
                const unsigned hold = __ballot_sync(kFull, src >= 0);
                const int sl = __ffs(hold) - 1;
                float4 pj = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    if (m == sm) pj = cpos[m];
                pj.x = __shfl_sync(kFull, pj.x, sl);
                pj.y = __shfl_sync(kFull, pj.y, sl);
                pj.z = __shfl_sync(kFull, pj.z, sl);
                prim = (int)pixel_key(a.cam, a.h, make_float3(pj.x, pj.y, pj.z));
            }
            const int64_t slot = slot_at(ns);
            if (lane == 0) {
                a.slot_rec[slot].x = tj;
                a.slot_rec[slot].y = __int_as_float(idj);
                if (ns > 0) a.slot_rec[slot_at(ns - 1)].z = tj - t_sel;
            }
            t_sel = tj;
            if (lane < K) {
                const bool ok = mine != ~0ull;
                a.slot_nbr[slot * K + lane] = ok ? (int)(uint32_t)mine : -1;
                a.slot_dist[slot * K + lane] = ok ? dsqrt(__uint_as_float((uint32_t)(mine >> 32))) : 0.0f;
            }
            if (++ns == n_max) {
                done = true;
                break;
            }
        }
        t_prev = tj;
        // w_k <= gamma T_k <= gamma T for every later k: nothing more can pass
        if (!(dmul(a.gamma, T) > a.eps_w)) {
            done = true;
            break;
        }
    }
    // the largest kept candidate depth (for the fallback rule)
    uint64_t lmax = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m)
        if (ckey[m] != ~0ull && ckey[m] > lmax) lmax = ckey[m];
    const uint64_t kmax = warp_max_u64(lmax);
    if (lane == 0 && ns > 0) a.slot_rec[slot_at(ns - 1)].z = 2.0f * radius_at(a.mode, a.r, ray, t_sel);
    if (lane == 0) {
        a.n_s[ri] = ns;
        a.primary[ri] = prim;
        a.cand_count[ri] = total;
        // fall back to the plain search when the restricted one is empty
        // (unless the whole window is), when the plain search accepts a
        // point in front of t0, or when the selection ran out of
        // candidates while the plain search has more behind t1
        // a point behind t1 cannot change the result when a sample was kept
        // and the last restricted candidate lies more than max(gap_k, 1) r
        // before t1: the gap rule stops the plain selection before it
        bool late_ok = false;
        if (interval && jstar >= 0 && a.gap_k > 0.0f && C > 0) {
            const float tl = __uint_as_float((uint32_t)(kmax >> 32));
            late_ok = dsub(tf, tl) > dmul(fmaxf(a.gap_k, 1.0f), radius_at(a.mode, a.r, ray, tl));
        }
        // nothing the plain test accepts in the plain search's own window:
        // the plain search would come back empty as well, so an empty result
        // needs no second search
        const bool plain_empty = total == 0 && !early_hit && !late_hit && hr == hw;
        const bool miss = (ns == 0 && !full_window_empty && !plain_empty) || early_hit || (!done && late_hit && !late_ok);
        if (interval && a.fallback && miss) a.fallback[atomicAdd(a.fallback_count, 1u)] = (int32_t)ri;
    }
    __syncwarp();
}

template <int KB>
__global__ void __launch_bounds__(kSearchWarps * 32) k_search_select_wide(const SearchArgs a)
{
    grid_dep_wait();
    grid_dep_trigger();
    extern __shared__ __align__(16) unsigned char smem[];
    const SearchSmem L = search_layout();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float4 *cp = reinterpret_cast<float4 *>(smem + L.cp) + warp * kCandCap;
    uint64_t *ck = reinterpret_cast<uint64_t *>(smem + L.ck) + warp * kCandCap;
    // a long fallback list went to the lane kernel: its wide rays come here
    const bool to_lanes = a.list_split && a.count_ptr && *a.count_ptr > a.list_split;
    const int32_t *map = to_lanes ? a.wide : a.ray_map;
    const uint32_t *cnt = to_lanes ? a.wide_count : a.count_ptr;
    const int64_t R_eff = cnt ? (int64_t)*cnt : a.R;

    // every warp pulls the next listed ray from a grid-wide counter, so heavy
    // rays never hold up a block; blocks past the list's end leave at once
    if ((int64_t)blockIdx.x * kSearchWarps >= R_eff) return;
    for (;;) {
        unsigned long long rl = 0;
        if (lane == 0) rl = atomicAdd(a.pull, 1ull);
        rl = __shfl_sync(kFull, rl, 0);
        if ((int64_t)rl >= R_eff) break;
        // ri: the ray's index in the outputs (listed passes: from the list)
        const int64_t ri = map ? (int64_t)__ldg(map + (int64_t)rl) : (int64_t)rl;
        wide_ray<KB>(a, a.interval, ri, cp, ck);
    }
}

// Lane-per-ray search.  A lane appends its accepted points, unsorted, to
// its own column of a [cap][32] shared-memory array (a few instructions
// per point, so lanes that accept at different times cost the warp little),
// then takes its candidates in (t, id) order, finding each next one with a
// scan of the column -- the selection usually stops after a few.  A ray whose
// window holds more than kLaneWalkMax points, or with more accepted points
// than the column holds, is listed for the warp-per-ray search instead
// (before walking, or as soon as the column overflows).
constexpr int kLaneWarps = 4;
// most points a lane walks for one ray; windows holding more go to the
// warp-per-ray search
constexpr uint32_t kLaneWalkMax = 384;

// The point-major selection (kMode 3) and the restricted walk (kMode 1) run
// with shorter columns, two position loads in flight instead of four and
// more blocks per SM (no register spills at those bounds); the plain and
// learned walks keep the longer column.
__host__ __device__ constexpr bool lane_short(int kMode) { return kMode == 3 || kMode == 1; }

// column entries per lane
__host__ __device__ constexpr int lane_cap(int kMode) { return lane_short(kMode) ? kLaneCapShort : kLaneCap; }

// resident blocks per SM for each K bucket and mode (K <= 8: 5 with the
// short columns -- 40 KB of shared memory and at most 102 registers a
// block -- else 4 (48 KB); K <= 16: 4 with the short columns, else 3; K >
// 16: 3, for the registers of the larger neighbour arrays)
__host__ __device__ constexpr int lane_blocks_per_sm(int KB, int kMode)
{
    return KB <= 8 ? (lane_short(kMode) ? 5 : 4) : (KB <= 16 && lane_short(kMode) ? 4 : 3);
}

__host__ __device__ constexpr size_t lane_smem_bytes(int kMode)
{
    return (size_t)kLaneWarps * lane_cap(kMode) * 32 * 8;
}

// One ray on one lane; lt / li point at this lane's column (depth lt[c * 32],
// table index li[c * 32]).  Returns false when the ray must go to the
// warp-per-ray search.
// kMode: 0 plain search, 1 restricted to given intervals, 2 restricted to
// intervals the proposal network infers here.
template <int KB, int kMode>
__device__ __forceinline__ bool lane_ray(const SearchArgs &a, int64_t ri, int pix, float *lt, uint32_t *li,
                                         const float *prop_w)
{
    const int W = a.cam.width;
    const int pv = pix / W, pu = pix - pv * W;
    const float4 rt = __ldg(a.raytab + pix);
    Ray ray;
    ray.dx = rt.x;
    ray.dy = rt.y;
    ray.dz = rt.z;
    ray.c = rt.w;

    // depth range and window of this ray (plain: [t_near, t_far] and h;
    // restricted: the ray's interval -- given, or inferred here by the
    // proposal network -- and the window bound of its t0, D12)
    constexpr bool kLearned = kMode == 2;
    constexpr bool restricted = kMode == 1 || kMode == 2;
    constexpr bool kPointMajor = kMode == 3;   // candidates from the point-major pass
    constexpr int kCap = lane_cap(kMode);      // column entries
    float tn = a.cam.t_near, tf = a.cam.t_far;
    float2 iv = make_float2(tn, tf);
    const int hw = plain_window(a);           // the plain search's window
    int hr = hw;
    bool full_window_empty = false;
    if constexpr (restricted) {
        if constexpr (kLearned) {
            float x[prop::kIn];
            prop::histogram(a.cam, a.start, a.spts, a.h, a.Wp, a.cam.height + 2 * a.h, pu, pv, x);
            iv = prop::interval(prop_w, x, a.cam);
        } else {
            iv = __ldg(a.interval + ri);
        }
        tn = fmaxf(tn, iv.x);
        tf = fminf(tf, iv.y);
        if (a.mode == HP_RADIUS_FIXED) {
            const float zlo = fmaxf(dsub(dmul(tn, a.cos_max), dmul(a.r, a.sin_max)), a.cam.z_near);
            const float lim = dadd(dmul(ddiv(a.win_fx, zlo), 1.001f), 1e-3f);
            if (lim < (float)a.h) hr = min(hr, (int)floorf(dadd(lim, 0.5f)));
        }
        const int fspan = 2 * a.h + 1;
        uint32_t flen = 0;
        for (int q = 0; q < fspan; ++q) {
            const int64_t kb = (int64_t)(pv + q) * a.Wp + pu;
            flen |= __ldg(a.start + kb + fspan) - __ldg(a.start + kb);
        }
        full_window_empty = flen == 0;
    }
    const int span = 2 * hr + 1, off = a.h - hr;
    const int64_t kb0 = (int64_t)(pv + off) * a.Wp + pu + off;

    // ---- window walk: s runs, the next row's bounds loaded one row ahead,
    // kPtBatch points of a run loaded before any of them is used
    constexpr int kPtBatch = 8;
    int total = 0;
    float t_max = 0.0f;
    bool early_hit = false, late_hit = false;
    // the smallest appended depth and its entry (candidate 0 unless another
    // entry has the same depth: then the ids decide, by a scan below)
    float t_lo = __int_as_float(0x7f800000);
    int c_lo = 0;                              // its column entry
    bool lo_tie = false;
    int n_col = 0;                             // entries in the column (the walk: every accepted point)
    if constexpr (kPointMajor) {
        // the pass left this ray's accepted points (any order) in its slots;
        // slots that overflowed hold an arbitrary subset: the warp search walks
        const uint32_t cnt = __ldg(a.pm_cnt + pix);
        if (cnt > (uint32_t)kPmCap) return true;   // searched already, from the overflow list
        // Candidates the selection can reach: it processes at most prune_m
        // candidates (every one multiplies T by at most 1 - alpha_min, and it
        // stops once gamma T <= eps_w), and a processed candidate's
        // neighbourhood lies within lim of its depth; so only the depths up
        // to the prune_m-th smallest plus that candidate's lim matter, a
        // prefix of the (t, id) order.  The column keeps that prefix.
        auto threshold = [&](float tl) {
            const float rl = radius_at(a.mode, a.r, ray, tl);
            return tl + (rl * 1.001f + 1e-5f * (1.0f + tl)) * 1.01f;
        };
        auto top_m = [&](float (&tm)[kPruneMax], float x) {
#pragma unroll
            for (int q = 0; q < kPruneMax; ++q) {
                const float lo = fminf(tm[q], x);
                x = fmaxf(tm[q], x);
                tm[q] = lo;
            }
        };
        auto mth = [&](const float (&tm)[kPruneMax]) {
            float tl = tm[0];
#pragma unroll
            for (int q = 1; q < kPruneMax; ++q)
                if (q < a.prune_m) tl = tm[q];
            return tl;
        };
        const bool prune = a.prune_m > 0 && cnt > (uint32_t)a.prune_m;
        float thr = __int_as_float(0x7f800000);
        auto keep = [&](float t, uint32_t ix) {
            lt[n_col * 32] = t;
            li[n_col * 32] = ix;
            t_max = fmaxf(t_max, t);
            lo_tie = t == t_lo ? true : (t < t_lo ? false : lo_tie);
            if (t < t_lo) {
                t_lo = t;
                c_lo = n_col;
            }
            ++n_col;
        };
        // the depths first (16-byte loads of four, kSlotBatch in flight; a
        // ray's slots are 16-byte aligned), the table indices of the kept
        // candidates after: most candidates lie beyond the reachable prefix
        const float4 *st = reinterpret_cast<const float4 *>(a.pm_t + (int64_t)pix * kPmCap);
        const uint32_t *si = a.pm_i + (int64_t)pix * kPmCap;
        constexpr int kSlotBatch = 3;
        const bool in_col = cnt <= (uint32_t)kCap;   // the depths fit the column
        {
            float tm[kPruneMax];
#pragma unroll
            for (int q = 0; q < kPruneMax; ++q) tm[q] = thr;
            for (uint32_t c0 = 0; c0 < cnt; c0 += 4 * kSlotBatch) {
                float4 e[kSlotBatch];
#pragma unroll
                for (int k = 0; k < kSlotBatch; ++k)
                    if (c0 + 4 * k < cnt) e[k] = __ldg(st + (c0 >> 2) + k);
#pragma unroll
                for (int k = 0; k < 4 * kSlotBatch; ++k) {
                    const uint32_t c = c0 + k;
                    if (c >= cnt) break;
                    const float4 q4 = e[k >> 2];
                    const float t = (k & 3) == 0 ? q4.x : (k & 3) == 1 ? q4.y : (k & 3) == 2 ? q4.z : q4.w;
                    if (in_col) lt[c * 32] = t;
                    if (prune) top_m(tm, t);
                }
            }
            if (prune) thr = threshold(mth(tm));
        }
        // the reachable prefix into the column, each entry's slot number in
        // place of its table index for now
        if (in_col) {
            for (uint32_t c = 0; c < cnt; ++c) {
                const float t = lt[c * 32];
                if (!(t <= thr)) continue;
                keep(t, c);                          // n_col <= c: in place
            }
        } else {
            // more than a column holds: the depths again from global memory
            for (uint32_t c0 = 0; c0 < cnt; c0 += 4 * kSlotBatch) {
                float4 e[kSlotBatch];
#pragma unroll
                for (int k = 0; k < kSlotBatch; ++k)
                    if (c0 + 4 * k < cnt) e[k] = __ldg(st + (c0 >> 2) + k);
#pragma unroll
                for (int k = 0; k < 4 * kSlotBatch; ++k) {
                    const uint32_t c = c0 + k;
                    if (c >= cnt) break;
                    const float4 q4 = e[k >> 2];
                    const float t = (k & 3) == 0 ? q4.x : (k & 3) == 1 ? q4.y : (k & 3) == 2 ? q4.z : q4.w;
                    if (!(t <= thr)) continue;
                    if (n_col == kCap) return false;   // more than the column holds
                    keep(t, c);
                }
            }
        }
        // the kept entries' table indices, their loads in flight together
        for (int c0 = 0; c0 < n_col; c0 += kSlotBatch) {
            uint32_t ix[kSlotBatch];
#pragma unroll
            for (int k = 0; k < kSlotBatch; ++k)
                if (c0 + k < n_col) ix[k] = __ldg(si + li[(c0 + k) * 32]);
#pragma unroll
            for (int k = 0; k < kSlotBatch; ++k)
                if (c0 + k < n_col) li[(c0 + k) * 32] = ix[k];
        }
        total = (int)cnt;
    } else {
        // a window holding many points (rays along a surface near a silhouette)
        // would keep one lane walking while the rest of its warp idles: the
        // warp-per-ray search, which walks 32 points at a time, takes the ray
        {
            uint32_t n_win = 0;
            for (int q = 0; q < span; ++q) {
                const int64_t kb = kb0 + (int64_t)q * a.Wp;
                n_win += __ldg(a.start + kb + span) - __ldg(a.start + kb);
            }
            if (n_win > kLaneWalkMax) {
                if (kLearned) a.interval_buf[ri] = iv;
                return false;
            }
        }

        uint32_t nlo = __ldg(a.start + kb0), nhi = __ldg(a.start + kb0 + span);
        for (int q = 0; q < span; ++q) {
            const uint32_t lo = nlo, hi = nhi;
            if (q + 1 < span) {
                const int64_t kb = kb0 + (int64_t)(q + 1) * a.Wp;
                nlo = __ldg(a.start + kb);
                nhi = __ldg(a.start + kb + span);
            }
            for (uint32_t i0 = lo; i0 < hi; i0 += kPtBatch) {
                float4 pb[kPtBatch];
#pragma unroll
                for (int k = 0; k < kPtBatch; ++k)
                    if (i0 + k < hi) pb[k] = __ldg(a.spts + i0 + k);
#pragma unroll
                for (int k = 0; k < kPtBatch; ++k) {
                    if (i0 + k >= hi) break;
                    float t = 0.0f;
                    bool acc;
                    if constexpr (!restricted) {
                        acc = accept_point(a, ray, pb[k], tn, tf, t);
                    } else {
                        const bool plain = accept_point(a, ray, pb[k], a.cam.t_near, a.cam.t_far, t);
                        acc = plain && t >= tn && t <= tf;
                        early_hit |= plain && t < tn;
                        late_hit |= plain && t > tf;
                    }
                    if (!acc) continue;
                    // more accepted points than the column holds: the warp-per-ray
                    // search takes the ray, so stop walking
                    if (total == kCap) {
                        if (kLearned) a.interval_buf[ri] = iv;
                        return false;
                    }
                    lt[total * 32] = t;
                    li[total * 32] = i0 + k;
                    t_max = fmaxf(t_max, t);
                    lo_tie = t == t_lo ? true : (t < t_lo ? false : lo_tie);
                    if (t < t_lo) {
                        t_lo = t;
                        c_lo = total;
                    }
                    ++total;
                }
            }
        }
    }
    if constexpr (!kPointMajor) n_col = total;
    // the cap rule is the warp search's (a pruned column is a prefix of the
    // (t, id) order: within the cap when it fits)
    if (n_col > a.cand_cap) {
        if (kLearned) a.interval_buf[ri] = iv;
        return false;
    }
    const int C = n_col;
    // the position (and id) of column entry c
    auto pos_of = [&](int c) -> float4 {
        const uint32_t ix = li[c * 32];
        return hp_check(ix < (uint64_t)a.n_points, a.err, ix) ? __ldg(a.spts + ix) : make_float4(0.f, 0.f, 0.f, 0.f);
    };

    // ---- adaptive primary surface sampling, candidates in (t, id) order.
    // Each pass over the column forms candidate j's neighbourhood and, in the
    // same loop, finds candidate j+1: the smallest (t, id) above (t_j, id_j)
    // (ids are looked up only for equal depths).
    const int K = a.K, n_max = a.n_max;
    float T = 1.0f, t_prev = 0.0f, t_sel = 0.0f;
    int id_sel = 0;
    int jstar = -1, ns = 0, prim = -1;
    bool done = false;
    // slot m of ray ri at m R + ri: sample-major planes, so the rays of a
    // tile write (and the pack reads) their first samples side by side
    auto slot_at = [&](int m) { return (int64_t)m * a.R + ri; };
    const float kInf = __int_as_float(0x7f800000);
    // candidate 0: the smallest (t, id)
    float tq = t_lo;
    int cq = c_lo;                             // column entry of the next candidate
    int idq = -2;                              // -2: not looked up yet
    if (lo_tie) tq = kInf;
    for (int c = 0; lo_tie && c < C; ++c) {
        const float tc = lt[c * 32];
        if (tc > tq) continue;
        if (tc == tq) {
            if (idq == -2) idq = __float_as_int(pos_of(cq).w);
            const int idc = __float_as_int(pos_of(c).w);
            if (idc >= idq) continue;
            idq = idc;
        } else {
            idq = -2;
        }
        tq = tc;
        cq = c;
    }
    for (int j = 0; j < C; ++j) {
        const float tj = tq;
        const float4 pj = pos_of(cq);
        const int idj = __float_as_int(pj.w);
        if (jstar >= 0 && a.gap_k > 0.0f) {
            const float gap = dsub(tj, t_prev);
            if (!(gap <= dmul(a.gap_k, radius_at(a.mode, a.r, ray, t_prev)))) {
                done = true;
                break;
            }
        }
        const float rad = radius_at(a.mode, a.r, ray, tj);
        const float rad2 = dmul(rad, rad);
        // |x_j - P_i| >= |t_j - t_i| up to float32 rounding (~1e-6 (1 + t)),
        // far inside the margin, so only candidates within lim in depth qualify
        const float lim = rad * 1.001f + 1e-5f * (1.0f + tj);
        uint64_t keys[KB];
#pragma unroll
        for (int m = 0; m < KB; ++m) keys[m] = ~0ull;
        int n_keys = 0;                        // keys held (the rest are empty)
        tq = kInf;
        idq = -2;
        // kNb column entries at a time: the positions of those within lim in
        // depth are loaded together before any is used (their latencies overlap)
        constexpr int kNb = lane_short(kMode) ? 2 : 4;
        for (int c0 = 0; c0 < C; c0 += kNb) {
            float tcs[kNb];
            float4 P[kNb];
#pragma unroll
            for (int k = 0; k < kNb; ++k) tcs[k] = c0 + k < C ? lt[(c0 + k) * 32] : kInf;
#pragma unroll
            for (int k = 0; k < kNb; ++k)
                if (c0 + k < C && fabsf(tcs[k] - tj) <= lim) P[k] = pos_of(c0 + k);
#pragma unroll
            for (int k = 0; k < kNb; ++k) {
                if (c0 + k >= C) break;
                const float tc = tcs[k];
                // next candidate
                if (tc >= tj && tc <= tq) {
                    bool take = true;
                    int idc = -2;
                    if (tc == tj || tc == tq) {
                        idc = __float_as_int(pos_of(c0 + k).w);
                        if (tc == tj && idc <= idj) take = false;
                        if (take && tc == tq) {
                            if (idq == -2) idq = __float_as_int(pos_of(cq).w);
                            if (idc >= idq) take = false;
                        }
                    }
                    if (take) {
                        tq = tc;
                        cq = c0 + k;
                        idq = idc;
                    }
                }
                // neighbourhood of candidate j
                if (fabsf(tc - tj) > lim) continue;
                const float4 Pi = P[k];
                const float ax = dfma(tj, ray.dx, -Pi.x);
                const float ay = dfma(tj, ray.dy, -Pi.y);
                const float az = dfma(tj, ray.dz, -Pi.z);
                const float d2 = dadd(dadd(dmul(ax, ax), dmul(ay, ay)), dmul(az, az));
                if (d2 <= rad2)
                    knn_insert_n<KB>(keys, ((uint64_t)__float_as_uint(d2) << 32) | (uint32_t)__float_as_int(Pi.w),
                                     n_keys);
            }
        }
        float s = 0.0f, dist[KB];
        int kp = 0;
#pragma unroll
        for (int m = 0; m < KB; ++m) {
            dist[m] = 0.0f;
            if (m < K && m < n_keys) {
                dist[m] = dsqrt(__uint_as_float((uint32_t)(keys[m] >> 32)));
                s = dadd(s, dist[m]);
                ++kp;
            }
        }
        const float dj = ddiv(s, (float)kp);
        const float alpha = dmul(a.gamma, exp32(-ddiv(dmul(dj, dj), a.beta2)));
        const float w = dmul(alpha, T);
        T = dmul(T, dsub(1.0f, alpha));
        if (w > a.eps_w) {
            if (jstar < 0) {
                jstar = j;
                prim = (int)pixel_key(a.cam, a.h, make_float3(pj.x, pj.y, pj.z));
            }
            const int64_t slot = slot_at(ns);
            // a record is written whole once its delta is known (next sample or the end)
            if (ns > 0) a.slot_rec[slot_at(ns - 1)] = make_float4(t_sel, __int_as_float(id_sel), tj - t_sel, 0.0f);
            t_sel = tj;
            id_sel = idj;
            if ((K & 3) == 0) {
                // 16-byte stores (a slot's K entries start 16-byte aligned)
                int4 *sn = reinterpret_cast<int4 *>(a.slot_nbr + slot * K);
                float4 *sd = reinterpret_cast<float4 *>(a.slot_dist + slot * K);
#pragma unroll
                for (int m = 0; m < KB; m += 4) {
                    if (m < K) {
                        int v[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) v[q] = keys[m + q] != ~0ull ? (int)(uint32_t)keys[m + q] : -1;
                        sn[m >> 2] = make_int4(v[0], v[1], v[2], v[3]);
                        sd[m >> 2] = make_float4(dist[m], dist[m + 1], dist[m + 2], dist[m + 3]);
                    }
                }
            } else {
#pragma unroll
                for (int m = 0; m < KB; ++m) {
                    if (m < K) {
                        const bool ok = keys[m] != ~0ull;
                        a.slot_nbr[slot * K + m] = ok ? (int)(uint32_t)keys[m] : -1;
                        a.slot_dist[slot * K + m] = dist[m];
                    }
                }
            }
            if (++ns == n_max) {
                done = true;
                break;
            }
        }
        t_prev = tj;
        if (!(dmul(a.gamma, T) > a.eps_w)) {
            done = true;
            break;
        }
    }
    if (ns > 0)
        a.slot_rec[slot_at(ns - 1)] =
            make_float4(t_sel, __int_as_float(id_sel), 2.0f * radius_at(a.mode, a.r, ray, t_sel), 0.0f);
    a.n_s[ri] = ns;
    a.primary[ri] = prim;
    a.cand_count[ri] = total;
    if (restricted && a.fallback) {
        // fallback rule of the restricted search (D12); the last candidate's
        // depth is the largest accepted depth (total <= cand_cap here)
        bool late_ok = false;
        if (jstar >= 0 && a.gap_k > 0.0f && total > 0)
            late_ok = dsub(tf, t_max) > dmul(fmaxf(a.gap_k, 1.0f), radius_at(a.mode, a.r, ray, t_max));
        // nothing the plain test accepts in the plain search's own window:
        // the plain search would come back empty as well, so an empty result
        // needs no second search
        const bool plain_empty = total == 0 && !early_hit && !late_hit && hr == hw;
        const bool miss = (ns == 0 && !full_window_empty && !plain_empty) || early_hit || (!done && late_hit && !late_ok);
        if (miss) a.fallback[atomicAdd(a.fallback_count, 1u)] = (int32_t)ri;
    }
    return true;
}

// Warps pull work units from a grid-wide counter: an 8 x 4 pixel tile (whole
// frames; ray i is pixel i) or 32 consecutive listed rays.
template <int KB, int kMode>
__global__ void __launch_bounds__(kLaneWarps * 32, lane_blocks_per_sm(KB, kMode)) k_search_select(const SearchArgs a)
{
    grid_dep_wait();
    grid_dep_trigger();
    constexpr bool kLearned = kMode == 2;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // this lane's candidate list: depth lt[c * 32] and table index li[c * 32]
    constexpr int kCap = lane_cap(kMode);
    float *lt = reinterpret_cast<float *>(smem) + warp * (kCap * 32) + lane;
    uint32_t *li = reinterpret_cast<uint32_t *>(smem) + kLaneWarps * kCap * 32 + warp * (kCap * 32) + lane;

    // proposal weights (FP32 copy of the BF16 ones) behind the columns
    float *pw = nullptr;
    if constexpr (kLearned) {
        pw = reinterpret_cast<float *>(smem + lane_smem_bytes(kMode));
        prop::load_weights(a.prop_w, pw);
        __syncthreads();
    }

    const int W = a.cam.width, H = a.cam.height;
    const int64_t npix = (int64_t)W * H;
    const bool frame = !a.rays && !a.ray_map;
    const int tiles_x = (W + 7) >> 3;
    const int64_t n_list = a.count_ptr ? (int64_t)*a.count_ptr : a.R;
    // a short fallback list is the warp-per-ray kernel's (list_split)
    const int64_t n_units = frame ? (int64_t)tiles_x * ((H + 3) >> 2)
                                  : (a.list_split && n_list <= (int64_t)a.list_split ? 0 : (n_list + 31) / 32);
    const int64_t R_eff = frame ? npix : (a.count_ptr ? (int64_t)*a.count_ptr : a.R);
    if constexpr (kMode == 3) {
        // the pixels whose slots overflowed walk their whole window with the
        // warp-per-ray search: the heaviest rays of the frame, so the warps
        // take them before any tile (their latency then overlaps the tiles)
        float4 *cp = reinterpret_cast<float4 *>(reinterpret_cast<float *>(smem) + warp * (kCap * 32));
        uint64_t *ck = reinterpret_cast<uint64_t *>(cp + kCandCap);
        static_assert(kCandCap * (sizeof(float4) + sizeof(uint64_t)) <= kCap * 32 * sizeof(float),
                      "the warp search's lists fit one warp's depth column");
        const uint32_t n_ovf = *a.ovf_count;
        for (;;) {
            uint32_t i = 0;
            if (lane == 0) i = atomicAdd(a.ovf_pull, 1u);
            i = __shfl_sync(kFull, i, 0);
            if (i >= n_ovf) break;
            wide_ray<KB>(a, nullptr, (int64_t)__ldg(a.ovf + i), cp, ck);
        }
        __syncwarp();
    }
    for (;;) {
        unsigned int u = 0;
        if (lane == 0) u = atomicAdd(a.lane_units, 1u);
        u = __shfl_sync(kFull, u, 0);
        if ((int64_t)u >= n_units) break;
        int64_t ri;
        int pix;
        if (frame) {
            const int64_t ty = (int64_t)u / tiles_x;
            const int pu = (int)((int64_t)u - ty * tiles_x) * 8 + (lane & 7);
            const int64_t pv = ty * 4 + (lane >> 3);
            if (pu >= W || pv >= H) continue;
            ri = pv * W + pu;
            pix = (int)ri;
        } else {
            const int64_t rl = (int64_t)u * 32 + lane;
            if (rl >= R_eff) continue;
            ri = a.ray_map ? (int64_t)__ldg(a.ray_map + rl) : rl;
            pix = a.rays ? __ldg(a.rays + ri) : (int)ri;
        }
        if (pix < 0 || pix >= npix) {
            set_error(a.err, HP_ERR_BAD_RAY, ri);
            a.n_s[ri] = 0;
            a.primary[ri] = -1;
            a.cand_count[ri] = 0;
            continue;
        }
        // a window too large for one lane, or more candidates than this lane
        // may answer for: the warp-per-ray search takes the ray
        if (!lane_ray<KB, kMode>(a, ri, pix, lt, li, pw)) a.wide[atomicAdd(a.wide_count, 1u)] = (int32_t)ri;
    }

}

// Packing (K6): exclusive scan of n_s with a decoupled look-back over
// uniform tiles of kPackRays rays; the tile's samples form one contiguous packed
// range, which the whole block copies with coalesced stores (each packed
// sample's slot is looked up in a shared-memory map).  When the caller leaves
// the neighbour lists in the slots (hp_samples.nbr NULL), only the per-sample
// records are copied and each sample's slot index is written instead.
constexpr int kPackRays = 1024;
constexpr int kPackWarps = kPackRays / 32;

__global__ void __launch_bounds__(kPackRays) k_pack_samples(const SearchArgs a)
{
    grid_dep_wait();
    grid_dep_trigger();
    __shared__ int64_t s_tile, s_prefix;
    __shared__ int s_warp[kPackWarps];
    __shared__ int s_total;
    __shared__ uint16_t s_slot[kPackRays * kMaxSamples];   // packed sample -> (ray in tile) << 4 | m
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(a.ticket, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t ri = tile * kPackRays + tid;
    const int ns = ri < a.R ? a.n_s[ri] : 0;
    const int incl = warp_incl_scan(ns);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int w = lane < kPackWarps ? s_warp[lane] : 0;
        const int wi = warp_incl_scan(w);
        if (lane < kPackWarps) s_warp[lane] = wi - w;
        const int tot = __shfl_sync(kFull, wi, kPackWarps - 1);
        const int64_t pre = lookback_prefix_warp(a.flags, tile, tot, a.err, a.spin_limit, true);
        if (lane == 0) {
            s_total = tot;
            s_prefix = pre;
        }
    }
    __syncthreads();
    const int local = s_warp[warp] + (incl - ns);     // this ray's first sample within the tile
    const int64_t base = s_prefix;
    const int64_t off = base + local;
    if (ri < a.R) a.sample_offset[ri] = off;
    if (ri == a.R - 1) {
        a.sample_offset[a.R] = off + ns;
        if (off + ns > a.capacity) set_error(a.err, HP_ERR_OVERFLOW, off + ns);
    }
    for (int m = 0; m < ns; ++m) s_slot[local + m] = (uint16_t)((tid << 4) | m);
    __syncthreads();
    // samples that fit the capacity
    int64_t total = s_total;
    if (base + total > a.capacity) total = a.capacity > base ? a.capacity - base : 0;
    const int64_t ray0 = tile * kPackRays;
    for (int p = tid; p < total; p += kPackRays) {
        const int v = s_slot[p];
        const int64_t r = ray0 + (v >> 4);
        const int64_t sl = (int64_t)(v & 15) * a.R + r;
        const float4 rec = a.slot_rec[sl];
        a.t[base + p] = rec.x;
        a.src[base + p] = __float_as_int(rec.y);
        a.delta[base + p] = rec.z;
        a.ray[base + p] = (int)r;
        if (!a.nbr) a.sample_slot[base + p] = (int32_t)sl;   // the lists stay in the slots
    }
    if (!a.nbr) return;
    // neighbour ids and distances
    const int K = a.K;
    auto slot_of = [&](int64_t p) {
        const int v = s_slot[p];
        return (int64_t)(v & 15) * a.R + ray0 + (v >> 4);
    };
    const bool vec = (K & 3) == 0 && (((uintptr_t)a.nbr | (uintptr_t)a.nbr_dist) & 15) == 0;
    if (vec) {
        // 16-byte chunks: lane (sample sub, chunk e), two samples per lane in
        // flight (the slots are spread over the tile's rays)
        const int q = K >> 2, spi = 32 / q, sub = lane / q, e = lane - sub * q;
        const int4 *sn = reinterpret_cast<const int4 *>(a.slot_nbr);
        const float4 *sd = reinterpret_cast<const float4 *>(a.slot_dist);
        int4 *on = reinterpret_cast<int4 *>(a.nbr);
        float4 *od = reinterpret_cast<float4 *>(a.nbr_dist);
        if (sub < spi) {
            for (int64_t p = (int64_t)warp * spi + sub; p < total; p += 2 * kPackWarps * spi) {
                const int64_t p2 = p + kPackWarps * spi;
                const bool two = p2 < total;
                const int64_t s0 = slot_of(p), s1 = two ? slot_of(p2) : s0;
                const int4 n0 = __ldg(sn + s0 * q + e), n1 = __ldg(sn + s1 * q + e);
                const float4 d0 = __ldg(sd + s0 * q + e), d1 = __ldg(sd + s1 * q + e);
                on[(base + p) * q + e] = n0;
                od[(base + p) * q + e] = d0;
                if (two) {
                    on[(base + p2) * q + e] = n1;
                    od[(base + p2) * q + e] = d1;
                }
            }
        }
    } else {
        // lane (sample sub, element e) per warp step
        const int per = 32 / K, sub = lane / K, e = lane - sub * K;
        if (sub < per) {
            for (int64_t p = (int64_t)warp * per + sub; p < total; p += kPackWarps * per) {
                const int64_t sl = slot_of(p);
                a.nbr[(base + p) * K + e] = a.slot_nbr[sl * K + e];
                a.nbr_dist[(base + p) * K + e] = a.slot_dist[sl * K + e];
            }
        }
    }
}

size_t search_smem_bytes() { return search_layout().total; }

namespace {

// One search pass over the rays `a` describes: the lane-per-ray kernel, then
// the warp-per-ray kernel over the rays the lanes listed as too wide.
// Whole frames, plain search: the point-major pass finds the candidates.
// Listed plain searches of at most this many rays per SM go warp-per-ray.
constexpr int64_t kSmallListPerSm = 64;

bool point_major_pass(const SearchArgs &a)
{
    return !a.prop_w && !a.interval && !a.rays && !a.ray_map && a.pm_t && a.pm_i && a.pm_cnt && a.pcell &&
           a.R == (int64_t)a.cam.width * a.cam.height;
}

cudaError_t search_pass(const SearchArgs &a, cudaStream_t st, Prof *prof, int kid)
{
    cudaError_t e;
    const bool point_major = point_major_pass(a);
    auto lane_k = a.prop_w ? (a.K <= 4 ? k_search_select<4, 2> : a.K <= 8 ? k_search_select<8, 2>
                              : a.K <= 16 ? k_search_select<16, 2> : k_search_select<32, 2>)
                  : a.interval ? (a.K <= 4 ? k_search_select<4, 1> : a.K <= 8 ? k_search_select<8, 1>
                                  : a.K <= 16 ? k_search_select<16, 1> : k_search_select<32, 1>)
                  : point_major ? (a.K <= 4 ? k_search_select<4, 3> : a.K <= 8 ? k_search_select<8, 3>
                                   : a.K <= 16 ? k_search_select<16, 3> : k_search_select<32, 3>)
                               : (a.K <= 4 ? k_search_select<4, 0> : a.K <= 8 ? k_search_select<8, 0>
                                  : a.K <= 16 ? k_search_select<16, 0> : k_search_select<32, 0>);
    auto wide_k = a.K <= 4 ? k_search_select_wide<4> : a.K <= 8 ? k_search_select_wide<8>
                : a.K <= 16 ? k_search_select_wide<16> : k_search_select_wide<32>;
    const int lane_mode = a.prop_w ? 2 : a.interval ? 1 : point_major ? 3 : 0;
    const size_t lsm = lane_smem_bytes(lane_mode) + (a.prop_w ? (size_t)(prop::kImage + 4) * 4 : 0),
                 wsm = search_smem_bytes();
    if ((e = cudaFuncSetAttribute(lane_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(wide_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm)) != cudaSuccess)
        return e;
    // wide_count, pull and lane_units: cleared with the tickets by launch_search
    int64_t units;
    if (!a.rays && !a.ray_map)
        units = div_up((int64_t)a.cam.width, 8) * div_up((int64_t)a.cam.height, 4);
    else
        units = div_up(a.R, 32);
    // persistent warps: as many blocks as stay resident, fewer for small work
    const int KB = a.K <= 4 ? 4 : a.K <= 8 ? 8 : a.K <= 16 ? 16 : 32;
    const int64_t blocks =
        std::min<int64_t>(div_up(units, kLaneWarps), (int64_t)a.n_sm * lane_blocks_per_sm(KB, lane_mode));
    // A short plain list of rays (a training batch) would give the lane
    // kernel a few hundred warps for the whole GPU: one warp per ray instead
    if (!point_major && !a.interval && !a.prop_w && a.rays && a.R <= (int64_t)a.n_sm * kSmallListPerSm) {
        SearchArgs w = a;
        w.pm_cnt = nullptr;                      // no point-major slots: the warps walk
        const int64_t wb = std::min<int64_t>(div_up(a.R, kSearchWarps), (int64_t)a.n_sm * 4);
        prof_begin(prof, st, kid);
        launch_chained(wide_k, (unsigned)wb, kSearchWarps * 32, wsm, st, w);
        prof_end(prof, st);
        return cudaGetLastError();
    }
    // pm_cnt: cleared with the tickets by launch_search
    prof_begin(prof, st, kid);
    const bool splat = point_major && a.n_points > 0;
    if (splat) launch_chained(k_search_splat, (unsigned)div_up(a.n_points, 256), 256, 0, st, a);
    launch_chained(lane_k, (unsigned)blocks, kLaneWarps * 32, lsm, st, a);
    prof_end(prof, st, splat ? 2 : 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    SearchArgs b = a;
    b.ray_map = a.wide;
    b.count_ptr = a.wide_count;
    if (!point_major) b.pm_cnt = nullptr;   // no slots to read the candidates from
    if (a.prop_w) {
        // the lanes left the inferred intervals of the rays they handed over
        b.interval = a.interval_buf;
        b.prop_w = nullptr;
    }
    const int64_t wblocks = std::min<int64_t>(div_up(a.R, kSearchWarps), (int64_t)a.n_sm * 4);
    prof_begin(prof, st, KID_SEARCH_WIDE);
    launch_chained(wide_k, (unsigned)wblocks, kSearchWarps * 32, wsm, st, b);
    prof_end(prof, st);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_search(const SearchArgs &a, cudaStream_t st, Prof *prof)
{
    cudaError_t e;
    if (a.raytab_stale) {
        const int64_t npix = (int64_t)a.cam.width * a.cam.height;
        prof_begin(prof, st, KID_RAY_TABLE);
        launch_chained(k_ray_table, (unsigned)div_up(npix, 256), 256, 0, st, a.cam, a.mode, a.rdd, a.raytab);
        prof_end(prof, st);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int64_t tiles = div_up(a.R, kPackRays);
    // the ticket words (pack ticket, fallback count, wide-ray count, lane
    // units, the 64-bit pull counter: words 0-5) and the pack's look-back
    // words after them: one memset
    const char *z0 = reinterpret_cast<const char *>(a.ticket);
    const char *zf = reinterpret_cast<const char *>(a.flags);
    const char *ze = reinterpret_cast<const char *>(a.flags + tiles);
    if (point_major_pass(a)) {
        // ... and the point-major pass's per-pixel counts, which follow
        if (reinterpret_cast<const char *>(a.pm_cnt) < ze) return cudaErrorInvalidValue;
        ze = reinterpret_cast<const char *>(a.pm_cnt + a.R);
    }
    if (!(zf >= z0 + 6 * sizeof(uint32_t) && reinterpret_cast<const char *>(a.wide_count) < zf &&
          reinterpret_cast<const char *>(a.lane_units) < zf && reinterpret_cast<const char *>(a.pull + 1) <= zf &&
          reinterpret_cast<const char *>(a.wide_count) >= z0 && reinterpret_cast<const char *>(a.lane_units) >= z0 &&
          reinterpret_cast<const char *>(a.pull) >= z0))
        return cudaErrorInvalidValue;
    if ((e = launch_clear(a.ticket, (size_t)(ze - z0), st, prof)) != cudaSuccess) return e;
    if ((e = search_pass(a, st, prof, KID_SEARCH)) != cudaSuccess) return e;
    if ((a.interval || a.prop_w) && a.fallback) {
        // plain search for the rays the restricted search flagged, one warp
        // per ray.  With K > 8 a list of more than kSmallListPerSm rays per
        // SM -- the count is on the device -- goes to the lane-per-ray kernel
        // instead, whose too-wide rays the warp kernel then takes: both
        // kernels launch, and each reads the count to see which part is its
        // own.  Measured: forward_1008 (K 16, 40k missed rays) 0.128 ms by
        // warps, 0.059 by lanes; objects_800 (K 8, a long list) 0.055 ms by
        // warps, 0.074 by lanes
        SearchArgs b = a;
        b.interval = nullptr;
        b.prop_w = nullptr;
        b.ray_map = a.fallback;
        b.count_ptr = a.fallback_count;
        b.raytab_stale = 0;
        b.pm_cnt = nullptr;
        const bool split = a.K > 8;
        b.list_split = split ? (uint32_t)std::min<int64_t>((int64_t)a.n_sm * kSmallListPerSm, 0x7fffffff) : 0u;
        // wide_count, lane_units and the 64-bit pull counter (ticket words 2-5)
        if (reinterpret_cast<const char *>(a.lane_units) != reinterpret_cast<const char *>(a.wide_count) + 4 ||
            reinterpret_cast<const char *>(a.pull) != reinterpret_cast<const char *>(a.wide_count) + 8)
            return cudaErrorInvalidValue;
        if ((e = launch_clear(a.wide_count, 4 * sizeof(uint32_t), st, prof)) != cudaSuccess) return e;
        auto lane0 = a.K <= 4 ? k_search_select<4, 0> : a.K <= 8 ? k_search_select<8, 0>
                   : a.K <= 16 ? k_search_select<16, 0> : k_search_select<32, 0>;
        auto wide_k = a.K <= 4 ? k_search_select_wide<4> : a.K <= 8 ? k_search_select_wide<8>
                    : a.K <= 16 ? k_search_select_wide<16> : k_search_select_wide<32>;
        const int KB = a.K <= 4 ? 4 : a.K <= 8 ? 8 : a.K <= 16 ? 16 : 32;
        const size_t lsm = lane_smem_bytes(0);
        if (split &&
            (e = cudaFuncSetAttribute(lane0, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm)) != cudaSuccess)
            return e;
        const int64_t lblocks =
            std::min<int64_t>(div_up(div_up(a.R, 32), kLaneWarps), (int64_t)a.n_sm * lane_blocks_per_sm(KB, 0));
        const int64_t wblocks = std::min<int64_t>(div_up(a.R, kSearchWarps), (int64_t)a.n_sm * 4);
        prof_begin(prof, st, KID_SEARCH_FALLBACK);
        if (split) launch_chained(lane0, (unsigned)lblocks, kLaneWarps * 32, lsm, st, b);
        launch_chained(wide_k, (unsigned)wblocks, kSearchWarps * 32, search_smem_bytes(), st, b);
        prof_end(prof, st, split ? 2 : 1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    prof_begin(prof, st, KID_PACK);
    launch_chained(k_pack_samples, (unsigned)tiles, kPackRays, 0, st, a);
    prof_end(prof, st);
    return cudaGetLastError();
}

}  // namespace hp
