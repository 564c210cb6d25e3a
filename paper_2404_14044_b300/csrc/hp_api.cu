// C-ABI of the HashPoint hot path: argument checks, the search-window bound,
// workspace carving and kernel launches.  See include/hashpoint.h.
#include <cmath>
#include <cstring>
#include <new>

#include "hp_kernels.cuh"

using namespace hp;

struct hp_ctx {
    hp_config cfg;
    int device = 0;
    int num_sms = 1;
    ErrWord *d_err = nullptr;
    // caller workspace (if set)
    char *ws = nullptr;
    size_t ws_bytes = 0;
    // self-owned regions (used when no caller workspace is set)
    char *own[3] = {nullptr, nullptr, nullptr};
    size_t own_bytes[3] = {0, 0, 0};
    uint32_t spin_limit = kSpinLimitDefault;
    int32_t skip_tile = -1;
    // table state
    bool built = false;
    Cam cam{};
    int h = 0, Wp = 0, Hp = 0;
    int64_t P = 0, N = 0;
    float r = 0.f, rdd = 0.f;
    size_t table_bytes = 0;
    uint32_t *cnt = nullptr, *start = nullptr, *scan_ticket = nullptr;
    uint2 *keyrank = nullptr;
    float4 *spts = nullptr;
    uint32_t *pcell = nullptr;           // bucket of each listed point (the scatter writes it)
    uint64_t *scan_flags = nullptr;
    float4 *raytab = nullptr;        // per-pixel rays, cached while the intrinsics are unchanged
    bool raytab_valid = false;
    float raytab_key[8] = {0};
    // search state
    bool searched = false;
    bool rendered = false;
    const int32_t *rays = nullptr;   // pixel list of the last search (caller-owned)
    const hp_samples *last_samples = nullptr;
    int64_t R = 0;
    int K = 0, n_max = 0;
    size_t search_bytes = 0;
    // the last search left its neighbour lists in the slots (hp_samples.nbr NULL)
    bool lists_in_slots = false;
    const int32_t *slot_nbr = nullptr, *sample_slot = nullptr;
    const float *slot_dist = nullptr;
    Prof prof;
};

namespace {

constexpr size_t kAlign = 256;
inline size_t al(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

bool is_finite32(float x) { return std::isfinite(x); }

hp_status check_config(const hp_config *c)
{
    if (!c) return HP_ERR_INVALID_ARG;
    if (c->radius_mode < HP_RADIUS_FIXED || c->radius_mode > HP_RADIUS_CONE_APPROX) return HP_ERR_INVALID_ARG;
    if (!(c->gamma > 0.f && c->gamma <= 1.f)) return HP_ERR_INVALID_ARG;
    if (!(c->beta2 > 0.f) || !is_finite32(c->beta2)) return HP_ERR_INVALID_ARG;
    if (!(c->eps_w >= 0.f) || !is_finite32(c->eps_w)) return HP_ERR_INVALID_ARG;
    if (!(c->gap_k >= 0.f) || !is_finite32(c->gap_k)) return HP_ERR_INVALID_ARG;
    if (!(c->eps_d > 0.f) || !is_finite32(c->eps_d)) return HP_ERR_INVALID_ARG;
    if (c->cand_cap < 1 || c->cand_cap > kCandCap) return HP_ERR_INVALID_ARG;
    if (c->bg_mode != 0 && c->bg_mode != 1) return HP_ERR_INVALID_ARG;
    if (c->window_h < 0 || c->window_h > kHMax) return HP_ERR_INVALID_ARG;
    if (!is_finite32(c->rho)) return HP_ERR_INVALID_ARG;
    return HP_OK;
}

hp_status check_camera(const hp_camera *c)
{
    if (!c) return HP_ERR_INVALID_ARG;
    if (c->width < 1 || c->height < 1 || (int64_t)c->width * c->height > 0x7fffffffLL) return HP_ERR_INVALID_ARG;
    const float *f = &c->fx;
    for (int i = 0; i < 4 + 9 + 3 + 3; ++i)
        if (!is_finite32(f[i])) return HP_ERR_INVALID_ARG;
    if (!(c->fx > 0.f) || !(c->fy > 0.f)) return HP_ERR_INVALID_ARG;
    if (!(c->t_near > 0.f) || !(c->t_far >= c->t_near) || !(c->z_near > 0.f)) return HP_ERR_INVALID_ARG;
    return HP_OK;
}

// Window half-width.  An accepted point lies at t >= t_near within r(t) of
// the ray: P = t d + e with e orthogonal to d.  Its image-plane offset from
// the ray's pixel centre is (e_x d_z - d_x e_z)/(Z d_z), bounded by
// |e| sqrt(1 + nx^2) / Z, and Z >= t d_z - |e| sin(theta).  Bounding these
// over all pixel centres gives the largest offset L in pixels; the point then
// lies at most floor(L + 1/2) pixels away.  Cone modes keep the paper's
// s = 2 ceil(r_ddot / r_dot) + 1 when it is larger (Sec. 3.2).
hp_status derive_window(const hp_camera &c, const hp_config &cfg, float r, int *h_out, float *rdd_out)
{
    const double fx = c.fx, fy = c.fy, cx = c.cx, cy = c.cy;
    const double ax = std::fmax(std::fabs(0.5 - cx), std::fabs(((double)c.width - 0.5) - cx)) / fx;
    const double ay = std::fmax(std::fabs(0.5 - cy), std::fabs(((double)c.height - 0.5) - cy)) / fy;
    const double q = ax * ax + ay * ay;
    const double cosm = 1.0 / std::sqrt(1.0 + q);
    const double sinm = std::sqrt(q / (1.0 + q));
    double lim_x, lim_y, rdd = 0.0, rho = 0.0;
    if (cfg.radius_mode == HP_RADIUS_FIXED) {
        const double rr = r;
        if (!(rr > 0)) return HP_ERR_INVALID_ARG;
        double zlo = (double)c.t_near * cosm - rr * sinm;
        if (zlo < (double)c.z_near) zlo = (double)c.z_near;
        lim_x = fx * rr * std::sqrt(1.0 + ax * ax) / zlo;
        lim_y = fy * rr * std::sqrt(1.0 + ay * ay) / zlo;
    } else {
        const double rdot = std::sqrt(1.0 / ((3.14159265358979323846 * fx) * fy));
        if (cfg.rho > 0) {
            rho = cfg.rho;
            rdd = rho * rdot;
        } else {
            // r_min at t_near on the central ray equals the given radius
            const double rr = r, tn = c.t_near;
            if (!(rr > 0) || !(tn > rr)) return HP_ERR_INVALID_ARG;
            rdd = (cfg.radius_mode == HP_RADIUS_CONE) ? rr / std::sqrt(tn * tn - rr * rr) : rr / tn;
            rho = rdd / rdot;
        }
        const double den = cosm - rdd * sinm;
        if (!(den > 0)) return HP_ERR_INVALID_ARG;
        lim_x = fx * rdd * std::sqrt(1.0 + ax * ax) / den;
        lim_y = fy * rdd * std::sqrt(1.0 + ay * ay) / den;
    }
    const double lim = std::fmax(lim_x, lim_y) * (1.0 + 1e-3) + 1e-3;
    if (!(lim < (double)kHMax)) return HP_ERR_INVALID_ARG;
    int h = (int)std::floor(lim + 0.5);
    if (cfg.radius_mode != HP_RADIUS_FIXED) {
        const int hp_paper = (int)std::ceil(rho);
        if (hp_paper > h) h = hp_paper;
    }
    if (cfg.window_h > 0) h = cfg.window_h;
    if (h > kHMax) return HP_ERR_INVALID_ARG;
    *h_out = h;
    *rdd_out = (float)rdd;
    return HP_OK;
}

size_t table_region_bytes(int64_t N, int64_t P, int64_t npix)
{
    size_t o = 0;
    o += al(16 * (size_t)npix);                              // ray table (first: depends on W*H only)
    o += al(256);                                            // tickets
    o += al(8 * (size_t)div_up(P + 1, kScanTile));           // scan flags
    o += al(4 * (size_t)(P + 1));                            // cnt
    o += al(4 * (size_t)(P + 1));                            // start
    o += al(8 * (size_t)N);                                  // keyrank
    o += al(16 * (size_t)N);                                 // spts
    o += al(4 * (size_t)N);                                  // bucket of each listed point
    return o;
}

// ticket + look-back words, then the per-ray sample slots
size_t search_region_bytes(int64_t R, int n_max, int K)
{
    const size_t slots = (size_t)(R > 0 ? R : 1) * n_max;
    return al(256) + al(8 * (size_t)div_up(R > 0 ? R : 1, 256)) + al(16 * slots) + 2 * al(4 * slots * K) +
           al(4 * slots) +                           // slot of each packed sample (lists left in the slots)
           al(4 * (size_t)(R > 0 ? R : 1)) +         // fallback list of the proposal-restricted search
           al(4 * (size_t)(R > 0 ? R : 1)) +         // rays handed to the warp-per-ray search
           al(4 * (size_t)(R > 0 ? R : 1)) +         // pixels whose point-major slots overflowed
           al(8 * (size_t)(R > 0 ? R : 1)) +         // intervals the learned search inferred for them
           al(4 * (size_t)(R > 0 ? R : 1)) +         // point-major pass: candidates per pixel
           al(8 * (size_t)kPmCap * (size_t)(R > 0 ? R : 1));   // ... and the candidates
}

// decoded samples, then the backward's per-sample scratch, then the
// tensor-core decode's weight image and tile counter
size_t render_region_bytes(int64_t cap)
{
    const size_t c = (size_t)(cap > 0 ? cap : 1);
    return al(16 * c) + al(16 * c) + al(4 * c) + al(kWsImageMax) + al(256);
}

// Region i of the workspace: 0 table, 1 search, 2 render.
hp_status region(hp_ctx *ctx, int i, size_t bytes, char **out)
{
    if (ctx->ws) {
        size_t off = 0;
        if (i >= 1) off += ctx->table_bytes;
        if (i >= 2) off += ctx->search_bytes;
        if (off + bytes > ctx->ws_bytes) return HP_ERR_NO_MEMORY;
        *out = ctx->ws + off;
        return HP_OK;
    }
    if (ctx->own_bytes[i] < bytes) {
        if (i == 0) ctx->raytab_valid = false;          // fresh memory: the cached ray table is gone
        if (ctx->own[i]) cudaFree(ctx->own[i]);
        ctx->own[i] = nullptr;
        ctx->own_bytes[i] = 0;
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return HP_ERR_NO_MEMORY;
        }
        ctx->own[i] = static_cast<char *>(p);
        ctx->own_bytes[i] = bytes;
    }
    *out = ctx->own[i];
    return HP_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

extern "C" {

const char *hp_status_string(hp_status s)
{
    switch (s) {
    case HP_OK: return "ok";
    case HP_ERR_INVALID_ARG: return "invalid argument";
    case HP_ERR_CUDA: return "CUDA error";
    case HP_ERR_OVERFLOW: return "sample capacity overflow";
    case HP_ERR_TIMEOUT: return "bounded wait timed out";
    case HP_ERR_NOT_BUILT: return "table or samples not built";
    case HP_ERR_NO_MEMORY: return "workspace too small or allocation failed";
    case HP_ERR_BAD_RAY: return "ray pixel out of range";
    case HP_ERR_TOO_LARGE: return "size exceeds the allocation-free limit";
    case HP_ERR_BOUNDS: return "index outside its array (bounds-check build)";
    }
    return "unknown status";
}

int32_t hp_version(void) { return 10000; }

hp_status hp_create(hp_ctx **out, const hp_config *cfg)
{
    if (!out) return HP_ERR_INVALID_ARG;
    *out = nullptr;
    hp_status s = check_config(cfg);
    if (s != HP_OK) return s;
    hp_ctx *ctx = new (std::nothrow) hp_ctx();
    if (!ctx) return HP_ERR_NO_MEMORY;
    ctx->cfg = *cfg;
    if (cudaGetDevice(&ctx->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return HP_ERR_CUDA;
    }
    void *p = nullptr;
    if (cudaMalloc(&p, 64) != cudaSuccess || cudaMemset(p, 0, 64) != cudaSuccess) {
        cudaGetLastError();
        if (p) cudaFree(p);
        delete ctx;
        return HP_ERR_CUDA;
    }
    ctx->d_err = static_cast<ErrWord *>(p);
    *out = ctx;
    return HP_OK;
}

static void prof_release(Prof &p)
{
    if (p.ev) {
        for (int i = 0; i < 2 * p.cap; ++i) cudaEventDestroy(p.ev[i]);
        delete[] p.ev;
    }
    delete[] p.kid;
    delete[] p.nk;
    p = Prof();
}

hp_status hp_profile_start(hp_ctx *ctx, int32_t max_launches)
{
    if (!ctx || max_launches < 1 || max_launches > (1 << 20)) return HP_ERR_INVALID_ARG;
    prof_release(ctx->prof);
    Prof &p = ctx->prof;
    p.ev = new (std::nothrow) cudaEvent_t[2 * (size_t)max_launches];
    p.kid = new (std::nothrow) int[max_launches];
    p.nk = new (std::nothrow) int[max_launches];
    if (!p.ev || !p.kid || !p.nk) {
        delete[] p.ev;
        delete[] p.kid;
        delete[] p.nk;
        p = Prof();
        return HP_ERR_NO_MEMORY;
    }
    for (int i = 0; i < 2 * max_launches; ++i) {
        if (cudaEventCreate(&p.ev[i]) != cudaSuccess) {
            cudaGetLastError();
            p.cap = i / 2;
            prof_release(p);
            return HP_ERR_CUDA;
        }
    }
    p.cap = max_launches;
    p.n = 0;
    p.on = true;
    return HP_OK;
}

hp_status hp_profile_stop(hp_ctx *ctx, double *ms, int32_t *launches, int32_t *kernels)
{
    if (!ctx) return HP_ERR_INVALID_ARG;
    Prof &p = ctx->prof;
    double acc[KID_COUNT] = {0};
    int32_t cnt[KID_COUNT] = {0}, nk[KID_COUNT] = {0};
    hp_status s = HP_OK;
    for (int i = 0; i < p.n; ++i) {
        float t = 0.f;
        if (cudaEventSynchronize(p.ev[2 * i + 1]) != cudaSuccess ||
            cudaEventElapsedTime(&t, p.ev[2 * i], p.ev[2 * i + 1]) != cudaSuccess) {
            cudaGetLastError();
            s = HP_ERR_CUDA;
            break;
        }
        acc[p.kid[i]] += t;
        cnt[p.kid[i]] += 1;
        nk[p.kid[i]] += p.nk[i];
    }
    for (int k = 0; k < KID_COUNT; ++k) {
        if (ms) ms[k] = acc[k];
        if (launches) launches[k] = cnt[k];
        if (kernels) kernels[k] = nk[k];
    }
    prof_release(p);
    return s;
}

const char *hp_profile_kernel_name(int32_t id)
{
    static const char *names[KID_COUNT] = {"k_project_count", "k_scan", "k_scatter", "k_bucket_sort",
                                           "k_search_select", "k_pack_samples", "k_aggregate_decode",
                                           "k_composite", "k_composite_bwd", "k_decode_bwd", "k_prop_infer",
                                           "k_search_select_fallback", "k_search_select_wide", "k_ray_table",
                                           "k_clear"};
    static_assert(KID_COUNT == HP_PROF_KERNELS, "profiler kernel count");
    return (id >= 0 && id < KID_COUNT) ? names[id] : "unknown";
}

hp_status hp_destroy(hp_ctx *ctx)
{
    if (!ctx) return HP_ERR_INVALID_ARG;
    prof_release(ctx->prof);
    for (int i = 0; i < 3; ++i)
        if (ctx->own[i]) cudaFree(ctx->own[i]);
    if (ctx->d_err) cudaFree(ctx->d_err);
    delete ctx;
    return HP_OK;
}

hp_status hp_workspace_size(const hp_config *cfg, const hp_camera *cam, float r, int64_t n_points, int64_t n_rays,
                            int32_t K, int32_t n_samples, size_t *bytes)
{
    hp_status s;
    if (!bytes || n_points < 0 || n_rays < 0 || n_samples < 1 || n_samples > kMaxSamples || K < 1 || K > kMaxK)
        return HP_ERR_INVALID_ARG;
    if ((s = check_config(cfg)) != HP_OK || (s = check_camera(cam)) != HP_OK) return s;
    int h;
    float rdd;
    if ((s = derive_window(*cam, *cfg, r, &h, &rdd)) != HP_OK) return s;
    const int64_t P = (int64_t)(cam->width + 2 * h) * (cam->height + 2 * h);
    *bytes = table_region_bytes(n_points, P, (int64_t)cam->width * cam->height) +
             search_region_bytes(n_rays, n_samples, K) +
             render_region_bytes(n_rays * n_samples);
    return HP_OK;
}

hp_status hp_window(const hp_config *cfg, const hp_camera *cam, float r, int32_t *h_out, float *rdd_out)
{
    hp_status s;
    if (!h_out || !rdd_out) return HP_ERR_INVALID_ARG;
    if ((s = check_config(cfg)) != HP_OK || (s = check_camera(cam)) != HP_OK) return s;
    int h;
    float rdd;
    if ((s = derive_window(*cam, *cfg, r, &h, &rdd)) != HP_OK) return s;
    *h_out = h;
    *rdd_out = rdd;
    return HP_OK;
}

hp_status hp_set_workspace(hp_ctx *ctx, void *d_ptr, size_t bytes)
{
    if (!ctx || (d_ptr && ((uintptr_t)d_ptr % kAlign) != 0)) return HP_ERR_INVALID_ARG;
    ctx->raytab_valid = false;
    ctx->ws = static_cast<char *>(d_ptr);
    ctx->ws_bytes = d_ptr ? bytes : 0;
    ctx->built = false;
    ctx->searched = false;
    return HP_OK;
}

hp_status hp_debug_fault(hp_ctx *ctx, int32_t skip_tile, int32_t spin_limit)
{
    if (!ctx || spin_limit < 0) return HP_ERR_INVALID_ARG;
    ctx->skip_tile = skip_tile;
    ctx->spin_limit = spin_limit > 0 ? (uint32_t)spin_limit : kSpinLimitDefault;
    return HP_OK;
}

hp_status hp_build_table(hp_ctx *ctx, const float *d_points, int64_t n_points, const hp_camera *cam, float r,
                         void *stream)
{
    hp_status s;
    if (!ctx || n_points < 0 || n_points > 0x7fffffffLL || (n_points > 0 && !d_points)) return HP_ERR_INVALID_ARG;
    if ((s = check_camera(cam)) != HP_OK) return s;
    if (!is_finite32(r)) return HP_ERR_INVALID_ARG;
    int h;
    float rdd;
    if ((s = derive_window(*cam, ctx->cfg, r, &h, &rdd)) != HP_OK) return s;
    const int Wp = cam->width + 2 * h, Hp = cam->height + 2 * h;
    const int64_t P = (int64_t)Wp * Hp;
    if (P + 1 > 0xffffffffLL) return HP_ERR_INVALID_ARG;
    ctx->built = false;
    ctx->searched = false;
    const int64_t npix = (int64_t)cam->width * cam->height;
    ctx->table_bytes = table_region_bytes(n_points, P, npix);
    char *base = nullptr;
    if ((s = region(ctx, 0, ctx->table_bytes, &base)) != HP_OK) return s;
    size_t o = 0;
    {
        // the ray table depends on the intrinsics, the radius mode and r_ddot only
        const float key[8] = {(float)cam->width, (float)cam->height, cam->fx, cam->fy, cam->cx, cam->cy,
                              (float)ctx->cfg.radius_mode, rdd};
        float4 *rt = reinterpret_cast<float4 *>(base);
        if (!ctx->raytab_valid || rt != ctx->raytab || std::memcmp(key, ctx->raytab_key, sizeof(key)) != 0) {
            ctx->raytab_valid = false;
            std::memcpy(ctx->raytab_key, key, sizeof(key));
        }
        ctx->raytab = rt;
        o += al(16 * (size_t)npix);
    }
    // tickets, look-back words and counts back to back: the build clears
    // them with one memset
    ctx->scan_ticket = reinterpret_cast<uint32_t *>(base + o); o += al(256);
    ctx->scan_flags = reinterpret_cast<uint64_t *>(base + o);  o += al(8 * (size_t)div_up(P + 1, kScanTile));
    ctx->cnt = reinterpret_cast<uint32_t *>(base + o);         o += al(4 * (size_t)(P + 1));
    ctx->start = reinterpret_cast<uint32_t *>(base + o);       o += al(4 * (size_t)(P + 1));
    ctx->keyrank = reinterpret_cast<uint2 *>(base + o);        o += al(8 * (size_t)n_points);
    ctx->spts = reinterpret_cast<float4 *>(base + o);          o += al(16 * (size_t)n_points);
    ctx->pcell = reinterpret_cast<uint32_t *>(base + o);

    Cam c{};
    std::memcpy(c.R, cam->R, sizeof(c.R));
    std::memcpy(c.t, cam->t, sizeof(c.t));
    c.fx = cam->fx; c.fy = cam->fy; c.cx = cam->cx; c.cy = cam->cy;
    c.t_near = cam->t_near; c.t_far = cam->t_far; c.z_near = cam->z_near;
    c.width = cam->width; c.height = cam->height;
    ctx->cam = c;
    ctx->h = h; ctx->Wp = Wp; ctx->Hp = Hp; ctx->P = P; ctx->N = n_points;
    ctx->r = r; ctx->rdd = rdd;

    BuildArgs a{};
    a.pts = d_points; a.N = n_points; a.cam = c; a.h = h; a.P = P;
    a.cnt = ctx->cnt; a.start = ctx->start; a.keyrank = ctx->keyrank; a.spts = ctx->spts;
    a.scan_flags = ctx->scan_flags; a.scan_ticket = ctx->scan_ticket; a.err = ctx->d_err;
    a.zmin_enc = ctx->scan_ticket + 1;
    a.pcell = ctx->pcell;
    a.spin_limit = ctx->spin_limit; a.skip_tile = ctx->skip_tile;
    if (launch_build(a, static_cast<cudaStream_t>(stream), &ctx->prof) != cudaSuccess) {
        cudaGetLastError();
        return HP_ERR_CUDA;
    }
    ctx->built = true;
    return HP_OK;
}

hp_status hp_table_info(const hp_ctx *ctx, hp_table *out)
{
    if (!ctx || !out) return HP_ERR_INVALID_ARG;
    if (!ctx->built) return HP_ERR_NOT_BUILT;
    out->h = ctx->h;
    out->padded_width = ctx->Wp;
    out->padded_height = ctx->Hp;
    out->n_buckets = ctx->P;
    out->r_ddot = ctx->rdd;
    out->d_start = ctx->start;
    out->d_points = reinterpret_cast<const float *>(ctx->spts);
    return HP_OK;
}

hp_status hp_table_copy(const hp_ctx *ctx, uint32_t *d_start, float *d_points, void *stream)
{
    if (!ctx || !d_start || (ctx->N > 0 && !d_points)) return HP_ERR_INVALID_ARG;
    if (!ctx->built) return HP_ERR_NOT_BUILT;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(d_start, ctx->start, 4 * (size_t)(ctx->P + 1), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        return HP_ERR_CUDA;
    }
    // the list in its canonical order: every bucket sorted by (z, x, y, id)
    // into the caller's buffer (the table itself keeps the scatter's order)
    if (ctx->N > 0 && launch_bucket_sort(ctx->P, ctx->start, ctx->spts, reinterpret_cast<float4 *>(d_points), ctx->cnt,
                                         ctx->scan_ticket + 2, st) != cudaSuccess) {
        cudaGetLastError();
        return HP_ERR_CUDA;
    }
    return HP_OK;
}

// Most candidates the selection (Sec. 3.3) can process on a ray: every
// processed candidate multiplies T by 1 - alpha_j <= 1 - alpha_min, alpha_min
// = gamma exp(-d_max^2 / beta^2) with d_max the largest radius a neighbour can
// lie within (the pseudo-UDF d_j is a mean of such distances), and the
// selection stops once gamma T <= eps_w.  The margins cover float32 rounding
// and exp32's error.  0 when the bound exceeds kPruneMax (or does not exist).
static int selection_bound(const hp_config &cfg, int mode, float r, float rdd, float t_far)
{
    const double g = cfg.gamma, b2 = cfg.beta2, eps = cfg.eps_w;
    if (!(g > 0.0) || !(b2 > 0.0) || !(eps > 0.0)) return 0;
    const double dmax = (mode == HP_RADIUS_FIXED ? (double)r : (double)t_far * (double)rdd) * 1.001;
    const double amin = g * std::exp(-dmax * dmax / b2) * (1.0 - 1e-4);
    if (!(amin > 0.0) || !(amin < 1.0)) return 0;
    double T = 1.0;
    for (int m = 1; m <= kPruneMax; ++m) {
        T *= (1.0 - amin) * (1.0 + 1e-5);
        if (g * T <= eps * (1.0 - 1e-5)) return m;
    }
    return 0;
}

static hp_status search_impl(hp_ctx *ctx, const int32_t *d_ray_pixels, int64_t n_rays, int32_t K, int32_t n_samples,
                             const hp_samples *out, const float *d_interval, const uint16_t *d_prop_w,
                             uint32_t *d_fallback_count, void *stream)
{
    if (!ctx || !out) return HP_ERR_INVALID_ARG;
    if (!ctx->built) return HP_ERR_NOT_BUILT;
    if (n_rays < 0 || n_rays > 0x7fffffffLL || K < 1 || K > kMaxK || n_samples < 1 || n_samples > kMaxSamples)
        return HP_ERR_INVALID_ARG;
    if (!d_ray_pixels && n_rays != 0 && n_rays != (int64_t)ctx->cam.width * ctx->cam.height)
        return HP_ERR_INVALID_ARG;
    if (!out->sample_offset || out->capacity < 0) return HP_ERR_INVALID_ARG;
    if (n_rays > 0 && (!out->n_s || !out->primary || !out->cand_count)) return HP_ERR_INVALID_ARG;
    if (out->capacity > 0 && (!out->t || !out->ray || !out->src || !out->delta))
        return HP_ERR_INVALID_ARG;
    // the neighbour lists: both packed, or both left in the search's slots
    // (slot indices must then fit int32)
    const bool lists_in_slots = !out->nbr;
    if ((!out->nbr) != (!out->nbr_dist)) return HP_ERR_INVALID_ARG;
    if (lists_in_slots && n_rays * (int64_t)n_samples > 0x7fffffffLL) return HP_ERR_INVALID_ARG;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    ctx->searched = false;
    ctx->lists_in_slots = false;
    ctx->search_bytes = search_region_bytes(n_rays, n_samples, K);
    char *base = nullptr;
    hp_status s;
    if ((s = region(ctx, 1, ctx->search_bytes, &base)) != HP_OK) return s;
    if (n_rays == 0) {
        if (cudaMemsetAsync(out->sample_offset, 0, sizeof(int64_t), st) != cudaSuccess) {
            cudaGetLastError();
            return HP_ERR_CUDA;
        }
    } else {
        SearchArgs a{};
        a.cam = ctx->cam; a.mode = ctx->cfg.radius_mode; a.r = ctx->r; a.rdd = ctx->rdd; a.h = ctx->h;
        a.Wp = ctx->Wp; a.gamma = ctx->cfg.gamma; a.beta2 = ctx->cfg.beta2; a.eps_w = ctx->cfg.eps_w;
        a.gap_k = ctx->cfg.gap_k; a.cand_cap = ctx->cfg.cand_cap; a.K = K; a.n_max = n_samples;
        a.prune_m = selection_bound(ctx->cfg, ctx->cfg.radius_mode, ctx->r, ctx->rdd, ctx->cam.t_far);
        a.start = ctx->start; a.spts = ctx->spts; a.rays = d_ray_pixels; a.R = n_rays;
        a.raytab = ctx->raytab; a.raytab_stale = ctx->raytab_valid ? 0 : 1;
        a.n_s = out->n_s; a.primary = out->primary; a.cand_count = out->cand_count;
        a.sample_offset = out->sample_offset; a.t = out->t; a.ray = out->ray; a.src = out->src;
        a.delta = out->delta; a.nbr = out->nbr; a.nbr_dist = out->nbr_dist; a.capacity = out->capacity;
        const size_t slots = (size_t)n_rays * n_samples;
        size_t o = 0;
        a.ticket = reinterpret_cast<uint32_t *>(base + o);   o += al(256);
        a.flags = reinterpret_cast<uint64_t *>(base + o);    o += al(8 * (size_t)div_up(n_rays, 256));
        // right after the look-back words: the search clears the tickets,
        // those words and the per-pixel candidate counts with one memset
        a.pm_cnt = reinterpret_cast<uint32_t *>(base + o);    o += al(4 * (size_t)n_rays);
        a.slot_rec = reinterpret_cast<float4 *>(base + o);   o += al(16 * slots);
        a.slot_nbr = reinterpret_cast<int32_t *>(base + o);  o += al(4 * slots * K);
        a.slot_dist = reinterpret_cast<float *>(base + o);   o += al(4 * slots * K);
        a.sample_slot = reinterpret_cast<int32_t *>(base + o); o += al(4 * slots);
        a.fallback = reinterpret_cast<int32_t *>(base + o);  o += al(4 * (size_t)n_rays);
        a.fallback_count = a.ticket + 1;
        a.wide = reinterpret_cast<int32_t *>(base + o);      o += al(4 * (size_t)n_rays);
        a.ovf = reinterpret_cast<int32_t *>(base + o);       o += al(4 * (size_t)n_rays);
        a.ovf_count = a.ticket + 6;
        a.ovf_pull = a.ticket + 7;
        a.interval_buf = reinterpret_cast<float2 *>(base + o); o += al(8 * (size_t)n_rays);
        a.pm_t = reinterpret_cast<float *>(base + o);
        a.pm_i = reinterpret_cast<uint32_t *>(base + o + 4 * (size_t)kPmCap * (size_t)n_rays);
        a.pcell = ctx->pcell;
        a.n_points = ctx->N;
        a.prop_w = d_prop_w;
        a.wide_count = a.ticket + 2;
        a.pull = reinterpret_cast<unsigned long long *>(a.ticket + 4);
        a.lane_units = a.ticket + 3;
        a.n_sm = ctx->num_sms;
        a.interval = reinterpret_cast<const float2 *>(d_interval);
        a.zmin_enc = ctx->scan_ticket + 1;
        if (ctx->cfg.radius_mode == HP_RADIUS_FIXED) {
            // window bound terms for a depth lower bound (same terms as derive_window)
            const double fx = ctx->cam.fx, fy = ctx->cam.fy, cx = ctx->cam.cx, cy = ctx->cam.cy;
            const double ax = std::fmax(std::fabs(0.5 - cx), std::fabs(((double)ctx->cam.width - 0.5) - cx)) / fx;
            const double ay = std::fmax(std::fabs(0.5 - cy), std::fabs(((double)ctx->cam.height - 0.5) - cy)) / fy;
            const double q = ax * ax + ay * ay;
            a.cos_max = (float)(1.0 / std::sqrt(1.0 + q));
            a.sin_max = (float)std::sqrt(q / (1.0 + q));
            a.win_fx = (float)std::fmax(fx * ctx->r * std::sqrt(1.0 + ax * ax), fy * ctx->r * std::sqrt(1.0 + ay * ay));
        }
        a.err = ctx->d_err;
        a.spin_limit = ctx->spin_limit;
        if (launch_search(a, st, &ctx->prof) != cudaSuccess) {
            cudaGetLastError();
            return HP_ERR_CUDA;
        }
        ctx->raytab_valid = true;
        if (lists_in_slots) {
            ctx->lists_in_slots = true;
            ctx->slot_nbr = a.slot_nbr;
            ctx->slot_dist = a.slot_dist;
            ctx->sample_slot = a.sample_slot;
        }
        if ((d_interval || d_prop_w) && d_fallback_count &&
            cudaMemcpyAsync(d_fallback_count, a.fallback_count, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) !=
                cudaSuccess) {
            cudaGetLastError();
            return HP_ERR_CUDA;
        }
    }
    ctx->R = n_rays;
    ctx->K = K;
    ctx->n_max = n_samples;
    ctx->rays = d_ray_pixels;
    ctx->searched = true;
    ctx->rendered = false;
    return HP_OK;
}

hp_status hp_search_sample(hp_ctx *ctx, const int32_t *d_ray_pixels, int64_t n_rays, int32_t K, int32_t n_samples,
                           const hp_samples *out, void *stream)
{
    return search_impl(ctx, d_ray_pixels, n_rays, K, n_samples, out, nullptr, nullptr, nullptr, stream);
}

hp_status hp_search_sample_proposal(hp_ctx *ctx, const int32_t *d_ray_pixels, int64_t n_rays, int32_t K,
                                    int32_t n_samples, const float *d_interval, const hp_samples *out,
                                    uint32_t *d_fallback_count, void *stream)
{
    if (!d_interval) return HP_ERR_INVALID_ARG;
    return search_impl(ctx, d_ray_pixels, n_rays, K, n_samples, out, d_interval, nullptr, d_fallback_count, stream);
}

hp_status hp_search_sample_learned(hp_ctx *ctx, const int32_t *d_ray_pixels, int64_t n_rays, int32_t K,
                                   int32_t n_samples, const uint16_t *d_weights_bf16, const hp_samples *out,
                                   uint32_t *d_fallback_count, void *stream)
{
    if (!d_weights_bf16) return HP_ERR_INVALID_ARG;
    return search_impl(ctx, d_ray_pixels, n_rays, K, n_samples, out, nullptr, d_weights_bf16, d_fallback_count,
                       stream);
}

static PropArgs prop_args(const hp_ctx *ctx, const int32_t *d_rays, int64_t n_rays)
{
    PropArgs a{};
    a.cam = ctx->cam; a.h = ctx->h; a.Wp = ctx->Wp; a.Hp = ctx->Hp; a.start = ctx->start; a.spts = ctx->spts;
    a.rays = d_rays; a.R = n_rays;
    return a;
}

hp_status hp_proposal_infer(hp_ctx *ctx, const int32_t *d_ray_pixels, int64_t n_rays, const uint16_t *d_weights_bf16,
                            float *d_interval, void *stream)
{
    if (!ctx || !d_weights_bf16 || n_rays < 0 || (n_rays > 0 && !d_interval)) return HP_ERR_INVALID_ARG;
    if (!ctx->built) return HP_ERR_NOT_BUILT;
    if (!d_ray_pixels && n_rays != 0 && n_rays != (int64_t)ctx->cam.width * ctx->cam.height) return HP_ERR_INVALID_ARG;
    PropArgs a = prop_args(ctx, d_ray_pixels, n_rays);
    a.weights_bf16 = d_weights_bf16;
    a.interval = reinterpret_cast<float2 *>(d_interval);
    if (launch_prop_infer(a, static_cast<cudaStream_t>(stream), &ctx->prof) != cudaSuccess) {
        cudaGetLastError();
        return HP_ERR_CUDA;
    }
    return HP_OK;
}

hp_status hp_proposal_train_step(hp_ctx *ctx, const int32_t *d_ray_pixels, int64_t n_rays, const hp_samples *plain,
                                 float *d_params, float *d_adam_m, float *d_adam_v, float *d_grad,
                                 uint16_t *d_weights_bf16, int32_t step, float lr, float *d_loss, void *stream)
{
    if (!ctx || !plain || !d_params || !d_adam_m || !d_adam_v || !d_grad || !d_weights_bf16 || step < 1 ||
        !(lr > 0.f) || n_rays < 0)
        return HP_ERR_INVALID_ARG;
    if (!ctx->built) return HP_ERR_NOT_BUILT;
    if (!d_ray_pixels && n_rays != 0 && n_rays != (int64_t)ctx->cam.width * ctx->cam.height) return HP_ERR_INVALID_ARG;
    PropArgs a = prop_args(ctx, d_ray_pixels, n_rays);
    a.params = d_params; a.grad = d_grad; a.loss = d_loss; a.weights_out = d_weights_bf16;
    a.n_s = plain->n_s; a.sample_offset = plain->sample_offset; a.t = plain->t;
    if (launch_prop_train(a, d_adam_m, d_adam_v, step, lr, static_cast<cudaStream_t>(stream)) != cudaSuccess) {
        cudaGetLastError();
        return HP_ERR_CUDA;
    }
    return HP_OK;
}

hp_status hp_aggregate_render(hp_ctx *ctx, const hp_samples *smp, int64_t n_rays, const float *d_feats, int32_t F,
                              const hp_mlp *mlp, float *d_rgb, float *d_wsum, void *stream)
{
    if (!ctx || !smp || !mlp) return HP_ERR_INVALID_ARG;
    if (!ctx->built || !ctx->searched || n_rays != ctx->R) return HP_ERR_NOT_BUILT;
    if (!(F == 4 || F == 8 || F == 16 || F == 32 || F == 64 || F == 128)) return HP_ERR_INVALID_ARG;
    if (mlp->n_layers < 1 || mlp->n_layers > HP_MLP_MAX_LAYERS || !mlp->d_params) return HP_ERR_INVALID_ARG;
    if (mlp->dims[0] != F || mlp->dims[mlp->n_layers] != 4) return HP_ERR_INVALID_ARG;
    int64_t n_par = 0;
    for (int l = 0; l < mlp->n_layers; ++l) {
        const int fo = mlp->dims[l + 1];
        if (l + 1 < mlp->n_layers && !(fo == 16 || fo == 32 || fo == 64 || fo == 128)) return HP_ERR_INVALID_ARG;
        n_par += (int64_t)mlp->dims[l] * fo + fo;
    }
    if (n_par > 40960) return HP_ERR_INVALID_ARG;
    if (n_rays > 0 && ((ctx->N > 0 && !d_feats) || !d_rgb || !d_wsum || !aligned16(d_feats)))
        return HP_ERR_INVALID_ARG;
    if (n_rays == 0) return HP_OK;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *base = nullptr;
    hp_status s;
    if ((s = region(ctx, 2, render_region_bytes(smp->capacity), &base)) != HP_OK) return s;
    RenderArgs a{};
    a.n_s = smp->n_s; a.sample_offset = smp->sample_offset; a.delta = smp->delta; a.nbr = smp->nbr;
    a.nbr_dist = smp->nbr_dist; a.capacity = smp->capacity; a.R = n_rays; a.K = ctx->K;
    if (!smp->nbr || !smp->nbr_dist) {
        // the lists stayed in the last search's slots
        if (smp->nbr || smp->nbr_dist || !ctx->lists_in_slots) return HP_ERR_INVALID_ARG;
        a.nbr = nullptr;
        a.nbr_dist = nullptr;
        a.slot_nbr = ctx->slot_nbr;
        a.slot_dist = ctx->slot_dist;
        a.sample_slot = ctx->sample_slot;
    }
    a.feats = d_feats; a.F = F; a.mlp = mlp->d_params; a.n_layers = mlp->n_layers;
    for (int l = 0; l <= mlp->n_layers; ++l) a.dims[l] = mlp->dims[l];
    a.eps_d = ctx->cfg.eps_d; a.bg_mode = ctx->cfg.bg_mode;
    a.decode = mlp->decode; a.err = ctx->d_err;
    if (a.decode < HP_DECODE_FP32 || a.decode > HP_DECODE_BF16) return HP_ERR_INVALID_ARG;
    if (a.decode == HP_DECODE_BF16 && !decode_tc_supported(a, true, nullptr)) return HP_ERR_INVALID_ARG;
    a.sample_out = reinterpret_cast<float4 *>(base);
    {
        const size_t c = (size_t)(smp->capacity > 0 ? smp->capacity : 1);
        const size_t o = al(16 * c) + al(16 * c) + al(4 * c);
        a.wimg = reinterpret_cast<unsigned char *>(base + o);
        a.tile_ctr = reinterpret_cast<uint32_t *>(base + o + al(kWsImageMax));
    }
    a.rgb = d_rgb; a.wsum = d_wsum; a.num_sms = ctx->num_sms;
    a.n_feats = ctx->N;
    a.n_slots = ctx->R * (int64_t)ctx->n_max;
    const bool tc_ok = a.decode != HP_DECODE_FP32_SIMT && decode_tc_supported(a, a.decode == HP_DECODE_BF16, nullptr);
    if (!tc_ok && render_smem_bytes(a) > 227 * 1024) return HP_ERR_INVALID_ARG;
    if (launch_render(a, st, &ctx->prof) != cudaSuccess) {
        cudaGetLastError();
        return HP_ERR_CUDA;
    }
    ctx->rendered = true;
    return HP_OK;
}

hp_status hp_aggregate_render_backward(hp_ctx *ctx, const hp_samples *smp, int64_t n_rays, const float *d_points,
                                       const float *d_feats, int32_t F, const hp_mlp *mlp, const float *d_grad_rgb,
                                       const float *d_grad_wsum, float *d_grad_feats, float *d_grad_points,
                                       void *stream)
{
    if (!ctx || !smp || !mlp) return HP_ERR_INVALID_ARG;
    if (!ctx->built || !ctx->searched || !ctx->rendered || n_rays != ctx->R) return HP_ERR_NOT_BUILT;
    if (mlp->n_layers < 1 || mlp->n_layers > HP_MLP_MAX_LAYERS || !mlp->d_params || mlp->dims[0] != F ||
        mlp->dims[mlp->n_layers] != 4)
        return HP_ERR_INVALID_ARG;
    for (int l = 0; l <= mlp->n_layers; ++l)
        if (mlp->dims[l] < 1 || mlp->dims[l] > HP_MLP_MAX_WIDTH) return HP_ERR_INVALID_ARG;
    // the backward reads the packed neighbour lists
    if (!smp->nbr || !smp->nbr_dist) return HP_ERR_INVALID_ARG;
    if (n_rays == 0) return HP_OK;
    if (!d_grad_rgb || (ctx->N > 0 && (!d_feats || !d_points))) return HP_ERR_INVALID_ARG;
    char *base = nullptr;
    hp_status s;
    if ((s = region(ctx, 2, render_region_bytes(smp->capacity), &base)) != HP_OK) return s;
    const size_t c = (size_t)(smp->capacity > 0 ? smp->capacity : 1);
    BwdArgs a{};
    a.n_s = smp->n_s; a.sample_offset = smp->sample_offset; a.t = smp->t; a.ray = smp->ray; a.src = smp->src;
    a.delta = smp->delta; a.nbr = smp->nbr; a.nbr_dist = smp->nbr_dist; a.capacity = smp->capacity;
    a.R = n_rays; a.K = ctx->K; a.rays = ctx->rays; a.raytab = ctx->raytab; a.cam = ctx->cam;
    a.mode = ctx->cfg.radius_mode; a.points = d_points; a.feats = d_feats; a.F = F; a.mlp = mlp->d_params;
    a.n_layers = mlp->n_layers;
    for (int l = 0; l <= mlp->n_layers; ++l) a.dims[l] = mlp->dims[l];
    a.eps_d = ctx->cfg.eps_d; a.bg_mode = ctx->cfg.bg_mode;
    a.sample_out = reinterpret_cast<const float4 *>(base);
    a.go = reinterpret_cast<float4 *>(base + al(16 * c));
    a.gt = reinterpret_cast<float *>(base + 2 * al(16 * c));
    a.grad_rgb = d_grad_rgb; a.grad_wsum = d_grad_wsum; a.grad_feats = d_grad_feats; a.grad_points = d_grad_points;
    a.n_points = ctx->N;
    a.err = ctx->d_err;
    a.num_sms = ctx->num_sms;
    if (backward_smem_bytes(a) > 227 * 1024) return HP_ERR_INVALID_ARG;
    if (launch_backward(a, static_cast<cudaStream_t>(stream), &ctx->prof) != cudaSuccess) {
        cudaGetLastError();
        return HP_ERR_CUDA;
    }
    return HP_OK;
}

hp_status hp_selftest_mma(hp_ctx *ctx, const uint16_t *d_a, const uint16_t *d_b, float *d_d, int32_t K, int32_t N,
                          int32_t flags, void *stream)
{
    if (!ctx || !d_a || !d_b || !d_d) return HP_ERR_INVALID_ARG;
    if (K < 16 || K > 128 || K % 16 != 0 || N < 16 || N > 256 || N % 16 != 0 || (flags & ~3) != 0)
        return HP_ERR_INVALID_ARG;
    if (launch_mma_selftest(d_a, d_b, d_d, K, N, flags, ctx->d_err, static_cast<cudaStream_t>(stream)) !=
        cudaSuccess) {
        cudaGetLastError();
        return HP_ERR_CUDA;
    }
    return HP_OK;
}

hp_status hp_get_status(hp_ctx *ctx, void *stream, int32_t *dev_status, int64_t *detail)
{
    if (!ctx) return HP_ERR_INVALID_ARG;
    ErrWord w{};
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess ||
        cudaMemcpy(&w, ctx->d_err, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(ctx->d_err, 0, sizeof(w)) != cudaSuccess) {
        cudaGetLastError();
        return HP_ERR_CUDA;
    }
    if (dev_status) *dev_status = w.status;
    if (detail) *detail = w.detail;
    return HP_OK;
}

}  // extern "C"
