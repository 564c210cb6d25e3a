/*
 * HashPoint CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-file restatement of the per-frame hot path of
 * "HashPoint: Accelerated Point Searching and Sampling for Neural Rendering"
 * (CVPR 2024): table build (Sec. 3.2, "Accelerated structure construction"),
 * window search (Sec. 3.2 "Searching", Eq. radius), adaptive primary surface
 * sampling (Sec. 3.3, the pseudo-UDF d_j, alpha_j and Eq. weight), then the
 * integration of Sec. 3.4: inverse-distance feature aggregation, a radiance
 * MLP and volume rendering (Eq. 2).
 *
 * Only the test-suite, the package smoke check and the benchmark's CPU
 * baseline may load this library.  It shares no code with the CUDA path.
 *
 * Precision.  Every *continuous* value (aggregated feature, MLP, density,
 * colour, compositing) is computed in double.  Every *discrete decision*
 * (pixel keys, accept/reject, orderings, K-nearest sets, alpha/weight
 * thresholds, clusters, sample counts) is taken in float32 under the
 * "decision arithmetic contract" below, so that a float32 GPU kernel that
 * follows the same contract reaches the same decisions bit for bit.  The
 * float32 quantities the contract defines (camera-space positions, ray
 * directions, sample depths t_j) are the inputs of the double-precision
 * continuous stages.
 *
 * Decision arithmetic contract (each + - * / is one IEEE binary32 operation
 * rounded to nearest-even, in the written order; sqrtf is correctly rounded;
 * fmaf is one rounding of a*b+c; nothing is contracted; build with
 * -ffp-contract=off):
 *   D1 camera space   X = ((R0*px + R1*py) + R2*pz) + t0   (rows 1, 2 alike)
 *   D2 key            u = fx*(X/Z) + cx, v = fy*(Y/Z) + cy, floor; keep iff
 *                     Z > z_near and the pixel lies in the image padded by h;
 *                     key = (floor(v)+h)*(W+2h) + (floor(u)+h)
 *   D3 ray            nx = ((u+0.5)-cx)/fx, ny = ((v+0.5)-cy)/fy,
 *                     q = nx*nx + ny*ny, n2 = q + 1, len = sqrtf(n2),
 *                     d = (nx/len, ny/len, 1/len); origin = camera centre
 *   D4 radius         fixed: r(t) = r; cone (Eq. radius, f = 1 plane):
 *                     g = sqrtf(q) - rdd, c = rdd/(len*sqrtf(g*g + 1));
 *                     cone approx (Eq. r_approx2): c = rdd/n2; r(t) = t*c
 *   D5 accept         t = (X*dx + Y*dy) + Z*dz;  e = fmaf(-t, d, P) per axis;
 *                     rho2 = (ex*ex + ey*ey) + ez*ez;
 *                     accept iff t_near <= t <= t_far and rho2 <= r(t)*r(t)
 *   D6 candidate order ascending (t, point id)
 *   D7 distance       a = fmaf(t_j, d, -P) per axis, dist2 = (ax*ax + ay*ay) + az*az,
 *                     dist = sqrtf(dist2)
 *   D8 pseudo-UDF     N_j = the candidates with dist2 <= r(t_j)*r(t_j) ("points within
 *                     its radius", Fig. 3), the K' = min(K, |.|) first by (dist2, id);
 *                     s = dist_1, s = s + dist_2, ...; d_j = s / K'.  N_j always holds
 *                     the candidate's own point (its dist2 is its D5 rho2).
 *   D9 confidence     alpha_j = gamma * exp32(-((d_j*d_j)/beta2))
 *   D10 weight        w_j = alpha_j * T_j,  T_1 = 1,  T_{j+1} = T_j * (1 - alpha_j)
 *   D11 primary       j* = first j with w_j > eps_w; the cluster runs on while
 *                     (t_{j+1} - t_j) <= gap_k * r(t_j); samples are its members
 *                     with w_j > eps_w, in order, at most n.  gap_k = 0 drops the
 *                     cluster gate: every candidate from j* on with w_j > eps_w
 *                     (the gamma-controlled move towards multi-surface sampling)
 *   D12 restricted    (learned-interval search) per-ray depth range [tn, tf] =
 *       search        [max(t_near, t0), min(t_far, t1)]; fixed radius: window
 *                     zlo = max((tn*cos_m) - (r*sin_m), z_near),
 *                     lim = ((win/zlo)*1.001) + 0.001, hr = floor(lim + 0.5) if lim < h
 *                     (cos_m, sin_m, win: float of the double image-corner terms);
 *                     candidates: accepted (D5) with t in [tn, tf] inside the hr
 *                     window; it falls back to the plain search when it keeps no
 *                     sample (and the full window is not empty), when D5 accepts
 *                     a point with t < tn, or when the selection ran out of
 *                     candidates (no gap / n / gamma*T <= eps_w stop) while D5
 *                     accepts a point with t > tf -- unless a sample was kept,
 *                     gap_k > 0 and (tf - t_last) > max(gap_k, 1) * r(t_last)
 *                     for the last restricted candidate t_last
 *   exp32             Cody & Waite range reduction (two-part ln 2) and a
 *                     degree-7 Taylor polynomial in Horner form, scaled by 2^k
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    float t_near, t_far, z_near;
} or_camera;

typedef struct {
    int32_t radius_mode;   /* 0 fixed, 1 cone (Eq. radius), 2 cone approx (Eq. r_approx2) */
    float r;               /* fixed radius; cone modes: r_min at t_near when rho <= 0 */
    float rho;             /* r_ddot / r_dot for the cone modes */
    float gamma, beta2, eps_w, gap_k, eps_d;
    int32_t cand_cap, K, n_max, bg_mode, window_h;
} or_params;

#define OR_HMAX 64

/* ------------------------------------------------------------------ exp32 */

static float bits_float(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }

/* exp(x) in binary32 for the decisions (D9).  Cody & Waite: x = k ln2 + r with
 * ln2 split as LN2_HI + LN2_LO where LN2_HI keeps 16 significant bits (so that
 * k*LN2_HI is exact for |k| < 256); exp(r) by the Taylor series to degree 7
 * (|r| <= ln2/2, truncation < 6e-9 relative); scale by 2^k built from the
 * exponent bits. */
float or_exp32(float x)
{
    const float L2E = (float)(1.0 / 0.69314718055994530942);
    const float LN2_HI = (float)(45426.0 / 65536.0);            /* floor(ln2 * 2^16) / 2^16 */
    const float LN2_LO = (float)(0.69314718055994530942 - 45426.0 / 65536.0);
    const float C2 = (float)(1.0 / 2.0), C3 = (float)(1.0 / 6.0), C4 = (float)(1.0 / 24.0);
    const float C5 = (float)(1.0 / 120.0), C6 = (float)(1.0 / 720.0), C7 = (float)(1.0 / 5040.0);
    if (x != x) return x;
    if (x < -104.0f) return 0.0f;
    if (x > 88.5f) return INFINITY;
    float kf = rintf(x * L2E);
    float r = (x - kf * LN2_HI) - kf * LN2_LO;
    float p = C7;
    p = p * r + C6;
    p = p * r + C5;
    p = p * r + C4;
    p = p * r + C3;
    p = p * r + C2;
    p = p * r + 1.0f;
    p = p * r + 1.0f;
    int k = (int)kf;
    if (k >= -126) return p * bits_float((uint32_t)(k + 127) << 23);
    return (p * bits_float((uint32_t)(k + 100 + 127) << 23)) * bits_float((uint32_t)(127 - 100) << 23);
}

/* --------------------------------------------------------- camera helpers */

/* D1 */
void or_cam_point(const or_camera *c, const float *p, float *out)
{
    float px = p[0], py = p[1], pz = p[2];
    out[0] = ((c->R[0] * px + c->R[1] * py) + c->R[2] * pz) + c->t[0];
    out[1] = ((c->R[3] * px + c->R[4] * py) + c->R[5] * pz) + c->t[1];
    out[2] = ((c->R[6] * px + c->R[7] * py) + c->R[8] * pz) + c->t[2];
}

/* D1 for N points (out: N x 3). */
void or_cam_points(const or_camera *c, const float *p, int64_t N, float *out)
{
    for (int64_t i = 0; i < N; ++i) or_cam_point(c, p + 3 * i, out + 3 * i);
}

/* D2: returns 1 and the padded key if the point is kept. */
static int project_key(const or_camera *c, int h, const float *X, uint32_t *key)
{
    float Z = X[2];
    if (!(Z > c->z_near)) return 0;
    float u = c->fx * (X[0] / Z) + c->cx;
    float v = c->fy * (X[1] / Z) + c->cy;
    float fu = floorf(u), fv = floorf(v);
    if (!(fu >= (float)(-h) && fu < (float)(c->width + h) && fv >= (float)(-h) && fv < (float)(c->height + h)))
        return 0;
    uint32_t iu = (uint32_t)((int)fu + h), iv = (uint32_t)((int)fv + h);
    *key = iv * (uint32_t)(c->width + 2 * h) + iu;
    return 1;
}

typedef struct {
    float d[3];
    float q, n2, len;
    float c;        /* cone coefficient, r(t) = t*c */
} ray_t;

/* D3 + D4 */
static void make_ray(const or_camera *c, const or_params *p, float rdd, int pu, int pv, ray_t *ray)
{
    float nx = (((float)pu + 0.5f) - c->cx) / c->fx;
    float ny = (((float)pv + 0.5f) - c->cy) / c->fy;
    float q = nx * nx + ny * ny;
    float n2 = q + 1.0f;
    float len = sqrtf(n2);
    ray->d[0] = nx / len;
    ray->d[1] = ny / len;
    ray->d[2] = 1.0f / len;
    ray->q = q;
    ray->n2 = n2;
    ray->len = len;
    ray->c = 0.0f;
    if (p->radius_mode == 1) {
        float g = sqrtf(q) - rdd;
        ray->c = rdd / (len * sqrtf(g * g + 1.0f));
    } else if (p->radius_mode == 2) {
        ray->c = rdd / n2;
    }
}

static float radius_at(const or_params *p, const ray_t *ray, float t)
{
    return p->radius_mode == 0 ? p->r : t * ray->c;
}

/* D5: returns 1 and t when the camera-space point P is accepted (depth
 * range [tn, tf], normally [t_near, t_far]). */
static int accept_point(const or_params *p, const ray_t *ray, const float *P, float tn, float tf, float *t_out)
{
    const float *d = ray->d;
    float t = (P[0] * d[0] + P[1] * d[1]) + P[2] * d[2];
    if (!(t >= tn && t <= tf)) return 0;
    float ex = fmaf(-t, d[0], P[0]);
    float ey = fmaf(-t, d[1], P[1]);
    float ez = fmaf(-t, d[2], P[2]);
    float rho2 = (ex * ex + ey * ey) + ez * ez;
    float rad = radius_at(p, ray, t);
    if (!(rho2 <= rad * rad)) return 0;
    *t_out = t;
    return 1;
}

/* ------------------------------------------------------ window half-width
 * A point accepted by D5 lies at t >= t_near within r(t) of the ray.  Writing
 * it as t*d + e with e orthogonal to d, its image-plane offset from the ray's
 * pixel centre is (e_x d_z - d_x e_z)/(Z d_z) <= |e| sqrt(1+nx^2)/Z and its
 * depth is Z >= t d_z - |e| sin(theta).  Bounding both over the image gives the
 * largest pixel offset L; a point whose projection is L pixels from a pixel
 * centre falls at most floor(L + 1/2) pixels away.  In the cone modes the
 * paper's kernel size s = 2*ceil(r_ddot/r_dot)+1 is kept when it is larger.
 * Returns 0, or a negative code for an unusable camera. */
int or_window(const or_camera *c, const or_params *p, int32_t *h_out, float *rdd_out)
{
    if (c->width <= 0 || c->height <= 0 || !(c->fx > 0) || !(c->fy > 0)) return -1;
    if (!(c->t_near > 0) || !(c->t_far >= c->t_near) || !(c->z_near > 0)) return -1;
    double fx = c->fx, fy = c->fy, cx = c->cx, cy = c->cy;
    double ax = fmax(fabs(0.5 - cx), fabs(((double)c->width - 0.5) - cx)) / fx;
    double ay = fmax(fabs(0.5 - cy), fabs(((double)c->height - 0.5) - cy)) / fy;
    double q = ax * ax + ay * ay;
    double cosm = 1.0 / sqrt(1.0 + q);
    double sinm = sqrt(q / (1.0 + q));
    double lim_x, lim_y, rdd = 0.0, rho = 0.0;
    if (p->radius_mode == 0) {
        double r = p->r;
        if (!(r > 0)) return -1;
        double zlo = (double)c->t_near * cosm - r * sinm;
        if (zlo < (double)c->z_near) zlo = (double)c->z_near;
        lim_x = fx * r * sqrt(1.0 + ax * ax) / zlo;
        lim_y = fy * r * sqrt(1.0 + ay * ay) / zlo;
    } else if (p->radius_mode == 1 || p->radius_mode == 2) {
        double rdot = sqrt(1.0 / ((3.14159265358979323846 * fx) * fy));
        if (p->rho > 0) {
            rho = p->rho;
            rdd = rho * rdot;
        } else {
            /* r_min at t_near equals the given radius on the central ray (Sec. 3.2) */
            double r = p->r, tn = c->t_near;
            if (!(r > 0) || !(tn > r)) return -1;
            rdd = (p->radius_mode == 1) ? r / sqrt(tn * tn - r * r) : r / tn;
            rho = rdd / rdot;
        }
        double den = cosm - rdd * sinm;
        if (!(den > 0)) return -2;
        lim_x = fx * rdd * sqrt(1.0 + ax * ax) / den;
        lim_y = fy * rdd * sqrt(1.0 + ay * ay) / den;
    } else {
        return -1;
    }
    double lim = fmax(lim_x, lim_y) * (1.0 + 1e-3) + 1e-3;
    if (!(lim < (double)OR_HMAX)) return -3;
    int h = (int)floor(lim + 0.5);
    if (p->radius_mode != 0) {
        int hp = (int)ceil(rho);
        if (hp > h) h = hp;
    }
    if (p->window_h > 0) h = p->window_h;
    if (h > OR_HMAX) return -3;
    *h_out = h;
    *rdd_out = (float)rdd;
    return 0;
}

/* ----------------------------------------------------------- table build */

typedef struct {
    uint32_t key;
    float X, Y, Z;
    int32_t id;
} rec_t;

static int cmp_rec(const void *a_, const void *b_)
{
    const rec_t *a = (const rec_t *)a_, *b = (const rec_t *)b_;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->Z != b->Z) return a->Z < b->Z ? -1 : 1;
    if (a->X != b->X) return a->X < b->X ? -1 : 1;
    if (a->Y != b->Y) return a->Y < b->Y ? -1 : 1;
    return (a->id > b->id) - (a->id < b->id);
}

/* The pixel-keyed table of Sec. 3.2: every kept point, grouped by pixel key
 * (bucket), each bucket ordered by (depth, x, y, id); start[k] is the first
 * position of bucket k in the list and start[k+1]-start[k] its count.
 * Outputs: start[(W+2h)(H+2h)+1], ids[N_v], pos[3 N_v] (camera space, D1).
 * Returns N_v, or -1 when out of memory. */
int64_t or_build_table(const float *pts, int64_t N, const or_camera *c, int32_t h,
                       uint32_t *start, int32_t *ids, float *pos)
{
    int64_t Wp = c->width + 2 * h, Hp = c->height + 2 * h, P = Wp * Hp;
    rec_t *rec = (rec_t *)malloc(sizeof(rec_t) * (size_t)(N > 0 ? N : 1));
    if (!rec) return -1;
    int64_t nv = 0;
    for (int64_t i = 0; i < N; ++i) {
        float X[3];
        uint32_t key;
        or_cam_point(c, pts + 3 * i, X);
        if (!project_key(c, h, X, &key)) continue;
        rec[nv].key = key;
        rec[nv].X = X[0];
        rec[nv].Y = X[1];
        rec[nv].Z = X[2];
        rec[nv].id = (int32_t)i;
        ++nv;
    }
    qsort(rec, (size_t)nv, sizeof(rec_t), cmp_rec);
    for (int64_t k = 0; k <= P; ++k) start[k] = 0;
    for (int64_t i = 0; i < nv; ++i) start[rec[i].key + 1] += 1;
    for (int64_t k = 0; k < P; ++k) start[k + 1] += start[k];
    for (int64_t i = 0; i < nv; ++i) {
        ids[i] = rec[i].id;
        pos[3 * i + 0] = rec[i].X;
        pos[3 * i + 1] = rec[i].Y;
        pos[3 * i + 2] = rec[i].Z;
    }
    free(rec);
    return nv;
}

/* ----------------------------------------------------------------- search */

typedef struct {
    float t;
    int32_t id;
    float P[3];
} cand_t;

static int cmp_cand(const void *a_, const void *b_)
{
    const cand_t *a = (const cand_t *)a_, *b = (const cand_t *)b_;
    if (a->t != b->t) return a->t < b->t ? -1 : 1;
    return (a->id > b->id) - (a->id < b->id);
}

typedef struct {
    const float *pts;
    int64_t N;
    const or_camera *cam;
    const or_params *prm;
    int32_t h;
    float rdd;
    const uint32_t *start;
    const int32_t *ids;
    const float *pos;
} frame_t;

/* All accepted points of one ray, sorted by (t, id) (D5, D6).  brute != 0
 * tests every input point (the brute-force search of Sec. 3.5); otherwise the
 * s x s window of buckets around the ray's pixel is walked and empty buckets
 * are skipped (Sec. 3.2).  Returns the count; *out is malloc'ed. */
static int64_t ray_candidates_w(const frame_t *f, const ray_t *ray, int pu, int pv, int brute, float tn, float tf,
                                int hr, int *early, int *late, cand_t **out);

static int64_t ray_candidates(const frame_t *f, const ray_t *ray, int pu, int pv, int brute, float tn, float tf,
                              cand_t **out)
{
    return ray_candidates_w(f, ray, pu, pv, brute, tn, tf, f->h, NULL, NULL, out);
}

/* As ray_candidates, over the window of half-width hr <= h; early / late (if
 * given) report points the plain range [t_near, t_far] accepts with t < tn /
 * t > tf. */
static int64_t ray_candidates_w(const frame_t *f, const ray_t *ray, int pu, int pv, int brute, float tn, float tf,
                                int hr, int *early, int *late, cand_t **out)
{
    int64_t cap = 64, n = 0;
    cand_t *cs = (cand_t *)malloc(sizeof(cand_t) * (size_t)cap);
    float t;
    if (brute) {
        for (int64_t i = 0; i < f->N; ++i) {
            float X[3];
            or_cam_point(f->cam, f->pts + 3 * i, X);
            if (!(X[2] > f->cam->z_near)) continue;
            if (!accept_point(f->prm, ray, X, tn, tf, &t)) continue;
            if (n == cap) { cap *= 2; cs = (cand_t *)realloc(cs, sizeof(cand_t) * (size_t)cap); }
            cs[n].t = t; cs[n].id = (int32_t)i;
            cs[n].P[0] = X[0]; cs[n].P[1] = X[1]; cs[n].P[2] = X[2];
            ++n;
        }
    } else {
        int h = f->h, off = h - hr;
        int64_t Wp = f->cam->width + 2 * h;
        for (int dy = 0; dy <= 2 * hr; ++dy) {
            for (int dx = 0; dx <= 2 * hr; ++dx) {
                /* pixel (pu-hr+dx, pv-hr+dy) has padded key (pv+off+dy)*Wp + (pu+off+dx) */
                int64_t k = (int64_t)(pv + off + dy) * Wp + (pu + off + dx);
                uint32_t a = f->start[k], b = f->start[k + 1];
                if (a == b) continue;     /* count check: nothing to test */
                for (uint32_t i = a; i < b; ++i) {
                    const float *X = f->pos + 3 * (int64_t)i;
                    if (early || late) {
                        float tp;
                        if (accept_point(f->prm, ray, X, f->cam->t_near, f->cam->t_far, &tp)) {
                            if (tp < tn && early) *early = 1;
                            if (tp > tf && late) *late = 1;
                        }
                    }
                    if (!accept_point(f->prm, ray, X, tn, tf, &t)) continue;
                    if (n == cap) { cap *= 2; cs = (cand_t *)realloc(cs, sizeof(cand_t) * (size_t)cap); }
                    cs[n].t = t; cs[n].id = f->ids[i];
                    cs[n].P[0] = X[0]; cs[n].P[1] = X[1]; cs[n].P[2] = X[2];
                    ++n;
                }
            }
        }
    }
    qsort(cs, (size_t)n, sizeof(cand_t), cmp_cand);
    *out = cs;
    return n;
}

/* D12: image-corner terms of the restricted window -- cos and sin of the
 * largest angle between a pixel-centre ray and the optical axis, and the
 * window's projected radius scale (float of double). */
static void d12_terms(const or_camera *cam, const or_params *prm, float *rcos, float *rsin, float *rwin)
{
    double fx = cam->fx, fy = cam->fy, cx = cam->cx, cy = cam->cy;
    double ax = fmax(fabs(0.5 - cx), fabs(((double)cam->width - 0.5) - cx)) / fx;
    double ay = fmax(fabs(0.5 - cy), fabs(((double)cam->height - 0.5) - cy)) / fy;
    double q = ax * ax + ay * ay;
    double rr = prm->r;
    *rcos = (float)(1.0 / sqrt(1.0 + q));
    *rsin = (float)sqrt(q / (1.0 + q));
    *rwin = (float)fmax(fx * rr * sqrt(1.0 + ax * ax), fy * rr * sqrt(1.0 + ay * ay));
}

/* D12: half-width of the window a ray restricted to depths t >= tn walks
 * (fixed radius; the cone modes keep h): zlo = max(tn cos - r sin, z_near),
 * lim = (win / zlo) 1.001 + 0.001, hr = min(h, floor(lim + 0.5)) when lim < h. */
static int d12_window(const or_camera *cam, const or_params *prm, int h, float tn, float rcos, float rsin, float rwin)
{
    int hr = h;
    if (prm->radius_mode == 0) {
        float zlo = tn * rcos - prm->r * rsin;
        if (!(zlo >= cam->z_near)) zlo = cam->z_near;
        float lim = (rwin / zlo) * 1.001f + 1e-3f;
        if (lim < (float)h) { int q = (int)floorf(lim + 0.5f); hr = q < h ? q : h; }
    }
    return hr;
}

/* ------------------------------------------------------------- selection */

typedef struct {
    float dist2;
    int32_t id;
} nd_t;

static int cmp_nd(const void *a_, const void *b_)
{
    const nd_t *a = (const nd_t *)a_, *b = (const nd_t *)b_;
    if (a->dist2 != b->dist2) return a->dist2 < b->dist2 ? -1 : 1;
    return (a->id > b->id) - (a->id < b->id);
}

typedef struct {
    int32_t n_s;
    int32_t primary;         /* padded key of the source point of j*, or -1 */
    int32_t cand_count;      /* accepted points before the capacity cut */
    float t[64];
    int32_t src[64];
    int32_t *nbr;            /* n_max * K */
    float *ndist;            /* n_max * K */
} ray_result_t;

/* Adaptive primary surface sampling (Sec. 3.3) for one ray, candidates in
 * (t, id) order.  For each candidate x_j = o + t_j d, the K nearest candidate
 * points within r(t_j) of x_j give the pseudo-UDF d_j (mean distance), alpha_j = gamma
 * exp(-d_j^2/beta^2), w_j = alpha_j prod_{k<j}(1-alpha_k) (Eq. weight); the
 * samples are the primary cluster's candidates with w_j > eps_w. */
static void select_samples(const frame_t *f, const ray_t *ray, const cand_t *cs, int64_t C, int32_t K,
                           int32_t n_max, ray_result_t *res, float *d_out, float *w_out, int *stopped)
{
    const or_params *p = f->prm;
    nd_t *nd = (nd_t *)malloc(sizeof(nd_t) * (size_t)(C > 0 ? C : 1));
    float *w = (float *)malloc(sizeof(float) * (size_t)(C > 0 ? C : 1));
    int32_t *knn = (int32_t *)malloc(sizeof(int32_t) * (size_t)(C > 0 ? C : 1) * (size_t)K);
    float *tafter = (float *)malloc(sizeof(float) * (size_t)(C > 0 ? C : 1));
    float *kd = (float *)malloc(sizeof(float) * (size_t)(C > 0 ? C : 1) * (size_t)K);
    float T = 1.0f;
    for (int64_t j = 0; j < C; ++j) {
        float tj = cs[j].t;
        float rad = radius_at(p, ray, tj);
        float rad2 = rad * rad;
        for (int64_t i = 0; i < C; ++i) {
            float ax = fmaf(tj, ray->d[0], -cs[i].P[0]);
            float ay = fmaf(tj, ray->d[1], -cs[i].P[1]);
            float az = fmaf(tj, ray->d[2], -cs[i].P[2]);
            nd[i].dist2 = (ax * ax + ay * ay) + az * az;
            nd[i].id = cs[i].id;
        }
        qsort(nd, (size_t)C, sizeof(nd_t), cmp_nd);
        int64_t Kp = 0;
        while (Kp < K && Kp < C && nd[Kp].dist2 <= rad2) ++Kp;
        float s = 0.0f;
        for (int64_t m = 0; m < Kp; ++m) {
            float dist = sqrtf(nd[m].dist2);
            s = s + dist;
            knn[j * K + m] = nd[m].id;
            kd[j * K + m] = dist;
        }
        for (int64_t m = Kp; m < K; ++m) { knn[j * K + m] = -1; kd[j * K + m] = 0.0f; }
        float dj = s / (float)Kp;
        float alpha = p->gamma * or_exp32(-((dj * dj) / p->beta2));
        w[j] = alpha * T;
        if (d_out) d_out[j] = dj;
        if (w_out) w_out[j] = w[j];
        T = T * (1.0f - alpha);
        tafter[j] = T;                 /* T after candidate j */
    }
    res->n_s = 0;
    res->primary = -1;
    int64_t jstar = -1;
    for (int64_t j = 0; j < C; ++j) {
        if (w[j] > p->eps_w) { jstar = j; break; }
    }
    if (jstar >= 0) {
        uint32_t key = 0;
        project_key(f->cam, f->h, cs[jstar].P, &key);
        res->primary = (int32_t)key;
        for (int64_t j = jstar; j < C && res->n_s < n_max; ++j) {
            if (j > jstar && p->gap_k > 0.0f) {
                float gap = cs[j].t - cs[j - 1].t;
                if (!(gap <= p->gap_k * radius_at(p, ray, cs[j - 1].t))) break;
            }
            if (w[j] > p->eps_w) {
                int m = res->n_s++;
                res->t[m] = cs[j].t;
                res->src[m] = cs[j].id;
                memcpy(res->nbr + (int64_t)m * K, knn + j * K, sizeof(int32_t) * (size_t)K);
                memcpy(res->ndist + (int64_t)m * K, kd + j * K, sizeof(float) * (size_t)K);
            }
        }
    }
    /* did the depth-ordered selection stop (gap after j*, n samples, or
     * gamma * T_j <= eps_w so that no later weight can pass) before running
     * out of candidates? */
    if (stopped) {
        *stopped = 0;
        int64_t js = -1;
        int32_t ns = 0;
        for (int64_t j = 0; j < C && !*stopped; ++j) {
            if (js >= 0 && p->gap_k > 0.0f) {
                float gap = cs[j].t - cs[j - 1].t;
                if (!(gap <= p->gap_k * radius_at(p, ray, cs[j - 1].t))) { *stopped = 1; break; }
            }
            if (w[j] > p->eps_w) {
                if (js < 0) js = j;
                if (++ns == n_max) { *stopped = 1; break; }
            }
            if (!(p->gamma * tafter[j] > p->eps_w)) *stopped = 1;
        }
    }
    free(nd);
    free(w);
    free(knn);
    free(kd);
    free(tafter);
}

/* ------------------------------------------- aggregation, decode, composite */

static double softplus_d(double x) { return x > 0 ? x + log1p(exp(-x)) : log1p(exp(x)); }
static double sigmoid_d(double x) { return 1.0 / (1.0 + exp(-x)); }

/* MLP y = W_L(...relu(W_1 x + b_1)...) + b_L in double; params packed
 * W0 (dims[1] x dims[0], row-major), b0, W1, b1, ... */
void or_mlp(const int32_t *dims, int32_t n_layers, const float *params, const double *x, double *y)
{
    double a[1024], b[1024];
    int32_t width = dims[0];
    for (int32_t i = 0; i < width; ++i) a[i] = x[i];
    const float *P = params;
    for (int32_t l = 0; l < n_layers; ++l) {
        int32_t fi = dims[l], fo = dims[l + 1];
        const float *W = P, *bias = P + (int64_t)fi * fo;
        for (int32_t o = 0; o < fo; ++o) {
            double acc = (double)bias[o];
            for (int32_t i = 0; i < fi; ++i) acc += (double)W[(int64_t)o * fi + i] * a[i];
            b[o] = (l + 1 < n_layers && acc < 0.0) ? 0.0 : acc;
        }
        for (int32_t o = 0; o < fo; ++o) a[o] = b[o];
        P += (int64_t)fi * fo + fo;
    }
    for (int32_t o = 0; o < dims[n_layers]; ++o) y[o] = a[o];
}

/* Sec. 3.4 integration for one ray: features of each sample's K' neighbours
 * blended by inverse distance (weights 1/max(dist, eps_d)), decoded by the
 * MLP into density sigma = softplus(o0) and colour sigmoid(o1..3), then
 * volume rendered with Eq. 2: tau_j = exp(-sum_{k<j} sigma_k Delta_k),
 * c = sum_j tau_j (1 - exp(-sigma_j Delta_j)) c_j, Delta_j = t_{j+1} - t_j and
 * 2 r(t) for the last sample; background weight 1 - sum.  Optional per-sample
 * outputs: feat (n_s x F), out4 (n_s x 4: sigma, r, g, b). */
static void shade_ray(const frame_t *f, const ray_t *ray, const float *feats, int32_t F, const int32_t *dims,
                      int32_t n_layers, const float *mlp, int32_t K, int32_t n_s, const float *ts,
                      const int32_t *nbr, double *rgb, double *wsum, double *feat_out, double *out4)
{
    const or_params *p = f->prm;
    double T = 1.0, ws = 0.0, c3[3] = {0, 0, 0};
    double fe[1024], o[8];
    for (int32_t j = 0; j < n_s; ++j) {
        double x[3];
        for (int a = 0; a < 3; ++a) x[a] = (double)ts[j] * (double)ray->d[a];
        double wsum_i = 0.0;
        for (int32_t k = 0; k < F; ++k) fe[k] = 0.0;
        for (int32_t m = 0; m < K; ++m) {
            int32_t id = nbr[(int64_t)j * K + m];
            if (id < 0) continue;
            float P[3];
            or_cam_point(f->cam, f->pts + 3 * (int64_t)id, P);
            double dx = x[0] - P[0], dy = x[1] - P[1], dz = x[2] - P[2];
            double dist = sqrt(dx * dx + dy * dy + dz * dz);
            double wi = 1.0 / (dist > p->eps_d ? dist : (double)p->eps_d);
            wsum_i += wi;
            for (int32_t k = 0; k < F; ++k) fe[k] += wi * (double)feats[(int64_t)id * F + k];
        }
        for (int32_t k = 0; k < F; ++k) fe[k] /= wsum_i;
        or_mlp(dims, n_layers, mlp, fe, o);
        double sigma = softplus_d(o[0]);
        double col[3] = {sigmoid_d(o[1]), sigmoid_d(o[2]), sigmoid_d(o[3])};
        if (feat_out) for (int32_t k = 0; k < F; ++k) feat_out[(int64_t)j * F + k] = fe[k];
        if (out4) { out4[4 * j] = sigma; for (int a = 0; a < 3; ++a) out4[4 * j + 1 + a] = col[a]; }
        double delta = (j + 1 < n_s) ? (double)ts[j + 1] - (double)ts[j]
                                     : 2.0 * (p->radius_mode == 0 ? (double)p->r : (double)ts[j] * (double)ray->c);
        double a = -expm1(-sigma * delta);
        double wj = T * a;
        for (int c = 0; c < 3; ++c) c3[c] += wj * col[c];
        ws += wj;
        T *= exp(-sigma * delta);
    }
    double bg = p->bg_mode == 1 ? 1.0 : 0.0;
    for (int c = 0; c < 3; ++c) rgb[c] = c3[c] + (1.0 - ws) * bg;
    *wsum = ws;
}

/* ------------------------------------------------------------ full frame */

typedef struct {
    int32_t n_s, primary, cand_count;
} ray_head_t;

/* The whole hot path for R rays (rays = pixel ids v*W+u, or NULL for all
 * W*H pixels in row-major order).  Sample outputs are packed ray by ray
 * (sample_offset[R+1]); per-sample arrays need capacity R*n_max.
 * brute != 0 replaces the window walk with brute force.  nthreads > 1 runs
 * rays in parallel (OpenMP).  Returns the sample count S, or a negative
 * error: -1 bad arguments, -2 out of memory, -3 a ray pixel out of range. */
int64_t or_render(const float *pts, int64_t N, const float *feats, int32_t F, const or_camera *cam,
                  const or_params *prm, const int32_t *dims, int32_t n_layers, const float *mlp,
                  const int32_t *rays, int64_t R, const float *intervals, int32_t brute, int32_t nthreads,
                  int32_t *n_s, int32_t *primary, int32_t *cand_count, int64_t *sample_offset,
                  float *s_t, int32_t *s_ray, int32_t *s_src, int32_t *s_nbr, float *s_dist,
                  double *rgb, double *wsum, double *s_feat, double *s_out4)
{
    int32_t h;
    float rdd;
    if (or_window(cam, prm, &h, &rdd) != 0) return -1;
    const int32_t K = prm->K, n_max = prm->n_max;
    if (K < 1 || K > 64 || n_max < 1 || n_max > 64 || prm->cand_cap < 1) return -1;
    if (F < 1 || F > 1024 || n_layers < 1 || dims[0] != F || dims[n_layers] != 4) return -1;
    int64_t W = cam->width, H = cam->height;
    if (!rays) R = W * H;
    int64_t P = (W + 2 * h) * (H + 2 * h);
    uint32_t *start = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(P + 1));
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    float *pos = (float *)malloc(sizeof(float) * 3 * (size_t)(N > 0 ? N : 1));
    ray_head_t *head = (ray_head_t *)malloc(sizeof(ray_head_t) * (size_t)(R > 0 ? R : 1));
    float *st = (float *)malloc(sizeof(float) * (size_t)(R > 0 ? R : 1) * n_max);
    int32_t *ssrc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(R > 0 ? R : 1) * n_max);
    int32_t *snbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(R > 0 ? R : 1) * n_max * K);
    float *sdist = (float *)malloc(sizeof(float) * (size_t)(R > 0 ? R : 1) * n_max * K);
    if (!start || !ids || !pos || !head || !st || !ssrc || !snbr || !sdist) return -2;
    if (!brute && or_build_table(pts, N, cam, h, start, ids, pos) < 0) return -2;
    frame_t fr = {pts, N, cam, prm, h, rdd, start, ids, pos};
    /* D12 image-corner terms of the restricted window (float of double) */
    float rcos, rsin, rwin;
    d12_terms(cam, prm, &rcos, &rsin, &rwin);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads > 0 ? nthreads : 1) reduction(| : bad)
    for (int64_t i = 0; i < R; ++i) {
        int64_t pix = rays ? rays[i] : i;
        if (pix < 0 || pix >= W * H) { bad = 1; head[i].n_s = 0; head[i].primary = -1; head[i].cand_count = 0; continue; }
        int pu = (int)(pix % W), pv = (int)(pix / W);
        ray_t ray;
        make_ray(cam, prm, rdd, pu, pv, &ray);
        cand_t *cs;
        ray_result_t res;
        res.nbr = snbr + i * n_max * K;
        res.ndist = sdist + i * n_max * K;
        int64_t C = 0;
        int fallback = 1;
        if (intervals) {
            /* restricted to the ray's interval (D12); fall back to the plain search on a miss */
            float tn = intervals[2 * i] > cam->t_near ? intervals[2 * i] : cam->t_near;
            float tf = intervals[2 * i + 1] < cam->t_far ? intervals[2 * i + 1] : cam->t_far;
            int hr = d12_window(cam, prm, h, tn, rcos, rsin, rwin);
            int early = 0, late = 0, stopped = 0;
            C = ray_candidates_w(&fr, &ray, pu, pv, brute, tn, tf, hr, &early, &late, &cs);
            int64_t Ck = C < prm->cand_cap ? C : prm->cand_cap;
            select_samples(&fr, &ray, cs, Ck, K, n_max, &res, NULL, NULL, &stopped);
            int full_empty = 1;
            for (int dy = 0; dy <= 2 * h && full_empty; ++dy) {
                int64_t kb = (int64_t)(pv + dy) * (W + 2 * h) + pu;
                if (start[kb + 2 * h + 1] != start[kb]) full_empty = 0;
            }
            int late_ok = 0;
            if (res.n_s > 0 && prm->gap_k > 0.0f && Ck > 0) {
                float tl = cs[Ck - 1].t;
                float g = prm->gap_k > 1.0f ? prm->gap_k : 1.0f;
                late_ok = (tf - tl) > g * radius_at(prm, &ray, tl);
            }
            fallback = (res.n_s == 0 && !full_empty) || early || (!stopped && late && !late_ok);
            if (fallback) { free(cs); cs = NULL; }
        }
        if (fallback) {
            C = ray_candidates(&fr, &ray, pu, pv, brute, cam->t_near, cam->t_far, &cs);
            int64_t Ck = C < prm->cand_cap ? C : prm->cand_cap;   /* keep the cand_cap smallest (t, id) */
            select_samples(&fr, &ray, cs, Ck, K, n_max, &res, NULL, NULL, NULL);
        }
        res.cand_count = (int32_t)C;
        head[i].n_s = res.n_s;
        head[i].primary = res.primary;
        head[i].cand_count = res.cand_count;
        memcpy(st + i * n_max, res.t, sizeof(float) * (size_t)res.n_s);
        memcpy(ssrc + i * n_max, res.src, sizeof(int32_t) * (size_t)res.n_s);
        free(cs);
        shade_ray(&fr, &ray, feats, F, dims, n_layers, mlp, K, res.n_s, st + i * n_max, snbr + i * n_max * K,
                  rgb + 3 * i, wsum + i, NULL, NULL);
    }
    /* pack samples ray by ray */
    int64_t S = 0;
    for (int64_t i = 0; i < R; ++i) {
        sample_offset[i] = S;
        n_s[i] = head[i].n_s;
        primary[i] = head[i].primary;
        cand_count[i] = head[i].cand_count;
        for (int32_t m = 0; m < head[i].n_s; ++m, ++S) {
            s_t[S] = st[i * n_max + m];
            s_ray[S] = (int32_t)i;
            s_src[S] = ssrc[i * n_max + m];
            memcpy(s_nbr + S * K, snbr + (i * n_max + m) * K, sizeof(int32_t) * (size_t)K);
            memcpy(s_dist + S * K, sdist + (i * n_max + m) * K, sizeof(float) * (size_t)K);
        }
    }
    sample_offset[R] = S;
    /* optional per-sample diagnostics: recompute the continuous stages per sample */
    if (s_feat || s_out4) {
        for (int64_t i = 0; i < R; ++i) {
            int64_t pix = rays ? rays[i] : i;
            if (pix < 0 || pix >= W * H || head[i].n_s == 0) continue;
            ray_t ray;
            double c3[3], ws;
            make_ray(cam, prm, rdd, (int)(pix % W), (int)(pix / W), &ray);
            int64_t o = sample_offset[i];
            shade_ray(&fr, &ray, feats, F, dims, n_layers, mlp, K, head[i].n_s, s_t + o, s_nbr + o * K, c3, &ws,
                      s_feat ? s_feat + o * F : NULL, s_out4 ? s_out4 + o * 4 : NULL);
        }
    }
    free(start); free(ids); free(pos); free(head); free(st); free(ssrc); free(snbr); free(sdist);
    return bad ? -3 : S;
}

/* Candidate list of a single ray (for search tests): returns the number of
 * accepted points and writes the first min(count, cap) by (t, id). */
int64_t or_ray_candidates(const float *pts, int64_t N, const or_camera *cam, const or_params *prm,
                          int32_t pixel, int32_t brute, int32_t cap, int32_t *cid, float *ct)
{
    int32_t h;
    float rdd;
    if (or_window(cam, prm, &h, &rdd) != 0) return -1;
    int64_t W = cam->width, H = cam->height;
    if (pixel < 0 || pixel >= W * H) return -3;
    int64_t P = (W + 2 * h) * (H + 2 * h);
    uint32_t *start = NULL;
    int32_t *ids = NULL;
    float *pos = NULL;
    if (!brute) {
        start = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(P + 1));
        ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
        pos = (float *)malloc(sizeof(float) * 3 * (size_t)(N > 0 ? N : 1));
        or_build_table(pts, N, cam, h, start, ids, pos);
    }
    frame_t fr = {pts, N, cam, prm, h, rdd, start, ids, pos};
    ray_t ray;
    make_ray(cam, prm, rdd, (int)(pixel % W), (int)(pixel / W), &ray);
    cand_t *cs;
    int64_t C = ray_candidates(&fr, &ray, (int)(pixel % W), (int)(pixel / W), brute, cam->t_near, cam->t_far, &cs);
    for (int64_t i = 0; i < C && i < cap; ++i) { cid[i] = cs[i].id; ct[i] = cs[i].t; }
    free(cs); free(start); free(ids); free(pos);
    return C;
}

/* Accepted points of one ray with t in [tn, tf] (D5 restricted to the
 * interval), in (t, id) order.  mode 0: brute force over all points; 1: the
 * hashed walk of the full window h; 2: the hashed walk of the D12 window hr
 * that t >= tn allows.  Returns the count (cid / ct get the first cap) and
 * the window half-width walked in *h_out. */
int64_t or_ray_candidates_interval(const float *pts, int64_t N, const or_camera *cam, const or_params *prm,
                                   int32_t pixel, int32_t mode, float tn, float tf, int32_t cap, int32_t *cid,
                                   float *ct, int32_t *h_out)
{
    int32_t h;
    float rdd;
    if (or_window(cam, prm, &h, &rdd) != 0) return -1;
    int64_t W = cam->width, H = cam->height;
    if (pixel < 0 || pixel >= W * H || mode < 0 || mode > 2) return -3;
    int64_t P = (W + 2 * h) * (H + 2 * h);
    uint32_t *start = NULL;
    int32_t *ids = NULL;
    float *pos = NULL;
    if (mode != 0) {
        start = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(P + 1));
        ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
        pos = (float *)malloc(sizeof(float) * 3 * (size_t)(N > 0 ? N : 1));
        or_build_table(pts, N, cam, h, start, ids, pos);
    }
    frame_t fr = {pts, N, cam, prm, h, rdd, start, ids, pos};
    ray_t ray;
    int pu = (int)(pixel % W), pv = (int)(pixel / W);
    make_ray(cam, prm, rdd, pu, pv, &ray);
    int hr = h;
    if (mode == 2) {
        float rcos, rsin, rwin;
        d12_terms(cam, prm, &rcos, &rsin, &rwin);
        hr = d12_window(cam, prm, h, tn, rcos, rsin, rwin);
    }
    if (h_out) *h_out = hr;
    cand_t *cs;
    int64_t C = ray_candidates_w(&fr, &ray, pu, pv, mode == 0, tn, tf, hr, NULL, NULL, &cs);
    for (int64_t i = 0; i < C && i < cap; ++i) { cid[i] = cs[i].id; ct[i] = cs[i].t; }
    free(cs); free(start); free(ids); free(pos);
    return C;
}

/* The continuous stages alone for caller-given samples of one ray (pixel),
 * for tests of Sec. 3.4 / Eq. 2 in isolation.  nbr is n_s x K (-1 = unused). */
void or_shade(const float *pts, const float *feats, int32_t F, const or_camera *cam, const or_params *prm,
              const int32_t *dims, int32_t n_layers, const float *mlp, int32_t pixel, int32_t n_s,
              const float *ts, const int32_t *nbr, double *rgb, double *wsum, double *feat_out, double *out4)
{
    int32_t h;
    float rdd;
    if (or_window(cam, prm, &h, &rdd) != 0) { h = 0; rdd = 0.0f; }
    frame_t fr = {pts, 0, cam, prm, h, rdd, NULL, NULL, NULL};
    ray_t ray;
    make_ray(cam, prm, rdd, pixel % cam->width, pixel / cam->width, &ray);
    shade_ray(&fr, &ray, feats, F, dims, n_layers, mlp, prm->K, n_s, ts, nbr, rgb, wsum, feat_out, out4);
}

/* The ray of pixel (u, v) under D3/D4: d[3], q, n2, len, c. */
void or_ray(const or_camera *cam, const or_params *prm, int32_t pu, int32_t pv, float *out6)
{
    int32_t h;
    float rdd = 0.0f;
    if (or_window(cam, prm, &h, &rdd) != 0) rdd = 0.0f;
    ray_t ray;
    make_ray(cam, prm, rdd, pu, pv, &ray);
    out6[0] = ray.d[0]; out6[1] = ray.d[1]; out6[2] = ray.d[2];
    out6[3] = ray.n2; out6[4] = ray.len; out6[5] = ray.c;
}

/* Selection alone on caller-given candidates of one ray (for the hand-worked
 * special cases of Sec. 3.3).  P is C x 3 camera-space positions, t[C] and
 * id[C] already in (t, id) order.  Returns n_s; writes t/src of the samples,
 * the primary index j* (or -1), and every candidate's pseudo-UDF d_j and
 * weight w_j (d_out[C], w_out[C]). */
int32_t or_select(const or_camera *cam, const or_params *prm, int32_t pixel, int32_t C, const float *t,
                  const int32_t *id, const float *P, float *out_t, int32_t *out_src, int32_t *out_nbr,
                  float *out_dist, int32_t *jstar_out, float *d_out, float *w_out)
{
    int32_t h;
    float rdd;
    if (or_window(cam, prm, &h, &rdd) != 0) { h = 0; rdd = 0.0f; }
    frame_t fr = {NULL, 0, cam, prm, h, rdd, NULL, NULL, NULL};
    ray_t ray;
    make_ray(cam, prm, rdd, pixel % cam->width, pixel / cam->width, &ray);
    cand_t *cs = (cand_t *)malloc(sizeof(cand_t) * (size_t)(C > 0 ? C : 1));
    for (int32_t i = 0; i < C; ++i) {
        cs[i].t = t[i]; cs[i].id = id[i];
        cs[i].P[0] = P[3 * i]; cs[i].P[1] = P[3 * i + 1]; cs[i].P[2] = P[3 * i + 2];
    }
    ray_result_t res;
    res.nbr = out_nbr;
    res.ndist = out_dist;
    select_samples(&fr, &ray, cs, C, prm->K, prm->n_max, &res, d_out, w_out, NULL);
    for (int32_t m = 0; m < res.n_s; ++m) { out_t[m] = res.t[m]; out_src[m] = res.src[m]; }
    *jstar_out = -1;
    if (res.n_s > 0) {
        for (int32_t i = 0; i < C; ++i) if (cs[i].id == res.src[0]) { *jstar_out = i; break; }
    }
    free(cs);
    return res.n_s;
}

/* ------------------------------------------------------------ backward
 * Gradients of the rendered colour c and weight sum W = sum_j w'_j (Eq. 2)
 * of every ray with respect to the point features and the point positions,
 * the discrete structure (neighbour sets, samples) held fixed.  Forward, per
 * sample j of a ray with direction d: x_j = t_j d; IDW weights
 * w_ij = 1/max(|x_j - P_i|, eps_d), f_j = sum_i w_ij f_i / sum_i w_ij; MLP ->
 * o_j; sigma_j = softplus(o_j0), c_j = sigmoid(o_j1..3); E_j =
 * exp(-sigma_j Delta_j), tau_1 = 1, tau_{j+1} = tau_j E_j, w'_j = tau_j (1 - E_j);
 * c = sum_j w'_j c_j + (1 - W) bg.  Sample depths depend on the source point:
 * t_j = t_j(0) + <P_src - P_src(0), d>; Delta_j = t_{j+1} - t_j, Delta_last =
 * 2 r(t_last).  Positions are camera space P = R p + t; world gradients are
 * R^T dL/dP.  All in double.  "pcam" holds the camera-space positions the
 * function is evaluated at (N x 3) and "pcam0" the base positions the sample
 * depths t_j(0) belong to. */

typedef struct {
    double P[3];
} v3_t;

static void mlp_forward_keep(const int32_t *dims, int32_t L, const float *params, const double *x, double *acts,
                             double *pre, double *out)
{
    /* acts: per layer input (L x 1024), pre: per layer pre-activation (L x 1024) */
    const float *P = params;
    for (int32_t i = 0; i < dims[0]; ++i) acts[i] = x[i];
    for (int32_t l = 0; l < L; ++l) {
        int32_t fi = dims[l], fo = dims[l + 1];
        const float *W = P, *b = P + (int64_t)fi * fo;
        double *in = acts + (int64_t)l * 1024, *z = pre + (int64_t)l * 1024;
        for (int32_t o = 0; o < fo; ++o) {
            double acc = (double)b[o];
            for (int32_t i = 0; i < fi; ++i) acc += (double)W[(int64_t)o * fi + i] * in[i];
            z[o] = acc;
            if (l + 1 < L) acts[(int64_t)(l + 1) * 1024 + o] = acc > 0.0 ? acc : 0.0;
            else out[o] = acc;
        }
        P += (int64_t)fi * fo + fo;
    }
}

/* Continuous forward (and optional backward) of one ray with frozen structure. */
static void ray_continuous(const or_camera *cam, const or_params *prm, const float *d32, float c_cone,
                           const double *pcam, const double *pcam0, const double *feats, int32_t F,
                           const int32_t *dims, int32_t L, const float *mlp, int32_t K, int32_t n_s,
                           const float *ts, const int32_t *src, const int32_t *nbr, double *rgb, double *wsum,
                           const double *grad_rgb, double grad_wsum, double *g_feats, double *g_pcam)
{
    double d[3] = {d32[0], d32[1], d32[2]};
    double bg = prm->bg_mode == 1 ? 1.0 : 0.0;
    enum { MS = 64 };
    double t[MS], sig[MS], col[MS][3], o[MS][4], delta[MS], E[MS], tau[MS], wp[MS];
    double Wsum[MS];
    double (*fe)[1024] = (double (*)[1024])malloc(sizeof(double) * 1024 * (size_t)(n_s > 0 ? n_s : 1));
    double *acts_all = (double *)malloc(sizeof(double) * (size_t)L * 1024 * (size_t)(n_s > 0 ? n_s : 1));
    double *pre_all = (double *)malloc(sizeof(double) * (size_t)L * 1024 * (size_t)(n_s > 0 ? n_s : 1));
#define ACTS(j) (acts_all + (int64_t)(j) * L * 1024)
#define PRE(j) (pre_all + (int64_t)(j) * L * 1024)
    double T = 1.0, ws = 0.0, c3[3] = {0, 0, 0};
    for (int32_t j = 0; j < n_s; ++j) {
        const double *Ps = pcam + 3 * (int64_t)src[j], *P0 = pcam0 + 3 * (int64_t)src[j];
        t[j] = (double)ts[j] + ((Ps[0] - P0[0]) * d[0] + (Ps[1] - P0[1]) * d[1] + (Ps[2] - P0[2]) * d[2]);
    }
    for (int32_t j = 0; j < n_s; ++j) {
        double x[3] = {t[j] * d[0], t[j] * d[1], t[j] * d[2]};
        double W = 0.0;
        for (int32_t k = 0; k < F; ++k) fe[j][k] = 0.0;
        for (int32_t m = 0; m < K; ++m) {
            int32_t id = nbr[(int64_t)j * K + m];
            if (id < 0) continue;
            const double *Pi = pcam + 3 * (int64_t)id;
            double dx = x[0] - Pi[0], dy = x[1] - Pi[1], dz = x[2] - Pi[2];
            double dist = sqrt(dx * dx + dy * dy + dz * dz);
            double w = 1.0 / (dist > prm->eps_d ? dist : (double)prm->eps_d);
            W += w;
            for (int32_t k = 0; k < F; ++k) fe[j][k] += w * feats[(int64_t)id * F + k];
        }
        for (int32_t k = 0; k < F; ++k) fe[j][k] /= W;
        Wsum[j] = W;
        mlp_forward_keep(dims, L, mlp, fe[j], ACTS(j), PRE(j), o[j]);
        sig[j] = softplus_d(o[j][0]);
        for (int a = 0; a < 3; ++a) col[j][a] = sigmoid_d(o[j][1 + a]);
    }
    for (int32_t j = 0; j < n_s; ++j) {
        delta[j] = (j + 1 < n_s) ? t[j + 1] - t[j]
                                 : 2.0 * (prm->radius_mode == 0 ? (double)prm->r : t[j] * (double)c_cone);
        E[j] = exp(-sig[j] * delta[j]);
        tau[j] = T;
        wp[j] = T * -expm1(-sig[j] * delta[j]);
        for (int a = 0; a < 3; ++a) c3[a] += wp[j] * col[j][a];
        ws += wp[j];
        T *= E[j];
    }
    for (int a = 0; a < 3; ++a) rgb[a] = c3[a] + (1.0 - ws) * bg;
    *wsum = ws;
    if (!grad_rgb) {
        free(fe); free(acts_all); free(pre_all);
        return;
    }

    /* composite backward */
    double gw[MS], gsig[MS], gdel[MS], gt[MS], suffix = 0.0;
    for (int32_t j = 0; j < n_s; ++j)
        gw[j] = grad_rgb[0] * (col[j][0] - bg) + grad_rgb[1] * (col[j][1] - bg) + grad_rgb[2] * (col[j][2] - bg) +
                grad_wsum;
    for (int32_t j = n_s - 1; j >= 0; --j) {
        double bracket = gw[j] * tau[j] * E[j] - suffix;   /* suffix = sum_{k>j} gw_k w'_k */
        gsig[j] = bracket * delta[j];
        gdel[j] = bracket * sig[j];
        suffix += gw[j] * wp[j];
    }
    for (int32_t j = 0; j < n_s; ++j) gt[j] = 0.0;
    for (int32_t j = 0; j < n_s; ++j) {
        if (j + 1 < n_s) {
            gt[j + 1] += gdel[j];
            gt[j] -= gdel[j];
        } else if (prm->radius_mode != 0) {
            gt[j] += gdel[j] * 2.0 * (double)c_cone;
        }
    }
    for (int32_t j = 0; j < n_s; ++j) {
        /* activations and MLP backward */
        double dz[1024], dh[1024];
        double go[4];
        go[0] = gsig[j] * sigmoid_d(o[j][0]);
        for (int a = 0; a < 3; ++a) go[1 + a] = grad_rgb[a] * wp[j] * col[j][a] * (1.0 - col[j][a]);
        for (int32_t k = 0; k < 4; ++k) dz[k] = go[k];
        const float *Pl[16];
        {
            const float *P = mlp;
            for (int32_t l = 0; l < L; ++l) { Pl[l] = P; P += (int64_t)dims[l] * dims[l + 1] + dims[l + 1]; }
        }
        for (int32_t l = L - 1; l >= 0; --l) {
            int32_t fi = dims[l], fo = dims[l + 1];
            const float *W = Pl[l];
            for (int32_t i = 0; i < fi; ++i) {
                double acc = 0.0;
                for (int32_t oo = 0; oo < fo; ++oo) acc += (double)W[(int64_t)oo * fi + i] * dz[oo];
                dh[i] = acc;
            }
            if (l > 0) {
                const double *z = PRE(j) + (int64_t)(l - 1) * 1024;
                for (int32_t i = 0; i < fi; ++i) dz[i] = z[i] > 0.0 ? dh[i] : 0.0;
            }
        }
        /* dh = dL/df_j ; IDW backward */
        double x[3] = {t[j] * d[0], t[j] * d[1], t[j] * d[2]};
        double gx[3] = {0, 0, 0};
        for (int32_t m = 0; m < K; ++m) {
            int32_t id = nbr[(int64_t)j * K + m];
            if (id < 0) continue;
            const double *Pi = pcam + 3 * (int64_t)id;
            double dv[3] = {x[0] - Pi[0], x[1] - Pi[1], x[2] - Pi[2]};
            double dist = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
            double w = 1.0 / (dist > prm->eps_d ? dist : (double)prm->eps_d);
            double gwi = 0.0;
            for (int32_t k = 0; k < F; ++k) {
                double fi_k = feats[(int64_t)id * F + k];
                if (g_feats) g_feats[(int64_t)id * F + k] += w / Wsum[j] * dh[k];
                gwi += dh[k] * (fi_k - fe[j][k]) / Wsum[j];
            }
            if (dist > prm->eps_d && g_pcam) {
                double gdist = gwi * (-1.0 / (dist * dist));
                for (int a = 0; a < 3; ++a) {
                    g_pcam[3 * (int64_t)id + a] -= gdist * dv[a] / dist;
                    gx[a] += gdist * dv[a] / dist;
                }
            }
        }
        gt[j] += gx[0] * d[0] + gx[1] * d[1] + gx[2] * d[2];
        if (g_pcam)
            for (int a = 0; a < 3; ++a) g_pcam[3 * (int64_t)src[j] + a] += gt[j] * d[a];
    }
    free(fe); free(acts_all); free(pre_all);
#undef ACTS
#undef PRE
}

/* Backward of the frame whose samples or_render produced.  grad_rgb (R x 3),
 * grad_wsum (R, or NULL); accumulates into grad_feats (N x F), grad_pcam
 * (N x 3, camera space) and grad_pworld (N x 3, world space); any output may
 * be NULL.  Evaluated at the float32 camera-space positions of the contract
 * (D1) and the float32 sample depths, so that it is the derivative of the
 * frame that or_render computes. */
int64_t or_backward(const float *pts, int64_t N, const float *feats, int32_t F, const or_camera *cam,
                    const or_params *prm, const int32_t *dims, int32_t n_layers, const float *mlp,
                    const int32_t *rays, int64_t R, const int64_t *sample_offset, const float *s_t,
                    const int32_t *s_src, const int32_t *s_nbr, const double *grad_rgb, const double *grad_wsum,
                    double *grad_feats, double *grad_pcam, double *grad_pworld)
{
    int32_t h;
    float rdd;
    if (or_window(cam, prm, &h, &rdd) != 0) return -1;
    const int32_t K = prm->K;
    int64_t W = cam->width, H = cam->height;
    double *pc = (double *)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    double *fd = (double *)malloc(sizeof(double) * (size_t)F * (size_t)(N > 0 ? N : 1));
    double *gp = (double *)calloc(3 * (size_t)(N > 0 ? N : 1), sizeof(double));
    for (int64_t i = 0; i < N; ++i) {
        float X[3];
        or_cam_point(cam, pts + 3 * i, X);
        for (int a = 0; a < 3; ++a) pc[3 * i + a] = X[a];
        for (int32_t k = 0; k < F; ++k) fd[i * F + k] = feats[i * F + k];
    }
    for (int64_t i = 0; i < R; ++i) {
        int64_t pix = rays ? rays[i] : i;
        if (pix < 0 || pix >= W * H) continue;
        int64_t a = sample_offset[i], b = sample_offset[i + 1];
        if (b == a) continue;
        ray_t ray;
        make_ray(cam, prm, rdd, (int)(pix % W), (int)(pix / W), &ray);
        double rgb[3], ws;
        ray_continuous(cam, prm, ray.d, ray.c, pc, pc, fd, F, dims, n_layers, mlp, K, (int32_t)(b - a), s_t + a,
                       s_src + a, s_nbr + a * K, rgb, &ws, grad_rgb + 3 * i, grad_wsum ? grad_wsum[i] : 0.0,
                       grad_feats, gp);
    }
    for (int64_t i = 0; i < N; ++i) {
        if (grad_pcam)
            for (int a = 0; a < 3; ++a) grad_pcam[3 * i + a] += gp[3 * i + a];
        if (grad_pworld) /* dL/dp = R^T dL/dP */
            for (int a = 0; a < 3; ++a)
                grad_pworld[3 * i + a] += (double)cam->R[0 + a] * gp[3 * i] + (double)cam->R[3 + a] * gp[3 * i + 1] +
                                          (double)cam->R[6 + a] * gp[3 * i + 2];
    }
    free(pc);
    free(fd);
    free(gp);
    return 0;
}

/* Forward with frozen structure at caller-given camera-space positions
 * (double, N x 3) and features (double, N x F), sample depths moving with
 * their source point from the base positions pcam0 -- the function whose
 * derivative or_backward returns (for finite-difference checks). */
int64_t or_forward_frozen(const double *pcam, const double *pcam0, const double *feats, int32_t F,
                          const or_camera *cam, const or_params *prm, const int32_t *dims, int32_t n_layers,
                          const float *mlp, const int32_t *rays, int64_t R, const int64_t *sample_offset,
                          const float *s_t, const int32_t *s_src, const int32_t *s_nbr, double *rgb, double *wsum)
{
    int32_t h;
    float rdd;
    if (or_window(cam, prm, &h, &rdd) != 0) return -1;
    int64_t W = cam->width, H = cam->height;
    for (int64_t i = 0; i < R; ++i) {
        int64_t pix = rays ? rays[i] : i;
        double bg = prm->bg_mode == 1 ? 1.0 : 0.0;
        rgb[3 * i] = rgb[3 * i + 1] = rgb[3 * i + 2] = bg;
        wsum[i] = 0.0;
        if (pix < 0 || pix >= W * H) continue;
        int64_t a = sample_offset[i], b = sample_offset[i + 1];
        if (b == a) continue;
        ray_t ray;
        make_ray(cam, prm, rdd, (int)(pix % W), (int)(pix / W), &ray);
        ray_continuous(cam, prm, ray.d, ray.c, pcam, pcam0, feats, F, dims, n_layers, mlp, prm->K,
                       (int32_t)(b - a), s_t + a, s_src + a, s_nbr + a * prm->K, rgb + 3 * i, wsum + i, NULL, 0.0,
                       NULL, NULL);
    }
    return 0;
}
