// Shared device definitions of the HashPoint CUDA path (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hashpoint.h"

namespace hp {

// ------------------------------------------------------------------ limits
constexpr int kHMax = 64;            // largest window half-width
constexpr int kCandCap = 128;        // candidate buffer per ray (power of two)
constexpr int kMaxK = 32;            // neighbours per candidate
constexpr int kMaxSamples = 16;      // samples per ray
constexpr int kSearchWarps = 8;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;        // per thread: tile = 8192 entries
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr uint32_t kSpinLimitDefault = 1u << 22;
constexpr uint32_t kNoKey = 0xFFFFFFFFu;

// ------------------------------------------- programmatic dependent launch
// The kernels of a frame are launched with programmatic stream serialization
// (launch_chained): a kernel's blocks may become resident while its
// predecessor in the stream is still running, and wait in grid_dep_wait()
// until that grid has completed and its memory operations are visible.  Every
// kernel calls grid_dep_wait() before it touches global memory (a no-op when
// it was launched without the attribute) and then grid_dep_trigger(), which
// lets its own successor launch once every block of this grid has started.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ------------------------------------------------------ device status word
struct ErrWord {
    int32_t status;
    int32_t pad;
    int64_t detail;
};

__device__ __forceinline__ void set_error(ErrWord *e, int32_t code, int64_t detail)
{
    if (atomicCAS(&e->status, 0, code) == 0) e->detail = detail;
}

// Bounds-check build (compiled with -DHP_CHECKS=1, libhashpoint_checks.so):
// hp_check(ok, err, index) records HP_ERR_BOUNDS with the index when an index
// check fails and returns false, so that the caller skips the access.  In the
// normal build it is the constant true and costs nothing.
#ifdef HP_CHECKS
__device__ __forceinline__ bool hp_check(bool ok, ErrWord *e, int64_t index)
{
    if (!ok) set_error(e, HP_ERR_BOUNDS, index);
    return ok;
}
#else
__device__ __forceinline__ bool hp_check(bool, ErrWord *, int64_t) { return true; }
#endif

// --------------------------------------------- decision arithmetic contract
// Every discrete decision is computed with single IEEE binary32 operations in
// a written order (no contraction), so that an independent CPU program that
// follows the same order reaches the same decisions bit for bit.
__device__ __forceinline__ float dadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float dsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float dmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float ddiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float dsqrt(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ float dfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Camera parameters as the kernels read them (by value, kernel argument).
struct Cam {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float t_near, t_far, z_near;
    int32_t width, height;
};

// Camera-space position: X = ((R0 px + R1 py) + R2 pz) + t0, rows alike.
__device__ __forceinline__ float3 cam_point(const Cam &c, float px, float py, float pz)
{
    float3 o;
    o.x = dadd(dadd(dadd(dmul(c.R[0], px), dmul(c.R[1], py)), dmul(c.R[2], pz)), c.t[0]);
    o.y = dadd(dadd(dadd(dmul(c.R[3], px), dmul(c.R[4], py)), dmul(c.R[5], pz)), c.t[1]);
    o.z = dadd(dadd(dadd(dmul(c.R[6], px), dmul(c.R[7], py)), dmul(c.R[8], pz)), c.t[2]);
    return o;
}

// Pixel key of a camera-space point in the image padded by h on each side;
// kNoKey when Z <= z_near or the pixel lies outside the padded image.
__device__ __forceinline__ uint32_t pixel_key(const Cam &c, int h, float3 X)
{
    if (!(X.z > c.z_near)) return kNoKey;
    float u = dadd(dmul(c.fx, ddiv(X.x, X.z)), c.cx);
    float v = dadd(dmul(c.fy, ddiv(X.y, X.z)), c.cy);
    float fu = floorf(u), fv = floorf(v);
    if (!(fu >= (float)(-h) && fu < (float)(c.width + h) && fv >= (float)(-h) && fv < (float)(c.height + h)))
        return kNoKey;
    uint32_t iu = (uint32_t)((int)fu + h), iv = (uint32_t)((int)fv + h);
    return iv * (uint32_t)(c.width + 2 * h) + iu;
}

// Ray through the centre of pixel (pu, pv) from the camera centre:
// d = (nx, ny, 1) / |(nx, ny, 1)|; c = cone coefficient (r(t) = t c).
struct Ray {
    float dx, dy, dz;
    float c;
};

__device__ __forceinline__ Ray make_ray(const Cam &cam, int mode, float rdd, int pu, int pv)
{
    float nx = ddiv(dsub(dadd((float)pu, 0.5f), cam.cx), cam.fx);
    float ny = ddiv(dsub(dadd((float)pv, 0.5f), cam.cy), cam.fy);
    float q = dadd(dmul(nx, nx), dmul(ny, ny));
    float n2 = dadd(q, 1.0f);
    float len = dsqrt(n2);
    Ray r;
    r.dx = ddiv(nx, len);
    r.dy = ddiv(ny, len);
    r.dz = ddiv(1.0f, len);
    r.c = 0.0f;
    if (mode == HP_RADIUS_CONE) {
        float g = dsub(dsqrt(q), rdd);
        r.c = ddiv(rdd, dmul(len, dsqrt(dadd(dmul(g, g), 1.0f))));
    } else if (mode == HP_RADIUS_CONE_APPROX) {
        r.c = ddiv(rdd, n2);
    }
    return r;
}

__device__ __forceinline__ float radius_at(int mode, float r, const Ray &ray, float t)
{
    return mode == HP_RADIUS_FIXED ? r : dmul(t, ray.c);
}

// exp(x) for the confidence alpha_j: Cody & Waite range reduction
// (x = k ln2 + r, ln2 = LN2_HI + LN2_LO with a 16-bit LN2_HI so k*LN2_HI is
// exact), the Taylor series of exp(r) to degree 7 in Horner form, and a scale
// by 2^k built from exponent bits (two steps below 2^-126).
__device__ __forceinline__ float exp32(float x)
{
    constexpr float kL2E = (float)(1.0 / 0.69314718055994530942);
    constexpr float kLn2Hi = (float)(45426.0 / 65536.0);
    constexpr float kLn2Lo = (float)(0.69314718055994530942 - 45426.0 / 65536.0);
    constexpr float kC2 = (float)(1.0 / 2.0), kC3 = (float)(1.0 / 6.0), kC4 = (float)(1.0 / 24.0);
    constexpr float kC5 = (float)(1.0 / 120.0), kC6 = (float)(1.0 / 720.0), kC7 = (float)(1.0 / 5040.0);
    if (x != x) return x;
    if (x < -104.0f) return 0.0f;
    if (x > 88.5f) return __int_as_float(0x7f800000);
    float kf = rintf(dmul(x, kL2E));
    float r = dsub(dsub(x, dmul(kf, kLn2Hi)), dmul(kf, kLn2Lo));
    float p = kC7;
    p = dadd(dmul(p, r), kC6);
    p = dadd(dmul(p, r), kC5);
    p = dadd(dmul(p, r), kC4);
    p = dadd(dmul(p, r), kC3);
    p = dadd(dmul(p, r), kC2);
    p = dadd(dmul(p, r), 1.0f);
    p = dadd(dmul(p, r), 1.0f);
    int k = (int)kf;
    if (k >= -126) return dmul(p, __int_as_float((k + 127) << 23));
    return dmul(dmul(p, __int_as_float((k + 227) << 23)), __int_as_float(27 << 23));
}

// ------------------------------------------------ decoupled look-back scan
// Single-pass prefix sums (Merrill & Garland, "Single-pass Parallel Prefix
// Scan with Decoupled Look-back", 2016).  Each tile publishes a 64-bit word
// holding a 2-bit state (1 = aggregate, 2 = inclusive prefix) and a 62-bit
// value; tiles are numbered by an atomic ticket so every predecessor is
// already running.  The wait is bounded: after `spin_limit` polls the tile
// records HP_ERR_TIMEOUT, treats the missing value as 0 and goes on.
constexpr uint64_t kLbAgg = 1ull << 62;
constexpr uint64_t kLbPre = 2ull << 62;
constexpr uint64_t kLbVal = kLbAgg - 1;

__device__ __forceinline__ void st_relaxed(uint64_t *p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Decoupled look-back (flags: 2-bit state -- 0 nothing, 1 the tile's
// aggregate, 2 its inclusive prefix -- over a 62-bit value), called by a
// whole warp with the tile's aggregate agg: returns the tile's exclusive
// prefix.  The warp inspects 32 predecessors per step, nearest in lane 0,
// and stops at the nearest one that has published its inclusive prefix.
__device__ __forceinline__ int64_t lookback_prefix_warp(uint64_t *flags, int64_t tile, int64_t agg, ErrWord *err,
                                                        uint32_t spin_limit, bool publish)
{
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (publish && lane == 0) st_relaxed(flags, kLbPre | (uint64_t)agg);
        return 0;
    }
    if (publish && lane == 0) st_relaxed(flags + tile, kLbAgg | (uint64_t)agg);
    int64_t excl = 0;
    int64_t j0 = tile - 1;
    uint32_t spins = 0;
    for (;;) {
        const int64_t j = j0 - lane;
        // before tile 0: an inclusive prefix of 0
        const uint64_t v = j >= 0 ? ld_relaxed(flags + j) : kLbPre;
        const uint64_t state = v >> 62;
        const unsigned m2 = __ballot_sync(0xffffffffu, state == 2), m0 = __ballot_sync(0xffffffffu, state == 0);
        const int first2 = m2 ? __ffs(m2) - 1 : 31;
        const unsigned need = first2 == 31 ? 0xffffffffu : ((2u << first2) - 1u);   // lanes 0 .. first2
        if (m0 & need) {
            // a needed predecessor has published nothing yet
            if (++spins > spin_limit) {
                if (lane == 0) set_error(err, HP_ERR_TIMEOUT, tile);
                break;
            }
            __nanosleep(64);
            continue;
        }
        int64_t x = lane <= first2 ? (int64_t)(v & kLbVal) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        excl += x;
        if (m2) break;
        j0 -= 32;
    }
    if (publish && lane == 0) st_relaxed(flags + tile, kLbPre | (uint64_t)(excl + agg));
    return excl;
}

// Inclusive warp scan of an int.
__device__ __forceinline__ int warp_incl_scan(int v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Inclusive warp scan of a uint32 (sums modulo 2^32).
__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

inline int64_t div_up(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace hp
