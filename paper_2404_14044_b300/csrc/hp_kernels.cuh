// Launch interfaces between the C-ABI layer and the kernels.
#pragma once

#include "hp_common.cuh"

#include <utility>

namespace hp {

// Launches a kernel with programmatic stream serialization: its blocks may
// become resident while the previous kernel in the stream still runs, and
// wait for it in grid_dep_wait() (every kernel of the library calls that
// first).  Launch errors are also left for cudaGetLastError().
template <typename... P, typename... A>
inline cudaError_t launch_chained(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A &&...args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}


// Kernel ids of the per-kernel profiler (hp_profile_*).
enum KernelId {
    KID_PROJECT = 0, KID_SCAN, KID_SCATTER, KID_SORT, KID_SEARCH, KID_PACK, KID_DECODE, KID_COMPOSITE,
    KID_COMPOSITE_BWD, KID_DECODE_BWD, KID_PROP_INFER, KID_SEARCH_FALLBACK, KID_SEARCH_WIDE, KID_RAY_TABLE, KID_CLEAR, KID_COUNT
};

// Optional CUDA-event pairs around each launch, on the launching stream.
struct Prof {
    bool on = false;
    int cap = 0;
    int n = 0;
    cudaEvent_t *ev = nullptr;   // 2 * cap
    int *kid = nullptr;          // cap
    int *nk = nullptr;           // cap: kernels launched between the two events
};

inline void prof_begin(Prof *p, cudaStream_t st, int kid)
{
    if (p && p->on && p->n < p->cap) {
        p->kid[p->n] = kid;
        cudaEventRecord(p->ev[2 * p->n], st);
    }
}

inline void prof_end(Prof *p, cudaStream_t st, int kernels = 1)
{
    if (p && p->on && p->n < p->cap) {
        cudaEventRecord(p->ev[2 * p->n + 1], st);
        p->nk[p->n] = kernels;
        ++p->n;
    }
}

// Zeroes `bytes` (a multiple of 4, 4-byte aligned) at p with a chained
// kernel (a memset would end the chain of programmatic launches).
cudaError_t launch_clear(void *p, size_t bytes, cudaStream_t st, Prof *prof);

struct BuildArgs {
    const float *pts;
    int64_t N;
    Cam cam;
    int h;
    int64_t P;              // buckets = (W+2h)(H+2h)
    uint32_t *cnt;          // [P+1]
    uint32_t *start;        // [P+1]
    uint2 *keyrank;         // [N]
    float4 *spts;           // [N] bucket by bucket, within a bucket in the atomics' order
    uint32_t *pcell;        // [N] bucket of each listed point (written by the scatter)
    uint64_t *scan_flags;   // [ceil((P+1)/kScanTile)]
    uint32_t *scan_ticket;
    uint32_t *zmin_enc;     // smallest depth of a tabled point, 0x7f800000 - bits (0: none), by atomicMax
    ErrWord *err;
    uint32_t spin_limit;
    int32_t skip_tile;
};

// Candidates per ray held by the lane-per-ray search (its shared-memory
// column); rays with more go to the warp-per-ray search.
constexpr int kLaneCap = 48;
// The column of the point-major selection and of the restricted walk: a
// shorter column leaves room for a fifth block per SM (K <= 8).
constexpr int kLaneCapShort = 40;
// Slots per ray of the point-major pass: the lane search reads rays of up to
// kLaneCap candidates from them, the warp-per-ray search rays of up to kPmCap.
constexpr int kPmCap = 128;
// Most candidates the selection can process for which the lane search prunes
// its column (prune_m; larger bounds switch the pruning off).
constexpr int kPruneMax = 4;

struct SearchArgs {
    Cam cam;                 // raytab is (re)computed from cam when raytab_stale
    int mode;
    float r;
    float rdd;
    int h;
    int Wp;
    float gamma, beta2, eps_w, gap_k;
    int cand_cap;
    int K;
    int n_max;
    int prune_m;             // at most this many candidates are processed per ray (0: no bound used)
    const uint32_t *start;
    const float4 *spts;
    float4 *raytab;          // [W*H] per-pixel (dx, dy, dz, cone c)
    int raytab_stale;        // recompute the ray table before searching
    const float2 *interval;  // per-ray [t0, t1] (proposal-restricted search), NULL: plain
    const uint16_t *prop_w;  // proposal weights (BF16): the search infers each ray's interval itself
    float2 *interval_buf;    // ... and leaves it here for the rays it hands to the warp-per-ray search
    float win_fx, cos_max, sin_max;  // window bound terms for a depth lower bound (fixed radius)
    const uint32_t *zmin_enc;        // smallest depth of a tabled point (as BuildArgs::zmin_enc)
    const uint32_t *pcell;   // bucket of each listed point (whole frames: point-major candidate pass)
    int64_t n_points;        // points given to the table build (bound of the tabled ones)
    uint32_t *pm_cnt;        // [W*H] candidates each pixel's ray received from the point-major pass
    float *pm_t;             // [W*H x kPmCap] depths t of those candidates
    uint32_t *pm_i;          // [W*H x kPmCap] their table indices
    int32_t *fallback;       // rays whose restricted search kept nothing (original indices)
    uint32_t *fallback_count;
    int32_t *wide;           // rays with more candidates than a lane holds (original indices)
    uint32_t *wide_count;
    int32_t *ovf;            // whole frames: pixels whose point-major slots overflowed (the pass lists them)
    uint32_t *ovf_count;
    uint32_t *ovf_pull;      // next of them for the lane kernel's warps
    unsigned long long *pull;    // next listed ray of the warp-per-ray search
    uint32_t *lane_units;    // next tile / group of 32 rays of the lane-per-ray search
    int n_sm;                // multiprocessors of the device (grid sizing)
    const int32_t *ray_map;  // fallback pass: original index of listed ray i
    const uint32_t *count_ptr;   // fallback pass: number of listed rays (device)
    // fallback pass (0: off): the lane-per-ray kernel takes the list only
    // when it holds more than list_split rays; the warp-per-ray kernel takes
    // the whole list up to that many, else the rays the lanes listed as wide
    uint32_t list_split;
    const int32_t *rays;     // NULL: ray i is pixel i
    int64_t R;
    int32_t *n_s;
    int32_t *primary;
    int32_t *cand_count;
    int64_t *sample_offset;
    float *t;
    int32_t *ray;
    int32_t *src;
    float *delta;
    int32_t *nbr;            // packed lists; NULL: left in the slots, sample_slot written instead
    float *nbr_dist;
    int64_t capacity;
    int32_t *sample_slot;    // [n_max x R] slot (m R + i) of each packed sample
    float4 *slot_rec;        // [n_max x R] sample slots (scratch), slot m of ray i at m R + i: t, source id bits, delta
    int32_t *slot_nbr;       // [n_max x R x K]
    float *slot_dist;        // [n_max x R x K]
    uint64_t *flags;         // [ceil(R / 256)] look-back words of the packing scan
    uint32_t *ticket;
    ErrWord *err;
    uint32_t spin_limit;
};

struct RenderArgs {
    const int32_t *n_s;
    const int64_t *sample_offset;
    const float *delta;
    const int32_t *nbr;
    const float *nbr_dist;
    int64_t capacity;
    int64_t R;
    int K;
    const float *feats;
    int F;
    const float *mlp;        // packed W0,b0,W1,b1,... (global)
    int n_layers;
    int dims[HP_MLP_MAX_LAYERS + 1];
    float eps_d;
    int bg_mode;
    int decode;              // HP_DECODE_*
    ErrWord *err;
    float4 *sample_out;      // [capacity] (sigma, r, g, b)
    float *rgb;              // [R*3]
    float *wsum;             // [R]
    int num_sms;
    unsigned char *wimg;     // [kWsImageMax] the tensor-core decode's weight image (16-byte aligned)
    uint32_t *tile_ctr;      // the tensor-core decode's tile counter
    // nbr == NULL: the lists stay in the search's slot rows (slot_nbr,
    // slot_dist: row m R + i holds the K entries of ray i's m-th sample), and
    // sample_slot[g] is the row of packed sample g
    const int32_t *slot_nbr;
    const float *slot_dist;
    const int32_t *sample_slot;
    int64_t n_feats;         // feature rows (the bounds-check build tests neighbour ids against it)
    int64_t n_slots;         // slot rows of the last search (the same, for sample_slot)
};

// Neighbour list of packed sample g: its row in the packed arrays, or its slot
// row when the search left the lists in the slots.
__device__ __forceinline__ int64_t list_row(const RenderArgs &a, int64_t g)
{
    if (a.nbr) return g;
    const int64_t r = __ldg(a.sample_slot + g);
    return hp_check(r >= 0 && r < a.n_slots, a.err, r) ? r : 0;   // (bounds-check build: row 0 instead)
}
__device__ __forceinline__ const int32_t *list_ids(const RenderArgs &a) { return a.nbr ? a.nbr : a.slot_nbr; }
__device__ __forceinline__ const float *list_dists(const RenderArgs &a) { return a.nbr ? a.nbr_dist : a.slot_dist; }

// Largest weight image of the tensor-core decode (its shared-memory limit).
constexpr int kWsImageMax = 227 * 1024;

__global__ void k_scan(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int64_t n, uint64_t *flags,
                       uint32_t *ticket, ErrWord *err, uint32_t spin_limit, int32_t skip_tile);

struct PropArgs {
    Cam cam;
    int h, Wp, Hp;
    const uint32_t *start;
    const float4 *spts;
    const int32_t *rays;
    int64_t R;
    const uint16_t *weights_bf16;   // inference weights
    float2 *interval;               // inference output
    float *params;                  // training: FP32 master weights
    float *grad;
    float *loss;                    // [2]: summed loss, rays used
    uint16_t *weights_out;          // training: refreshed BF16 copy
    const int32_t *n_s;             // training targets: the plain search's samples
    const int64_t *sample_offset;
    const float *t;
};

struct BwdArgs {
    const int32_t *n_s;
    const int64_t *sample_offset;
    const float *t;
    const int32_t *ray;
    const int32_t *src;
    const float *delta;
    const int32_t *nbr;
    const float *nbr_dist;
    int64_t capacity;
    int64_t R;
    int K;
    const int32_t *rays;     // pixel of each ray (NULL: ray i is pixel i)
    const float4 *raytab;    // per-pixel (d, cone c)
    Cam cam;
    int mode;
    const float *points;     // world N x 3
    const float *feats;
    int F;
    const float *mlp;
    int n_layers;
    int dims[HP_MLP_MAX_LAYERS + 1];
    float eps_d;
    int bg_mode;
    const float4 *sample_out;   // forward (sigma, r, g, b) per sample
    const float *grad_rgb;      // R x 3
    const float *grad_wsum;     // R or NULL
    float4 *go;                 // scratch: dL/d(MLP output) per sample
    float *gt;                  // scratch: dL/dt_j through the Delta's
    int64_t n_points;           // N (the bounds-check build tests neighbour ids against it)
    ErrWord *err;
    float *grad_feats;          // N x F, accumulated (NULL: skip)
    float *grad_points;         // N x 3 world, accumulated (NULL: skip)
    int num_sms;
};

cudaError_t launch_build(const BuildArgs &a, cudaStream_t st, Prof *prof);
// The list of a built table in its canonical order: each bucket's points of
// `list` sorted by (z, x, y, id) into `out`; big / n_big: scratch for the list
// of large buckets (P + 1 words) and its counter.
cudaError_t launch_bucket_sort(int64_t P, const uint32_t *start, const float4 *list, float4 *out, uint32_t *big,
                               uint32_t *n_big, cudaStream_t st);
size_t backward_smem_bytes(const BwdArgs &a);
cudaError_t launch_prop_infer(const PropArgs &a, cudaStream_t st, Prof *prof);
cudaError_t launch_prop_train(const PropArgs &a, float *m, float *v, int step, float lr, cudaStream_t st);
cudaError_t launch_backward(const BwdArgs &a, cudaStream_t st, Prof *prof);
size_t search_smem_bytes();
cudaError_t launch_search(const SearchArgs &a, cudaStream_t st, Prof *prof);
size_t render_smem_bytes(const RenderArgs &a);
cudaError_t launch_render(const RenderArgs &a, cudaStream_t st, Prof *prof);
bool decode_tc_supported(const RenderArgs &a, bool bf16, size_t *smem);
// n_kernels: CUDA kernels launched (the weight image and the decode, or the decode alone)
cudaError_t launch_decode_tc(const RenderArgs &a, bool bf16, cudaStream_t st, int *n_kernels);
cudaError_t launch_mma_selftest(const uint16_t *A, const uint16_t *B, float *D, int K, int N, int flags, ErrWord *err,
                                cudaStream_t st);

}  // namespace hp
