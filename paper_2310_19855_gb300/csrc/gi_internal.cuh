// Internal declarations shared by the translation units of libgi.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gi.h"

namespace gi {

constexpr uint32_t kEmpty = 0u;          // fingerprint word of an empty slot
constexpr int kFixShift = 24;            // fixed point: 2^-24 radiance units
constexpr float kRadMax = 32768.0f;      // radiance clamp before quantisation
constexpr int kQBits = 19;               // bits per quantised coordinate
constexpr uint32_t kQMask = (1u << kQBits) - 1u;

// 32-byte per-slot accumulator: one sector.  stamp = 1 + frame of the last
// resolve that found samples in the cell (0 = never resolved).
struct __align__(16) Accum {
    unsigned long long sum[3];
    uint32_t count;
    uint32_t stamp;
};
static_assert(sizeof(Accum) == 32, "accumulator must fill one 32-byte sector");

// Device counters of a cache (one 128-byte line).
struct __align__(128) Counters {
    uint32_t touch_count;   // entries in the touch list since the last resolve
    uint32_t ticket;        // last-block ticket of the resolve kernel
    uint32_t occupied;      // slots holding a fingerprint
    uint32_t max_probe;     // longest probing run seen
    unsigned long long dropped;
    unsigned long long clamped;
    uint32_t error_word;
    uint32_t pad[23];
};

// Per-view constants of the cell descriptor (Algorithm 6 + LOD reading).
struct KeyParams {
    float cam[3];
    float thr[3];      // squared-distance thresholds of LODs 1..3
    float side[4];     // s0 * 2^l
    float inv_side[4]; // (1/s0) * 2^-l
    int num_lods;
};

#ifdef __CUDACC__
// PCG hash (Jarzynski & Olano 2020): one LCG step, then PCG's RXS-M-XS output.
__host__ __device__ __forceinline__ uint32_t pcg_hash(uint32_t v) {
    uint32_t state = v * 747796405u + 2891336453u;
    uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
    return (word >> 22u) ^ word;
}

// LOD of the cell descriptor: the float32 squared camera distance (fixed order, no contraction)
// against the Algorithm-6 thresholds.
__device__ __forceinline__ int key_lod(const KeyParams &k, float px, float py, float pz) {
    const float dx = __fsub_rn(px, k.cam[0]);
    const float dy = __fsub_rn(py, k.cam[1]);
    const float dz = __fsub_rn(pz, k.cam[2]);
    const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    int lod = 0;
    if (k.num_lods > 1 && d2 >= k.thr[0]) lod = 1;
    if (k.num_lods > 2 && d2 >= k.thr[1]) lod = 2;
    if (k.num_lods > 3 && d2 >= k.thr[2]) lod = 3;
    return lod;
}
#endif

// Host helpers (gi_common.cu)
void set_error(const char *fmt, ...);
gi_status cuda_status(cudaError_t e, const char *what);
KeyParams key_params(float cell_size, uint32_t num_lods, const gi_view *v);
double distance_scale(double fov_y, uint32_t width, uint32_t height);
bool view_ok(const gi_view *v);

// Pinhole camera constants for device code.
struct CamParams {
    float pos[3], fwd[3], right[3], up[3];
    float sx_scale, sy_scale; // tan(fov/2) * W/H, tan(fov/2)
    float inv_w, inv_h;
    uint32_t width, height;
};
CamParams cam_params(const gi_view *v);


// ---------------------------------------------------------------- per-pass arguments
typedef uint32_t SlotWord;  // tag = fingerprint << 8 | (home mod 256); 0 = empty
__device__ __forceinline__ uint32_t word_tag(SlotWord w) { return w; }

struct UpdateArgs {
    const float *p[3];
    const float *nrm[3];
    const float *rad[3];
    const float *len;
    const float *dir[3];
    uint32_t *slot_ids;
    unsigned long long n;
    SlotWord *tags;
    Accum *accum;
    uint32_t acc_stride;  // Accum units between consecutive slots
    uint32_t *touch;
    uint32_t *bitmap;     // touched slots, one bit each (NULL: first touches go to the touch list)
    Counters *ctr;
    uint32_t mask;
    uint32_t max_probe;
    KeyParams kp;
    // far hits to the surrogate (gi_cache_route_far): while the network's judged error stats
    // (route_stats[1] <= route_trust * route_stats[2], route_stats[2] > 0) allow it, hits with
    // LOD >= route_lod are left out of the table; route_stats NULL: no routing
    const float *route_stats;
    float route_trust;
    uint32_t route_lod;
}; // UpdateArgs

struct ResolveArgs {
    const uint32_t *touch;
    uint32_t *bitmap;     // touched slots (walked and cleared by the resolve)
    uint32_t words;       // bitmap words = slots / 32
    Accum *accum;
    uint32_t acc_stride;
    void *resolved;
    uint32_t res_stride;  // bytes between consecutive resolved values
    Counters *ctr;
    float alpha;
    uint32_t stamp_now;   // frame + 1
    uint32_t has_lr;      // a resolve happened before
    uint32_t lr;          // frame of that resolve
    uint32_t evict;       // E
    int f16;
    uint32_t *occ_out;    // host-mapped {occupied slots, stamp_now}, written by the last block
};

struct LiveRule {
    uint32_t has_lr, lr, evict;
};

struct MipInfo {
    int count;
    int w[GI_MAX_MIPS], h[GI_MAX_MIPS], off[GI_MAX_MIPS];
};

struct SpawnArgs {
    const float4 *gbuf;
    uint32_t width, height;
    CamParams cam;
    int jx, jy;            // jitter inside the spawn tile of 8 upscale x 8 upscale pixels
    uint32_t upscale;      // 1: every 8x8 tile spawns; u: one tile per spawn tile
    uint32_t keep;         // tiles without a fresh probe keep their level-0 mask, position, normal
    uint32_t *mask;
    float4 *pos;
    float4 *nrm;
    uint32_t tiles_x, tiles_y;
    MipInfo mi;
};

// Screen-probe reprojection (Algorithm 1).
struct ReprojArgs {
    const float4 *gbuf;
    const float2 *motion;  // per pixel: offset to the previous frame's position of its surface point
    uint32_t width, height, tiles_x, tiles_y;
    CamParams cam;
    float dscale;          // cell_size(d) = dscale * d
    const uint32_t *prev_mask;
    const float4 *prev_pos, *prev_nrm;
    uint32_t *mask;
    float4 *pos, *nrm;
    uint32_t *src;         // source probe of each tile (GI_PROBE_NONE: none)
};


struct IntegrateArgs {
    const uint32_t *slot_ids;
    const void *resolved;
    uint32_t res_stride;
    int f16;
    uint32_t slots;
    const float4 *nrm;
    float *sh;
    uint32_t probes;
    uint32_t rpp;
    float env[3];
    const uint32_t *ovr_bits;  // surrogate answers: bit r set -> record r takes ovr[r] (or NULL)
    const float4 *ovr;
    const float *ray_len;      // ray lengths of the records (probe atlas: mean hit distance per cell)
};

// Frame atlas of the temporal path: fresh probes gather their spawn tile's rays (blended with the
// tile's reprojected probe by Algorithm 4), reprojected-only probes carry their source's cells.
struct TemporalArgs {
    IntegrateArgs g;       // records of the spawn tiles (g.probes = spawn tiles)
    const float4 *gbuf;
    uint32_t width, height, tiles_x, probes, upscale, spawn_x;
    int jx, jy;
    const uint32_t *src;
    const float4 *prev_atlas;
    float4 *atlas;
};

struct InterpArgs {
    const float4 *gbuf;
    uint32_t width, height;
    CamParams cam;
    float dscale;
    const uint32_t *mask;
    MipInfo mi;
    const float4 *ppos;
    const float4 *pnrm;
    const float *sh;
    uint32_t tiles_x;
    float4 *out;
};

// ---------------------------------------------------------------- tile table (gi_tiles.cu)
// Two-level cache (Section 2.2.3): a slot holds a tile of 8 x 8 cells; cell e = slot * 64 + cell.
constexpr int kTileCells = 64;
constexpr int kTileMips = 21;  // 4x4 + 2x2 + 1x1 values above the cells

struct TileArrays {
    SlotWord *tags;              // [T] tile tags
    Accum *accum;                // [T * 64] sums and count since the last resolve (stamp field unused)
    uint32_t *stamp;             // [T * 64] 1 + frame of the last resolve with samples; 0 = never
    float4 *state;               // [T * 64] blended radiance; w = sample count (u32 bits)
    void *resolved;              // [T * 64] answer of each live cell (float4 or half4, w = cold)
    float4 *mips;                // [T * 21] MIP values; w = sample count (u32 bits), 0 = none
    unsigned long long *omask;   // [T] cells live after the tile's last resolve
};

struct TileUpdateArgs {
    UpdateArgs u;                // u.tags / u.accum / u.mask / u.ctr of the tile table
    unsigned long long *tmask;   // [T] cells touched since the last resolve (one array for both copies)
    uint32_t *cidx;              // [T] accumulator block of each touched tile (one array for both copies)
    uint32_t *tlist;             // [T] tile of each block
};

struct TileResolveArgs {
    TileArrays t;
    uint32_t tiles;              // T (a multiple of 32)
    unsigned long long *tmask;
    uint32_t *cidx;
    uint32_t *tlist;
    Counters *ctr;
    uint32_t res_stride;
    int f16;
    float alpha;
    uint32_t frame, stamp_now;   // frame and frame + 1
    uint32_t has_lr, lr, evict;  // previous resolve (for the no-history test) and E
    uint32_t min_samples;
    uint32_t *occ_out;
};

gi_status tile_update_launch(const TileUpdateArgs &a, int key_dir, int resident_blocks, cudaStream_t st);
gi_status tile_resolve_launch(const TileResolveArgs &a, int blocks, cudaStream_t st);
int tile_resolve_blocks_per_sm();
gi_status tile_query_points_launch(const TileUpdateArgs &a, const TileArrays &t, uint32_t res_stride, int f16,
                                   LiveRule rule, float4 *out, int blocks, int key_dir, cudaStream_t st);
gi_status tile_rebuild_launch(const TileArrays &from, const TileArrays &to, unsigned long long *tmask,
                              uint32_t res_bytes, uint32_t mask, uint32_t max_probe, LiveRule rule, Counters *ctr,
                              int blocks, cudaStream_t st);
gi_status tile_scan_launch(const TileArrays &t, const unsigned long long *tmask, uint32_t tiles, LiveRule rule,
                           unsigned long long *out, int blocks, cudaStream_t st);

// Grid of the interpolation: blocks of 32x16 pixels starting at (-4, -4), one 8x8-pixel region
// sharing a base tile per warp.
__host__ __device__ inline uint32_t interp_grid_x(uint32_t width) { return (width + 4u + 31u) / 32u; }
__host__ __device__ inline uint32_t interp_grid_y(uint32_t height) { return (height + 4u + 15u) / 16u; }

// Cache internals needed by the probe kernels.
struct CacheView {
    const void *resolved;      // resolved radiance of slot 0: float4, or half4 (ushort4)
    uint32_t resolved_stride;  // bytes between the resolved values of consecutive slots
    int resolved_f16;
    uint32_t slots;
};
CacheView cache_view(gi_cache_t c);

// Answers of the latest gi_nrc_query_frame for a view of n records (gi_nrc.cu).
gi_status nrc_override(gi_nrc_t nrc, uint64_t n, const uint32_t **bits, const float4 **ovr);

// Host helpers of the cache used by the batched pass chain (gi_cache.cu).
bool hits_ok(const gi_hits *h, uint32_t key_dir);
UpdateArgs cache_update_args(gi_cache_t c, const gi_hits *h, const gi_view *v, uint32_t *slot_ids);
gi_status cache_before_update(gi_cache_t c, cudaStream_t st);  // compaction check, counters
void cache_after_update(gi_cache_t c);
ResolveArgs cache_resolve_args(gi_cache_t c, uint32_t frame);
void cache_after_resolve(gi_cache_t c, uint32_t frame);
int cache_key_dir(const gi_cache_s *c);
bool cache_tiled(const gi_cache_s *c);
int cache_device(const gi_cache_s *c);
int64_t cache_last_resolved(const gi_cache_s *c);
gi_nrc_t cache_route_nrc(const gi_cache_s *c);  // the surrogate the cache routes far hits to, or NULL

// Blocks of a resident grid of `kernel` (threads per block, dynamic shared memory 0) on the
// current device, at most `items`.
template <typename K>
inline uint32_t resident_grid(K kernel, int threads, uint32_t items) {
    int dev = 0, sms = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    const uint32_t g = (uint32_t)(sms * (per_sm > 0 ? per_sm : 1));
    return items < g ? items : g;
}

// Launchers of the batched passes: one launch per pass over every view; args and prefix tables
// (nviews + 1 block-count prefixes) live in device memory.
uint32_t update_blocks_for(unsigned long long n, uint32_t records_per_block);
gi_status launch_update_batched(const UpdateArgs *args, const uint32_t *prefix, uint32_t nviews, uint32_t blocks,
                                int key_dir, cudaStream_t st);
gi_status launch_resolve_batched(const ResolveArgs *args, const uint32_t *prefix, uint32_t nviews, uint32_t blocks,
                                 cudaStream_t st);
gi_status launch_spawn_batched(const SpawnArgs *args, const uint32_t *prefix, uint32_t nviews, uint32_t blocks,
                               cudaStream_t st);
gi_status launch_integrate_batched(const IntegrateArgs *args, const uint32_t *prefix, uint32_t nviews,
                                   uint32_t blocks, uint32_t threads, uint32_t rays_per_probe, cudaStream_t st);
gi_status launch_interpolate_batched(const InterpArgs *args, const uint32_t *prefix, uint32_t nviews,
                                     uint32_t blocks, cudaStream_t st);

// Host helpers of the probe passes used by the batched pass chain (gi_probes.cu).
gi_status ensure_moments();
gi_status spawn_check(const gi_gbuffer *gbuf, const gi_view *view, const gi_probes *pr);
SpawnArgs spawn_args(const gi_gbuffer *gbuf, const gi_view *view, const gi_probes *pr);
gi_status integrate_check(gi_cache_t cache, const gi_probes *pr, const uint32_t *slot_ids, uint32_t rays_per_probe);
IntegrateArgs integrate_args(gi_cache_t cache, const gi_probes *pr, const uint32_t *slot_ids, uint32_t rpp,
                             const float env[3]);
gi_status interp_check(const gi_gbuffer *gbuf, const gi_view *view, const gi_probes *pr, const float *out);
InterpArgs interp_args(const gi_gbuffer *gbuf, const gi_view *view, const gi_probes *pr, float *out);

} // namespace gi

// ---------------------------------------------------------------- device helpers
namespace gi {

// View of a flat block index through the prefix table of per-view block counts (prefix[0] = 0,
// prefix[nviews] = total): the v with prefix[v] <= blk < prefix[v + 1].
__device__ __forceinline__ uint32_t view_of_block(const uint32_t *prefix, uint32_t nviews, uint32_t blk) {
    uint32_t lo = 0, hi = nviews;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= blk) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Persistent batched passes: a resident grid takes the flat work items of every view (the prefix
// table's blocks) one at a time from a counter that follows the prefix table (prefix[nviews + 1],
// zero when the pass starts), so that blocks that drew cheap items take more; a view's arguments
// are reloaded into shared memory only when an item belongs to another view than the last.  The
// body sees `item` (the view-local block) and `items` (the view's block count).
#define GI_BATCHED_ITEMS(prefix, nviews, sa, args, body)                                   \
    do {                                                                                 \
        __shared__ uint32_t s_w_;                                                        \
        const uint32_t total_ = __ldg((prefix) + (nviews));                              \
        uint32_t *ctr_ = const_cast<uint32_t *>(prefix) + (nviews) + 1;                  \
        uint32_t cur_ = 0xFFFFFFFFu;                                                     \
        for (;;) {                                                                       \
            if (threadIdx.x == 0) s_w_ = atomicAdd(ctr_, 1u);                            \
            __syncthreads();                                                             \
            const uint32_t w_ = s_w_;                                                    \
            if (w_ >= total_) break;                                                     \
            const uint32_t v_ = view_of_block((prefix), (nviews), w_);                   \
            if (v_ != cur_) {                                                            \
                load_view_args((sa), (args) + v_);                                       \
                __syncthreads();                                                         \
                cur_ = v_;                                                               \
            }                                                                            \
            const uint32_t p0_ = __ldg((prefix) + v_), p1_ = __ldg((prefix) + v_ + 1);   \
            const uint32_t item = w_ - p0_, items = p1_ - p0_;                           \
            (void)items;                                                                 \
            body;                                                                        \
            __syncthreads();                                                             \
        }                                                                                \
    } while (0)

// Copy one view's pass arguments from global to shared memory (whole block; sync after).
template <typename T>
__device__ __forceinline__ void load_view_args(T &dst, const T *src) {
    static_assert(sizeof(T) % 4 == 0, "argument structs are copied as 32-bit words");
    const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d = reinterpret_cast<uint32_t *>(&dst);
    for (uint32_t i = threadIdx.x; i < sizeof(T) / 4; i += blockDim.x) d[i] = __ldg(s + i);
}

// World position of pixel (x, y) at distance d along its camera ray, every operation in float32
// round-to-nearest in a fixed order (no contraction): probe positions and the reprojection's
// decisions are then reproducible bit for bit.
__device__ __forceinline__ float3 pixel_world_exact(const CamParams &c, uint32_t x, uint32_t y, float d) {
    const float sx = __fmul_rn(__fsub_rn(__fmul_rn(__fmul_rn(2.0f, __fadd_rn((float)x, 0.5f)), c.inv_w), 1.0f),
                               c.sx_scale);
    const float sy = __fmul_rn(__fsub_rn(1.0f, __fmul_rn(__fmul_rn(2.0f, __fadd_rn((float)y, 0.5f)), c.inv_h)),
                               c.sy_scale);
    const float dx = __fadd_rn(__fadd_rn(c.fwd[0], __fmul_rn(sx, c.right[0])), __fmul_rn(sy, c.up[0]));
    const float dy = __fadd_rn(__fadd_rn(c.fwd[1], __fmul_rn(sx, c.right[1])), __fmul_rn(sy, c.up[1]));
    const float dz = __fadd_rn(__fadd_rn(c.fwd[2], __fmul_rn(sx, c.right[2])), __fmul_rn(sy, c.up[2]));
    const float ln = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)));
    const float s = __fdiv_rn(d, ln);
    return make_float3(__fadd_rn(c.pos[0], __fmul_rn(dx, s)), __fadd_rn(c.pos[1], __fmul_rn(dy, s)),
                       __fadd_rn(c.pos[2], __fmul_rn(dz, s)));
}

__device__ __forceinline__ float3 cam_ray_dir(const CamParams &c, float x, float y) {
    // sx = (2(x+0.5)/W - 1) tan(fov/2) W/H, sy = (1 - 2(y+0.5)/H) tan(fov/2)
    float sx = (2.0f * (x + 0.5f) * c.inv_w - 1.0f) * c.sx_scale;
    float sy = (1.0f - 2.0f * (y + 0.5f) * c.inv_h) * c.sy_scale;
    float dx = c.fwd[0] + sx * c.right[0] + sy * c.up[0];
    float dy = c.fwd[1] + sx * c.right[1] + sy * c.up[1];
    float dz = c.fwd[2] + sx * c.right[2] + sy * c.up[2];
    float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
    return make_float3(dx * inv, dy * inv, dz * inv);
}

} // namespace gi

namespace gi {
// The trust test's inputs of a surrogate (gi_nrc.cu): device stats {loss, sum m|y - t|, sum m|t|},
// the trust threshold, and whether it has taken an Adam step.
void nrc_route_inputs(gi_nrc_t nrc, const float **stats, float *trust, bool *trained);
} // namespace gi
