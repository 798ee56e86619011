/*
 * gi.h -- C ABI of the world-space radiance cache and the screen-probe stage
 * of GI-1.0 (two-level radiance caching), GPU implementation for sm_103a.
 *
 * Scope: the world cache of Section 2.2 (a spatial hash of cells keyed by a
 * descriptor of the secondary vertex: quantised position, quantised
 * direction, distance LOD and the light-leak bit of Section 2.2.2; bucket
 * hash + fingerprint with linear probing; per-frame radiance accumulation;
 * resolve with an exponential moving average (Section 2.2.3) and decay of
 * untouched cells (Section 2.2.1); lookups for the screen-probe rays), and the
 * screen probes it feeds (spawn per 8x8 tile with a Halton jitter, Section
 * 2.1.1; probe mask + MIP chain and Algorithm 3, Section 2.1.5; probe
 * irradiance through 3-band spherical harmonics, Section 2.4.2; per-pixel
 * interpolation, Section 2.4.1).
 *
 * Conventions shared by every entry point:
 *  - Pointers named *device* point to CUDA device memory owned by the caller;
 *    the library reads/writes them asynchronously on the given stream.  The
 *    caller keeps them alive until the stream has passed the call.
 *  - Every call is asynchronous on `stream` (a cudaStream_t; 0 = the legacy
 *    default stream) and does not synchronise, except gi_cache_stats and
 *    gi_cache_export, which synchronise `stream`.
 *  - Arguments are validated on the host before anything is launched; a
 *    failed validation returns GI_ERR_INVALID_ARG and launches nothing.
 *    gi_last_error() then holds a message (per host thread).
 *  - Nothing on the device traps.  Device-side anomalies (dropped hits,
 *    bounded waits that ran out) are counted in device counters and surface
 *    at the next gi_cache_stats.
 *  - The library fails loudly: there is no CPU fallback.  Without a usable
 *    CUDA device every launching call returns GI_ERR_CUDA.
 */
#ifndef GI_H
#define GI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gi_status {
    GI_OK = 0,
    GI_ERR_INVALID_ARG = 1,   /* bad pointer, size, alignment or configuration */
    GI_ERR_OOM = 2,           /* device or pinned-host allocation failed */
    GI_ERR_CUDA = 3,          /* a CUDA runtime call failed (no device, launch error, ...) */
    GI_ERR_TIMEOUT = 4,       /* a bounded device-side wait ran out */
    GI_ERR_DEVICE_FAULT = 5,  /* the device error word is set */
    GI_ERR_CAPACITY = 6,      /* an export buffer is too small */
    GI_WARN_DROPPED = 100     /* stats: some hits found no slot within max_probe (table too full) */
} gi_status;

/* Slot-id codes written by gi_cache_update for records that do not name a cell. */
#define GI_SLOT_MISS 0xFFFFFFFEu  /* the ray left the scene: its radiance is the environment */
#define GI_SLOT_NONE 0xFFFFFFFFu  /* no sample: invalid record, or a hit dropped for lack of a slot */
#define GI_SLOT_FAR 0xFFFFFFFDu   /* a far hit left to the surrogate (gi_cache_route_far): no cell */

/* Probe-mask sentinel of a tile without probe (Section 2.1.5). */
#define GI_PROBE_NONE 0xFFFFFFFFu

/* Per-pixel flags written in the alpha channel by gi_probes_interpolate (Section 2.4.1). */
#define GI_INTERP_OK 0       /* edge-aware weighted average */
#define GI_INTERP_RELAXED 1  /* every weight was zero: equal weights over the neighbours found */
#define GI_INTERP_NONE 2     /* no neighbour probe found: irradiance 0 */
#define GI_INTERP_SKY 3      /* the pixel sees no surface: irradiance 0 */

enum { GI_KEY_DIR_NORMAL = 0, GI_KEY_DIR_RAY = 1 };
enum { GI_RESOLVED_F32 = 0, GI_RESOLVED_F16 = 1 };
enum { GI_FIRST_TOUCH_AUTO = 0, GI_FIRST_TOUCH_LIST = 1, GI_FIRST_TOUCH_BITMAP = 2 };
enum { GI_MERGE_NONE = 0, GI_MERGE_WARP = 1 };

typedef struct gi_cache_s *gi_cache_t;
typedef void *gi_stream_t; /* cudaStream_t */

/*
 * Cache configuration.
 *   log2_slots      table size N = 2^log2_slots slots, 10..28
 *   cell_size       s0: side of a LOD-0 cell in world units (> 0)
 *   num_lods        distance LODs 1..4; LOD l has side s0 * 2^l and is used
 *                   where the screen-space cell size of Algorithm 6 is in
 *                   [s0 2^l, s0 2^(l+1)) (the last LOD takes everything above)
 *   alpha           blend weight of a new frame mean, (0, 1]
 *   evict_frames    E >= 1: a cell untouched at E consecutive resolves is evicted
 *   max_probe       longest linear-probing run, 1..255
 *   key_dir         GI_KEY_DIR_NORMAL: direction term from the surface normal;
 *                   GI_KEY_DIR_RAY: from the outgoing direction (minus the ray)
 *   resolved_format GI_RESOLVED_F32 (16 B per slot) or GI_RESOLVED_F16 (8 B)
 *   rebuild_load    fraction of slots occupied (live + stale cells) above which the
 *                   next update first compacts the table, in [0.25, 0.95]
 *   first_touch     how the update accumulates and records the slots touched since the
 *                   last resolve: GI_FIRST_TOUCH_LIST (per group of same-cell records of a warp,
 *                   three 64-bit additions and a returning count addition; the first toucher of
 *                   a slot appends it to a list, staged per block), GI_FIRST_TOUCH_BITMAP (the
 *                   group's sums and count in one 32-byte bulk reduction from shared memory,
 *                   cp.reduce.async.bulk, and a non-returning set of the slot's bit in a bitmap
 *                   of one bit per slot that the resolve walks in slot order: fewer L2
 *                   operations per record), or GI_FIRST_TOUCH_AUTO (the bitmap).  Results are
 *                   identical.
 *   tiles           0: a slot holds one cell.  1: two-level cache of Section 2.2.3 ("Prefiltering
 *                   Radiance"): a slot holds a tile of 8 x 8 cells on the plane that drops the
 *                   direction code's axis (in-plane cell coordinates floor-divided by 8 form the
 *                   tile descriptor, their remainders (u mod 8) + 8 (v mod 8) the cell), plus
 *                   box-filtered MIP levels 4x4, 2x2 and 1x1 rebuilt at every resolve that
 *                   touches the tile.  log2_slots then counts tiles (10..22); slot ids are
 *                   tile slot * 64 + cell; first_touch must be AUTO (a tile cache records the
 *                   cells touched since the last resolve in a 64-bit mask per tile).
 *   min_samples     tiles only, >= 1: a cell answers queries from the finest of its levels
 *                   (the cell, then its 4x4, 2x2 and 1x1 ancestors) whose sample count reaches
 *                   min_samples, else from the 1x1 level.  The sample count of a cell is the
 *                   number of samples blended into it since it last started without history;
 *                   a MIP value averages its children that hold a value and sums their counts.
 *   merge           GI_MERGE_NONE: every hit record is inserted and accumulated on its own (records
 *                   of one cell add into its accumulator in separate reductions; the integer sums
 *                   are the same).  GI_MERGE_WARP: the hits of a warp (32 consecutive records) that
 *                   name the same cell are merged first (__match_any_sync), so one of them probes
 *                   and accumulates for all.  Results are identical; the merge pays only where
 *                   consecutive records share cells.  Ignored by tile caches and by
 *                   gi_batch_frame, whose update never merges.
 */
typedef struct gi_cache_config {
    uint32_t log2_slots;
    float cell_size;
    uint32_t num_lods;
    float alpha;
    uint32_t evict_frames;
    uint32_t max_probe;
    uint32_t key_dir;
    uint32_t resolved_format;
    float rebuild_load;
    uint32_t first_touch;
    uint32_t tiles;
    uint32_t min_samples;
    uint32_t merge;
} gi_cache_config;

/*
 * View of a frame: pinhole camera at cam_pos looking along cam_fwd with unit
 * cam_right / cam_up; the ray through pixel (x, y) (row 0 on top) has
 * direction normalize(fwd + sx right + sy up), sx = (2(x+0.5)/W - 1) tan(fov_y/2) W/H,
 * sy = (1 - 2(y+0.5)/H) tan(fov_y/2).  fov_y and the size also give the
 * screen-space cell size of Algorithm 6.  frame is the frame index (monotone).
 */
typedef struct gi_view {
    uint32_t frame;
    uint32_t width, height;
    float cam_pos[3];
    float cam_fwd[3];
    float cam_right[3];
    float cam_up[3];
    double fov_y; /* radians */
} gi_view;

/*
 * Hit records, structure of arrays, n records; each pointer is a device array
 * of n float32 (any 4-byte alignment).  Record i is a hit when ray_len[i] is
 * finite and >= 0 and pos is finite; ray_len = +inf marks a ray that left the
 * scene; anything else (negative, NaN) marks no sample.  ray_dir is the unit
 * probe-ray direction and is read only with GI_KEY_DIR_RAY (else may be NULL).
 */
typedef struct gi_hits {
    const float *pos[3];
    const float *nrm[3];
    const float *rad[3];
    const float *ray_len;
    const float *ray_dir[3];
    uint64_t n;
} gi_hits;

/* G-buffer: device float4 per pixel (nx, ny, nz, distance along the pixel ray;
 * +inf = sky), row-major height x width, 16-byte aligned. */
typedef struct gi_gbuffer {
    const float *nd;
    uint32_t width, height;
} gi_gbuffer;

#define GI_MAX_MIPS 16
#define GI_SH_STRIDE 28 /* floats per probe: 9 coefficients x RGB (k*3 + c), 1 pad */

/* Layout of the probe buffers of a width x height view (filled by gi_probes_layout). */
typedef struct gi_probe_layout {
    uint32_t tiles_x, tiles_y, num_probes, mip_count;
    uint32_t mip_w[GI_MAX_MIPS], mip_h[GI_MAX_MIPS], mip_offset[GI_MAX_MIPS];
    uint32_t mask_words; /* total u32 words of all mask levels */
} gi_probe_layout;

/*
 * Probe buffers (device, caller-owned, sized by gi_probe_layout):
 *   mask  u32[mask_words]: level k at mip_offset[k], mip_w[k] x mip_h[k] row-major;
 *         a probe is packed as y << 16 | x (its pixel), GI_PROBE_NONE if absent
 *   pos   float4[num_probes]: world position, distance along the pixel ray
 *   nrm   float4[num_probes]: unit normal, w = 1 for a probe, 0 for none
 *   sh    float[num_probes * GI_SH_STRIDE]: SH coefficients of the probe radiance
 * Probe p is the probe of tile (p mod tiles_x, p / tiles_x).
 */
typedef struct gi_probes {
    gi_probe_layout layout;
    uint32_t *mask;
    float *pos;
    float *nrm;
    float *sh;
} gi_probes;

/* Cumulative counters and table state (gi_cache_stats).  In a tile cache slots, occupied and
 * touched count tiles, live counts cells. */
typedef struct gi_cache_stats_t {
    uint64_t slots;           /* N */
    uint64_t occupied;        /* slots holding a cell (tile), live or stale */
    uint64_t live;            /* cells not evicted as of the last resolve, plus cells touched since */
    uint64_t touched;         /* cells (tiles) touched since the last resolve */
    uint64_t dropped;         /* hits that found no slot within max_probe (cumulative) */
    uint64_t clamped;         /* hit records whose radiance was clamped to [0, 32768] or was NaN */
    uint64_t rebuilds;        /* table compactions so far */
    uint64_t updates, resolves;
    uint32_t max_probe_seen;  /* longest probing run so far */
    uint32_t error_word;      /* device error word (0 = none) */
    int64_t last_resolved;    /* frame of the last resolve, -1 before the first */
} gi_cache_stats_t;

/* One live cell, as exported by gi_cache_export (host memory).  In a tile cache the identity is
 * (tile's home slot << 24 | tile fingerprint) << 6 | cell, value is the cell's own blended
 * radiance (level 0) and slot is tile slot * 64 + cell. */
typedef struct gi_cell {
    uint64_t identity;  /* home slot << 24 | 24-bit fingerprint */
    uint64_t sum[3];    /* fixed-point sums accumulated since the last resolve (2^-24 units) */
    uint32_t count;     /* samples accumulated since the last resolve */
    uint32_t stamp;     /* 1 + last frame this cell was resolved with samples; 0 = never */
    float value[3];     /* resolved radiance */
    uint32_t slot;      /* current slot index (changes when the table is compacted) */
} gi_cell;

/* One tile of a tile cache with at least one live cell, as exported by gi_cache_export_tiles
 * (host memory).  Values 0..63 are the cells (level 0, cell (i, j) at i + 8 j), 64..79 the 4x4
 * level, 80..83 the 2x2 level, 84 the 1x1 level; level k + 1 value (i, j) covers level-k values
 * (2i + di, 2j + dj).  samples = 0 marks a value that holds nothing (a cell not live, a MIP value
 * without live cell below it).  Levels 1..3 are those of the last resolve that touched the tile. */
#define GI_TILE_VALUES 85
typedef struct gi_tile {
    uint64_t identity;                 /* home slot << 24 | 24-bit fingerprint of the tile */
    uint32_t slot;                     /* tile slot */
    uint32_t live;                     /* live cells */
    float value[GI_TILE_VALUES][3];
    uint32_t samples[GI_TILE_VALUES];
} gi_tile;

/* ---------------------------------------------------------------- errors */
/* Message of the last failed call on this host thread ("" if none). */
const char *gi_last_error(void);
/* Name of a status code. */
const char *gi_status_string(gi_status s);
/* Library version, major * 10000 + minor * 100 + patch. */
uint32_t gi_version(void);

/* ---------------------------------------------------------------- world cache */
/*
 * Create a cache (Section 2.2.1): allocates the slot table (fingerprints,
 * 32-byte fixed-point accumulators, resolved radiance), a spare table for
 * compaction, the record of touched slots (a bitmap of one bit per slot, or a
 * touch list of 4 bytes per slot in the list form) and counters, on the
 * current CUDA device.  The library owns this memory until gi_cache_destroy.
 * Synchronous.
 * Errors: GI_ERR_INVALID_ARG (cfg out of range), GI_ERR_OOM, GI_ERR_CUDA.
 */
gi_status gi_cache_create(const gi_cache_config *cfg, gi_cache_t *out);

/* Free every resource of the cache (synchronises the device first). NULL is a no-op. */
gi_status gi_cache_destroy(gi_cache_t cache);

/*
 * Accumulate one batch of hit records into the cache (Sections 2.2.1-2.2.3):
 * per hit, the cell descriptor (quantised position, dominant-axis direction,
 * distance LOD from Algorithm 6's cell size, light-leak bit), bucket hash +
 * fingerprint, linear probing with atomicCAS on the fingerprint to find or
 * insert the cell, then 64-bit fixed-point sums round(r * 2^24) per channel
 * and a sample count (see first_touch for the two forms of the accumulation and
 * merge for the optional merge of a warp's same-cell hits).  Between two
 * resolves a cell takes fewer than 2^32 records (its 32-bit count) and sums
 * below 2^64 (2^25 records at the clamp radiance 32768): the records of many
 * frames, far above what a frame brings.  slot_ids (device, n u32,
 * caller-owned) receives each record's slot, GI_SLOT_MISS or GI_SLOT_NONE: the
 * cached index of Section 2.2.1, valid until the next gi_cache_update.
 * Several updates may precede one resolve.
 * If the previous resolve left the table fuller than rebuild_load, this call
 * first compacts it (live cells only; slot indices change).
 * Errors: GI_ERR_INVALID_ARG (NULL record plane, NULL slot_ids with n > 0,
 * view size 0, non-positive fov), GI_ERR_CUDA.
 */
gi_status gi_cache_update(gi_cache_t cache, const gi_hits *hits, const gi_view *view, uint32_t *slot_ids,
                          gi_stream_t stream);

/*
 * Resolve the frame (Section 2.2.3 and the decay rule of Section 2.2.1): for
 * every cell touched since the last resolve, mean m = sum / (count 2^24);
 * a cell without history (new, or evicted earlier) takes v = m, others
 * v <- v + alpha (m - v); accumulators are cleared and the cell's stamp set to
 * this frame.  Cells whose last touch is E or more frames before `frame` are
 * evicted (they stay in the table until the next compaction but no longer
 * answer queries, and restart without history if hit again).  A tile cache
 * then rebuilds the MIP levels of every tile touched since the last resolve
 * and stores, for each of its live cells, the value of the level that answers
 * it (see min_samples): the resolved radiance that queries by slot return.
 * Errors: GI_ERR_INVALID_ARG (frame earlier than the previous resolve), GI_ERR_CUDA.
 */
gi_status gi_cache_resolve(gi_cache_t cache, uint32_t frame, gi_stream_t stream);

/*
 * Query the cache (Section 2.1.3: the radiance returned to a probe ray).
 * By slot: slot_ids (device, n) as written by gi_cache_update; out (device float4[n])
 * = (r, g, b, 1) for a slot, (env, 1) for GI_SLOT_MISS, (0, 0, 0, 0) for GI_SLOT_NONE.
 * By point: hits (device, n records) + view; descriptor lookup without insertion;
 * out = (r, g, b, 1) for a live cell, (0, 0, 0, 0) otherwise (a miss of the cache).
 */
typedef struct gi_query {
    const uint32_t *slot_ids; /* by slot when non-NULL */
    const gi_hits *points;    /* by point when slot_ids is NULL */
    const gi_view *view;      /* by point: camera and view size for the descriptor */
    uint64_t n;
    float env[3];
} gi_query;
gi_status gi_cache_query(gi_cache_t cache, const gi_query *q, float *out, gi_stream_t stream);

/*
 * Counters and table state.  Synchronises `stream`, then scans the table.
 * Returns GI_WARN_DROPPED when hits were dropped, GI_ERR_DEVICE_FAULT when the
 * device error word is set (stats are filled in both cases).
 */
gi_status gi_cache_stats(gi_cache_t cache, gi_cache_stats_t *out, gi_stream_t stream);

/*
 * Copy every live cell (see gi_cache_stats_t.live) to host memory, sorted by
 * identity.  Synchronises `stream`.  *count receives the number of live cells;
 * if it exceeds capacity nothing is written and GI_ERR_CAPACITY is returned.
 * out may be NULL with capacity 0 to ask for the count.
 */
gi_status gi_cache_export(gi_cache_t cache, gi_cell *out, uint64_t capacity, uint64_t *count, gi_stream_t stream);

/*
 * Tile caches: copy every tile holding a live cell, with its levels, to host memory, sorted by
 * identity.  Synchronises `stream`.  Count and capacity as for gi_cache_export.
 * Errors: GI_ERR_INVALID_ARG (not a tile cache, NULL argument), GI_ERR_CAPACITY, GI_ERR_CUDA.
 */
gi_status gi_cache_export_tiles(gi_cache_t cache, gi_tile *out, uint64_t capacity, uint64_t *count,
                                gi_stream_t stream);

/* ---------------------------------------------------------------- screen probes */
/* Probe buffer sizes of a width x height view (host only, no device access). */
gi_status gi_probes_layout(uint32_t width, uint32_t height, gi_probe_layout *out);

/*
 * Spawn one probe per 8x8 tile (Section 2.1.1, upscale 1x1): the pixel
 * 8 * tile + j, j = (floor(8 H_2(f+1)), floor(8 H_3(f+1))) the Halton point of
 * frame f shared by every tile, clamped to the image; no probe on a sky pixel.
 * Writes mask level 0 and its MIP chain (Section 2.1.5: first valid probe of
 * each 2x2 block in the order (0,0), (1,0), (0,1), (1,1)), positions rebuilt
 * from the G-buffer distance and the camera, normals from the G-buffer.
 * Positions: the camera ray through the pixel centre times the distance, in
 * float32 round-to-nearest operations in a fixed order (sx = (2(x+0.5)/W - 1)
 * tan(fov/2) W/H, sy = (1 - 2(y+0.5)/H) tan(fov/2), dir = (fwd + sx right) + sy up,
 * world = cam + dir (d / |dir|)), so that they are reproducible bit for bit.
 * `probes` must have been laid out for the view size.
 */
gi_status gi_probes_spawn(const gi_gbuffer *gbuf, const gi_view *view, const gi_probes *probes, gi_stream_t stream);

/* ---------------------------------------------------------------- temporal path */
#define GI_MAX_UPSCALE 8

/*
 * Spawn with temporal upscale u (Section 2.1.1, "Temporal Upscale"): spawn tiles of 8u x 8u
 * pixels share the jitter j = (floor(8u H_2(f+1)), floor(8u H_3(f+1))); the probe pixel of spawn
 * tile S is min(8u S + j, (W-1, H-1)) and the 8x8 tile containing it receives a fresh probe
 * (position and normal as gi_probes_spawn) unless the pixel is sky.  keep = 0: every other tile
 * gets no probe (u = 1, keep = 0 is gi_probes_spawn).  keep != 0: every other tile, and a tile
 * whose spawn pixel is sky, keeps its level-0 mask, position and normal (those written by
 * gi_probes_reproject).  Then the MIP chain.  1 <= u <= GI_MAX_UPSCALE.
 * The frame's hit records belong to the spawn tiles, row by row: probe S traces records
 * S * rays_per_probe ... (S + 1) * rays_per_probe - 1.
 */
gi_status gi_probes_spawn_upscaled(const gi_gbuffer *gbuf, const gi_view *view, uint32_t upscale, uint32_t keep,
                                   const gi_probes *probes, gi_stream_t stream);

/*
 * Screen-probe reprojection (Algorithm 1) into `cur` from the previous frame's probes `prev`
 * (same layout, distinct buffers).  motion: device float2 per pixel (row-major, 8-byte aligned),
 * the offset in pixels from the pixel centre to where its surface point was in the previous
 * frame.  Per 8x8 tile, each non-sky pixel p looks up q = floor(p + 0.5 + motion(p)); if q is in
 * the image and the previous level-0 mask has a probe at q's tile, that probe bids when
 * |dot(pos_probe - pos_p, n_p)| < cell_size(d_p) (Algorithm 6's distance_scale x d_p) and
 * dot(n_probe, n_p) > 0.95, with the score (half(|pos_probe - pos_p|) << 16) | lane, lane =
 * 8 ly + lx; the smallest score places the tile's probe on its pixel (position and normal of that
 * pixel), src[tile] = the previous probe's index.  A tile without bid gets no probe and
 * src = GI_PROBE_NONE.  All decisions in float32 round-to-nearest operations (positions as in
 * gi_probes_spawn).  Writes cur's level-0 mask, pos, nrm; the MIP chain comes with the spawn
 * that follows (gi_probes_spawn_upscaled with keep).  src: device u32[num_probes].
 */
gi_status gi_probes_reproject(const gi_gbuffer *gbuf, const gi_view *view, const float *motion,
                              const gi_probes *prev, const gi_probes *cur, uint32_t *src, gi_stream_t stream);

/*
 * The frame's probe atlas (float4[num_probes * 64], (radiance rgb, mean hit distance)) for the
 * temporal path.  A tile whose fresh probe exists this frame (see gi_probes_spawn_upscaled)
 * gathers its spawn tile's rays as gi_probes_gather does; when src[tile] names a previous probe,
 * each cell's radiance is then blended with that probe's same cell in prev_atlas by the biased
 * temporal hysteresis of Algorithm 4 (l = mean of rgb; alpha = max(l1 - l2 - min(l1, l2), 0) /
 * max(l1, l2, 1e-4), clamped to [0, 0.95] and squared; lerp(current, previous, alpha)), keeping
 * the fresh hit distance.  A tile with a reprojected probe and no fresh one copies the source's
 * 64 cells; a tile with neither gets zeros.  slot_ids / ray_len: the spawn tiles' records
 * (slot_ids 16-byte aligned).  prev_atlas and atlas are distinct, 16-byte aligned.  gi_probes_project then gives the SH.
 */
gi_status gi_probes_gather_temporal(gi_cache_t cache, const gi_gbuffer *gbuf, const gi_view *view, uint32_t upscale,
                                    const gi_probes *probes, const uint32_t *slot_ids, const float *ray_len,
                                    uint32_t rays_per_probe, const uint32_t *src, const float *prev_atlas,
                                    float *atlas, const float env[3], gi_stream_t stream);

/*
 * Probe irradiance (Sections 2.1.4, 2.4.2): ray k of probe p is record
 * p * rays_per_probe + k and samples hemi-octahedral cell k mod 64
 * (cell 8j + i covers u in [-1 + i/4, -1 + (i+1)/4], v likewise with j, in
 * the probe frame (t, b, n) of Duff et al. 2017; direction from (u, v):
 * x = (u+v)/2, y = (u-v)/2, z = 1 - |x| - |y|, normalised).  Each ray's
 * radiance is the cache's resolved value at its slot (the environment `env`
 * for GI_SLOT_MISS; no sample for GI_SLOT_NONE); per-cell means, with the
 * mean of populated cells copied into cells without sample; projection to 3
 * SH bands through exact per-cell direction moments.  Writes probes->sh.
 * rays_per_probe must be a positive multiple of 64; slot_ids 16-byte aligned (it is read 16 bytes
 * at a time; GI_ERR_INVALID_ARG otherwise).  Call after gi_cache_resolve.
 */
gi_status gi_probes_integrate(gi_cache_t cache, const gi_probes *probes, const uint32_t *slot_ids,
                              uint32_t rays_per_probe, const float env[3], gi_stream_t stream);

/*
 * The same probe irradiance in three passes, with the probe filter of Section 2.3 (Algorithm 5)
 * in between.  The probe atlas is a device float4 array of num_probes x 64 entries (16-byte
 * aligned, caller-owned): entry p * 64 + c = (radiance rgb, hit distance) of cell c of probe p.
 *
 * gi_probes_gather: per cell the mean radiance of its rays as in gi_probes_integrate (radiance
 * backup included) and the mean ray length of its rays that hit a surface (+inf when none did);
 * ray_len = the records' ray lengths (device, num_probes * rays_per_probe floats).  slot_ids
 * 16-byte aligned.  Zeros for a tile without probe.
 *
 * gi_probes_filter: one pass of the separable 7x7 sparse blur along axis 0 (x) or 1 (y) of the
 * probe grid: each cell is averaged with the same cell of the probes that Algorithm 3 finds at
 * steps -1, +1, -2, +2, -3, +3, skipping a neighbour farther than cell_size(d_p) (Algorithm 6)
 * from the probe's plane, a cell whose direction points behind the neighbour's normal, and a
 * neighbour whose hit point (at the smaller of the two hit distances) lies more than pi/50 off the
 * cell direction seen from the probe; weight 1 (the probe) and 1 / (1 + |d_p - d_q| / cell_size(d_p))
 * per accepted neighbour; the running hit distance is the weighted mean.  atlas_out must not alias
 * atlas_in.
 *
 * gi_probes_project: SH coefficients of every probe from its atlas into probes->sh, as
 * gi_probes_integrate does from the rays (gather + project == integrate).
 */
gi_status gi_probes_gather(gi_cache_t cache, const gi_probes *probes, const uint32_t *slot_ids, const float *ray_len,
                           uint32_t rays_per_probe, const float env[3], float *atlas, gi_stream_t stream);
gi_status gi_probes_filter(const gi_probes *probes, const gi_view *view, const float *atlas_in, float *atlas_out,
                           uint32_t axis, gi_stream_t stream);
gi_status gi_probes_project(const gi_probes *probes, const float *atlas, gi_stream_t stream);

/*
 * Per-pixel interpolation (Section 2.4.1): the four neighbours found by
 * Algorithm 3 at offsets (0,0), (1,0), (0,1), (1,1) from tile floor((pixel - 4) / 8);
 * weight = bilinear * max(0, n_p . n_q)^8 * max(0, 1 - plane_dist / cell_size(d_p));
 * irradiance E = sum w E_q(n_p) / sum w with E_q(n) = sum_lm A_l L_lm Y_lm(n),
 * A = (pi, 2pi/3, pi/4).  out: device float4 per pixel (E rgb, flag GI_INTERP_*).
 */
gi_status gi_probes_interpolate(const gi_gbuffer *gbuf, const gi_view *view, const gi_probes *probes, float *out,
                                gi_stream_t stream);

/* Per-cell direction moments used by gi_probes_integrate (host memory, 64 x 10
 * doubles: solid angle, first moment xyz, second moment xx yy zz xy xz yz; local
 * frame), computed in closed form for the spherical quadrilateral of each cell. */
gi_status gi_cell_moments(double *out640);

/* ---------------------------------------------------------------- many views per frame */
/*
 * The same pass chain for many independent views (each with its own cache, camera, G-buffer and
 * records) with one kernel launch per pass over all views: per frame, gi_batch_frame runs spawn,
 * update, resolve, probe irradiance and interpolation for every view, exactly as the single-view
 * calls gi_probes_spawn, gi_cache_update, gi_cache_resolve(resolve_frame), gi_probes_integrate and
 * gi_probes_interpolate would, with the same results.  With use_graph != 0 the launches are
 * captured into a CUDA graph the first time (and again whenever a view's size changes) on a
 * stream of the batch's own, then replayed on `stream`.
 */
#define GI_BATCH_MAX_VIEWS 256

typedef struct gi_batch_s *gi_batch_t;

/* Launch shapes, chosen by an autotuner (defaults: 2048, 3, 256). */
typedef struct gi_batch_tuning {
    uint32_t update_records_per_block; /* records per update block, multiple of 256 in [256, 2048] */
    uint32_t resolve_blocks_per_sm;    /* resolve blocks per SM over all views, 1..4 */
    uint32_t integrate_threads;        /* threads per integrate block (four per probe), 32..128 */
} gi_batch_tuning;

/* One view of a frame.  All pointers are device pointers owned by the caller; hits.n must equal
 * probes.layout.num_probes * rays_per_probe; every cache of a batch uses the same key_dir and
 * holds cells, not tiles. */
typedef struct gi_batch_view {
    gi_cache_t cache;
    gi_view view;            /* view.frame drives the spawn jitter */
    uint32_t resolve_frame;  /* frame at which this view's cache is resolved (never decreasing) */
    gi_hits hits;
    gi_gbuffer gbuf;
    gi_probes probes;
    uint32_t *slot_ids;      /* 16-byte aligned */
    float *irradiance; /* float4 per pixel */
    float env[3];
} gi_batch_view;

/* Create a batch of n_views views (1..GI_BATCH_MAX_VIEWS); tuning may be NULL (defaults). */
gi_status gi_batch_create(uint32_t n_views, uint32_t rays_per_probe, const gi_batch_tuning *tuning, gi_batch_t *out);
/* Change the launch shapes (synchronises the device; captured graphs are dropped). */
gi_status gi_batch_set_tuning(gi_batch_t b, const gi_batch_tuning *tuning);
/* Run one frame of every view (views: n_views entries).  Asynchronous on stream. */
gi_status gi_batch_frame(gi_batch_t b, const gi_batch_view *views, uint32_t use_graph, gi_stream_t stream);
gi_status gi_batch_destroy(gi_batch_t b);

/* ---------------------------------------------------------------- learned radiance surrogate */
/*
 * An online-trained network that maps a hit (position, normal) to radiance.  The paper has no
 * learned part: its world cache answers every query from hash cells.  The surrogate is trained
 * on the cache's own resolved cells and answers the queries the cache serves worst: hits whose
 * insertion was dropped (GI_SLOT_NONE), hits on cells resolved for the first time (no history
 * yet), and hits at coarse LODs.  The cache stays the reference: the error of the network on its
 * latest training batch, measured against the cache's values, decides whether it answers at all.
 *
 * Model (published methods, not the paper's):
 *  - multiresolution hash encoding (Mueller et al. 2022): GI_NRC_LEVELS levels, level l a grid of
 *    resolution[l] cells per axis over the box [aabb_lo, aabb_hi] (positions are clamped into it);
 *    each level holds 2^log2_table entries of GI_NRC_FEATURES float16 features; the point's
 *    features are the trilinear interpolation of the 8 vertices of its cell; a vertex is
 *    addressed densely when 6 (resolution + 1)^3 <= 2^log2_table, else by the spatial hash
 *    x * 1 ^ y * 2654435761 ^ z * 805459861 ^ d * 2246822519 (mod 2^log2_table), where
 *    d in 0..5 is the normal's dominant axis and sign (the cell key's direction code);
 *  - a network 32 -> 64 -> ReLU -> 64 -> ReLU -> 3 without bias terms, bfloat16 weights and
 *    activations, float32 accumulation, on the tensor cores; radiance = max(output, 0);
 *  - loss over a batch of B samples: (1/B) sum_s m_s sum_c (y - t)^2 / (y^2 + loss_eps), with no
 *    gradient through the denominator (relative L2, Mueller et al. 2021); m_s = 0 skips a sample;
 *  - Adam with bias correction on float32 master copies of every parameter; on the table it is
 *    sparse: an entry no sample of the step touched (gradient exactly 0) keeps its value and its
 *    moments, as in PyTorch's SparseAdam.
 */
#define GI_NRC_LEVELS 16
#define GI_NRC_FEATURES 2
#define GI_NRC_HIDDEN 64
#define GI_NRC_OUTPUTS 3
#define GI_NRC_MAX_BATCH (1u << 20)

typedef struct gi_nrc_s *gi_nrc_t;

/*
 * Surrogate configuration.
 *   log2_table   entries per level, 2^10 .. 2^24
 *   resolution   cells per axis of each level, 1 .. 2^20
 *   aabb_lo/hi   box the positions are normalised into (hi > lo on every axis)
 *   lr, beta1, beta2, adam_eps   Adam (lr > 0, betas in [0, 1), eps >= 0)
 *   loss_eps     relative-L2 denominator term (> 0)
 *   batch        training samples per gi_nrc_train_frame, 128 .. GI_NRC_MAX_BATCH
 *   train_steps  minibatches (and Adam steps) those samples are split into; batch must be a
 *                multiple of train_steps with at least 128 samples per minibatch
 *   max_records  largest record count of a view passed to gi_nrc_train_frame / gi_nrc_query_frame
 *   max_queries  most records gi_nrc_query_frame answers per call (the rest keep the cache's value)
 *   trust        the network answers only while its L1 error on the latest training batch,
 *                relative to the targets' L1 norm, is at most trust (>= 0)
 *   query_lod    hits whose cell LOD is >= query_lod are answered by the network (>= 4: none)
 *   seed         parameter initialisation: table features uniform in [-1e-4, 1e-4], weights
 *                uniform in +-sqrt(6 / (fan_in + fan_out)), from a splitmix64 stream
 */
typedef struct gi_nrc_config {
    uint32_t log2_table;
    uint32_t resolution[GI_NRC_LEVELS];
    float aabb_lo[3], aabb_hi[3];
    float lr, beta1, beta2, adam_eps;
    float loss_eps;
    uint32_t batch;
    uint32_t train_steps;
    uint32_t max_records;
    uint32_t max_queries;
    float trust;
    uint32_t query_lod;
    uint64_t seed;
} gi_nrc_config;

/* Sample points (device planes of n float32, any 4-byte alignment). */
typedef struct gi_points {
    const float *pos[3];
    const float *nrm[3];
    uint32_t n;
} gi_points;

/* Counters of a surrogate (gi_nrc_stats). */
typedef struct gi_nrc_stats_t {
    uint64_t steps;        /* Adam steps taken */
    float loss;            /* loss of the latest gi_nrc_backward batch, or the mean over the
                              minibatches of the latest gi_nrc_train_frame */
    float judged_error;    /* sum m |y - t| / sum m |t| over those samples, each evaluated before
                              its own Adam step */
    uint32_t trusted;      /* judged_error <= trust and steps > 0 */
    uint32_t queries;      /* records answered by the latest gi_nrc_query_frame */
} gi_nrc_stats_t;

/* The library's defaults in every field of *cfg: log2_table 19; resolution[l] = floor(16 b^l),
 * b = (2048 / 16)^(1 / (GI_NRC_LEVELS - 1)), the last level exactly 2048 (a geometric schedule from
 * 16 to 2048 cells per axis, Mueller et al. 2022); the unit box [0, 1]^3; lr 1e-2, beta1 0.9, beta2
 * 0.99, adam_eps 1e-15; loss_eps 0.01; batch 65536 in 4 train_steps; max_records 2^22; max_queries
 * 2^20; trust 0.05; query_lod 2; seed 1.  Host only.  Errors: GI_ERR_INVALID_ARG for a NULL cfg. */
gi_status gi_nrc_config_defaults(gi_nrc_config *cfg);

/* Create (allocates every parameter, Adam state and scratch buffer; initialises from cfg->seed).
 * Synchronous.  Errors: GI_ERR_INVALID_ARG, GI_ERR_OOM, GI_ERR_CUDA. */
gi_status gi_nrc_create(const gi_nrc_config *cfg, gi_nrc_t *out);
gi_status gi_nrc_destroy(gi_nrc_t nrc);

/*
 * Parameters as float32 host arrays: table [GI_NRC_LEVELS][2^log2_table][2], w1 [64][32] (output
 * unit, encoded feature 2l + f), w2 [64][64], w3 [3][64].  set_params replaces the master copies
 * and resets Adam (moments and step count) and the gradient accumulators; any pointer may be
 * NULL to leave that part alone.  get_params copies the masters out.  Both synchronise the device.
 */
gi_status gi_nrc_set_params(gi_nrc_t nrc, const float *table, const float *w1, const float *w2, const float *w3);
gi_status gi_nrc_get_params(gi_nrc_t nrc, float *table, float *w1, float *w2, float *w3);
/* Gradient accumulators, same layouts (host arrays; NULL skips a part).  Synchronise the device. */
gi_status gi_nrc_set_gradients(gi_nrc_t nrc, const float *table, const float *w1, const float *w2, const float *w3);
gi_status gi_nrc_get_gradients(gi_nrc_t nrc, float *table, float *w1, float *w2, float *w3);

/* Radiance of n points: out (device float4[n]) = (max(y, 0), 1).  n <= GI_NRC_MAX_BATCH. */
gi_status gi_nrc_infer(gi_nrc_t nrc, const gi_points *pts, float *out, gi_stream_t stream);

/*
 * Loss gradients of one batch, added to the gradient accumulators (which an Adam step clears).
 * target: device planes [3][n] float32; mask: device float[n] of 0/1, or NULL for all 1;
 * batch_norm: B of the loss (0: B = n).  The loss and judged error go to gi_nrc_stats.
 */
gi_status gi_nrc_backward(gi_nrc_t nrc, const gi_points *pts, const float *const target[3], const float *mask,
                          uint32_t batch_norm, gi_stream_t stream);

/* One Adam step of every parameter from the gradient accumulators, which it then clears. */
gi_status gi_nrc_adam(gi_nrc_t nrc, gi_stream_t stream);

/*
 * Adam's step size (cfg.lr) for the Adam steps enqueued after the call, gi_nrc_adam's and
 * gi_nrc_train_frame's, so that a caller can lower it as training goes on (no counterpart in the
 * paper, which has no learned part).  Host only, no synchronisation.  Errors: GI_ERR_INVALID_ARG
 * for a NULL surrogate or a step size that is not finite and > 0.
 */
gi_status gi_nrc_set_learning_rate(gi_nrc_t nrc, float lr);

/*
 * Training on a view's resolved cells (call after gi_cache_resolve of the frame): sample
 * k < cfg.batch is record pcg(k ^ pcg(frame + 1)) mod hits->n (PCG hash: one LCG step with
 * multiplier 747796405 and increment 2891336453, then the RXS-M-XS output permutation); its
 * target is the cache's resolved radiance of the record's cell (slot_ids from gi_cache_update),
 * masked out for records without a cell.  Minibatch j = samples [j b, (j + 1) b), b = batch /
 * train_steps, each followed by its Adam step (loss normalised by b).
 */
gi_status gi_nrc_train_frame(gi_nrc_t nrc, gi_cache_t cache, const gi_hits *hits, const uint32_t *slot_ids,
                             uint32_t frame, gi_stream_t stream);

/*
 * Pick the records of a view the network answers and evaluate it there (call after
 * gi_cache_resolve and gi_nrc_train_frame): hits whose slot is GI_SLOT_NONE, hits on cells
 * resolved this frame for the first time, and hits whose cell LOD (the view's Algorithm 6
 * thresholds, as in the cell key) is >= cfg.query_lod -- only while the judged error of the
 * latest training batch is <= cfg.trust, and at most cfg.max_queries records.  The answers stay
 * in the surrogate for gi_probes_integrate_nrc.
 */
gi_status gi_nrc_query_frame(gi_nrc_t nrc, gi_cache_t cache, const gi_hits *hits, const uint32_t *slot_ids,
                             const gi_view *view, gi_stream_t stream);

/*
 * The records answered by the latest gi_nrc_query_frame, in increasing record order: records
 * (device u32[capacity]) and their radiance rad (device float4[capacity], (r, g, b, 1)); *count
 * (host) receives the number answered.  Synchronises `stream`.  GI_ERR_CAPACITY (nothing copied)
 * when count > capacity; NULL records and rad with capacity 0 ask for the count only.
 */
gi_status gi_nrc_answers(gi_nrc_t nrc, uint32_t *records, float *rad, uint32_t capacity, uint32_t *count,
                         gi_stream_t stream);

/* gi_probes_integrate with the radiance of the records picked by the latest gi_nrc_query_frame
 * taken from the network instead of the cache. */
gi_status gi_probes_integrate_nrc(gi_cache_t cache, gi_nrc_t nrc, const gi_probes *probes, const uint32_t *slot_ids,
                                  uint32_t rays_per_probe, const float env[3], gi_stream_t stream);

/* Counters (synchronises `stream`). */
gi_status gi_nrc_stats(gi_nrc_t nrc, gi_nrc_stats_t *out, gi_stream_t stream);

/*
 * Far hits to the surrogate instead of the table (no counterpart in the paper, whose far field is
 * the tile cache's MIP prefilter, Section 2.2.3).  From the next gi_cache_update of `cache` on,
 * while `nrc` is trusted (its judged error on its latest training batch within its trust, tested
 * by the update on the device, so that no call synchronises), hits whose cell LOD is >= far_lod
 * are neither inserted nor accumulated: their slot id is GI_SLOT_FAR, and gi_nrc_query_frame
 * answers every GI_SLOT_FAR record with the network (the plain probe pass treats them as rays
 * without sample).  The network keeps training on the cells the table still holds.  nrc NULL or
 * far_lod >= 4 ends the routing.  One-level caches only; in a batch, only with the view's
 * surrogate in the batch (gi_batch_set_surrogate, gi_batch_set_view_surrogates).  nrc must outlive
 * the routing.  Host only, no
 * synchronisation.  Errors: GI_ERR_INVALID_ARG for a NULL or tile cache.
 */
gi_status gi_cache_route_far(gi_cache_t cache, gi_nrc_t nrc, uint32_t far_lod);

/*
 * The surrogate in a batch (no counterpart in the paper): with nrc set, gi_batch_frame keeps the
 * far-hit routing of the views whose caches route to nrc (gi_cache_route_far), and its probe pass
 * becomes, view after view, gi_nrc_query_frame and gi_probes_integrate_nrc on the view's records
 * (the network's answer buffers hold one view at a time), with the same results as those calls;
 * the other passes stay one launch over all views.  That form runs without the CUDA graph
 * (use_graph is ignored).  nrc NULL restores the plain form; a view whose cache routes to another
 * surrogate than the batch's is rejected by gi_batch_frame.  Training stays the caller's
 * (gi_nrc_train_frame on any view's records).  nrc must outlive its use.  Host only.
 * Errors: GI_ERR_INVALID_ARG for a NULL batch.
 */
gi_status gi_batch_set_surrogate(gi_batch_t b, gi_nrc_t nrc);

/*
 * One surrogate per view (no counterpart in the paper), for views of different scenes, which one
 * network cannot share: nrcs is a host array of the batch's n_views handles (an entry may be NULL),
 * read during the call.  The probe pass of the views whose entry is NULL stays one launch over
 * them; each view v with a network takes gi_nrc_query_frame and gi_probes_integrate_nrc with
 * nrcs[v] on one of the batch's four internal streams, forked from `stream` after the resolve and
 * joined back before the interpolation: distinct networks run side by side, the views of one
 * network in view order on one stream (its answer buffers hold one view at a time).  The results
 * are those of the single-view calls.  The other passes stay one launch over all views, and the
 * form runs without the CUDA graph while any entry is set.  nrcs NULL restores
 * the plain form.  gi_batch_frame rejects a view whose cache routes far hits to a network other
 * than nrcs[v].  gi_batch_set_surrogate(b, nrc) is this call with every entry nrc.  Each network
 * must outlive its use.  Host only.  Errors: GI_ERR_INVALID_ARG for a NULL batch.
 */
gi_status gi_batch_set_view_surrogates(gi_batch_t b, const gi_nrc_t *nrcs);

/* ---------------------------------------------------------------- allocation-free variant */
/*
 * Per-record cell means of one batch, without allocating device memory.  The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc -- a renderer plugin whose
 * host engine owns the whole GPU memory budget, or a thread that must never block in the
 * allocator -- and so cannot create a cache with gi_cache_create.
 *
 * Result: out (device float4[n], caller-owned) = (mean radiance of the record's cell, 1) for a
 * hit, (env, 1) for a ray that left the scene (ray_len = +inf), (0, 0, 0, -1) for a hit whose cell
 * found no free slot within 255 slots of its bucket (dropped; at most GI_NOALLOC_MAX_RECORDS cells
 * in 2^GI_NOALLOC_LOG2_SLOTS slots make this very unlikely), (0, 0, 0, 0) for a record that is no
 * sample (non-finite position, negative or NaN ray length).  stats_out (device uint64[2],
 * caller-owned, 8-byte aligned, or NULL) receives, on `stream` after the means, the number of
 * dropped hits and the number of hits whose radiance was clamped to [0, 32768] before fixed-point
 * accumulation (the means of clamped hits use the clamped values).  It
 * equals gi_cache_create(log2_slots = GI_NOALLOC_LOG2_SLOTS, cell_size, num_lods, key_dir,
 * max_probe = 255) followed by gi_cache_update, gi_cache_resolve and gi_cache_query by slot on the
 * same records: the cell descriptor, fixed-point sums and float32 mean are the same, with no
 * temporal history (every call starts from an empty table).
 *
 * Scratch: one file-scope device array of GI_NOALLOC_SCRATCH_BYTES (about 10.5 MB) holds the
 * table, touch list, counters and slot ids.  Every GPU that loads the library holds it until the
 * process exits.  Each call clears the table and counters first, then overwrites the rest.  The
 * first call on a device looks the array's address up (cudaGetSymbolAddress, with that device
 * current) and caches it for the life of the process; make that first call before any stream
 * capture.  A device reset (cudaDeviceReset, or anything else that destroys the primary context)
 * unloads the module and leaves that cached address stale: do not call this entry point on a
 * device after its context was reset.  Every call on a device
 * shares the one array: calls that overlap on the GPU (other streams, other host threads) race
 * and give wrong results -- serialise them.  Calls no cudaMalloc, cudaFree or allocating library.
 *
 * Errors: GI_ERR_INVALID_ARG for n > GI_NOALLOC_MAX_RECORDS, a NULL plane or output, a bad view,
 * cell_size <= 0, num_lods outside 1..4, an unknown key_dir or a misaligned stats_out; GI_ERR_CUDA
 * if a launch fails.
 */
#define GI_NOALLOC_LOG2_SLOTS 18
#define GI_NOALLOC_MAX_RECORDS 131072u
#define GI_NOALLOC_SCRATCH_BYTES \
    ((4u + 32u + 4u) * (1u << GI_NOALLOC_LOG2_SLOTS) + 4u * GI_NOALLOC_MAX_RECORDS + 128u)
gi_status gi_cell_means_noalloc(const gi_hits *hits, const gi_view *view, float cell_size, uint32_t num_lods,
                                uint32_t key_dir, const float env[3], float *out, uint64_t *stats_out,
                                gi_stream_t stream);

/* ---------------------------------------------------------------- diagnostics
 * Not a step of the path.  gi_cache_update ends, per hit record (GI_MERGE_NONE), in L2
 * operations on the cell's 32-byte accumulator (Section 2.2.1's accumulation in 64-bit fixed
 * point): in the list form (GI_FIRST_TOUCH_LIST) three 64-bit additions of the sums and one
 * returning 32-bit addition of the count, whose old value flags the first touch; in the bitmap
 * form (GI_FIRST_TOUCH_BITMAP, and AUTO) one 32-byte bulk reduction of the sums and count from
 * shared memory and a non-returning set of the slot's bit.  gi_diag_update_atomics issues exactly
 * those operations of the given form for n slot ids (records with slot_ids[i] >= 2^log2_slots are
 * skipped; one reduction per record, as the update without merge) and nothing else: no record
 * stream, key, probe or slot-id store.  Timed beside gi_cache_update on the same frame's slot ids
 * it gives the floor of the update's accumulation on this GPU.
 *   slot_ids       device uint32[n] (4-byte aligned), e.g. the slot_ids_out of an update
 *   first_touch    the form: GI_FIRST_TOUCH_LIST, GI_FIRST_TOUCH_BITMAP or AUTO (the bitmap)
 *   scratch        device, caller-owned, zeroed by the caller, 32-byte aligned: 2^log2_slots
 *                  32-byte accumulators (receiving sums 1, 2, 3 and count 1 per record), followed
 *                  in the bitmap form by the bitmap, 2^log2_slots / 8 bytes
 *   first_touches  list form: device uint32 (caller-owned), incremented by the number of slots
 *                  whose count left 0; unused (may be NULL) in the bitmap form
 * Errors: GI_ERR_INVALID_ARG for log2_slots outside [10, 30], an unknown form, a NULL or
 * misaligned buffer. */
gi_status gi_diag_update_atomics(const uint32_t *slot_ids, uint64_t n, uint32_t log2_slots, uint32_t first_touch,
                                 void *scratch, uint32_t *first_touches, gi_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* GI_H */
