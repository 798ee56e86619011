// Two-level world cache (Section 2.2.3, "Prefiltering Radiance"): the hash table indexes tiles of
// 8 x 8 cells instead of single cells, and every resolve that touches a tile rebuilds its
// box-filtered MIP levels (4x4, 2x2, 1x1) after the temporal blend.  A cell then answers from the
// finest of its levels that holds at least min_samples samples.
//
// Tile descriptor: the cell descriptor's LOD, leak bit and direction code; of the quantised
// position, the two coordinates on the plane that drops the direction code's axis (in increasing
// axis order u, v) floor-divided by 8 (16 bits each) and the main-axis coordinate (19 bits).  The
// cell inside the tile is (u mod 8) + 8 (v mod 8), so a surface facing one axis fills its tiles
// densely.
//
// Layout (T tile slots, cell e = slot * 64 + cell):
//   tags     u32[T]          tile fingerprint << 8 | (home mod 256); 0 = empty
//   tmask    u64[T]          cells touched since the last resolve (set by the update, walked in
//                            slot order and cleared by the resolve: the touched tiles are its
//                            non-zero words)
//   omask    u64[T]          cells live after the last resolve that touched the tile (a superset of
//                            its live cells until the next one: cells only die without a touch)
//   cidx     u32[T]          accumulator block of a tile touched since the last resolve, in the
//                            order the update handed them out; GI_SLOT_NONE otherwise
//   accum    Accum[T * 64]   block b holds the fixed-point sums and counts of the 64 cells of the
//                            tile whose cidx is b, since the last resolve
//   stamp    u32[T * 64]     1 + frame of the last resolve that found samples; 0 = never
//   state    float4[T * 64]  blended radiance, w = samples since the cell last started without history
//   resolved [T * 64]        the answer of each live cell (float4 or half4; w = resolved without history)
//   mips     float4[T * 21]  levels 1..3 (16 + 4 + 1 values), w = summed sample count, 0 = no value
//   tlist    u32[T]          the touched tiles in block order (entry b = the tile of block b)
// The per-cell arrays of one tile are contiguous.  The update issues no returning atomic but one
// counter add per CTA of the compaction: sums, counts and the touched bit are reductions.  The
// resolve of a tile is one warp that issues the loads of all its cells at once: 256 B of stamps,
// the state of the cells in omask | tmask, the accumulators of the touched cells.
#include <algorithm>

#include "gi_cache_dev.cuh"

namespace gi {

// Tile descriptor and cell index of a record (the cell descriptor's float ops, in the same order).
__device__ __forceinline__ unsigned long long tile_key(const KeyParams &k, float px, float py, float pz, float sx,
                                                       float sy, float sz, float len, uint32_t flip, uint32_t &cell) {
    const int lod = key_lod(k, px, py, pz);
    const float inv = pick4(k.inv_side, lod);
    const float side = pick4(k.side, lod);
    const int qx = __float2int_rd(__fmul_rn(px, inv));
    const int qy = __float2int_rd(__fmul_rn(py, inv));
    const int qz = __float2int_rd(__fmul_rn(pz, inv));
    const unsigned long long leak = (len < side) ? 1ull : 0ull;
    const float ax = fabsf(sx), ay = fabsf(sy), az = fabsf(sz);
    const int axis = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
    const float comp = axis == 0 ? sx : (axis == 1 ? sy : sz);
    const uint32_t sgn = (__float_as_uint(comp) >> 31) ^ flip;
    const unsigned long long code = (unsigned long long)(2 * axis + (int)sgn);
    const int qu = axis == 0 ? qy : qx;
    const int qv = axis == 2 ? qy : qz;
    const int qw = axis == 0 ? qx : (axis == 1 ? qy : qz);
    cell = (uint32_t)(qu & 7) + 8u * (uint32_t)(qv & 7);
    const unsigned long long tu = (uint32_t)(qu >> 3) & 0xFFFFu;
    const unsigned long long tv = (uint32_t)(qv >> 3) & 0xFFFFu;
    const unsigned long long w = (uint32_t)qw & kQMask;
    return ((unsigned long long)lod << 61) | (leak << 60) | (code << 57) | (tu << 35) | (tv << 19) | w;
}

__device__ __forceinline__ uint32_t sat_add(uint32_t a, uint32_t b) { return a > 0xFFFFFFFFu - b ? 0xFFFFFFFFu : a + b; }

// ---------------------------------------------------------------- update
// Three launches.  (1) k_tile_key: per record the tile descriptor, bucket + fingerprint of the
// tile and the cell; the leader of each group of same-cell hits in a warp finds or inserts the
// tile by linear probing and sets the cell's bit in the tile's touched mask (a reduction); the
// record's slot id is tile slot * 64 + cell.  (2) k_tile_compact: every tile touched since the
// last resolve that has no accumulator block yet gets the next one (a per-frame index, cidx).
// (3) k_tile_accumulate: per record the fixed-point radiance, merged per cell within the warp
// and added into the cell's accumulator of its tile's block with one 32-byte bulk reduction.  The accumulator
// blocks of one frame are contiguous (touched tiles x 2 KB), so the reductions of a frame span
// that range only, not the whole table: the cost of scattered reductions grows with the span.
template <int KEY_DIR>
__global__ void __launch_bounds__(kUpdThreads, 8) k_tile_key(TileUpdateArgs ta) {
    const UpdateArgs &a = ta.u;
    __shared__ uint32_t s_clamped, s_maxp, s_new;
    if (threadIdx.x == 0) {
        s_clamped = 0;
        s_maxp = 0;
        s_new = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * kUpdThreads;
    uint32_t my_clamped = 0, my_maxp = 0, my_new = 0;
    unsigned long long my_dropped = 0;
    for (unsigned long long base = (unsigned long long)blockIdx.x * kUpdThreads; base < a.n; base += stride) {
        const unsigned long long i = base + threadIdx.x;
        const bool inr = i < a.n;
        // the key's planes of an in-range record in one round trip; the radiance is read by
        // k_tile_accumulate, which also counts its clamps (here only those of dropped hits)
        float len = -1.0f, px = 0.f, py = 0.f, pz = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
        if (inr) {
            len = __ldcs(a.len + i);
            px = __ldcs(a.p[0] + i);
            py = __ldcs(a.p[1] + i);
            pz = __ldcs(a.p[2] + i);
            const float *const *sd = KEY_DIR == GI_KEY_DIR_NORMAL ? a.nrm : a.dir;
            sx = __ldcs(sd[0] + i);
            sy = __ldcs(sd[1] + i);
            sz = __ldcs(sd[2] + i);
        }
        const bool hit = inr && isfinite(len) && len >= 0.0f && isfinite3(px, py, pz);
        const bool miss = inr && len == INFINITY;
        uint32_t home = 0, tag = 0, cell = 0;
        if (hit) {
            const unsigned long long key =
                tile_key(a.kp, px, py, pz, sx, sy, sz, len, KEY_DIR == GI_KEY_DIR_NORMAL ? 0u : 1u, cell);
            cell_of_key(key, a.mask, home, tag);
        }
        // same cell = same (home, tag, cell); home < 2^22, so the cell fits above it
        const unsigned hm = __ballot_sync(kFull, hit);
        unsigned peers = 0;
        if (hit) peers = __match_any_sync(hm, ((unsigned long long)(home | (cell << 26)) << 32) | tag);
        const bool leader = hit && (peers & ((1u << lane) - 1u)) == 0u;
        uint32_t slot = GI_SLOT_NONE;
        if (leader) {
            uint32_t s = home, k = 0;
            for (; k < a.max_probe; ++k) {
                const uint32_t t = __ldcg(a.tags + s);
                if (t == tag) {
                    slot = s;
                    break;
                }
                if (t == kEmpty) {
                    const uint32_t old = atomicCAS(a.tags + s, kEmpty, tag);
                    if (old == kEmpty) ++my_new;
                    if (old == kEmpty || old == tag) {
                        slot = s;
                        break;
                    }
                }
                s = (s + 1u) & a.mask;
            }
            my_maxp = max(my_maxp, k + 1u);
            if (slot != GI_SLOT_NONE) atomicOr(ta.tmask + slot, 1ull << cell);
            else my_dropped += (unsigned long long)__popc(peers);
        }
        const int lead = hit ? (__ffs(peers) - 1) : lane;
        const uint32_t my_slot = __shfl_sync(kFull, slot, lead);
        uint32_t id = miss ? GI_SLOT_MISS : GI_SLOT_NONE;
        if (hit && my_slot != GI_SLOT_NONE) id = my_slot * kTileCells + cell;
        if (hit && my_slot == GI_SLOT_NONE) {
            uint32_t bad = 0;
            quantize(__ldcs(a.rad[0] + i), bad);
            quantize(__ldcs(a.rad[1] + i), bad);
            quantize(__ldcs(a.rad[2] + i), bad);
            my_clamped += bad;
        }
        if (inr) __stcs(a.slot_ids + i, id);
    }
    my_clamped = __reduce_add_sync(kFull, my_clamped);
    my_maxp = __reduce_max_sync(kFull, my_maxp);
    my_new = __reduce_add_sync(kFull, my_new);
    if (my_dropped) atomicAdd(&a.ctr->dropped, my_dropped);
    if (lane == 0) {
        if (my_clamped) atomicAdd(&s_clamped, my_clamped);
        if (my_new) atomicAdd(&s_new, my_new);
        atomicMax(&s_maxp, my_maxp);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_clamped) atomicAdd(&a.ctr->clamped, (unsigned long long)s_clamped);
        if (s_maxp) atomicMax(&a.ctr->max_probe, s_maxp);
        if (s_new) atomicAdd(&a.ctr->occupied, s_new);
    }
}

constexpr int kCompactThreads = 256;

// One warp per 32 tile slots: the touched tiles without a block take the next indices (one
// counter add per CTA) and are listed at that index.  ctr->touch_count counts the blocks handed
// out since the last resolve.
__global__ void __launch_bounds__(kCompactThreads) k_tile_compact(const unsigned long long *tmask, uint32_t *cidx,
                                                                  uint32_t *tlist, uint32_t tiles, Counters *ctr) {
    __shared__ uint32_t s_cnt[kCompactThreads / 32];
    __shared__ uint32_t s_base;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t t = blockIdx.x * kCompactThreads + threadIdx.x;
    bool need = false;
    if (t < tiles) need = __ldcg(tmask + t) != 0ull && __ldcg(cidx + t) == GI_SLOT_NONE;
    const unsigned b = __ballot_sync(kFull, need);
    if (lane == 0) s_cnt[w] = (uint32_t)__popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t tot = 0;
        for (int k = 0; k < kCompactThreads / 32; ++k) {
            const uint32_t c = s_cnt[k];
            s_cnt[k] = tot;
            tot += c;
        }
        s_base = tot ? atomicAdd(&ctr->touch_count, tot) : 0u;
    }
    __syncthreads();
    if (need) {
        const uint32_t k = s_base + s_cnt[w] + (uint32_t)__popc(b & ((1u << lane) - 1u));
        cidx[t] = k;
        tlist[k] = t;
    }
}

__global__ void __launch_bounds__(kUpdThreads, 8) k_tile_accumulate(const uint32_t *slot_ids, const float *r0,
                                                                    const float *r1, const float *r2,
                                                                    unsigned long long n, const uint32_t *cidx,
                                                                    uint32_t cells, Accum *accum, Counters *ctr) {
    __shared__ __align__(32) unsigned long long s_red[kUpdThreads][4];
    __shared__ uint32_t s_clamped;
    if (threadIdx.x == 0) s_clamped = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    uint32_t my_clamped = 0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < n; base += stride) {
        const unsigned long long i = base + threadIdx.x;
        const uint32_t id = i < n ? __ldcs(slot_ids + i) : GI_SLOT_NONE;
        bool ok = id < cells;
        unsigned long long q0 = 0, q1 = 0, q2 = 0;
        uint32_t blk = 0;
        if (ok) {
            uint32_t bad = 0;
            q0 = quantize(__ldcs(r0 + i), bad);
            q1 = quantize(__ldcs(r1 + i), bad);
            q2 = quantize(__ldcs(r2 + i), bad);
            my_clamped += bad;
            blk = __ldcg(cidx + id / kTileCells);
        }
        // a tile with a slot id always has a block (the compaction ran after the keys); a missing
        // one would be a broken invariant: the record is skipped rather than written out of range
        ok = ok && blk < cells / kTileCells;
        const unsigned vm = __ballot_sync(kFull, ok);
        unsigned peers = 0;
        if (ok) peers = __match_any_sync(vm, id);
        const unsigned above = peers & (0xFFFFFFFEu << lane);
        int nxt = above ? (__ffs(above) - 1) : -1;
        uint32_t cnt = ok ? 1u : 0u;
        while (__any_sync(kFull, nxt >= 0)) {
            const int src = nxt >= 0 ? nxt : lane;
            const unsigned long long o0 = __shfl_sync(kFull, q0, src);
            const unsigned long long o1 = __shfl_sync(kFull, q1, src);
            const unsigned long long o2 = __shfl_sync(kFull, q2, src);
            const uint32_t oc = __shfl_sync(kFull, cnt, src);
            const int on = __shfl_sync(kFull, nxt, src);
            if (nxt >= 0) {
                q0 += o0;
                q1 += o1;
                q2 += o2;
                cnt += oc;
                nxt = on;
            }
        }
        if (ok && (peers & ((1u << lane) - 1u)) == 0u) {
            // the group's sums and count in one 32-byte bulk reduction (the stamp half of the
            // last lane is unused in the blocks)
            Accum *ac = accum + (size_t)blk * kTileCells + (id % kTileCells);
            bulk_wait_read();  // the previous reduction has read the slot
            s_red[threadIdx.x][0] = q0;
            s_red[threadIdx.x][1] = q1;
            s_red[threadIdx.x][2] = q2;
            s_red[threadIdx.x][3] = cnt;
            bulk_add_accum(ac, s_red[threadIdx.x]);
        }
    }
    bulk_wait_all();
    // hits with a tile whose radiance was clamped (k_tile_key counts those of dropped hits)
    my_clamped = __reduce_add_sync(kFull, my_clamped);
    if (lane == 0 && my_clamped) atomicAdd(&s_clamped, my_clamped);
    __syncthreads();
    if (threadIdx.x == 0 && s_clamped) atomicAdd(&ctr->clamped, (unsigned long long)s_clamped);
}

// ---------------------------------------------------------------- resolve
constexpr int kTileResThreads = 256;
constexpr int kTileResWarps = kTileResThreads / 32;

__device__ __forceinline__ float recip_children(uint32_t k) {
    // 1 / k for the children holding a value (k <= 4): exact for 1, 2, 4, within half an ulp for 3
    return k == 1u ? 1.0f : (k == 2u ? 0.5f : (k == 3u ? 0.333333343f : (k == 4u ? 0.25f : 0.0f)));
}

// One MIP value from four values of the level below (xyz, w = sample count bits; count 0 = no
// value): the mean of those holding a value and their summed (saturating) count.
__device__ __forceinline__ float4 box4(const float4 &a, const float4 &b, const float4 &c, const float4 &d) {
    const uint32_t na = __float_as_uint(a.w), nb = __float_as_uint(b.w), nc = __float_as_uint(c.w),
                   nd = __float_as_uint(d.w);
    float sx = 0.f, sy = 0.f, sz = 0.f;
    uint32_t k = 0, n = 0;
    if (na) {
        sx += a.x;
        sy += a.y;
        sz += a.z;
        ++k;
        n = sat_add(n, na);
    }
    if (nb) {
        sx += b.x;
        sy += b.y;
        sz += b.z;
        ++k;
        n = sat_add(n, nb);
    }
    if (nc) {
        sx += c.x;
        sy += c.y;
        sz += c.z;
        ++k;
        n = sat_add(n, nc);
    }
    if (nd) {
        sx += d.x;
        sy += d.y;
        sz += d.z;
        ++k;
        n = sat_add(n, nd);
    }
    const float r = recip_children(k);
    return make_float4(sx * r, sy * r, sz * r, __uint_as_float(n));
}

// The touched tiles are listed in block order by the compaction; warps take entries i, i + warps,
// ... (the next entry's tile and masks are loaded before the current one is computed).  A tile is
// resolved by one warp, lane l holding cells l and l + 32: the blended cells go to shared memory,
// lanes 0..15 build the 4x4 level, lanes 0..3 the 2x2 level and lane 0 the 1x1 level, each value
// from its four children; then each live cell takes the finest level with enough samples.
// Completion is counted per warp, so warps never wait for one another.
__global__ void __launch_bounds__(kTileResThreads) k_tile_resolve(TileResolveArgs a) {
    __shared__ float4 s_lv[kTileResWarps][kTileCells + kTileMips];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float4 *lv = s_lv[w];
    const uint32_t warp = (blockIdx.x * kTileResThreads + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * kTileResThreads) >> 5;
    const uint32_t n = __ldcg(&a.ctr->touch_count);
    uint32_t i = warp;
    uint32_t t = 0;
    unsigned long long m = 0, o = 0;
    if (i < n) {
        t = __ldcg(a.tlist + i);
        m = __ldcg(a.tmask + t);
        o = __ldcg(a.t.omask + t);
    }
    while (i < n) {
        const size_t base = (size_t)t * kTileCells;
        Accum *acc = a.t.accum + (size_t)i * kTileCells;
        const unsigned long long want = m | o;
        // every load of the tile: stamps, state of the cells that may hold a value, accumulators
        uint32_t st[2];
        float4 sv[2];
        uint4 lo[2], hi[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t c = (uint32_t)lane + 32u * h;
            st[h] = __ldcg(a.t.stamp + base + c);
            sv[h] = make_float4(0.f, 0.f, 0.f, 0.f);
            if ((want >> c) & 1ull) sv[h] = __ldcg(a.t.state + base + c);
            if ((m >> c) & 1ull) {
                const uint4 *src = reinterpret_cast<const uint4 *>(acc + c);
                lo[h] = __ldcg(src);
                hi[h] = __ldcg(src + 1);
            }
        }
        // the next entry's tile and masks
        const uint32_t inext = i + nwarps;
        uint32_t tn = 0;
        unsigned long long mn = 0, on = 0;
        if (inext < n) {
            tn = __ldcg(a.tlist + inext);
            mn = __ldcg(a.tmask + tn);
            on = __ldcg(a.t.omask + tn);
        }
        bool live[2], cold[2];
        float4 cv[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t c = (uint32_t)lane + 32u * h;
            const size_t e = base + c;
            cv[h] = sv[h];
            cold[h] = false;
            if ((m >> c) & 1ull) {
                // no history: never resolved, or evicted by an earlier resolve (untouched E frames)
                const bool fresh = st[h] == 0u || (a.has_lr && (a.lr - (st[h] - 1u)) >= a.evict);
                const unsigned long long s0 = ((unsigned long long)lo[h].y << 32) | lo[h].x;
                const unsigned long long s1 = ((unsigned long long)lo[h].w << 32) | lo[h].z;
                const unsigned long long s2 = ((unsigned long long)hi[h].y << 32) | hi[h].x;
                // mean = sum / (count 2^24): one reciprocal, three products (within an ulp of the quotient)
                const float rc = __frcp_rn((float)hi[h].z) * 5.9604644775390625e-8f;
                float3 val = make_float3(__ull2float_rn(s0) * rc, __ull2float_rn(s1) * rc, __ull2float_rn(s2) * rc);
                uint32_t samples = hi[h].z;
                if (!fresh) {
                    val = make_float3(sv[h].x + a.alpha * (val.x - sv[h].x), sv[h].y + a.alpha * (val.y - sv[h].y),
                                      sv[h].z + a.alpha * (val.z - sv[h].z));
                    samples = sat_add(__float_as_uint(sv[h].w), samples);
                }
                cv[h] = make_float4(val.x, val.y, val.z, __uint_as_float(samples));
                uint4 *dst = reinterpret_cast<uint4 *>(acc + c);
                dst[0] = make_uint4(0u, 0u, 0u, 0u);
                dst[1] = make_uint4(0u, 0u, 0u, 0u);
                live[h] = true;
                cold[h] = fresh;
            } else {
                live[h] = st[h] != 0u && (a.frame - (st[h] - 1u)) < a.evict;
            }
            // a live cell's sample count is >= 1, so count 0 marks "no value" in the levels
            if (!live[h]) cv[h] = make_float4(0.f, 0.f, 0.f, 0.f);
            lv[c] = cv[h];
        }
        // State and stamps go back in whole 32-byte sectors wherever a sector holds a touched cell
        // (a partly written sector costs the DRAM a read of it): the touched cells' new values, the
        // untouched cells' unchanged ones -- or zeros for a cell that holds no value (a dead cell's
        // state is never read: it restarts without history when touched again).
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t c = (uint32_t)lane + 32u * h;
            const size_t e = base + c;
            const bool touched = (m >> c) & 1ull;
            const unsigned tm = __ballot_sync(kFull, touched);
            if ((tm >> (lane & ~1)) & 3u) a.t.state[e] = touched ? cv[h] : sv[h];
            if ((tm >> (lane & ~7)) & 0xFFu) a.t.stamp[e] = touched ? a.stamp_now : st[h];
        }
        __syncwarp();
        if (lane < 16) {  // 4x4 value (I, J) = (lane & 3, lane >> 2): cells 2I + 16J + {0, 1, 8, 9}
            const int c0 = 2 * (lane & 3) + 16 * (lane >> 2);
            lv[kTileCells + lane] = box4(lv[c0], lv[c0 + 1], lv[c0 + 8], lv[c0 + 9]);
        }
        __syncwarp();
        if (lane < 4) {  // 2x2 value (I, J) = (lane & 1, lane >> 1): 4x4 values 2I + 8J + {0, 1, 4, 5}
            const int c0 = kTileCells + 2 * (lane & 1) + 8 * (lane >> 1);
            lv[kTileCells + 16 + lane] = box4(lv[c0], lv[c0 + 1], lv[c0 + 4], lv[c0 + 5]);
        }
        __syncwarp();
        if (lane == 0) {
            const int c0 = kTileCells + 16;
            lv[kTileCells + 20] = box4(lv[c0], lv[c0 + 1], lv[c0 + 2], lv[c0 + 3]);
        }
        __syncwarp();
        // answers in whole sectors too: a cell without value shares its sector with a live one
        // (2 cells per sector in float32, 4 in float16) writes zeros, never read (not live)
        const uint32_t span = a.f16 ? 4u : 2u;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t c = (uint32_t)lane + 32u * h;
            const unsigned lm = __ballot_sync(kFull, live[h]);
            if (!live[h]) {
                if ((lm >> (lane & ~(span - 1u))) & ((1u << span) - 1u))
                    store_resolved(a.t.resolved, a.res_stride, a.f16, (uint32_t)(base + c),
                                   make_float3(0.f, 0.f, 0.f), false);
                continue;
            }
            // finest level with enough samples; a live cell has a value at every level above it
            const float4 l1 = lv[kTileCells + ((c & 7u) >> 1) + 4u * (c >> 4)];
            const float4 l2 = lv[kTileCells + 16u + ((c >> 2) & 1u) + 2u * (c >> 5)];
            float4 ans = lv[kTileCells + 20];
            if (__float_as_uint(cv[h].w) >= a.min_samples) ans = cv[h];
            else if (__float_as_uint(l1.w) >= a.min_samples) ans = l1;
            else if (__float_as_uint(l2.w) >= a.min_samples) ans = l2;
            store_resolved(a.t.resolved, a.res_stride, a.f16, (uint32_t)(base + c), make_float3(ans.x, ans.y, ans.z),
                           cold[h]);
        }
        if (lane < kTileMips) a.t.mips[(size_t)t * kTileMips + lane] = lv[kTileCells + lane];
        const unsigned live0 = __ballot_sync(kFull, live[0]), live1 = __ballot_sync(kFull, live[1]);
        if (lane == 0) {
            a.t.omask[t] = ((unsigned long long)live1 << 32) | live0;
            a.tmask[t] = 0ull;
            a.cidx[t] = GI_SLOT_NONE;
        }
        __syncwarp();
        i = inext;
        t = tn;
        m = mn;
        o = on;
    }
    // the last warp to finish resets the block counter and publishes the occupancy
    resolve_finish(a.ctr, a.occ_out, a.stamp_now, nwarps, 0u);
}

// ---------------------------------------------------------------- lookup by point
template <int KEY_DIR>
__global__ void k_tile_query_points(TileUpdateArgs ta, TileArrays t, uint32_t res_stride, int f16, LiveRule rule,
                                    float4 *out) {
    const UpdateArgs &a = ta.u;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < a.n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const float len = a.len[i];
        const float px = a.p[0][i], py = a.p[1][i], pz = a.p[2][i];
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (isfinite(len) && len >= 0.0f && isfinite3(px, py, pz)) {
            const float *src0 = KEY_DIR == GI_KEY_DIR_NORMAL ? a.nrm[0] : a.dir[0];
            const float *src1 = KEY_DIR == GI_KEY_DIR_NORMAL ? a.nrm[1] : a.dir[1];
            const float *src2 = KEY_DIR == GI_KEY_DIR_NORMAL ? a.nrm[2] : a.dir[2];
            uint32_t cell;
            const unsigned long long key = tile_key(a.kp, px, py, pz, src0[i], src1[i], src2[i], len,
                                                    KEY_DIR == GI_KEY_DIR_NORMAL ? 0u : 1u, cell);
            uint32_t home, tag;
            cell_of_key(key, a.mask, home, tag);
            uint32_t s = home;
            for (uint32_t k = 0; k < a.max_probe; ++k) {
                const uint32_t w = __ldg(t.tags + s);
                if (w == kEmpty) break;
                if (w == tag) {
                    const uint32_t e = s * kTileCells + cell;
                    if (answers(__ldg(t.stamp + e), rule)) {
                        const float3 v = load_resolved(t.resolved, res_stride, f16, e);
                        o = make_float4(v.x, v.y, v.z, 1.0f);
                    }
                    break;
                }
                s = (s + 1u) & a.mask;
            }
        }
        out[i] = o;
    }
}

// ---------------------------------------------------------------- compaction
// One warp per slot of the current table: a tile with a live cell moves to the clean spare table
// (home recovered from the slot and the tag's low byte) with its stamps, state, answers and MIP
// values; the current slot is cleared behind it.  Runs right after a resolve, when every
// accumulator and touched mask is clear.
__global__ void k_tile_rebuild(TileArrays from, TileArrays to, unsigned long long *tmask, uint32_t res_bytes,
                               uint32_t mask, uint32_t max_probe, LiveRule rule, Counters *ctr) {
    const int lane = threadIdx.x & 31;
    const uint32_t N = mask + 1u;
    uint32_t live_tiles = 0, dropped = 0;
    for (uint32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < N; s += (gridDim.x * blockDim.x) >> 5) {
        const uint32_t tg = from.tags[s];
        if (tg == kEmpty) continue;
        const size_t e0 = (size_t)s * kTileCells + lane, e1 = e0 + 32;
        const uint32_t st0 = from.stamp[e0], st1 = from.stamp[e1];
        const unsigned live0 = __ballot_sync(kFull, answers(st0, rule));
        const unsigned live1 = __ballot_sync(kFull, answers(st1, rule));
        if (live0 | live1) {
            uint32_t ns = GI_SLOT_NONE;
            if (lane == 0) {
                const uint32_t home = (s - ((s - (tg & 0xFFu)) & 0xFFu)) & mask;
                uint32_t p = home;
                for (uint32_t k = 0; k < max_probe; ++k) {
                    if (atomicCAS(to.tags + p, kEmpty, tg) == kEmpty) {
                        ns = p;
                        break;
                    }
                    p = (p + 1u) & mask;
                }
            }
            ns = __shfl_sync(kFull, ns, 0);
            if (ns != GI_SLOT_NONE) {
                const size_t d0 = (size_t)ns * kTileCells + lane, d1 = d0 + 32;
                to.stamp[d0] = st0;
                to.stamp[d1] = st1;
                to.state[d0] = from.state[e0];
                to.state[d1] = from.state[e1];
                if (res_bytes == 8) {
                    reinterpret_cast<uint2 *>(to.resolved)[d0] = reinterpret_cast<const uint2 *>(from.resolved)[e0];
                    reinterpret_cast<uint2 *>(to.resolved)[d1] = reinterpret_cast<const uint2 *>(from.resolved)[e1];
                } else {
                    reinterpret_cast<uint4 *>(to.resolved)[d0] = reinterpret_cast<const uint4 *>(from.resolved)[e0];
                    reinterpret_cast<uint4 *>(to.resolved)[d1] = reinterpret_cast<const uint4 *>(from.resolved)[e1];
                }
                if (lane < kTileMips)
                    to.mips[(size_t)ns * kTileMips + lane] = from.mips[(size_t)s * kTileMips + lane];
                if (lane == 0) {
                    to.omask[ns] = ((unsigned long long)live1 << 32) | live0;
                    ++live_tiles;
                }
            } else if (lane == 0) {
                dropped += (uint32_t)(__popc(live0) + __popc(live1));
            }
        }
        from.stamp[e0] = 0u;
        from.stamp[e1] = 0u;
        __syncwarp();
        if (lane == 0) {
            from.tags[s] = kEmpty;
            from.omask[s] = 0ull;
            tmask[s] = 0ull;
        }
    }
    live_tiles = __reduce_add_sync(kFull, live_tiles);
    dropped = __reduce_add_sync(kFull, dropped);
    if (lane == 0) {
        if (live_tiles) atomicAdd(&ctr->occupied, live_tiles);
        if (dropped) atomicAdd(&ctr->dropped, (unsigned long long)dropped);
    }
}

// ---------------------------------------------------------------- table scan for stats
__global__ void k_tile_scan(TileArrays t, const unsigned long long *tmask, uint32_t tiles, LiveRule rule,
                            unsigned long long *out /* occupied, live, touched tiles */) {
    unsigned long long occ = 0, live = 0, touched = 0;
    const size_t cells = (size_t)tiles * kTileCells;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < cells; e += (size_t)gridDim.x * blockDim.x) {
        if ((e % kTileCells) == 0 && tmask[e / kTileCells]) ++touched;
        if (t.tags[e / kTileCells] == kEmpty) continue;
        if ((e % kTileCells) == 0) ++occ;
        if (((tmask[e / kTileCells] >> (e % kTileCells)) & 1ull) || answers(t.stamp[e], rule)) ++live;
    }
    for (int o = 16; o; o >>= 1) {
        occ += __shfl_xor_sync(kFull, occ, o);
        live += __shfl_xor_sync(kFull, live, o);
        touched += __shfl_xor_sync(kFull, touched, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, occ);
        atomicAdd(out + 1, live);
        atomicAdd(out + 2, touched);
    }
}

// ---------------------------------------------------------------- launchers
gi_status tile_update_launch(const TileUpdateArgs &a, int key_dir, int resident_blocks, cudaStream_t st) {
    // neither pass stages anything per block: at least a resident grid striding over the records,
    // and no block with more than kUpdBlockRecords records (1080p: 92 us with the resident grid
    // against 97 us with blocks of 2048 records; 4K: 315 us with blocks of 2048 against 348 us)
    const unsigned long long chunks = (a.u.n + kUpdBlockRecords - 1) / kUpdBlockRecords;
    const int blocks = (int)std::min<unsigned long long>(
        std::max<unsigned long long>((unsigned long long)resident_blocks, chunks), (a.u.n + kUpdThreads - 1) / kUpdThreads);
    if (blocks == 0) return GI_OK;
    if (key_dir == GI_KEY_DIR_NORMAL)
        k_tile_key<GI_KEY_DIR_NORMAL><<<blocks, kUpdThreads, 0, st>>>(a);
    else
        k_tile_key<GI_KEY_DIR_RAY><<<blocks, kUpdThreads, 0, st>>>(a);
    gi_status s = cuda_status(cudaGetLastError(), "k_tile_key launch");
    if (s != GI_OK) return s;
    const uint32_t tiles = a.u.mask + 1u;
    k_tile_compact<<<(tiles + kCompactThreads - 1) / kCompactThreads, kCompactThreads, 0, st>>>(a.tmask, a.cidx,
                                                                                                a.tlist, tiles, a.u.ctr);
    s = cuda_status(cudaGetLastError(), "k_tile_compact launch");
    if (s != GI_OK) return s;
    k_tile_accumulate<<<blocks, kUpdThreads, 0, st>>>(a.u.slot_ids, a.u.rad[0], a.u.rad[1], a.u.rad[2], a.u.n, a.cidx,
                                                      tiles * (uint32_t)kTileCells, a.u.accum, a.u.ctr);
    return cuda_status(cudaGetLastError(), "k_tile_accumulate launch");
}

int tile_resolve_blocks_per_sm() {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_resolve, kTileResThreads, 0) != cudaSuccess)
        return 1;
    return per_sm > 0 ? per_sm : 1;
}

gi_status tile_resolve_launch(const TileResolveArgs &a, int blocks, cudaStream_t st) {
    // no more warps than tiles
    blocks = std::min<int>(blocks, (int)((a.tiles + kTileResWarps - 1) / kTileResWarps));
    k_tile_resolve<<<blocks, kTileResThreads, 0, st>>>(a);
    return cuda_status(cudaGetLastError(), "k_tile_resolve launch");
}

gi_status tile_query_points_launch(const TileUpdateArgs &a, const TileArrays &t, uint32_t res_stride, int f16,
                                   LiveRule rule, float4 *out, int blocks, int key_dir, cudaStream_t st) {
    if (key_dir == GI_KEY_DIR_NORMAL)
        k_tile_query_points<GI_KEY_DIR_NORMAL><<<blocks, 256, 0, st>>>(a, t, res_stride, f16, rule, out);
    else
        k_tile_query_points<GI_KEY_DIR_RAY><<<blocks, 256, 0, st>>>(a, t, res_stride, f16, rule, out);
    return cuda_status(cudaGetLastError(), "k_tile_query_points launch");
}

gi_status tile_rebuild_launch(const TileArrays &from, const TileArrays &to, unsigned long long *tmask,
                              uint32_t res_bytes, uint32_t mask, uint32_t max_probe, LiveRule rule, Counters *ctr,
                              int blocks, cudaStream_t st) {
    k_tile_rebuild<<<blocks, 256, 0, st>>>(from, to, tmask, res_bytes, mask, max_probe, rule, ctr);
    return cuda_status(cudaGetLastError(), "k_tile_rebuild launch");
}

gi_status tile_scan_launch(const TileArrays &t, const unsigned long long *tmask, uint32_t tiles, LiveRule rule,
                           unsigned long long *out, int blocks, cudaStream_t st) {
    k_tile_scan<<<blocks, 256, 0, st>>>(t, tmask, tiles, rule, out);
    return cuda_status(cudaGetLastError(), "k_tile_scan launch");
}

} // namespace gi
