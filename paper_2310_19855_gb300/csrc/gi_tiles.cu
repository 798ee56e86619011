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
//   tmask    u64[T]          cells touched since the last resolve (set by the update, cleared by
//                            the resolve); its first bit in a frame lists the tile for the resolve
//   accum    Accum[T * 64]   fixed-point sums and count since the last resolve
//   stamp    u32[T * 64]     1 + frame of the last resolve that found samples; 0 = never
//   state    float4[T * 64]  blended radiance, w = samples since the cell last started without history
//   resolved [T * 64]        the answer of each live cell (float4 or half4; w = resolved without history)
//   mips     float4[T * 21]  levels 1..3 (16 + 4 + 1 values), w = summed sample count, 0 = no value
// The per-cell arrays of one tile are contiguous: the resolve of a tile is one warp reading 256 B
// of stamps and 1 KB of state, the accumulators of touched cells only.
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
// Per record: tile descriptor, bucket + fingerprint of the tile, cell.  Hits of a warp naming the
// same cell are merged (integer sums, order-free); the group leader finds or inserts the tile by
// linear probing, adds the sums into the cell's accumulator and sets the cell's bit in the tile's
// touched mask; the add that finds the mask empty lists the tile for the resolve.
template <int KEY_DIR>
__global__ void __launch_bounds__(kUpdThreads, 8) k_tile_update(TileUpdateArgs ta) {
    const UpdateArgs &a = ta.u;
    __shared__ uint32_t s_touch[kUpdBlockRecords];
    __shared__ uint32_t s_n, s_base, s_clamped, s_maxp, s_new;
    if (threadIdx.x == 0) {
        s_n = 0;
        s_clamped = 0;
        s_maxp = 0;
        s_new = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * kUpdThreads;
    uint32_t my_clamped = 0, my_maxp = 0, my_new = 0;
    for (unsigned long long base = (unsigned long long)blockIdx.x * kUpdThreads; base < a.n; base += stride) {
        const unsigned long long i = base + threadIdx.x;
        const bool inr = i < a.n;
        const float len = inr ? __ldcs(a.len + i) : -1.0f;
        float px = 0.f, py = 0.f, pz = 0.f;
        if (inr) {
            px = __ldcs(a.p[0] + i);
            py = __ldcs(a.p[1] + i);
            pz = __ldcs(a.p[2] + i);
        }
        const bool hit = inr && isfinite(len) && len >= 0.0f && isfinite3(px, py, pz);
        const bool miss = inr && len == INFINITY;
        unsigned long long q0 = 0, q1 = 0, q2 = 0;
        uint32_t home = 0, tag = 0, cell = 0;
        if (hit) {
            float sx, sy, sz;
            if (KEY_DIR == GI_KEY_DIR_NORMAL) {
                sx = __ldcs(a.nrm[0] + i);
                sy = __ldcs(a.nrm[1] + i);
                sz = __ldcs(a.nrm[2] + i);
            } else {
                sx = __ldcs(a.dir[0] + i);
                sy = __ldcs(a.dir[1] + i);
                sz = __ldcs(a.dir[2] + i);
            }
            uint32_t bad = 0;
            q0 = quantize(__ldcs(a.rad[0] + i), bad);
            q1 = quantize(__ldcs(a.rad[1] + i), bad);
            q2 = quantize(__ldcs(a.rad[2] + i), bad);
            my_clamped += bad;
            const unsigned long long key =
                tile_key(a.kp, px, py, pz, sx, sy, sz, len, KEY_DIR == GI_KEY_DIR_NORMAL ? 0u : 1u, cell);
            cell_of_key(key, a.mask, home, tag);
        }
        // same cell = same (home, tag, cell); home < 2^22, so the cell fits above it
        const unsigned hm = __ballot_sync(kFull, hit);
        unsigned peers = 0;
        if (hit) peers = __match_any_sync(hm, ((unsigned long long)(home | (cell << 26)) << 32) | tag);
        const unsigned above = peers & (0xFFFFFFFEu << lane);
        int nxt = above ? (__ffs(above) - 1) : -1;
        uint32_t cnt = hit ? 1u : 0u;
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
            if (slot != GI_SLOT_NONE) {
                Accum *ac = a.accum + (size_t)slot * kTileCells + cell;
                atomicAdd(&ac->sum[0], q0);
                atomicAdd(&ac->sum[1], q1);
                atomicAdd(&ac->sum[2], q2);
                atomicAdd(&ac->count, cnt);
                if (atomicOr(ta.tmask + slot, 1ull << cell) == 0ull) s_touch[atomicAdd(&s_n, 1u)] = slot;
            } else {
                atomicAdd(&a.ctr->dropped, (unsigned long long)cnt);
            }
        }
        const int lead = hit ? (__ffs(peers) - 1) : lane;
        const uint32_t my_slot = __shfl_sync(kFull, slot, lead);
        uint32_t id = miss ? GI_SLOT_MISS : GI_SLOT_NONE;
        if (hit && my_slot != GI_SLOT_NONE) id = my_slot * kTileCells + cell;
        if (inr) __stcs(a.slot_ids + i, id);
    }
    my_clamped = __reduce_add_sync(kFull, my_clamped);
    my_maxp = __reduce_max_sync(kFull, my_maxp);
    my_new = __reduce_add_sync(kFull, my_new);
    if (lane == 0) {
        if (my_clamped) atomicAdd(&s_clamped, my_clamped);
        if (my_new) atomicAdd(&s_new, my_new);
        atomicMax(&s_maxp, my_maxp);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        s_base = s_n ? atomicAdd(&a.ctr->touch_count, s_n) : 0u;
        if (s_clamped) atomicAdd(&a.ctr->clamped, (unsigned long long)s_clamped);
        if (s_maxp) atomicMax(&a.ctr->max_probe, s_maxp);
        if (s_new) atomicAdd(&a.ctr->occupied, s_new);
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < s_n; j += kUpdThreads) a.touch[s_base + j] = s_touch[j];
}

// ---------------------------------------------------------------- resolve
// Sum of a value over the lanes lane ^ {0, o1, o2, o1 ^ o2}: every lane of the group gets the same
// bits (each add is commutative).
struct Box {
    float3 s;
    uint32_t k, n;
};

__device__ __forceinline__ Box box_xor(Box b, int o) {
    Box r;
    r.s.x = b.s.x + __shfl_xor_sync(kFull, b.s.x, o);
    r.s.y = b.s.y + __shfl_xor_sync(kFull, b.s.y, o);
    r.s.z = b.s.z + __shfl_xor_sync(kFull, b.s.z, o);
    r.k = b.k + __shfl_xor_sync(kFull, b.k, o);
    r.n = sat_add(b.n, __shfl_xor_sync(kFull, b.n, o));
    return r;
}

__device__ __forceinline__ Box box_of(bool has, float3 v, uint32_t n) {
    Box b;
    b.s = has ? v : make_float3(0.f, 0.f, 0.f);
    b.k = has ? 1u : 0u;
    b.n = has ? n : 0u;
    return b;
}

// mean of the children holding a value (their count k), zero when none does
__device__ __forceinline__ float3 box_mean(const Box &b) {
    if (!b.k) return make_float3(0.f, 0.f, 0.f);
    const float fk = (float)b.k;
    return make_float3(__fdiv_rn(b.s.x, fk), __fdiv_rn(b.s.y, fk), __fdiv_rn(b.s.z, fk));
}

__device__ __forceinline__ float4 mip_word(const Box &b) {
    const float3 m = box_mean(b);
    return make_float4(m.x, m.y, m.z, __uint_as_float(b.k ? b.n : 0u));
}

constexpr int kTileResThreads = 256;

// One warp per touched tile; lane l holds cells l and l + 32 (rows 0..3 and 4..7).  Cell (i, j)
// = i + 8 j, so the level-1 siblings of a cell differ in lane bits 0 and 3, level-2 siblings (of
// level-1 values) in bits 1 and 4, level-3 siblings in bit 2 and in the half.
__global__ void __launch_bounds__(kTileResThreads) k_tile_resolve(TileResolveArgs a) {
    const uint32_t n = __ldcg(&a.ctr->touch_count);
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * kTileResThreads + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * kTileResThreads) >> 5;
    for (uint32_t ti = warp; ti < n; ti += nwarps) {
        const uint32_t t = __ldcs(a.touch + ti);
        const unsigned long long m = __ldcg(a.tmask + t);
        __syncwarp();
        if (lane == 0) a.tmask[t] = 0ull;
        const size_t base = (size_t)t * kTileCells;
        float3 v[2];
        uint32_t ns[2];
        bool live[2], cold[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t c = (uint32_t)lane + 32u * h;
            const size_t e = base + c;
            const uint32_t st = __ldcg(a.t.stamp + e);
            v[h] = make_float3(0.f, 0.f, 0.f);
            ns[h] = 0;
            live[h] = false;
            cold[h] = false;
            if ((m >> c) & 1ull) {
                const uint4 *src = reinterpret_cast<const uint4 *>(a.t.accum + e);
                const uint4 lo = __ldcg(src), hi = __ldcg(src + 1);
                // no history: never resolved, or evicted by an earlier resolve (untouched E frames)
                const bool fresh = st == 0u || (a.has_lr && (a.lr - (st - 1u)) >= a.evict);
                const unsigned long long s0 = ((unsigned long long)lo.y << 32) | lo.x;
                const unsigned long long s1 = ((unsigned long long)lo.w << 32) | lo.z;
                const unsigned long long s2 = ((unsigned long long)hi.y << 32) | hi.x;
                const float fc = (float)hi.z;
                float3 val = make_float3(__fdiv_rn(__ull2float_rn(s0), fc) * 5.9604644775390625e-8f,
                                         __fdiv_rn(__ull2float_rn(s1), fc) * 5.9604644775390625e-8f,
                                         __fdiv_rn(__ull2float_rn(s2), fc) * 5.9604644775390625e-8f);
                uint32_t samples = hi.z;
                if (!fresh) {
                    const float4 o = __ldcg(a.t.state + e);
                    val = make_float3(o.x + a.alpha * (val.x - o.x), o.y + a.alpha * (val.y - o.y),
                                      o.z + a.alpha * (val.z - o.z));
                    samples = sat_add(__float_as_uint(o.w), samples);
                }
                a.t.state[e] = make_float4(val.x, val.y, val.z, __uint_as_float(samples));
                a.t.stamp[e] = a.stamp_now;
                uint4 *dst = reinterpret_cast<uint4 *>(a.t.accum + e);
                dst[0] = make_uint4(0u, 0u, 0u, 0u);
                dst[1] = make_uint4(0u, 0u, 0u, 0u);
                v[h] = val;
                ns[h] = samples;
                live[h] = true;
                cold[h] = fresh;
            } else if (st != 0u && (a.frame - (st - 1u)) < a.evict) {
                const float4 o = __ldcg(a.t.state + e);
                v[h] = make_float3(o.x, o.y, o.z);
                ns[h] = __float_as_uint(o.w);
                live[h] = true;
            }
        }
        // level 1 (4x4): siblings at lane ^ 1 and lane ^ 8
        Box b1[2], b2[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) b1[h] = box_xor(box_xor(box_of(live[h], v[h], ns[h]), 1), 8);
        // level 2 (2x2): level-1 siblings at lane ^ 2 and lane ^ 16
#pragma unroll
        for (int h = 0; h < 2; ++h) b2[h] = box_xor(box_xor(box_of(b1[h].k > 0, box_mean(b1[h]), b1[h].n), 2), 16);
        // level 3 (1x1): level-2 siblings at lane ^ 4 and in the other half
        Box c3[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) c3[h] = box_xor(box_of(b2[h].k > 0, box_mean(b2[h]), b2[h].n), 4);
        Box b3;
        b3.s = make_float3(c3[0].s.x + c3[1].s.x, c3[0].s.y + c3[1].s.y, c3[0].s.z + c3[1].s.z);
        b3.k = c3[0].k + c3[1].k;
        b3.n = sat_add(c3[0].n, c3[1].n);
        const float3 m3 = box_mean(b3);
        float4 *mips = a.t.mips + (size_t)t * kTileMips;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t c = (uint32_t)lane + 32u * h;
            if (live[h]) {
                // finest level with enough samples; a live cell has a value at every level above it
                float3 ans = m3;
                if (ns[h] >= a.min_samples) ans = v[h];
                else if (b1[h].n >= a.min_samples) ans = box_mean(b1[h]);
                else if (b2[h].n >= a.min_samples) ans = box_mean(b2[h]);
                store_resolved(a.t.resolved, a.res_stride, a.f16, (uint32_t)(base + c), ans, cold[h]);
            }
            if ((c & 9u) == 0u) mips[((c & 7u) >> 1) + 4u * (c >> 4)] = mip_word(b1[h]);
            if ((c & 27u) == 0u) mips[16u + ((c >> 2) & 1u) + 2u * (c >> 5)] = mip_word(b2[h]);
        }
        if (lane == 0) mips[20] = mip_word(b3);
    }
    resolve_finish(a.ctr, a.occ_out, a.stamp_now, gridDim.x, 0u);
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
                if (lane == 0) ++live_tiles;
            } else if (lane == 0) {
                dropped += (uint32_t)(__popc(live0) + __popc(live1));
            }
        }
        from.stamp[e0] = 0u;
        from.stamp[e1] = 0u;
        __syncwarp();
        if (lane == 0) {
            from.tags[s] = kEmpty;
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
__global__ void k_tile_scan(TileArrays t, uint32_t tiles, LiveRule rule, unsigned long long *out /* occupied, live */) {
    unsigned long long occ = 0, live = 0;
    const size_t cells = (size_t)tiles * kTileCells;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < cells; e += (size_t)gridDim.x * blockDim.x) {
        if (t.tags[e / kTileCells] == kEmpty) continue;
        if ((e % kTileCells) == 0) ++occ;
        if (t.accum[e].count > 0u || answers(t.stamp[e], rule)) ++live;
    }
    for (int o = 16; o; o >>= 1) {
        occ += __shfl_xor_sync(kFull, occ, o);
        live += __shfl_xor_sync(kFull, live, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, occ);
        atomicAdd(out + 1, live);
    }
}

// ---------------------------------------------------------------- launchers
gi_status tile_update_launch(const TileUpdateArgs &a, int key_dir, cudaStream_t st) {
    const int blocks = (int)((a.u.n + kUpdBlockRecords - 1) / kUpdBlockRecords);
    if (blocks == 0) return GI_OK;
    if (key_dir == GI_KEY_DIR_NORMAL)
        k_tile_update<GI_KEY_DIR_NORMAL><<<blocks, kUpdThreads, 0, st>>>(a);
    else
        k_tile_update<GI_KEY_DIR_RAY><<<blocks, kUpdThreads, 0, st>>>(a);
    return cuda_status(cudaGetLastError(), "k_tile_update launch");
}

int tile_resolve_blocks_per_sm() {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_resolve, kTileResThreads, 0) != cudaSuccess)
        return 1;
    return per_sm > 0 ? per_sm : 1;
}

gi_status tile_resolve_launch(const TileResolveArgs &a, int blocks, cudaStream_t st) {
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

gi_status tile_scan_launch(const TileArrays &t, uint32_t tiles, LiveRule rule, unsigned long long *out, int blocks,
                           cudaStream_t st) {
    k_tile_scan<<<blocks, 256, 0, st>>>(t, tiles, rule, out);
    return cuda_status(cudaGetLastError(), "k_tile_scan launch");
}

} // namespace gi
